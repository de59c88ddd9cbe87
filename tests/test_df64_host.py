"""The double-float arithmetic of csrc/df64.cuh (used for the mixed solvers' true
residuals), compiled for the host and checked against properties that fix it:
two-sum and the FMA product are error-free (the pair represents the exact sum or
product, checked in exact rational arithmetic), and the lazy sums and products
of one stencil-sized chain (~10^2 operations, every product with one normalised
factor) stay within 2^-44 of the exact value."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r'''
#include <cstdio>
#include <cstdlib>
#include "df64.cuh"
using namespace qxd;
int main() {
    float a, b;
    double x[64], y[64];
    // pairs: two_sum and the exact product
    while (scanf("%a %a", &a, &b) == 2 && !(a == 0.f && b == 0.f)) {
        dfl s = df_two_sum(a, b);
        dfl p = dfl(a, 0.f) * dfl(b, 0.f);
        printf("%a %a %a %a\n", s.hi, s.lo, p.hi, p.lo);
    }
    // chains: sum_k x_k y_k with both factors double-float rounded, lazily accumulated
    int n;
    while (scanf("%d", &n) == 1 && n > 0) {
        for (int k = 0; k < n; ++k) scanf("%la %la", &x[k], &y[k]);
        dfl acc(0.f, 0.f);
        for (int k = 0; k < n; ++k) acc = fma(dfl(x[k]), dfl(y[k]), acc);
        acc = df_norm(acc);
        printf("%a %a\n", acc.hi, acc.lo);
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not os.path.isdir(cuda_inc):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("df64")
    src = d / "df64_host.cpp"
    src.write_text(PROGRAM)
    exe = d / "df64_host"
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", cuda_inc,
                    "-I", os.path.join(ROOT, "paper_1908_11673_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True)
    return str(exe)


def run(exe, text):
    return subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")


def test_two_sum_and_product_are_exact(prog):
    rng = np.random.default_rng(11)
    a = (rng.normal(size=400) * np.exp2(rng.integers(-20, 20, 400))).astype(np.float32)
    b = (rng.normal(size=400) * np.exp2(rng.integers(-20, 20, 400))).astype(np.float32)
    text = "".join(f"{float(x).hex()} {float(y).hex()}\n" for x, y in zip(a, b)) + "0x0p+0 0x0p+0\n0\n"
    out = run(prog, text)
    for line, x, y in zip(out, a, b):
        sh, sl, ph, pl = (float.fromhex(t) for t in line.split())
        fx, fy = Fraction(float(x)), Fraction(float(y))
        assert Fraction(sh) + Fraction(sl) == fx + fy
        assert Fraction(ph) + Fraction(pl) == fx * fy


def test_lazy_chain_accuracy(prog):
    rng = np.random.default_rng(12)
    chains = []
    text = "0x0p+0 0x0p+0\n"
    for n in (8, 50, 64):
        x = rng.normal(size=n)
        y = rng.normal(size=n)
        chains.append((x, y))
        text += f"{n}\n" + "".join(f"{float(u).hex()} {float(v).hex()}\n" for u, v in zip(x, y))
    text += "0\n"
    out = [l for l in run(prog, text) if l.strip()]
    for line, (x, y) in zip(out, chains):
        hi, lo = (float.fromhex(t) for t in line.split())
        exact = sum(Fraction(float(u)) * Fraction(float(v)) for u, v in zip(x, y))
        scale = sum(abs(Fraction(float(u)) * Fraction(float(v))) for u, v in zip(x, y))
        err = abs(Fraction(hi) + Fraction(lo) - exact)
        assert err <= scale * Fraction(1, 2 ** 44), float(err / scale)
