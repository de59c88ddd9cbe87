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


CONVERSIONS = r'''
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include "df64.cuh"
using namespace qxd;
// df_split and df_widen (integer forms) against the conversion operators they replace:
// (float)d, (float)(d - (double)(float)d) and (double)f, compared bit for bit
int main() {
    std::mt19937_64 rng(7);
    long long bad = 0, n = 0;
    auto check = [&](double d) {
        const dfl a = df_split(d);
        const float rh = (float)d, rl = (float)(d - (double)rh);
        const double w = df_widen(rh), rw = (double)rh;
        ++n;
        if (std::memcmp(&a.hi, &rh, 4) || std::memcmp(&a.lo, &rl, 4) || std::memcmp(&w, &rw, 8)) {
            if (bad < 5) std::printf("mismatch %a\n", d);
            ++bad;
        }
    };
    std::uniform_real_distribution<double> U(-4.0, 4.0);
    for (int i = 0; i < 1000000; ++i) {
        unsigned long long u = rng();
        double d;
        std::memcpy(&d, &u, 8);
        check(d);  // any bit pattern: subnormal, inf, nan, huge and tiny values included
        check(U(rng) * std::ldexp(1.0, (int)(rng() % 80) - 40));
        u = (rng() & ~0x1FFFFFFFull) | 0x10000000ull;  // ties of the leading part
        std::memcpy(&d, &u, 8);
        check(d);
        u = (rng() & 0xFFF0000000000000ull) | 0xFFFFFF0000000ull | (rng() & 0x1FFFFFFFull);  // carries
        std::memcpy(&d, &u, 8);
        check(d);
    }
    const double edge[] = {0.0, -0.0, 1.0, -1.0, 0x1p-74, 0x1p-75, 0x1.fffffffffffffp-75, 0x1p127,
                           0x1.fffffep127, 0x1.ffffffp127, 0x1.fffffffffffffp126, 1e300, -1e-300, 5e-324,
                           INFINITY, -INFINITY, NAN, 0x1.000001p0, 0x1.0000008p0, 0x1.0000018p0, 0x1.ffffff8p0};
    for (double d : edge) check(d);
    std::printf("%lld %lld\n", n, bad);
    return 0;
}
'''


def test_integer_conversions_match_the_conversion_operators(tmp_path):
    """df_split / df_widen (integer forms used by the solver's conversion kernels) give the
    same bits as the IEEE conversions (round to nearest even) on 4 M random doubles:
    arbitrary bit patterns, values of spinor magnitude, exact ties and rounding carries
    of the leading part, and edge cases (signed zeros, range limits, inf, nan)."""
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not os.path.isdir(cuda_inc):
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "conv.cpp"
    src.write_text(CONVERSIONS)
    exe = tmp_path / "conv"
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", cuda_inc,
                    "-I", os.path.join(ROOT, "paper_1908_11673_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    n, bad = int(out[-2]), int(out[-1])
    assert n > 4_000_000 and bad == 0, out
