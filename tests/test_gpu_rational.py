"""Rational factors, reweighting exponents and the small determinant on the GPU
(App. A.2, A.3; Sec. 2.3) against the oracle (oracle/reweighting.py) on the
same seeded fields.

Tolerances.  Both sides take every shifted inverse from a multi-shift CG to a
relative residual tol; a quantity built from them differs between the sides by
about tol times the condition number of Q2 + mu_j^2 relative to |phi|^2.  The
pseudofermion action and P_{k,l} phi are dominated by the identity part and
agree to 1e-8; the W_rat series terms (eta, Z^n eta) are small differences
(|Z| ~ v delta) and agree to 1e-4 relative plus 1e-9 |eta|^2 absolute.
S_sdet is a sum of site-local FP64 factorisations: 1e-12 relative."""
import os

import numpy as np
import pytest

from oracle import ratapprox
from oracle import reweighting as rw
from paper_1908_11673_gb300 import workload
from tests.gpu_helpers import relerr, setup

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rational_deg10_pow_m1_4.txt")


def gpu_rational(qxd, r):
    return qxd.rational(r.A, r.nu, r.mu)


def spinor_e(op, seed):
    return workload.spinor(len(op.even_sites()), seed)


@pytest.mark.parametrize("L,cstar,qhat", [((8, 8, 8, 8), 0, -2), ((4, 4, 8, 4), 1, 4), ((8, 4, 4, 4), 3, -2)])
def test_sdet_parity(L, cstar, qhat):
    qxd, ctx, op, _, _ = setup(L, cstar, (np.pi, 0, 0, 0) if cstar == 0 else (np.pi, 0, 0, 0), qhat=qhat,
                               kappa=0.13, seed=9300, stout=1)
    got, nneg = ctx.sdet(0)
    want, wneg = rw.sdet(op)
    assert abs(got - want) <= 1e-12 * abs(want)
    assert nneg == wneg
    ctx.close()


@pytest.mark.parametrize("k,l", [(0, 9), (0, 4), (5, 9)])
def test_pf_action_and_factor_parity(k, l):
    qxd, ctx, op, _, _ = setup((8, 8, 8, 8), 0, (np.pi, 0, 0, 0), qhat=-2, kappa=0.13, seed=9310, stout=1)
    r = ratapprox.load(GOLDEN)
    gr = gpu_rational(qxd, r)
    phi = spinor_e(op, 9311)
    Q2 = rw.NormalOperator(op)
    S, info = ctx.pf_action(0, gr, k, l, phi, tol=1e-11)
    assert info.status == 0 and info.true_relres <= 1e-11
    S_or = rw.pf_action(Q2, r, k, l, phi, tol=1e-12)
    assert abs(S - S_or) <= 1e-8 * abs(S_or)
    out = np.empty_like(phi)
    ctx.rat_apply(0, gr, k, l, phi, out, tol=1e-11)
    assert relerr(out, rw.factor_apply(Q2, r, k, l, phi, tol=1e-12)) <= 1e-8
    # S = (phi, P phi) from the returned field
    assert abs(np.vdot(phi, out).real - S) <= 1e-10 * abs(S)
    ctx.close()


def test_rw_rat_parity():
    qxd, ctx, op, _, _ = setup((4, 4, 8, 4), 1, (np.pi, 0, 0, 0), qhat=-2, kappa=0.13, seed=9320, stout=1)
    r = ratapprox.load(GOLDEN)
    eta = spinor_e(op, 9321)
    u, v, nterms = 1, 4, 2
    terms, expo, info = ctx.rw_rat(0, gpu_rational(qxd, r), u, v, nterms, eta, tol=1e-12)
    assert info.status == 0
    want = rw.wrat_terms(rw.NormalOperator(op), r, u, v, nterms, eta, tol=1e-12)
    nrm = np.vdot(eta, eta).real
    for t, w in zip(terms, want):
        assert abs(t - w) <= 1e-4 * abs(w) + 1e-9 * nrm, (t, w)
    assert abs(expo - rw.wrat_exponent(want, v)) <= 1e-4 * abs(expo) + 1e-9 * nrm
    ctx.close()


@pytest.mark.parametrize("k,l", [(0, 9), (2, 6)])
def test_rw_rtm_parity(k, l):
    qxd, ctx, op, _, _ = setup((8, 8, 8, 8), 0, (np.pi, 0, 0, 0), qhat=-2, kappa=0.13, seed=9330, stout=1)
    r_t = ratapprox.load(GOLDEN)
    r_mu = rw.shifted(r_t, 0.02)
    eta = spinor_e(op, 9331)
    e, info = ctx.rw_rtm(0, gpu_rational(qxd, r_mu), gpu_rational(qxd, r_t), k, l, eta, tol=1e-11)
    assert info.status == 0
    want = rw.wrtm_exponent(rw.NormalOperator(op), r_mu, r_t, k, l, eta, tol=1e-12)
    assert abs(e - want) <= 1e-6 * abs(want) + 1e-11 * np.vdot(eta, eta).real, (e, want)
    ctx.close()


def test_rational_argument_errors():
    qxd, ctx, op, _, _ = setup((4, 4, 4, 4), 0, (np.pi, 0, 0, 0))
    r = ratapprox.load(GOLDEN)
    gr = gpu_rational(qxd, r)
    phi = spinor_e(op, 1)
    for k, l in [(3, 2), (-1, 4), (0, 10)]:
        with pytest.raises(qxd.QxdError) as e:
            ctx.pf_action(0, gr, k, l, phi)
        assert e.value.code == 1
    same = qxd.rational(1.0, [1.0, 2.0], [0.5, 0.5])
    with pytest.raises(qxd.QxdError) as e:
        ctx.pf_action(0, same, 0, 1, phi)
    assert e.value.code == 1
    with pytest.raises(qxd.QxdError) as e:
        ctx.rw_rat(0, gr, 1, 0, 2, phi)
    assert e.value.code == 1
    ctx.close()
