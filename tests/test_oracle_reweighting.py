"""Pins of the rational factors on lattice fields (App. A.2, A.3) and of the
small-determinant action (Sec. 2.3), against what the mathematics fixes:

 * the residues of Ptilde_{k,l} - 1 reproduce the product form at arbitrary q2
   (and vanish when both approximations are the same);
 * the Taylor coefficients c_{v,n} sum to (1 + z)^(-1/v) - 1;
 * on a small lattice, the field functions equal the spectral definitions
   through the dense eigendecomposition of Q2 = Dhat^+ Dhat built by LAPACK:
   P_{k,l} phi, (phi, P_{k,l} phi), (eta, Z^n eta) with Z = Q2^u R^v - 1, and
   (eta, [Ptilde_{k,l} - 1] eta), each evaluated from the product forms;
 * S_sdet: det D = det D_oo det Dhat (Schur), so sum_odd log|det D_oo(x)| =
   log|det D| - log|det Dhat| from dense LU; and the free-field value
   12 V/2 log(1/(2 kappa)).
"""
import functools
import os

import numpy as np
import pytest

from oracle import ratapprox
from oracle import reweighting as rw
from tests.oracle_helpers import dense, make_op

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rational_deg10_pow_m1_4.txt")


def printed():
    return ratapprox.load(GOLDEN)


def product(rat, k, l, q2):
    out = np.ones_like(q2)
    for j in range(k, l + 1):
        out = out * (q2 + rat.nu[j] ** 2) / (q2 + rat.mu[j] ** 2)
    return out


def ptilde(r_mu, r_t, k, l, q2):
    out = np.ones_like(q2)
    for j in range(k, l + 1):
        out = out * (q2 + r_mu.mu[j] ** 2) * (q2 + r_t.nu[j] ** 2) / ((q2 + r_mu.nu[j] ** 2) * (q2 + r_t.mu[j] ** 2))
    return out


@pytest.mark.parametrize("k,l", [(0, 9), (0, 4), (5, 8), (9, 9)])
def test_rtm_residues_reproduce_product(k, l):
    r_t = printed()
    r_mu = rw.shifted(r_t, 0.01)
    sig, sigt = rw.rtm_sigma(r_mu, r_t, k, l)
    q2 = np.geomspace(1e-7, 1e3, 501)
    pf = np.ones_like(q2)
    for i, j in enumerate(range(k, l + 1)):
        pf += sig[i] / (q2 + r_mu.nu[j] ** 2) + sigt[i] / (q2 + r_t.mu[j] ** 2)
    want = ptilde(r_mu, r_t, k, l, q2)
    assert np.abs(pf - want).max() <= 1e-10 * np.abs(want).max()


def test_rtm_residues_vanish_for_equal_approximations():
    r = printed()
    sig, sigt = rw.rtm_sigma(r, r, 0, 9)
    assert np.all(sig == 0.0) and np.all(sigt == 0.0)


def test_factor_residues_reproduce_product():
    r = printed()
    for k, l in [(0, 9), (0, 4), (5, 8), (3, 3)]:
        q2 = np.geomspace(1e-7, 1e3, 301)
        pf = np.ones_like(q2)
        for s, j in zip(r.sigma(k, l), range(k, l + 1)):
            pf += s / (q2 + r.mu[j] ** 2)
        assert np.abs(pf / product(r, k, l, q2) - 1).max() < 1e-12


@pytest.mark.parametrize("v", [1, 2, 4])
def test_taylor_coefficients(v):
    for z in (0.3, -0.2, 1e-3):
        s = sum(rw.c_vn(v, n) * z ** n for n in range(1, 80))
        assert abs(s - ((1 + z) ** (-1.0 / v) - 1)) < 1e-13
    assert rw.c_vn(v, 1) == -1.0 / v


def test_shifted_approximation_keeps_the_error():
    r = printed()
    mh = 0.05
    rs = rw.shifted(r, mh)
    q2 = np.geomspace(r.r_a ** 2, r.r_b ** 2, 20001)
    err = 1 - (q2 + mh * mh) ** r.alpha * rs.rho(q2)
    # rs(q2) = rho(q2 + mh^2), so the error at q2 is rho's error at q2 + mh^2, within delta where that stays in range
    inside = q2 + mh * mh <= r.r_b ** 2
    assert np.abs(err[inside]).max() <= r.delta * (1 + 1e-9)


CASES = [((4, 2, 2, 4), 0, (np.pi, 0, 0, 0)), ((2, 4, 2, 4), 1, (np.pi, 0, 0, 0))]


@functools.lru_cache(maxsize=None)
def spectral(L, cstar, theta, seed=131):
    """Dense Q2 = M^+ M from LAPACK on the matrix M of Dhat, its eigendecomposition, and
    Q2 as a fast callable (checked once against the oracle's NormalOperator)."""
    op, _, _ = make_op(L, cstar, theta, qhat=-2, kappa=0.13, seed=seed)
    ne = len(op.even_sites())
    Dinv = op.Doo_inv()
    M = dense(lambda v: op.Dhat(v, Dinv), ne * 12, (ne, 4, 3))
    H = M.conj().T @ M
    w, Q = np.linalg.eigh(H)
    v = np.random.default_rng(seed).normal(size=(ne, 4, 3)) + 0j
    Hv = (H @ v.reshape(-1)).reshape(v.shape)
    assert np.linalg.norm(rw.NormalOperator(op)(v) - Hv) <= 1e-13 * np.linalg.norm(Hv)
    return op, ne, w, Q, lambda x: (H @ x.reshape(-1)).reshape(x.shape)


def fn_of(Q, w, f, v):
    return (Q @ (f(w) * (Q.conj().T @ v.reshape(-1)))).reshape(v.shape)


def quad(Q, w, f, v):
    c = Q.conj().T @ v.reshape(-1)
    return float(np.sum(np.abs(c) ** 2 * f(w)))


@pytest.mark.parametrize("L,cstar,theta", CASES)
def test_factor_and_action_spectral(L, cstar, theta):
    op, ne, w, Q, Q2 = spectral(L, cstar, theta)
    r = printed()
    phi = np.random.default_rng(5).normal(size=(ne, 4, 3)) + 1j * np.random.default_rng(6).normal(size=(ne, 4, 3))
    for k, l in [(0, 9), (0, 4), (5, 9)]:
        got = rw.factor_apply(Q2, r, k, l, phi)
        want = fn_of(Q, w, lambda x: product(r, k, l, x), phi)
        assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)
        S = rw.pf_action(Q2, r, k, l, phi)
        assert abs(S - quad(Q, w, lambda x: product(r, k, l, x), phi)) <= 1e-9 * abs(S)
    got = rw.rat_apply(Q2, r, phi)
    assert np.linalg.norm(got - fn_of(Q, w, r.rho, phi)) <= 1e-9 * np.linalg.norm(got)


@pytest.mark.parametrize("L,cstar,theta", CASES)
def test_wrat_terms_spectral(L, cstar, theta):
    op, ne, w, Q, Q2 = spectral(L, cstar, theta)
    r = printed()
    eta = np.random.default_rng(7).normal(size=(ne, 4, 3)) + 1j * np.random.default_rng(8).normal(size=(ne, 4, 3))
    u, v = 1, 4  # alpha = 1/4
    terms = rw.wrat_terms(Q2, r, u, v, 3, eta)
    zeta = w ** u * r.rho(w) ** v - 1.0
    # the approximation holds on the spectrum: |Z| <= (1 + delta)^v - 1
    assert np.abs(zeta).max() <= (1 + r.delta) ** v - 1 + 1e-12
    for n, t in enumerate(terms, start=1):
        want = quad(Q, w, lambda x: (x ** u * r.rho(x) ** v - 1.0) ** n, eta)
        assert abs(t - want) <= 1e-6 * abs(want) + 1e-12 * np.vdot(eta, eta).real, (n, t, want)
    want = quad(Q, w, lambda x: (1 + (x ** u * r.rho(x) ** v - 1.0)) ** (-1.0 / v) - 1.0, eta)
    assert abs(rw.wrat_exponent(terms, v) - want) <= 1e-4 * abs(want)


@pytest.mark.parametrize("L,cstar,theta", CASES)
def test_wrtm_exponent_spectral(L, cstar, theta):
    op, ne, w, Q, Q2 = spectral(L, cstar, theta)
    r_t = printed()
    r_mu = rw.shifted(r_t, 0.02)
    eta = np.random.default_rng(9).normal(size=(ne, 4, 3)) + 1j * np.random.default_rng(10).normal(size=(ne, 4, 3))
    for k, l in [(0, 9), (0, 4), (5, 9), (9, 9)]:
        got = rw.wrtm_exponent(Q2, r_mu, r_t, k, l, eta)
        want = quad(Q, w, lambda x: ptilde(r_mu, r_t, k, l, x) - 1.0, eta)
        assert abs(got - want) <= 1e-8 * abs(want) + 1e-14 * np.vdot(eta, eta).real, (k, l, got, want)


@pytest.mark.parametrize("L,cstar,theta", CASES)
def test_sdet_schur(L, cstar, theta):
    op, _, _ = make_op(L, cstar, theta, qhat=4, kappa=0.13, seed=141)
    V = op.geom.V
    D = dense(lambda v: op.apply(v), V * 12, (V, 4, 3))
    ne = len(op.even_sites())
    Dinv = op.Doo_inv()
    Dh = dense(lambda v: op.Dhat(v, Dinv), ne * 12, (ne, 4, 3))
    _, l_full = np.linalg.slogdet(D)
    _, l_hat = np.linalg.slogdet(Dh)
    got, nneg = rw.sdet(op)
    assert abs(got - (l_full - l_hat)) <= 1e-10 * abs(l_full)
    assert nneg == 0


def test_sdet_free_field():
    kappa = 0.125
    op, _, _ = make_op((4, 4, 2, 2), 0, (np.pi, 0, 0, 0), kappa=kappa, free=True)
    got, nneg = rw.sdet(op)
    assert abs(got - 12 * (op.geom.V // 2) * np.log(1 / (2 * kappa))) < 1e-12 * abs(got) + 1e-12
    assert nneg == 0
