"""Dense brute force on small lattices: the even-odd (Schur) identities behind
Dhat (Sec. 2.3) and the solvers (Sec. 4.4) against LAPACK."""
import numpy as np
import pytest

from oracle.solvers import cgne_solve, gcr, mscg, cg
from tests.oracle_helpers import dense, make_op

CASES = [((4, 4, 2, 2), 0, (np.pi, 0.3, 0, 0)), ((2, 4, 2, 4), 1, (np.pi, 0, 0, 0)),
         ((2, 2, 4, 2), 3, (np.pi, 0, 0, 0))]


def full_matrix(op):
    V = op.geom.V
    return dense(lambda v: op.apply(v), V * 12, (V, 4, 3))


@pytest.mark.parametrize("L,cstar,theta", CASES)
def test_schur_identities(L, cstar, theta):
    op, _, _ = make_op(L, cstar, theta, qhat=4, kappa=0.13, seed=61)
    geom = op.geom
    D = full_matrix(op)
    ev, od = op.even_sites(), op.odd_sites()
    ie = (ev[:, None] * 12 + np.arange(12)).reshape(-1)
    io = (od[:, None] * 12 + np.arange(12)).reshape(-1)
    Dee, Deo, Doe, Doo = D[np.ix_(ie, ie)], D[np.ix_(ie, io)], D[np.ix_(io, ie)], D[np.ix_(io, io)]
    # hops join opposite parities: D_ee and D_oo are site diagonal
    for blk, sites in ((Dee, ev), (Doo, od)):
        n = len(sites)
        mask = np.kron(np.eye(n), np.ones((12, 12)))
        assert np.abs(blk * (1 - mask)).max() == 0.0
    Dhat_schur = Dee - Deo @ np.linalg.solve(Doo, Doe)
    Dinv = op.Doo_inv()
    ne = len(ev)
    Dhat = dense(lambda v: op.Dhat(v, Dinv), ne * 12, (ne, 4, 3))
    assert np.abs(Dhat - Dhat_schur).max() < 1e-13 * np.abs(Dhat).max()
    # det D = det D_oo det Dhat, and Dhat^-1 = (D^-1)_ee
    s1, l1 = np.linalg.slogdet(D)
    s2, l2 = np.linalg.slogdet(Doo)
    s3, l3 = np.linalg.slogdet(Dhat)
    assert abs(l1 - (l2 + l3)) < 1e-9 * abs(l1)
    assert abs(s1 - s2 * s3) < 1e-9
    Dinv_full = np.linalg.inv(D)
    assert np.abs(np.linalg.inv(Dhat) - Dinv_full[np.ix_(ie, ie)]).max() < 1e-10 * np.abs(Dinv_full).max()


@pytest.mark.parametrize("L,cstar,theta", CASES)
def test_cgne_solve_matches_lapack(L, cstar, theta):
    op, _, _ = make_op(L, cstar, theta, qhat=-2, kappa=0.13, seed=71)
    V = op.geom.V
    eta = np.random.default_rng(1).normal(size=(V, 4, 3)) + 0j
    psi, it, res = cgne_solve(op, eta, 1e-10, 5000)
    assert it > 0 and res <= 1e-10
    D = full_matrix(op)
    x = np.linalg.solve(D, eta.reshape(-1)).reshape(V, 4, 3)
    cond = np.linalg.cond(D)
    assert np.abs(psi - x).max() <= 10 * cond * 1e-10 * np.abs(x).max()


def test_gcr_and_mscg_match_lapack():
    op, _, _ = make_op((4, 2, 2, 4), 0, (np.pi, 0, 0, 0), qhat=4, kappa=0.13, seed=81)
    ev = op.even_sites()
    ne = len(ev)
    Dinv = op.Doo_inv()
    Dh = lambda v: op.Dhat(v, Dinv)
    M = dense(Dh, ne * 12, (ne, 4, 3))
    b = np.random.default_rng(2).normal(size=(ne, 4, 3)) + 1j
    x, it = gcr(Dh, b, 1e-11, 8, 2000)
    assert it > 0
    ref = np.linalg.solve(M, b.reshape(-1)).reshape(ne, 4, 3)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref) * np.linalg.cond(M)
    H = M.conj().T @ M
    shifts = [0.0, 0.01, 0.5, 3.0]
    apply_H = lambda v: (H @ v.reshape(-1)).reshape(v.shape)
    xs, it = mscg(apply_H, b, shifts, 1e-11, 5000)
    assert it > 0
    for s, xj in zip(shifts, xs):
        ref = np.linalg.solve(H + s * np.eye(len(H)), b.reshape(-1)).reshape(b.shape)
        assert np.linalg.norm(xj - ref) <= 1e-8 * np.linalg.norm(ref)
    # single-shift CG agrees with the zero shift
    x0, _ = cg(apply_H, b, 1e-11, 5000)
    assert np.linalg.norm(x0 - xs[0]) <= 1e-8 * np.linalg.norm(x0)
