"""Pins of the learned-preconditioner oracle (oracle/ptc.py)."""
import numpy as np
import pytest

from oracle import ptc
from oracle import DiracOperator, Flavour, GaugeField, Geometry
from paper_1908_11673_gb300 import workload
from tests.oracle_helpers import make_op


def rand_weights(rng, nlayers, nch, scale=0.3):
    Ws = ptc.identity_weights(nlayers, nch)
    for W in Ws:
        W += scale * (rng.normal(size=W.shape) + 1j * rng.normal(size=W.shape))
    return Ws


def test_identity_weights_give_identity():
    op, _, _ = make_op((4, 4, 2, 4), 1, (np.pi, 0, 0, 0), qhat=4)
    T = ptc.Transport(op)
    r = workload.spinor(op.geom.V // 2, 1)
    out = ptc.network(T, ptc.identity_weights(4, 3), r)
    assert np.abs(out - r).max() == 0.0


@pytest.mark.parametrize("cstar", [0, 2])
def test_transport_and_layer_adjoints(cstar):
    op, _, _ = make_op((4, 4, 2, 4), cstar, (np.pi if cstar else 0.7, 0, 0, 0), qhat=-2)
    T = ptc.Transport(op)
    V = op.geom.V
    a = workload.spinor(V, 2)
    g = workload.spinor(V, 3)
    for d in range(ptc.NDIR):
        lhs = np.vdot(g, T.apply(d, a))
        rhs = np.vdot(T.apply(ptc.opposite(d), g), a)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    rng = np.random.default_rng(4)
    W = rng.normal(size=(3, 2, 9, 4, 4)) + 1j * rng.normal(size=(3, 2, 9, 4, 4))
    A = workload.spinor(V, 5, nrhs=2)
    Gf = workload.spinor(V, 6, nrhs=3)
    lhs = np.vdot(Gf, ptc.layer(T, W, A))
    rhs = np.vdot(ptc.layer_adjoint(T, W, Gf), A)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_transport_plane_wave_eigenvalues():
    """Free field: T_{1+mu} e^{ipx} chi = e^{i p_mu} e^{ipx} chi and
    T_{5+mu} e^{ipx} chi = e^{-i p_mu} e^{ipx} chi for momenta allowed by the
    boundary conditions (here antiperiodic time, periodic space)."""
    L = (4, 4, 6, 4)
    geom = Geometry(L, 0, (np.pi, 0, 0, 0))
    U, A = workload.unit_gauge_field(L)
    op = DiracOperator(GaugeField(geom, U, A, 6.0), Flavour(0, 0.13, 0.0, 0.0))
    T = ptc.Transport(op)
    p = np.array([3 * np.pi / 4, 2 * np.pi / 4, 2 * np.pi * 2 / 6, 2 * np.pi / 4])
    x = geom.coords(geom.sites())
    chi = np.arange(12).reshape(4, 3) + 1j
    psi = np.exp(1j * np.tensordot(p, x, axes=(0, 0)))[:, None, None] * chi
    for mu in range(4):
        assert np.abs(T.apply(1 + mu, psi) - np.exp(1j * p[mu]) * psi).max() < 1e-13
        assert np.abs(T.apply(5 + mu, psi) - np.exp(-1j * p[mu]) * psi).max() < 1e-13


def test_gauge_covariance_of_the_network():
    from tests.test_oracle_symmetries import random_su3
    qhat = 4
    op, U, A = make_op((4, 4, 2, 4), 0, (np.pi, 0, 0, 0), qhat=qhat, seed=9)
    geom = op.geom
    rng = np.random.default_rng(1)
    g = random_su3(rng, geom.V)
    lam = rng.uniform(-np.pi, np.pi, geom.V)
    s = geom.sites()
    Un, An = np.empty_like(U), np.empty_like(A)
    for mu in range(4):
        nb, _ = geom.neighbour(s, mu, +1)
        Un[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[nb], -1, -2))
        An[:, mu] = lam + A[:, mu] - lam[nb]
    op2 = DiracOperator(GaugeField(geom, Un, An, 6.0), op.fl)
    Ws = rand_weights(np.random.default_rng(2), 3, 2)
    ev = op.even_sites()
    omega = (g * np.exp(1j * qhat * lam)[:, None, None])[ev]
    rot = lambda v: np.einsum('nij,naj->nai', omega, v)
    r = workload.spinor(geom.V // 2, 3)
    got = ptc.network(ptc.Transport(op2), Ws, rot(r))
    want = rot(ptc.network(ptc.Transport(op), Ws, r))
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("norm", ["error", "residual"])
def test_gradient_matches_central_differences(norm):
    op, _, _ = make_op((2, 4, 2, 4), 1, (np.pi, 0, 0, 0), qhat=-2, seed=13)
    T = ptc.Transport(op)
    rng = np.random.default_rng(7)
    Ws = rand_weights(rng, 3, 2, scale=0.2)
    ne = op.geom.V // 2
    pairs = [(workload.spinor(ne, 20 + i), workload.spinor(ne, 40 + i)) for i in range(2)]
    L0, G = ptc.loss_and_grad(T, Ws, pairs, norm=norm)
    assert abs(L0 - ptc.loss(T, Ws, pairs, norm=norm)) < 1e-12 * L0
    h = 1e-6
    for l, c, cp, d, s, t in [(0, 1, 0, 0, 2, 3), (1, 0, 1, 3, 0, 0), (1, 1, 1, 7, 1, 2), (2, 0, 0, 5, 3, 1),
                              (2, 0, 1, 8, 2, 2)]:
        for part in (1.0, 1j):
            Wp = [W.copy() for W in Ws]
            Wm = [W.copy() for W in Ws]
            Wp[l][c, cp, d, s, t] += h * part
            Wm[l][c, cp, d, s, t] -= h * part
            fd = (ptc.loss(T, Wp, pairs, norm=norm) - ptc.loss(T, Wm, pairs, norm=norm)) / (2 * h)
            an = 2 * (G[l][c, cp, d, s, t].real if part == 1.0 else G[l][c, cp, d, s, t].imag)
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * L0), (l, c, cp, d, s, t, part, fd, an)


def test_residual_norm_special_cases():
    """The residual-norm loss of one pair: 1 for the zero map, |r - Dhat r|^2 / |r|^2
    for the identity network (Dhat from the dense matrix of the oracle's operator),
    and equal to the error loss weighted by Dhat, |Dhat (M r - e)|^2 / |Dhat e|^2,
    for a pair with Dhat e = r."""
    op, _, _ = make_op((2, 4, 2, 4), 0, (np.pi, 0, 0, 0), qhat=3, seed=17)
    T = ptc.Transport(op)
    ne = op.geom.V // 2
    Dinv = op.Doo_inv()
    Dmat = np.stack([op.Dhat(np.eye(12 * ne)[k].reshape(ne, 4, 3), Dinv).reshape(-1) for k in range(12 * ne)], axis=1)
    e = workload.spinor(ne, 51)
    r = (Dmat @ e.reshape(-1)).reshape(ne, 4, 3)
    zero = [np.zeros_like(W) for W in ptc.identity_weights(3, 2)]
    assert abs(ptc.loss(T, zero, [(r, e)], norm="residual") - 1.0) < 1e-14
    ident = ptc.identity_weights(3, 2)
    want = np.linalg.norm(r.reshape(-1) - Dmat @ r.reshape(-1)) ** 2 / np.linalg.norm(r) ** 2
    assert abs(ptc.loss(T, ident, [(r, e)], norm="residual") - want) < 1e-12 * want
    Ws = rand_weights(np.random.default_rng(9), 3, 2, scale=0.2)
    out = ptc.network(T, Ws, r)
    dnorm = np.linalg.norm(Dmat @ (out - e).reshape(-1)) ** 2 / np.linalg.norm(Dmat @ e.reshape(-1)) ** 2
    assert abs(ptc.loss(T, Ws, [(r, e)], norm="residual") - dnorm) < 1e-10 * dnorm
