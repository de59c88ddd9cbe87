"""Pins of the oracle against closed forms of the free and constant-background
operator (Sec. 2.1 boundary conditions, Sec. 2.3 operator).

Free field, U = 1, z = 1: a plane wave psi(x) = exp(i p.x) chi is an
eigenfunction of the hopping term and
    D psi = exp(i p.x) [1/(2 kappa) - sum_mu cos p_mu + i sum_mu gamma_mu sin p_mu] chi
for every momentum allowed by the boundary conditions:
  * phase-periodic direction:  p_mu = (2 pi n + theta_mu) / L_mu;
  * C* extended direction 1:   p_1 = pi n_1 / L_1,  n_1 = 0 .. 2L_1 - 1;
  * C* direction k = 2, 3:     p_k = pi (2 m + n_1) / L_k  (the shifted identification
    x + L_k e_k ~ x + L_1 e_1 of eq. ext-shifted-bc).
"""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from oracle import DiracOperator, Flavour, GaugeField, Geometry
from oracle.dirac import GAMMA
from paper_1908_11673_gb300 import workload
from tests.oracle_helpers import dense, make_op


def plane_wave(geom, p, chi):
    x = geom.coords(geom.sites())
    ph = np.exp(1j * np.tensordot(np.asarray(p), x, axes=(0, 0)))
    return ph[:, None, None] * chi[None, :, :]


def free_matrix(kappa, p):
    M = np.eye(4, dtype=np.complex128) * (1.0 / (2 * kappa) - np.sum(np.cos(p)))
    for mu in range(4):
        M = M + 1j * np.sin(p[mu]) * GAMMA[mu]
    return M


def allowed_momenta(geom, rng, count):
    L, N = geom.L, geom.N
    out = []
    for _ in range(count):
        p = np.zeros(4)
        p[0] = (2 * np.pi * rng.integers(L[0]) + geom.theta[0]) / L[0]
        if geom.cstar:
            n1 = rng.integers(N[1])
            p[1] = np.pi * n1 / L[1]
            for k in (2, 3):
                if k <= geom.cstar:
                    p[k] = np.pi * (2 * rng.integers(L[k]) + n1) / L[k]
                else:
                    p[k] = 2 * np.pi * rng.integers(L[k]) / L[k]
        else:
            for k in (1, 2, 3):
                p[k] = (2 * np.pi * rng.integers(L[k]) + geom.theta[k]) / L[k]
        out.append(p)
    return out


GEOMS = [
    ((4, 6, 4, 8), 0, (np.pi, 0.0, 0.0, 0.0)),
    ((6, 4, 4, 4), 0, (0.3, 0.7, -1.1, 2.0)),
    ((4, 4, 6, 4), 1, (np.pi, 0.0, 0.0, 0.0)),
    ((4, 4, 4, 6), 2, (np.pi, 0.0, 0.0, 0.0)),
    ((4, 6, 4, 4), 3, (np.pi, 0.0, 0.0, 0.0)),
    ((4, 4, 6, 8), 3, (0.0, 0.0, 0.0, 0.0)),
]


@pytest.mark.parametrize("L,cstar,theta", GEOMS)
def test_free_plane_waves(L, cstar, theta):
    geom = Geometry(L, cstar, theta)
    U, A = workload.unit_gauge_field(L)
    kappa = 0.13
    op = DiracOperator(GaugeField(geom, U, A, 6.0), Flavour(-2, kappa, 1.9, 1.0))
    rng = np.random.default_rng(5)
    for p in allowed_momenta(geom, rng, 6):
        chi = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        psi = plane_wave(geom, p, chi)
        got = op.apply(psi)
        want = plane_wave(geom, p, free_matrix(kappa, p) @ chi)
        assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def test_free_field_forbidden_momentum_fails():
    """A momentum that violates the boundary condition is not an eigenfunction
    (guards the test above against accepting any wave)."""
    geom = Geometry((4, 4, 4, 4), 0, (np.pi, 0, 0, 0))
    U, A = workload.unit_gauge_field(geom.L)
    op = DiracOperator(GaugeField(geom, U, A, 6.0), Flavour(0, 0.13, 0.0, 0.0))
    p = np.array([0.0, 0, 0, 0])  # periodic in time: not allowed with theta_0 = pi
    chi = np.ones((4, 3), dtype=np.complex128)
    psi = plane_wave(geom, p, chi)
    assert np.abs(op.apply(psi) - plane_wave(geom, p, free_matrix(0.13, p) @ chi)).max() > 0.1


@pytest.mark.parametrize("qhat", [-2, 1, 4])
def test_constant_u1_background_shifts_momentum(qhat):
    """A constant photon field A_mu = phi_mu (no C*) enters the hopping term as
    z^qhat = exp(i qhat phi_mu), i.e. p -> p + qhat phi; all U(1) plaquettes are 1,
    so the U(1) SW term vanishes."""
    L = (4, 4, 6, 4)
    geom = Geometry(L, 0, (np.pi, 0, 0, 0))
    U, _ = workload.unit_gauge_field(L)
    phi = np.array([0.31, -0.17, 0.52, 0.09])
    A = np.broadcast_to(phi, (geom.Vphys, 4)).copy()
    kappa = 0.125
    op = DiracOperator(GaugeField(geom, U, A, 6.0), Flavour(qhat, kappa, 1.9, 1.7))
    rng = np.random.default_rng(2)
    for p in allowed_momenta(geom, rng, 4):
        chi = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        got = op.apply(plane_wave(geom, p, chi))
        want = plane_wave(geom, p, free_matrix(kappa, p + qhat * phi) @ chi)
        assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def test_sw_term_vanishes_on_unit_links():
    op, _, _ = make_op((4, 4, 4, 4), cstar=2, free=True)
    assert np.abs(op.sw_term(op.geom.sites())).max() == 0.0


def test_qcd_only_limit_ignores_photon():
    """qhat = 0: the U(1) field drops out (hopping and SW term)."""
    L = (4, 4, 4, 4)
    geom = Geometry(L, 1, (np.pi, 0, 0, 0))
    U, A = workload.gauge_field(L, 3, device="cpu")
    fl = Flavour(0, 0.13, 1.9, 1.0)
    op1 = DiracOperator(GaugeField(geom, U, A, 6.0), fl)
    op2 = DiracOperator(GaugeField(geom, U, np.zeros_like(A), 6.0), fl)
    psi = workload.spinor(geom.V, 4)
    assert np.abs(op1.apply(psi) - op2.apply(psi)).max() < 1e-14


def test_qed_only_limit_is_colour_diagonal():
    """U = 1: D is the identity in colour space (each colour sees the same operator)."""
    L = (4, 4, 4, 4)
    geom = Geometry(L, 2, (np.pi, 0, 0, 0))
    U, _ = workload.unit_gauge_field(L)
    _, A = workload.gauge_field(L, 3, device="cpu")
    op = DiracOperator(GaugeField(geom, U, A, 6.0), Flavour(4, 0.13, 1.9, 1.0))
    psi = workload.spinor(geom.V, 4)
    psi[:, :, 1:] = 0.0
    out = op.apply(psi)
    assert np.abs(out[:, :, 1:]).max() == 0.0
    psi2 = np.roll(psi, 2, axis=2)  # same spin field in colour 2
    assert np.abs(op.apply(psi2)[:, :, 2] - out[:, :, 0]).max() < 1e-14


def dhat_free_eigenvalues(geom, kappa):
    """Closed form of the free even-odd operator: with h = -c +- i s the
    eigenvalues of the free hopping matrix (c = sum cos p, s = |sin p|),
    Dhat = m - h^2/m (m = 1/(2 kappa)); p and p + (pi,pi,pi,pi) give the same values."""
    m = 1.0 / (2 * kappa)
    vals = []
    L, N = geom.L, geom.N
    import itertools
    ranges = [range(N[0]), range(N[1]), range(L[2]), range(L[3])]
    for n0, n1, n2, n3 in itertools.product(*ranges):
        p = np.zeros(4)
        p[0] = (2 * np.pi * n0 + geom.theta[0]) / L[0]
        if geom.cstar:
            p[1] = np.pi * n1 / L[1]
            p[2] = np.pi * (2 * n2 + n1) / L[2] if geom.cstar >= 2 else 2 * np.pi * n2 / L[2]
            p[3] = np.pi * (2 * n3 + n1) / L[3] if geom.cstar >= 3 else 2 * np.pi * n3 / L[3]
        else:
            p[1] = (2 * np.pi * n1 + geom.theta[1]) / L[1]
            p[2] = (2 * np.pi * n2 + geom.theta[2]) / L[2]
            p[3] = (2 * np.pi * n3 + geom.theta[3]) / L[3]
        c = np.sum(np.cos(p))
        s = np.sqrt(np.sum(np.sin(p) ** 2))
        for h in (-c + 1j * s, -c - 1j * s):
            vals += [m - h * h / m] * 6   # 2 spin x 3 colour
    vals = np.array(vals)
    return vals  # every value appears twice as often as in Dhat


@pytest.mark.parametrize("L,cstar,theta", [((4, 4, 2, 2), 0, (np.pi, 0.4, 0, 0)),
                                           ((4, 2, 4, 2), 1, (np.pi, 0, 0, 0)),
                                           ((2, 2, 4, 4), 3, (np.pi, 0, 0, 0))])
def test_free_dhat_spectrum_dense(L, cstar, theta):
    geom = Geometry(L, cstar, theta)
    U, A = workload.unit_gauge_field(L)
    kappa = 0.13
    op = DiracOperator(GaugeField(geom, U, A, 6.0), Flavour(-2, kappa, 1.9, 1.0))
    ne = len(op.even_sites())
    Dinv = op.Doo_inv()
    M = dense(lambda v: op.Dhat(v, Dinv), ne * 12, (ne, 4, 3))
    ev = np.linalg.eigvals(M)
    closed = np.sort_complex(dhat_free_eigenvalues(geom, kappa))[::2]
    cost = np.abs(ev[:, None] - closed[None, :])
    r, c = linear_sum_assignment(cost)
    assert cost[r, c].max() < 1e-9
