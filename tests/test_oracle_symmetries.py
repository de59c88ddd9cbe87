"""Pins of the oracle by symmetries the operator must have (Sec. 4.2 test list):
gamma5-hermiticity, SU(3) x U(1) gauge covariance, translation covariance on the
extended lattice, and the C* structure (Sec. 2.1: CTD antisymmetric, which is
what makes pf(CTD) well defined)."""
import numpy as np
import pytest

from oracle import DiracOperator, Flavour, GaugeField, Geometry
from oracle.dirac import GAMMA, gamma5
from paper_1908_11673_gb300 import workload
from tests.oracle_helpers import dense, make_op

BCS = [((4, 4, 4, 6), 0, (np.pi, 0.0, 0.0, 0.0)),
       ((4, 6, 4, 4), 0, (0.4, -0.3, 1.2, 0.0)),
       ((4, 4, 4, 4), 1, (np.pi, 0.0, 0.0, 0.0)),
       ((6, 4, 4, 4), 2, (np.pi, 0.0, 0.0, 0.0)),
       ((4, 4, 6, 4), 3, (0.0, 0.0, 0.0, 0.0))]


def vdot(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


@pytest.mark.parametrize("L,cstar,theta", BCS)
def test_gamma5_hermiticity(L, cstar, theta):
    op, _, _ = make_op(L, cstar, theta, qhat=4, seed=21)
    V = op.geom.V
    phi = workload.spinor(V, 1)
    psi = workload.spinor(V, 2)
    lhs = vdot(phi, gamma5(op.apply(gamma5(psi))))
    rhs = vdot(op.apply(phi), psi)
    assert abs(lhs - rhs) < 1e-13 * abs(rhs) + 1e-12
    # and not trivially: D itself is not Hermitian
    assert abs(vdot(phi, op.apply(psi)) - vdot(op.apply(phi), psi)) > 1e-3 * abs(rhs)
    ne = len(op.even_sites())
    a = workload.spinor(ne, 3)
    b = workload.spinor(ne, 4)
    Dinv = op.Doo_inv()
    lhs = vdot(a, gamma5(op.Dhat(gamma5(b), Dinv)))
    rhs = vdot(op.Dhat(a, Dinv), b)
    assert abs(lhs - rhs) < 1e-13 * abs(rhs)


def random_su3(rng, n):
    m = rng.normal(size=(n, 3, 3)) + 1j * rng.normal(size=(n, 3, 3))
    q, r = np.linalg.qr(m)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[:, None, None]


@pytest.mark.parametrize("L,cstar,theta", BCS)
def test_gauge_covariance(L, cstar, theta):
    """U(x,mu) -> g(x) U(x,mu) g(x+mu)^+,  z(x,mu) -> l(x) z(x,mu) l(x+mu)^*,
    psi -> g l^qhat psi  gives  D' psi' = (D psi)'.  With C* the transformation
    respects the orbifold (g, l on the mirror are the conjugates of the physical
    ones), so the transformed field is again a physical-lattice field."""
    qhat = -2
    op, U, A = make_op(L, cstar, theta, qhat=qhat, seed=31)
    geom = op.geom
    rng = np.random.default_rng(7)
    gp = random_su3(rng, geom.Vphys)
    ap = rng.uniform(-np.pi, np.pi, size=geom.Vphys)
    ext = geom.sites()
    pidx, mirror = geom.physical_index(ext)
    g = np.where(mirror[:, None, None], np.conj(gp[pidx]), gp[pidx])
    lam_angle = np.where(mirror, -ap[pidx], ap[pidx])
    phys = ext[~mirror]  # physical sites in physical lexicographic order
    Un = np.empty_like(U)
    An = np.empty_like(A)
    gf = op.g
    for mu in range(4):
        nb, _ = geom.neighbour(phys, mu, +1)
        Un[:, mu] = g[phys] @ gf.U(phys, mu) @ np.conj(np.swapaxes(g[nb], -1, -2))
        An[:, mu] = lam_angle[phys] + gf.A(phys, mu) - lam_angle[nb]
    op2 = DiracOperator(GaugeField(geom, Un, An, 6.0), op.fl)
    psi = workload.spinor(geom.V, 5)
    omega = g * np.exp(1j * qhat * lam_angle)[:, None, None]
    rot = lambda v: np.einsum('nij,naj->nai', omega, v)
    got = op2.apply(rot(psi))
    want = rot(op.apply(psi))
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("L,cstar,theta,shift", [
    ((4, 4, 4, 6), 0, (np.pi, 0.0, 0.0, 0.0), (1, 2, 0, 3)),
    ((4, 4, 4, 4), 1, (np.pi, 0.0, 0.0, 0.0), (0, 1, 0, 0)),
    ((4, 4, 6, 4), 3, (np.pi, 0.0, 0.0, 0.0), (1, 1, 2, 1)),
])
def test_translation_covariance(L, cstar, theta, shift):
    """Translating fields by a lattice vector t on the extended torus commutes
    with D.  With the phase-periodic time boundary a spinor transported across it
    picks up exp(-+i theta_0); with C* the translation by e_1 maps the physical
    lattice partly onto the mirror, where the fields are the conjugates."""
    op, _, _ = make_op(L, cstar, theta, qhat=4, seed=41)
    geom = op.geom
    s = geom.sites()
    # back-translated site x - t and the accumulated spinor phase
    src = s.copy()
    phase = np.ones(geom.V, dtype=np.complex128)
    for mu in range(4):
        for _ in range(shift[mu]):
            src, ph = geom.neighbour(src, mu, -1)
            phase = phase * ph
    pidx, mirror = geom.physical_index(s)
    phys = s[~mirror]
    Un = np.stack([op.g.U(src[phys], mu) for mu in range(4)], axis=1)
    An = np.stack([op.g.A(src[phys], mu) for mu in range(4)], axis=1)
    op2 = DiracOperator(GaugeField(geom, Un, An, 6.0), op.fl)
    psi = workload.spinor(geom.V, 9)
    T = lambda v: phase[:, None, None] * v[src]
    got = op2.apply(T(psi))
    want = T(op.apply(psi))
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def charge_conjugation_matrix():
    """C with C^-1 gamma_mu C = -gamma_mu^T for all mu (Sec. 2.1), found as the
    null space of the linear conditions gamma_mu C + C gamma_mu^T = 0 and
    normalised to be unitary."""
    rows = []
    for g in GAMMA:
        # vec(g C + C g^T) = (I (x) g + g (x) I) vec(C) in column-major vec
        rows.append(np.kron(np.eye(4), g) + np.kron(g, np.eye(4)))
    Mt = np.concatenate(rows, axis=0)
    _, sv, vh = np.linalg.svd(Mt)
    assert sv[-1] < 1e-12 and sv[-2] > 1e-3
    C = vh[-1].conj().reshape(4, 4, order='F')
    C = C / np.sqrt(abs(np.linalg.det(C))) ** 0.5
    return C


def test_charge_conjugation_properties():
    C = charge_conjugation_matrix()
    assert np.allclose(C.T, -C, atol=1e-12)
    assert np.allclose(C.conj().T @ C, np.eye(4), atol=1e-12)
    for g in GAMMA:
        assert np.allclose(np.linalg.inv(C) @ g @ C, -g.T, atol=1e-12)


@pytest.mark.parametrize("L,cstar", [((4, 2, 4, 2), 1), ((2, 2, 4, 2), 2), ((2, 2, 2, 4), 3)])
def test_cstar_CTD_is_antisymmetric(L, cstar):
    """With C* boundaries the Pfaffian pf(CTD) exists because C T D is
    antisymmetric (Sec. 2.1, T psi(x) = psi(x + L1 e1)).  This fails if the mirror
    gauge field is not the conjugate of the physical one, or if the shifted
    boundary of eq. ext-shifted-bc is wrong."""
    op, _, _ = make_op(L, cstar, (np.pi, 0, 0, 0), qhat=4, seed=51, sigma_h=0.6, sigma_a=0.5)
    geom = op.geom
    V = geom.V
    D = dense(lambda v: op.apply(v), V * 12, (V, 4, 3))
    C = charge_conjugation_matrix()
    shift = np.zeros(4, dtype=int)
    shift[1] = geom.L[1]
    Tsrc = geom.translate(geom.sites(), shift)
    T = np.zeros((V, V))
    T[np.arange(V), Tsrc] = 1.0
    CT = np.kron(T, np.kron(C, np.eye(3)))
    M = CT @ D
    assert np.abs(M + M.T).max() < 1e-12 * np.abs(M).max()
    # planted mistake: a mirror field that is a copy (not the conjugate) of the
    # physical one must break the antisymmetry
    class CopiedMirror(GaugeField):
        def U(self, idx, mu):
            p, _ = self.geom.physical_index(idx)
            return self.Up[p, mu]

        def A(self, idx, mu):
            p, _ = self.geom.physical_index(idx)
            return self.Ap[p, mu]

    bad = DiracOperator(CopiedMirror(geom, op.g.Up, op.g.Ap, 6.0), op.fl)
    Mb = CT @ dense(lambda v: bad.apply(v), V * 12, (V, 4, 3))
    assert np.abs(Mb + Mb.T).max() > 1e-3 * np.abs(Mb).max()


def test_cstar_mirror_links_are_conjugate():
    op, U, A = make_op((4, 4, 4, 4), 3, (np.pi, 0, 0, 0))
    geom = op.geom
    s = geom.sites()
    p, mirror = geom.physical_index(s)
    for mu in range(4):
        assert np.array_equal(op.g.U(s[mirror], mu), np.conj(U[p[mirror], mu]))
        assert np.array_equal(op.g.A(s[mirror], mu), -A[p[mirror], mu])


@pytest.mark.parametrize("cstar", [0, 1, 2, 3])
def test_neighbour_map_is_a_bijection_with_inverse(cstar):
    geom = Geometry((4, 6, 4, 8), cstar, (np.pi, 0, 0, 0))
    s = geom.sites()
    for mu in range(4):
        f, ph_f = geom.neighbour(s, mu, +1)
        assert len(np.unique(f)) == geom.V
        b, ph_b = geom.neighbour(f, mu, -1)
        assert np.array_equal(b, s)
        assert np.allclose(ph_f * ph_b, 1.0)
        # hops join opposite parities (even-odd preconditioning needs this)
        assert np.all(geom.parity(f) != geom.parity(s))
