"""Pins of the oracle's open time boundary (Sec. 2.3 eq. dirac, term dD_b; the
definition the paper defers to openQCD, Luescher and Schaefer, Comput. Phys.
Commun. 184 (2013) 519):

  * closed form: on the free field the operator restricted to spatially constant
    fields is block triangular in time, with determinant
    [(a + cF - 1)^2 a^(L0-2)]^12 and trace 12 [L0 a + 2 (cF - 1)], a = 1/(2 kappa) - 3
    (a dropped wrap-around hop, a dD_b on one boundary only or with another
    coefficient all change one of them);
  * time reflection x0 -> L0 - 1 - x0 with gamma0 gamma5 commutes with the free
    operator (dD_b on the wrong slices breaks it);
  * D does not depend on the links that would cross the boundary (a clover leaf
    or a hop kept across it would);
  * away from the boundary (1 <= x0 <= L0 - 2) D is the periodic operator, whose
    own pins are in test_oracle_free_field.py and test_oracle_symmetries.py;
  * gamma5-hermiticity and SU(3) x U(1) gauge covariance with the boundary open;
  * cF = 1 (tree level) gives dD_b = 0: D(cF) - D(1) is (cF - 1) on the boundary
    slices and nothing else.
"""
import numpy as np
import pytest

from oracle import DiracOperator, Flavour, GaugeField, Geometry
from oracle.dirac import GAMMA, GAMMA5
from paper_1908_11673_gb300 import workload

KAPPA = 0.13
CF = 1.37


def make(L, cstar=0, cF=CF, U=None, A=None, seed=17, qhat=-2, free=False):
    geom = Geometry(L, cstar, (0.0, 0.0, 0.0, 0.0), tbc="open", cF=cF)
    if U is None:
        U, A = workload.unit_gauge_field(L) if free else workload.gauge_field(L, seed, device="cpu")
    op = DiracOperator(GaugeField(geom, U, A, 6.0), Flavour(qhat, KAPPA, 1.90952, 1.0))
    return op, U, A


def test_free_zero_momentum_block_closed_form():
    L = (6, 4, 4, 4)
    op, _, _ = make(L, free=True)
    geom = op.geom
    T = L[0]
    nsp = geom.V // T
    # basis of spatially constant fields: time slice t, spin-colour component k
    M = np.zeros((12 * T, 12 * T), dtype=np.complex128)
    x0 = geom.coords(geom.sites())[0]
    for t in range(T):
        for k in range(12):
            psi = np.zeros((geom.V, 12), dtype=np.complex128)
            psi[x0 == t, k] = 1.0
            out = op.apply(psi.reshape(-1, 4, 3)).reshape(geom.V, 12)
            # project back on spatially constant fields (the free operator keeps them)
            for s in range(T):
                M[12 * s:12 * s + 12, 12 * t + k] = out[x0 == s].sum(axis=0) / nsp
    a = 1.0 / (2.0 * KAPPA) - 3.0
    sign, logdet = np.linalg.slogdet(M)
    expect = 12 * (2 * np.log(a + CF - 1.0) + (T - 2) * np.log(a))
    assert abs(logdet - expect) < 1e-10 and abs(sign - 1.0) < 1e-10
    assert abs(np.trace(M) - 12 * (T * a + 2 * (CF - 1.0))) < 1e-10
    # nothing couples the two ends of the chain
    assert np.abs(M[:12, 12 * (T - 1):]).max() == 0 and np.abs(M[12 * (T - 1):, :12]).max() == 0


def test_free_time_reflection_symmetry():
    L = (6, 4, 4, 4)
    op, _, _ = make(L, free=True)
    geom = op.geom
    x = geom.coords(geom.sites())
    xr = x.copy()
    xr[0] = L[0] - 1 - x[0]
    refl = geom.index(xr)
    R = GAMMA[0] @ GAMMA5

    def reflect(psi):
        return np.einsum("ab,nbi->nai", R, psi[refl])

    psi = workload.spinor(geom.V, 3)
    assert np.linalg.norm(op.apply(reflect(psi)) - reflect(op.apply(psi))) < 1e-12 * np.linalg.norm(psi)
    # an improvement term on the slices 1 and L0 - 1 (not symmetric) is caught
    wrong = op.apply(psi) + (CF - 1.0) * np.where((x[0] == 1)[:, None, None], psi, 0)
    wrong_r = op.apply(reflect(psi)) + (CF - 1.0) * np.where((x[0] == 1)[:, None, None], reflect(psi), 0)
    assert np.linalg.norm(wrong_r - reflect(wrong)) > 1e-3 * np.linalg.norm(psi)


@pytest.mark.parametrize("cstar", [0, 1])
def test_independent_of_links_across_the_boundary(cstar):
    L = (4, 4, 4, 6)
    op, U, A = make(L, cstar)
    geom = Geometry(L, 0)
    x0 = geom.coords(geom.sites())[0]
    last = x0 == L[0] - 1
    rng = np.random.default_rng(5)
    U2, A2 = U.copy(), A.copy()
    U2[last, 0] = workload.gauge_field(L, 99, device="cpu")[0][last, 0]
    A2[last, 0] = rng.normal(0.0, 1.0, size=last.sum())
    op2, _, _ = make(L, cstar, U=U2, A=A2)
    psi = workload.spinor(op.geom.V, 4)
    assert np.array_equal(op.apply(psi), op2.apply(psi))
    # the periodic operator does depend on them
    per = lambda u, a: DiracOperator(GaugeField(Geometry(L, cstar, (0.0, 0, 0, 0)), u, a, 6.0),
                                     Flavour(-2, KAPPA, 1.90952, 1.0))
    assert np.linalg.norm(per(U, A).apply(psi) - per(U2, A2).apply(psi)) > 1e-3 * np.linalg.norm(psi)


@pytest.mark.parametrize("cstar", [0, 2])
def test_interior_equals_periodic_operator(cstar):
    L = (6, 4, 4, 4)
    op, U, A = make(L, cstar)
    per = DiracOperator(GaugeField(Geometry(L, cstar, (0.0, 0, 0, 0)), U, A, 6.0), Flavour(-2, KAPPA, 1.90952, 1.0))
    geom = op.geom
    x0 = geom.coords(geom.sites())[0]
    inner = geom.sites()[(x0 >= 1) & (x0 <= L[0] - 2)]
    edge = geom.sites()[(x0 == 0) | (x0 == L[0] - 1)]
    psi = workload.spinor(geom.V, 5)
    assert np.linalg.norm(op.apply(psi, inner) - per.apply(psi, inner)) < 1e-13 * np.linalg.norm(psi[inner])
    assert np.linalg.norm(op.apply(psi, edge) - per.apply(psi, edge)) > 1e-2 * np.linalg.norm(psi[edge])


@pytest.mark.parametrize("cstar", [0, 3])
def test_gamma5_hermiticity(cstar):
    op, _, _ = make((4, 4, 4, 4), cstar)
    V = op.geom.V
    phi, psi = workload.spinor(V, 6), workload.spinor(V, 7)
    g5 = lambda v: np.einsum("ab,nbi->nai", GAMMA5, v)
    lhs = np.vdot(phi, g5(op.apply(g5(psi))))
    rhs = np.vdot(op.apply(phi), psi)
    assert abs(lhs - rhs) < 1e-13 * np.linalg.norm(phi) * np.linalg.norm(psi) * 10


def test_gauge_covariance():
    L = (4, 4, 4, 4)
    qhat = 3
    op, U, A = make(L, qhat=qhat)
    geom = op.geom
    V = geom.V
    rng = np.random.default_rng(8)
    g = workload.gauge_field(L, 123, device="cpu")[0][:, 0]  # one SU(3) matrix per site
    lam = rng.uniform(-np.pi, np.pi, size=V)
    Ug = np.empty_like(U)
    Ag = np.empty_like(A)
    for mu in range(4):
        xp, _ = Geometry(L, 0).neighbour(geom.sites(), mu, +1)
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[xp], -1, -2))
        Ag[:, mu] = A[:, mu] + lam - lam[xp]
    opg, _, _ = make(L, U=Ug, A=Ag, qhat=qhat)
    psi = workload.spinor(V, 9)
    Om = lambda v: np.exp(1j * qhat * lam)[:, None, None] * np.einsum("nij,naj->nai", g, v)
    Om_dag = lambda v: np.exp(-1j * qhat * lam)[:, None, None] * np.einsum("nji,naj->nai", np.conj(g), v)
    assert np.linalg.norm(opg.apply(psi) - Om(op.apply(Om_dag(psi)))) < 1e-12 * np.linalg.norm(psi)


def test_tree_level_coefficient_gives_no_boundary_term():
    L = (4, 4, 4, 4)
    op, U, A = make(L, cF=1.0)
    opc, _, _ = make(L, cF=CF, U=U, A=A)
    geom = op.geom
    psi = workload.spinor(geom.V, 10)
    bnd = geom.boundary_slice(geom.sites())
    diff = opc.apply(psi) - op.apply(psi)
    assert np.linalg.norm(diff[~bnd]) == 0.0
    assert np.linalg.norm(diff[bnd] - (CF - 1.0) * psi[bnd]) < 1e-13 * np.linalg.norm(psi[bnd])


def test_geometry_rejects_time_phase_with_open_boundary():
    with pytest.raises(ValueError):
        Geometry((4, 4, 4, 4), 0, (np.pi, 0, 0, 0), tbc="open")
