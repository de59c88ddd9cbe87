"""Pins of the SW term normalisation (eq. sw-term and the U(1) field tensor of
Sec. 2.3) by a constant abelian flux.

On a torus, the U(1) field z_2(x) = exp(i phi x1) for 0 <= x1 < L1, and
z_1(x) = exp(-i phi L1 x2) on the links leaving x1 = L1 - 1 (1 elsewhere) with
phi = 2 pi n / (L1 L2), has every (1,2) plaquette equal to exp(i phi) and all
other plaquettes equal to 1.  Then all four clover leaves are equal and
  * U(1):  q Ahat_12 = i qhat sin(phi)    (Ahat = i/(4 qel) Im{4 e^{i phi}}, q = qhat qel),
           dD_sw = q csw_u1 [ (i/4) s_12 Ahat_12 + (i/4) s_21 Ahat_21 ]
                 = -(qhat csw_u1 sin phi / 2) s_12 (x) 1_colour;
  * SU(3) (the same construction with a diagonal flux phi_a per colour,
    sum_a n_a = 0): Fhat_12 = i diag(sin phi_a) and
           dD_sw = -(csw_su3 / 2) s_12 (x) diag(sin phi_a).
s_12 = (i/2)[g_1, g_2] squares to one, so its eigenvalues are +-1 (twice each).
Hence the 12 eigenvalues of the SW term are +-(csw/2) sin(phi_a) for SU(3) and
+-(qhat csw_u1/2) sin(phi) for U(1), whatever the gamma basis.  A wrong 1/8,
i/4, the factor 2 from ordered pairs, or sin(qhat phi) in place of
qhat sin(phi) changes these numbers.
"""
import numpy as np
import pytest

from oracle import DiracOperator, Flavour, GaugeField, Geometry
from paper_1908_11673_gb300 import workload


def flux_angles(L, n):
    """A_1, A_2 angles of the constant-flux U(1) field in the (1,2) plane."""
    geom = Geometry(L, 0)
    x = geom.coords(geom.sites())
    phi = 2 * np.pi * n / (L[1] * L[2])
    A = np.zeros((geom.V, 4))
    A[:, 2] = phi * x[1]
    A[:, 1] = np.where(x[1] == L[1] - 1, -phi * L[1] * x[2], 0.0)
    return A, phi


@pytest.mark.parametrize("qhat,csw", [(1, 1.0), (-2, 1.0), (4, 1.7)])
def test_u1_sw_term_constant_flux(qhat, csw):
    L = (4, 4, 6, 4)
    A, phi = flux_angles(L, 1)
    U, _ = workload.unit_gauge_field(L)
    geom = Geometry(L, 0, (np.pi, 0, 0, 0))
    op = DiracOperator(GaugeField(geom, U, A, 6.0), Flavour(qhat, 0.13, 1.9, csw))
    sites = geom.sites()[::7]
    ev = np.sort(np.linalg.eigvalsh(op.sw_term(sites)), axis=1)
    a = qhat * csw * np.sin(phi) / 2
    want = np.sort(np.array([-abs(a)] * 6 + [abs(a)] * 6))
    assert np.abs(ev - want).max() < 1e-13
    assert abs(np.sin(qhat * phi) - qhat * np.sin(phi)) > 1e-3 or abs(qhat) == 1


def test_su3_sw_term_constant_flux():
    L = (4, 6, 4, 4)
    n = np.array([1, 2, -3])
    geom = Geometry(L, 0, (np.pi, 0, 0, 0))
    U, _ = workload.unit_gauge_field(L)
    phis = []
    for a in range(3):
        Aa, ph = flux_angles(L, n[a])
        phis.append(ph)
        for mu in (1, 2):
            U[:, mu, a, a] = np.exp(1j * Aa[:, mu])
    assert np.allclose(np.linalg.det(U), 1.0)
    csw = 1.90952
    op = DiracOperator(GaugeField(geom, U, np.zeros((geom.V, 4)), 6.0), Flavour(-2, 0.13, csw, 1.0))
    sites = geom.sites()[::5]
    ev = np.sort(np.linalg.eigvalsh(op.sw_term(sites)), axis=1)
    vals = []
    for ph in phis:
        vals += [csw * np.sin(ph) / 2, -csw * np.sin(ph) / 2] * 2
    want = np.sort(np.array(vals))
    assert np.abs(ev - want).max() < 1e-13


def test_sw_term_is_hermitian_and_chirally_block_diagonal():
    """The field tensors are anti-Hermitian (Sec. 2.3), so dD_sw is Hermitian, and
    sigma_{mu nu} commutes with gamma_5: the 12x12 term splits into two 6x6
    blocks of definite chirality (the structure the CUDA path stores)."""
    from oracle.dirac import GAMMA5
    L = (4, 4, 4, 4)
    geom = Geometry(L, 2, (np.pi, 0, 0, 0))
    U, A = workload.gauge_field(L, 8, device="cpu")
    op = DiracOperator(GaugeField(geom, U, A, 6.0), Flavour(4, 0.13, 1.9, 1.0))
    M = op.sw_term(geom.sites())
    assert np.abs(M - np.conj(np.swapaxes(M, 1, 2))).max() < 1e-14
    g5 = np.kron(GAMMA5, np.eye(3))
    assert np.abs(g5 @ M - M @ g5).max() < 1e-14
