"""O(a)-improved Wilson-Dirac operator with SU(3) x U(1) links (Sec. 2.3).

    D = m0 + D_w + dD_sw + dD_b               (eq. dirac; dD_b = 0 for periodic time)
    D_w = sum_mu 1/2 {gamma_mu (nabla_mu + nabla*_mu) - nabla*_mu nabla_mu}
    nabla_mu  psi(x) = U(x,mu) z(x,mu)^qhat psi(x+mu) - psi(x)            (eq. frw-covder)
    nabla*_mu psi(x) = psi(x) - U(x-mu,mu)^+ z(x-mu,mu)^-qhat psi(x-mu)    (eq. bkw-covder)
    dD_sw = csw_su3 sum_{mu,nu} (i/4) sigma_{mu nu} Fhat_{mu nu}
          + q csw_u1 sum_{mu,nu} (i/4) sigma_{mu nu} Ahat_{mu nu}        (eq. sw-term)
    Ahat_{mu nu}(x) = i/(4 qel) Im{z_{mu nu}(x) + z_{mu nu}(x-mu) + z_{mu nu}(x-nu)
                                   + z_{mu nu}(x-mu-nu)}
    z_{mu nu}(x) = z(x,mu) z(x+mu,nu) z(x+nu,mu)^* z(x,nu)^*
    q = qhat * qel,   a m0 = 1/(2 kappa) - 4   (Sec. 4.4, kappa relation).

Expanding the covariant derivatives gives, site by site,

    (D psi)(x) = [1/(2 kappa) + dD_sw(x)] psi(x)
                 - 1/2 sum_mu [(1 - gamma_mu) V(x,mu) psi(x+mu)
                               + (1 + gamma_mu) V(x-mu,mu)^+ psi(x-mu)],
    V(x,mu) = U(x,mu) z(x,mu)^qhat,

which is what `DiracOperator.apply` evaluates literally, with explicit 4x4
gamma matrices and 3x3 colour products.

Open time boundary (the definition the paper defers to openQCD; Luescher and
Schaefer, Comput. Phys. Commun. 184 (2013) 519): the fields live on
0 <= x0 <= L0 - 1, the hops that would cross the boundary are absent (phase 0
from Geometry.neighbour), the clover leaves whose plaquette would cross it are
absent from Fhat and Ahat, and
    dD_b psi(x) = (cF - 1) (delta_{x0,0} + delta_{x0,L0-1}) psi(x),
with cF the boundary improvement coefficient (tree level cF = 1: dD_b = 0).

Readings where the paper is silent (each used identically by every test):
  * gamma basis: chiral Euclidean basis, gamma_0 = [[0,-1],[-1,0]],
    gamma_k = [[0,-i s_k],[i s_k,0]] (s_k Pauli), gamma_5 = g0 g1 g2 g3 = diag(1,1,-1,-1);
  * sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu];
  * Fhat_{mu nu} = (Q_{mu nu} - Q_{mu nu}^+)/8 with Q the sum of the four clover
    leaves at x (the construction the paper takes from Luescher et al. 1996),
    without a traceless projection;
  * the SW sums run over all ordered pairs (mu, nu) as printed.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU baseline, never by the library.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .lattice import Geometry

# --- Dirac algebra ----------------------------------------------------------
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_PAULI = [np.array([[0, 1], [1, 0]], dtype=np.complex128),
          np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
          np.array([[1, 0], [0, -1]], dtype=np.complex128)]

GAMMA = [np.block([[_Z2, -_I2], [-_I2, _Z2]])] + \
        [np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in _PAULI]
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
SIGMA = [[0.5j * (GAMMA[m] @ GAMMA[n] - GAMMA[n] @ GAMMA[m]) for n in range(4)]
         for m in range(4)]
ONE4 = np.eye(4, dtype=np.complex128)
ONE3 = np.eye(3, dtype=np.complex128)


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


@dataclass
class Flavour:
    """Parameters of one quark flavour (input-file section [Flavour n])."""
    qhat: int
    kappa: float
    su3csw: float
    u1csw: float


class GaugeField:
    """SU(3) links U and photon field A given on the physical lattice.

    On the mirror lattice (x1 >= L1 with C*) the fields are fixed by the
    orbifold constraint U(x + L1 e1) = U(x)^*, A(x + L1 e1) = -A(x)
    (eq. cstar-bc-gauge); `U` and `A` return the extended-lattice values.
    """

    def __init__(self, geom: Geometry, U_phys: np.ndarray, A_phys: np.ndarray, invqel: float = 1.0):
        self.geom = geom
        self.Up = np.asarray(U_phys, dtype=np.complex128).reshape(geom.Vphys, 4, 3, 3)
        self.Ap = np.asarray(A_phys, dtype=np.float64).reshape(geom.Vphys, 4)
        self.qel = 1.0 / float(invqel)

    def U(self, idx, mu):
        p, mirror = self.geom.physical_index(idx)
        u = self.Up[p, mu]
        return np.where(mirror[:, None, None], np.conj(u), u)

    def A(self, idx, mu):
        p, mirror = self.geom.physical_index(idx)
        a = self.Ap[p, mu]
        return np.where(mirror, -a, a)

    def z(self, idx, mu):
        """Compact U(1) link z = exp(iA) (Sec. 2)."""
        return np.exp(1j * self.A(idx, mu))


class DiracOperator:
    def __init__(self, gauge: GaugeField, flavour: Flavour):
        self.g = gauge
        self.geom = gauge.geom
        self.fl = flavour
        self._diag = None
        self._Vfull = [None] * 4
        self._nbfull = {}

    # --- links ----------------------------------------------------------------
    def V(self, idx, mu):
        """Hopping link U(x,mu) z(x,mu)^qhat (eq. frw-covder); memoised for the
        whole lattice once a large part of it is asked for."""
        idx = np.asarray(idx, dtype=np.int64)
        if self._Vfull[mu] is None and 8 * len(idx) >= self.geom.V:
            s = self.geom.sites()
            self._Vfull[mu] = self.g.U(s, mu) * (self.g.z(s, mu) ** self.fl.qhat)[:, None, None]
        if self._Vfull[mu] is not None:
            return self._Vfull[mu][idx]
        return self.g.U(idx, mu) * (self.g.z(idx, mu) ** self.fl.qhat)[:, None, None]

    def _hop(self, s, mu, sign):
        """Neighbour and boundary phase, memoised for the whole lattice."""
        if s is None:
            key = (mu, sign)
            if key not in self._nbfull:
                self._nbfull[key] = self.geom.neighbour(self.geom.sites(), mu, sign)
            return self._nbfull[key]
        return self.geom.neighbour(s, mu, sign)

    def _nb(self, idx, mu, sign):
        return self.geom.neighbour(idx, mu, sign)[0]

    # --- field tensors (eq. sw-term and the U(1) definition below it) ----------
    def Fhat(self, idx, mu, nu):
        """SU(3) clover field tensor (Q_{mu nu} - Q_{mu nu}^+)/8 at the sites idx."""
        U = self.g.U
        x = idx
        xpm = self._nb(x, mu, +1)
        xpn = self._nb(x, nu, +1)
        xmm = self._nb(x, mu, -1)
        xmn = self._nb(x, nu, -1)
        xmm_pn = self._nb(xmm, nu, +1)
        xmm_mn = self._nb(xmm, nu, -1)
        xmn_pm = self._nb(xmn, mu, +1)
        leaf1 = U(x, mu) @ U(xpm, nu) @ dag(U(xpn, mu)) @ dag(U(x, nu))
        leaf2 = U(x, nu) @ dag(U(xmm_pn, mu)) @ dag(U(xmm, nu)) @ U(xmm, mu)
        leaf3 = dag(U(xmm, mu)) @ dag(U(xmm_mn, nu)) @ U(xmm_mn, mu) @ U(xmn, nu)
        leaf4 = dag(U(xmn, nu)) @ U(xmn, mu) @ U(xmn_pm, nu) @ dag(U(x, mu))
        # leaf k is the plaquette with lower corner x, x-mu, x-mu-nu, x-nu
        inside = self.geom.plaquette_inside
        w = [inside(c, mu, nu)[:, None, None] for c in (x, xmm, xmm_mn, xmn)]
        Q = w[0] * leaf1 + w[1] * leaf2 + w[2] * leaf3 + w[3] * leaf4
        return (Q - dag(Q)) / 8.0

    def zplaq(self, idx, mu, nu):
        """U(1) plaquette z_{mu nu}(x)."""
        z = self.g.z
        return (z(idx, mu) * z(self._nb(idx, mu, +1), nu)
                * np.conj(z(self._nb(idx, nu, +1), mu)) * np.conj(z(idx, nu)))

    def Ahat(self, idx, mu, nu):
        """U(1) field tensor Ahat_{mu nu}(x) (purely imaginary scalar)."""
        xmm = self._nb(idx, mu, -1)
        xmn = self._nb(idx, nu, -1)
        xmmn = self._nb(xmm, nu, -1)
        s = sum(self.geom.plaquette_inside(c, mu, nu) * self.zplaq(c, mu, nu) for c in (idx, xmm, xmn, xmmn))
        return 1j / (4.0 * self.g.qel) * s.imag

    def sw_term(self, idx):
        """dD_sw at the sites idx as 12x12 matrices, index = 3*spin + colour."""
        n = len(idx)
        q = self.fl.qhat * self.g.qel
        M = np.zeros((n, 4, 3, 4, 3), dtype=np.complex128)
        for mu in range(4):
            for nu in range(4):
                if mu == nu:
                    continue
                G = (self.fl.su3csw * self.Fhat(idx, mu, nu)
                     + q * self.fl.u1csw * self.Ahat(idx, mu, nu)[:, None, None] * ONE3)
                M += 0.25j * np.einsum('ab,nij->naibj', SIGMA[mu][nu], G)
        return M.reshape(n, 12, 12)

    def diag_term(self, idx):
        """Site-diagonal part m0 + 4 + dD_sw + dD_b = 1/(2 kappa) + dD_sw + dD_b (12x12).

        It depends on the gauge field only, so once a large part of the lattice
        is asked for, it is computed for every site and kept."""
        idx = np.asarray(idx, dtype=np.int64)
        if self._diag is None and 8 * len(idx) >= self.geom.V:
            self._diag = self._diag_at(self.geom.sites())
        if self._diag is not None:
            return self._diag[idx]
        return self._diag_at(idx)

    def _diag_at(self, idx):
        dDb = (self.geom.cF - 1.0) * self.geom.boundary_slice(idx)  # dD_b (open boundary)
        return self.sw_term(idx) + (1.0 / (2.0 * self.fl.kappa) + dDb)[:, None, None] * np.eye(12)

    # --- the operator ---------------------------------------------------------
    def apply(self, psi, sites=None):
        """(D psi)(x) for x in `sites` (all extended sites by default).

        psi: complex [V][4][3] on the extended lattice.  Returns [len(sites)][4][3].
        """
        geom = self.geom
        psi = np.asarray(psi, dtype=np.complex128).reshape(geom.V, 4, 3)
        s = geom.sites() if sites is None else np.asarray(sites, dtype=np.int64)
        out = (self.diag_term(s) @ psi[s].reshape(-1, 12, 1)).reshape(-1, 4, 3)
        for mu in range(4):
            f, ph_f = self._hop(sites if sites is None else s, mu, +1)
            b, ph_b = self._hop(sites if sites is None else s, mu, -1)
            Vf = self.V(s, mu)
            Vb = self.V(b, mu)
            # colour: (V psi)_{a i} = sum_j V_ij psi_{a j};  spin: (1 -+ gamma_mu) on index a
            fwd = (ONE4 - GAMMA[mu]) @ (ph_f[:, None, None] * psi[f] @ np.swapaxes(Vf, -1, -2))
            bwd = (ONE4 + GAMMA[mu]) @ (ph_b[:, None, None] * psi[b] @ np.conj(Vb))
            out -= 0.5 * (fwd + bwd)
        return out

    # --- even-odd preconditioning (Sec. 2.3, definition of D-hat) -------------
    def even_sites(self):
        return self.geom.sites(0)

    def odd_sites(self):
        return self.geom.sites(1)

    def Doo_inv(self):
        """Inverse of the odd-odd block: D_oo is site diagonal (no hop joins two
        odd sites), so its inverse is the inverse of each 12x12 diagonal term."""
        return np.linalg.inv(self.diag_term(self.odd_sites()))

    def _embed(self, v, sites):
        full = np.zeros((self.geom.V, 4, 3), dtype=np.complex128)
        full[sites] = np.asarray(v).reshape(-1, 4, 3)
        return full

    def Doe(self, psi_e):
        return self.apply(self._embed(psi_e, self.even_sites()), self.odd_sites())

    def Deo(self, psi_o):
        return self.apply(self._embed(psi_o, self.odd_sites()), self.even_sites())

    def Dee(self, psi_e):
        return self.apply(self._embed(psi_e, self.even_sites()), self.even_sites())

    def Doo(self, psi_o):
        return self.apply(self._embed(psi_o, self.odd_sites()), self.odd_sites())

    def Dhat(self, psi_e, Doo_inv=None):
        """Dhat psi_e = D_ee psi_e - D_eo D_oo^-1 D_oe psi_e, on even sites in
        lexicographic order."""
        Dinv = self.Doo_inv() if Doo_inv is None else Doo_inv
        t = np.einsum('nab,nb->na', Dinv, self.Doe(psi_e).reshape(-1, 12)).reshape(-1, 4, 3)
        return self.Dee(psi_e) - self.Deo(t)


def gamma5(psi):
    """Multiply a spinor field [..][4][3] by gamma_5 in spin space."""
    return np.einsum('ab,...bi->...ai', GAMMA5, psi)
