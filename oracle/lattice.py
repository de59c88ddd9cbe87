"""Extended-lattice geometry of openQ*D (Sec. 2.1).

Physical lattice L0 x L1 x L2 x L3 (mu = 0 is time).  With C* boundary
conditions in `cstar` >= 1 spatial directions (turned on in the order 1, 2, 3;
Sec. 2.1, footnote on the input file) the code allocates the extended lattice
L0 x 2L1 x L2 x L3; sites with x1 >= L1 form the mirror lattice.

Neighbours on the extended lattice:
  * direction 1 with C*: periodic with period 2 L1 (eq. ext-periodic-bc);
  * C* directions k = 2, 3: crossing L_k shifts x1 by L1 (eq. ext-shifted-bc,
    Fig. cstar);
  * all other directions (time, and spatial directions without C*): periodic,
    and a spinor picks up exp(+-i theta_mu) when it is transported across the
    boundary (eq. periodic-bc-quark).  theta must vanish in the spatial
    directions when C* is on (Sec. 2.1); theta_0 = pi gives antiperiodic time.
  * open time boundary (tbc = "open"; the paper lists open and SF boundaries in
    time, Sec. 2.3 eq. dirac, and defers their definition to openQCD, Luescher
    and Schaefer, Comput. Phys. Commun. 184 (2013) 519): the lattice ends at
    x0 = 0 and x0 = L0 - 1.  Nothing is transported across: the phase of a step
    across the time boundary is 0, and a plaquette in a plane containing time
    whose lower corner has x0 = L0 - 1 does not exist (plaquette_inside).  The
    boundary improvement coefficient cF enters dD_b (dirac.py).

Site index: lexicographic with x0 slowest, idx = ((x0*N1 + x1)*N2 + x2)*N3 + x3
where N = extended extents.  Parity = (x0 + x1 + x2 + x3) mod 2 (0 = even).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU baseline, never by the library.
"""
from __future__ import annotations

import numpy as np


class Geometry:
    def __init__(self, L, cstar: int = 0, theta=(0.0, 0.0, 0.0, 0.0), tbc: str = "periodic", cF: float = 1.0):
        self.L = tuple(int(v) for v in L)
        self.cstar = int(cstar)
        self.theta = tuple(float(t) for t in theta)
        self.tbc = str(tbc)
        self.cF = float(cF)
        if self.tbc not in ("periodic", "open"):
            raise ValueError("tbc must be 'periodic' or 'open'")
        if self.tbc == "open" and self.theta[0] != 0.0:
            raise ValueError("theta_0 must vanish with an open time boundary")
        if not 0 <= self.cstar <= 3:
            raise ValueError("cstar must be 0..3")
        if any(v <= 0 or v % 2 for v in self.L):
            raise ValueError("every extent must be even and positive (even-odd ordering)")
        if self.cstar and any(self.theta[k] != 0.0 for k in (1, 2, 3)):
            raise ValueError("spatial theta must vanish with C* boundary conditions")
        L0, L1, L2, L3 = self.L
        self.N = (L0, 2 * L1 if self.cstar else L1, L2, L3)
        self.V = int(np.prod(self.N))
        self.Vphys = int(np.prod(self.L))

    # --- coordinates -------------------------------------------------------
    def coords(self, idx):
        idx = np.asarray(idx, dtype=np.int64)
        N0, N1, N2, N3 = self.N
        x3 = idx % N3
        x2 = (idx // N3) % N2
        x1 = (idx // (N3 * N2)) % N1
        x0 = idx // (N3 * N2 * N1)
        return np.stack([x0, x1, x2, x3])

    def index(self, x):
        N0, N1, N2, N3 = self.N
        return ((x[0] * N1 + x[1]) * N2 + x[2]) * N3 + x[3]

    def parity(self, idx):
        return self.coords(idx).sum(axis=0) % 2

    def sites(self, parity=None):
        allsites = np.arange(self.V, dtype=np.int64)
        if parity is None:
            return allsites
        return allsites[self.parity(allsites) == parity]

    # --- neighbours --------------------------------------------------------
    def neighbour(self, idx, mu: int, sign: int):
        """Site reached from idx by one step sign*mu-hat, and the phase a spinor
        field picks up on the way (1 unless a phase-periodic boundary is crossed).
        """
        x = self.coords(idx).copy()
        N = self.N
        x[mu] += sign
        phase = np.ones(x.shape[1], dtype=np.complex128)
        crossed = (x[mu] < 0) | (x[mu] >= N[mu])
        x[mu] %= N[mu]
        shifted = self.cstar >= 1 and mu >= 2 and mu <= self.cstar
        if mu == 0 and self.tbc == "open":
            # open boundary: no transport across x0 = L0 - 1 <-> 0
            phase = np.where(crossed, 0.0 + 0j, 1.0 + 0j)
        elif shifted:
            # eq. ext-shifted-bc: x + L_k e_k is identified with x + L_1 e_1
            x[1] = np.where(crossed, (x[1] + self.L[1]) % N[1], x[1])
        elif not (self.cstar >= 1 and mu == 1):
            phase = np.where(crossed, np.exp(1j * sign * self.theta[mu]), 1.0 + 0j)
        return self.index(x), phase

    def plaquette_inside(self, corner, mu: int, nu: int):
        """True for the plaquettes (lower corner `corner`, plane mu nu) that lie on
        the lattice: all of them unless the time boundary is open, where those in
        a plane containing time with corner x0 = L0 - 1 would cross it."""
        corner = np.asarray(corner, dtype=np.int64)
        if self.tbc != "open" or (mu != 0 and nu != 0):
            return np.ones(corner.shape, dtype=bool)
        return self.coords(corner)[0] != self.N[0] - 1

    def boundary_slice(self, idx):
        """True on the time slices x0 = 0 and x0 = L0 - 1 of an open lattice."""
        if self.tbc != "open":
            return np.zeros(np.shape(idx), dtype=bool)
        x0 = self.coords(idx)[0]
        return (x0 == 0) | (x0 == self.N[0] - 1)

    def translate(self, idx, shift):
        """Site idx + shift (an extended-lattice vector) on the extended torus."""
        out = np.asarray(idx, dtype=np.int64)
        for mu in range(4):
            s = int(shift[mu])
            step = 1 if s > 0 else -1
            for _ in range(abs(s)):
                out, _ = self.neighbour(out, mu, step)
        return out

    # --- physical <-> extended --------------------------------------------
    def physical_index(self, idx):
        """For an extended site: (index of its physical partner, is_mirror)."""
        x = self.coords(idx)
        mirror = np.zeros(x.shape[1], dtype=bool)
        if self.cstar:
            mirror = x[1] >= self.L[1]
            x = x.copy()
            x[1] = np.where(mirror, x[1] - self.L[1], x[1])
        L0, L1, L2, L3 = self.L
        return ((x[0] * L1 + x[1]) * L2 + x[2]) * L3 + x[3], mirror
