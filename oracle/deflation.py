"""Inexact deflation with SAP (DFL+SAP+GCR; Sec. 4.4, solver list and the
deflation-subspace discussion).  Plain FP64 NumPy.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU baseline, never by the library.

The paper names the method (inexact deflation with SAP, one subspace per
charge) and defers its definition to the literature on local coherence and
inexact deflation.  The reading implemented here, step by step:

1. Blocks.  The lattice is tiled by blocks of b^4 sites (the SAP block grid).
2. Subspace generation.  Ns fields phi_1..phi_Ns start from given random
   fields.  ninv times: phi_k <- M_sap phi_k for every k (M_sap: the SAP
   approximation of D^-1, oracle.sap), then block orthonormalisation.
3. Block orthonormalisation.  On every block, modified Gram-Schmidt of the
   restrictions phi_k|_B in the order k = 1..Ns; the global fields are replaced
   by the concatenation of their orthonormal block pieces.
4. Prolongation and restriction.  P c = sum_{B,k} c_{B,k} phi_k|_B and
   (P^+ v)_{B,k} = <phi_k|_B, v>; P^+ P = 1.
5. Little Dirac operator.  A = P^+ D P, an (Ns Nb)^2 matrix whose (B, B') block
   vanishes unless B' = B or a nearest-neighbour block of B.
6. Preconditioner.  M_dfl v = P A^-1 P^+ v + M_sap (v - D P A^-1 P^+ v), i.e. the
   coarse correction followed by SAP on the deflated residual.  The oracle
   solves the little system exactly (dense LU).
7. As a right preconditioner of FGCR on Dhat: z_e = (M_dfl (r_e, 0))_e, as for SAP.
"""
from __future__ import annotations

import numpy as np

from .dirac import DiracOperator
from .sap import SAP


class Deflation:
    def __init__(self, op: DiracOperator, sap: SAP, seeds, ninv: int = 2):
        """seeds: complex [Ns][V][4][3] random start fields; sap: the SAP map used both
        for generating the subspace and as the smoother of the preconditioner."""
        self.op, self.sap, self.geom = op, sap, op.geom
        self.block = sap.block
        self.nblocks = sap.nblocks
        phis = np.array(seeds, dtype=np.complex128)
        self.Ns = len(phis)
        self.phis = self.orthonormalise(phis)
        for _ in range(ninv):
            phis = np.array([sap.apply(p) for p in self.phis])
            self.phis = self.orthonormalise(phis)
        self.A = self.little_operator()

    @classmethod
    def from_basis(cls, op: DiracOperator, sap: SAP, phis):
        """The same construction for a given basis (taken as it is, not regenerated
        or re-orthonormalised): lets a test evaluate A and M_dfl on another
        implementation's subspace."""
        self = cls.__new__(cls)
        self.op, self.sap, self.geom = op, sap, op.geom
        self.block = sap.block
        self.nblocks = sap.nblocks
        self.phis = np.array(phis, dtype=np.complex128)
        self.Ns = len(self.phis)
        self.A = self.little_operator()
        return self

    # --- blocks ---------------------------------------------------------------
    def block_dot(self, a, b):
        """<a|_B, b|_B> for every block B (complex, length Nb)."""
        d = np.einsum('nij,nij->n', np.conj(a), b)
        return np.bincount(self.block, weights=d.real, minlength=self.nblocks) + \
            1j * np.bincount(self.block, weights=d.imag, minlength=self.nblocks)

    def orthonormalise(self, phis):
        """Modified Gram-Schmidt of the block restrictions, block by block."""
        out = np.array(phis, dtype=np.complex128)
        for k in range(len(out)):
            for j in range(k):
                c = self.block_dot(out[j], out[k])
                out[k] = out[k] - c[self.block][:, None, None] * out[j]
            nrm = np.sqrt(self.block_dot(out[k], out[k]).real)
            out[k] = out[k] / nrm[self.block][:, None, None]
        return out

    # --- prolongation, restriction, little operator -----------------------------
    def restrict(self, v):
        """(P^+ v) as an array [Nb][Ns]."""
        return np.stack([self.block_dot(p, v) for p in self.phis], axis=1)

    def prolong(self, c):
        """P c for c [Nb][Ns]."""
        c = np.asarray(c).reshape(self.nblocks, self.Ns)
        out = np.zeros((self.geom.V, 4, 3), dtype=np.complex128)
        for k in range(self.Ns):
            out += c[self.block, k][:, None, None] * self.phis[k]
        return out

    def basis_vector(self, B, k):
        v = np.zeros((self.geom.V, 4, 3), dtype=np.complex128)
        m = self.block == B
        v[m] = self.phis[k][m]
        return v

    def little_operator(self):
        """Dense A[(B, k), (B', l)] = <phi_k|_B, D phi_l|_B'>, index B * Ns + k."""
        n = self.nblocks * self.Ns
        A = np.zeros((n, n), dtype=np.complex128)
        for Bp in range(self.nblocks):
            for l in range(self.Ns):
                w = self.op.apply(self.basis_vector(Bp, l))
                A[:, Bp * self.Ns + l] = self.restrict(w).reshape(-1)
        return A

    # --- preconditioner -----------------------------------------------------------
    def coarse_solve(self, v):
        """P A^-1 P^+ v."""
        c = np.linalg.solve(self.A, self.restrict(v).reshape(-1))
        return self.prolong(c)

    def apply(self, v):
        """M_dfl v = P A^-1 P^+ v + M_sap (v - D P A^-1 P^+ v)."""
        v = np.asarray(v, dtype=np.complex128)
        u = self.coarse_solve(v)
        return u + self.sap.apply(v - self.op.apply(u))

    def apply_even(self, r_e):
        """(M_dfl (r_e, 0))_e for an even-site field."""
        full = np.zeros((self.geom.V, 4, 3), dtype=np.complex128)
        ev = self.op.even_sites()
        full[ev] = r_e
        return self.apply(full)[ev]


def block_neighbours(sap: SAP, geom):
    """For every block B and slot s (0: B itself; 1 + 2 mu: the block containing
    x + mu for the sites x on B's +mu face; 2 + 2 mu: the -mu face), the block
    index, read off the neighbour map of the lattice (C* shifts included)."""
    nb = np.zeros((sap.nblocks, 9), dtype=np.int64)
    s = geom.sites()
    for B in range(sap.nblocks):
        nb[B, 0] = B
    for mu in range(4):
        f, _ = geom.neighbour(s, mu, +1)
        b, _ = geom.neighbour(s, mu, -1)
        for slot, nbr in ((1 + 2 * mu, f), (2 + 2 * mu, b)):
            cross = sap.block[nbr] != sap.block
            for B in range(sap.nblocks):
                tgt = np.unique(sap.block[nbr[(sap.block == B) & cross]])
                if len(tgt) != 1:
                    raise ValueError("a block face must face exactly one block")
                nb[B, slot] = tgt[0]
    return nb
