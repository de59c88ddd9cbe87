"""Schwarz alternating procedure (SAP) preconditioner (Sec. 4.1 and 4.4: SAP+GCR
with block size 4^4, ncy = 5 cycles, nmr = 5 minimal-residual steps).  Plain
FP64 NumPy.

The lattice is tiled by non-overlapping blocks of b^4 sites, coloured like a
checkerboard by the parity of the block coordinates.  Every extent must hold an
even number of blocks: then blocks of one colour never touch (across the
periodic boundary included), no hop joins a block to itself, and every block
face is a Dirichlet boundary.  The block operator D_B
is D restricted to a block with Dirichlet boundary conditions: hops that leave
the block are dropped.  One application of the preconditioner M to a source eta:

    psi = 0, rho = eta
    repeat ncy times, for colour in (0, 1):
        on every block B of that colour (independently):
            solve D_B d = rho|_B approximately, with the even-odd system of the block
                b_e   = rho_e - H^B_eo A_oo^-1 rho_o
                nmr minimal-residual steps on Dhat_B y = b_e from y = 0
                    (p = Dhat_B r, alpha = <p, r>/<p, p>, y += alpha r, r -= alpha p)
                d_e = y,  d_o = A_oo^-1 (rho_o - H^B_oe y)
            psi|_B += d
        rho = eta - D psi
    M eta = psi

The minimal-residual steps and the colouring are as in Luescher's SAP (which
the paper uses through openQCD); the block even-odd splitting is the standard
one.  As a preconditioner of the even-odd operator Dhat the project uses
(M (r_e, 0))_e, because Dhat^-1 = (D^-1)_ee.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU baseline, never by the library.
"""
from __future__ import annotations

import numpy as np

from .dirac import DiracOperator, GAMMA, ONE4


class SAP:
    def __init__(self, op: DiracOperator, bsize: int = 4, ncy: int = 5, nmr: int = 5):
        geom = op.geom
        if any(n % (2 * bsize) for n in geom.N):
            raise ValueError("every simulated extent must hold an even number of blocks")
        self.op, self.geom = op, geom
        self.b, self.ncy, self.nmr = bsize, ncy, nmr
        s = geom.sites()
        x = geom.coords(s)
        bc = x // bsize
        nb = [n // bsize for n in geom.N]
        self.block = ((bc[0] * nb[1] + bc[1]) * nb[2] + bc[2]) * nb[3] + bc[3]
        self.colour = bc.sum(axis=0) % 2
        self.parity = geom.parity(s)
        self.nblocks = int(np.prod(nb))
        # neighbours that stay inside the block
        self.nb = {}
        for mu in range(4):
            f, ph_f = geom.neighbour(s, mu, +1)
            b, ph_b = geom.neighbour(s, mu, -1)
            self.nb[mu] = (f, ph_f, self.block[f] == self.block, b, ph_b, self.block[b] == self.block)
        self.Vlink = [op.V(s, mu) for mu in range(4)]
        self.diag = op.diag_term(s)
        self.diag_inv = np.linalg.inv(self.diag)

    # hopping term with Dirichlet block boundaries, on the sites of parity `p_out`
    def hop_block(self, v, p_out):
        op = self.op
        out = np.zeros_like(v)
        for mu in range(4):
            f, ph_f, in_f, b, ph_b, in_b = self.nb[mu]
            Vf = self.Vlink[mu]
            Vb = np.conj(np.swapaxes(self.Vlink[mu][b], -1, -2))
            fwd = (ONE4 - GAMMA[mu]) @ ((ph_f * in_f)[:, None, None] * v[f] @ np.swapaxes(Vf, -1, -2))
            bwd = (ONE4 + GAMMA[mu]) @ ((ph_b * in_b)[:, None, None] * v[b] @ np.swapaxes(Vb, -1, -2))
            out -= 0.5 * (fwd + bwd)
        out[self.parity != p_out] = 0.0
        return out

    def mul_diag(self, M, v, p):
        out = np.zeros_like(v)
        m = self.parity == p
        out[m] = (M[m] @ v[m].reshape(-1, 12, 1)).reshape(-1, 4, 3)
        return out

    def block_dot(self, a, b, mask):
        """<a, b> summed over the sites of each block (only sites in mask)."""
        d = np.einsum('nij,nij->n', np.conj(a), b) * mask
        return np.bincount(self.block, weights=d.real, minlength=self.nblocks) + \
            1j * np.bincount(self.block, weights=d.imag, minlength=self.nblocks)

    def block_solve(self, rho, colour):
        """Approximate solution of D_B d = rho|_B on all blocks of one colour."""
        sel = (self.colour == colour)
        ev = sel & (self.parity == 0)
        od = sel & (self.parity == 1)
        rho = np.where(sel[:, None, None], rho, 0.0)
        t = self.mul_diag(self.diag_inv, rho, 1)
        b = np.where(ev[:, None, None], rho - self.hop_block(t, 0), 0.0)
        y = np.zeros_like(b)
        r = b.copy()
        for _ in range(self.nmr):
            t = self.mul_diag(self.diag_inv, self.hop_block(r, 1), 1)
            p = np.where(ev[:, None, None], self.mul_diag(self.diag, r, 0) - self.hop_block(t, 0), 0.0)
            pr = self.block_dot(p, r, ev)
            pp = self.block_dot(p, p, ev).real
            alpha = np.where(pp > 0, pr / np.where(pp > 0, pp, 1.0), 0.0)[self.block]
            y = y + alpha[:, None, None] * r
            r = r - alpha[:, None, None] * p
        d = y.copy()
        d_o = self.mul_diag(self.diag_inv, rho - self.hop_block(y, 1), 1)
        d[od] = d_o[od]
        return np.where(sel[:, None, None], d, 0.0)

    def apply(self, eta):
        """psi = M eta for a full-lattice field eta [V][4][3]."""
        eta = np.asarray(eta, dtype=np.complex128)
        psi = np.zeros_like(eta)
        rho = eta.copy()
        for _ in range(self.ncy):
            for colour in (0, 1):
                psi = psi + self.block_solve(rho, colour)
                rho = eta - self.op.apply(psi)
        return psi

    def apply_even(self, r_e):
        """(M (r_e, 0))_e for an even-site field."""
        full = np.zeros((self.geom.V, 4, 3), dtype=np.complex128)
        ev = self.op.even_sites()
        full[ev] = r_e
        return self.apply(full)[ev]
