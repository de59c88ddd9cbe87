"""Learned preconditioner: a gauge-covariant network of parallel-transport
layers (not part of the paper; the network shape is the one this project
trains).  Plain FP64 NumPy.

Layer l maps c_in channels of spinor fields to c_out channels:

    b_c(x) = sum_{c'} sum_{d=0..8} W[c][c'][d] (T_d a_{c'})(x),

    T_0 a(x)      = a(x)
    T_{1+mu} a(x) = V(x,mu) a(x+mu)            (forward transport)
    T_{5+mu} a(x) = V(x-mu,mu)^+ a(x-mu)       (backward transport)

with V = U z^qhat and the same boundary conditions (phases, C* shifts) as the
Dirac operator, and W[c][c'][d] a complex 4x4 matrix acting on the spin index.
The transports commute with gauge transformations, so the network is gauge
covariant; it has no nonlinearity, so it is a linear map M.  Used as a
preconditioner of the even-odd operator Dhat, M acts on an even-site field r
embedded in the full lattice (zero on odd sites) and its output is restricted
to the even sites: Dhat^-1 = (D^-1)_ee, so M is trained to approximate D^-1.

Loss over pairs (r_i, e_i) with Dhat e_i = r_i, in one of two norms:
    L = sum_i |(M r_i)_e - e_i|^2 / |e_i|^2                  ("error": Euclidean norm)
    L = sum_i |r_i - Dhat (M r_i)_e|^2 / |r_i|^2            ("residual")
The second is the error of M r_i measured in the norm |Dhat .|, since
Dhat e_i = r_i; it weighs each mode by |Dhat|, as the residual of a right-
preconditioned Krylov solver does, and is 1 for M = 0.
Gradient (Wirtinger): G = dL/dW^* = sum_x delta_c(x) (T_d a_{c'}(x))^+ per
layer, with delta = (out - e)/|e|^2 at the output and delta' = layer^+ delta
propagated backwards (layer^+ uses W^+ and T_d^+ = T_{opposite d}).
The gradient with respect to the real and imaginary parts of W is 2 Re G, 2 Im G.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU baseline, never by the library.
"""
from __future__ import annotations

import numpy as np

from .dirac import DiracOperator

NDIR = 9


def opposite(d: int) -> int:
    if d == 0:
        return 0
    return d + 4 if d <= 4 else d - 4


def layer_shapes(nlayers: int, nch: int):
    return [(1 if l == 0 else nch, 1 if l == nlayers - 1 else nch) for l in range(nlayers)]


def identity_weights(nlayers: int, nch: int):
    """W[c][c][0] = 1 for c < min(c_in, c_out): the network is the identity."""
    Ws = []
    for cin, cout in layer_shapes(nlayers, nch):
        W = np.zeros((cout, cin, NDIR, 4, 4), dtype=np.complex128)
        for c in range(min(cin, cout)):
            W[c, c, 0] = np.eye(4)
        Ws.append(W)
    return Ws


class Transport:
    """The nine transports T_d of a Dirac operator's links and boundaries."""

    def __init__(self, op: DiracOperator):
        self.op = op
        self.geom = op.geom
        s = self.geom.sites()
        self.nb = {}
        for mu in range(4):
            f, ph_f = self.geom.neighbour(s, mu, +1)
            b, ph_b = self.geom.neighbour(s, mu, -1)
            Vf = op.V(s, mu)
            Vb = np.conj(np.swapaxes(op.V(b, mu), -1, -2))
            self.nb[1 + mu] = (f, ph_f, Vf)
            self.nb[5 + mu] = (b, ph_b, Vb)

    def apply(self, d: int, a):
        """T_d a for a field a [V][4][3]."""
        if d == 0:
            return a.copy()
        idx, ph, M = self.nb[d]
        # (M a(y))_{s,i} = sum_j M_ij a(y)_{s,j}
        return ph[:, None, None] * (a[idx] @ np.swapaxes(M, -1, -2))


def layer(T: Transport, W, a):
    """b[c] = sum_{c',d} W[c][c'][d] T_d a[c']  (a: [c_in][V][4][3])."""
    cout, cin = W.shape[0], W.shape[1]
    V = a.shape[1]
    b = np.zeros((cout, V, 4, 3), dtype=np.complex128)
    for cp in range(cin):
        for d in range(NDIR):
            s = T.apply(d, a[cp])
            for c in range(cout):
                b[c] += np.einsum('st,vtj->vsj', W[c, cp, d], s)
    return b


def layer_adjoint(T: Transport, W, g):
    """a[c'] = sum_{c,d} W[c][c'][d]^+ T_d^+ g[c], with T_d^+ = T_{opposite(d)}."""
    cout, cin = W.shape[0], W.shape[1]
    V = g.shape[1]
    a = np.zeros((cin, V, 4, 3), dtype=np.complex128)
    for c in range(cout):
        for d in range(NDIR):
            for cp in range(cin):
                t = np.einsum('ts,vtj->vsj', np.conj(W[c, cp, d]), g[c])
                a[cp] += T.apply(opposite(d), t)
    return a


def embed_even(op: DiracOperator, r_e):
    full = np.zeros((op.geom.V, 4, 3), dtype=np.complex128)
    full[op.even_sites()] = r_e
    return full


def network(T: Transport, Ws, r_e, keep=False):
    """(M r)_e for an even-site field r_e [V/2][4][3]."""
    op = T.op
    a = embed_even(op, r_e)[None]
    acts = [a]
    for W in Ws:
        a = layer(T, W, a)
        acts.append(a)
    out = a[0][op.even_sites()]
    return (out, acts) if keep else out


def _dhat_pair(op):
    """Dhat and Dhat^+ = gamma5 Dhat gamma5 on even-site fields."""
    from .dirac import gamma5
    Dinv = op.Doo_inv()
    return (lambda v: op.Dhat(v, Dinv)), (lambda v: gamma5(op.Dhat(gamma5(v), Dinv)))


def loss(T: Transport, Ws, pairs, norm="error"):
    tot = 0.0
    if norm == "residual":
        D, _ = _dhat_pair(T.op)
    for r, e in pairs:
        out = network(T, Ws, r)
        if norm == "residual":
            res = r - D(out)
            tot += float(np.vdot(res, res).real / np.vdot(r, r).real)
        else:
            tot += float(np.vdot(out - e, out - e).real / np.vdot(e, e).real)
    return tot


def loss_and_grad(T: Transport, Ws, pairs, norm="error"):
    """L and G_l = dL/dW_l^* (complex arrays shaped like W_l).  The output
    adjoint is (out - e)/|e|^2 for the Euclidean error and
    Dhat^+ (Dhat out - r)/|r|^2 for the residual norm."""
    op = T.op
    ev = op.even_sites()
    G = [np.zeros_like(W) for W in Ws]
    tot = 0.0
    if norm == "residual":
        D, Ddag = _dhat_pair(op)
    for r, e in pairs:
        out, acts = network(T, Ws, r, keep=True)
        delta = np.zeros((1, op.geom.V, 4, 3), dtype=np.complex128)
        if norm == "residual":
            rr = float(np.vdot(r, r).real)
            res = D(out) - r
            tot += float(np.vdot(res, res).real) / rr
            delta[0][ev] = Ddag(res) / rr
        else:
            ee = float(np.vdot(e, e).real)
            res = out - e
            tot += float(np.vdot(res, res).real) / ee
            delta[0][ev] = res / ee
        for l in range(len(Ws) - 1, -1, -1):
            a = acts[l]
            W = Ws[l]
            for cp in range(W.shape[1]):
                for d in range(NDIR):
                    s = T.apply(d, a[cp])
                    for c in range(W.shape[0]):
                        # sum_x sum_colour delta_c(x)[s][i] conj(s(x)[t][i])
                        G[l][c, cp, d] += np.einsum('vsi,vti->st', delta[c], np.conj(s))
            if l > 0:
                delta = layer_adjoint(T, W, delta)
    return tot, G
