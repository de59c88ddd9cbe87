"""Textbook Krylov solvers used by openQ*D (Sec. 4.4): CG on the normal
equations (CGNE), multi-shift CG (MSCG, for the shifted systems of the rational
approximation, App. A.2) and flexible restarted GCR.  Plain NumPy, FP64.
Vectors are complex arrays of any shape; inner products are <a,b> = sum conj(a) b.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU baseline, never by the library.
"""
from __future__ import annotations

import numpy as np

from .dirac import DiracOperator, gamma5


def dot(a, b):
    return np.vdot(a, b)


def norm(a):
    return float(np.sqrt(np.vdot(a, a).real))


def cg(apply_A, b, tol, nmx, x0=None):
    """Conjugate gradient for a Hermitian positive-definite A; stops when the
    recursive residual satisfies |r| <= tol |b|.  Returns (x, iterations)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = dot(r, r).real
    bnorm = norm(b)
    for k in range(1, nmx + 1):
        Ap = apply_A(p)
        alpha = rr / dot(p, Ap).real
        x += alpha * p
        r -= alpha * Ap
        rr_new = dot(r, r).real
        if np.sqrt(rr_new) <= tol * bnorm:
            return x, k
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, -1


def dhat_dagger(op: DiracOperator, psi_e, Dinv):
    """Dhat^+ = gamma5 Dhat gamma5 (gamma5-hermiticity of D carries over to Dhat
    because the site-diagonal blocks commute with gamma5)."""
    return gamma5(op.Dhat(gamma5(psi_e), Dinv))


def cgnr(apply_D, apply_Ddag, b, tol, nmx, x0=None, bnorm=None):
    """CG on the normal equations D^+ D x = D^+ b, tracking the residual
    s = b - D x of the original system and stopping when |s| <= tol * bnorm
    (bnorm defaults to |b|).  Returns (x, iterations, |s|)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    s = b - apply_D(x) if x0 is not None else b.copy()
    bnorm = norm(b) if bnorm is None else bnorm
    z = apply_Ddag(s)
    p = z.copy()
    zz = dot(z, z).real
    for k in range(1, nmx + 1):
        w = apply_D(p)
        alpha = zz / dot(w, w).real
        x += alpha * p
        s -= alpha * w
        if norm(s) <= tol * bnorm:
            return x, k, norm(s)
        z = apply_Ddag(s)
        zz_new = dot(z, z).real
        p = z + (zz_new / zz) * p
        zz = zz_new
    return x, -nmx, norm(s)


def cgne_solve(op: DiracOperator, eta, tol=1e-10, nmx=10000):
    """Solve D psi = eta on the full lattice through the even-odd system:
        eta_hat_e = eta_e - D_eo D_oo^-1 eta_o,
        CG on Dhat^+ Dhat y = Dhat^+ eta_hat_e (stopping on |eta_hat_e - Dhat y|),
        psi_e = y,  psi_o = D_oo^-1 (eta_o - D_oe psi_e).
    The CG is restarted from the current y until the full-lattice residual
    |eta - D psi| / |eta| <= tol.  Returns (psi, CG iterations, true relative residual)."""
    geom = op.geom
    ev, od = op.even_sites(), op.odd_sites()
    Dinv = op.Doo_inv()
    mul = lambda M, v: np.einsum('nab,nb->na', M, v.reshape(-1, 12)).reshape(-1, 4, 3)
    eta = np.asarray(eta, dtype=np.complex128).reshape(geom.V, 4, 3)
    eta_hat = eta[ev] - op.Deo(mul(Dinv, eta[od]))
    Dh = lambda v: op.Dhat(v, Dinv)
    Dhd = lambda v: dhat_dagger(op, v, Dinv)
    enorm = norm(eta)
    y = np.zeros_like(eta_hat)
    psi = np.zeros_like(eta)
    iters, res = 0, np.inf
    for _ in range(20):
        y, k, _ = cgnr(Dh, Dhd, eta_hat, tol * 0.5, nmx - iters, x0=y, bnorm=enorm)
        iters += abs(k)
        psi[ev] = y
        psi[od] = mul(Dinv, eta[od] - op.Doe(y))
        res = norm(eta - op.apply(psi)) / enorm
        if res <= tol or k < 0:
            break
    return psi, (iters if res <= tol else -iters), res


def mscg(apply_A, b, shifts, tol, nmx):
    """Multi-shift CG: solves (A + s_j) x_j = b for all shifts s_j >= 0 in one
    Krylov space (Jegerlehner's recursion for the shifted coefficients).
    Each shift stops when its residual |r_j| <= tol |b|.
    Returns (list of x_j, iterations)."""
    ns = len(shifts)
    x = [np.zeros_like(b) for _ in range(ns)]
    p = [b.copy() for _ in range(ns)]
    r = b.copy()
    rr = dot(r, r).real
    bn = norm(b)
    zeta_prev = np.ones(ns)
    zeta = np.ones(ns)
    alpha_prev, beta_prev = 1.0, 0.0
    active = np.ones(ns, dtype=bool)
    # base system: the smallest shift s0 (the others are shifted by s_j - s0)
    s0 = min(shifts)
    ds = np.array([s - s0 for s in shifts])
    pb = r.copy()
    for k in range(1, nmx + 1):
        Ap = apply_A(pb) + s0 * pb
        alpha = rr / dot(pb, Ap).real
        zeta_next = np.empty(ns)
        for j in range(ns):
            if not active[j]:
                continue
            denom = (alpha * beta_prev * (zeta_prev[j] - zeta[j])
                     + zeta_prev[j] * alpha_prev * (1.0 + ds[j] * alpha))
            zeta_next[j] = zeta[j] * zeta_prev[j] * alpha_prev / denom
            alpha_j = alpha * zeta_next[j] / zeta[j]
            x[j] += alpha_j * p[j]
        r_new = r - alpha * Ap
        rr_new = dot(r_new, r_new).real
        beta = rr_new / rr
        for j in range(ns):
            if not active[j]:
                continue
            beta_j = beta * (zeta_next[j] / zeta[j]) ** 2
            p[j] = zeta_next[j] * r_new + beta_j * p[j]
            if abs(zeta_next[j]) * np.sqrt(rr_new) <= tol * bn:
                active[j] = False
            zeta_prev[j], zeta[j] = zeta[j], zeta_next[j]
        pb = r_new + beta * pb
        r, rr = r_new, rr_new
        alpha_prev, beta_prev = alpha, beta
        if not active.any():
            return x, k
    return x, -nmx


def gcr(apply_A, b, tol, nkv, nmx, precond=None, x0=None):
    """Flexible GCR restarted every nkv steps (right preconditioner M, which may
    change between steps).  Stops when |b - A x| <= tol |b| (residual recomputed
    at every restart).  Returns (x, iterations)."""
    M = precond if precond is not None else (lambda v: v)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bn = norm(b)
    r = b - apply_A(x)
    it = 0
    while it < nmx:
        Z, W, WW = [], [], []
        for _ in range(nkv):
            z = M(r)
            w = apply_A(z)
            for zj, wj, wwj in zip(Z, W, WW):
                beta = dot(wj, w) / wwj
                w = w - beta * wj
                z = z - beta * zj
            ww = dot(w, w).real
            a = dot(w, r) / ww
            x = x + a * z
            r = r - a * w
            Z.append(z); W.append(w); WW.append(ww)
            it += 1
            if norm(r) <= tol * bn or it >= nmx:
                break
        r = b - apply_A(x)
        if norm(r) <= tol * bn:
            return x, it
    return x, -it
