"""Rational factors of the quark determinant on lattice fields: the pseudofermion
action of a factor P_{k,l} (App. A.2, eqs. Pfactor, Spf, Spf2), the stochastic
exponents of the reweighting factors W_rat and W_rtm (App. A.3), and the
small-determinant action S_sdet (Sec. 2.3, even-odd preconditioning).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU baseline, never by the library.  Plain FP64 NumPy.

Conventions.  Q2 = Dhat^+ Dhat on even fields.  Factor indices k, l are
0-based and inclusive (the paper's j = k+1 .. l+1).  Every shifted inverse
(Q2 + s)^-1 is taken from the multi-shift CG of oracle.solvers, each shift to a
relative residual `tol`.

Readings where the paper is silent or garbled:
  * S_sdet.  The printed form "-sum_f alpha_f tr log(1 + D_f,oo)" does not match
    the normalisation of D used everywhere else (D_oo = 1/(2 kappa) + clover).
    The factorisation det D = det D_oo det Dhat fixes the term as
    S_sdet = -sum_f alpha_f sum_{x odd} log det D_oo(x), D_oo(x) the 12x12
    site-diagonal block; `sdet` returns sum_{x odd} log |det D_oo(x)| (the
    caller applies -alpha_f).  A normalisation in which the diagonal mass term
    is 1 differs by the field-independent constant 12 V/2 log(2 kappa).
  * W_rtm.  The exponent (eta, [Ptilde_{k,l} - 1] eta) is evaluated in the
    combined form the paper recommends for stability, rewritten with the
    solutions x_j = (Q2 + nu_j^2)^-1 eta and y_j = (Q2 + mutilde_j^2)^-1 eta as
    (sigma_j + sigmatilde_j) (eta, x_j) + sigmatilde_j (nu_j^2 - mutilde_j^2) (x_j, y_j)
    (the numerator (s+st) Q2 + s mt^2 + st nu^2 equals
    (s+st)(Q2 + mt^2) + st (nu^2 - mt^2)).
"""
from __future__ import annotations

import math

import numpy as np

from .dirac import DiracOperator
from .ratapprox import Rational
from .solvers import dhat_dagger, mscg


class NormalOperator:
    """Q2 = Dhat^+ Dhat on even-site fields [V/2][4][3]."""

    def __init__(self, op: DiracOperator):
        self.op = op
        self.Dinv = op.Doo_inv()

    def __call__(self, v):
        return dhat_dagger(self.op, self.op.Dhat(v, self.Dinv), self.Dinv)


def _shifted_inverses(Q2, b, shifts, tol, nmx):
    xs, it = mscg(Q2, b, list(shifts), tol, nmx)
    if it < 0:
        raise RuntimeError("multi-shift CG did not converge")
    return xs


def factor_apply(Q2, rat: Rational, k, l, phi, tol=1e-12, nmx=20000):
    """P_{k,l} phi = phi + sum_{j=k..l} sigma_j (Q2 + mu_j^2)^-1 phi (partial fractions of eq. Pfactor)."""
    sig = rat.sigma(k, l)
    xs = _shifted_inverses(Q2, phi, [rat.mu[j] ** 2 for j in range(k, l + 1)], tol, nmx)
    out = phi.copy()
    for s, x in zip(sig, xs):
        out = out + s * x
    return out


def pf_action(Q2, rat: Rational, k, l, phi, tol=1e-12, nmx=20000):
    """S_pf,k,l = (phi, phi) + sum_j sigma_j (phi, (Q2 + mu_j^2)^-1 phi)  (eq. Spf2)."""
    sig = rat.sigma(k, l)
    xs = _shifted_inverses(Q2, phi, [rat.mu[j] ** 2 for j in range(k, l + 1)], tol, nmx)
    S = np.vdot(phi, phi).real
    for s, x in zip(sig, xs):
        S += s * np.vdot(phi, x).real
    return float(S)


def rat_apply(Q2, rat: Rational, phi, tol=1e-12, nmx=20000):
    """R phi = A P_{0,n-1} phi."""
    return rat.A * factor_apply(Q2, rat, 0, rat.degree - 1, phi, tol, nmx)


def c_vn(v, n):
    """Taylor coefficient of (1 + Z)^(-1/v) = 1 + sum_n c_{v,n} Z^n (App. A.3)."""
    c = 1.0
    for i in range(n):
        c *= (1.0 / v + i)
    return (-1) ** n * c / math.factorial(n)


def wrat_terms(Q2, rat: Rational, u, v, nterms, eta, tol=1e-12, nmx=20000):
    """(eta, Z^n eta) for n = 1..nterms, Z = Q2^u R^v - 1 (eq. Wrat2)."""
    terms = []
    w = eta.copy()
    for _ in range(nterms):
        t = w
        for _ in range(v):
            t = rat_apply(Q2, rat, t, tol, nmx)
        for _ in range(u):
            t = Q2(t)
        w = t - w
        terms.append(float(np.vdot(eta, w).real))
    return terms


def wrat_exponent(terms, v):
    """(eta, [(1 + Z)^(-1/v) - 1] eta) from the series terms (eq. Wrat3)."""
    return float(sum(c_vn(v, n + 1) * t for n, t in enumerate(terms)))


def rtm_sigma(r_mu: Rational, r_t: Rational, k, l):
    """Residues (sigma_j, sigmatilde_j), j = k..l, of Ptilde_{k,l} - 1 at the poles
    q2 = -nu_j^2 and q2 = -mutilde_j^2, where
    Ptilde_{k,l}(q2) = prod_j (q2 + mu_j^2)(q2 + nutilde_j^2) / ((q2 + nu_j^2)(q2 + mutilde_j^2))."""
    js = range(k, l + 1)
    nu2 = {j: r_mu.nu[j] ** 2 for j in js}
    mu2 = {j: r_mu.mu[j] ** 2 for j in js}
    nt2 = {j: r_t.nu[j] ** 2 for j in js}
    mt2 = {j: r_t.mu[j] ** 2 for j in js}
    sig, sigt = [], []
    for j in js:
        # residue at q2 = -nu_j^2: drop the vanishing factor (q2 + nu_j^2)
        p = -nu2[j]
        s = (mu2[j] + p) * (nt2[j] + p) / (mt2[j] + p)
        for m in js:
            if m != j:
                s *= (mu2[m] + p) * (nt2[m] + p) / ((nu2[m] + p) * (mt2[m] + p))
        sig.append(s)
        # residue at q2 = -mutilde_j^2
        p = -mt2[j]
        s = (mu2[j] + p) * (nt2[j] + p) / (nu2[j] + p)
        for m in js:
            if m != j:
                s *= (mu2[m] + p) * (nt2[m] + p) / ((nu2[m] + p) * (mt2[m] + p))
        sigt.append(s)
    return np.array(sig), np.array(sigt)


def wrtm_exponent(Q2, r_mu: Rational, r_t: Rational, k, l, eta, tol=1e-12, nmx=20000):
    """(eta, [Ptilde_{k,l} - 1] eta), the exponent of the stochastic estimate of
    det Ptilde_{k,l}^-1 (App. A.3, W_rtm)."""
    sig, sigt = rtm_sigma(r_mu, r_t, k, l)
    js = list(range(k, l + 1))
    shifts = [r_mu.nu[j] ** 2 for j in js] + [r_t.mu[j] ** 2 for j in js]
    xs = _shifted_inverses(Q2, eta, shifts, tol, nmx)
    n = len(js)
    e = 0.0
    for i, j in enumerate(js):
        x, y = xs[i], xs[n + i]
        e += (sig[i] + sigt[i]) * np.vdot(eta, x).real
        e += sigt[i] * (r_mu.nu[j] ** 2 - r_t.mu[j] ** 2) * np.vdot(x, y).real
    return float(e)


def shifted(rat: Rational, muhat: float) -> Rational:
    """rho(q2 + muhat^2) written as a rational function of q2: nu_j -> sqrt(nu_j^2 + muhat^2),
    mu_j -> sqrt(mu_j^2 + muhat^2).  If rho approximates (q2)^-alpha on [r_a^2, r_b^2], the
    result approximates (q2 + muhat^2)^-alpha with the same relative error on the shifted range."""
    return Rational(power=rat.power, degree=rat.degree, r_a=rat.r_a, r_b=rat.r_b, muhat=muhat,
                    delta=rat.delta, A=rat.A, nu=np.sqrt(rat.nu ** 2 + muhat ** 2),
                    mu=np.sqrt(rat.mu ** 2 + muhat ** 2), x=rat.x)


def sdet(op: DiracOperator):
    """sum over odd sites of log |det D_oo(x)| (12x12 site-diagonal block), and the number
    of odd sites whose determinant is negative."""
    odd = op.odd_sites()
    sign, logdet = np.linalg.slogdet(op.diag_term(odd))
    return float(np.sum(logdet)), int(np.sum(sign.real < 0))
