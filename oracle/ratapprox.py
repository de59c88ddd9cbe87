"""Rational approximation of (q^2)^-alpha and its partial fractions (App. A.1, A.2).

    rho(q^2) = A prod_j (q^2 + nu_j^2) / (q^2 + mu_j^2)                   (eq. ratfunc)
    delta    = max_{q in [r_a, r_b]} |1 - (q^2 + muhat^2)^alpha rho(q^2)|   (eq. error)
    P_{k,l}  = 1 + sum_{j=k..l} sigma_j / (Dhat^+ Dhat + mu_j^2)
    sigma_j  = (nu_j^2 - mu_j^2) prod_{m != j} (nu_m^2 - mu_j^2) / (mu_m^2 - mu_j^2)

The coefficients are inputs (the paper prints a degree-10 example in its sample
input file, App. C); `load` reads them from a text record.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU baseline, never by the library.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Rational:
    power: tuple
    degree: int
    r_a: float   # range in |Q| (the printed 'range' gives r_a, r_b)
    r_b: float
    muhat: float
    delta: float
    A: float
    nu: np.ndarray
    mu: np.ndarray
    x: np.ndarray  # extremal points of the error (in q^2)

    @property
    def alpha(self) -> float:
        return -self.power[0] / self.power[1]

    def rho(self, q2):
        q2 = np.asarray(q2, dtype=np.float64)
        out = np.full_like(q2, self.A)
        for n, m in zip(self.nu, self.mu):
            out = out * (q2 + n * n) / (q2 + m * m)
        return out

    def rel_error(self, q2):
        """1 - (q^2 + muhat^2)^alpha rho(q^2)."""
        q2 = np.asarray(q2, dtype=np.float64)
        return 1.0 - (q2 + self.muhat ** 2) ** self.alpha * self.rho(q2)

    def sigma(self, k=0, l=None):
        """Partial-fraction residues sigma_j for the factor P_{k,l} (0-based, inclusive)."""
        l = self.degree - 1 if l is None else l
        out = []
        for j in range(k, l + 1):
            s = self.nu[j] ** 2 - self.mu[j] ** 2
            for m in range(k, l + 1):
                if m != j:
                    s *= (self.nu[m] ** 2 - self.mu[j] ** 2) / (self.mu[m] ** 2 - self.mu[j] ** 2)
            out.append(s)
        return np.array(out)

    def rho_partial_fractions(self, q2):
        """A (1 + sum_j sigma_j / (q^2 + mu_j^2))."""
        q2 = np.asarray(q2, dtype=np.float64)
        s = np.ones_like(q2)
        for sj, mj in zip(self.sigma(), self.mu):
            s = s + sj / (q2 + mj * mj)
        return self.A * s


def load(path) -> Rational:
    vals = {}
    nu, mu, x = {}, {}, {}
    with open(path) as f:
        for line in f:
            line = line.split('#')[0].strip()
            if not line or line.startswith('['):
                continue
            key, *rest = line.split()
            if key.startswith('nu['):
                nu[int(key[3:-1])] = float(rest[0])
            elif key.startswith('mu['):
                mu[int(key[3:-1])] = float(rest[0])
            elif key.startswith('x['):
                x[int(key[2:-1])] = float(rest[0])
            else:
                vals[key] = rest
    n = int(vals['degree'][0])
    return Rational(power=(int(vals['power'][0]), int(vals['power'][1])), degree=n,
                    r_a=float(vals['range'][0]), r_b=float(vals['range'][1]),
                    muhat=float(vals['mu'][0]), delta=float(vals['delta'][0]),
                    A=float(vals['A'][0]),
                    nu=np.array([nu[i] for i in range(n)]),
                    mu=np.array([mu[i] for i in range(n)]),
                    x=np.array([x[i] for i in range(len(x))]))
