"""Pins of the rational-approximation code (App. A.1, A.2) by the paper's
printed degree-10 example (sample input file, App. C, [Rational 0]):
 * the printed extremal points x_0 = r_a^2 and x_21 = r_b^2 (in q^2);
 * the optimal (minmax) error equioscillates: 1 - x_i^alpha rho(x_i) = +-delta with
   alternating sign at all 22 printed extremal points (Chebyshev alternation);
 * max |error| over the whole range equals the printed delta (eq. error);
 * the partial fractions of App. A.2 reproduce rho;
 * rho(Dhat^+ Dhat) phi = A (phi + sum_j sigma_j (Dhat^+ Dhat + mu_j^2)^-1 phi)
   with the shifted solves done by the oracle's MSCG (dense check on a small lattice).
"""
import os

import numpy as np

from oracle import ratapprox
from oracle.solvers import mscg
from tests.oracle_helpers import dense, make_op

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rational_deg10_pow_m1_4.txt")


def test_printed_record():
    r = ratapprox.load(GOLDEN)
    assert r.degree == 10 and r.alpha == 0.25 and len(r.x) == 22
    assert abs(r.x[0] - r.r_a ** 2) < 1e-15 * r.x[0]
    assert abs(r.x[-1] - r.r_b ** 2) < 1e-14 * r.x[-1]
    assert np.all(np.diff(r.nu) < 0) and np.all(np.diff(r.mu) < 0)


def test_equioscillation_at_printed_extrema():
    r = ratapprox.load(GOLDEN)
    e = r.rel_error(r.x)
    assert np.abs(np.abs(e) - r.delta).max() < 1e-9 * r.delta
    assert np.all(np.sign(e[1:]) == -np.sign(e[:-1]))


def test_uniform_error_is_delta():
    r = ratapprox.load(GOLDEN)
    q2 = np.geomspace(r.r_a ** 2, r.r_b ** 2, 200001)
    assert abs(np.abs(r.rel_error(q2)).max() - r.delta) < 1e-9 * r.delta


def test_partial_fractions_reproduce_rho():
    r = ratapprox.load(GOLDEN)
    q2 = np.geomspace(1e-6, 1e2, 1001)
    assert np.abs(r.rho_partial_fractions(q2) / r.rho(q2) - 1).max() < 1e-13


def test_rational_function_of_operator_via_mscg():
    r = ratapprox.load(GOLDEN)
    op, _, _ = make_op((4, 2, 2, 4), 0, (np.pi, 0, 0, 0), qhat=-2, kappa=0.13, seed=91)
    ne = len(op.even_sites())
    Dinv = op.Doo_inv()
    M = dense(lambda v: op.Dhat(v, Dinv), ne * 12, (ne, 4, 3))
    H = M.conj().T @ M
    w, Q = np.linalg.eigh(H)
    phi = np.random.default_rng(3).normal(size=(ne, 4, 3)) + 0j
    want = (Q @ (r.rho(w) * (Q.conj().T @ phi.reshape(-1)))).reshape(phi.shape)
    shifts = list(r.mu ** 2)
    xs, it = mscg(lambda v: (H @ v.reshape(-1)).reshape(v.shape), phi, shifts, 1e-12, 5000)
    assert it > 0
    got = r.A * (phi + sum(s * x for s, x in zip(r.sigma(), xs)))
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
