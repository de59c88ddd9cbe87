"""Small helpers shared by the oracle pin tests (no method arithmetic)."""
import numpy as np

from oracle import DiracOperator, Flavour, GaugeField, Geometry
from paper_1908_11673_gb300 import workload


def make_op(L, cstar=0, theta=(np.pi, 0, 0, 0), qhat=-2, kappa=0.136377,
            su3csw=1.90952, u1csw=1.0, seed=11, invqel=6.0, free=False, sigma_h=0.3, sigma_a=0.2):
    g = Geometry(L, cstar, theta)
    if free:
        U, A = workload.unit_gauge_field(L)
    else:
        U, A = workload.gauge_field(L, seed, sigma_h=sigma_h, sigma_a=sigma_a, device="cpu")
    gf = GaugeField(g, U, A, invqel)
    return DiracOperator(gf, Flavour(qhat, kappa, su3csw, u1csw)), U, A


def dense(apply, n_in, shape_in):
    """Matrix of a linear map given as a function on arrays of shape shape_in."""
    cols = []
    for k in range(n_in):
        e = np.zeros(n_in, dtype=np.complex128)
        e[k] = 1.0
        cols.append(np.asarray(apply(e.reshape(shape_in))).reshape(-1))
    return np.stack(cols, axis=1)
