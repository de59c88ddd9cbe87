"""Shared set-up of the GPU parity tests: the same seeded input bytes go to the
CUDA library and to the oracle."""
import numpy as np
import pytest

from oracle import DiracOperator, Flavour, GaugeField, Geometry
from paper_1908_11673_gb300 import workload

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_11673_gb300 import build, qxd
    build.build()
    return qxd


def setup(L, cstar, theta, qhat=-2, kappa=0.136377, su3csw=1.90952, u1csw=1.0, seed=1000, stout=0,
          invqel=6.0, device="cpu", tbc="periodic", cF=1.0):
    """Library context and oracle operator on the same seeded field; tbc "open"
    gives both an open time boundary with improvement coefficient cF."""
    qxd = need_gpu()
    U, A = workload.gauge_field(L, seed, stout_steps=stout, device=device)
    geom = Geometry(L, cstar, theta, tbc=tbc, cF=cF)
    op = DiracOperator(GaugeField(geom, U, A, invqel), Flavour(qhat, kappa, su3csw, u1csw))
    ctx = qxd.Context(L, cstar, theta, tbc=qxd.TBC_OPEN if tbc == "open" else qxd.TBC_PERIODIC, cF=cF)
    ctx.set_links(U, A, invqel)
    ctx.set_clover(0, qhat, kappa, su3csw, u1csw)
    return qxd, ctx, op, U, A


def relerr(a, b):
    return float(np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1)))
