"""SAP preconditioner on the GPU against the oracle (oracle/sap.py), and SAP+FGCR solves.

Tolerance of the preconditioner application: FP32 arithmetic with FP32 block
sums in the minimal-residual steps (the map is nonlinear in its input through
alpha = <p, r>/<p, p>): 2e-5 norm-relative."""
import numpy as np
import pytest

from oracle.sap import SAP
from paper_1908_11673_gb300 import workload
from tests.gpu_helpers import relerr, setup

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,cstar,ncy,nmr", [((8, 8, 8, 8), 0, 1, 1), ((8, 8, 8, 8), 0, 5, 5),
                                              ((16, 8, 8, 8), 0, 1, 2), ((8, 4, 8, 8), 1, 2, 3),
                                              ((8, 4, 8, 8), 3, 5, 5)])
def test_sap_apply_parity(L, cstar, ncy, nmr):
    qxd, ctx, op, _, _ = setup(L, cstar, (np.pi, 0, 0, 0), qhat=4, kappa=0.13, seed=9100, stout=1)
    ctx.set_sap(ncy, nmr)
    eta = workload.spinor(op.geom.V, 9101).astype(np.complex64)
    out = np.empty_like(eta)
    ctx.sap_apply(0, eta, out)
    ref = SAP(op, bsize=4, ncy=ncy, nmr=nmr).apply(eta.astype(np.complex128))
    assert relerr(out.astype(np.complex128), ref) <= 2e-5
    ctx.close()


@pytest.mark.parametrize("inner", [1, 2])
def test_sap_fgcr_solves(inner):
    """16^4, smeared, qhat=-2, kappa=0.136377: the case where restarted GCR
    without a preconditioner stalls.  SAP+FGCR reaches 1e-10 in far fewer
    iterations than FGCR without it."""
    qxd, ctx, op, _, _ = setup((16, 16, 16, 16), 0, (np.pi, 0, 0, 0), qhat=-2, seed=4100, stout=5)
    eta = workload.spinor(op.geom.V, 41000)
    psi = np.empty_like(eta)
    plain = ctx.solve(0, eta, psi, kind=1, tol=1e-10, inner=inner, nkv=16)
    info = ctx.solve(0, eta, psi, kind=1, tol=1e-10, inner=inner, nkv=16, precond=2)
    assert info.status == 0 and info.true_relres <= 1e-10
    assert info.iters < plain.iters, (info.iters, plain.iters)
    sites = np.random.default_rng(0).choice(op.geom.V, 1000, replace=False)
    r = eta[sites] - op.apply(psi, sites)
    assert np.linalg.norm(r) / np.linalg.norm(eta[sites]) < 1e-9
    ctx.close()


@pytest.mark.parametrize("L", [(6, 8, 8, 8), (8, 8, 4, 8), (12, 8, 8, 8)])
def test_sap_rejects_unsupported_lattices(L):
    """Extents must hold an even number of 4^4 blocks."""
    qxd, ctx, op, _, _ = setup(L, 0, (np.pi, 0, 0, 0))
    eta = workload.spinor(op.geom.V, 1).astype(np.complex64)
    with pytest.raises(qxd.QxdError) as e:
        ctx.sap_apply(0, eta, np.empty_like(eta))
    assert e.value.code == 1
    ctx.close()
