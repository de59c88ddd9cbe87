"""Open time boundary (Sec. 2.3 eq. dirac, term dD_b; definition of openQCD,
Luescher and Schaefer, Comput. Phys. Commun. 184 (2013) 519) on the GPU against
the oracle: D_w in every precision and Dhat, with and without C* in the spatial
directions, and solves checked by the oracle's residual.  Tolerances are those
of test_gpu_operator.py."""
import numpy as np
import pytest

from oracle.dirac import gamma5
from paper_1908_11673_gb300 import workload
from tests.gpu_helpers import relerr, setup

pytestmark = pytest.mark.gpu

BF16_U = 2.0 ** -9
TOL = {0: 1e-13, 1: 2e-6, 2: 2 * BF16_U, 3: 1e-12}
TOL_DHAT = {0: 1e-13, 1: 2e-6, 2: 3 * BF16_U}
NOPHASE = (0.0, 0.0, 0.0, 0.0)
GEOMS = [((6, 4, 4, 6), 0, -2, 1.37), ((4, 4, 6, 4), 1, 4, 0.9), ((6, 4, 6, 4), 3, -2, 1.0)]


@pytest.mark.parametrize("L,cstar,qhat,cF", GEOMS)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_open_Dw_parity(L, cstar, qhat, cF, prec):
    qxd, ctx, op, _, _ = setup(L, cstar, NOPHASE, qhat=qhat, seed=9000 + sum(L), tbc="open", cF=cF)
    psi = workload.spinor(op.geom.V, 9001)
    if prec in (1, 2):
        psi = psi.astype(np.complex64)
    out = np.empty_like(psi)
    ctx.apply_Dw(0, prec, psi, out)
    ref = op.apply(psi.astype(np.complex128))
    assert relerr(out.astype(np.complex128), ref) <= TOL[prec]
    ctx.close()


@pytest.mark.parametrize("L,cstar,qhat,cF", GEOMS)
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_open_Dhat_parity(L, cstar, qhat, cF, prec):
    qxd, ctx, op, _, _ = setup(L, cstar, NOPHASE, qhat=qhat, seed=9100 + sum(L), tbc="open", cF=cF)
    ne = op.geom.V // 2
    psi = workload.spinor(ne, 9101)
    if prec:
        psi = psi.astype(np.complex64)
    p = psi.astype(np.complex128)
    for dagger in (False, True):
        out = np.empty_like(psi)
        ctx.apply_Dhat_eo(0, prec, psi, out, dagger=dagger)
        ref = gamma5(op.Dhat(gamma5(p))) if dagger else op.Dhat(p)
        assert relerr(out.astype(np.complex128), ref) <= TOL_DHAT[prec]
    ctx.close()


@pytest.mark.parametrize("kind,inner,precond", [(0, 0, 0), (1, 1, 0), (1, 2, 0), (1, 1, 2)])
def test_open_solves(kind, inner, precond):
    """CGNE (FP64), FGCR with FP32 and BF16 inner solves, and SAP-preconditioned
    FGCR on an 8^4 lattice with an open time boundary (cF = 1.2), smeared links:
    the oracle's residual of the returned solution."""
    qxd, ctx, op, _, _ = setup((8, 8, 8, 8), 0, NOPHASE, qhat=-2, kappa=0.13, seed=9200, stout=3, tbc="open",
                               cF=1.2)
    eta = workload.spinor(op.geom.V, 9201)
    psi = np.empty_like(eta)
    info = ctx.solve(0, eta, psi, kind=kind, tol=1e-10, inner=inner, nkv=16, precond=precond)
    assert info.status == 0 and info.true_relres <= 1e-10, info.asdict()
    res = np.linalg.norm(eta - op.apply(psi)) / np.linalg.norm(eta)
    assert res <= 1.5e-10, res
    ctx.close()
