"""Solves on the GPU checked by the oracle: the returned psi must satisfy
|eta - D psi| / |eta| <= tol with D applied by the oracle (FP64)."""
import numpy as np
import pytest

from paper_1908_11673_gb300 import workload
from tests.gpu_helpers import setup

pytestmark = pytest.mark.gpu


def oracle_residual(op, eta, psi):
    return float(np.linalg.norm(eta - op.apply(psi)) / np.linalg.norm(eta))


@pytest.mark.parametrize("kind,inner", [(0, 0), (1, 1), (1, 0), (1, 2)])
def test_config1_solves(kind, inner):
    """8^4, antiperiodic time, qhat=-2, kappa=0.136377, csw=1.90952/1.0, one
    Gaussian source: CGNE (FP64) and FGCR with FP32 / FP64 / BF16 inner solves."""
    qxd, ctx, op, _, _ = setup((8, 8, 8, 8), 0, (np.pi, 0, 0, 0), qhat=-2, seed=1000)
    eta = workload.spinor(op.geom.V, 1001)
    psi = np.empty_like(eta)
    info = ctx.solve(0, eta, psi, kind=kind, tol=1e-10, inner=inner, nkv=16)
    assert info.status == 0
    assert info.true_relres <= 1e-10
    assert oracle_residual(op, eta, psi) <= 1.5e-10
    ctx.close()


@pytest.mark.parametrize("cstar", [1, 3])
def test_cstar_solves(cstar):
    qxd, ctx, op, _, _ = setup((4, 4, 6, 4), cstar, (np.pi, 0, 0, 0), qhat=4, kappa=0.13, seed=77, stout=2)
    eta = workload.spinor(op.geom.V, 78)
    for kind, inner in ((0, 0), (1, 1)):
        psi = np.empty_like(eta)
        info = ctx.solve(0, eta, psi, kind=kind, tol=1e-10, inner=inner)
        assert info.true_relres <= 1e-10
        assert oracle_residual(op, eta, psi) <= 1.5e-10
    ctx.close()


def test_solver_failures_are_reported():
    qxd, ctx, op, _, _ = setup((4, 4, 4, 4), 0, (np.pi, 0, 0, 0))
    eta = workload.spinor(op.geom.V, 3)
    psi = np.empty_like(eta)
    info = ctx.solve(0, eta, psi, kind=0, tol=1e-10, nmx=2, check=False)
    assert info.status == 2  # QXD_ENOCONV
    bad = eta.copy()
    bad[5, 1, 2] = np.nan
    with pytest.raises(qxd.QxdError) as e:
        ctx.solve(0, bad, psi, kind=1, tol=1e-10)
    assert e.value.code == 4  # QXD_ENAN
    with pytest.raises(qxd.QxdError) as e:
        ctx.apply_Dw(3, 0, eta, psi)  # flavour slot never set
    assert e.value.code == 7
    ctx.close()


def test_mixed_fgcr_residual_certified_in_fp64():
    """The mixed solver takes its outer residual with the FP64 data in double-float
    arithmetic; an FP64 residual of the returned solution agrees with its report."""
    qxd, ctx, op, _, _ = setup((8, 8, 8, 8), 0, (np.pi, 0, 0, 0), qhat=-2, seed=5600, stout=2)
    eta = workload.spinor(op.geom.V, 5601)
    psi = np.empty_like(eta)
    info = ctx.solve(0, eta, psi, kind=1, tol=1e-10, inner=1, nkv=16)
    assert info.status == 0 and info.true_relres <= 1e-10
    dpsi = np.empty_like(psi)
    ctx.apply_Dw(0, 0, psi, dpsi)
    rel64 = np.linalg.norm(eta - dpsi) / np.linalg.norm(eta)
    assert rel64 <= 1e-10
    assert abs(rel64 - info.true_relres) <= 1e-3 * rel64
    ctx.close()
