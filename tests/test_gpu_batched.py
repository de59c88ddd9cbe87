"""Batched (multi-right-hand-side) mixed-precision solves, checked by the oracle."""
import numpy as np
import pytest

from paper_1908_11673_gb300 import workload
from tests.gpu_helpers import relerr, setup

pytestmark = pytest.mark.gpu


def oracle_residuals(op, eta, psi, sites=None):
    out = []
    for e, p in zip(eta, psi):
        if sites is None:
            out.append(float(np.linalg.norm(e - op.apply(p)) / np.linalg.norm(e)))
        else:
            out.append(float(np.linalg.norm(e[sites] - op.apply(p, sites)) / np.linalg.norm(e[sites])))
    return out


@pytest.mark.parametrize("inner", [1, 2])
def test_batched_fgcr_four_rhs(inner):
    qxd, ctx, op, _, _ = setup((4, 6, 4, 4), 3, (np.pi, 0, 0, 0), qhat=4, kappa=0.13, seed=8100, stout=2)
    eta = workload.spinor(op.geom.V, 8101, nrhs=4)
    psi = np.empty_like(eta)
    info = ctx.solve(0, eta, psi, kind=1, tol=1e-10, inner=inner, nkv=8, nrhs=4)
    assert info.status == 0 and info.true_relres <= 1e-10
    assert max(oracle_residuals(op, eta, psi)) <= 1.5e-10
    # each right-hand side also solved alone: same solutions to the solver tolerance
    for r in range(4):
        one = np.empty_like(eta[r])
        ctx.solve(0, eta[r], one, kind=1, tol=1e-10, inner=inner, nkv=8)
        assert relerr(psi[r], one) < 1e-8
    ctx.close()


def test_config5_48c96_two_flavours_bf16_batched():
    """48^3 x 96 with C* in the three spatial directions (simulated 96x96x48x48,
    V = 21,233,664), smeared links, u1csw = su3csw = 1.90952, both flavours
    (qhat=-2, kappa=0.136377; qhat=4, kappa=0.137312) in turn, 4 right-hand sides
    in one batch, BF16 spinor storage in the inner solves, FP64 outer to 1e-10.
    The oracle checks the residual at 800 sampled sites per right-hand side."""
    import torch
    from oracle import DiracOperator, Flavour, GaugeField, Geometry
    from paper_1908_11673_gb300 import build, qxd
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    L = (96, 48, 48, 48)
    U, A = workload.gauge_field(L, 5000, stout_steps=5, device="cuda")
    torch.cuda.empty_cache()
    geom = Geometry(L, 3, (np.pi, 0, 0, 0))
    gauge = GaugeField(geom, U, A, 6.0)
    ctx = qxd.Context(L, 3, (np.pi, 0, 0, 0))
    ctx.set_links(U, A, 6.0)
    assert ctx.V == 21233664
    sites = np.random.default_rng(5).choice(ctx.V, 800, replace=False)
    import time
    t0 = time.time()
    for fl, (qhat, kappa) in enumerate([(4, 0.137312), (-2, 0.136377)]):
        ctx.set_clover(0, qhat, kappa, 1.90952, 1.90952)
        eta = torch.from_numpy(workload.spinor(ctx.V, 5001 + fl, nrhs=4)).cuda()
        psi = torch.empty_like(eta)
        info = ctx.solve(0, eta, psi, kind=1, tol=1e-10, inner=2, nkv=8, nrhs=4)
        print(f"config5 flavour qhat={qhat}: {info.asdict()} at {time.time() - t0:.1f} s", flush=True)
        assert info.status == 0 and info.true_relres <= 1e-10, info.asdict()
        op = DiracOperator(gauge, Flavour(qhat, kappa, 1.90952, 1.90952))
        res = oracle_residuals(op, eta.cpu().numpy(), psi.cpu().numpy(), sites)
        assert max(res) < 1e-9, res
        del eta, psi
    ctx.close()
