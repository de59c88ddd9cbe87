"""Batched (multi-right-hand-side) mixed-precision solves, checked by the oracle."""
import numpy as np
import pytest

from paper_1908_11673_gb300 import workload
from tests.gpu_helpers import relerr, setup

pytestmark = pytest.mark.gpu

# bfloat16 storage of input and output spinors: 2u, u = 2^-9 (derivation in
# test_gpu_operator.py)
BF16_TOL = 2 * 2.0 ** -9


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
    V = 21,233,664), u1csw = su3csw = 1.90952, both flavours (qhat=-2,
    kappa=0.136377; qhat=4, kappa=0.137312), 5 stout steps on the SU(3) and on
    the U(1) links (the configuration's "stout-smeared links" read as the
    combined links U z).
    Unsmeared photon angles first: the small-determinant action counts the odd
    sites whose 12x12 site-diagonal block has a negative determinant for qhat = 4
    (an eigenvalue has crossed zero, so others sit near zero and Dhat is nearly
    singular there); printed, it is the reason the U(1) links are smeared.
    Then, on the smeared field, for both flavours: FP64 and BF16-storage D_w on 4
    right-hand sides in one launch against the oracle at 400 sampled sites, and
    the batched solve of the 4 right-hand sides with BF16 storage in the inner
    solves, FP64 outer to 1e-10, oracle residual at 800 sampled sites."""
    import time

    import torch
    from oracle import DiracOperator, Flavour, GaugeField, Geometry
    from paper_1908_11673_gb300 import build, qxd
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    L = (96, 48, 48, 48)
    t0 = time.time()
    U, A0 = workload.gauge_field(L, 5000, stout_steps=5, device="cuda")
    torch.cuda.empty_cache()
    ctx = qxd.Context(L, 3, (np.pi, 0, 0, 0))
    try:
        ctx.set_links(U, A0, 6.0)
        assert ctx.V == 21233664
        ctx.set_clover(0, 4, 0.137312, 1.90952, 1.90952)
        ld0, nneg0 = ctx.sdet(0)
        A = workload.u1_stout(A0, L, 5, 0.1, device="cuda")
        del A0
        ctx.set_links(U, A, 6.0)
        ctx.set_clover(0, 4, 0.137312, 1.90952, 1.90952)
        ld1, nneg1 = ctx.sdet(0)
        print(f"config5 qhat=4 odd sites with det D_oo < 0: unsmeared photon field {nneg0}, smeared {nneg1}; "
              f"sum log|det D_oo| {ld0:.6e} / {ld1:.6e}", flush=True)
        geom = Geometry(L, 3, (np.pi, 0, 0, 0))
        gauge = GaugeField(geom, U, A, 6.0)
        rng = np.random.default_rng(5)
        for qhat, kappa in [(4, 0.137312), (-2, 0.136377)]:
            ctx.set_clover(0, qhat, kappa, 1.90952, 1.90952)
            op = DiracOperator(gauge, Flavour(qhat, kappa, 1.90952, 1.90952))
            sites = rng.choice(ctx.V, 400, replace=False)
            eta = torch.from_numpy(workload.spinor(ctx.V, 5001, nrhs=4)).cuda()
            out = torch.empty_like(eta)
            ctx.apply_Dw(0, 0, eta, out, nrhs=4)
            for r in range(4):
                ref = op.apply(eta[r].cpu().numpy(), sites)
                assert relerr(out[r].cpu().numpy()[sites], ref) <= 1e-13
            e32 = eta.to(torch.complex64)
            o32 = torch.empty_like(e32)
            ctx.apply_Dw(0, 2, e32, o32, nrhs=4)
            for r in range(4):
                ref = op.apply(e32[r].cpu().numpy().astype(np.complex128), sites)
                assert relerr(o32[r].cpu().numpy()[sites].astype(np.complex128), ref) <= BF16_TOL
            del out, e32, o32
            psi = torch.empty_like(eta)
            t1 = time.time()
            info = ctx.solve(0, eta, psi, kind=1, tol=1e-10, inner=2, nkv=8, nrhs=4)
            torch.cuda.synchronize()
            print(f"config5 qhat={qhat}: {info.asdict()} solve {time.time() - t1:.1f} s at {time.time() - t0:.1f} s",
                  flush=True)
            assert info.status == 0 and info.true_relres <= 1e-10, info.asdict()
            sites = rng.choice(ctx.V, 800, replace=False)
            res = oracle_residuals(op, eta.cpu().numpy(), psi.cpu().numpy(), sites)
            assert max(res) < 1e-9, res
            del psi, eta
    finally:
        ctx.close()  # also when an assertion fails: the context holds most of the device memory
