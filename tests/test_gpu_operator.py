"""GPU parity of the operator applications against the FP64 oracle.

Tolerances (norm-relative over the whole output):
  FP64              1e-13 (operator parity bar);
  FP32              2e-6: inputs, links and site-diagonal terms are rounded to
                    binary32 (2^-24 relative each) and each output component sums
                    ~10^2 products of O(1) terms; observed errors are a few 1e-7;
  BF16 spinors      2u = 2^-8 (3.9e-3) for D_w, 3u for Dhat, u = 2^-9 the unit
                    roundoff of bfloat16 (8-bit significand, round to nearest).
                    The kernel rounds the input spinor (each component to within
                    u relative) and its output to bfloat16 and computes in FP32
                    (1e-6 relative, negligible).  The error is D delta_in + delta_out
                    with |delta_out| <= u |D psi| and |delta_in| <= u |psi|; for the
                    Gaussian inputs of these tests delta_in is a random vector like
                    psi, so |D delta_in| / |D psi| ~ |delta_in| / |psi| <= u, and the
                    norm-relative error stays below 2u.  Dhat stores its odd-site
                    intermediate in bfloat16 as well: one rounding more, 3u;
  DF64              1e-12: FP64 data in double-float arithmetic, each real held to
                    2^-48 relative and each output component a sum of ~10^2 products.
"""
import numpy as np
import pytest

from oracle.dirac import gamma5
from paper_1908_11673_gb300 import workload
from tests.gpu_helpers import relerr, setup

pytestmark = pytest.mark.gpu

GEOMS = [
    ((6, 4, 4, 6), 0, (np.pi, 0.0, 0.0, 0.0), -2),
    ((4, 6, 4, 8), 0, (0.3, 0.7, -1.1, 2.0), 4),
    ((4, 4, 6, 4), 1, (np.pi, 0.0, 0.0, 0.0), 4),
    ((6, 4, 6, 4), 2, (np.pi, 0.0, 0.0, 0.0), -2),
    ((4, 6, 4, 4), 3, (np.pi, 0.0, 0.0, 0.0), 1),
    ((8, 8, 8, 8), 0, (np.pi, 0.0, 0.0, 0.0), -2),
]
BF16_U = 2.0 ** -9
TOL = {0: 1e-13, 1: 2e-6, 2: 2 * BF16_U, 3: 1e-12}
# Dhat: BF16 keeps one more rounded field (the odd-site intermediate)
TOL_DHAT = {0: 1e-13, 1: 2e-6, 2: 3 * BF16_U}


@pytest.mark.parametrize("L,cstar,theta,qhat", GEOMS)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_apply_Dw_parity(L, cstar, theta, qhat, prec):
    qxd, ctx, op, _, _ = setup(L, cstar, theta, qhat=qhat, seed=1000 + sum(L))
    psi = workload.spinor(op.geom.V, 5)
    if prec in (1, 2):
        psi = psi.astype(np.complex64)
    out = np.empty_like(psi)
    ctx.apply_Dw(0, prec, psi, out)
    ref = op.apply(psi.astype(np.complex128))
    assert relerr(out.astype(np.complex128), ref) <= TOL[prec]
    ctx.close()


@pytest.mark.parametrize("L,cstar,theta,qhat", GEOMS)
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_Dhat_parity(L, cstar, theta, qhat, prec, dagger):
    qxd, ctx, op, _, _ = setup(L, cstar, theta, qhat=qhat, seed=2000 + sum(L))
    ne = op.geom.V // 2
    psi = workload.spinor(ne, 6)
    if prec != 0:
        psi = psi.astype(np.complex64)
    out = np.empty_like(psi)
    ctx.apply_Dhat_eo(0, prec, psi, out, dagger=dagger)
    p = psi.astype(np.complex128)
    ref = gamma5(op.Dhat(gamma5(p))) if dagger else op.Dhat(p)
    assert relerr(out.astype(np.complex128), ref) <= TOL_DHAT[prec]
    ctx.close()


def test_apply_Dw_multiple_rhs_and_device_buffers():
    qxd, ctx, op, _, _ = setup((4, 4, 6, 4), 1, (np.pi, 0, 0, 0), qhat=4)
    import torch
    V = op.geom.V
    psi = workload.spinor(V, 9, nrhs=3)
    d_in = torch.from_numpy(psi).cuda()
    d_out = torch.empty_like(d_in)
    ctx.apply_Dw(0, 0, d_in, d_out, nrhs=3)
    torch.cuda.synchronize()
    out = d_out.cpu().numpy()
    for r in range(3):
        assert relerr(out[r], op.apply(psi[r])) <= 1e-13
    ctx.close()


def test_full_size_sampled_parity():
    """32^3 x 64 physical lattice with C* in 3 directions (extended 64x64x32x32,
    V = 4,194,304), stout-smeared links, qhat = 4: FP64 and FP32 outputs at 3000
    sampled sites against the oracle evaluated at those sites only."""
    import torch
    L = (64, 32, 32, 32)
    qxd, ctx, op, _, _ = setup(L, 3, (np.pi, 0, 0, 0), qhat=4, kappa=0.137312, seed=2000, stout=5,
                               device="cuda")
    V = op.geom.V
    assert V == 4194304
    psi = workload.spinor(V, 2001)
    sites = np.random.default_rng(0).choice(V, 3000, replace=False)
    ref = op.apply(psi, sites)
    d_in = torch.from_numpy(psi).cuda()
    d_out = torch.empty_like(d_in)
    ctx.apply_Dw(0, 0, d_in, d_out)
    out = d_out.cpu().numpy()
    assert relerr(out[sites], ref) <= 1e-13
    ctx.apply_Dw(0, 3, d_in, d_out)
    assert relerr(d_out.cpu().numpy()[sites], ref) <= TOL[3]
    d_in32 = d_in.to(torch.complex64)
    d_out32 = torch.empty_like(d_in32)
    ctx.apply_Dw(0, 1, d_in32, d_out32)
    ref32 = op.apply(d_in32.cpu().numpy().astype(np.complex128), sites)
    assert relerr(d_out32.cpu().numpy()[sites].astype(np.complex128), ref32) <= TOL[1]
    ctx.close()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("nrhs", [2, 3, 5, 12])
def test_multi_rhs_fused_kernel_parity(prec, nrhs):
    """The fused multi-right-hand-side kernel (one link load for all right-hand
    sides, autotuned tile) against the oracle, right-hand side by right-hand side,
    for D_w and for Dhat (which also uses the fused inverse-diagonal epilogue)."""
    import torch
    qxd, ctx, op, _, _ = setup((6, 4, 6, 4), 2, (np.pi, 0, 0, 0), qhat=4, seed=6000 + nrhs)
    V = op.geom.V
    psi = workload.spinor(V, 6001, nrhs=nrhs).astype(np.complex64)
    d_in = torch.from_numpy(psi).cuda()
    d_out = torch.empty_like(d_in)
    ctx.apply_Dw(0, prec, d_in, d_out, nrhs=nrhs)
    out = d_out.cpu().numpy()
    for r in range(nrhs):
        assert relerr(out[r].astype(np.complex128), op.apply(psi[r].astype(np.complex128))) <= TOL[prec]
    ne = V // 2
    pe = workload.spinor(ne, 6002, nrhs=nrhs).astype(np.complex64)
    e_in = torch.from_numpy(pe).cuda()
    e_out = torch.empty_like(e_in)
    ctx.apply_Dhat_eo(0, prec, e_in, e_out, nrhs=nrhs, dagger=True)
    eo = e_out.cpu().numpy()
    for r in range(nrhs):
        ref = gamma5(op.Dhat(gamma5(pe[r].astype(np.complex128))))
        assert relerr(eo[r].astype(np.complex128), ref) <= TOL_DHAT[prec]
    ctx.close()
