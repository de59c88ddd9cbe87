"""The allocation-free even-odd operator (qxd_apply_Dhat_eo_noalloc) gives the
same result as qxd_apply_Dhat_eo.

It is for callers that cannot allocate device memory during the call (their
own pool owns the device memory, or a device-wide synchronisation from
cudaMalloc is not acceptable).  It keeps its temporaries in a fixed device
array of the library.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1908_11673_gb300 import workload
from tests.gpu_helpers import relerr, setup

pytestmark = pytest.mark.gpu

# the operator-parity tolerances of test_gpu_operator.py (FP64, FP32, and for
# bfloat16 storage 3u, u = 2^-9: input, odd intermediate and output rounded)
TOL = {0: 1e-13, 1: 2e-6, 2: 3 * 2.0 ** -9}


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("dagger", [False, True])
def test_noalloc_matches_apply_Dhat_eo_on_two_calls(prec, dagger):
    """Two calls in a row with different inputs.  The first noalloc call comes
    before any qxd_apply_Dhat_eo on the context, so it runs with the launch
    shape that was never tuned (the default); the second after it."""
    import torch
    qxd, ctx, op, _, _ = setup((6, 4, 6, 4), 2, (np.pi, 0.0, 0.0, 0.0), qhat=-2, seed=5100)
    ne = op.geom.V // 2
    dt = torch.complex128 if prec == 0 else torch.complex64
    outs = []
    for call in range(2):
        psi = torch.from_numpy(workload.spinor(ne, 5200 + call)).to(dt).cuda()
        ref = torch.empty_like(psi)
        got = torch.empty_like(psi)
        ctx.apply_Dhat_eo_noalloc(0, prec, psi, got, dagger=dagger)
        ctx.apply_Dhat_eo(0, prec, psi, ref, dagger=dagger)
        torch.cuda.synchronize()
        r = ref.cpu().numpy().astype(np.complex128)
        assert relerr(got.cpu().numpy().astype(np.complex128), r) <= TOL[prec]
        outs.append(r)
    assert relerr(outs[0], outs[1]) > 0.1  # two different inputs, two different results
    ctx.close()


def test_noalloc_rejects_host_arrays_and_large_lattices():
    qxd, ctx, op, _, _ = setup((4, 4, 4, 4), 0, (np.pi, 0.0, 0.0, 0.0))
    psi = workload.spinor(op.geom.V // 2, 1)
    out = np.empty_like(psi)
    with pytest.raises(qxd.QxdError) as e:
        ctx.apply_Dhat_eo_noalloc(0, 0, psi, out)
    assert e.value.code == 1 and "device arrays" in str(e.value)
    ctx.close()
    big = qxd.Context((16, 16, 16, 18), 0, (np.pi, 0.0, 0.0, 0.0))
    U, A = workload.unit_gauge_field(big.L)
    big.set_links(U, A)
    big.set_clover(0, -2, 0.13, 1.9, 1.0)
    import torch
    x = torch.zeros((big.Vh, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(qxd.QxdError) as e:
        big.apply_Dhat_eo_noalloc(0, 0, x, torch.empty_like(x))
    assert e.value.code == 1 and "at most 32768" in str(e.value)
    big.close()


def test_noalloc_call_records_into_a_cuda_graph():
    """No allocation and no host wait inside the call: after a first call (which looks up
    the scratch array's address) it records into a CUDA graph, and the replay gives
    qxd_apply_Dhat_eo's result for the input present at replay time."""
    import torch
    qxd, ctx, op, _, _ = setup((6, 4, 6, 4), 2, (np.pi, 0.0, 0.0, 0.0), qhat=-2, seed=5100)
    ne = op.geom.V // 2
    psi = torch.from_numpy(workload.spinor(ne, 5300)).to(torch.complex64).cuda()
    got = torch.empty_like(psi)
    ref = torch.empty_like(psi)
    ctx.apply_Dhat_eo_noalloc(0, 1, psi, got)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.apply_Dhat_eo_noalloc(0, 1, psi, got, stream=s)
    psi.copy_(torch.from_numpy(workload.spinor(ne, 5301)).to(torch.complex64))
    got.zero_()
    g.replay()
    torch.cuda.synchronize()
    ctx.apply_Dhat_eo(0, 1, psi, ref)
    torch.cuda.synchronize()
    r = ref.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(r) > 0
    assert relerr(got.cpu().numpy().astype(np.complex128), r) <= TOL[1]
    ctx.close()
