"""Inexact deflation with SAP on the GPU (Sec. 4.4, DFL+SAP+GCR) against the
oracle (oracle/deflation.py) on the same seeded fields and random start fields.

Tolerances.  The subspace passes through FP32 SAP applications and FP32
Gram-Schmidt on the GPU against FP64 on the oracle: 1e-4 per basis field.
The little operator and the preconditioner are compared on the GPU's own basis
(read back), so only FP32 arithmetic separates the sides: 1e-5 of max |A|, and
1e-4 for M_dfl with the little system solved to 1e-7 on the GPU (exactly on the
oracle)."""
import numpy as np
import pytest

from oracle.deflation import Deflation, block_neighbours
from oracle.sap import SAP
from paper_1908_11673_gb300 import workload
from tests.gpu_helpers import relerr, setup

pytestmark = pytest.mark.gpu

CASES = [((8, 8, 8, 8), 0, 4), ((8, 4, 8, 8), 1, 3)]  # L, cstar, Ns


def seeds(V, Ns, seed):
    return np.stack([workload.spinor(V, seed + k) for k in range(Ns)]).astype(np.complex64)


def gpu_basis(ctx, V, Ns):
    out = []
    for k in range(Ns):
        b = np.empty((V, 4, 3), dtype=np.complex64)
        ctx.dfl_basis(0, k, b)
        out.append(b)
    return np.array(out)


@pytest.mark.parametrize("L,cstar,Ns", CASES)
def test_dfl_subspace_and_little_operator(L, cstar, Ns):
    qxd, ctx, op, _, _ = setup(L, cstar, (np.pi, 0, 0, 0), qhat=-2, kappa=0.13, seed=9400, stout=1)
    V = op.geom.V
    sd = seeds(V, Ns, 9401)
    ctx.set_sap(2, 3)
    ctx.dfl_setup(0, sd, Ns, ninv=1)
    sap = SAP(op, bsize=4, ncy=2, nmr=3)
    ref = Deflation(op, sap, sd.astype(np.complex128), ninv=1)
    basis = gpu_basis(ctx, V, Ns)
    for k in range(Ns):
        assert relerr(basis[k].astype(np.complex128), ref.phis[k]) <= 1e-4, k
    # the little operator on the GPU's own basis
    A, nbr = ctx.dfl_little(0, Ns)
    assert np.array_equal(nbr, block_neighbours(sap, op.geom))
    mine = Deflation.from_basis(op, sap, basis.astype(np.complex128))
    # the slots of one block pair add up (with two blocks in a direction the +mu
    # and -mu faces face the same block)
    dense = np.zeros_like(mine.A)
    for B in range(mine.nblocks):
        for s in range(9):
            Bp = nbr[B, s]
            dense[B * Ns:(B + 1) * Ns, Bp * Ns:(Bp + 1) * Ns] += A[B, s].T  # [k][l]
    assert np.abs(dense - mine.A).max() <= 1e-5 * np.abs(mine.A).max()
    ctx.close()


def test_dfl_apply_parity():
    qxd, ctx, op, _, _ = setup((8, 8, 8, 8), 0, (np.pi, 0, 0, 0), qhat=4, kappa=0.13, seed=9410, stout=1)
    V = op.geom.V
    Ns = 4
    ctx.set_sap(2, 3)
    ctx.dfl_setup(0, seeds(V, Ns, 9411), Ns, ninv=1, ctol=1e-7, cnmx=1000, cnkv=16)
    sap = SAP(op, bsize=4, ncy=2, nmr=3)
    mine = Deflation.from_basis(op, sap, gpu_basis(ctx, V, Ns).astype(np.complex128))
    v = workload.spinor(V, 9412).astype(np.complex64)
    out = np.empty_like(v)
    info = ctx.dfl_apply(0, v, out)
    assert info.true_relres <= 1e-7
    assert relerr(out.astype(np.complex128), mine.apply(v.astype(np.complex128))) <= 1e-4
    ctx.close()


@pytest.mark.parametrize("inner", [1, 2])
def test_dfl_fgcr_solves(inner):
    qxd, ctx, op, _, _ = setup((16, 16, 16, 16), 0, (np.pi, 0, 0, 0), qhat=-2, seed=4100, stout=5)
    V = op.geom.V
    ctx.set_sap(3, 4)
    ctx.dfl_setup(0, seeds(V, 8, 9420), 8, ninv=3)
    eta = workload.spinor(V, 41000)
    psi = np.empty_like(eta)
    info = ctx.solve(0, eta, psi, kind=1, tol=1e-10, inner=inner, nkv=16, precond=3)
    assert info.status == 0 and info.true_relres <= 1e-10
    sites = np.random.default_rng(0).choice(V, 1000, replace=False)
    r = eta[sites] - op.apply(psi, sites)
    assert np.linalg.norm(r) / np.linalg.norm(eta[sites]) < 1e-9
    ctx.close()


def test_dfl_errors():
    qxd, ctx, op, _, _ = setup((8, 8, 8, 8), 0, (np.pi, 0, 0, 0))
    V = op.geom.V
    v = workload.spinor(V, 1).astype(np.complex64)
    with pytest.raises(qxd.QxdError) as e:
        ctx.dfl_apply(0, v, np.empty_like(v))
    assert e.value.code == 7
    eta = workload.spinor(V, 2)
    with pytest.raises(qxd.QxdError) as e:
        ctx.solve(0, eta, np.empty_like(eta), kind=1, precond=3)
    assert e.value.code == 7
    with pytest.raises(qxd.QxdError) as e:
        ctx.dfl_setup(0, seeds(V, 33, 3), 33)
    assert e.value.code == 1
    ctx.close()


@pytest.mark.parametrize("Ns,cnkv,ctas,cancel", [(12, 6, None, None), (12, 6, "1", None), (7, 5, "1", "2"),
                                                 (20, 4, None, "2")])
def test_dfl_little_solver(monkeypatch, Ns, cnkv, ctas, cancel):
    """The little-system GCR (one cooperative launch, grid barriers, sums reduced on every
    CTA): M_dfl v against the oracle's exact little solve on the GPU's own basis, on 32
    blocks, with restarts (cnkv below the step count), several blocks per warp
    (QXD_DFL_CTAS=1: one CTA of 16 warps), Ns that leaves lanes idle (7: four rows of A side
    by side in 28 lanes), and the explicit-norm step forced (QXD_DFL_CANCEL=2)."""
    if ctas:
        monkeypatch.setenv("QXD_DFL_CTAS", ctas)
    if cancel:
        monkeypatch.setenv("QXD_DFL_CANCEL", cancel)
    qxd, ctx, op, _, _ = setup((16, 8, 8, 8), 0, (np.pi, 0, 0, 0), qhat=-2, kappa=0.13, seed=9430, stout=1)
    V = op.geom.V
    ctx.set_sap(2, 3)
    ctx.dfl_setup(0, seeds(V, Ns, 9431), Ns, ninv=1, ctol=1e-7, cnmx=5000, cnkv=cnkv)
    sap = SAP(op, bsize=4, ncy=2, nmr=3)
    mine = Deflation.from_basis(op, sap, gpu_basis(ctx, V, Ns).astype(np.complex128))
    assert mine.nblocks == 32
    v = workload.spinor(V, 9432).astype(np.complex64)
    out = np.empty_like(v)
    info = ctx.dfl_apply(0, v, out)
    assert info.true_relres <= 1e-7
    assert info.iters > cnkv  # restarted at least once
    assert relerr(out.astype(np.complex128), mine.apply(v.astype(np.complex128))) <= 1e-4
    ctx.close()
