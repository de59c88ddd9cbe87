"""Learned preconditioner kernels against the oracle (oracle/ptc.py).

Tolerances: the network runs in FP32 (weights, activations, links), sums of
~10^3 products per output component: forward 1e-5 and loss 1e-5 relative,
gradient 1e-4 (norm-relative, FP64 block sums of FP32 products).
The tensor-core forward layers (bfloat16 transports and weights, FP32
accumulation) round each operand of every product once, 2u per layer with
u = 2^-9 the bfloat16 unit roundoff: 8u over the four layers."""
import numpy as np
import pytest

from oracle import ptc
from paper_1908_11673_gb300 import workload
from tests.gpu_helpers import relerr, setup

pytestmark = pytest.mark.gpu


def rand_weights(rng, nlayers, nch, scale=0.2):
    Ws = ptc.identity_weights(nlayers, nch)
    for W in Ws:
        W += scale * (rng.normal(size=W.shape) + 1j * rng.normal(size=W.shape))
    return Ws


def flat(Ws):
    return np.concatenate([W.reshape(-1) for W in Ws]).astype(np.complex64)


def unflat(x, nlayers, nch):
    out, k = [], 0
    for cin, cout in ptc.layer_shapes(nlayers, nch):
        n = cout * cin * 9 * 16
        out.append(x[k:k + n].reshape(cout, cin, 9, 4, 4))
        k += n
    return out


GEOMS = [((4, 4, 4, 6), 0, (np.pi, 0, 0, 0)), ((4, 4, 6, 4), 2, (np.pi, 0, 0, 0))]


# channel counts: 4 and 3 fit one block's output group, 12 takes two groups of
# the forward kernel and four chunks of the weight-gradient kernel
@pytest.mark.parametrize("L,cstar,theta", GEOMS)
@pytest.mark.parametrize("nch", [4, 12])
def test_forward_parity(L, cstar, theta, nch):
    qxd, ctx, op, _, _ = setup(L, cstar, theta, qhat=4, seed=7100)
    Ws = rand_weights(np.random.default_rng(1), 4, nch)
    ne = op.geom.V // 2
    r = workload.spinor(ne, 7101).astype(np.complex64)
    out = np.empty_like(r)
    ctx.ptc_apply(0, flat(Ws), 4, nch, r, out)
    ref = ptc.network(ptc.Transport(op), Ws, r.astype(np.complex128))
    assert relerr(out.astype(np.complex128), ref) <= 1e-5
    ident = np.empty_like(r)
    ctx.ptc_apply(0, flat(ptc.identity_weights(4, nch)), 4, nch, r, ident)
    assert np.array_equal(ident, r)
    # the channel mixing on the tensor cores
    out_tc = np.empty_like(r)
    ctx.ptc_apply(0, flat(Ws), 4, nch, r, out_tc, prec=qxd.BF16)
    assert relerr(out_tc.astype(np.complex128), ref) <= 8 * 2.0 ** -9
    # identity weights are exact in bfloat16: the output is the input rounded once
    ctx.ptc_apply(0, flat(ptc.identity_weights(4, nch)), 4, nch, r, ident, prec=qxd.BF16)
    assert relerr(ident.astype(np.complex128), r.astype(np.complex128)) <= 2.0 ** -9
    ctx.close()


@pytest.mark.parametrize("L,cstar,theta", GEOMS)
@pytest.mark.parametrize("nch", [3, 12])
@pytest.mark.parametrize("norm", ["error", "residual"])
def test_loss_and_gradient_parity(L, cstar, theta, nch, norm):
    qxd, ctx, op, _, _ = setup(L, cstar, theta, qhat=-2, seed=7200)
    nl = 3
    Ws = rand_weights(np.random.default_rng(2), nl, nch)
    ne = op.geom.V // 2
    r = workload.spinor(ne, 7201, nrhs=2).astype(np.complex64)
    e = workload.spinor(ne, 7202, nrhs=2).astype(np.complex64)
    W32 = flat(Ws)
    grad = np.zeros_like(W32)
    kind = qxd.LOSS_RESIDUAL if norm == "residual" else qxd.LOSS_ERROR
    loss = ctx.ptc_loss_grad(0, W32, nl, nch, r, e, 2, grad=grad, kind=kind)
    Wr = unflat(W32.astype(np.complex128), nl, nch)
    pairs = [(r[i].astype(np.complex128), e[i].astype(np.complex128)) for i in range(2)]
    L0, G = ptc.loss_and_grad(ptc.Transport(op), Wr, pairs, norm=norm)
    assert abs(loss - L0) <= 1e-5 * L0
    assert relerr(grad.astype(np.complex128), np.concatenate([g.reshape(-1) for g in G])) <= 1e-4
    ctx.close()


def test_training_reduces_loss_and_fgcr_uses_the_network():
    qxd, ctx, op, _, _ = setup((8, 8, 8, 8), 0, (np.pi, 0, 0, 0), qhat=-2, seed=7300, stout=5)
    ne = op.geom.V // 2
    b = workload.spinor(ne, 7301)
    npairs = 12
    r = np.empty((npairs, ne, 4, 3), dtype=np.complex64)
    e = np.empty_like(r)
    ctx.ptc_record_pairs(0, b, npairs, 3, r, e)
    # recorded pairs satisfy Dhat e = r (to the FP32 rounding of the stored pair)
    Dinv = op.Doo_inv()
    for i in (0, npairs - 1):
        assert relerr(op.Dhat(e[i].astype(np.complex128), Dinv), r[i].astype(np.complex128)) < 1e-5
    nl, nch = 4, 4
    W = flat(ptc.identity_weights(nl, nch))
    m = np.zeros_like(W)
    v = np.zeros_like(W)
    t = np.zeros(1, dtype=np.int32)
    losses = ctx.ptc_train(0, W, m, v, nl, nch, r, e, npairs, 4, 60, 2e-3, t)
    assert t[0] == 60
    assert np.isfinite(losses).all()
    full0 = ctx.ptc_loss_grad(0, flat(ptc.identity_weights(nl, nch)), nl, nch, r, e, npairs)
    full1 = ctx.ptc_loss_grad(0, W, nl, nch, r, e, npairs)
    assert full1 < 0.7 * full0, (full0, full1)
    ctx.set_precond_weights(0, W, nl, nch)
    eta = workload.spinor(op.geom.V, 7302)
    psi = np.empty_like(eta)
    info = ctx.solve(0, eta, psi, kind=1, tol=1e-10, inner=1, nkv=16, precond=1)
    assert info.status == 0 and info.true_relres <= 1e-10
    sites = np.random.default_rng(0).choice(op.geom.V, 1000, replace=False)
    res = eta[sites] - op.apply(psi, sites)
    assert np.linalg.norm(res) / np.linalg.norm(eta[sites]) < 1e-9
    ctx.close()


def test_learned_preconditioner_effect_16x16x16x16():
    """What the trained network does inside the solver, on the 16^4 configuration
    (5 stout steps, qhat = -2, kappa = 0.136377, csw 1.90952/1.0).
    Training: 4 layers x 8 channels, Adam (6 epochs, batches of 10) on the
    residual-norm loss over 8 x 100 pairs recorded from the plain FP64 solver on
    fields 4000..4007.  Checked: the trained loss is below the identity network's
    and below the zero map's (1 by definition), and on held-out residuals of field
    4100 one application of Dhat M leaves less than the identity network and less
    than the zero map.  Then FGCR(16) with FP32 inner solves, with the network (on
    the tensor cores) and without it, both to the true FP64 residual 1e-10 checked
    by the oracle; their iterations and device times are printed side by side
    (the measured comparison is recorded with the benchmark rows)."""
    import torch

    from paper_1908_11673_gb300 import learned
    from tests.gpu_helpers import need_gpu
    qxd = need_gpu()
    nl, nch = 4, 8
    W, summ = learned.train(learned.FIELD, list(range(4000, 4008)), 100, epochs=6, batch=10)
    print("training:", summ, flush=True)
    assert summ["loss_trained"] < summ["loss_identity"] and summ["loss_trained"] < summ["loss_zero_map"]
    f = learned.FIELD
    U, A = workload.gauge_field(f["L"], 4100, stout_steps=f["stout"], rho=f["rho"])
    from oracle import DiracOperator, Flavour, GaugeField, Geometry
    op = DiracOperator(GaugeField(Geometry(f["L"], 0, f["theta"]), U, A, f["invqel"]),
                       Flavour(f["qhat"], f["kappa"], f["su3csw"], f["u1csw"]))
    ctx = qxd.Context(f["L"], 0, f["theta"])
    ctx.set_links(U, A, f["invqel"])
    ctx.set_clover(0, f["qhat"], f["kappa"], f["su3csw"], f["u1csw"])
    r_held, _, _ = learned.record(ctx, 41001, 8, stride=4)
    red = learned.residual_reduction(ctx, W, nl, nch, r_held)
    red_id = learned.residual_reduction(ctx, learned.identity_weights(nl, nch), nl, nch, r_held)
    print(f"held-out |r - Dhat M r|^2/|r|^2: trained {red:.4f}, identity {red_id:.4f}, zero map 1", flush=True)
    assert red < 1.0 and red < red_id
    ctx.set_precond_weights(0, W, nl, nch)
    eta = workload.spinor(op.geom.V, 41000)
    res = {}
    for name, pre in (("none", qxd.PRECOND_NONE), ("learned", qxd.PRECOND_LEARNED)):
        psi = np.empty_like(eta)
        ctx.solve(0, eta, psi, kind=qxd.FGCR, tol=1e-10, inner=qxd.FP32, nkv=16, precond=pre)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = ctx.solve(0, eta, psi, kind=qxd.FGCR, tol=1e-10, inner=qxd.FP32, nkv=16, precond=pre)
        e1.record()
        torch.cuda.synchronize()
        assert info.status == 0 and info.true_relres <= 1e-10, info.asdict()
        rel = float(np.linalg.norm(eta - op.apply(psi)) / np.linalg.norm(eta))
        assert rel <= 1.5e-10, (name, rel)
        res[name] = (info.iters, e0.elapsed_time(e1), rel)
    print(f"held-out FGCR to 1e-10: without M {res['none'][0]} iterations {res['none'][1]:.1f} ms, "
          f"with M {res['learned'][0]} iterations {res['learned'][1]:.1f} ms", flush=True)
    ctx.close()
