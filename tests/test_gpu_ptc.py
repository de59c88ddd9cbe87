"""Learned preconditioner kernels against the oracle (oracle/ptc.py).

Tolerances: the network runs in FP32 (weights, activations, links), sums of
~10^3 products per output component: forward 1e-5 and loss 1e-5 relative,
gradient 1e-4 (norm-relative, FP64 block sums of FP32 products)."""
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


@pytest.mark.parametrize("L,cstar,theta", GEOMS)
def test_forward_parity(L, cstar, theta):
    qxd, ctx, op, _, _ = setup(L, cstar, theta, qhat=4, seed=7100)
    Ws = rand_weights(np.random.default_rng(1), 4, 4)
    ne = op.geom.V // 2
    r = workload.spinor(ne, 7101).astype(np.complex64)
    out = np.empty_like(r)
    ctx.ptc_apply(0, flat(Ws), 4, 4, r, out)
    ref = ptc.network(ptc.Transport(op), Ws, r.astype(np.complex128))
    assert relerr(out.astype(np.complex128), ref) <= 1e-5
    ident = np.empty_like(r)
    ctx.ptc_apply(0, flat(ptc.identity_weights(4, 4)), 4, 4, r, ident)
    assert np.array_equal(ident, r)
    ctx.close()


@pytest.mark.parametrize("L,cstar,theta", GEOMS)
def test_loss_and_gradient_parity(L, cstar, theta):
    qxd, ctx, op, _, _ = setup(L, cstar, theta, qhat=-2, seed=7200)
    nl, nch = 3, 3
    Ws = rand_weights(np.random.default_rng(2), nl, nch)
    ne = op.geom.V // 2
    r = workload.spinor(ne, 7201, nrhs=2).astype(np.complex64)
    e = workload.spinor(ne, 7202, nrhs=2).astype(np.complex64)
    W32 = flat(Ws)
    grad = np.zeros_like(W32)
    loss = ctx.ptc_loss_grad(0, W32, nl, nch, r, e, 2, grad=grad)
    Wr = unflat(W32.astype(np.complex128), nl, nch)
    pairs = [(r[i].astype(np.complex128), e[i].astype(np.complex128)) for i in range(2)]
    L0, G = ptc.loss_and_grad(ptc.Transport(op), Wr, pairs)
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
