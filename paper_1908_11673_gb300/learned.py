"""Learned preconditioner experiment on 16^4 lattices.

Training: a gauge-covariant network (4 parallel-transport layers, 8 channels,
FP32 weights, identity start) is trained with Adam on residual/error pairs
(r_k, x* - x_k) that the plain FP64 solver (CG on the normal equations of
Dhat) produces on seeded smeared gauge fields.  Evaluation: on held-out fields,
FGCR (FP32 inner solves, FP64 defect correction) to a true relative residual of
1e-10 with and without the network as right preconditioner, and the plain FP64
CGNE on the same systems: iterations and device time.

Everything runs through the C ABI (qxd_ptc_record_pairs, qxd_ptc_train,
qxd_set_precond_weights, qxd_solve).

    python -m paper_1908_11673_gb300.learned [--train-fields 20] [--pairs 100] ...
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import qxd, workload

FIELD = dict(L=(16, 16, 16, 16), cstar=0, theta=(math.pi, 0.0, 0.0, 0.0), qhat=-2, kappa=0.136377,
             su3csw=1.90952, u1csw=1.0, invqel=6.0, stout=5, rho=0.1)


def identity_weights(nlayers, nch):
    """Weights of the identity network: W[c][c][0] = 1 (4x4) for c < min(c_in, c_out)
    in every layer, complex64 [layers][cout][cin][9][4][4] flattened."""
    parts = []
    for l in range(nlayers):
        cin = 1 if l == 0 else nch
        cout = 1 if l == nlayers - 1 else nch
        W = np.zeros((cout, cin, 9, 4, 4), dtype=np.complex64)
        for c in range(min(cin, cout)):
            W[c, c, 0] = np.eye(4)
        parts.append(W.reshape(-1))
    return np.concatenate(parts)


def make_context(seed, device=0, field=FIELD):
    U, A = workload.gauge_field(field["L"], seed, sigma_h=field.get("sigma_h", 0.3), stout_steps=field["stout"],
                                rho=field["rho"], u1_stout_steps=field.get("u1_stout", 0))
    ctx = qxd.Context(field["L"], field["cstar"], field["theta"], device=device)
    ctx.set_links(U, A, field["invqel"])
    ctx.set_clover(0, field["qhat"], field["kappa"], field["su3csw"], field["u1csw"])
    return ctx


def record(ctx, seed, npairs, stride=None):
    """npairs pairs spread over one plain FP64 solve of Dhat x = b (b Gaussian):
    every `stride`-th iterate, or (stride None) the largest stride for which the
    solve has npairs * stride iterations (found by bisection)."""
    ne = ctx.Vh
    b = workload.spinor(ne, seed)
    lo = stride
    if lo is None:
        # count the iterations of the plain solve first, then sample its iterates evenly
        probe_r = np.empty((1, ne, 4, 3), dtype=np.complex64)
        probe_e = np.empty_like(probe_r)
        lo, hi = 1, 4096
        while lo < hi:  # largest stride s with npairs * s iterations available
            mid = (lo + hi + 1) // 2
            try:
                ctx.ptc_record_pairs(0, b, 1, mid * npairs, probe_r, probe_e)
                lo = mid
            except qxd.QxdError:
                hi = mid - 1
    r = np.empty((npairs, ne, 4, 3), dtype=np.complex64)
    e = np.empty_like(r)
    ctx.ptc_record_pairs(0, b, npairs, lo, r, e)
    return r, e, lo


def train(field, seeds, npairs, epochs=6, batch=10, lr=2e-3, nlayers=4, nch=8, stride=None, device=0,
          loss="residual"):
    """Train the network on pairs recorded on the fields of `seeds` (one context
    per field, all on the GPU): Adam from the identity network, `epochs` passes
    over every field's pairs in batches, on the residual-norm loss
    |r - Dhat M r|^2/|r|^2 (loss="residual", the pair error in the norm |Dhat .|)
    or the Euclidean error |M r - e|^2/|e|^2 (loss="error").  Returns (W, summary)
    with the mean loss per epoch and the mean loss of the identity, the zero map
    (1 by definition) and the trained network over all pairs."""
    kind = qxd.LOSS_RESIDUAL if loss == "residual" else qxd.LOSS_ERROR
    t0 = time.time()
    W = identity_weights(nlayers, nch)
    if loss == "residual":
        # start from M = 2 kappa (the inverse of the mass term of Dhat), the last layer scaled
        nlast = 16 * 9 * nch  # weights of the last layer (nch -> 1)
        W[-nlast:] *= np.complex64(2.0 * field["kappa"])
    m = np.zeros_like(W)
    v = np.zeros_like(W)
    t = np.zeros(1, dtype=np.int32)
    data = []
    for i, sd in enumerate(seeds):
        ctx = make_context(sd, device, field)
        r, e, st = record(ctx, 10 * sd + 1, npairs, stride)
        data.append((ctx, r, e))
    t_pairs = time.time() - t0
    history = []
    steps = max(1, npairs // batch)
    for _ in range(epochs):
        el = []
        for ctx, r, e in data:
            el.extend(ctx.ptc_train(0, W, m, v, nlayers, nch, r, e, npairs, batch, steps, lr, t, kind=kind).tolist())
        history.append(float(np.mean(el)))
    t_train = time.time() - t0 - t_pairs
    ident = identity_weights(nlayers, nch)
    loss_id = float(np.mean([ctx.ptc_loss_grad(0, ident, nlayers, nch, r, e, npairs, kind=kind) / npairs
                             for ctx, r, e in data]))
    loss_tr = float(np.mean([ctx.ptc_loss_grad(0, W, nlayers, nch, r, e, npairs, kind=kind) / npairs
                             for ctx, r, e in data]))
    for ctx, _, _ in data:
        ctx.close()
    return W, {"fields": len(seeds), "pairs": len(seeds) * npairs, "network": f"{nlayers} layers x {nch} channels",
               "loss": loss, "epochs": epochs, "loss_zero_map": 1.0, "loss_identity": loss_id, "loss_trained": loss_tr,
               "loss_history": history, "seconds_pairs": t_pairs, "seconds_training": t_train}


def residual_reduction(ctx, W, nlayers, nch, r):
    """Mean of |r - Dhat M r|^2 / |r|^2 over the residuals r [n][V/2][4][3]
    (complex64): how much of r one application of M Dhat removes (1 for M = 0),
    through qxd_ptc_apply and qxd_apply_Dhat_eo (FP32)."""
    out = []
    Mr = np.empty_like(r[0])
    DMr = np.empty_like(r[0])
    for ri in r:
        ctx.ptc_apply(0, W, nlayers, nch, ri, Mr)
        ctx.apply_Dhat_eo(0, qxd.FP32, Mr, DMr)
        out.append(float(np.linalg.norm(ri - DMr) ** 2 / np.linalg.norm(ri) ** 2))
    return float(np.mean(out))


def evaluate(ctx, W, nlayers, nch, seed, nkv=16):
    eta = workload.spinor(ctx.V, seed)
    psi = np.empty_like(eta)
    out = {}
    import torch
    for name, kind, pre in (("fgcr", qxd.FGCR, qxd.PRECOND_NONE), ("fgcr_learned", qxd.FGCR, qxd.PRECOND_LEARNED),
                            ("cgne_fp64", qxd.CGNE, qxd.PRECOND_NONE)):
        if pre == qxd.PRECOND_LEARNED:
            ctx.set_precond_weights(0, W, nlayers, nch)
        ctx.solve(0, eta, psi, kind=kind, tol=1e-10, inner=qxd.FP32, nkv=nkv, precond=pre)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = ctx.solve(0, eta, psi, kind=kind, tol=1e-10, inner=qxd.FP32, nkv=nkv, precond=pre)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"iters": info.iters, "ms": e0.elapsed_time(e1), "true_relres": info.true_relres,
                     "status": info.status}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--train-fields", type=int, default=20)
    ap.add_argument("--eval-fields", type=int, default=10)
    ap.add_argument("--pairs", type=int, default=100, help="pairs per training field")
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=10)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--nlayers", type=int, default=4)
    ap.add_argument("--nch", type=int, default=8)
    ap.add_argument("--loss", choices=["residual", "error"], default="residual")
    ap.add_argument("--out", default=None, help="write the JSON summary here")
    ap.add_argument("--weights", default=None, help="save the trained weights (.npy)")
    args = ap.parse_args(argv)

    W, summ_train = train(FIELD, [4000 + i for i in range(args.train_fields)], args.pairs, args.epochs, args.batch,
                          args.lr, args.nlayers, args.nch, loss=args.loss)
    evals = []
    for i in range(args.eval_fields):
        ctx = make_context(4100 + i)
        evals.append(evaluate(ctx, W, args.nlayers, args.nch, 41000 + i))
        ctx.close()
    summ = {k: {"iters_mean": float(np.mean([e[k]["iters"] for e in evals])),
                "ms_mean": float(np.mean([e[k]["ms"] for e in evals])),
                "max_true_relres": float(max(e[k]["true_relres"] for e in evals))} for k in evals[0]}
    result = summ_train | {"eval_fields": args.eval_fields, "held_out": summ}
    print(json.dumps(result, indent=1))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(result, f, indent=1)
    if args.weights:
        np.save(args.weights, W)
    return result


if __name__ == "__main__":
    main()
