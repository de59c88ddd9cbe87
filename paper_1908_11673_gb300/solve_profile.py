"""Per-kernel profile of one solve on a seeded synthetic field.

Runs `reps` solves of D psi = eta to a true relative residual of 1e-10 through
the C ABI (qxd_solve) with the library's kernel profiling on (qxd_profile mode 2:
launch counts and CUDA-event time of every kernel class on its launching
stream) and prints, per solve, the solver report and the kernel table.

    python -m paper_1908_11673_gb300.solve_profile --L 24,24,24,48 --precond sap [--ncy 5 --nmr 5]
    python -m paper_1908_11673_gb300.solve_profile --L 24,24,24,48 --precond dfl --Ns 12 --ninv 2
    python -m paper_1908_11673_gb300.solve_profile --L 64,32,32,32 --cstar 3 --qhat 4 --kappa 0.137312 \
        --seed 2100 --sigma-h 0.6 --precond dfl --ncy 3 --nmr 4      # rough fields, C* boundary

With --precond dfl the deflation subspace is built first (qxd_dfl_setup) from
Ns Gaussian fields drawn on the device with a seeded torch generator; its
setup time is printed.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import build, qxd, workload


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--L", default="24,24,24,48", help="physical lattice extents x0,x1,x2,x3")
    ap.add_argument("--cstar", type=int, default=0)
    ap.add_argument("--qhat", type=int, default=-2)
    ap.add_argument("--kappa", type=float, default=0.136377)
    ap.add_argument("--seed", type=int, default=2000)
    ap.add_argument("--stout", type=int, default=5)
    ap.add_argument("--sigma-h", type=float, default=0.3,
                    help="width of the random Hermitian generators (0.6: rough fields, plaquette about 0.63)")
    ap.add_argument("--solver", choices=["fgcr", "cgne"], default="fgcr")
    ap.add_argument("--precond", choices=["none", "sap", "dfl"], default="none")
    ap.add_argument("--Ns", type=int, default=12)
    ap.add_argument("--ninv", type=int, default=2)
    ap.add_argument("--ctol", type=float, default=1e-2)
    ap.add_argument("--cnmx", type=int, default=64)
    ap.add_argument("--ncy", type=int, default=5)
    ap.add_argument("--nmr", type=int, default=5)
    ap.add_argument("--nkv", type=int, default=16)
    ap.add_argument("--inner", choices=["fp32", "bf16"], default="fp32")
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides solved in lockstep (FGCR)")
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--top", type=int, default=10)
    args = ap.parse_args(argv)
    import torch

    build.build()
    L = tuple(int(v) for v in args.L.split(","))
    U, A = workload.gauge_field(L, args.seed, sigma_h=args.sigma_h, stout_steps=args.stout)
    ctx = qxd.Context(L, args.cstar, (np.pi, 0.0, 0.0, 0.0))
    ctx.set_links(U, A, 6.0)
    ctx.set_clover(0, args.qhat, args.kappa, 1.90952, 1.0)
    if args.nrhs == 1:
        eta = torch.from_numpy(workload.spinor(ctx.V, args.seed + 1)).cuda()
    else:
        eta = torch.from_numpy(np.stack([workload.spinor(ctx.V, args.seed + 1 + j) for j in range(args.nrhs)])).cuda()
    psi = torch.empty_like(eta)
    ctx.set_sap(args.ncy, args.nmr)
    kind = qxd.FGCR if args.solver == "fgcr" else qxd.CGNE
    pre = {"none": qxd.PRECOND_NONE, "sap": qxd.PRECOND_SAP, "dfl": qxd.PRECOND_DFL}[args.precond]
    if args.precond == "dfl":
        gen = torch.Generator(device="cuda").manual_seed(args.seed + 7)
        seeds = torch.randn((args.Ns, ctx.V, 4, 3), dtype=torch.complex64, device="cuda", generator=gen)
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx.dfl_setup(0, seeds, args.Ns, ninv=args.ninv, ctol=args.ctol, cnmx=args.cnmx)
        torch.cuda.synchronize()
        print(json.dumps({"dfl_setup_ms": round((time.perf_counter() - t) * 1e3, 1), "Ns": args.Ns,
                          "ninv": args.ninv}))
        del seeds
    inner = qxd.FP32 if args.inner == "fp32" else qxd.BF16
    for _ in range(args.reps):
        ctx.profile(2)
        torch.cuda.synchronize()
        t = time.perf_counter()
        info = ctx.solve(0, eta, psi, kind=kind, tol=1e-10, inner=inner, nkv=args.nkv, precond=pre, nrhs=args.nrhs)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        prof = ctx.profile_entries()
        ctx.profile(0)
        print(json.dumps({"ms": round(dt * 1e3, 2)} | info.asdict()))
        tot = sum(p["ms"] for p in prof) or 1.0
        for p in sorted(prof, key=lambda p: -p["ms"])[: args.top]:
            gbs = p["bytes"] / p["ms"] / 1e6 if p["ms"] else 0.0
            print(f"  {p['name']:28s} {p['launches']:7d} {p['ms']:10.3f} ms {p['ms'] / p['launches'] * 1e3:9.1f} us/launch"
                  f"  share {p['ms'] / tot:.3f}  {gbs:8.1f} GB/s")
    ctx.close()


if __name__ == "__main__":
    main()
