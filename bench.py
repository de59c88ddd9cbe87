#!/usr/bin/env python
"""Benchmark of the Wilson-clover QCD+QED Dirac operator and its solvers on one
GB300 (or N replicas under torchrun).

Workload (one step): solve D psi = eta to a true FP64 relative residual of 1e-10
on the 32^3 x 64 lattice with C* boundary conditions in the three spatial
directions (simulated extended lattice 64 x 64 x 32 x 32, V = 4,194,304 sites),
antiperiodic time, stout-smeared synthetic SU(3) links (5 steps, rho = 0.1) and
Gaussian U(1) angles, flavour qhat = 4, kappa = 0.137312, csw = 1.90952 / 1.0,
with the mixed-precision solver (flexible GCR on Dhat in FP32 inside FP64
defect correction).

Reported:
  value      operator throughput inside the timed solves in Gflop/s: every
             half-lattice hopping launch counts 2112 flop per output site (so one
             D_w or one Dhat application = 2112 V flop), divided by the device time;
  time_to_solution   the same solve (ms_per_step) against the plain FP64 CGNE solve;
  roofline   the dominant kernel's algorithmic bytes per launch / its mean
             CUDA-event duration, against the measured HBM copy bandwidth;
  e2e        the same metric through the C ABI with pinned HOST buffers (the
             library copies eta in and psi out inside the timed call);
  cpu_baseline  the FP64 oracle applying D_w to a bounded sample of sites;
  next_rows  outside the timed region, on the same system: the SAP-preconditioned
             solve (Sec. 4.4 SAP+GCR) and the deflated one (DFL+SAP+GCR, subspace
             setup timed apart) against the unpreconditioned one, and the
             pseudofermion action of the printed degree-10 rational approximation
             (App. A.2: one 10-shift multi-shift CG plus FP64 assembly) and the
             small-determinant action (Sec. 2.3), each timed with CUDA events.

--impl reference times the oracle (the plain CPU implementation) on the same
metric, each step a bounded sample of sites of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Dw Gflop/s & % HBM roofline; time-to-1e-10 residual vs plain FP64 GPU solve"
FLOP_PER_SITE = 2112
# FP64 FMA throughput of this GPU, measured with a dependent-chain FMA probe
# (8 chains per thread, 4-8 blocks of 256 threads per SM): 1.19 TFLOP/s.
FP64_PEAK_TFLOPS = 1.19


# DRAM bytes per output site measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum)
# on the 24^3x48 lattice for the current kernels;
# a launch on another lattice moves these bytes times its V/2 sites.
NCU_BYTES_PER_SITE = {"hop_fp32_self1_post0": 1000.6, "hop_fp32_self0_post1": 898.4}
# DRAM bytes over algorithmic bytes, measured the same way, for kernels whose bytes per
# launch vary (the hop with fused inner products reads one field per earlier basis field)
NCU_TRAFFIC_RATIO = {"hop_fp32_self1_post0_dots": 0.998}


GOLDEN_RATIONAL = os.path.join(ROOT, "tests", "golden", "rational_deg10_pow_m1_4.txt")


def read_rational(path):
    """(A, nu[], mu[]) from a [Rational] record (key value lines, '#' comments)."""
    vals, nu, mu = {}, {}, {}
    with open(path) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line or line.startswith("["):
                continue
            key, *rest = line.split()
            if key.startswith("nu["):
                nu[int(key[3:-1])] = float(rest[0])
            elif key.startswith("mu["):
                mu[int(key[3:-1])] = float(rest[0])
            else:
                vals[key] = rest
    n = int(vals["degree"][0])
    return float(vals["A"][0]), np.array([nu[i] for i in range(n)]), np.array([mu[i] for i in range(n)])


def hop_bytes_per_launch(entry, V):
    """Algorithmic bytes of one FP64 hopping launch without right-hand-side scaling
    (used to recover the number of right-hand sides of a profile entry)."""
    self_mode = int(entry["name"].split("_self")[1][0])
    post = int(entry["name"].split("_post")[1][0])
    per = 2 * 192 + 8 * 144 + (192 if self_mode else 0) + 576 * ((self_mode == 1) + (post == 1))
    return (V // 2) * per

WORKLOADS = {
    "32^3x64-cstar3": dict(L=(64, 32, 32, 32), cstar=3, theta=(math.pi, 0.0, 0.0, 0.0), qhat=4,
                           kappa=0.137312, su3csw=1.90952, u1csw=1.0, invqel=6.0, field_seed=2000,
                           src_seed=2001, stout=5, rho=0.1),
    # the bench lattice and couplings on rougher fields (H entries N(0, 0.6^2), plaquette about 0.63
    # after the 5 stout steps, the value the configurations aim at): the preconditioner comparison
    "32^3x64-cstar3-rough": dict(L=(64, 32, 32, 32), cstar=3, theta=(math.pi, 0.0, 0.0, 0.0), qhat=4,
                                 kappa=0.137312, su3csw=1.90952, u1csw=1.0, invqel=6.0, field_seed=2100,
                                 src_seed=2101, stout=5, rho=0.1, sigma_h=0.6),
    # 24^3 x 48, antiperiodic time (larger than L2, a few GB on the device: profiler captures)
    "24^3x48": dict(L=(48, 24, 24, 24), cstar=0, theta=(math.pi, 0.0, 0.0, 0.0), qhat=-2, kappa=0.136377,
                    su3csw=1.90952, u1csw=1.0, invqel=6.0, field_seed=3000, src_seed=3001, stout=5, rho=0.1),
    # small case for quick checks (8^4, antiperiodic time)
    "8^4": dict(L=(8, 8, 8, 8), cstar=0, theta=(math.pi, 0.0, 0.0, 0.0), qhat=-2, kappa=0.136377,
                su3csw=1.90952, u1csw=1.0, invqel=6.0, field_seed=1000, src_seed=1001, stout=0, rho=0.1),
    "16^4": dict(L=(16, 16, 16, 16), cstar=0, theta=(math.pi, 0.0, 0.0, 0.0), qhat=-2, kappa=0.136377,
                 su3csw=1.90952, u1csw=1.0, invqel=6.0, field_seed=4000, src_seed=4001, stout=5, rho=0.1),
}


def workload_desc(name, w, args, world=1):
    """The `config` object: identical keys on the native and the reference arm."""
    L = w["L"]
    ext = (L[0], 2 * L[1] if w["cstar"] else L[1], L[2], L[3])
    return {
        "workload": f"{name}: Wilson-clover SU(3)xU(1) Dirac solve to 1e-10, physical {L[3]}x{L[2]}x{L[1]}x{L[0]}"
                    f" (x,y,z,t), C* dirs={w['cstar']}, simulated {'x'.join(map(str, ext))}",
        "V": int(np.prod(ext)),
        "qhat": w["qhat"], "kappa": w["kappa"], "su3csw": w["su3csw"], "u1csw": w["u1csw"],
        "stout_steps": w["stout"], "rho": w["rho"], "field_seed": w["field_seed"], "source_seed": w["src_seed"],
        "solver": "FGCR on Dhat, inner solve in FP32 (or BF16 basis storage), FP64 defect correction",
        "tol": 1e-10,
        "l2": "working set (links, SW terms, Krylov vectors) >> 129 MB L2; no flush",
        "nkv": args.nkv, "inner": args.inner,
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
    }


# ----------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------------
def oracle_rate(w, U, A, psi, seconds, rng_seed=0):
    """FP64 oracle applying D_w at a random sample of sites; returns (Gflop/s, sites, s)."""
    from oracle import DiracOperator, Flavour, GaugeField, Geometry
    geom = Geometry(w["L"], w["cstar"], w["theta"])
    op = DiracOperator(GaugeField(geom, U, A, w["invqel"]),
                       Flavour(w["qhat"], w["kappa"], w["su3csw"], w["u1csw"]))
    rng = np.random.default_rng(rng_seed)
    n = 512
    t0 = time.perf_counter()
    op.apply(psi, rng.choice(geom.V, n, replace=False))
    dt = time.perf_counter() - t0
    n = int(min(geom.V // 8 - 1, max(512, n * seconds / max(dt, 1e-3))))
    sites = rng.choice(geom.V, n, replace=False)
    t0 = time.perf_counter()
    op.apply(psi, sites)
    dt = time.perf_counter() - t0
    return FLOP_PER_SITE * n / dt / 1e9, n, dt


def _oracle_worker(job):
    """One process of the all-core oracle timing: D_w at its share of the sites,
    fields read from memory-mapped .npy files.  Returns (sites, wall start, wall end)."""
    import sys as _sys
    _sys.path.insert(0, job["root"])
    from oracle import DiracOperator, Flavour, GaugeField, Geometry
    w = job["w"]
    U = np.load(job["U"], mmap_mode="r")
    A = np.load(job["A"], mmap_mode="r")
    psi = np.load(job["psi"], mmap_mode="r")
    geom = Geometry(w["L"], w["cstar"], w["theta"])
    op = DiracOperator(GaugeField(geom, U, A, w["invqel"]), Flavour(w["qhat"], w["kappa"], w["su3csw"], w["u1csw"]))
    sites = np.asarray(job["sites"], dtype=np.int64)
    op.apply(psi, sites[:64])  # touch the pages of the code path before the clock starts
    t0 = time.time()
    op.apply(psi, sites)
    return len(sites), t0, time.time()


def oracle_rate_all_cores(w, U, A, psi, seconds, single_rate):
    """The oracle on every core of this process's affinity set: one spawned worker
    per core (OMP/BLAS threads pinned to 1), each applying D_w at its own share of
    a random sample of sites sized for about `seconds` of wall time from the
    single-core rate.  Returns (Gflop/s, cores, sites, wall s)."""
    import multiprocessing as mp
    import shutil
    import tempfile
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    V = psi.shape[0]
    per_core = max(256, int(single_rate * 1e9 / FLOP_PER_SITE * seconds))
    n = int(min(V // 2, per_core * cores))
    sites = np.random.default_rng(7).choice(V, n, replace=False)
    tmp = tempfile.mkdtemp(prefix="qxd_oracle_")
    try:
        paths = {}
        for key, arr in (("U", U), ("A", A), ("psi", psi)):
            paths[key] = os.path.join(tmp, key + ".npy")
            np.save(paths[key], np.ascontiguousarray(arr))
        env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env:
            os.environ[k] = "1"
        try:
            jobs = [dict(root=ROOT, w=w, sites=chunk, **paths) for chunk in np.array_split(sites, cores)]
            with mp.get_context("spawn").Pool(cores) as pool:
                res = pool.map(_oracle_worker, jobs)
        finally:
            for k, v in env.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    nsites = sum(r[0] for r in res)
    return FLOP_PER_SITE * nsites / wall / 1e9, cores, nsites, wall


def make_inputs(w, device):
    from paper_1908_11673_gb300 import workload
    U, A = workload.gauge_field(w["L"], w["field_seed"], sigma_h=w.get("sigma_h", 0.3), stout_steps=w["stout"],
                                rho=w["rho"], device=device)
    V = int(np.prod(w["L"])) * (2 if w["cstar"] else 1)
    eta = workload.spinor(V, w["src_seed"])
    return U, A, eta


# ----------------------------------------------------------------------------------
# whole-job aggregation over ranks (replicas: each rank solves its own system)
def max_over_ranks(dist, value, device):
    """The largest per-rank value (the job's time); `dist` None means one process."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value, device):
    """The sum of the per-rank values (the job's work)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t)
    return float(t.item())


def run_reference(args, w, name):
    """The oracle on the host cores: each step a bounded sample of sites."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    U, A, eta = make_inputs(w, "cpu")
    seconds = float(os.environ.get("QXD_REF_STEP_SECONDS", "5"))
    for i in range(args.warmup):
        oracle_rate(w, U, A, eta, min(seconds, 1.0), rng_seed=100 + i)
    flops, secs, nsites = 0.0, 0.0, 0
    for i in range(args.steps):
        rate, n, dt = oracle_rate(w, U, A, eta, seconds, rng_seed=i)
        flops += rate * dt * 1e9
        secs += dt
        nsites += n
    value = flops / secs / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gflop/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_desc(name, w, args, world),
        "cpu_baseline": {"value": value, "unit": "Gflop/s", "cores": 1, "kind": "oracle",
                         "sample": f"D_w at {nsites} random sites of the workload over {args.steps} steps "
                                   f"(NumPy FP64, one process)"},
        "e2e": {"value": value, "unit": "Gflop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def spectral_range(ctx, qxd, torch, dev, stream, V, n_power=40, n_inverse=5):
    """Estimates of the extreme eigenvalues of Dhat^+ Dhat through the C ABI:
    lambda_max by power iteration with the FP64 operator (a lower bound that
    converges from below), lambda_min by inverse iteration with the multi-shift
    solver at one shift sigma = 0 (the Rayleigh quotient of the last iterate, an
    upper bound converging from above).  The printed approximation assumes the
    spectrum of |Qhat| = sqrt(Dhat^+ Dhat) inside [r_a, r_b] (App. A.1, eq. normbound)."""
    ne = V // 2
    gen = torch.Generator(device=dev).manual_seed(77)
    x = torch.randn((ne, 4, 3), dtype=torch.complex128, device=dev, generator=gen)
    y = torch.empty_like(x)
    t = torch.empty_like(x)
    lam_max = 0.0
    for _ in range(n_power):
        x /= torch.linalg.vector_norm(x)
        ctx.apply_Dhat_eo(0, qxd.FP64, x, t, stream=stream)
        ctx.apply_Dhat_eo(0, qxd.FP64, t, y, dagger=True, stream=stream)
        lam_max = float(torch.vdot(x.reshape(-1), y.reshape(-1)).real)
        x, y = y, x
    x = torch.randn((ne, 4, 3), dtype=torch.complex128, device=dev, generator=gen)
    lam_min = None
    iters = 0
    for _ in range(n_inverse):
        x /= torch.linalg.vector_norm(x)
        info = ctx.solve_multishift(0, [0.0], x, y, tol=1e-10, inner=qxd.FP32, stream=stream)
        iters += info.iters
        # Rayleigh quotient of Dhat^+ Dhat at y = (Dhat^+ Dhat)^-1 x: <y, x> / <y, y>
        lam_min = float(torch.vdot(y.reshape(-1), x.reshape(-1)).real / torch.vdot(y.reshape(-1), y.reshape(-1)).real)
        x, y = y, x
    ra, rb = 1.98e-3, 7.62  # range of the printed degree-10 approximation (App. C, [Rational 0])
    return {"lambda_max_estimate": lam_max, "lambda_min_estimate": lam_min,
            "power_iterations": n_power, "inverse_iterations": n_inverse, "inverse_cg_iterations": iters,
            "printed_range_squared": [ra * ra, rb * rb],
            "inside_printed_range": bool(lam_max <= rb * rb and lam_min >= ra * ra)}


def precond_rows(ctx, qxd, torch, dev, stream, timed, eta_d, psi_d, solve_kw, V, sap=((5, 5), (3, 4))):
    """SAP(ncy,nmr)- and DFL+SAP(3,4)-preconditioned FGCR (Sec. 4.4) on the
    context's system, each timed with CUDA events (one solve after a warm-up)."""
    nxt = {}
    for ncy, nmr in sap:
        ctx.set_sap(ncy, nmr)
        ctx.solve(0, eta_d, psi_d, **(solve_kw | {"precond": qxd.PRECOND_SAP, "nkv": 16}))
        ctx.profile(2)
        ms_sap, inf_sap = timed(lambda: ctx.solve(0, eta_d, psi_d, **(solve_kw | {"precond": qxd.PRECOND_SAP,
                                                                                  "nkv": 16})), 1)
        ps = {p["name"]: p for p in ctx.profile_entries()}
        ctx.profile(0)
        blk = ps.get("sap_sweep")
        nxt[f"sap_fgcr_ncy{ncy}_nmr{nmr}"] = {
            "ms": ms_sap, "iters": inf_sap[0].iters, "true_relres": inf_sap[0].true_relres,
            "sap_sweep_ms_per_launch": blk["ms"] / blk["launches"] if blk else None,
            "sap_sweep_launches": blk["launches"] if blk else None,
            "sap_sweep_GBps": blk["bytes"] / (blk["ms"] * 1e-3) / 1e9 if blk else None}
    # inexact deflation (DFL+SAP+GCR): subspace from Ns Gaussian fields drawn on the
    # device with a seeded generator, SAP(3,4) as smoother and for the inverse iteration
    ctx.set_sap(3, 4)
    gen = torch.Generator(device=dev).manual_seed(4242)
    seeds = torch.randn((12, V, 4, 3), dtype=torch.complex64, device=dev, generator=gen)
    torch.cuda.synchronize()
    t0d = time.perf_counter()
    ctx.dfl_setup(0, seeds, 12, ninv=2, ctol=1e-2, cnmx=64, stream=stream)
    torch.cuda.synchronize()
    dfl_setup_ms = (time.perf_counter() - t0d) * 1e3
    del seeds
    dkw = solve_kw | {"precond": qxd.PRECOND_DFL, "nkv": 16}
    ms_dfl, inf_dfl = timed(lambda: ctx.solve(0, eta_d, psi_d, **dkw), 1)
    nxt["dfl_fgcr_Ns12_ninv2_sap3_4"] = {"setup_ms": dfl_setup_ms, "ms": ms_dfl, "iters": inf_dfl[0].iters,
                                          "true_relres": inf_dfl[0].true_relres}
    return nxt


def rough_row(args, qxd, torch, dev, stream, timed, fp32_kw):
    """The bench lattice and couplings on rougher synthetic fields (plaquette about
    0.63 after smearing, the value the configurations aim at): plain FP64 CGNE,
    the unpreconditioned mixed FGCR, SAP(3,4) and DFL+SAP(3,4), to 1e-10 each."""
    from paper_1908_11673_gb300 import workload
    w = WORKLOADS["32^3x64-cstar3-rough"]
    U, A, eta = make_inputs(w, str(dev))
    ctx = qxd.Context(w["L"], w["cstar"], w["theta"], device=dev.index or 0)
    ctx.set_links(U, A, w["invqel"], stream=stream)
    ctx.set_clover(0, w["qhat"], w["kappa"], w["su3csw"], w["u1csw"], stream=stream)
    V = ctx.V
    row = {"field": "H entries N(0, 0.6^2), 5 stout steps rho 0.1, seed 2100",
           "plaquette": workload.plaquette(U, w["L"])}
    del U, A
    eta_d = torch.from_numpy(eta).to(dev)
    psi_d = torch.empty_like(eta_d)
    ctx.solve(0, eta_d, psi_d, **fp32_kw)
    ms, inf = timed(lambda: ctx.solve(0, eta_d, psi_d, **fp32_kw), 1)
    row["fgcr_mixed"] = {"ms": ms, "iters": inf[0].iters, "true_relres": inf[0].true_relres}
    ms64, inf64 = timed(lambda: ctx.solve(0, eta_d, psi_d, kind=qxd.CGNE, tol=1e-10, nmx=200000, stream=stream), 1)
    row["fp64_cgne"] = {"ms": ms64, "iters": inf64[0].iters, "true_relres": inf64[0].true_relres}
    row.update(precond_rows(ctx, qxd, torch, dev, stream, timed, eta_d, psi_d, fp32_kw, V, sap=((3, 4),)))
    del eta_d, psi_d
    ctx.close()
    return row


def learned_row(ctx, qxd, torch, dev, stream, timed, w, V, fp64_cgne_ms):
    """The mixed-precision, batched, learned-preconditioned solve on the bench
    system: the network (4 layers x 8 channels) is trained on four 16 x 8^3 lattices
    with the bench system's couplings, boundary conditions and smearing (the
    network is local and gauge covariant, so its weights carry over to the large
    lattice), then FGCR(16) with FP32 inner solves and the network as right
    preconditioner solves 4 right-hand sides in lockstep (one multi-right-hand-side
    operator launch per iteration) to the true FP64 residual 1e-10; beside it the
    same batch without the network, and the plain FP64 CGNE time per right-hand side."""
    from paper_1908_11673_gb300 import learned
    field = dict(L=(16, 8, 8, 8), cstar=w["cstar"], theta=w["theta"], qhat=w["qhat"], kappa=w["kappa"],
                 su3csw=w["su3csw"], u1csw=w["u1csw"], invqel=w["invqel"], stout=w["stout"], rho=w["rho"],
                 sigma_h=w.get("sigma_h", 0.3))
    nl, nch, nrhs = 4, 8, 4
    W, summ = learned.train(field, [7000 + i for i in range(4)], 50, epochs=4, batch=10, nlayers=nl, nch=nch,
                            device=dev.index or 0)
    ctx.set_precond_weights(0, W, nl, nch)
    gen = torch.Generator(device=dev).manual_seed(2002)
    eta = torch.randn((nrhs, V, 4, 3), dtype=torch.complex128, device=dev, generator=gen)
    psi = torch.empty_like(eta)
    row = {"training": {k: v for k, v in summ.items() if k != "loss_history"}, "nrhs": nrhs}
    for name, pre in (("learned", qxd.PRECOND_LEARNED), ("none", qxd.PRECOND_NONE)):
        kw = dict(kind=qxd.FGCR, tol=1e-10, inner=qxd.FP32, nkv=16, precond=pre, nrhs=nrhs, nmx=100000,
                  stream=stream)
        ms, inf = timed(lambda: ctx.solve(0, eta, psi, **kw), 1)
        chk = torch.empty_like(psi)
        ctx.apply_Dw(0, qxd.FP64, psi, chk, nrhs=nrhs, stream=stream)
        rel = [float(torch.linalg.vector_norm(eta[j] - chk[j]) / torch.linalg.vector_norm(eta[j]))
               for j in range(nrhs)]
        del chk
        row[name] = {"ms": ms, "ms_per_rhs": ms / nrhs, "iters": inf[0].iters, "true_relres": inf[0].true_relres,
                     "fp64_check_worst": max(rel), "status": inf[0].status}
    if fp64_cgne_ms:
        row["fp64_cgne_ms_per_rhs"] = fp64_cgne_ms
        row["speedup_learned_vs_fp64_cgne"] = fp64_cgne_ms / row["learned"]["ms_per_rhs"]
    del eta, psi
    return row


def batched_row(qxd, torch, dev, stream, timed):
    """24^3 x 48 (V = 663,552, antiperiodic time, 5 stout steps, qhat = -2,
    kappa = 0.136377): the FP32 multi-right-hand-side D_w at nrhs = 1, 4, 12
    (algorithmic bytes per output site per right-hand side and GB/s of the hop
    launches, CUDA events around each launch) and the ten-shift multi-shift CG of
    the printed degree-10 approximation (FP32 Krylov space, FP64 refinement)."""
    w = WORKLOADS["24^3x48"]
    U, A, _ = make_inputs(w, str(dev))
    ctx = qxd.Context(w["L"], w["cstar"], w["theta"], device=dev.index or 0)
    ctx.set_links(U, A, w["invqel"], stream=stream)
    ctx.set_clover(0, w["qhat"], w["kappa"], w["su3csw"], w["u1csw"], stream=stream)
    del U, A
    V = ctx.V
    peak, _ = measured_peaks()
    row = {"lattice": "24^3x48", "V": V, "mrhs": []}
    gen = torch.Generator(device=dev).manual_seed(3)
    for nrhs in (1, 4, 12):
        x = torch.randn((nrhs, V, 4, 3), dtype=torch.complex64, device=dev, generator=gen)
        y = torch.empty_like(x)
        ctx.apply_Dw(0, qxd.FP32, x, y, nrhs=nrhs, stream=stream)  # tunes the launch shape
        torch.cuda.synchronize()
        ctx.profile(2)
        for _ in range(10):
            ctx.apply_Dw(0, qxd.FP32, x, y, nrhs=nrhs, stream=stream)
        hops = [p for p in ctx.profile_entries() if p["name"].startswith("hop_")]
        ctx.profile(0)
        ms = sum(p["ms"] for p in hops)
        by = sum(p["bytes"] for p in hops)
        n = sum(p["launches"] for p in hops)
        row["mrhs"].append({"nrhs": nrhs, "hop_launches": n, "ms_per_Dw": 2 * ms / n,
                            "bytes_per_site_per_rhs": by / n / (V // 2) / nrhs,
                            "GBps": by / (ms * 1e-3) / 1e9, "frac_of_hbm": by / (ms * 1e-3) / 1e9 / peak,
                            "Gflops": n * (V // 2) * nrhs * FLOP_PER_SITE / (ms * 1e-3) / 1e9})
        del x, y
    A_r, nu_r, mu_r = read_rational(GOLDEN_RATIONAL)
    sigma = list(mu_r ** 2)
    phi = torch.randn((V // 2, 4, 3), dtype=torch.complex128, device=dev, generator=gen)
    xs = torch.empty((len(sigma), V // 2, 4, 3), dtype=torch.complex128, device=dev)
    ctx.solve_multishift(0, sigma, phi, xs, tol=1e-10, inner=qxd.FP32, stream=stream)
    ms_ms, inf = timed(lambda: ctx.solve_multishift(0, sigma, phi, xs, tol=1e-10, inner=qxd.FP32, stream=stream), 1)
    row["mscg_10_shifts"] = {"ms": ms_ms, "cg_iters": inf[0].iters, "worst_shift_relres": inf[0].true_relres}
    del phi, xs
    ctx.close()
    return row


def run_native(args, w, name):
    import torch

    from paper_1908_11673_gb300 import build, qxd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    U, A, eta = make_inputs(w, f"cuda:{local}")
    ctx = qxd.Context(w["L"], w["cstar"], w["theta"], device=local)
    t0 = time.perf_counter()
    ctx.set_links(U, A, w["invqel"], stream=stream)
    ctx.set_clover(0, w["qhat"], w["kappa"], w["su3csw"], w["u1csw"], stream=stream)
    setup_s = time.perf_counter() - t0
    V = ctx.V
    eta_d = torch.from_numpy(eta).to(dev)
    psi_d = torch.empty_like(eta_d)
    inner = {"fp32": qxd.FP32, "bf16": qxd.BF16}[args.inner]
    solve_kw = dict(kind=qxd.FGCR, tol=1e-10, inner=inner, nkv=args.nkv, nmx=args.nmx, stream=stream,
                    check=args.nmx >= 100000)

    for _ in range(args.warmup):
        ctx.solve(0, eta_d, psi_d, **solve_kw)
    torch.cuda.synchronize()

    def timed(fn, k):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = [fn() for _ in range(k)]
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = max_over_ranks(dist, e0.elapsed_time(e1), dev)
        return ms, infos

    def timed_local(fn, k):
        """timed() without the barriers, for work that rank 0 does alone"""
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = [fn() for _ in range(k)]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), infos

    # ---- timed region: K mixed-precision solves; launches counted, not timed --------
    sampler = ClockSampler(local)
    sampler.start()
    ctx.profile(1)
    ms, infos = timed(lambda: ctx.solve(0, eta_d, psi_d, **solve_kw), args.steps)
    counts = ctx.profile_entries()
    ctx.profile(0)
    clocks = sampler.stop()
    hop_launches = sum(p["launches"] for p in counts if p["name"].startswith("hop_"))
    flops = hop_launches * (V // 2) * FLOP_PER_SITE
    launches = sum(p["launches"] for p in counts)

    # the mixed solver's outer residual runs in double-float: check the last timed
    # solution with the FP64 operator before any other solve overwrites it
    dpsi = torch.empty_like(psi_d)
    ctx.apply_Dw(0, qxd.FP64, psi_d, dpsi, stream=stream)
    torch.cuda.synchronize()
    rel64 = float(torch.linalg.vector_norm(eta_d - dpsi) / torch.linalg.vector_norm(eta_d))
    del dpsi

    # ---- kernel table: the same K solves again, every launch bracketed by CUDA events
    # recorded on its stream (a second pass, so that the events cost nothing above) ----
    ctx.profile(2)
    ms_prof, infos_prof = timed(lambda: ctx.solve(0, eta_d, psi_d, **solve_kw), args.steps)
    prof = ctx.profile_entries()
    ctx.profile(0)
    total_ms_k = sum(p["ms"] for p in prof)

    # ---- e2e: pinned host buffers through the C ABI ----------------------------------
    eta_h = torch.from_numpy(eta).pin_memory()
    psi_h = torch.empty_like(eta_h).pin_memory()
    ctx.solve(0, eta_h, psi_h, **solve_kw)  # warm-up: the library's staging buffers are allocated here
    k_e2e = max(1, min(args.steps, 3))
    ms_e2e, infos_e2e = timed(lambda: ctx.solve(0, eta_h, psi_h, **solve_kw), k_e2e)
    e2e_value = flops / args.steps * k_e2e / (ms_e2e * 1e-3) / 1e9

    # ---- plain FP64 CGNE on the same system ---------------------------------------------
    base = None
    if not args.no_fp64_baseline:
        ms64, inf64 = timed(lambda: ctx.solve(0, eta_d, psi_d, kind=qxd.CGNE, tol=1e-10, nmx=200000,
                                              stream=stream), 1)
        base = {"fp64_cgne_ms": ms64, "fp64_cgne_iters": inf64[0].iters,
                "fp64_cgne_true_relres": inf64[0].true_relres}

    # ---- next rows of the method on the same system (not part of the timed step) --------
    nxt = None
    spec = None
    if not args.no_extras:
        spec = spectral_range(ctx, qxd, torch, dev, stream, V)
        nxt = {}
        nxt.update(precond_rows(ctx, qxd, torch, dev, stream, timed, eta_d, psi_d, solve_kw, V))
        A_r, nu_r, mu_r = read_rational(GOLDEN_RATIONAL)
        rat = qxd.rational(A_r, nu_r, mu_r)
        phi_e = torch.from_numpy(np.ascontiguousarray(eta[: V // 2])).to(dev)
        ctx.pf_action(0, rat, 0, 9, phi_e, tol=1e-10, stream=stream)
        ms_pf, _ = timed(lambda: ctx.pf_action(0, rat, 0, 9, phi_e, tol=1e-10, stream=stream), 1)
        S_pf, inf_pf = ctx.pf_action(0, rat, 0, 9, phi_e, tol=1e-10, stream=stream)
        nxt["pf_action_deg10"] = {"ms": ms_pf, "S_over_phi2": S_pf / float(np.vdot(eta[: V // 2], eta[: V // 2]).real),
                                  "cg_iters": inf_pf.iters, "worst_shift_relres": inf_pf.true_relres}
        ctx.sdet(0, stream=stream)
        ms_sd, _ = timed(lambda: ctx.sdet(0, stream=stream), 3)
        nxt["sdet"] = {"ms": ms_sd / 3, "logdet_per_odd_site": ctx.sdet(0, stream=stream)[0] / (V // 2)}
        del phi_e
        nxt["learned_batched_mixed"] = learned_row(ctx, qxd, torch, dev, stream, timed, w, V,
                                                   base["fp64_cgne_ms"] if base else None)

    # ---- aggregate over ranks ----------------------------------------------------------
    total_value = sum_over_ranks(dist, flops, dev) / (ms * 1e-3) / 1e9
    if rank != 0:
        ctx.close()
        dist.destroy_process_group()
        return 0
    if not args.no_extras:
        # the batched configuration on its own lattice (rank 0 only, after the others are done)
        ctx.close()
        ctx = None
        del eta_d, psi_d
        torch.cuda.empty_cache()
        nxt["batched_24x24x24x48"] = batched_row(qxd, torch, dev, stream, timed_local)
        try:
            nxt["rough_fields_32x32x32x64_cstar3"] = rough_row(args, qxd, torch, dev, stream, timed_local, solve_kw)
        except qxd.QxdError as e:  # a solve that misses 1e-10 within nmx is reported, not fatal
            nxt["rough_fields_32x32x32x64_cstar3"] = {"error": str(e)}

    peak, peak_kind = measured_peaks()
    dom = max(prof, key=lambda p: p["ms"])
    mean_ms = dom["ms"] / dom["launches"]
    bytes_per_launch = dom["bytes"] / dom["launches"]
    timing = f"CUDA events around every launch on its stream, in a second pass of the same {args.steps} solves"
    if dom["name"].startswith("hop_fp64"):
        # the FP64 hopping kernel is bound by the FP64 pipe (1/64 of the FP32 rate on
        # this GPU), not by HBM: 2112 flop per output site against the FP64 FMA peak
        flops_per_launch = (V // 2) * FLOP_PER_SITE * (dom["bytes"] / dom["launches"]) / hop_bytes_per_launch(dom, V)
        achieved = flops_per_launch / (mean_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": dom["name"], "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "peak_kind": "measured FP64 FMA rate of this GPU (2 flop per DFMA)",
                    "flops_per_launch": flops_per_launch, "mean_launch_ms": mean_ms,
                    "hbm_GBps": bytes_per_launch / (mean_ms * 1e-3) / 1e9, "traffic": None, "timing": timing}
    else:
        achieved = bytes_per_launch / (mean_ms * 1e-3) / 1e9
        per_site = NCU_BYTES_PER_SITE.get(dom["name"])
        ratio = NCU_TRAFFIC_RATIO.get(dom["name"])
        if per_site:
            traffic, source = per_site * (V // 2), "ncu dram bytes per site on 24^3x48 scaled to this lattice"
        elif ratio:
            traffic = ratio * bytes_per_launch
            source = "ncu dram bytes / algorithmic bytes on 24^3x48 times this launch's mean algorithmic bytes"
        else:
            traffic, source = None, None
        roofline = {"bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_kind": f"{peak_kind} (HBM copy bandwidth)",
                    "bytes_per_launch": bytes_per_launch, "mean_launch_ms": mean_ms,
                    "traffic": traffic, "traffic_source": source, "timing": timing}
    kernels = []
    for p in sorted(prof, key=lambda p: -p["ms"]):
        gbs = p["bytes"] / (p["ms"] * 1e-3) / 1e9 if p["ms"] > 0 else None
        kernels.append({"name": p["name"], "launches": p["launches"], "ms": round(p["ms"], 3),
                        "share": round(p["ms"] / total_ms_k, 4) if total_ms_k else None,
                        "GB/s": round(gbs, 1) if gbs else None})
    info = infos[-1]
    tts = {"mixed_ms": ms / args.steps, "iters_inner": info.iters, "outer_restarts": info.restarts,
           "true_relres": info.true_relres, "true_relres_fp64_check": rel64, "status": info.status,
           "profiled_pass_ms": ms_prof / args.steps, "profiled_pass_iters": infos_prof[-1].iters}
    if base:
        tts.update(base)
        tts["speedup_vs_fp64_cgne"] = base["fp64_cgne_ms"] / (ms / args.steps)

    cpu = None
    if not args.no_cpu_baseline:
        sec = float(os.environ.get("QXD_CPU_SECONDS", "10"))
        rate, n, dt = oracle_rate(w, U, A, eta, sec)
        rate_all, cores, n_all, dt_all = oracle_rate_all_cores(w, U, A, eta, sec, rate)
        cpu = {"value": rate_all, "unit": "Gflop/s", "cores": cores, "kind": "oracle",
               "sample": f"D_w at {n_all} random sites of the workload, one spawned NumPy FP64 process per "
                         f"core ({dt_all:.1f} s wall)",
               "single_core": {"value": rate, "cores": 1,
                               "sample": f"D_w at {n} random sites ({dt:.1f} s, one process)"}}

    line = {
        "metric": METRIC, "value": total_value, "unit": "Gflop/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.inner == "fp32" else "bf16+f32+f64", "data": "synthetic",
        "config": workload_desc(name, w, args, world),
        "time_to_solution": tts,
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "Gflop/s", "h2d_bytes_per_step": int(eta.nbytes),
                "d2h_bytes_per_step": int(eta.nbytes), "ms_per_step": ms_e2e / k_e2e},
        "gpu_launches": launches,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "setup_s": setup_s,
        "spectral_range": spec,
        "next_rows": nxt,
        "kernels": kernels,
    }
    print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="32^3x64-cstar3")
    ap.add_argument("--no-fp64-baseline", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the SAP and rational-function measurements")
    ap.add_argument("--nmx", type=int, default=100000,
                    help="operator applications per solve; below 100000 a solve that stops early is reported, "
                         "not raised (profiler captures)")
    ap.add_argument("--nkv", type=int, default=8, help="GCR restart length (8: fastest of 8, 16, 32 here)")
    ap.add_argument("--inner", choices=["fp32", "bf16"], default="fp32",
                    help="storage of the inner solve's Krylov basis and operator (residual FP32 either way)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w, args.workload)
    return run_native(args, w, args.workload)


if __name__ == "__main__":
    sys.exit(main())
