#!/usr/bin/env python3
"""Benchmark: 12-RHS Wilson-clover propagator solve to a 1e-10 true residual.

Workload (one "step"): lattice 32^3x64, links exp(i 0.3 sum_a r_a lambda_a/2)
(seed 0), kappa 0.1235, c_sw 1.0, antiperiodic time; the 12 spin-colour point
sources at site 0; one wcl_invert call (even-odd BiCGStab, FP32 inner solver,
reliable updates at delta = 3e-4 checked every 2 iterations, double-float
intermediate and FP64 final residual replacements, true residual and solution
accumulation in FP64; --sloppy f16/bf16 streams 16-bit fields with per-site norms) -- source preparation, solve, odd-site
reconstruction and the FP64 true residual included.  Inputs are resident in
HBM when the timed region starts; the solve working set (tens of GB) is far
larger than L2.

Printed JSON line: value = 12-RHS solves per second over all ranks (solves
replayed as CUDA graphs, no per-launch events); roofline = the inner-precision
12-RHS fused dslash (the dominant kernel), from CUDA events around each launch
on the library's stream during one extra, profiled solve; fp64_dslash = the
FP64 launches of that solve against the FP64 ALU rate;
e2e = the same solve through the C ABI with b and x in pinned host memory (the
library's import/export kernels move them over the host link, timed);
cpu_baseline = the FP64 oracle on the host cores, on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (32, 32, 32, 64)
EPS, SEED, KAPPA, CSW, TOL = 0.3, 0, 0.1235, 1.0, 1e-10
METRIC = "clover dslash GB/s & roofline %; 12-RHS solve time to 1e-10 true residual"
PREC_INDEX = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3, "df64": 4}
FP64_PEAK_GFLOPS = 1250.0  # GB300 FP64 vector rate, nominal
# DRAM bytes (read + written) per site and right-hand side of the 12-RHS FP32 fused dslash,
# averaged over the solve's launch mix (2 x A^-1 D x, 1 x alpha-fused, 1 x omega-fused), from
# one ncu capture of 8 such launches of the same solve on 32^3x16 -- the bench lattice's
# spatial volume, so the t neighbours lie as far apart as at 32^3x64, with a few GB on the
# device: 998/1145/967/1455 MB per launch for 3.15 M site-RHS, 362.8 B against 320 algorithmic
TRAFFIC_F32_12RHS_PER_SITE_RHS = 362.8
UNIT = "12-RHS solves/s"
WORKLOAD = "32^3x64 Wilson-clover, eps 0.3, kappa 0.1235, c_sw 1.0, 12 spin-colour point sources, tol 1e-10"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sloppy", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--delta", type=float, default=3e-4, help="reliable-update threshold")
    ap.add_argument("--check-every", type=int, default=2, help="iterations per graph replay / convergence check")
    ap.add_argument("--sloppy-updates", type=int, default=0,
                    help="16-bit inner solvers: updates above 10^-k ||b|| with the FP32 operator (0: off)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pairs", type=int, default=2000, help="training pairs of --case compare")
    ap.add_argument("--epochs", type=int, default=4, help="training epochs of --case compare")
    ap.add_argument("--case", default="solve",
                    choices=["solve", "mhat", "compare", "batch", "throughput", "precond", "propagator", "mg",
                             "staggered", "force"],
                    help="mhat: only apply the Schur operator (the small case used for ncu captures); "
                         "batch: four uneven lattices x 12 Z2 sources in one batched solve vs single-RHS "
                         "solves; throughput: 16^3x32 FP32 operator applies and one point-source solve; "
                         "propagator: the Sec. III.B sequence (wall propagators, sequential propagator, "
                         "two- and three-point functions) on --dims, with the contraction kernel's roofline; "
                         "mg: the two-level multigrid (setup, then FGCR-MG on the 12 point sources) against "
                         "the batched BiCGStab solve on --dims at --kappa; staggered: the HISQ-form staggered "
                         "operator on --dims (FP64 and FP32 applies, GB/s) and its even-odd CG solve; force: "
                         "the FP64 clover fermion force (HMC) on --dims")
    ap.add_argument("--tol", type=float, default=1e-10, help="solver tolerance of --case propagator / mg")
    ap.add_argument("--kappa", type=float, default=KAPPA, help="hopping parameter of --case mg")
    ap.add_argument("--mg-block", default="4,4,4,4", help="--case mg: block size per direction")
    ap.add_argument("--mg-nvec", type=int, default=24, help="--case mg: null vectors")
    ap.add_argument("--mg-nkrylov", type=int, default=20, help="--case mg: restart length of the outer FGCR")
    ap.add_argument("--mg-smooth", default="2,2", help="--case mg: pre,post minimal-residual steps of the K-cycle")
    ap.add_argument("--mg-coarse-steps", type=int, default=8,
                    help="--case mg: coarse GCR steps of the batched K-cycle (solver fgcr_mg_batched)")
    ap.add_argument("--mg-single", type=int, default=1,
                    help="--case mg: also time the one-right-hand-side-at-a-time multigrid FGCR")
    ap.add_argument("--lattice", default="24,24,24,48", help="lattice of --case mhat")
    ap.add_argument("--dims", default="32,32,32,64", help="lattice of --case solve (the bench line uses 32^3x64)")
    ap.add_argument("--nrhs", type=int, default=12, help="right-hand sides of --case mhat")
    ap.add_argument("--prec", default="f32", choices=["f64", "df64", "f32", "f16", "bf16"], help="precision of --case mhat")
    ap.add_argument("--tensor-cores", type=int, default=0, help="--case mhat: 16-bit multi-RHS kernel on tensor cores")
    ap.add_argument("--shared-links", type=int, default=1,
                    help="--case mhat: multi-RHS kernel with links and clover staged in shared memory (tile)")
    ap.add_argument("--staged-spinors", type=int, default=0,
                    help="--case mhat: multi-RHS kernel with cp.async-staged neighbour spinors (tuner off)")
    ap.add_argument("--autotune", type=int, default=1, help="--case mhat: dslash autotuner on/off")
    ap.add_argument("--paired-rhs", type=int, default=0,
                    help="--case mhat: packed-pair multi-RHS kernel (two RHS per thread, FFMA2) when the tuner is off")
    ap.add_argument("--blocked-tiles", type=int, default=0, help="--case mhat: z-blocked tile order (tuner off)")
    ap.add_argument("--tma-staging", type=int, default=0,
                    help="--case mhat: TMA-staged kernel, 1 persistent / 2 one CTA per tile (tuner off)")
    ap.add_argument("--prefetch-spinors", type=int, default=0,
                    help="--case mhat: next hop's spinor prefetched in registers (tuner off)")
    return ap.parse_args()


def dist_init(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        import torch

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(max_ms, world):
    """Whole-job solves per second: every rank finished one solve per step, timed by
    the slowest rank."""
    return world * 1e3 / max_ms


def replica_seed(rank):
    """Replicas only: every rank solves its own gauge field, seeded by its rank."""
    return SEED + rank


class Clocks:
    """nvidia-smi sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_baseline_sample(gpu_iters_per_rhs: float, budget_s: float = 20.0):
    """Time the FP64 oracle's Schur BiCGStab iterations on 16^3x32 (same recipe) and
    scale by volume (x16), by the GPU solve's iterations per RHS and by 12 RHS."""
    import numpy as np

    import workloads as W
    from oracle import dirac, solvers
    from oracle import lattice as L

    dims = (16, 16, 16, 32)
    gauge = W.gauge_links(dims, EPS, SEED)
    op = dirac.from_qdp_problem(gauge, dims, KAPPA, CSW)
    b = L.from_qdp(W.point_source(dims, 0, 0), dims)
    bhat = op.schur_source(b)
    n = 1
    t0 = time.perf_counter()
    while True:
        solvers.bicgstab(op.Mhat, bhat, tol=0.0, maxiter=n)
        el = time.perf_counter() - t0
        if el > budget_s * 0.25 or n >= 8:
            break
        n *= 2
    t0 = time.perf_counter()
    solvers.bicgstab(op.Mhat, bhat, tol=0.0, maxiter=n)
    per_iter = (time.perf_counter() - t0) / n
    scale = (DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3]) / (dims[0] * dims[1] * dims[2] * dims[3])
    est = per_iter * scale * gpu_iters_per_rhs * 12
    cores = 1  # numpy elementwise and einsum kernels run on one thread
    try:
        affinity = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        affinity = None
    threads = ", ".join(f"{k}={os.environ.get(k, 'unset')}" for k in
                        ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"))
    return {"value": 1.0 / est, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} BiCGStab iterations of the FP64 oracle on 16^3x32 (same links/kappa/c_sw), "
                      f"{per_iter:.2f} s/iteration, scaled x{scale:.0f} by volume, x{gpu_iters_per_rhs:.0f} "
                      f"iterations/RHS (the GPU solve's count) and x12 RHS; host has {os.cpu_count()} cores, "
                      f"{affinity} in this process's affinity mask, {threads}; numpy's elementwise "
                      f"kernels are single-threaded"}


def oracle_true_residuals(gauge, x, b, dims):
    """||b - M x|| / ||b|| per right-hand side by the FP64 oracle over the whole lattice,
    slab by slab in a pool of spawned processes (one per host core, at most 16)."""
    import numpy as np

    from oracle import residual

    procs = min(16, os.cpu_count() or 1)
    t0 = time.perf_counter()
    r = residual.true_residuals(gauge, x, b, dims, KAPPA, CSW, t_boundary=-1, processes=procs)
    sec = time.perf_counter() - t0
    return {"worst": float(np.max(r)), "per_rhs": [float(v) for v in r], "seconds": sec, "processes": procs,
            "seconds_per_rhs": sec / len(r),
            "what": f"FP64 oracle: M x on the whole {'x'.join(map(str, dims))} lattice for each of the "
                    f"{len(r)} solutions (4-timeslice slabs with one halo timeslice each side, clover built "
                    f"per slab), ||b - M x|| / ||b||"}


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is one bounded sample (oracle
    BiCGStab iterations on 16^3x32, scaled to a 12-RHS 32^3x64 solve)."""
    if rank != 0:
        return 0
    # BiCGStab iterations per RHS on this workload: the GPU solve's measured count (47-51)
    iters_per_rhs = float(os.environ.get("WCL_REF_ITERS", "48"))
    vals = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline_sample(iters_per_rhs, budget_s=8.0)
        if k >= args.warmup:
            vals.append(r)
    v = statistics.median([r["value"] for r in vals])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle sample)", "parallelism": "host cores"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[-1]["cores"], "kind": "oracle",
                             "sample": vals[-1]["sample"] + f"; assumed {iters_per_rhs:.0f} iterations/RHS"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    import paper_2411_08461_gb300 as pkg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    seed = replica_seed(rank)
    dims = tuple(int(v) for v in args.dims.split(","))
    gauge = W.gauge_links(dims, EPS, seed)
    src = np.stack([W.point_source(dims, s, c) for s in range(4) for c in range(3)])
    ctx = pkg.Context(dims, t_boundary=-1, device=local, stream=stream)
    ctx.wcl_load_gauge(torch.from_numpy(gauge).to(dev), KAPPA, CSW)
    b = torch.from_numpy(src).to(dev)
    x = torch.zeros_like(b)
    prm = pkg.wcl_default_params(solver="bicgstab", sloppy=args.sloppy, tol=TOL, check_every=args.check_every,
                                 delta_reliable=args.delta)
    if args.sloppy_updates:
        from paper_2411_08461_gb300.wcl import WCL_OPT_SLOPPY_UPDATES
        ctx.wcl_set_option(WCL_OPT_SLOPPY_UPDATES, args.sloppy_updates)

    infos = None
    for _ in range(args.warmup):
        _, infos = ctx.wcl_invert(x, b, 12, prm)
    # timed solves: graphs on, no per-launch events
    ctx.wcl_get_stats(reset=True)
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, infos = ctx.wcl_invert(x, b, 12, prm)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world)
    launches = ctx.wcl_get_stats(reset=True)["kernel_launches"]
    worst = max(i["true_residual"] for i in infos)
    assert worst <= TOL and all(i["status"] == 0 for i in infos), infos
    iters = statistics.mean(i["iters"] for i in infos)

    # the comparison method on the same GPU and workload: plain FP32 single-RHS BiCGStab,
    # twelve sequential solves restarted from the IEEE FP64 true residual (pure FP32 stalls
    # near 1e-7), timed with CUDA events like the batched solve
    plain = pkg.wcl_default_params(sloppy="f32", outer="f64", tol=TOL, restart_on_update=1, delta_reliable=1e-5)
    xp = torch.zeros_like(b)
    ctx.wcl_invert(xp[:1], b[:1], 1, plain)  # warm-up of the single-RHS configurations
    p_runs, p_infos = [], []
    for _ in range(max(1, min(args.steps, 2))):
        barrier(world)
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        p_infos = [ctx.wcl_invert(xp[k:k + 1], b[k:k + 1], 1, plain)[1][0] for k in range(12)]
        q1.record(stream)
        torch.cuda.synchronize()
        p_runs.append(q0.elapsed_time(q1))
    plain_ms = max_over_ranks(statistics.median(p_runs), world)
    assert all(i["status"] == 0 and i["true_residual"] <= TOL for i in p_infos), p_infos
    del xp

    # one more solve with every dslash launch timed by events (direct launches, no graphs)
    ctx.wcl_set_profiling(True)
    ctx.wcl_get_stats(reset=True)
    _, pinfos = ctx.wcl_invert(x, b, 12, prm)
    torch.cuda.synchronize()
    st = ctx.wcl_get_stats(reset=True)
    ctx.wcl_set_profiling(False)

    # end to end: b and x in pinned host memory, passed to wcl_invert as they are;
    # the library's import kernel reads b and its export kernel writes x over the
    # host link inside the timed region
    bh = torch.from_numpy(src).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    barrier(world)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        ctx.wcl_invert(xh, bh, 12, prm)
    t1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, world)
    e2e_ok = float(np.abs(xh.numpy() - x.cpu().numpy()).max()) == 0.0

    # FP32 fused dslash alone at 32^3x64 (two launches per M_hat), for the roofline target
    ctx.wcl_set_profiling(True)
    ctx.wcl_get_stats(reset=True)
    pin = torch.from_numpy(W.gaussian_fermion(dims, 1)[0]).to(dev)
    pout = torch.empty_like(pin)
    for _ in range(10):
        ctx.wcl_apply_Mpc(pout, pin, "f32")
    f32 = ctx.wcl_get_stats(reset=True)
    ctx.wcl_set_profiling(False)

    # FP64 12-RHS operator alone (every RHS active), for its ALU roofline
    ctx.wcl_set_profiling(True)
    pin12 = torch.zeros((12,) + tuple(pin.shape), dtype=pin.dtype, device=dev)
    pin12[:] = pin
    pout12 = torch.empty_like(pin12)
    ctx.wcl_apply_Mpc(pout12, pin12, "f64", nrhs=12)
    ctx.wcl_get_stats(reset=True)
    ctx.wcl_apply_Mpc(pout12, pin12, "f64", nrhs=12)
    f64 = ctx.wcl_get_stats(reset=True)
    ctx.wcl_set_profiling(False)
    del pin12, pout12

    peak, peak_kind = measured_peaks()
    sp = PREC_INDEX[args.sloppy]
    s_ms, s_n, s_bytes, s_flops = st["prec_ms"][sp], st["prec_timed"][sp], st["prec_bytes"][sp], st["prec_flops"][sp]
    gbs = s_bytes / (s_ms * 1e-3) / 1e9 if s_ms > 0 else None
    d_ms, d_n = st["prec_ms"][0], st["prec_timed"][0]
    df_ms, df_n = st["prec_ms"][4], st["prec_timed"][4]
    f64_gflops = f64["dslash_flops"] / (f64["dslash_ms"] * 1e-3) / 1e9 if f64["dslash_ms"] > 0 else None
    f32_gbs = f32["dslash_bytes"] / (f32["dslash_ms"] * 1e-3) / 1e9 if f32["dslash_ms"] > 0 else None
    # DRAM bytes per launch of the dominant kernel: the per-(site, RHS) traffic measured on
    # the small case (same kernel variant, same launch mix) times the units of one launch
    # here (sites per parity x 12); only for the FP32 inner solver it was measured for
    units = dims[0] * dims[1] * dims[2] * dims[3] // 2 * 12
    traffic = TRAFFIC_F32_12RHS_PER_SITE_RHS * units if args.sloppy == "f32" else None
    value = replicas_value(ms, world)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"{args.sloppy} storage / f32 arithmetic / f64 residual", "data": "synthetic",
        "config": {"workload": WORKLOAD if dims == DIMS else WORKLOAD.replace("32^3x64", "x".join(map(str, dims))),
                   "lattice": "x".join(map(str, dims)), "nrhs": 12, "solver": "bicgstab even-odd",
                   "sloppy": args.sloppy, "delta_reliable": args.delta, "sloppy_updates": args.sloppy_updates,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "working set >> L2 (no flush needed)"},
        "solve": {"seconds": ms / 1e3, "iters_per_rhs": iters, "worst_true_residual": worst,
                  "reliable_updates": statistics.mean(i["reliable_updates"] for i in infos)},
        "plain_f32_single_rhs": {"seconds": plain_ms / 1e3, "runs": len(p_runs),
                                 "iters_per_rhs": statistics.mean(i["iters"] for i in p_infos),
                                 "worst_true_residual": max(i["true_residual"] for i in p_infos),
                                 "speedup_of_this_solve": plain_ms / ms,
                                 "method": "12 sequential wcl_invert calls with nrhs 1: FP32 BiCGStab restarted "
                                           "from the IEEE FP64 true residual at each 1e-5 reduction, same GPU, "
                                           "same workload, CUDA events"},
        "roofline": {"bound": "hbm", "kernel": f"{args.sloppy} 12-RHS fused dslash+clover (inner solver, tuned variant)",
                     "achieved": gbs, "peak": peak, "unit": "GB/s",
                     "frac": (gbs / peak) if gbs else None, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": s_bytes / max(1, s_n), "launches_timed": s_n,
                     "avg_launch_ms": s_ms / max(1, s_n),
                     "traffic": traffic,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of 8 launches of this "
                                       "kernel in the same solve on 32^3x16 (362.8 B per site-RHS against 320 "
                                       "algorithmic, 1.13x), scaled by the site-RHS of one launch here",
                     "gflops": s_flops / (s_ms * 1e-3) / 1e9 if s_ms > 0 else None,
                     "share_of_profiled_solve": s_ms / max(1e-9, pinfos[0]["seconds"] * 1e3)},
        "fp64_dslash": {"bound": "alu", "kernel": "FP64 12-RHS fused dslash (final residual replacements)",
                        "gflops": f64_gflops, "peak_gflops": FP64_PEAK_GFLOPS, "peak_kind": "nominal",
                        "frac": (f64_gflops / FP64_PEAK_GFLOPS) if f64_gflops else None,
                        "rate_measured_on": "M_hat, 12 RHS all active, 2 launches",
                        "launches_in_profiled_solve": d_n, "ms_in_profiled_solve": d_ms,
                        "double_float_launches_in_profiled_solve": df_n, "double_float_ms_in_profiled_solve": df_ms},
        "dslash_f32": {"achieved": f32_gbs, "frac": (f32_gbs / peak) if f32_gbs else None, "unit": "GB/s",
                       "launches": f32["dslash_timed"],
                       "config": "x".join(map(str, dims)) + ", 1 RHS, M_hat (864 + 960 B/site)"},
        "clocks": clk,
        "e2e": {"value": world * 1e3 / e2e_ms, "unit": UNIT, "h2d_bytes_per_step": bh.numel() * 16,
                "d2h_bytes_per_step": xh.numel() * 16, "ms_per_step": e2e_ms, "copied_back_matches": e2e_ok},
        "gpu_launches": launches,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(iters)
        # the oracle's own FP64 true residual of every right-hand side of the benchmark's
        # solve, over the whole lattice (slab by slab, spawned processes), and its time
        rec = oracle_true_residuals(gauge, x.cpu().numpy(), src, dims)
        line["cpu_baseline"]["true_residual_recompute"] = rec
        line["solve"]["worst_true_residual_oracle"] = rec["worst"]
    del gauge
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_mhat_case(args):
    """Apply M_hat a few times on one lattice: the small case for kernel captures.
    Prints the dslash GB/s measured with CUDA events around each launch."""
    import torch

    import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    import paper_2411_08461_gb300 as pkg

    dims = tuple(int(v) for v in args.lattice.split(","))
    ctx = pkg.Context(dims)
    ctx.wcl_set_option(pkg.wcl.WCL_OPT_TENSOR_CORES, args.tensor_cores)
    ctx.wcl_set_option(pkg.wcl.WCL_OPT_SHARED_LINKS, args.shared_links)
    ctx.wcl_set_option(pkg.wcl.WCL_OPT_STAGED_SPINORS, args.staged_spinors)
    ctx.wcl_set_option(pkg.wcl.WCL_OPT_AUTOTUNE, args.autotune)
    ctx.wcl_set_option(pkg.wcl.WCL_OPT_PAIRED_RHS, args.paired_rhs)
    ctx.wcl_set_option(pkg.wcl.WCL_OPT_BLOCKED_TILES, args.blocked_tiles)
    ctx.wcl_set_option(pkg.wcl.WCL_OPT_TMA_STAGING, args.tma_staging)
    ctx.wcl_set_option(pkg.wcl.WCL_OPT_PREFETCH_SPINORS, args.prefetch_spinors)
    ctx.wcl_load_gauge(torch.from_numpy(W.gauge_links(dims, EPS, SEED)).cuda(), KAPPA, CSW)
    vh = dims[0] * dims[1] * dims[2] * dims[3] // 2
    psi = torch.from_numpy(W.gaussian_fermion(dims, 1, nrhs=args.nrhs)[:, 0].copy()).cuda().reshape(-1)
    assert psi.numel() == args.nrhs * vh * 12
    out = torch.empty_like(psi)
    for _ in range(args.warmup):
        ctx.wcl_apply_Mpc(out, psi, args.prec, nrhs=args.nrhs)
    ctx.wcl_set_profiling(True)
    ctx.wcl_get_stats(reset=True)
    for _ in range(args.steps):
        ctx.wcl_apply_Mpc(out, psi, args.prec, nrhs=args.nrhs)
    st = ctx.wcl_get_stats(reset=True)
    peak, kind = measured_peaks()
    gbs = st["dslash_bytes"] / (st["dslash_ms"] * 1e-3) / 1e9
    print(json.dumps({"case": "mhat", "lattice": dims, "nrhs": args.nrhs, "prec": args.prec,
                      "tensor_cores": args.tensor_cores, "shared_links": args.shared_links,
                      "staged_spinors": args.staged_spinors, "autotune": args.autotune,
                      "paired_rhs": args.paired_rhs, "blocked_tiles": args.blocked_tiles,
                      "tma_staging": args.tma_staging, "prefetch_spinors": args.prefetch_spinors,
                      "dslash_launches": st["dslash_timed"], "avg_launch_ms": st["dslash_ms"] / st["dslash_timed"],
                      "gbs": gbs, "frac": gbs / peak, "peak": peak, "peak_kind": kind}))
    ctx.close()
    return 0


def _ctx_for(pkg, dims, seed, dev):
    import torch

    import workloads as W

    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(torch.from_numpy(W.gauge_links(dims, EPS, seed)).to(dev), KAPPA, CSW)
    return ctx


def run_batch_case(args):
    """Four uneven lattices, 12 Z2-noise sources each, to a 1e-10 true residual:
    one batched, graph-captured wcl_invert_batch over all 48 systems, against one
    12-RHS wcl_invert per lattice and against 12 single-RHS solves per lattice."""
    import numpy as np
    import torch

    import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    import paper_2411_08461_gb300 as pkg

    dev = torch.device("cuda", 0)
    shapes = [(8, 8, 8, 16), (12, 12, 12, 24), (16, 16, 16, 32), (24, 24, 24, 48)]
    ctxs = [_ctx_for(pkg, d, 200 + k, dev) for k, d in enumerate(shapes)]
    bs = [torch.from_numpy(W.z2_fermion(d, 300 + k, nrhs=12)).to(dev) for k, d in enumerate(shapes)]
    xs = [torch.zeros_like(b) for b in bs]
    prm = pkg.wcl_default_params(solver="bicgstab", sloppy=args.sloppy, tol=TOL, check_every=args.check_every,
                                 delta_reliable=args.delta)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        out = None
        for _ in range(args.steps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps / 1e3, out

    def batched():
        _, info = pkg.wcl_invert_batch(ctxs, xs, bs, 12, prm)
        return info

    t_batch, info_b = timed(batched)
    res = {"case": "batch", "lattices": ["x".join(map(str, d)) for d in shapes], "sources": "12 Z2 per lattice",
           "sloppy": args.sloppy, "tol": TOL,
           "batched": {"seconds": t_batch, "worst_true_residual": max(i["true_residual"] for i in info_b),
                       "iters_per_rhs": statistics.mean(i["iters"] for i in info_b)}}
    t_multi, worst_m, t_single, worst_s = 0.0, 0.0, 0.0, 0.0
    per = []
    for k, (c, b, x) in enumerate(zip(ctxs, bs, xs)):
        tm, info_m = timed(lambda: c.wcl_invert(x, b, 12, prm)[1])
        worst_m = max(worst_m, max(i["true_residual"] for i in info_m))
        x1 = torch.zeros_like(b[0])

        def singles():
            out = []
            for r in range(12):
                x1.zero_()
                out += c.wcl_invert(x1, b[r].contiguous(), 1, prm)[1]
            return out

        ts, info_s = timed(singles)
        worst_s = max(worst_s, max(i["true_residual"] for i in info_s))
        t_multi += tm
        t_single += ts
        per.append({"lattice": res["lattices"][k], "twelve_rhs_s": tm, "single_rhs_x12_s": ts})
    res["per_lattice_12rhs"] = {"seconds": t_multi, "worst_true_residual": worst_m}
    res["single_rhs"] = {"seconds": t_single, "worst_true_residual": worst_s}
    res["per_lattice"] = per
    res["speedup_batched_vs_single"] = t_single / t_batch
    res["speedup_batched_vs_per_lattice_12rhs"] = t_multi / t_batch
    print(json.dumps(res))
    for c in ctxs:
        c.close()
    return 0


def run_throughput_case(args):
    """16^3x32, FP32 fields and arithmetic: 100 applies of the full operator M
    (two fused dslash+clover launches each, 10 warm-up) on Gaussian spinors, then
    one BiCGStab solve from a point source to a 1e-10 true residual (FP32 inner
    solver, FP64 reliable updates and true residual)."""
    import torch

    import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    import paper_2411_08461_gb300 as pkg

    dev = torch.device("cuda", 0)
    dims = (16, 16, 16, 32)
    ctx = _ctx_for(pkg, dims, SEED, dev)
    psi = torch.from_numpy(W.gaussian_fermion(dims, 1)).to(dev)
    out = torch.empty_like(psi)
    for _ in range(10):
        ctx.wcl_apply_D(out, psi, "f32")
    ctx.wcl_set_profiling(True)
    ctx.wcl_get_stats(reset=True)
    for _ in range(100):
        ctx.wcl_apply_D(out, psi, "f32")
    st = ctx.wcl_get_stats(reset=True)
    ctx.wcl_set_profiling(False)
    peak, kind = measured_peaks()
    gbs = st["dslash_bytes"] / (st["dslash_ms"] * 1e-3) / 1e9
    b = torch.from_numpy(W.point_source(dims, 0, 0)).to(dev)
    x = torch.zeros_like(b)
    prm = pkg.wcl_default_params(solver="bicgstab", sloppy="f32", tol=TOL, delta_reliable=args.delta)
    ctx.wcl_invert(x, b, 1, prm)  # warm-up (tuning)
    x.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, info = ctx.wcl_invert(x, b, 1, prm)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"case": "throughput", "lattice": "16x16x16x32", "storage": "f32",
                      "applies": 100, "fused_launches": st["dslash_timed"],
                      "avg_launch_us": 1e3 * st["dslash_ms"] / st["dslash_timed"],
                      "gbs": gbs, "frac": gbs / peak, "peak": peak, "peak_kind": kind,
                      "gflops": st["dslash_flops"] / (st["dslash_ms"] * 1e-3) / 1e9,
                      "note": "the 16^3x32 FP32 working set (about 57 MB per launch) can stay in L2",
                      "solve": {"seconds": e0.elapsed_time(e1) / 1e3, "iters": info[0]["iters"],
                                "true_residual": info[0]["true_residual"],
                                "reliable_updates": info[0]["reliable_updates"]}}))
    ctx.close()
    return 0


def run_precond_case(args):
    """Apply the learned preconditioner's PTC network (random weights of the trained
    shape) to --nrhs Gaussian fields on --lattice: FP32 SIMT layers, BF16 SIMT layers,
    BF16 layers on mma.sync and on tcgen05 (inputs split into 3, 2 or 1 BF16 terms);
    CUDA-event time per application."""
    import torch

    import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    import paper_2411_08461_gb300 as pkg

    dims = tuple(int(v) for v in args.lattice.split(","))
    ctx = _ctx_for(pkg, dims, SEED, torch.device("cuda", 0))
    ctx.wcl_precond_load(pkg.ptc_flatten(W.ptc_weights(pkg.wcl.PTC_CHANNELS, seed=1, scale=0.3)))
    vh = dims[0] * dims[1] * dims[2] * dims[3] // 2
    r = torch.from_numpy(W.gaussian_fermion(dims, 2, nrhs=args.nrhs)[:, 0].copy()).cuda().reshape(args.nrhs, vh * 12)
    z = torch.empty_like(r)
    res = {"case": "precond", "lattice": dims, "nrhs": args.nrhs}
    for name, bf16, tc, split in (("fp32_simt", 0, 0, 3), ("bf16_simt", 1, 0, 3), ("bf16_tensor_cores", 1, 1, 3),
                                  ("bf16_tcgen05", 1, 2, 3), ("bf16_tcgen05_split2", 1, 2, 2),
                                  ("bf16_tcgen05_split1", 1, 2, 1)):
        ctx.wcl_set_option(pkg.wcl.WCL_OPT_PTC_TENSOR_CORES, tc)
        ctx.wcl_set_option(pkg.wcl.WCL_OPT_PTC_SPLIT, split)
        for _ in range(max(1, args.warmup)):
            ctx.wcl_precond_apply(z, r, args.nrhs, bf16=bf16)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            ctx.wcl_precond_apply(z, r, args.nrhs, bf16=bf16)
        e1.record()
        torch.cuda.synchronize()
        res[name + "_ms"] = e0.elapsed_time(e1) / args.steps
    print(json.dumps(res))
    ctx.close()
    return 0


def run_propagator_case(args):
    """The Sec. III.B sequence on --dims with the FP32 mixed-precision 12-RHS solver
    (FP64 reliable updates, tolerance --tol): wall sources at t0 = 0 with p = 0 and
    p = (0, 0, 1), the two propagators, the sequential source at t = Lt/2, the
    sequential propagator, the two-point (Eq. 6) and three-point (Eq. 7) functions.
    Then --steps timed calls of each contraction (CUDA events, after --warmup) for the
    contraction kernel's roofline: 4608 algorithmic bytes (two complex128
    propagators) and 1152 FP64 flops (144 complex multiply-adds) per site."""
    import torch

    import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    import paper_2411_08461_gb300 as pkg

    dev = torch.device("cuda", 0)
    dims = tuple(int(v) for v in args.dims.split(","))
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    t0, ts, mom = 0, lt // 2, (0, 0, 1)
    ctx = _ctx_for(pkg, dims, SEED, dev)
    prm = pkg.wcl_default_params(solver="bicgstab", sloppy=args.sloppy, tol=args.tol, check_every=args.check_every,
                                 delta_reliable=args.delta)
    f12 = lambda: torch.zeros((12, V * 12), dtype=torch.complex128, device=dev)
    b0, bp, x, S0, Sp, X, Sseq = f12(), f12(), f12(), f12(), f12(), f12(), f12()
    two = torch.zeros(lt, dtype=torch.complex128, device=dev)
    three = torch.zeros_like(two)
    g53 = pkg.wcl_gamma(15) @ pkg.wcl_gamma(4)
    ctx.wcl_wall_source(b0, t0)
    ctx.wcl_invert(x, b0, 12, prm)  # warm-up: tuning and graph capture
    torch.cuda.synchronize()
    iters = []

    def solve_into(prop, b):
        x.zero_()
        _, info = ctx.wcl_invert(x, b, 12, prm)
        iters.append(max(i["iters"] for i in info))
        assert all(i["true_residual"] <= args.tol for i in info), info
        ctx.wcl_fermions_to_propagator(prop, x)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.wcl_wall_source(b0, t0)
    ctx.wcl_wall_source(bp, t0, mom)
    solve_into(S0, b0)
    solve_into(Sp, bp)
    ctx.wcl_sequential_source(X, S0, ts, mom)
    ctx.wcl_propagator_to_fermions(b0, X)
    solve_into(Sseq, b0)
    ctx.wcl_contract(two, S0, Sp, None, mom)
    ctx.wcl_contract(three, Sseq, Sp, g53)
    e1.record()
    torch.cuda.synchronize()
    workflow_s = e0.elapsed_time(e1) / 1e3

    timings = {}
    for name, call in (("two_point", lambda: ctx.wcl_contract(two, S0, Sp, None, mom)),
                       ("three_point", lambda: ctx.wcl_contract(three, Sseq, Sp, g53))):
        for _ in range(max(3, args.warmup)):
            call()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            call()
        e1.record()
        torch.cuda.synchronize()
        timings[name] = e0.elapsed_time(e1) / args.steps
    peak, kind = measured_peaks()
    byts, flops = 4608.0 * V, 1152.0 * V
    roof = {}
    for name, ms in timings.items():
        gbs = byts / (ms * 1e-3) / 1e9
        tfl = flops / (ms * 1e-3) / 1e12
        roof[name] = {"ms_per_call": ms, "gbs": gbs, "hbm_frac": gbs / peak, "fp64_tflops": tfl,
                      "fp64_frac": tfl / (FP64_PEAK_GFLOPS / 1e3)}
    print(json.dumps({"case": "propagator", "lattice": dims, "tol": args.tol, "sloppy": args.sloppy,
                      "workflow_s": workflow_s, "max_iters_per_solve": iters,
                      "two_point": [[c.real, c.imag] for c in two.cpu().tolist()[:4]],
                      "contraction": roof, "hbm_peak_gbs": peak, "hbm_peak_kind": kind,
                      "fp64_peak_tflops": (FP64_PEAK_GFLOPS / 1e3), "fp64_peak_kind": "nominal",
                      "note": "each contraction call includes its finaliser and, with momentum, the phase table"}))
    ctx.close()
    return 0


def run_compare_case(args):
    """12 point sources on 32^3x64 solved four ways, each to a 1e-10 true residual:
    plain FP32 single-RHS BiCGStab (12 sequential solves, FP64 restarts), the
    batched 12-RHS mixed-precision BiCGStab, batched GCR(20), and batched
    flexible GCR(20) with the PTC network trained on the GPU on pairs from
    16^3x32 fields (kappa 0.124) and applied to a fresh 32^3x64 configuration."""
    import numpy as np
    import torch

    import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    import paper_2411_08461_gb300 as pkg

    dev = torch.device("cuda", 0)
    res = {"case": "compare", "workload": WORKLOAD}
    # ---- training on 16^3x32, kappa 0.124 -----------------------------------
    tdims, tkappa = (16, 16, 16, 32), 0.124
    tctx = pkg.Context(tdims)
    tctx.wcl_load_gauge(torch.from_numpy(W.gauge_links(tdims, EPS, 100)).to(dev), tkappa, CSW)
    rng = np.random.default_rng(101)
    w0 = []
    for cin, cout in zip(pkg.wcl.PTC_CHANNELS[:-1], pkg.wcl.PTC_CHANNELS[1:]):
        w = 1e-3 * (rng.standard_normal((cout, cin, 9, 4, 4)) + 1j * rng.standard_normal((cout, cin, 9, 4, 4)))
        w[0, 0, 0] += np.eye(4)
        w0.append(w)
    tctx.wcl_precond_load(pkg.ptc_flatten(w0))
    # pairs (r, e) = (M_hat e, e): half Gaussian e, half partial BiCGStab solutions (low-mode rich)
    n = args.pairs
    vh = tdims[0] * tdims[1] * tdims[2] * tdims[3] // 2
    es = torch.empty((n, vh * 12), dtype=torch.complex128, device=dev)
    ng = n // 2
    for k in range(0, ng, 64):
        m = min(64, ng - k)
        es[k:k + m] = torch.from_numpy(W.gaussian_fermion(tdims, 200 + k, nrhs=m)[:, 0].reshape(m, -1).copy()).to(dev)
    k = ng
    it = 4
    while k < n:
        m = min(12, n - k)
        b = torch.from_numpy(W.z2_fermion(tdims, 300 + k, nrhs=m).reshape(m, -1)).to(dev)
        x = torch.zeros_like(b)
        tctx.wcl_invert(x, b, m, pkg.wcl_default_params(sloppy="f32", tol=1e-10, maxiter=it, check_every=2),
                        check=False)
        es[k:k + m] = x.reshape(m, 2, -1)[:, 0]
        k += m
        it = 4 + (it + 4) % 60
    rs = torch.empty_like(es)
    for k in range(0, n, 64):
        m = min(64, n - k)
        tctx.wcl_apply_Mpc(rs[k:k + m], es[k:k + m].contiguous(), "f64", nrhs=m)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = tctx.wcl_precond_train(rs, es, n, pkg.wcl_default_train_params(epochs=args.epochs, batch=8, lr=2e-3))
    torch.cuda.synchronize()
    res["training"] = {"lattice": "16x16x16x32", "kappa": tkappa, "pairs": n, "epochs": args.epochs,
                       "seconds": time.perf_counter() - t0, "loss_per_epoch": [float(v) for v in losses]}
    weights = tctx.wcl_precond_get()
    tctx.close()
    del es, rs

    # ---- the four solves on 32^3x64 --------------------------------------------
    gauge = W.gauge_links(DIMS, EPS, 7)  # a configuration the network never saw
    src = np.stack([W.point_source(DIMS, s, c) for s in range(4) for c in range(3)])
    ctx = pkg.Context(DIMS)
    ctx.wcl_load_gauge(torch.from_numpy(gauge).to(dev), KAPPA, CSW)
    del gauge
    ctx.wcl_precond_load(weights)
    b = torch.from_numpy(src).to(dev)
    x = torch.zeros_like(b)

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t, out

    def solve(params, nrhs=12):
        return ctx.wcl_invert(x, b, nrhs, params)[1]

    # the baseline: FP32 BiCGStab restarted from the IEEE FP64 true residual (defect correction)
    plain = pkg.wcl_default_params(sloppy="f32", outer="f64", tol=TOL, restart_on_update=1, delta_reliable=1e-5)
    solve(pkg.wcl_default_params(sloppy="f32", tol=TOL))  # warm-up (12 RHS: tuner, workspace)
    ctx.wcl_invert(x[:1], b[:1], 1, plain)  # warm-up of the single-RHS configurations
    sec, infos = timed(lambda: [ctx.wcl_invert(x[k:k + 1], b[k:k + 1], 1, plain)[1][0] for k in range(12)])
    res["plain_f32_single_rhs"] = {"seconds": sec, "iters": [i["iters"] for i in infos],
                                   "worst_true_residual": max(i["true_residual"] for i in infos)}
    for name, prm in [("batched_bicgstab_f32", pkg.wcl_default_params(sloppy="f32", tol=TOL, delta_reliable=3e-4,
                                                                      check_every=2)),
                      ("batched_bicgstab_f16", pkg.wcl_default_params(sloppy="f16", tol=TOL, delta_reliable=0.01)),
                      ("batched_gcr20_f32", pkg.wcl_default_params(solver="gcr", sloppy="f32", tol=TOL,
                                                                   delta_reliable=1e-3)),
                      ("batched_fgcr20_learned_f32", pkg.wcl_default_params(solver="fgcr_learned", sloppy="f32",
                                                                            tol=TOL, delta_reliable=1e-3))]:
        sec, infos = timed(lambda: solve(prm))
        res[name] = {"seconds": sec, "iters_per_rhs": float(np.mean([i["iters"] for i in infos])),
                     "worst_true_residual": max(i["true_residual"] for i in infos),
                     "reliable_updates": float(np.mean([i["reliable_updates"] for i in infos]))}
    base = res["plain_f32_single_rhs"]["seconds"]
    for k2 in list(res):
        if isinstance(res[k2], dict) and "seconds" in res[k2] and k2 != "training":
            res[k2]["speedup_vs_plain"] = base / res[k2]["seconds"]
    print(json.dumps(res))
    ctx.close()
    return 0


def run_staggered_case(args):
    """HISQ staggered workload on --dims (mass 0.1): the thin links of the seeded gauge
    field (eps 0.3) smeared on the GPU into fat and long links (wcl_hisq_smear, FP64,
    CUDA events; FP64 flops per site counted from its staple passes), the staggered
    operator M = 2 m + D on those links, whole-lattice applies in FP64 and FP32
    (algorithmic bytes per output site = 16 links read once per launch + the input
    vector + the output + the 2 m x term), and one mixed-precision CG solve from a point
    source to --tol."""
    import numpy as np
    import torch

    import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    import paper_2411_08461_gb300 as pkg

    dims = tuple(int(v) for v in args.dims.split(","))
    lx, ly, lz, lt = dims
    vol = lx * ly * lz * lt
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = pkg.Context(dims, stream=stream)
    thin = torch.from_numpy(W.gauge_links(dims, EPS, SEED)).to(dev)
    fat, lng = torch.empty_like(thin), torch.empty_like(thin)
    ctx.wcl_hisq_smear(fat, lng, thin, 0.0)  # warm-up
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    ctx.wcl_hisq_smear(fat, lng, thin, 0.0)
    b.record(stream)
    torch.cuda.synchronize()
    smear_ms = a.elapsed_time(b)
    # FP64 flops per site: a one-sign staple is two 3x3 complex products (2 x 216); per
    # link direction the first level runs 15 two-sign staple passes, the second 15 plus
    # 12 one-sign Lepage passes; the U(3) projection about 750 per link, the Naik link 432
    mm = 216
    flops_site = 4 * (15 * 2 * 2 * mm) + 4 * (15 * 2 * 2 * mm + 12 * 2 * mm) + 4 * 750 + 4 * 2 * mm
    ctx.wcl_load_staggered(fat, lng, 0.1)
    del fat, lng, thin
    chi = torch.from_numpy(W.gaussian_complex((2, lt, lz, ly, lx // 2, 3), 602)).to(dev)
    out = torch.empty_like(chi)
    peak, kind = measured_peaks()
    res = {"case": "staggered", "lattice": dims, "mass": 0.1, "peak": peak, "peak_kind": kind,
           "links": "HISQ smearing of the eps 0.3 thin links on the GPU",
           "hisq_smear": {"ms": smear_ms, "fp64_gflop": vol * flops_site / 1e9,
                          "fp64_tflops": vol * flops_site / (smear_ms * 1e-3) / 1e12,
                          "fp64_nominal_tflops": 1.25,
                          "frac_of_nominal": vol * flops_site / (smear_ms * 1e-3) / 1e12 / 1.25}}
    for prec, real in (("f64", 8), ("f32", 4)):
        for _ in range(3):
            ctx.wcl_apply_staggered(out, chi, prec)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        n = 10
        for _ in range(n):
            ctx.wcl_apply_staggered(out, chi, prec)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / n
        # per output site: 16 links x 18 reals, input vector 6 reals, output 6, 2 m x term 6
        byts = vol * (16 * 18 + 18) * real
        res[prec] = {"ms_per_apply_with_io": ms, "algorithmic_gb_per_apply": byts / 1e9,
                     "note": "the call time includes the QDP import and export kernels around the two dslash launches"}
    ctx.wcl_set_profiling(True)
    ctx.wcl_get_stats(reset=True)
    src = torch.zeros_like(chi)
    src[0, 0, 0, 0, 0, 0] = 1.0
    x = torch.zeros_like(src)
    prm = pkg.wcl_default_params(sloppy="f32", tol=args.tol)
    ctx.wcl_invert_staggered(x, src, 1, prm)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    _, info = ctx.wcl_invert_staggered(x, src, 1, prm)
    b.record(stream)
    torch.cuda.synchronize()
    res["cg_solve"] = {"seconds": a.elapsed_time(b) / 1e3, "iters": info[0]["iters"],
                       "restarts": info[0]["reliable_updates"], "true_residual": info[0]["true_residual"]}
    print(json.dumps(res))
    ctx.close()
    return 0


def run_mg_case(args):
    """Two-level multigrid on --dims at --kappa: the hierarchy's setup (null-space relaxation,
    prolongator, coarse stencil) timed, then FGCR preconditioned by the K-cycle on the 12
    spin-colour point sources to --tol, against the batched 12-RHS BiCGStab solve of the
    bench line on the same field (CUDA events on the library's stream)."""
    import numpy as np
    import torch

    import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    import paper_2411_08461_gb300 as pkg

    dims = tuple(int(v) for v in args.dims.split(","))
    block = tuple(int(v) for v in args.mg_block.split(","))
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = pkg.Context(dims, stream=stream)
    ctx.wcl_load_gauge(torch.from_numpy(W.gauge_links(dims, EPS, SEED)).to(dev), args.kappa, CSW)
    src = torch.from_numpy(np.stack([W.point_source(dims, s, c) for s in range(4) for c in range(3)])).to(dev)
    x = torch.zeros_like(src)

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3, out

    starts = torch.from_numpy(W.gaussian_fermion(dims, 500, nrhs=args.mg_nvec)).to(dev)
    mprm = pkg.wcl_default_mg_params(block=block, nvec=args.mg_nvec)
    ctx.wcl_mg_setup(starts, mprm)  # warm-up (tuner, module loading)
    setup_s, _ = timed(lambda: ctx.wcl_mg_setup(starts, mprm))
    del starts
    line = {"case": "mg", "lattice": dims, "kappa": args.kappa, "block": block, "nvec": args.mg_nvec,
            "relax_steps": mprm.relax_steps, "setup_seconds": setup_s}
    if args.mg_single:
        mg = pkg.wcl_default_params(solver="fgcr_mg", tol=args.tol, gcr_nkrylov=args.mg_nkrylov)
        ctx.wcl_invert(x[:1], src[:1], 1, mg)  # warm-up
        mg_s, infos = timed(lambda: ctx.wcl_invert(x, src, 12, mg)[1])
        line["mg_fgcr"] = {"seconds": mg_s, "outer_iters_per_rhs": float(np.mean([i["iters"] for i in infos])),
                           "restarts_per_rhs": float(np.mean([i["reliable_updates"] for i in infos])),
                           "worst_true_residual": max(i["true_residual"] for i in infos)}
    # all twelve right-hand sides at once: FGCR on M_hat preconditioned by the batched
    # K-cycle (a fixed number of coarse steps, every coefficient on the device)
    starts = torch.from_numpy(W.gaussian_fermion(dims, 500, nrhs=args.mg_nvec)).to(dev)
    pre, post = (int(v) for v in args.mg_smooth.split(","))
    bprm = pkg.wcl_default_mg_params(block=block, nvec=args.mg_nvec, coarse_maxiter=args.mg_coarse_steps, pre=pre,
                                     post=post)
    ctx.wcl_mg_setup(starts, bprm)
    del starts
    mgb = pkg.wcl_default_params(solver="fgcr_mg_batched", sloppy="f32", tol=args.tol, gcr_nkrylov=args.mg_nkrylov,
                                 delta_reliable=3e-4)
    ctx.wcl_invert(x, src, 12, mgb)  # warm-up (tuner, work space)
    mgb_s, binf = timed(lambda: ctx.wcl_invert(x, src, 12, mgb)[1])
    line["mg_fgcr_batched"] = {"seconds": mgb_s, "coarse_steps": args.mg_coarse_steps, "nkrylov": args.mg_nkrylov,
                               "smoothing": [pre, post],
                               "iters_per_rhs": float(np.mean([i["iters"] for i in binf])),
                               "reliable_updates_per_rhs": float(np.mean([i["reliable_updates"] for i in binf])),
                               "worst_true_residual": max(i["true_residual"] for i in binf)}
    bi = pkg.wcl_default_params(solver="bicgstab", sloppy="f32", tol=args.tol, check_every=2, delta_reliable=3e-4)
    ctx.wcl_invert(x, src, 12, bi)
    bi_s, binfos = timed(lambda: ctx.wcl_invert(x, src, 12, bi)[1])
    line["batched_bicgstab_f32"] = {"seconds": bi_s, "iters_per_rhs": float(np.mean([i["iters"] for i in binfos])),
                                    "worst_true_residual": max(i["true_residual"] for i in binfos)}
    if args.mg_single:
        line["mg_over_bicgstab_time"] = (line["mg_fgcr"]["seconds"] + setup_s) / bi_s
    line["mg_batched_over_bicgstab_time"] = mgb_s / bi_s
    line["mg_batched_with_setup_over_bicgstab_time"] = (mgb_s + setup_s) / bi_s
    print(json.dumps(line))
    ctx.close()
    return 0


def run_force_case(args):
    """FP64 clover fermion force of the two-flavour even-odd action on --dims (kappa
    0.1235, c_sw 1, clover determinant term included) for a Gaussian X, timed through
    wcl_clover_force with CUDA events (the call applies M_hat and two FP64 half-dslashes,
    then the per-site Omega kernel and the per-link force kernel).  FP64 flops counted
    per link (hopping outer products 1.4 k, 24 clover-leaf terms of four 3x3 complex
    products 21 k, U G and the projection 0.3 k) and per site (the sigma traces and the
    determinant term 7.9 k), against the FP64 nominal rate."""
    import numpy as np
    import torch

    import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    import paper_2411_08461_gb300 as pkg

    dims = tuple(int(v) for v in args.dims.split(","))
    vol = dims[0] * dims[1] * dims[2] * dims[3]
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = pkg.Context(dims, stream=stream)
    gauge = torch.from_numpy(W.gauge_links(dims, EPS, SEED)).to(dev)
    ctx.wcl_load_gauge(gauge, KAPPA, CSW)
    x = torch.from_numpy(np.ascontiguousarray(W.gaussian_fermion(dims, 1)[0])).to(dev)
    out = torch.empty_like(gauge)
    ctx.wcl_clover_force(out, x, True)  # warm-up (work space, module load)
    torch.cuda.synchronize()
    runs = []
    for _ in range(max(1, args.steps)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.wcl_clover_force(out, x, True)
        b.record(stream)
        torch.cuda.synchronize()
        runs.append(a.elapsed_time(b))
    ms = statistics.median(runs)
    flops = 4 * vol * (1.44e3 + 21.1e3 + 0.3e3) + vol * 7.9e3 + 4 * (vol // 2) * 1824
    line = {"case": "force", "lattice": dims, "ms": ms, "runs": len(runs),
            "fp64_gflop": flops / 1e9, "fp64_tflops": flops / (ms * 1e-3) / 1e12, "fp64_nominal_tflops": 1.25,
            "frac_of_nominal": flops / (ms * 1e-3) / 1e12 / 1.25,
            "what": "wcl_clover_force, FP64, two-flavour even-odd clover action with the odd clover determinant"}
    print(json.dumps(line))
    ctx.close()
    return 0


def main():
    args = parse()
    if args.case == "mhat":
        return run_mhat_case(args)
    if args.case == "batch":
        return run_batch_case(args)
    if args.case == "throughput":
        return run_throughput_case(args)
    if args.case == "compare":
        return run_compare_case(args)
    if args.case == "precond":
        return run_precond_case(args)
    if args.case == "propagator":
        return run_propagator_case(args)
    if args.case == "mg":
        return run_mg_case(args)
    if args.case == "staggered":
        return run_staggered_case(args)
    if args.case == "force":
        return run_force_case(args)
    if args.impl == "reference":
        # the oracle runs on rank 0's host cores only; other ranks exit without work
        return run_reference(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
    rank, world, local = dist_init(args.gpus)
    if True:
        rc = run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
