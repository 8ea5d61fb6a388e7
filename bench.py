#!/usr/bin/env python3
"""Benchmark: Parareal solves/s at 1e-8 relative error versus the FP64 oracle.

Workload (one step = one pass of the whole hot path): the 1D advection-
diffusion-reaction problem u_t = 0.01 u_xx - u_x - 0.1 u, n = 4095 interior
nodes, T = 1 in N = 64 intervals of M = 256 backward-Euler steps, rank
R = 16 with p = 8 oversampling, u0 = 5 seeded Gaussian bumps, f = 0.  A step
builds the coarse solvers (randomized SVD: forward sketch, orthonormalisation,
adjoint sketch, orthonormalisation, small SVD, lift) and runs one Parareal
solve to the a posteriori tolerance 1e-8 (fine solves, coarse sweeps, bounds).
The default arithmetic is the mixed mode (FP32 sketches, FP64 Parareal on
the FP64 fine-solve kernels).  Beside it the line times the same step with
the fine backward-Euler steps computed from FP32 solves and one correction
round per step whose residual is formed in pairs of FP32 numbers
(`fine_refined`; about 48-bit steps, 2.7e-12 from the FP64 kernels' steps
over an interval of 256 steps); --tri-refine R times that variant as the
headline instead.

value: solves/s with inputs resident in HBM (device-timed with CUDA events on
the library's stream).  e2e: the same through the C ABI with host buffers (the
operator coefficients and u0 uploaded, the iterate read back inside the timed
region).  --impl reference times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores.

Multi-GPU: the path does not shard; --gpus N runs N independent replicas (one
process per GPU under torchrun), value = all solves / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Parareal solves/s at 1e-8 rel err vs FP64 oracle"
UNIT = "solves/s"
TOL = 1e-8
# DRAM bytes per system of the FP64 fine-solve kernel, from one ncu capture of
# k_tri_cluster_wt<13, 3> (62 systems: 2.1978 MB read, 0 written)
F64_DRAM_BYTES_PER_SYSTEM = 2.1978e6 / 62
# and of the refined FP32 fine-solve kernel k_tri_irt<16> (62 systems:
# 2.1652 MB read, 0 written)
IRT_DRAM_BYTES_PER_SYSTEM = 2.165248e6 / 62
WORKLOAD = "adr1d n=4095 N=64 M=256 R=16 p=8 tol=1e-8"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="time only the headline step (no amortised, classical, two-sided or "
                         "host-buffer legs): the launch list of a profiler then holds the "
                         "warm-up and timed steps alone")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of oracle work for the cpu_baseline samples (all cores, then "
                         "one core)")
    ap.add_argument("--batch-per-grid", type=int, default=2,
                    help="batch mode: problems per grid size of the uneven 2D batch")
    ap.add_argument("--mode", default="solve",
                    choices=["solve", "serve", "krylov", "batch", "cfg3", "trisweep", "exp3", "fp64probe"],
                    help="solve: the headline step; serve: Poisson request stream on resident "
                         "coarse solvers (p50/p99 latency per offered rate); krylov: bandwidth "
                         "of the 2D Krylov fine propagator (HBM GB/s fraction)")
    ap.add_argument("--krylov-precs", default="mixed,f64",
                    help="krylov mode: precisions to time (mixed = FP32 sketch settings)")
    ap.add_argument("--krylov-systems", default="64,16",
                    help="krylov mode: systems per launch for each precision")
    ap.add_argument("--krylov-block", type=int, default=0, choices=[0, 4],
                    help="--mode krylov: solve the systems four at a time by block CG")
    ap.add_argument("--krylov-block-clusters", type=int, default=0,
                    help="--mode krylov: clusters in flight of the block CG (0: automatic)")
    ap.add_argument("--krylov-m", type=int, default=511,
                    help="krylov mode: grid size m of the diff2d m x m operator")
    ap.add_argument("--krylov-refine", type=int, default=0, choices=[0, 1, 2],
                    help="krylov mode: 1 forces the FP64 iterative refinement where the FP32 "
                         "on-chip kernel takes the grid (0: the library's default); batch "
                         "mode: 2 runs the FP64 fine steps on the FP64 Krylov kernels")
    ap.add_argument("--krylov-stage", type=int, default=0, choices=[0, 1],
                    help="krylov mode: 1 stages the FP32 global-memory kernel's stencil inputs "
                         "in shared memory by bulk copies (0: read from global memory)")
    ap.add_argument("--krylov-adv", action="store_true",
                    help="krylov mode: the nonsymmetric advection-diffusion operator (BiCGStab)")
    ap.add_argument("--refine-digits", default="",
                    help="krylov mode: also time the FP64 iterative refinement with these inner "
                         "FP32 tolerances 10^-d (comma list)")
    ap.add_argument("--krylov-onchip", type=int, default=0, choices=[0, 2],
                    help="krylov mode: 0 the on-chip CG where it applies, 2 the kernel with "
                         "its Krylov vectors in global memory")
    ap.add_argument("--sweep-systems", default="16,32,48,64,96,128",
                    help="trisweep mode: batch sizes of the FP64 adr1d fine-solve sweep")
    ap.add_argument("--sweep-chunks", default="8,9,10,11,12,13,14,15,16",
                    help="trisweep mode: chunk lengths (tri_wchunk) of the one-warp kernel")
    ap.add_argument("--sweep-refine", default="1,2",
                    help="trisweep: round counts of the refined FP32 fine solves to time ('' = none)")
    ap.add_argument("--tri-refine", type=int, default=0, choices=[0, 1, 2, 3],
                    help="timed step's 1D fine solves from FP32 solves refined by pair residuals: "
                         "rounds per step (0 = the FP64 kernels, the workload's precision; the other "
                         "variant is timed beside it unless --headline-only)")
    ap.add_argument("--rates", default="10,30,100,300,1000")
    ap.add_argument("--serve-targets", default="",
                    help="serve mode: extra passes 'rate:adr1d_target_ms,...' with admission "
                         "control on the adr1d handle")
    ap.add_argument("--serve-seconds", type=float, default=6.0,
                    help="arrival window per rate (at most 2000 requests)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate_over_ranks(ms_step: float, world: int, device=None):
    """Whole-job throughput of `world` independent replicas (one solve per rank
    and step): the step time is the slowest rank's (max over ranks, through
    the initialised process group), and value = world * 1000 / that time.
    Returns (ms_step, solves per second)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_step], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    return ms_step, world * 1000.0 / ms_step


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm / cpu baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(P, budget_s: float, threads: int = 0, iters: int = 3):
    """Time the FP64 oracle on a bounded sample of the workload and extrapolate
    to one solve: the rSVD of as many intervals as fit in 60% of the budget
    (at least one), scaled by N / intervals done, plus `iters` real Parareal
    iterations over all N intervals (coarse solvers of the sampled intervals
    reused for the others; the N fine solves of an iteration run as one
    batched call), scaled by the iteration count of the solve.  threads:
    the oracle's OpenMP threads (0: all host cores)."""
    from oracle import oracle as orc
    orc.set_num_threads(threads)
    try:
        oop = orc.Tridiag(P.lo, P.di, P.up)
        t0 = time.perf_counter()
        coarse = []
        while len(coarse) < P.N:
            coarse.append(orc.rsvd_interval(oop, P.dt, P.M, len(coarse), P.R, P.p, P.seed))
            if time.perf_counter() - t0 > 0.6 * budget_s:
                break
        nb = len(coarse)
        t_build = (time.perf_counter() - t0) * P.N / nb
        co = orc.Coarse([coarse[i % nb] for i in range(P.N)], P.R, P.p)
        t1 = time.perf_counter()
        orc.parareal(oop, P.dt, P.M, P.N, co, P.u0, K=iters)
        t_iter = (time.perf_counter() - t1) / iters
        cores = orc.num_threads()
    finally:
        orc.set_num_threads(0)
    wall = time.perf_counter() - t0
    return {"t_build": t_build, "t_iter": t_iter, "intervals": nb, "iters": iters,
            "cores": cores, "wall_s": wall}


def cpu_baseline_entry(P, budget_s: float, k_iters: int, threads: int) -> dict:
    smp = oracle_sample(P, budget_s, threads)
    est = smp["t_build"] + smp["t_iter"] * k_iters
    return {"value": 1.0 / est, "unit": UNIT, "cores": smp["cores"], "kind": "oracle",
            "sample": "rSVD of %d/%d intervals scaled to %d, plus %d real Parareal iterations "
                      "(all %d intervals) scaled to the %d of the solve: %.1f s per solve "
                      "(%.1f s of oracle work timed)"
                      % (smp["intervals"], P.N, P.N, smp["iters"], P.N, k_iters, est,
                         smp["wall_s"])}


def run_reference(args, P, k_iters: int):
    """The reference arm: the FP64 oracle as it stands on the host cores.  Each
    step times one bounded sample (oracle_sample, about 4 s); value = the
    solves/s that sample extrapolates to; ms_per_step = the measured time of
    a step's sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    ests, walls = [], []
    smp = None
    budget = min(args.cpu_budget, 4.0)
    for s in range(args.warmup + args.steps):
        smp = oracle_sample(P, budget_s=budget)
        if s >= args.warmup:
            ests.append(smp["t_build"] + smp["t_iter"] * k_iters)
            walls.append(smp["wall_s"])
    sec = statistics.mean(ests)
    val = 1.0 / sec
    sample = ("per step: oracle rSVD of %d of %d intervals scaled to %d, plus %d real Parareal "
              "iterations (all intervals) scaled to the %d of the solve; %.1f s per solve "
              "extrapolated, %.2f s measured per step"
              % (smp["intervals"], P.N, P.N, smp["iters"], k_iters, sec, statistics.mean(walls)))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(walls) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "solve_estimate_s": sec,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": smp["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------
FP64_PEAK_GFLOPS = 152 * 4 * 2.070      # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_GFLOPS = 152 * 256 * 2.070    # 128 FP32 FMA/clk/SM


def serve_leg(ctx, rates, seconds: float, quiet: bool = False, targets=None) -> dict:
    """Requests with new sources f = sum_{i<4} a_i sin(w_i t) exp(-(x-c_i)^2/w_i^2) and new
    u0 on coarse solvers prebuilt (mixed mode) for the 1D heat (n=255, N=16, M=64) and the
    1D advection-diffusion-reaction (n=4095, N=64, M=256) operators, 50/50, tol 1e-8,
    Poisson arrivals at each offered rate for `seconds` (at most 2000 requests);
    latency = submit -> result on the host.  targets: (rate, adr1d latency
    target in ms) passes run after the plain ones, with requests turned away
    (LRP_EBUSY) counted."""
    from paper_2508_08873_gb300 import _native
    from paper_2508_08873_gb300 import api, workloads as W
    probs = [W.heat1d(), W.adr1d()]
    ops = [api.Operator.tridiag(ctx, P.lo, P.di, P.up) for P in probs]
    cos = [api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="mixed")
           for op, P in zip(ops, probs)]
    pool = []
    rng = np.random.default_rng(2)
    for k in range(64):
        j = k % 2
        P = probs[j]
        pool.append((j,) + tuple(W.serving_request(P.n, P.N, P.M, P.dt, k)))
    srv = api.Server(ctx, max_slots=128, max_terms=4)
    # warm-up: every kernel configuration once
    for j in (0, 1):
        _, u0, g, c = pool[j]
        srv.wait(srv.submit(cos[j], u0, g, c, K=probs[j].N, tol=TOL), timeout=600)
    results = []
    passes = [(float(r), None) for r in rates] + [(float(r), float(t)) for r, t in (targets or [])]
    for rate, target in passes:
        srv.set_latency_target(cos[1], target or 0.0)
        nreq = int(min(2000, max(8, rate * seconds)))
        gaps = rng.exponential(1.0 / rate, nreq)
        tickets = []
        rejected = [0, 0]
        t0 = time.perf_counter()
        t_next = t0
        for i in range(nreq):
            t_next += gaps[i]
            while time.perf_counter() < t_next:
                time.sleep(min(0.0005, max(0.0, t_next - time.perf_counter())))
            j, u0, g, c = pool[i % len(pool)]
            try:
                tickets.append((j, srv.submit(cos[j], u0, g, c, K=probs[j].N, tol=TOL)))
            except _native.LrpError as e:
                if e.status != _native.LRP_EBUSY:
                    raise
                rejected[j] += 1
        lat = []
        lat_by = {0: [], 1: []}
        for j, t in tickets:
            u, info = srv.wait(t, timeout=1200)
            lat.append(info["latency_ms"])
            lat_by[j].append(info["latency_ms"])
        span = time.perf_counter() - t0

        def pct(v, q):
            return float(np.percentile(v, q)) if v else None
        results.append({"offered_per_s": rate, "requests": nreq,
                        "adr1d_latency_target_ms": target,
                        "rejected_busy": {"heat1d": rejected[0], "adr1d": rejected[1]},
                        "achieved_per_s": len(tickets) / span,
                        "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                        "p50_ms_heat1d": pct(lat_by[0], 50), "p99_ms_heat1d": pct(lat_by[0], 99),
                        "p50_ms_adr1d": pct(lat_by[1], 50), "p99_ms_adr1d": pct(lat_by[1], 99)})
        if not quiet:
            print(json.dumps(results[-1]), flush=True)
    srv.set_latency_target(cos[1], 0.0)
    stats = srv.stats()
    srv.close()
    for co in cos:
        co.close()
    for op in ops:
        op.close()
    return {"workload": "heat1d n=255 N=16 + adr1d n=4095 N=64, 50/50, tol=1e-8, Poisson "
                        "arrivals, mixed coarse solvers prebuilt",
            "saturation_per_s": max((r["achieved_per_s"] for r in results), default=0.0),
            "rates": results, "server": stats}


def run_serve(args):
    import torch
    from paper_2508_08873_gb300 import api
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ctx = api.Context(local)
    tg = [tuple(float(x) for x in v.split(":")) for v in args.serve_targets.split(",") if v]
    res = serve_leg(ctx, [float(r) for r in args.rates.split(",")], args.serve_seconds,
                    targets=tg)
    line = {"metric": "served Parareal solves/s (continuous batching)",
            "value": res["saturation_per_s"], "unit": "solves/s", "n_gpus": 1,
            "higher_is_better": True, "mode": "serve",
            "config": {"workload": "serve " + res["workload"]},
            "rates": res["rates"], "server": res["server"]}
    print(json.dumps(line), flush=True)


HBM_PEAK_GBS_FALLBACK = 6800.0


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s (generated file),
    else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                v = d[k]
                return float(v["value"] if isinstance(v, dict) else v), "measured"
    except Exception:
        pass
    return HBM_PEAK_GBS_FALLBACK, "fallback"


# DRAM bytes of one on-chip CG launch on diff2d 511^2 (16 FP32 systems, one
# step, 788 CG iterations each), from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum: 38.77 + 1.02 MB): the coefficients' and vectors'
# first reads and the results' writes; the Krylov vectors stay on chip.
ONCHIP_DRAM_BYTES_PER_SYSTEM = (38.77e6 + 1.02e6) / 16


def krylov_leg(ctx, precs, nsyss, steps: int, warmup: int, onchip: int = 0, block: int = 0,
               block_clusters: int = 0, refine_digits=(), m: int = 511,
               refine_mode: int = 0, adv: bool = False, stage: int = 0) -> dict:
    """The 2D fine propagator's bandwidth (the 'HBM GB/s frac' part of the
    metric): diff2d (511^2, kappa checkerboard, dt = 1/4096), Jacobi-PCG per
    backward-Euler step, FP32 sketch propagations (rtol 1e-6) and FP64 fine
    propagations (rtol 1e-12), one step per system.  Algorithmic traffic of a
    CG iteration: x, r, p read and written (6 words per grid point);
    achieved = that x iterations / kernel time (CUDA events on the library's
    stream).  With block = 4 the systems are solved four at a time in one
    block Krylov space (fewer iterations per system; `us_per_system_step`
    compares the kernels per system and step).  The "f64" entry times the
    FP64 Krylov kernel itself (krylov_refine = 2); "f64_refine" times the
    library's default FP64 step for this grid, iterative refinement (FP64
    residuals, FP32 on-chip CG corrections), by CUDA events on the library's
    stream around whole propagations (its kernels of both precisions and the
    host's checks between rounds)."""
    import torch
    from paper_2508_08873_gb300 import api, workloads as W
    P = W.diff2d(m=m, T=128 * 32 / 4096)            # dt = 1/4096 at every grid size
    if adv:                                         # the nonsymmetric operator (BiCGStab)
        P.st = W.adv2d_op(m, 0.01)
    op = api.Operator.stencil5(ctx, P.mx, P.my, P.st)
    op.set_krylov(1e-12, 1e-6, 20000)
    ctx.set_param("krylov_refine", 2)
    ctx.set_param("krylov_stage", stage)
    ctx.set_param("krylov_onchip", onchip)
    ctx.set_param("krylov_block", block)
    ctx.set_param("krylov_block_clusters", block_clusters)
    peak, peak_src = hbm_peak_gbs()
    rng = np.random.default_rng(0)
    out = {}
    try:
        for prec, nsys in zip(precs, nsyss):
            X = rng.standard_normal((nsys, P.n))
            for _ in range(max(1, warmup)):
                api.propagate(ctx, op, P.dt, 1, X, prec=prec)
            fam = "propagate_f64" if prec == "f64" else "propagate_f32"
            it0 = op.krylov_iterations()
            ctx.set_kernel_timing(True)
            ctx.reset_kernel_time()
            for _ in range(steps):
                api.propagate(ctx, op, P.dt, 1, X, prec=prec)
            nl, ms = ctx.kernel_time(fam)
            ctx.set_kernel_timing(False)
            its = op.krylov_iterations() - it0
            es = 8 if prec == "f64" else 4
            gbs = its * 6 * P.n * es / (ms * 1e-3) / 1e9
            onchip_used = ctx.get_param("krylov_onchip_rows") > 0
            block_used = ctx.get_param("krylov_block_last_systems") > 0
            key = "f64" if prec == "f64" else "f32"
            out[key] = {"systems": nsys, "cg_iterations_per_step": its / (nsys * steps),
                        "us_per_iteration_and_system": ms * 1e3 / its,
                        "us_per_system_step": ms * 1e3 / (nsys * steps), "achieved_gbs": gbs,
                        "peak_gbs": peak, "frac": gbs / peak, "launches": nl,
                        "rtol": 1e-12 if prec == "f64" else 1e-6,
                        "kernel": "k_bcg" if block_used else "k_cg_onchip" if onchip_used
                        else "k_krylov",
                        "block_shape": {"systems_per_block": ctx.get_param("krylov_block_last_systems"),
                                        "ctas_per_cluster": ctx.get_param("krylov_block_last_cs"),
                                        "clusters": ctx.get_param("krylov_block_last_clusters")},
                        "dram_traffic_per_launch": ONCHIP_DRAM_BYTES_PER_SYSTEM * nsys
                        if onchip_used and key == "f32" else None,
                        "onchip_shape": {"rows_per_cta": ctx.get_param("krylov_onchip_rows"),
                                         "ctas_per_cluster": ctx.get_param("krylov_onchip_cs"),
                                         "clusters": ctx.get_param("krylov_onchip_clusters")}}
            if prec == "f64" and onchip == 0 and block == 0:
                # the default FP64 path for this grid: iterative refinement
                Xd = torch.from_numpy(X).cuda()
                Yd = torch.empty_like(Xd)
                strm = torch.cuda.ExternalStream(ctx.stream)

                def refine(digits):
                    ctx.set_param("krylov_refine", refine_mode)
                    ctx.set_param("krylov_refine_digits", digits)
                    try:
                        for _ in range(max(1, warmup)):
                            api.propagate(ctx, op, P.dt, 1, Xd, prec=prec, out=Yd)
                        it0 = op.krylov_iterations()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        torch.cuda.synchronize()
                        e0.record(strm)
                        for _ in range(steps):
                            api.propagate(ctx, op, P.dt, 1, Xd, prec=prec, out=Yd)
                        e1.record(strm)
                        e1.synchronize()
                        return e0.elapsed_time(e1), op.krylov_iterations() - it0
                    finally:
                        ctx.set_param("krylov_refine", 2)
                        ctx.set_param("krylov_refine_digits", 0)

                ms_r, its_r = refine(0)
                out["f64_refine"] = {
                    "systems": nsys, "rtol": 1e-12,
                    "us_per_system_step": ms_r * 1e3 / (nsys * steps),
                    "speedup_vs_f64_kernel": out["f64"]["us_per_system_step"] / (ms_r * 1e3 / (nsys * steps)),
                    "fp32_cg_iterations_per_step": its_r / (nsys * steps),
                    "inner_rtol": 1e-3,
                    "kernels": "k_ir_resid + k_ir_reduce (FP64 residual, scaled-norm test), "
                               "k_ir_scale, k_cg_onchip<float> (correction), k_ir_apply"}
                for d in refine_digits:
                    ms_d, its_d = refine(d)
                    out["f64_refine"].setdefault("by_inner_digits", {})[str(d)] = {
                        "us_per_system_step": ms_d * 1e3 / (nsys * steps),
                        "fp32_cg_iterations_per_step": its_d / (nsys * steps)}
    finally:
        ctx.set_param("krylov_refine", 0)
        ctx.set_param("krylov_stage", 0)
        ctx.set_param("krylov_onchip", 0)
        ctx.set_param("krylov_block", 0)
        ctx.set_param("krylov_block_clusters", 0)
        op.close()
    return {"workload": (f"adv2d {m}^2 nu=0.01, dt=1/4096, Jacobi-BiCGStab" if adv else
                         f"diff2d {m}^2 kappa 8x8 checkerboard, dt=1/4096, Jacobi-PCG") +
                        ", one backward-Euler step per system",
            "peak_source": peak_src, "algorithmic_bytes": "6 words per grid point and CG "
                                                          "iteration (x, r, p read + written)",
            **out}


def run_krylov(args):
    import torch
    from paper_2508_08873_gb300 import api
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ctx = api.Context(local)
    precs = args.krylov_precs.split(",")
    nsyss = [int(v) for v in args.krylov_systems.split(",")]
    res = krylov_leg(ctx, precs, nsyss, args.steps, args.warmup, args.krylov_onchip,
                     args.krylov_block, args.krylov_block_clusters,
                     [int(v) for v in args.refine_digits.split(",") if v], args.krylov_m,
                     args.krylov_refine, args.krylov_adv, args.krylov_stage)
    head = res["f64" if precs[0] == "f64" else "f32"]
    line = {"metric": "2D fine-propagator algorithmic bandwidth (HBM GB/s frac)",
            "value": head["achieved_gbs"], "unit": "GB/s", "n_gpus": 1,
            "higher_is_better": True, "mode": "krylov", "steps": args.steps,
            "warmup": args.warmup, "dtype": "f64" if precs[0] == "f64" else "f32",
            "data": "synthetic", "config": {"workload": res["workload"]},
            "roofline": {"bound": "hbm", "achieved": head["achieved_gbs"],
                         "peak": head["peak_gbs"], "unit": "GB/s", "frac": head["frac"],
                         "peak_source": res["peak_source"],
                         "traffic": head["dram_traffic_per_launch"],
                         "note": "algorithmic bytes (x, r, p read + written per CG iteration) "
                                 "over kernel time; the on-chip kernel keeps the Krylov vectors "
                                 "in registers and shared memory"},
            "precisions": res}
    print(json.dumps(line), flush=True)


def all_fp64_leg(args, ctx, op, P, stream, flush) -> dict:
    """The same step (build + solve to tol 1e-8) with every stage in FP64 (the
    plain all-FP64 form the mixed one is compared with), device-timed like the
    headline, L2 flushed between steps."""
    import torch
    from paper_2508_08873_gb300 import api
    dev = flush.device
    u0 = torch.tensor(P.u0, dtype=torch.float64, device=dev)
    out = torch.empty((P.N + 1, P.n), dtype=torch.float64, device=dev)

    def step():
        co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64")
        _, info = api.parareal_solve(ctx, co, u0, K=P.N, tol=TOL, out=out, bounds=False)
        co.close()
        return info
    step()
    nsteps = max(3, args.steps // 3)
    ms = []
    for _ in range(nsteps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return {"solves_per_s": 1000.0 / statistics.mean(ms), "ms_per_step": statistics.mean(ms),
            "steps": nsteps, "iterations": info["k_done"], "rel_err_vs_oracle": None,
            "note": "FP64 sketches, orthonormalisation, small SVD, coarse applies and fine "
                    "solves; same workload and tolerance as the headline", "out": out}


def run_batch(args):
    """The uneven 2D batch (64 independent advection-diffusion problems
    u_t = nu Lap u - b.grad u on grids drawn from {63^2, 127^2, 255^2, 511^2},
    N = 32, M = 64, R = 24, p = 8, BiCGStab per step): a bounded subset with
    args.batch_per_grid problems of every grid size, one step = the batched
    graph-captured coarse build (mixed mode) plus the device-driven batched
    Parareal solve to tol 1e-8; solves/s = problems per second of device time.
    The full 64-problem batch is this subset scaled by its grid mix."""
    import torch
    from paper_2508_08873_gb300 import api, workloads as W
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ctx = api.Context(local)
    stream = torch.cuda.ExternalStream(ctx.stream, device=torch.device("cuda", local))
    Ps = []
    for m in W.ADV2D_GRIDS:
        for j in range(args.batch_per_grid):
            Ps.append(W.adv2d(len(Ps), m=m))
    ops = [api.Operator.stencil5(ctx, P.mx, P.my, P.st) for P in Ps]
    P0 = Ps[0]
    ctx.set_param("krylov_refine", args.krylov_refine)

    def step():
        ctx.set_kernel_timing(True)
        ctx.reset_kernel_time()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cos = api.build_coarse_batch(ctx, ops, P0.dt, P0.M, P0.N, P0.R, P0.p, 0, prec="mixed")
        e1.record(stream)
        outs, kd = api.parareal_solve_batch(ctx, cos, [P.u0 for P in Ps], K=P0.N, tol=TOL)
        e2.record(stream)
        torch.cuda.synchronize()
        kt = {f: ctx.kernel_time(f) for f in ("propagate_f32", "propagate_f64")}
        ctx.set_kernel_timing(False)
        for co in cos:
            co.close()
        return e0.elapsed_time(e1), e1.elapsed_time(e2), list(kd), outs, kt
    for _ in range(max(1, args.warmup)):
        step()
    ms_b, ms_s = [], []
    for _ in range(args.steps):
        b, sv, kd, outs, kt = step()
        ms_b.append(b)
        ms_s.append(sv)
    ms = statistics.mean(ms_b) + statistics.mean(ms_s)
    line = {"metric": "uneven 2D batch: Parareal solves/s at tol 1e-8 (build + solve)",
            "value": 1000.0 * len(Ps) / ms, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "mode": "batch",
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "adv2d uneven batch, %d problems (%d per grid of %s), N=32, M=64, "
                                   "R=24, p=8, BiCGStab, tol=1e-8" % (len(Ps), args.batch_per_grid,
                                                                       list(W.ADV2D_GRIDS))},
            "build_ms": statistics.mean(ms_b), "solve_ms": statistics.mean(ms_s),
            "fp64_steps": "FP64 Krylov kernels" if args.krylov_refine == 2
                          else "in-kernel iterative refinement (FP32 BiCGStab corrections)",
            "iterations": [int(k) for k in kd], "grids": [P.mx for P in Ps],
            "kernels": {f: {"launches": v[0], "ms_total": v[1]} for f, v in kt.items()}}
    print(json.dumps(line), flush=True)


def run_cfg3(args):
    """The 2D diffusion workload at its own size (511^2, kappa checkerboard,
    N = 128, M = 32, R = 32, p = 10, Jacobi-PCG at rtol 1e-6 for the FP32
    sketches and 1e-12 for the FP64 fine solves).  A full build (~10^4
    propagations of 32 steps) and every Parareal iteration (128 FP64 fine
    solves) take minutes, so the leg measures at full size, on the device:
      * the CG rates of both precisions (us per iteration and system, CG
        iterations per step) on full batches of one step;
      * a complete build with M = 1 (all N intervals, the same sketches,
        orthonormalisation, small SVDs and lift at n = 261121, l = 42): its
        time less its propagation time is the dense part of the build;
      * one Parareal iteration on that build (the coarse sweep's time);
    and states the full-size figures they give:
      T_build = dense + 2 N l M it32 t32,   T_iter = N M it64 t64 + sweep,
      solves/s(k) = 1 / (T_build + k T_iter)."""
    import torch
    from paper_2508_08873_gb300 import api, workloads as W
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ctx = api.Context(local)
    P = W.diff2d()
    kr = krylov_leg(ctx, ["mixed", "f64"], [64, 128], 1, 1)
    op = api.Operator.stencil5(ctx, P.mx, P.my, P.st)
    op.set_krylov(1e-12, 1e-6, 20000)
    ell = P.R + P.p
    api.Coarse(ctx, op, P.dt, 1, P.N, P.R, P.p, P.seed, prec="mixed").close()   # warm-up
    ctx.set_kernel_timing(True)
    ctx.reset_kernel_time()
    t0 = time.perf_counter()
    co = api.Coarse(ctx, op, P.dt, 1, P.N, P.R, P.p, P.seed, prec="mixed")
    torch.cuda.synchronize()
    t_b1 = time.perf_counter() - t0
    kt = {f: ctx.kernel_time(f) for f in ("propagate_f32", "orth", "svd", "lift")}
    ctx.reset_kernel_time()
    u, info = api.parareal_solve(ctx, co, P.u0, K=1)
    sweep = ctx.kernel_time("sweep")
    ctx.set_kernel_timing(False)
    dense = t_b1 - kt["propagate_f32"][1] * 1e-3
    f32, f64 = kr["f32"], kr["f64"]
    prop32 = 2 * P.N * ell * P.M * f32["cg_iterations_per_step"] * f32["us_per_iteration_and_system"] * 1e-6
    t_build = dense + prop32
    # FP64 fine solves: the library's default for this grid (iterative
    # refinement) when measured, else the FP64 Krylov kernel
    us64 = kr["f64_refine"]["us_per_system_step"] if "f64_refine" in kr \
        else f64["cg_iterations_per_step"] * f64["us_per_iteration_and_system"]
    t_iter = P.N * P.M * us64 * 1e-6 + sweep[1] * 1e-3
    t_iter_f64_kernel = P.N * P.M * f64["cg_iterations_per_step"] * f64["us_per_iteration_and_system"] \
        * 1e-6 + sweep[1] * 1e-3
    line = {"metric": "diff2d 511^2 Parareal: build and iteration times at full size (extrapolated "
                      "from full-size measurements)",
            "value": t_build, "unit": "s (build)", "mode": "cfg3", "n_gpus": 1,
            "higher_is_better": False, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "diff2d 511^2 kappa 8x8 checkerboard, N=128, M=32, R=32, p=10, "
                                   "Jacobi-PCG rtol 1e-6 (FP32 sketches) / 1e-12 (FP64 fine)"},
            "krylov": kr,
            "build_M1_s": t_b1, "build_M1_kernels_ms": {f: v[1] for f, v in kt.items()},
            "dense_part_s": dense, "sketch_propagation_s": prop32, "build_s": t_build,
            "sweep_ms": sweep[1], "iteration_s": t_iter,
            "iteration_s_f64_krylov_kernel": t_iter_f64_kernel,
            "solves_per_s": {str(k): 1.0 / (t_build + k * t_iter) for k in (1, 4, 16, P.N)},
            "formula": "T_build = dense + 2 N l M it32 t32; T_iter = N M t64 + sweep (t64 the "
                       "FP64 time per system and step: iterative refinement); "
                       "solves/s(k) = 1 / (T_build + k T_iter)"}
    co.close()
    print(json.dumps(line), flush=True)


def run_extras(args, ctx, op, P, step, stream, u0_d, out_d, flush, world):
    """The legs beside the headline: solves on prebuilt coarse solvers, the
    classical comparator, the two-sided sketch build and the host-buffer (e2e)
    timing through the C ABI."""
    import torch
    from paper_2508_08873_gb300 import api
    # amortised (serving view): solves only, coarse solvers built once
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec=args.prec)
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(args.steps):
        api.parareal_solve(ctx, co, u0_d, K=P.N, tol=TOL, out=out_d, bounds=False)
    a1.record(stream)
    torch.cuda.synchronize()
    amort = 1000.0 * args.steps / a0.elapsed_time(a1)
    # comparison: classical Parareal (one backward-Euler coarse step per
    # interval), same fine solver, stopped on its increment at the same tol
    cls_out = torch.empty_like(out_d)
    api.parareal_solve_classical(ctx, op, P.dt, P.M, P.N, u0_d, K=P.N, tol=TOL, out=cls_out)
    torch.cuda.synchronize()
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    _, cls_info = api.parareal_solve_classical(ctx, op, P.dt, P.M, P.N, u0_d, K=P.N, tol=TOL,
                                               out=cls_out)
    c1.record(stream)
    torch.cuda.synchronize()
    cls_ms = c0.elapsed_time(c1)
    # variant of Sec. 2.2: adjoint sketch on independent random vectors
    ts_out = torch.empty_like(out_d)

    def step_two_sided():
        co2 = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec=args.prec,
                         independent_adjoint=True)
        u2, inf2 = api.parareal_solve(ctx, co2, u0_d, K=P.N, tol=TOL, out=ts_out, bounds=False)
        co2.close()
        return inf2
    step_two_sided()
    torch.cuda.synchronize()
    d0 = torch.cuda.Event(enable_timing=True)
    d1 = torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    ts_info = step_two_sided()
    d1.record(stream)
    torch.cuda.synchronize()
    ts_ms = d0.elapsed_time(d1)
    # ---- e2e: host buffers through the C ABI ---------------------------------
    u0_h = torch.tensor(P.u0, dtype=torch.float64).pin_memory()
    out_h = torch.empty((P.N + 1, P.n), dtype=torch.float64).pin_memory()
    lo_h, di_h, up_h = (torch.tensor(a, dtype=torch.float64).pin_memory() for a in (P.lo, P.di, P.up))
    e2e_ms = []
    for s in range(max(2, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op_h = api.Operator.tridiag(ctx, lo_h.numpy(), di_h.numpy(), up_h.numpy())
        info_h = step(op_h, u0_h.numpy(), out_h.numpy())
        op_h.close()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_val = world * 1000.0 / statistics.mean(e2e_ms)
    # the 1D heat configuration of Experiment 1 (n=255, N=16, M=64, R=8, p=4,
    # source sin(2 pi t) exp(-100 (x - 1/2)^2)): latency-bound, reported in us
    # per solve (to tol 1e-10), with and without the coarse build
    from paper_2508_08873_gb300 import workloads as W
    H = W.heat1d()
    op_h = api.Operator.tridiag(ctx, H.lo, H.di, H.up)
    g_d = torch.tensor(H.g, dtype=torch.float64, device=u0_d.device)
    c_d = torch.tensor(H.c, dtype=torch.float64, device=u0_d.device)
    hu0 = torch.tensor(H.u0, dtype=torch.float64, device=u0_d.device)
    hout = torch.empty((H.N + 1, H.n), dtype=torch.float64, device=u0_d.device)

    def heat_step(build):
        co_h = api.Coarse(ctx, op_h, H.dt, H.M, H.N, H.R, H.p, H.seed, prec=args.prec) \
            if build else heat_step.co
        _, inf_h = api.parareal_solve(ctx, co_h, hu0, g_d, c_d, K=H.N, tol=1e-10, out=hout,
                                      bounds=False)
        if build:
            co_h.close()
        return inf_h
    heat_step.co = api.Coarse(ctx, op_h, H.dt, H.M, H.N, H.R, H.p, H.seed, prec=args.prec)
    heat = {}
    for build in (True, False):
        for _ in range(2):
            heat_step(build)
        torch.cuda.synchronize()
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        reps = 10
        for _ in range(reps):
            inf_h = heat_step(build)
        h1.record(stream)
        torch.cuda.synchronize()
        heat["us_per_solve_with_build" if build else "us_per_solve"] = \
            1000.0 * h0.elapsed_time(h1) / reps
    heat["iterations"] = inf_h["k_done"]
    heat["workload"] = "heat1d n=255 N=16 M=64 R=8 p=4 tol=1e-10"
    heat_step.co.close()
    return {"amortised_solves_per_s": amort * world,
            "heat1d": heat,
            "two_sided_sketch": {"iterations": ts_info["k_done"], "solves_per_s": 1000.0 / ts_ms,
                                 "rel_err_vs_oracle": None,
                                 "note": "build_coarse with F'^* on 2(R+p) independent random "
                                         "vectors (Sec. 2.2 variant) + the same solve"},
            "classical_parareal": {"iterations": cls_info["k_done"],
                                   "solves_per_s": 1000.0 / cls_ms,
                                   "rel_err_vs_oracle": None,
                                   "note": "one backward-Euler coarse step per interval, "
                                           "stopped on its increment at the same tol"},
            "e2e": {"value": e2e_val, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * (P.n + 3 * P.n),
                    "d2h_bytes_per_step": 8 * (P.N + 1) * P.n},
            "cls_out": cls_out, "ts_out": ts_out}


def run_exp3(args):
    """Experiment 3's time-dependent 2D heat equation at its own size (99^2
    grid, N = 10 intervals of M = 10 steps, R = 6, p = 1; every fine step its
    own operator): one step = the mixed coarse build + the Parareal solve to
    tol 1e-8, backward Euler and the SDIRK2-L stepper (the operator at both
    stage times), CUDA events on the library's stream; the error of the last
    timed result against the oracle's sequential FP64 fine solution."""
    import torch
    from paper_2508_08873_gb300 import api, workloads as W
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ctx = api.Context(local)
    stream = torch.cuda.ExternalStream(ctx.stream, device=torch.device("cuda", local))
    P = W.heat2d_td()
    legs = {}
    outs = {}
    for scheme in ("be", "sdirk2l"):
        if scheme == "be":
            st, c = P.extra["st_t"], P.c
        else:
            gam = (2.0 - 2.0 ** 0.5) / 2.0        # SDIRK2-L stage times t_J + (gamma, 1) dt
            ts = np.array([[(J + cs) * P.dt for cs in (gam, 1.0)] for J in range(P.N * P.M)]).ravel()
            st = W.heat2d_td_at(P.mx, ts)
            c = np.sin(5 * np.pi * ts).reshape(P.N * P.M, 2, 1)
        op = api.Operator.stencil5_td(ctx, P.mx, P.my, st, stepper=scheme)

        def step():
            co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="mixed")
            u, info = api.parareal_solve(ctx, co, P.u0, P.g, c, K=P.N, tol=1e-8)
            co.close()
            return u, info

        for _ in range(max(1, args.warmup)):
            step()
        ms = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            u, info = step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        outs[scheme] = (u, st, c)
        legs[scheme] = {"ms_per_step": statistics.mean(ms), "solves_per_s": 1e3 / statistics.mean(ms),
                        "iterations": info["k_done"], "final_bound": info["final_bound"],
                        "krylov_iterations_total": op.krylov_iterations()}
        op.close()
    if rank == 0:
        from oracle import oracle as orc
        for scheme, (u, st, c) in outs.items():
            oop = orc.Stencil5TD(P.mx, P.my, *(st[k] for k in "CWESN"), stepper=scheme)
            ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0, P.g, c)
            legs[scheme]["rel_err_vs_oracle"] = orc.rel_err(u, ref)
    be = legs["be"]
    line = {"metric": "Parareal solves/s at 1e-8 rel err vs FP64 oracle", "value": be["solves_per_s"],
            "unit": "solves/s", "mode": "exp3", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": be["ms_per_step"], "higher_is_better": True,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "heat2d_td 99^2 (Experiment 3: time-dependent conductivity, "
                                   "source) N=10 M=10 R=6 p=1 tol=1e-8",
                       "step": "build_coarse (mixed) + parareal_solve"},
            "backward_euler": be, "sdirk2l": legs["sdirk2l"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def fine_roofline(P, kern, k_list, ms_step, steps, rounds):
    """Roofline entry of the dominant kernel family of the headline step.
    Algorithmic flops per row and step: the FP64 kernels, Thomas with
    precomputed pivots (5: one FMA forward, one MUL and one FMA backward);
    the refined FP32 kernel, per step one solve (5) and per round a solve (5),
    the pair residual (3 split products 9, six low-part FMAs 12, three
    two-sums 18, the tail 7) and the pair update (9): 5 + 60 R."""
    fam = max(("propagate_f64", "propagate_f32"), key=lambda f: kern[f][1])
    nl, tot = kern[fam]
    k_mean = statistics.mean(k_list)
    systems_per_step = (P.N * k_mean - k_mean * (k_mean - 1) / 2) if fam == "propagate_f64" \
        else 2 * P.N * (P.R + P.p)
    per_row = (5.0 + 60.0 * rounds) if (fam == "propagate_f64" and rounds) else 5.0
    flops_step = per_row * P.n * P.M * systems_per_step
    launches_per_step = nl / steps
    achieved = flops_step / (tot / steps) / 1e6 if tot > 0 else 0.0   # GFLOP/s
    refined = fam == "propagate_f64" and rounds > 0
    peak = FP32_PEAK_GFLOPS if (refined or fam == "propagate_f32") else FP64_PEAK_GFLOPS
    # per-launch figures over the launches that propagate (one per Parareal
    # iteration; the launches enqueued after the device-side stop return at
    # once and are counted apart)
    real_launches = k_mean if fam == "propagate_f64" else launches_per_step
    systems_per_launch = systems_per_step / max(real_launches, 1)
    # DRAM traffic of the FP64 fine-solve kernel, from one ncu capture on GB300
    # (dram__bytes_read.sum + dram__bytes_write.sum of a 62-system launch of
    # the 12-row-chunk variant: 2.31 MB read, nothing written back within the
    # launch), per propagated system, times this run's systems per launch; of
    # the refined kernel from its own capture (one 62-system launch)
    traffic = None
    if fam == "propagate_f64":
        per_sys = IRT_DRAM_BYTES_PER_SYSTEM if refined else F64_DRAM_BYTES_PER_SYSTEM
        traffic = per_sys * systems_per_launch if per_sys else None
    return {"bound": "alu", "kernel": ("k_tri_irt (FP32 + pair residuals)" if refined else fam),
            "achieved": achieved / 1e3, "peak": peak / 1e3,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "flops_per_row_step": per_row,
            "algorithmic_bytes": 16.0 * P.n * systems_per_launch,
            "systems_per_launch": systems_per_launch,
            "launches_per_step": launches_per_step,
            "noop_launches_per_step": launches_per_step - real_launches,
            "share_of_step": (tot / steps) / ms_step,
            "peak_note": "FP64: 152 SMs x 2 FMA/clk x 2.07 GHz nominal (a throughput probe "
                         "reaches 1.6 FMA/clk/SM = 1.007 TFLOP/s); FP32: 128 FMA/clk/SM; the "
                         "refined kernel holds one system per SM (62 of 152 SMs at 62 systems)"}


# FP64 FMA issue probe: one CTA of w warps per SM, 8 independent FMA chains
# per thread, `active` lanes of each warp computing (the others branch past
# the loop); printed as one JSON list by the probe program
FP64_PROBE_SRC = r"""
#include <cstdio>
#include <cuda_runtime.h>
__global__ void k_fp64_fma(double* out, int iters, int active) {
  const int lane = threadIdx.x & 31;
  double a[8];
  for (int c = 0; c < 8; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  const double x = 0.9999999, y = 1e-7;
  if (lane < active) {
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int c = 0; c < 8; ++c) a[c] = fma(a[c], x, y);
    }
  }
  double s = 0.0;
  for (int c = 0; c < 8; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return 1;
  double* out = nullptr;
  if (cudaMalloc(&out, (size_t)sms * 512 * sizeof(double)) != cudaSuccess) return 1;
  const int iters = 1 << 15;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int ws[] = {1, 2, 3, 4, 5, 6, 8};
  const int acts[] = {1, 8, 32};
  printf("[");
  bool first = true;
  for (int w : ws)
    for (int act : acts) {
      k_fp64_fma<<<sms, 32 * w>>>(out, iters, act);
      cudaEventRecord(e0);
      k_fp64_fma<<<sms, 32 * w>>>(out, iters, act);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess) return 2;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      printf("%s{\"warps_per_sm\": %d, \"active_lanes\": %d, \"ms\": %.6f, \"sms\": %d, "
             "\"warp_fma_per_sm\": %.1f}", first ? "" : ", ", w, act, ms, sms, 8.0 * iters * w);
      first = false;
    }
  printf("]\n");
  cudaFree(out);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
"""


def run_fp64probe(args):
    """FP64 FMA issue rate of GB300 (the facts behind the FP64 roofline):
    warps per SM 1..8 (one CTA per SM) with 1, 8 or 32 active lanes; per
    case the FP64 warp instructions and lanes each SM retires per cycle at
    the SM clock sampled during the probe.  Compiles the probe with nvcc."""
    import tempfile
    rank, world, local = dist_env()
    if rank != 0:
        return
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "probe.cu")
        exe = os.path.join(td, "probe")
        with open(src, "w") as f:
            f.write(FP64_PROBE_SRC)
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src],
                       check=True)
        clocks = ClockSampler(local)
        clocks.start()
        res = subprocess.run([exe], check=True, capture_output=True, text=True,
                             env=dict(os.environ, CUDA_VISIBLE_DEVICES=str(local)))
        clk = clocks.stop()
    rows = json.loads(res.stdout)
    mhz = clk.get("sm_mhz") or 2070.0
    for r in rows:
        cycles = r["ms"] * 1e-3 * mhz * 1e6
        r["warp_fma_per_clk_per_sm"] = r["warp_fma_per_sm"] / cycles
        r["lanes_per_clk_per_sm"] = r["warp_fma_per_clk_per_sm"] * r["active_lanes"]
        r["cycles_per_warp_fma_per_subpartition"] = min(r["warps_per_sm"], 4) / r["warp_fma_per_clk_per_sm"]
    full = [r for r in rows if r["active_lanes"] == 32]
    best = max(full, key=lambda r: r["lanes_per_clk_per_sm"])
    line = {"metric": "FP64 FMA lanes per clock per SM", "mode": "fp64probe", "n_gpus": 1,
            "value": best["lanes_per_clk_per_sm"], "unit": "lanes/clk/SM", "higher_is_better": True,
            "data": "synthetic", "clocks": clk,
            "fp64_tflops_at_best": best["lanes_per_clk_per_sm"] * 2 * best["sms"] * mhz * 1e-6,
            "table": rows}
    print(json.dumps(line), flush=True)


def run_trisweep(args):
    """CUDA-event time per launch of the FP64 fine-solve kernels on adr1d
    (n = 4095, 256 steps) over batch sizes and chunk lengths: the general
    one-warp cluster kernel (tri_wtoep = 2) and its constant-coefficient
    variant (tri_wtoep = 1, chunk lengths with n mod MM in {0, MM - 1}), the
    table the library's chunk rule was read from."""
    import torch
    from paper_2508_08873_gb300 import api, workloads as W
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ctx = api.Context(local)
    P = W.adr1d()
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    rng = np.random.default_rng(0)
    table = {}
    for nsys in [int(v) for v in args.sweep_systems.split(",")]:
        X = torch.from_numpy(rng.standard_normal((nsys, P.n))).cuda()
        Y = torch.empty_like(X)
        row = {}
        for mm in [int(v) for v in args.sweep_chunks.split(",")]:
            for toep, key in ((2, "general"), (1, "constant")):
                if toep == 1 and P.n % mm and (P.n + 1) % mm:
                    continue
                ctx.set_param("tri_wchunk", mm)
                ctx.set_param("tri_warp", 2)
                ctx.set_param("tri_wtoep", toep)
                try:
                    for _ in range(max(1, args.warmup)):
                        api.propagate(ctx, op, P.dt, P.M, X, out=Y)
                    ctx.set_kernel_timing(True)
                    ctx.reset_kernel_time()
                    for _ in range(args.steps):
                        api.propagate(ctx, op, P.dt, P.M, X, out=Y)
                    nl, ms = ctx.kernel_time("propagate_f64")
                    ctx.set_kernel_timing(False)
                    row.setdefault(key, {})[str(mm)] = ms / max(nl, 1)
                finally:
                    ctx.set_param("tri_wchunk", 0)
                    ctx.set_param("tri_warp", 0)
                    ctx.set_param("tri_wtoep", 0)
        # the library's own choice for this batch
        for _ in range(max(1, args.warmup)):
            api.propagate(ctx, op, P.dt, P.M, X, out=Y)
        ctx.set_kernel_timing(True)
        ctx.reset_kernel_time()
        for _ in range(args.steps):
            api.propagate(ctx, op, P.dt, P.M, X, out=Y)
        nl, ms = ctx.kernel_time("propagate_f64")
        ctx.set_kernel_timing(False)
        row["default"] = ms / max(nl, 1)
        # FP32 solves refined by pair residuals (tri_refine = 1), per round
        # count: time per launch and the largest relative difference from the
        # FP64 kernel's result
        Yr = torch.empty_like(X)
        for rounds, (vname, clus, chunk) in [(int(v), var) for v in args.sweep_refine.split(",") if v
                                             for var in (("", 0, 0), ("_cta8", 0, 8), ("_cta12", 0, 12),
                                                         ("_cluster", 1, 0))]:
            ctx.set_param("tri_refine", 1)
            ctx.set_param("tri_refine_rounds", rounds)
            ctx.set_param("tri_refine_cluster", clus)
            ctx.set_param("tri_wchunk", chunk)
            try:
                for _ in range(max(1, args.warmup)):
                    api.propagate(ctx, op, P.dt, P.M, X, out=Yr)
                ctx.set_kernel_timing(True)
                ctx.reset_kernel_time()
                for _ in range(args.steps):
                    api.propagate(ctx, op, P.dt, P.M, X, out=Yr)
                nl, ms = ctx.kernel_time("propagate_f64")
                ctx.set_kernel_timing(False)
            finally:
                ctx.set_param("tri_refine", 0)
                ctx.set_param("tri_refine_rounds", 2)
                ctx.set_param("tri_refine_cluster", 0)
                ctx.set_param("tri_wchunk", 0)
            d = (torch.linalg.vector_norm(Yr - Y, dim=1) / torch.linalg.vector_norm(Y, dim=1)).max()
            row["refine_%d%s" % (rounds, vname)] = {"ms": ms / max(nl, 1), "max_rel_diff_vs_f64": float(d)}
        table[str(nsys)] = row
    line = {"metric": "FP64 fine-solve kernel time per launch (adr1d n=4095, M=256)",
            "unit": "ms", "mode": "trisweep", "n_gpus": 1, "higher_is_better": False,
            "dtype": "f64", "data": "synthetic", "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "adr1d n=4095 M=256, FP64, one-warp cluster kernels"},
            "table": table}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.mode == "trisweep":
        run_trisweep(args)
        return
    if args.mode == "fp64probe":
        run_fp64probe(args)
        return
    if args.mode == "exp3":
        run_exp3(args)
        return
    if args.mode == "serve":
        run_serve(args)
        return
    if args.mode == "krylov":
        run_krylov(args)
        return
    if args.mode == "batch":
        run_batch(args)
        return
    if args.mode == "cfg3":
        run_cfg3(args)
        return
    from paper_2508_08873_gb300 import workloads as W
    P = W.adr1d()
    K_ITERS_REF = 29          # iterations the tol-1e-8 solve performs (measured on the oracle)
    if args.impl == "reference":
        run_reference(args, P, K_ITERS_REF)
        return

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2508_08873_gb300 import api

    ctx = api.Context(local)
    if args.tri_refine:
        ctx.set_param("tri_refine", 1)
        ctx.set_param("tri_refine_rounds", args.tri_refine)
    stream = torch.cuda.ExternalStream(ctx.stream, device=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    u0_d = torch.tensor(P.u0, dtype=torch.float64, device=dev)
    out_d = torch.empty((P.N + 1, P.n), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)

    def step(op_, u0, out):
        co = api.Coarse(ctx, op_, P.dt, P.M, P.N, P.R, P.p, P.seed, prec=args.prec)
        u, info = api.parareal_solve(ctx, co, u0, K=P.N, tol=TOL, out=out, bounds=False)
        co.close()
        return info

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    for _ in range(args.warmup):
        info = step(op, u0_d, out_d)
    # ---- timed region (device time, inputs resident) -------------------------
    ctx.set_kernel_timing(True)
    ctx.reset_kernel_time()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    ev = []
    launches0 = ctx.launch_count()
    k_list = []
    t_wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = step(op, u0_d, out_d)
        e1.record(stream)
        ev.append((e0, e1))
        k_list.append(info["k_done"])
    barrier()
    t_wall = time.perf_counter() - t_wall0
    launches = ctx.launch_count() - launches0
    ms = [a.elapsed_time(b) for a, b in ev]
    kern = {f: ctx.kernel_time(f) for f in ("propagate_f64", "propagate_f32", "sweep", "orth",
                                            "svd", "lift")}
    ctx.set_kernel_timing(False)
    clk = clocks.stop()
    ms_step, value = aggregate_over_ranks(statistics.mean(ms), world, dev)
    # ---- the same step with the other fine solves: the refined FP32 steps
    # (one pair-residual round) beside the FP64 kernels, or the reverse -------
    alt = None
    alt_rounds = 0 if args.tri_refine else 1
    if not args.headline_only:
        ctx.set_param("tri_refine", 1 if alt_rounds else 0)
        ctx.set_param("tri_refine_rounds", max(alt_rounds, 1))
        out_alt = torch.empty_like(out_d)
        for _ in range(max(2, args.warmup // 2)):
            step(op, u0_d, out_alt)
        ctx.set_kernel_timing(True)
        ctx.reset_kernel_time()
        barrier()
        ev_alt, k_alt = [], []
        for s in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info_alt = step(op, u0_d, out_alt)
            e1.record(stream)
            ev_alt.append((e0, e1))
            k_alt.append(info_alt["k_done"])
        barrier()
        kern_alt = {f: ctx.kernel_time(f) for f in ("propagate_f64", "propagate_f32")}
        ctx.set_kernel_timing(False)
        ctx.set_param("tri_refine", 1 if args.tri_refine else 0)
        ctx.set_param("tri_refine_rounds", max(args.tri_refine, 1))
        ms_alt, value_alt = aggregate_over_ranks(statistics.mean([a.elapsed_time(b) for a, b in ev_alt]),
                                             world, dev)
        alt = {"solves_per_s": value_alt, "ms_per_step": ms_alt, "iterations": k_alt[-1],
                "fine": ("FP32 solves, one pair-residual correction round per step (k_tri_irt; "
                         "about 48-bit steps, not the FP64 arithmetic of the workload)")
                        if alt_rounds else "FP64 one-warp cluster kernels",
                "roofline": fine_roofline(P, kern_alt, k_alt, ms_alt, args.steps, alt_rounds), "out": out_alt}
    if args.headline_only:
        extras = None
    else:
        extras = run_extras(args, ctx, op, P, step, stream, u0_d, out_d, flush, world)
        ctx.set_param("tri_refine", 0)        # all FP64: the FP64 fine-solve kernels
        extras["all_fp64"] = all_fp64_leg(args, ctx, op, P, stream, flush)
        ctx.set_param("tri_refine", 1 if args.tri_refine else 0)
        extras["krylov_hbm_frac"] = krylov_leg(ctx, ["mixed", "f64"], [64, 16], 3, 1)
        extras["serve"] = serve_leg(ctx, [10.0, 30.0, 100.0], 3.0, quiet=True,
                                    targets=[(100.0, 1000.0)])
    # ---- accuracy of the timed solve vs the oracle's sequential fine solution -
    err = None
    if rank == 0:
        from oracle import oracle as orc
        ref = orc.sequential_fine(orc.Tridiag(P.lo, P.di, P.up), P.dt, P.M, P.N, P.u0)
        err = orc.rel_err(out_d.cpu().numpy(), ref)
        if extras is not None:
            extras["classical_parareal"]["rel_err_vs_oracle"] = orc.rel_err(
                extras.pop("cls_out").cpu().numpy(), ref)
            extras["two_sided_sketch"]["rel_err_vs_oracle"] = orc.rel_err(
                extras.pop("ts_out").cpu().numpy(), ref)
            extras["all_fp64"]["rel_err_vs_oracle"] = orc.rel_err(
                extras["all_fp64"].pop("out").cpu().numpy(), ref)
        if alt is not None:
            alt["rel_err_vs_oracle"] = orc.rel_err(alt.pop("out").cpu().numpy(), ref)
    # ---- roofline of the dominant kernel ---------------------------------------
    roof = fine_roofline(P, kern, k_list, ms_step, args.steps, args.tri_refine)
    kernels = {f: {"launches": v[0], "ms_total": v[1]} for f, v in kern.items()}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_entry(P, 0.4 * args.cpu_budget, K_ITERS_REF, 0)
        cpu["one_core"] = cpu_baseline_entry(P, 0.6 * args.cpu_budget, K_ITERS_REF, 1)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.prec == "f64" else "f32+f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "precision": args.prec,
                           "step": "build_coarse + parareal_solve(tol=1e-8)",
                           "l2": "flushed (256 MB write) between timed steps",
                           "parallelism": "replicas" if world > 1 else "1 GPU"},
                "iterations": k_list[-1], "rel_err_vs_oracle": err,
                "fine_solves": ("FP32 solves, %d pair-residual correction round(s) per step "
                                "(k_tri_irt)" % args.tri_refine) if args.tri_refine
                               else "FP64 one-warp cluster kernels",
                ("fine_f64_kernel" if args.tri_refine else "fine_refined"): alt,
                **(extras or {"e2e": None}),
                "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
                "roofline": roof, "kernels": kernels, "clocks": clk, "cpu_baseline": cpu,
                "wall_s_timed": t_wall}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
