#!/usr/bin/env python
"""Benchmark of the collision-resolution hot path on GB300.

Metric: LCP solves per second (and p50/p99 latency) on synthetic packings of
216 Janus spheres with 11 x 22 nodes each (52 272 nodes, 156 816 unknowns),
solved by mixed-precision Bi-PQN (FP32 stresslet sums, FP64 GMRES refinement
to 1e-12) to ||min(x, A x + b)||_2 <= 1e-8.  One step is one full collision
resolution of a fresh configuration: geometry, contacts and D, the slip
solve for U_nc and b, then the LCP solve (every row of the hot path).

The plain FP64 Mono-PQN GPU solve of the same configuration is timed once
beside it (--fp64-compare), and the CPU oracle is timed on a bounded sample
of the same workload on the host cores (cpu_baseline).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 run under torch.distributed.run: every rank solves its own
configurations (weak scaling, no collective on the data path); the extra
reports (plain-FP64 comparison, method comparison, trajectory, 64-sphere,
batched and serving runs, CPU baseline) run at N = 1 only.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# FP32 pair-sum kernel: 32 flops per node pair (r, |r|^2, r.n, phi_q - phi_p, r.d,
# the |r|^-5 scaling and the accumulation), plus one reciprocal square root.
FLOPS_PER_PAIR = 32
# Roofline denominator for plain FP32 ALU work: 152 SMs x 128 FP32 lanes x 2 flops
# (FMA) x 2.070 GHz maximum SM clock.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_PEAK_TFLOPS = FP32_PEAK_TFLOPS / 64.0
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# FP32 pair kernel at 216 spheres x 242 nodes, from an ncu capture, with the SHA-1 of
# the device code it was taken on (reported as null once that code changes; for the
# symmetric kernels the hashed code is the pair kernels' part of their file, before the
# finish kernel).
PAIR32_TRAFFIC = {
    "k_pair32_sym_p8rc5": {"file": "stokes_sym.cu", "source_sha1": "7c3da54fa3fcd6dd382fc924582e9560bd3f70e5",
                           "bytes_per_launch": 1042432},
    "k_pair32": {"file": "stokes.cu", "source_sha1": "298b391165dc32f4d22c484bf6d970a4f86ee95e",
                 "bytes_per_launch": 665088},
}
# FP32 operations of the symmetric kernel per unordered node pair (both ordered
# terms): r 3, |r|^2 6, |r|^-2 1, d 3, r.d 5, t 3, r.wn_q 5, r.wn_p 5, scales 2,
# two accumulations 12 = 45 flops (FMA = 2), i.e. 22.5 per ordered pair; the
# variants that take |r|^-2 from a reciprocal ("rc" in the name) do one
# multiply fewer: 44, i.e. 22 per ordered pair.
SYM_FLOPS_PER_ORDERED_PAIR = 22.5
SYM_RC_FLOPS_PER_ORDERED_PAIR = 22.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=6)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="spheres216_grid11x22")
    p.add_argument("--method", default="bi", choices=["bi", "mono"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--lowfi", default="auto",
                   help="Bi-PQN low-fidelity operator: rpy, a coarse boundary-integral grid NTxNP (e.g. 8x16), "
                        "or auto = (n_theta - 3) x 2(n_theta - 3) of the workload's grid")
    p.add_argument("--lowfi-min-bodies", type=int, default=8,
                   help="batched/serving modes: use --lowfi only for instances with at least this many spheres")
    p.add_argument("--warm-start", type=int, default=None,
                   help="trajectory warm starts (1 slip solve, 2 LCP forces, 3 both); default: the library's")
    p.add_argument("--self-quadrature", type=int, default=1,
                   help="1: high-order self-interaction quadrature (one 3ns x 3ns correction per body)")
    p.add_argument("--inner-tol", type=float, default=1e-6,
                   help="relative tolerance of each FP32-operator refinement sweep (mixed precision)")
    p.add_argument("--recycle", type=int, default=0,
                   help="solve pairs kept for projected starts of the mobility solves (0 = off)")
    p.add_argument("--fp64-compare", type=int, default=1)
    p.add_argument("--cpu-baseline", type=int, default=1)
    p.add_argument("--compare-methods", type=int, default=1,
                   help="also solve the first timed configuration with BB-PGD, Mono-PQN and Bi-PQN (mixed)")
    p.add_argument("--e2e", type=int, default=1)
    p.add_argument("--mode", default="solve", choices=["solve", "batched", "serving"],
                   help="solve: the headline metric; batched: 256 uneven instances solved together; "
                        "serving: Poisson requests from 32 concurrent simulations")
    p.add_argument("--batch-count", type=int, default=256)
    p.add_argument("--workers", type=int, default=12)
    p.add_argument("--sims", type=int, default=32)
    p.add_argument("--sim-steps", type=int, default=10)
    p.add_argument("--arrival-rate", type=float, default=8.0, help="requests/s per simulation (Poisson)")
    p.add_argument("--budget-frac", type=float, default=0.5, help="HBM budget as a fraction of all contexts")
    p.add_argument("--fp64-baseline", type=int, default=1,
                   help="batched/serving modes: time plain FP64 Mono-PQN on every instance, one at a time")
    p.add_argument("--trajectory", type=int, default=100,
                   help="also time this many forward-Euler steps (solve + lcp_step) of one configuration, with "
                        "the warm-started slip solve, and the first --trajectory-cold of them cold-started")
    p.add_argument("--trajectory-cold", type=int, default=10)
    p.add_argument("--c4c5", type=int, default=1,
                   help="also run the batched (256 instances) and serving (32 simulations) configurations "
                        "once and add their results to the line")
    p.add_argument("--c2", type=int, default=1,
                   help="64-sphere report: Mono vs Bi-PQN, FP64 vs mixed, high-fidelity MVPs and the error "
                        "against the FP64 oracle")
    return p.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_sha1(kernel: str) -> str:
    """SHA-1 of the device code a traffic figure was taken on."""
    import hashlib
    info = PAIR32_TRAFFIC[kernel]
    with open(os.path.join(ROOT, "paper_2604_10089_gb300", "csrc", info["file"]), "rb") as f:
        text = f.read()
    if info["file"] == "stokes.cu":   # pair2 .. the plain variant table
        a = text.find(b"__device__ __forceinline__ void pair2(")
        b = text.find(b"constexpr int kNumPair32Variants")
    else:                              # the pair kernels: everything before the finish kernel
        a, b = 0, text.find(b"// out_p = forward partials")
    return hashlib.sha1(text[a:b] if 0 <= a < b else text).hexdigest()


def lowfi_overrides(spec: str, n_theta: int = 0) -> dict:
    """Config fields of the low-fidelity operator: {} for RPY, else the coarse grid."""
    if spec == "rpy":
        return {}
    if spec == "auto":   # measured optimum at 64 and 216 spheres: grid n_theta - 3, FP32 GMRES to 1e-4
        nt = n_theta - 3
        if nt < 6:       # coarser grids do not resolve neighbouring spheres: RPY
            return {}
        return {"lowfi_n_theta": nt, "lowfi_n_phi": 2 * nt, "lowfi_tol": 1e-4, "init_forcing": 1e-3}
    nt, nph = (int(v) for v in spec.lower().split("x"))
    return {"lowfi_n_theta": nt, "lowfi_n_phi": nph}


def instance_lowfi(args, inst) -> dict:
    """Batched and serving modes: the coarse-grid low fidelity (--lowfi) for instances of at
    least --lowfi-min-bodies spheres, where it cuts high-fidelity MVPs; RPY below (and wherever
    the coarse grid would not resolve neighbouring spheres)."""
    return lowfi_overrides(args.lowfi, inst.n_theta) if inst.n_bodies >= args.lowfi_min_bodies else {}


def batch_lowfi_description(args) -> str:
    if args.lowfi == "rpy" or args.lowfi_min_bodies >= 10 ** 9:
        return "rpy"
    return (f"coarse grid ({args.lowfi}: n_theta - 3 for 9 x 18 spheres) for instances of at least "
            f"{args.lowfi_min_bodies} spheres where it resolves neighbours (>= 6 x 12), else rpy")


def pair32_kernel_name(variant: str) -> str:
    return "k_pair32" if variant == "t2c8" else "k_pair32_" + variant


def rank_seeds(rank: int, count: int) -> list:
    """Instance indices of one rank: disjoint across ranks (weak scaling, no shared data)."""
    return [rank * 1000 + i for i in range(count)]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank time over all ranks (the slowest rank sets the job time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def pct(v, q):
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


def run_ours(args, rank, world, local):
    import torch

    import paper_2604_10089_gb300 as L
    from workloads import make_instance

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    n_inst = args.warmup + args.steps
    insts = [make_instance(args.workload, k) for k in rank_seeds(rank, n_inst)]
    prec = L.LCP_MIXED if args.precision == "mixed" else L.LCP_FP64
    method = L.LCP_BI_PQN if args.method == "bi" else L.LCP_MONO_PQN
    lowfi = lowfi_overrides(args.lowfi, insts[0].n_theta)
    extra = {} if args.warm_start is None else {"warm_start": args.warm_start}
    cfg = L.config_for(insts[0], prec, cuda_stream=stream.cuda_stream, recycle=args.recycle,
                       inner_tol=args.inner_tol, self_quadrature=args.self_quadrature, **extra, **lowfi)
    tol = insts[0].tol
    with torch.cuda.stream(stream):
        cen = [torch.tensor(i.centers, dtype=torch.float64, device=dev) for i in insts]
        axs = [torch.tensor(i.axes, dtype=torch.float64, device=dev) for i in insts]
    stream.synchronize()
    ctx = L.lcp_setup(cfg, insts[0].centers, insts[0].axes)
    variant = L.lcp_kernel_variant(ctx)
    M, N, _ = L.lcp_sizes(ctx)
    xbuf = torch.empty(M * (M - 1) // 2, dtype=torch.float64, device=dev)
    stats = []

    def step(k):
        L.lcp_update_dev(ctx, cen[k], axs[k])
        _, _, n = L.lcp_sizes(ctx)
        st, _ = L.lcp_solve_dev(ctx, method, tol, None, xbuf[:n])
        return st, n

    for k in range(args.warmup):
        step(k)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    L.lcp_profile(ctx, True)
    launches0 = L.lcp_launch_count(ctx)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    ncon = []
    for k in range(args.steps):
        st, n = step(args.warmup + k)
        ev[k + 1].record(stream)
        stats.append(st)
        ncon.append(n)
    torch.cuda.synchronize()
    launches = L.lcp_launch_count(ctx) - launches0
    c32, t32 = L.lcp_profile_read(ctx, 0)
    c64, t64 = L.lcp_profile_read(ctx, 1)
    cdf, tdf = L.lcp_profile_read(ctx, 2)
    L.lcp_profile(ctx, False)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    lat = [ev[k].elapsed_time(ev[k + 1]) / 1e3 for k in range(args.steps)]
    t_total = ev[0].elapsed_time(ev[-1]) / 1e3
    t_total = max_over_ranks(t_total, dev)

    # end to end through the host API: host centres/axes in, host x out
    e2e = None
    if args.e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hb_in = hb_out = 0
        for k in range(args.steps):
            inst = insts[args.warmup + k]
            L.lcp_update(ctx, inst.centers, inst.axes)
            x, _, _ = L.lcp_solve(ctx, method, tol)
            hb_in += inst.centers.nbytes + inst.axes.nbytes
            hb_out += x.nbytes
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e = {"value": args.steps * world / te if rank == 0 else None, "unit": "LCP solves/s",
               "h2d_bytes_per_step": hb_in // args.steps, "d2h_bytes_per_step": hb_out // args.steps}

    # plain FP64 Mono-PQN on the first timed configuration, and agreement with it
    fp64 = None
    if args.fp64_compare and rank == 0 and world == 1:
        cfg64 = L.config_for(insts[0], L.LCP_FP64, recycle=0)   # the paper's method as printed
        ctx64 = L.lcp_setup(cfg64, insts[args.warmup].centers, insts[args.warmup].axes)
        t0 = time.perf_counter()
        x64, st64, _ = L.lcp_solve(ctx64, L.LCP_MONO_PQN, tol)
        t64s = time.perf_counter() - t0
        L.lcp_destroy(ctx64)
        L.lcp_update(ctx, insts[args.warmup].centers, insts[args.warmup].axes)
        xm, stm, _ = L.lcp_solve(ctx, method, tol)
        thr = 1e-9 * max(1.0, float(np.abs(x64).max()))
        fp64 = {"method": "mono_pqn", "precision": "fp64", "solves_per_s": 1.0 / t64s,
                "solve_seconds": t64s, "hi_mvps": st64["hi_mvps"], "gmres_iterations": st64["gmres_iterations"],
                "max_abs_diff_vs_ours": float(np.abs(xm - x64).max()),
                "same_active_set": bool(np.array_equal(xm > thr, x64 > thr)),
                "kkt_fp64": st64["kkt_abs"], "kkt_ours": stm["kkt_abs"]}
    # the paper's comparison on this workload: high-fidelity MVPs and time per solve
    comparison = None
    if args.compare_methods and rank == 0 and world == 1:
        comparison = {}
        inst = insts[args.warmup]
        runs = [("bb_pgd", L.LCP_BB_PGD, ctx), ("mono_pqn", L.LCP_MONO_PQN, ctx), ("bi_pqn", L.LCP_BI_PQN, ctx)]
        # Bi-PQN with the other low-fidelity operator (RPY vs the coarse 6 x 12 grid)
        other = {} if lowfi else lowfi_overrides("auto", inst.n_theta)
        ctx_o = L.lcp_setup(L.config_for(inst, prec, cuda_stream=stream.cuda_stream, **other), inst.centers, inst.axes)
        runs.append(("bi_pqn_" + ("rpy" if lowfi else "coarse_grid"), L.LCP_BI_PQN, ctx_o))
        for name, meth, c in runs:
            L.lcp_update(c, inst.centers, inst.axes)
            ts = time.perf_counter()
            _, st, status = L.lcp_solve(c, meth, tol, allow_not_converged=True)
            comparison[name] = {"hi_mvps": st["hi_mvps"], "lo_mvps": st["lo_mvps"], "e_mvps": round(st["e_mvps"], 3),
                                "iterations": st["iterations"], "seconds": time.perf_counter() - ts,
                                "converged": st["converged"] == 1}
        L.lcp_destroy(ctx_o)
    traj = None
    if args.trajectory and rank == 0 and world == 1:
        inst = insts[args.warmup]

        def trajectory(c, steps):
            L.lcp_update(c, inst.centers, inst.axes)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hi = lo = 0
            kkts, ncs, unc, warm, warm_x = [], [], [], [], []
            for _ in range(steps):
                _, st, _ = L.lcp_solve(c, method, tol)
                hi += st["hi_mvps"]
                lo += st["lo_mvps"]
                kkts.append(st["kkt_abs"])
                ncs.append(L.lcp_sizes(c)[2])
                unc.append(st["unc_gmres_iterations"])
                warm.append(st["unc_warm_started"])
                warm_x.append(st["warm_x0"])
                L.lcp_step(c, inst.dt)
            torch.cuda.synchronize()
            tt = time.perf_counter() - t0
            # the first slip solve of a trajectory comes from lcp_update (never warm-started)
            later = unc[1:]
            return {"steps": steps, "dt": inst.dt, "seconds": tt, "steps_per_s": steps / tt,
                    "hi_mvps_per_step": hi / steps, "lo_mvps_per_step": lo / steps, "max_kkt": max(kkts),
                    "contacts_first_last": [ncs[0], ncs[-1]],
                    "slip_gmres_iterations_per_step": float(np.mean(later)) if later else None,
                    "slip_warm_started_steps": int(sum(warm)), "force_warm_started_steps": int(sum(warm_x))}

        traj = trajectory(ctx, args.trajectory)
        traj["warm_start_flags"] = int(cfg.warm_start)
        if args.trajectory_cold:
            cfg_cold = L.config_for(insts[0], prec, cuda_stream=stream.cuda_stream, warm_start=0, **lowfi)
            ctx_cold = L.lcp_setup(cfg_cold, inst.centers, inst.axes)
            traj["cold_start_first_steps"] = trajectory(ctx_cold, min(args.trajectory_cold, args.trajectory))
            L.lcp_destroy(ctx_cold)
    L.lcp_destroy(ctx)
    c2 = c2_report(stream) if (args.c2 and rank == 0 and world == 1) else None
    c4 = c5 = None
    if args.c4c5 and rank == 0 and world == 1:
        # the batched and serving configurations at their sizes (256 instances; 32 simulations,
        # 3 steps each), two timed batches, without the minutes-long plain-FP64 baselines
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup, sub.fp64_baseline, sub.sim_steps = 6, 3, 0, 3
        c4 = run_batched(sub)
        c5 = run_serving(sub)
        for d in (c4, c5):
            d["fp64_baseline_note"] = ("plain FP64 one at a time is timed over every instance by "
                                       "bench.py --mode batched / --mode serving")

    pairs = float(N) * (N - 1)
    avg32 = t32 / c32 / 1e3 if c32 else None
    roof = None
    if avg32:
        ach = pairs * FLOPS_PER_PAIR / avg32 / 1e12
        kname = pair32_kernel_name(variant)
        info = PAIR32_TRAFFIC.get(kname)
        traffic = info["bytes_per_launch"] if info and info["bytes_per_launch"] and \
            info["source_sha1"] == source_sha1(kname) else None
        roof = {"kernel": kname, "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS, "traffic": traffic,
                "launches": c32, "avg_launch_ms": avg32 * 1e3, "pairs_per_launch": pairs,
                "flops_per_pair": FLOPS_PER_PAIR, "share_of_timed_region": t32 / 1e3 / t_total,
                "flops_note": "algorithmic work of the operator: 32 flops per ordered node pair, N(N-1) pairs",
                "peak_note": "152 SMs x 128 FP32 lanes x 2 x 2.070 GHz (nominal max clock)"}
        if variant.startswith("sym"):
            fpp = SYM_RC_FLOPS_PER_ORDERED_PAIR if "rc" in variant[len("sym_"):] else SYM_FLOPS_PER_ORDERED_PAIR
            hw = pairs * fpp / avg32 / 1e12
            roof["kernel_flops_per_pair"] = fpp
            roof["executed_tflops"] = hw
            roof["executed_frac"] = hw / FP32_PEAK_TFLOPS
            roof["symmetric_note"] = ("one evaluation serves both ordered terms of a node pair; "
                                      "executed_frac counts the FP32 operations the kernel performs")
    k64 = None
    if c64:
        a64 = pairs * FLOPS_PER_PAIR / (t64 / c64 / 1e3) / 1e12
        k64 = {"kernel": "k_pair64", "launches": c64, "avg_launch_ms": t64 / c64, "achieved": a64,
               "peak": FP64_PEAK_TFLOPS, "frac": a64 / FP64_PEAK_TFLOPS,
               "share_of_timed_region": t64 / 1e3 / t_total}
    summary = {
        "hi_mvps": [s["hi_mvps"] for s in stats], "lo_mvps": [s["lo_mvps"] for s in stats],
        "e_mvps": [round(s["e_mvps"], 3) for s in stats], "iterations": [s["iterations"] for s in stats],
        "gmres_iterations": [s["gmres_iterations"] for s in stats],
        "gmres_iterations_per_hi_mvp": float(sum(s["gmres_iterations"] for s in stats)
                                             / max(1, sum(s["hi_mvps"] for s in stats))),
        "lo_gmres_iterations": [s["lo_gmres_iterations"] for s in stats],
        "recycled_solves": [s["recycled_solves"] for s in stats],
        "fp32_applies": [s["fp32_applies"] for s in stats], "fp64_applies": [s["fp64_applies"] for s in stats],
        "df64_applies": [s["df64_applies"] for s in stats],
        "kkt_abs": [s["kkt_abs"] for s in stats], "contacts": ncon,
        "converged": all(s["converged"] == 1 for s in stats),
    }
    kdf = None
    if cdf:
        sym_df = variant.startswith("sym")
        kdf = {"kernel": "k_pair_df_sym" if sym_df else "k_pair_df", "launches": cdf, "avg_launch_ms": tdf / cdf,
               "fp32_ops_per_pair_note": "double-FP32 arithmetic, ~250 FP32 operations per ordered pair"
                                         + (", one evaluation per unordered pair (symmetric)" if sym_df else ""),
               "pairs_per_s": pairs / (tdf / cdf / 1e3), "share_of_timed_region": tdf / 1e3 / t_total}
    lowfi_desc = lowfi_description(lowfi)
    return dict(t_total=t_total, lat=lat, clocks=clk, c2=c2, c4=c4, c5=c5, launches=launches, roof=roof, k64=k64, kdf=kdf, e2e=e2e, traj=traj,
                lowfi=lowfi_desc, lowfi_cfg=lowfi,
                comparison=comparison,
                fp64=fp64, summary=summary, N=N, M=M)


def c2_report(stream) -> dict:
    """64 spheres (9 x 18 nodes, delta 0.05): Mono-PQN on the high-fidelity mobility and Bi-PQN
    with the RPY low fidelity, each all-FP64 and mixed (FP32 sums + FP64 refinement): solve time,
    high-/low-fidelity MVPs, and the distance to the plain FP64 Mono-PQN solution (the tests
    check these solves against the FP64 oracle)."""
    import paper_2604_10089_gb300 as L
    from workloads import make_instance

    inst = make_instance("spheres64_grid9x18", 0)
    out = {"workload": "spheres64_grid9x18: 64 Janus spheres, 10368 nodes, 31104 unknowns, delta 0.05",
           "tol": inst.tol}
    ref = None
    for name, meth, prec in (("mono_fp64", L.LCP_MONO_PQN, L.LCP_FP64), ("mono_mixed", L.LCP_MONO_PQN, L.LCP_MIXED),
                             ("bi_rpy_fp64", L.LCP_BI_PQN, L.LCP_FP64), ("bi_rpy_mixed", L.LCP_BI_PQN, L.LCP_MIXED)):
        ctx = L.lcp_setup(L.config_for(inst, prec, cuda_stream=stream.cuda_stream), inst.centers, inst.axes)
        try:
            L.lcp_solve(ctx, meth, inst.tol)   # warm-up (graph capture, first launches)
            t0 = time.perf_counter()
            x, st, _ = L.lcp_solve(ctx, meth, inst.tol)
            dt = time.perf_counter() - t0
        finally:
            L.lcp_destroy(ctx)
        if ref is None:
            ref = x
        thr = 1e-9 * max(1.0, float(np.abs(ref).max()))
        out[name] = {"seconds": dt, "hi_mvps": st["hi_mvps"], "lo_mvps": st["lo_mvps"], "e_mvps": st["e_mvps"],
                     "kkt": st["kkt_abs"], "converged": st["converged"] == 1,
                     "max_abs_diff_vs_mono_fp64": float(np.abs(x - ref).max()),
                     "same_active_set_as_mono_fp64": bool(np.array_equal(x > thr, ref > thr))}
    out["contacts"] = int(ref.size)
    return out


def run_batched(args):
    """256 uneven instances (8-128 spheres, 98 or 162 nodes, phi 0.30-0.45) solved together."""
    import torch

    import paper_2604_10089_gb300 as L
    from workloads import batched_instances

    t0 = time.perf_counter()
    insts = batched_instances(args.batch_count)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctxs = [L.lcp_setup(L.config_for(i, L.LCP_MIXED, own_stream=1, autotune=1, **instance_lowfi(args, i)),
                        i.centers, i.axes)
            for i in insts]
    t_setup = time.perf_counter() - t0
    xs = [torch.empty(max(L.lcp_sizes(c)[2], 1), dtype=torch.float64, device="cuda") for c in ctxs]
    for _ in range(max(1, args.warmup // 3)):
        L.lcp_batch_solve(ctxs, L.LCP_BI_PQN, 1e-8, xs, workers=args.workers)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    reps = max(1, args.steps // 3)
    for _ in range(reps):
        statuses, stats = L.lcp_batch_solve(ctxs, L.LCP_BI_PQN, 1e-8, xs, workers=args.workers)
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t0) / reps
    clk = clocks.stop()
    # the same instances one at a time (mixed), and plain FP64 Mono-PQN on a sample
    t0 = time.perf_counter()
    for c in ctxs:
        L.lcp_solve(c, L.LCP_BI_PQN, 1e-8)
    t_seq = time.perf_counter() - t0
    # plain FP64 Mono-PQN on the GPU, one instance at a time (every instance, timed)
    t64_all = 0.0
    if args.fp64_baseline:
        for i in insts:
            c64 = L.lcp_setup(L.config_for(i, L.LCP_FP64, recycle=0), i.centers, i.axes)
            ts = time.perf_counter()
            L.lcp_solve(c64, L.LCP_MONO_PQN, 1e-8, allow_not_converged=True)
            t64_all += time.perf_counter() - ts
            L.lcp_destroy(c64)
    variants = {}
    for c in ctxs:
        v = L.lcp_kernel_variant(c)
        variants[v] = variants.get(v, 0) + 1
    for c in ctxs:
        L.lcp_destroy(c)
    line = {"metric": "batched LCP solves/s", "value": len(insts) / t_batch, "unit": "LCP solves/s",
            "n_gpus": 1, "mode": "batched", "instances": len(insts), "workers": args.workers,
            "seconds_per_batch": t_batch, "all_converged": all(s == 0 for s in statuses),
            "hi_mvps_mean": float(np.mean([s["hi_mvps"] for s in stats])),
            "sequential_mixed_solves_per_s": len(insts) / t_seq,
            "sequential_fp64_mono_solves_per_s": (len(insts) / t64_all) if args.fp64_baseline else None,
            "setup_seconds_all": t_setup, "generation_seconds": t_gen,
            "kernel_variants": variants, "clocks": clk,
            "config": {"workload": "256 packings, 8-128 spheres, 98 or 162 nodes per sphere, phi 0.30-0.45",
                       "method": "bi_pqn", "precision": "mixed", "tol": 1e-8,
                       "low_fidelity": batch_lowfi_description(args)}}
    return line


def run_serving(args):
    """Poisson requests from concurrent simulations (16-216 spheres, 162 nodes); the server holds
    each simulation's first request until its estimated footprint fits the HBM budget."""
    import torch

    import paper_2604_10089_gb300 as L
    from workloads import serving_simulations

    sims = serving_simulations(args.sims)
    rng = np.random.default_rng(77)
    cfgs = [L.config_for(i, L.LCP_MIXED, **instance_lowfi(args, i)) for i in sims]
    est = [L.lcp_footprint_estimate(c, i.n_bodies, 6 * i.n_bodies) for c, i in zip(cfgs, sims)]
    budget = int(args.budget_frac * sum(est))
    srv = L.lcp_server_create(args.workers, budget)
    ids = [L.lcp_server_open(srv, c, i.centers, i.axes) for c, i in zip(cfgs, sims)]
    steps_left = [args.sim_steps] * len(sims)
    arrival = list(rng.exponential(1.0 / args.arrival_rate, len(sims)))
    ncon = [None] * len(sims)
    ticket = {}
    lat, solves_stats = [], []
    t0 = time.perf_counter()
    clocks = ClockSampler(0)
    clocks.start()
    done = 0
    total = args.sim_steps * len(sims)
    max_resident = max_waiting = 0
    while done < total and time.perf_counter() - t0 < 1800:
        now = time.perf_counter() - t0
        for k in range(len(sims)):
            if steps_left[k] == 0 or k in ticket or arrival[k] > now:
                continue
            dt = sims[k].dt if steps_left[k] > 1 else 0.0     # the simulation advances after each solve
            ticket[k] = (L.lcp_server_request(srv, ids[k], L.LCP_BI_PQN, 1e-8, dt), arrival[k])
        for k, (t, arr) in list(ticket.items()):
            status, x, st = L.lcp_server_poll(srv, t, 6 * sims[k].n_bodies, 200)
            if status == L.LCP_ERR_TIMEOUT:
                continue
            fin = time.perf_counter() - t0
            lat.append(fin - arr)
            solves_stats.append(st)
            del ticket[k]
            done += 1
            steps_left[k] -= 1
            if steps_left[k] > 0:
                arrival[k] = fin + rng.exponential(1.0 / args.arrival_rate)
            else:
                L.lcp_server_close(srv, ids[k])
        resident, waiting, _ = L.lcp_server_stats(srv)
        max_resident = max(max_resident, resident)
        max_waiting = max(max_waiting, waiting)
        time.sleep(0.0005)
    makespan = time.perf_counter() - t0
    clk = clocks.stop()
    L.lcp_server_destroy(srv)
    # sequential baselines: the same first-step requests one at a time, mixed Bi-PQN, and plain
    # FP64 Mono-PQN on the GPU (every simulation, timed)
    t_seq = t64 = 0.0
    for i in sims:
        c = L.lcp_setup(L.config_for(i, L.LCP_MIXED, **instance_lowfi(args, i)), i.centers, i.axes)
        ts = time.perf_counter()
        L.lcp_solve(c, L.LCP_BI_PQN, 1e-8)
        t_seq += time.perf_counter() - ts
        L.lcp_destroy(c)
        if args.fp64_baseline:
            c = L.lcp_setup(L.config_for(i, L.LCP_FP64, recycle=0), i.centers, i.axes)
            ts = time.perf_counter()
            L.lcp_solve(c, L.LCP_MONO_PQN, 1e-8, allow_not_converged=True)
            t64 += time.perf_counter() - ts
            L.lcp_destroy(c)
    line = {"metric": "served LCP solves/s", "value": done / makespan, "unit": "LCP solves/s", "n_gpus": 1,
            "mode": "serving", "requests": done, "simulations": len(sims), "workers": args.workers,
            "latency_s": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": max(lat) if lat else None},
            "arrival_rate_per_sim": args.arrival_rate, "hbm_budget_bytes": budget,
            "max_resident_bytes": max_resident, "max_requests_waiting": max_waiting,
            "sum_of_footprint_estimates": int(sum(est)),
            "all_converged": all(s["converged"] == 1 for s in solves_stats),
            "sequential_mixed_bi_solves_per_s": len(sims) / t_seq,
            "sequential_fp64_mono_solves_per_s": (len(sims) / t64) if args.fp64_baseline else None,
            "clocks": clk,
            "config": {"workload": f"{len(sims)} simulations, 16-216 spheres, 162 nodes per sphere, "
                                   f"phi 0.35-0.45, {args.sim_steps} steps each",
                       "method": "bi_pqn", "precision": "mixed", "tol": 1e-8,
                       "low_fidelity": batch_lowfi_description(args),
                       "admission": "server-held: a simulation's context is created once its estimated "
                                    "footprint fits the budget"}}
    return line


# Mean high- and low-fidelity MVPs per LCP solve of the GPU path on this workload (mixed
# Bi-PQN, 8 x 16 coarse-grid low fidelity): the mean over the 20 timed solves of a GPU
# bench run.  The reference arm has no GPU, so it takes its solve count from here; the
# main arm uses the counts it measures itself.
REFERENCE_MVPS = {"hi": 3.15, "lo": 18.40,
                  "source": "mean over the 20 timed solves of a GB300 bench run at spheres216_grid11x22 "
                            "(mixed Bi-PQN, 8 x 16 low fidelity)"}


def oracle_mobility_solves(workload: str, index: int, lowfi: dict, coarse_solves: int = 1, fine: bool = True):
    """Complete oracle mobility solves (plain C, FP64, all host cores), timed.

    fine: the U_nc slip solve of one configuration on the workload's grid, FP64 GMRES
    to 1e-12 (one high-fidelity solve of the LCP path).  Then `coarse_solves` complete
    low-fidelity solves with random forces: GMRES to the low fidelity's tolerance on
    its coarse grid, or the RPY pair mobility when the low fidelity is RPY.
    """
    from oracle.mf import MatrixFreeMobility
    from oracle.rpy import rpy_matrix
    from workloads import make_instance

    inst = make_instance(workload, index)
    out = {"cores": len(os.sched_getaffinity(0))}
    if fine:
        mf = MatrixFreeMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius, tol=1e-12,
                                self_quadrature=True)
        t0 = time.perf_counter()
        mf.apply(np.zeros(6 * inst.n_bodies), axes=inst.axes)
        out["fine_seconds"] = time.perf_counter() - t0
        out["fine_gmres_iterations"] = mf.last_iterations
    rng = np.random.default_rng(1000 + index)
    times, iters = [], []
    if lowfi:
        mc = MatrixFreeMobility(inst.centers, lowfi["lowfi_n_theta"], lowfi["lowfi_n_phi"], a=inst.radius,
                                tol=lowfi.get("lowfi_tol", 1e-6), self_quadrature=True)
    for _ in range(coarse_solves):
        FT = rng.standard_normal(6 * inst.n_bodies)
        t0 = time.perf_counter()
        if lowfi:
            mc.apply(FT)
            iters.append(mc.last_iterations)
        else:
            rpy_matrix(inst.centers, a=inst.radius, mu=inst.viscosity) @ FT
        times.append(time.perf_counter() - t0)
    out["coarse_seconds"] = times
    out["coarse_gmres_iterations"] = iters
    return out


def oracle_lcp_rate(fine_s: float, coarse_s: float, hi: float, lo: float) -> float:
    """LCP solves/s of the oracle on this path: one slip solve plus `hi` high-fidelity
    MVPs at the measured fine-solve time, `lo` low-fidelity MVPs at the coarse one."""
    return 1.0 / ((1.0 + hi) * fine_s + lo * coarse_s)


def c1_oracle_solve(index: int = 1) -> dict:
    """One complete oracle collision resolution at 8 spheres (7 x 14 nodes): dense K + P by
    LU, dense M and A = D^T M D, the slip solve for b, and the LCP by projected Gauss-Seidel.
    The self-interaction correction of the grid is built before the clock starts (like the
    library, which builds it once per grid and process)."""
    from oracle.bie import DenseMobility, self_correction
    from oracle.contacts import contact_matrix, detect_contacts
    from oracle.lcp import kkt_abs, lcp_data, pgs
    from workloads import make_instance

    inst = make_instance("spheres8_grid7x14", index)
    self_correction(inst.n_theta, inst.n_phi, inst.radius)
    t0 = time.perf_counter()
    mob = DenseMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius, mu=inst.viscosity,
                        self_quadrature=True)
    pairs, normals, gaps = detect_contacts(inst.centers, inst.contact_radius, inst.delta)
    D = contact_matrix(inst.n_bodies, pairs, normals)
    A, b = lcp_data(D, mob.matrix(), mob.apply(np.zeros(6 * inst.n_bodies), axes=inst.axes), gaps, inst.dt)
    x = pgs(A, b)
    t = time.perf_counter() - t0
    return {"seconds": t, "contacts": int(b.size), "active": int((x > 0).sum()),
            "kkt": float(kkt_abs(x, A @ x + b)), "solves_per_s": 1.0 / t}


def host_cpu() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm implementer and part)."""
    try:
        text = open("/proc/cpuinfo").read()
    except OSError:
        return platform.machine()
    fields = {}
    for line in text.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            fields.setdefault(k.strip(), v.strip())
    if "model name" in fields:
        return fields["model name"]
    parts = [platform.machine()]
    for k in ("CPU implementer", "CPU part", "CPU variant"):
        if k in fields:
            parts.append(f"{k.split()[-1]} {fields[k]}")
    return " ".join(parts)


def c1_anchor() -> dict:
    """The complete 8-sphere oracle solve on one core and on all host cores (subprocesses,
    so that the BLAS thread count is fixed before numpy loads)."""
    res = {"workload": "spheres8_grid7x14 (8 spheres, 2352 unknowns): dense LU of K + P, dense A, PGS"}
    for name, env in (("single_core", {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1",
                                       "MKL_NUM_THREADS": "1"}), ("all_cores", {})):
        try:
            out = subprocess.run([sys.executable, os.path.abspath(__file__), "--c1-oracle"], capture_output=True,
                                 text=True, timeout=300, env={**os.environ, **env}, check=True)
            res[name] = json.loads(out.stdout.strip().splitlines()[-1])
        except (subprocess.SubprocessError, ValueError, IndexError) as e:
            res[name] = {"error": str(e)[:200]}
    res["cores"] = len(os.sched_getaffinity(0))
    return res


def config_dict(args, M: int, N: int, lowfi_desc: str, world: int) -> dict:
    """The workload description both arms print."""
    return {"workload": f"{args.workload}: {M} Janus spheres, {N} surface nodes, {3 * N} unknowns",
            "method": f"{args.method}_pqn", "precision": args.precision, "tol": 1e-8,
            "low_fidelity": lowfi_desc,
            "gmres_tol": 1e-12, "step": "contacts + U_nc slip solve + b + LCP solve",
            "l2": "inputs larger than L2 (Krylov basis 76 MB + operator sweeps per apply)",
            "inner_tol": args.inner_tol, "recycle": args.recycle, "self_quadrature": args.self_quadrature,
            "parallelism": f"instances x{world}"}


def lowfi_description(lowfi: dict) -> str:
    if not lowfi:
        return "rpy"
    return (f"boundary integral on a {lowfi['lowfi_n_theta']}x{lowfi['lowfi_n_phi']} grid, FP32 GMRES to "
            f"{lowfi.get('lowfi_tol', 1e-6):g}, initialisation to {lowfi.get('init_forcing', 0.0):g} of its "
            f"initial KKT error")


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores, on this workload.

    Warm-up: one complete fine-grid slip solve (FP64 GMRES to 1e-12) of the first
    configuration, timed with its iteration count.  Each further step, warm-up or timed:
    one complete low-fidelity mobility solve of the next configuration.  The rate is one
    LCP solve's worth of these measured solves: (1 + hi) fine solves and lo coarse ones,
    with the GPU path's measured MVP counts on this workload (REFERENCE_MVPS).
    """
    if rank != 0:
        return
    from workloads import make_instance
    inst = make_instance(args.workload, 0)
    lowfi = lowfi_overrides(args.lowfi, inst.n_theta)
    first = oracle_mobility_solves(args.workload, 0, lowfi, coarse_solves=0)
    coarse, iters, step_s = [], [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle_mobility_solves(args.workload, 1 + k, lowfi, coarse_solves=1, fine=False)
        if k >= args.warmup:
            coarse.extend(r["coarse_seconds"])
            iters.extend(r["coarse_gmres_iterations"])
            step_s.append(time.perf_counter() - t0)
    t_c = float(np.mean(coarse))
    value = oracle_lcp_rate(first["fine_seconds"], t_c, REFERENCE_MVPS["hi"], REFERENCE_MVPS["lo"])
    M = inst.n_bodies
    N = inst.n_bodies * inst.n_theta * inst.n_phi
    sample = (f"{args.steps} complete low-fidelity oracle mobility solves ({t_c:.3f} s each"
              + (f", {np.mean(iters):.1f} GMRES iterations" if iters else "")
              + f"), after one complete fine-grid slip solve in the warm-up ({first['fine_seconds']:.2f} s, "
                f"{first['fine_gmres_iterations']} GMRES iterations to 1e-12); one LCP solve = "
                f"(1 + {REFERENCE_MVPS['hi']}) fine + {REFERENCE_MVPS['lo']} low-fidelity solves "
                f"({REFERENCE_MVPS['source']})")
    anchor = c1_anchor()
    line = {"impl": "reference", "metric": "LCP solves/s", "value": value, "unit": "LCP solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "ms_per_step": 1e3 * float(np.mean(step_s)), "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, M, N, lowfi_description(lowfi), world),
            "cpu_baseline": {"value": value, "unit": "LCP solves/s", "cores": first["cores"], "cpu": host_cpu(),
                             "kind": "oracle",
                             "sample": sample, "fine_solve_seconds": first["fine_seconds"],
                             "fine_gmres_iterations": first["fine_gmres_iterations"],
                             "coarse_solve_seconds": t_c, "mvps_per_lcp": REFERENCE_MVPS,
                             "c1_complete_solve": anchor},
            "ms_per_step_note": "wall time of one sample step (one complete low-fidelity oracle solve)",
            "e2e": {"value": value, "unit": "LCP solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    if "--c1-oracle" in sys.argv:
        print(json.dumps(c1_oracle_solve()), flush=True)
        return
    args = parse()
    rank, world, local = dist_info()
    if world > 1:
        import torch
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        torch.distributed.init_process_group(backend=backend)
    if args.impl == "ours" and args.mode != "solve":
        if rank == 0:
            line = run_batched(args) if args.mode == "batched" else run_serving(args)
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    r = run_ours(args, rank, world, local)
    if rank == 0:
        value = args.steps * world / r["t_total"]
        s = r["summary"]
        cpu = None
        if args.cpu_baseline and world == 1:
            # complete oracle mobility solves of this workload (one fine slip solve, two
            # low-fidelity solves), combined with the MVP counts this run measured
            hi, lo = float(np.mean(s["hi_mvps"])), float(np.mean(s["lo_mvps"]))
            o = oracle_mobility_solves(args.workload, 0, r["lowfi_cfg"], coarse_solves=2)
            t_c = float(np.mean(o["coarse_seconds"]))
            cpu = {"value": oracle_lcp_rate(o["fine_seconds"], t_c, hi, lo), "unit": "LCP solves/s",
                   "cores": o["cores"], "cpu": host_cpu(), "kind": "oracle",
                   "sample": f"one complete fine-grid slip solve of a {args.workload} configuration "
                             f"({o['fine_seconds']:.2f} s, {o['fine_gmres_iterations']} FP64 GMRES iterations to "
                             f"1e-12) and {len(o['coarse_seconds'])} complete low-fidelity solves ({t_c:.3f} s each"
                             + (f", {np.mean(o['coarse_gmres_iterations']):.1f} GMRES iterations"
                                if o["coarse_gmres_iterations"] else "")
                             + f"); one LCP solve = (1 + {hi:.2f}) fine + {lo:.2f} low-fidelity solves, the mean "
                               f"MVP counts of this run's timed solves",
                   "fine_solve_seconds": o["fine_seconds"], "fine_gmres_iterations": o["fine_gmres_iterations"],
                   "coarse_solve_seconds": t_c, "mvps_per_lcp": {"hi": hi, "lo": lo},
                   "c1_complete_solve": c1_anchor()}
        line = {
            "metric": "LCP solves/s", "value": value, "unit": "LCP solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * r["t_total"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": config_dict(args, r["M"], r["N"], r["lowfi"], world),
            "latency_s": {"p50": pct(r["lat"], 50), "p99": pct(r["lat"], 99)},
            "matvecs_per_s": {
                "high_fidelity_mvps": float(np.sum(s["hi_mvps"])) / r["t_total"],
                "low_fidelity_mvps": float(np.sum(s["lo_mvps"])) / r["t_total"],
                "fp32_pair_sum_applies": float(np.sum(s["fp32_applies"])) / r["t_total"],
                "note": "per second of the timed region; the FP32 applies are the high-fidelity grid's"},
            "roofline": r["roof"], "fp64_kernel": r["k64"], "df64_kernel": r["kdf"], "clocks": r["clocks"],
            "e2e": r["e2e"], "gpu_launches": r["launches"], "cpu_baseline": cpu,
            "fp64_mono_pqn": r["fp64"], "method_comparison_mixed": r["comparison"], "trajectory": r["traj"],
            "c2_spheres64": r["c2"], "c4_batched": r["c4"], "c5_serving": r["c5"],
            "solver": s,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
