#!/usr/bin/env python3
"""Benchmark of the all-at-once multigrid solvers for the Poisson and Stokes control problems.

Workload (one "step"): the scaling configuration at its largest size -- unit
square, h = 2^-11 (2049 x 2049 nodes, 8.4M unknowns y and lambda), y_D =
sin(2 pi x) sin(2 pi y) + 0.1 N(0,1) (seed 1), one solve from x = 0 to a
relative residual of 1e-8 for each alpha in {1, 1e-2, 1e-4, 1e-6, 1e-8}, with
the LSGS smoother, W-cycle, 2+2 steps, down to h = 1/2, FP32 cycles inside FP64
iterative refinement (4 FP32 cycles per refinement step: all five alphas then
converge in the same number of refinement steps; the other lines use the
library's default of 3).  Inputs are resident in HBM when timing starts; L2 is
flushed (256 MB write) before every timed step.

Printed JSON line: value = solved unknowns/s over all ranks; fp64_plain = the
same workload with every operation in FP64; e2e = through mg_batch_solve_host
with pinned host buffers (copies inside the timed region); roofline = the
finest-level smoother sweep (CUDA events inside a solve) against the measured
HBM copy bandwidth; roofs_measured = the library's own FMA-rate and bandwidth
microbenchmarks; l12, batch256, autograd16 = the largest instance, 256 batched
instances, 16 differentiated instances; stokes = the Stokes control problem at
h = 2^-9; cpu_baseline = the FP64 CPU oracle on a bounded sample.
`--impl reference` times the CPU oracle alone on the same workload.

Other modes (not timed against the reference): `--batch N` solves N
independent instances of mixed size (levels 6..10, alpha log-uniform in
[1e-8, 1]) in one batch graph; `--protocol` / `--protocol-stokes` print the
iteration counts of the paper's section 3 protocol in the layout of its
Table 1 / Table 2; `--profile-band`, `--profile-stokes`,
`--profile-stokes-step` run small launch sequences for ncu.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ALPHAS = [1.0, 1e-2, 1e-4, 1e-6, 1e-8]
METRIC = "solved unknowns/s at 1e-8 rel. residual, FP32+refine vs FP64; smoother GB/s"
UNIT = "unknowns/s"
SWEEP_BYTES_FP32 = 24  # per node and sweep: read y, lambda, f_y, f_lambda; write y, lambda (4 B each)
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_L{L}.json")

# DRAM bytes (read + written) of one finest-level LSGS step (the band kernel)
# from ncu captures (profiles/k_lsgs_band_l11.md, profiles/k_lsgs_band_l12.md),
# per level; valid while the kernel's sources hash to SHA.
BAND_TRAFFIC = {"bytes": {11: 73_746_432, 12: 388_791_808},
                "sha256": "09fba05ae0c3f3a41a8226b017ce1ac2b22041927767adceea023ae604fdccf1",
                "files": ["lsgs_band.cu", "band.h", "lean.cuh", "stencil.cuh", "common.cuh", "pair.cuh"]}


def band_traffic(level):
    """The captured traffic per launch, or None when the level was not
    captured or the kernel has changed since the capture."""
    import hashlib

    if level not in BAND_TRAFFIC["bytes"]:
        return None
    h = hashlib.sha256()
    try:
        for f in BAND_TRAFFIC["files"]:
            with open(os.path.join(ROOT, "paper_1502_03917_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return BAND_TRAFFIC["bytes"][level] if h.hexdigest() == BAND_TRAFFIC["sha256"] else None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--level", type=int, default=11)
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--smoother", default="lsgs", choices=["ne", "lsgs", "slsgs", "cgs"])
    p.add_argument("--cycle", default="W", choices=["V", "W"])
    p.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 comparison")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-vcycle", action="store_true", help="skip the V-cycle comparison")
    p.add_argument("--inner-cycles", type=int, default=4,
                   help="FP32 cycles per refinement step of the five-solve workload (its e2e, roofline and by-time "
                        "solves too; with 4 the five alphas all converge in the same number of refinement steps); "
                        "0: the library default, 3, which the h = 2^-12, 256-instance and differentiation lines use")
    p.add_argument("--small-max", type=int, default=0,
                   help="largest level (nodes per side) smoothed in one launch per call (0: library default 513; "
                        "257: per-phase launches on 513^2)")
    p.add_argument("--autotune", action="store_true",
                   help="let the library time each level's candidate kernels at set-up")
    p.add_argument("--batch", type=int, default=0,
                   help="time N independent instances of mixed size through mg_solve_batch instead")
    p.add_argument("--protocol", action="store_true",
                   help="print the iteration counts of the paper's protocol (Table 1 layout) instead of timing")
    p.add_argument("--profiling-run", action="store_true",
                   help="for runs under an external profiler: no CUDA events inside the solver graphs and no "
                        "nvidia-smi sampling (roofline and clocks are then not reported)")
    p.add_argument("--serial", action="store_true",
                   help="solve the alphas one after another instead of concurrently on separate streams")
    p.add_argument("--no-l12", action="store_true", help="skip the h = 2^-12 single-instance line")
    p.add_argument("--no-batch256", action="store_true", help="skip the 256-instance batched-solve line")
    p.add_argument("--no-autograd", action="store_true", help="skip the 16-instance differentiation line")
    p.add_argument("--no-stokes", action="store_true", help="skip the Stokes control line")
    p.add_argument("--protocol-stokes", action="store_true",
                   help="the section 3 protocol for the Stokes control problem on the GPU, in the layout of Table 2")
    p.add_argument("--profile-stokes", type=int, default=0, metavar="L",
                   help="profiling run: one Stokes W-cycle at h = 2^-L (bench workload, after a warm-up cycle) "
                        "inside cudaProfilerStart/Stop (ncu --profile-from-start off)")
    p.add_argument("--profile-stokes-step", type=int, default=0, metavar="L",
                   help="profiling run: one finest-level Stokes LSGS step at h = 2^-L without the dense map "
                        "inside cudaProfilerStart/Stop")
    p.add_argument("--profile-band", type=int, default=0, metavar="L",
                   help="for ncu captures: set up one FP32 LSGS handle at h = 2^-L and run --steps finest-level "
                        "smoothing steps (mg_smooth) after --warmup untimed ones; prints the CUDA-event time")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# ----------------------------------------------------------- multi-rank --
def rank_max(v: float, world: int, device: str) -> float:
    """The largest v over all ranks (the slowest replica's time); v itself for
    one rank.  Uses the default process group (NCCL on GPUs, gloo on CPU)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank_step: float, steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units all replicas processed in `steps` steps
    divided by the slowest replica's time (ms)."""
    return world * units_per_rank_step * steps / (ms_max / 1e3)


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200", "-i",
                 str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
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
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- our arm ----
def run_ours(args, rank, world, local):
    import torch

    from paper_1502_03917_gb300 import build as B
    from paper_1502_03917_gb300 import inputs
    import paper_1502_03917_gb300.aaomg as mg

    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    L = args.level
    yD = torch.tensor(inputs.yd_sine_noise(L, 1), dtype=torch.float64, device="cuda")

    def make(precision, profile):
        return {a: mg.Solver(L, a, smoother=args.smoother, precision=precision, cycle=args.cycle, max_iter=100,
                             profile=profile, inner_cycles=args.inner_cycles, autotune=args.autotune,
                             small_max=args.small_max)
                for a in ALPHAS}

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2

    streams = {a: torch.cuda.Stream() for a in ALPHAS}

    def run_all(fn):
        """fn(alpha) for every alpha: concurrently, one host thread and one CUDA
        stream per alpha (independent problems), or one after another."""
        if args.serial:
            for a in ALPHAS:
                fn(a)
            return
        main = torch.cuda.current_stream()
        ready = torch.cuda.Event()
        ready.record(main)
        errs = []

        def work(a):
            try:
                with torch.cuda.stream(streams[a]):
                    streams[a].wait_event(ready)
                    fn(a)
            except BaseException as e:  # surfaced below
                errs.append(e)

        ts = [threading.Thread(target=work, args=(a,)) for a in ALPHAS]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        if errs:
            raise errs[0]
        for a in ALPHAS:
            main.wait_stream(streams[a])

    def timed_steps(solvers, K, W):
        fs = {a: s.rhs_from_yd(yD) for a, s in solvers.items()}
        xs = {a: torch.zeros_like(fs[a]) for a in solvers}
        its = {}
        # all alphas in one graph-captured batch: one graph launch per step runs
        # every solve to its own convergence (tests on the device)
        batch = None if args.serial else mg.Batch([solvers[a] for a in ALPHAS])
        torch.cuda.synchronize()

        def one(a):
            xs[a].zero_()
            it, rr, code = solvers[a].solve(fs[a], xs[a], tol=args.tol)
            its[a] = it

        def step():
            if args.serial:
                run_all(one)
                return
            for a in ALPHAS:
                xs[a].zero_()
            it, rr, st, code = batch.solve([fs[a] for a in ALPHAS], [xs[a] for a in ALPHAS], tol=args.tol)
            for a, k in zip(ALPHAS, it):
                its[a] = k

        for _ in range(W):
            step()
        for s in solvers.values():
            s.reset_profile()
        l0 = sum(s.launches() for s in solvers.values())
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        clk = ClockSampler(local if not args.profiling_run else -1)
        if not args.profiling_run:
            clk.start()
        for k in range(K):
            flush.fill_(float(k))
            ev[k][0].record()
            step()
            ev[k][1].record()
        torch.cuda.synchronize()
        clocks = clk.stop()
        if world > 1:
            torch.distributed.barrier()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        launches = sum(s.launches() for s in solvers.values()) - l0
        prof = [s.profile() for s in solvers.values()]
        if batch is not None:
            batch.close()
        return ms, its, launches, prof, clocks, xs

    def max_over_ranks(v):
        return rank_max(v, world, "cuda")

    K, W = args.steps, args.warmup
    N = ((1 << L) + 1) ** 2
    unknowns_step = len(ALPHAS) * 2 * N

    sol32 = make("fp32_refine", False)
    ms, its32, launches, prof, clocks, xs32 = timed_steps(sol32, K, W)
    ms = max_over_ranks(ms)
    value = job_value(unknowns_step, K, world, ms)

    # roofline of the finest-level smoother sweep, timed with nothing else in
    # flight (one solve, in-graph CUDA events around each finest-level call)
    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    roofline = None
    roofs = None
    if not args.profiling_run:
        roofline = sweep_roofline(mg, L, yD, 1e-4, args, peak, pk is not None)
        # the project's own measurements of the roofs (FMA rates, L2-resident
        # and HBM bandwidth): at 2049^2 the sweep's x and f (67 MB) fit in L2
        roofs = mg.device_peaks()
        if roofline and roofline.get("achieved"):
            roofline["l2_gbs"] = roofs["l2_gbs"]
            roofline["frac_of_l2"] = roofline["achieved"] / roofs["l2_gbs"]
        # share of the timed steps: the isolated sweep time times the finest
        # sweeps the timed solves ran (refinement steps x inner cycles x 4)
        per_iter = roofline.pop("sweeps_per_iteration")
        sweeps = per_iter * sum(its32.values()) * K
        roofline["share_of_step"] = roofline["sweep_ms"] * sweeps / ms if roofline["sweep_ms"] else None

    # By device time the W-cycle is dominated by the latency-bound one-launch
    # smoothing calls on level 6 (the top kernel of the ncu launch list): time
    # them inside one real solve (alpha = 1) with in-graph events around each call.
    by_time = None
    LT = 6
    if not args.profiling_run and L > LT + 1:
        sp = mg.Solver(L, ALPHAS[0], smoother=args.smoother, precision="fp32_refine", cycle=args.cycle, max_iter=100,
                       profile=True, profile_level=LT, inner_cycles=args.inner_cycles)
        fa = sp.rhs_from_yd(yD)
        xa = torch.zeros_like(fa)
        sp.solve(fa, xa, tol=args.tol)
        sp.reset_profile()
        xa.zero_()
        sp.solve(fa, xa, tol=args.tol)
        t_ms, nsw = sp.profile()
        sp.close()
        NT = ((1 << LT) + 1) ** 2
        nu = 2
        if nsw:
            call_us = t_ms * 1e3 / (nsw / nu)
            ach = SWEEP_BYTES_FP32 * NT * nsw / (t_ms * 1e-3) / 1e9
            by_time = {"kernel": f"level-{LT} smoothing call ({(1 << LT) + 1}^2 nodes, {nu} LSGS steps, one block)",
                       "bound": "latency", "us_per_call": call_us, "us_per_step": call_us / nu,
                       "achieved": ach, "unit": "GB/s", "frac_of_hbm": ach / peak, "calls_timed": nsw // nu}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
           "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": f"Poisson control, h=2^-{L} ({(1 << L) + 1}^2 nodes, {2 * N} unknowns), "
                                  f"alpha in {ALPHAS}, y_D=sin(2pi x)sin(2pi y)+0.1N(0,1) seed 1, "
                                  f"{args.smoother.upper()} {args.cycle}(2,2) to h=1/2, FP32 cycles in FP64 "
                                  f"refinement, tol {args.tol}",
                      "level": L, "unknowns_per_solve": 2 * N, "solves_per_step": len(ALPHAS),
                      "smoother": args.smoother, "cycle": args.cycle, "precision": "fp32_refine",
                      "l2": "flushed (256 MB write) before every timed step", "parallelism": f"replicas x{world}",
                      "concurrency": 1 if args.serial else len(ALPHAS),
                      "inner_cycles": args.inner_cycles if args.inner_cycles > 0 else "library default (3)",
                      "kernels": "autotuned at set-up" if args.autotune else "measured defaults"},
           "iterations": {str(a): its32[a] for a in ALPHAS},
           "roofline": roofline, "roofline_by_time": by_time, "roofs_measured": roofs, "clocks": clocks,
           "gpu_launches": launches}

    out["error_vs_oracle"] = error_vs_golden(L, {a: xs32[a] for a in ALPHAS}, args.smoother)

    if not args.no_l12 and L == 11 and not args.profiling_run:
        out["l12"] = run_l12(args, mg, peak, pk is not None, flush)
    if not args.no_batch256 and not args.profiling_run:
        out["batch256"] = batch_line(args, 256, steps=2, warmup=1)
    if not args.no_autograd and not args.profiling_run:
        out["autograd16"] = run_autograd16(args)
    if not args.no_stokes and not args.profiling_run:
        out["stokes"] = run_stokes(args, peak, pk is not None, flush, cpu=(rank == 0 and world == 1 and not args.no_cpu))

    if not args.no_fp64:
        sol64 = make("fp64", False)
        K64 = max(1, min(K, 2))
        ms64, its64, _, _, _, xs64 = timed_steps(sol64, K64, 1)
        ms64 = max_over_ranks(ms64)
        # error of the FP32+refine solutions against the FP64 ones (both at tol)
        err = 0.0
        for a in ALPHAS:
            d = (xs32[a] - xs64[a]).norm() / xs64[a].norm()
            err = max(err, float(d))
        out["fp64_plain"] = {"value": world * unknowns_step * K64 / (ms64 / 1e3), "ms_per_step": ms64 / K64,
                             "iterations": {str(a): its64[a] for a in ALPHAS},
                             "max_rel_diff_fp32refine_vs_fp64": err}
        if roofs and args.smoother == "lsgs" and not args.profiling_run:
            out["fp64_plain"]["roofline"] = sweep_roofline_fp64(mg, L, yD, args, roofs)
        for s in sol64.values():
            s.close()

    if not args.no_vcycle and args.cycle == "W":
        # the same workload with the V-cycle (one coarse-grid step per level)
        solv = {a: mg.Solver(L, a, smoother=args.smoother, precision="fp32_refine", cycle="V", max_iter=100)
                for a in ALPHAS}
        msv, itsv, _, _, _, _ = timed_steps(solv, max(1, min(K, 2)), 1)
        msv = max_over_ranks(msv)
        out["vcycle"] = {"value": world * unknowns_step * max(1, min(K, 2)) / (msv / 1e3),
                         "ms_per_step": msv / max(1, min(K, 2)), "iterations": {str(a): itsv[a] for a in ALPHAS}}
        for s in solv.values():
            s.close()

    if not args.no_e2e:
        out["e2e"] = run_e2e(args, sol32, yD, K, world, max_over_ranks, run_all)

    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(L, args, its_gpu=out.get("fp64_plain", {}).get("iterations"))
    for s in sol32.values():
        s.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def sweep_roofline(mg, L, yD, alpha, args, peak, measured):
    """The finest-level LSGS sweep timed with nothing else in flight: one solve
    (after a warm-up solve) with CUDA events recorded inside the solver's graph
    around every finest-level smoothing call; 24 algorithmic bytes per node and
    sweep against the measured HBM copy bandwidth."""
    import torch

    s = mg.Solver(L, alpha, smoother=args.smoother, precision="fp32_refine", cycle=args.cycle, max_iter=100,
                  profile=True, inner_cycles=args.inner_cycles, autotune=args.autotune)
    f = s.rhs_from_yd(yD)
    x = torch.zeros_like(f)
    s.solve(f, x, tol=args.tol)
    s.reset_profile()
    x.zero_()
    it, _, _ = s.solve(f, x, tol=args.tol)
    t_ms, nsw = s.profile()
    s.close()
    N = ((1 << L) + 1) ** 2
    sweep_ms = t_ms / nsw if nsw else None
    achieved = SWEEP_BYTES_FP32 * N / (sweep_ms * 1e-3) / 1e9 if sweep_ms else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": band_traffic(L),
            "kernel": f"finest-level LSGS smoothing sweep (FP32, h=2^-{L}, {(1 << L) + 1}^2 nodes)",
            "peak_source": "measured" if measured else "fallback", "sweep_ms": sweep_ms, "sweeps_timed": nsw,
            "algorithmic_bytes_per_sweep": SWEEP_BYTES_FP32 * N,
            "timing": f"one solve alone (alpha={alpha:g}), CUDA events in the solver graph around each "
                      "finest-level smoothing call",
            "sweeps_per_iteration": nsw / it if it else 0}


FLOPS_LSGS_NODE = 114  # Algorithm 2 per node and step: two unknowns, each 14 gather + 14 scatter FMAs and p


def sweep_roofline_fp64(mg, L, yD, args, roofs):
    """The FP64 path's finest-level LSGS sweep (per-colour launches), timed as
    `sweep_roofline` does, against the FP64 FMA rate measured by
    mg_device_peaks: algorithmic flops per node and step = Algorithm 2's, two
    unknowns each with 14 gather and 14 scatter FMAs (A has 14 entries per
    node row over both fields) and one multiply: 114."""
    s = mg.Solver(L, 1e-4, smoother="lsgs", precision="fp64", cycle=args.cycle, max_iter=100, profile=True)
    f = s.rhs_from_yd(yD)
    import torch

    x = torch.zeros_like(f)
    s.solve(f, x, tol=args.tol)
    s.reset_profile()
    x.zero_()
    s.solve(f, x, tol=args.tol)
    t_ms, nsw = s.profile()
    s.close()
    N = ((1 << L) + 1) ** 2
    sweep_ms = t_ms / nsw if nsw else None
    tflops = FLOPS_LSGS_NODE * N / (sweep_ms * 1e-3) / 1e12 if sweep_ms else None
    return {"bound": "fp64", "kernel": f"finest-level FP64 LSGS sweep (per-colour launches, h=2^-{L})",
            "achieved": tflops, "peak": roofs["fp64_tflops"], "unit": "TFLOP/s",
            "frac": tflops / roofs["fp64_tflops"] if tflops else None, "peak_source": "mg_device_peaks",
            "sweep_ms": sweep_ms, "sweeps_timed": nsw, "algorithmic_flops_per_sweep": FLOPS_LSGS_NODE * N,
            "hbm_gbs": 48 * N / (sweep_ms * 1e-3) / 1e9 if sweep_ms else None}


def error_vs_golden(L, xs, smoother):
    """Element-wise error of GPU solutions against the FP64 oracle's at the
    sampled nodes of tests/golden/oracle_L{L}.json (written by the oracle
    alone): max |x - x_oracle| / max |x_oracle| over y and lambda, per alpha."""
    try:
        g = json.load(open(GOLDEN.format(L=L)))
    except (OSError, ValueError):
        return None
    import numpy as np

    idx = np.array(g["sample_nodes"])
    nn = ((1 << L) + 1) ** 2
    out = {}
    for a, x in xs.items():
        ref = next((r for r in g["runs"] if r["smoother"] == smoother and r["alpha"] == a), None)
        if ref is None:
            continue
        xh = x.cpu().numpy()
        e = 0.0
        for got, want in ((xh[idx], np.array(ref["y"])), (xh[nn + idx], np.array(ref["lambda"]))):
            e = max(e, float(np.abs(got - want).max() / np.abs(want).max()))
        out[str(a)] = e
    return out


def run_l12(args, mg, peak, measured, flush):
    """The largest single instance: h = 2^-12 (4097^2 nodes, 33.6M unknowns),
    alpha = 1e-6, y_D = +-1 piecewise constant plus U(-0.05, 0.05) noise (seed
    5); one solve at a time to the tolerance, FP32+refine against plain FP64,
    each solution's error against the FP64 oracle, and the finest sweep's
    roofline (at this size x and f, 268 MB, exceed the 129 MB L2)."""
    import torch

    from paper_1502_03917_gb300 import inputs

    L, a = 12, 1e-6
    N = ((1 << L) + 1) ** 2
    yD = torch.tensor(inputs.yd_piecewise(L, 5), dtype=torch.float64, device="cuda")

    def timed(precision, K):
        s = mg.Solver(L, a, smoother=args.smoother, precision=precision, cycle=args.cycle, max_iter=100)
        f = s.rhs_from_yd(yD)
        x = torch.zeros_like(f)
        s.solve(f, x, tol=args.tol)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        it = rr = None
        for k in range(K):
            flush.fill_(float(k))
            x.zero_()
            ev[k][0].record()
            it, rr, _ = s.solve(f, x, tol=args.tol)
            ev[k][1].record()
        torch.cuda.synchronize()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / K
        err = error_vs_golden(L, {a: x}, args.smoother)
        s.close()
        return {"value": 2 * N / (ms / 1e3), "ms_per_solve": ms, "iterations": it, "relres": rr,
                "error_vs_oracle": err.get(str(a)) if err else None, "solves_timed": K}

    out = {"workload": f"Poisson control, h=2^-{L} ({(1 << L) + 1}^2 nodes, {2 * N} unknowns), alpha={a:g}, "
                       f"y_D=+-1 piecewise + U(-0.05,0.05) seed 5, {args.smoother.upper()} {args.cycle}(2,2) to "
                       f"h=1/2, tol {args.tol}, one solve at a time, L2 flushed before each; FP32+refine with 3 FP32 "
                       f"cycles per refinement step (library default)",
           "unit": UNIT}
    out["fp32_refine"] = timed("fp32_refine", 3)
    out["fp64_plain"] = timed("fp64", 1)
    out["roofline"] = sweep_roofline(mg, L, yD, a, args, peak, measured)
    out["roofline"].pop("sweeps_per_iteration", None)
    return out


def run_profile_band(args):
    """A small, self-contained launch sequence for ncu: one FP32 LSGS handle
    at h = 2^-L with the default kernels (the band kernel on the finest level
    from 1025^2 nodes), `warmup` + `steps` finest-level smoothing steps through
    mg_smooth, one step per call."""
    import torch

    from paper_1502_03917_gb300 import build as B
    from paper_1502_03917_gb300 import inputs
    import paper_1502_03917_gb300.aaomg as mg

    B.build()
    L = args.profile_band
    with mg.Solver(L, 1e-4, smoother="lsgs", precision="fp32_refine") as s:
        f = torch.tensor(inputs.x_uniform(L, 1), dtype=torch.float64, device="cuda")
        x = torch.tensor(inputs.x_uniform(L, 2), dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            s.smooth(f, x, 1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            s.smooth(f, x, 1)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"profile_band": L, "kernels": s.level_kernels()[L], "steps": args.steps,
                          "ms_per_call": e0.elapsed_time(e1) / max(1, args.steps),
                          "note": "one mg_smooth call = FP64->FP32 conversion, one LSGS step, FP32->FP64"}))


def host_cpu():
    """The host's core count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        outp = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in outp.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "model": model}


def run_e2e(args, solvers, yD, K, world, max_over_ranks, run_all):
    """Same metric through the public host-buffer API: f and x in pinned host
    memory, the host-to-device and device-to-host copies inside the timed
    region; the five solves as one batch (mg_batch_solve_host), or one after
    another through mg_solve_host with --serial."""
    import torch

    import paper_1502_03917_gb300.aaomg as mg

    N = next(iter(solvers.values())).N
    host_f = {}
    for a, s in solvers.items():
        f = s.rhs_from_yd(yD)
        hf = torch.empty(2 * N, dtype=torch.float64, pin_memory=True)
        hf.copy_(f)
        host_f[a] = hf
    hx = {a: torch.empty(2 * N, dtype=torch.float64, pin_memory=True) for a in solvers}
    batch = None if args.serial else mg.Batch([solvers[a] for a in ALPHAS])
    torch.cuda.synchronize()

    def one(a):
        hx[a].zero_()
        solvers[a].solve_host(host_f[a].numpy(), hx[a].numpy(), tol=args.tol)

    def step():
        if batch is None:
            run_all(one)
            return
        for a in ALPHAS:
            hx[a].zero_()
        batch.solve_host([host_f[a].numpy() for a in ALPHAS], [hx[a].numpy() for a in ALPHAS], tol=args.tol)

    step()  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        step()
    torch.cuda.synchronize()
    sec = max_over_ranks(time.perf_counter() - t0)
    if batch is not None:
        batch.close()
    n = len(solvers)
    return {"value": world * n * 2 * N * K / sec, "unit": UNIT, "h2d_bytes_per_step": n * 2 * (2 * N * 8),
            "d2h_bytes_per_step": n * 2 * N * 8, "ms_per_step": 1e3 * sec / K,
            "api": "mg_solve_host per alpha" if batch is None else "mg_batch_solve_host (five alphas, one graph)"}


def oracle_iterations(L, smoother, tol):
    """Iteration counts of the FP64 oracle to `tol`, from the committed
    full-size reference file (written by oracle/make_golden.py)."""
    try:
        g = json.load(open(GOLDEN.format(L=L)))
    except (OSError, ValueError):
        return None
    out = {}
    for r in g["runs"]:
        if r["smoother"] == smoother:
            h = r["history"]
            out[str(r["alpha"])] = next((i for i, v in enumerate(h) if v <= tol), None)
    return out if out and None not in out.values() else None


def cpu_baseline(L, args, its_gpu=None):
    """The FP64 CPU oracle (single-threaded C) timed on one W-cycle of the same
    workload (alpha = 1e-4), scaled by the oracle's iteration counts to the
    tolerance for the five alphas."""
    import numpy as np

    import oracle
    from paper_1502_03917_gb300 import inputs

    oracle.build()
    its = oracle_iterations(L, args.smoother, args.tol) or its_gpu
    o = oracle.Oracle(L, 1e-4, smoother=args.smoother, gamma=2 if args.cycle == "W" else 1)
    f = o.rhs(inputs.yd_sine_noise(L, 1))
    x = np.zeros_like(f)
    t0 = time.perf_counter()
    o.cycle(f, x)
    t_cycle = time.perf_counter() - t0
    o.close()
    N = ((1 << L) + 1) ** 2
    total_it = sum(its.values()) if its else None
    value = len(ALPHAS) * 2 * N / (t_cycle * total_it) if total_it else None
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
            "sample": f"one {args.smoother.upper()} {args.cycle}(2,2) cycle at h=2^-{L}, alpha=1e-4, from x=0 "
                      f"({t_cycle:.2f} s), scaled by the oracle's iteration counts to {args.tol} for the five "
                      f"alphas ({total_it} cycles); assembly excluded",
            "seconds_per_cycle": t_cycle}


# ------------------------------------------------------------ reference arm --
def run_reference(args, rank, world):
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1502_03917_gb300 import inputs

    oracle.build()
    L = args.level
    N = ((1 << L) + 1) ** 2
    its = oracle_iterations(L, args.smoother, args.tol)
    if its is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle iteration counts for h=2^-{L}"}))
        return
    yD = inputs.yd_sine_noise(L, 1)
    # Each step is one oracle W-cycle at full size, alphas in turn, timed as it
    # runs; a cycle does 1/iterations of that alpha's solve, so a step counts
    # 2N / iterations solved unknowns (the value is projected from measured
    # cycle times: a whole oracle solve at this size takes minutes).
    hier = {}
    times, units = [], []
    for k in range(args.warmup + args.steps):
        a = ALPHAS[k % len(ALPHAS)]
        if a not in hier:
            o = oracle.Oracle(L, a, smoother=args.smoother, gamma=2 if args.cycle == "W" else 1)
            hier[a] = (o, o.rhs(yD))
        o, f = hier[a]
        x = np.zeros_like(f)
        t0 = time.perf_counter()
        o.cycle(f, x)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            units.append(2 * N / its[str(a)])
    for o, _ in hier.values():
        o.close()
    sec = sum(times)
    value = sum(units) / sec
    host = host_cpu()
    sample = ("per step one oracle W-cycle at full size (alphas in turn), measured; it counts as 1/iterations of "
              "that alpha's solve (iterations from tests/golden), so the value is projected from cycle times")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "projected": True,
           "config": {"workload": f"Poisson control, h=2^-{L}, alpha in {ALPHAS}, {args.smoother.upper()} "
                                  f"{args.cycle}(2,2), FP64 CPU oracle", "level": L},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host,
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_protocol(args):
    """Section 3's protocol on the GPU, laid out like Table 1: zero right-hand
    side, random start U(-1,1) (seed 7), W-cycles with 2+2 steps (sLSGS 1+1)
    until the error in the L norm has dropped by 1e-6, for k = 5..8 and
    alpha in {1, 1e-6, 1e-12}.  Counts in FP64 and with one FP32 cycle per
    refinement step, beside the paper's (natural order of Algorithm 2; the GPU
    visits the unknowns in the multicolour order)."""
    import torch

    from paper_1502_03917_gb300 import build as B
    from paper_1502_03917_gb300 import inputs
    import paper_1502_03917_gb300.aaomg as mg

    B.build()
    paper = {}
    with open(os.path.join(ROOT, "tests", "golden", "table1_iterations.txt")) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) == 4 and not line.startswith("#"):
                paper[(parts[0], int(parts[1]), float(parts[2]))] = int(parts[3])
    rows = []
    t0 = time.time()
    for sm in ("ne", "lsgs", "slsgs", "cgs"):
        nu = 1 if sm == "slsgs" else 2
        for k in (5, 6, 7, 8):
            x0 = torch.tensor(inputs.x_uniform(k, 7), dtype=torch.float64, device="cuda")
            for a in (1.0, 1e-6, 1e-12):
                row = {"smoother": sm, "k": k, "alpha": a, "paper": paper.get((sm, k, a))}
                for prec in ("fp64", "fp32_refine"):
                    with mg.Solver(k, a, smoother=sm, precision=prec, nu_pre=nu, nu_post=nu, inner_cycles=1) as s:
                        row[prec] = s.protocol_iterations(x0, 1e-6, 300)
                rows.append(row)
    print(json.dumps({"protocol": "section 3 (Table 1 layout), W-cycle, coarsest h = 1/2, multicolour order",
                      "seconds": time.time() - t0, "rows": rows}))


def run_protocol_stokes(args):
    """Section 3's protocol for the Stokes control problem on the GPU, laid out
    like Table 2: zero right-hand side, random start U(-1,1) (seed 7),
    W-cycles with 2+2 steps (sLSGS 1+1, NE damped with tau = 0.35) until the
    error in the L norm (means of p and mu removed) has dropped by 1e-6, for
    k = 4..7 and alpha in {1, 1e-6, 1e-12}, beside the paper's counts (natural
    order of Algorithm 2; the GPU visits the unknowns in the multicolour
    order)."""
    import numpy as np
    import torch

    from paper_1502_03917_gb300 import build as B
    from paper_1502_03917_gb300 import inputs
    from paper_1502_03917_gb300 import stokes

    B.build()
    paper = {}
    with open(os.path.join(ROOT, "tests", "golden", "table2_iterations.txt")) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) == 4 and not line.startswith("#"):
                paper[(parts[0], int(parts[1]), float(parts[2]))] = int(parts[3])
    rows = []
    t0 = time.time()
    for sm in ("ne", "lsgs", "slsgs"):
        for k in (4, 5, 6, 7):
            x0 = torch.tensor(np.random.default_rng(7).uniform(-1.0, 1.0, inputs.stokes_sizes(k)[2]),
                              dtype=torch.float64, device="cuda")
            for a in (1.0, 1e-6, 1e-12):
                with stokes.StokesSolver(k, a, smoother=sm) as s:
                    rows.append({"smoother": sm, "k": k, "alpha": a, "paper": paper.get((sm, k, a)),
                                 "gpu_fp64": s.protocol_iterations(x0, 1e-6, 300)})
    print(json.dumps({"protocol": "section 3 (Table 2 layout), Stokes control, Taylor-Hood, W-cycle, coarsest "
                                  "h = 1/2, multicolour order", "seconds": time.time() - t0, "rows": rows}))


def batch_line(args, count, steps, warmup):
    """The batched-solve configuration: `count` independent instances with
    levels uniform in 6..10, alpha log-uniform in [1e-8, 1], y_D ~ U(-1, 1)
    (one generator, seed 2), LSGS W(2,2), FP32 cycles in FP64 refinement, all
    solved by one launch of a recorded batch graph (mg_batch_solve: the
    convergence tests on the device); value = unknowns solved per second over
    all instances (set-up and graph recording excluded and reported)."""
    import torch

    from paper_1502_03917_gb300 import build as B
    from paper_1502_03917_gb300 import inputs
    import paper_1502_03917_gb300.aaomg as mg

    B.build()
    levels, alphas, yds = inputs.batch_instances(count, 2)
    t0 = time.time()
    solvers = [mg.Solver(L, a, smoother=args.smoother, precision="fp32_refine", cycle=args.cycle, max_iter=100,
                         autotune=args.autotune) for L, a in zip(levels, alphas)]
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    t0 = time.time()
    batch = mg.Batch(solvers)
    graph_s = time.time() - t0
    fs = [s.rhs_from_yd(torch.tensor(y, dtype=torch.float64, device="cuda")) for s, y in zip(solvers, yds)]
    xs = [torch.zeros_like(f) for f in fs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def step():
        for x in xs:
            x.zero_()
        its, rrs, st, code = batch.solve(fs, xs, tol=args.tol)
        return its, rrs, code

    for _ in range(warmup):
        step()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    its = rrs = None
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record()
        its, rrs, code = step()
        ev[k][1].record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    unknowns = sum(2 * (((1 << L) + 1) ** 2) for L in levels)
    hist = {}
    for k in its:
        hist[str(k)] = hist.get(str(k), 0) + 1
    batch.close()
    for s in solvers:
        s.close()
    return {"metric": "batched solves: unknowns/s at %g rel. residual" % args.tol,
            "value": unknowns * steps / (ms / 1e3), "unit": UNIT, "instances": count,
            "unknowns_per_step": unknowns, "steps": steps, "warmup": warmup, "ms_per_step": ms / steps,
            "setup_s": setup_s, "graph_s": graph_s, "iterations": hist, "max_relres": max(rrs),
            "levels": {str(L): levels.count(L) for L in sorted(set(levels))},
            "config": "levels U{6..10}, log10 alpha ~ U[-8,0], y_D ~ U(-1,1), seed 2; "
                      f"{args.smoother.upper()} {args.cycle}(2,2), FP32 cycles in FP64 refinement (3 per step, the "
                      "library default), one batch graph launch per step, L2 flushed before each"}


def run_batch(args):
    print(json.dumps(batch_line(args, args.batch, args.steps, args.warmup)))


def run_autograd16(args):
    """The differentiation configuration: 16 instances at h = 2^-10, alpha =
    1e-2, y_D ~ U(-1,1) (seed 4), u_target ~ N(0,1) (seed 3), loss
    L = 1/2 sum_k ||u_k - u_target,k||^2 with u = lambda / alpha; one step = the
    batched forward solve (FP32 + FP64 refinement, one batch graph) and the
    batched adjoint solve (dL/dy_D and dL/dlog alpha).  Checked against central
    finite differences (step 1e-6) of the same loss from FP64 solves, along a
    random direction in y_D and in log alpha."""
    import numpy as np
    import torch

    from paper_1502_03917_gb300.autograd import clear_cache, control

    L, alpha, B = 10, 1e-2, 16
    N = ((1 << L) + 1) ** 2
    yD = torch.tensor(np.random.default_rng(4).uniform(-1.0, 1.0, (B, N)), dtype=torch.float64, device="cuda")
    ut = torch.tensor(np.random.default_rng(3).standard_normal((B, N)), dtype=torch.float64, device="cuda")
    tol = 1e-10

    def grads():
        y = yD.clone().requires_grad_(True)
        la = torch.tensor(np.log(alpha), dtype=torch.float64, requires_grad=True)
        u = control(y, la, L, tol=tol, precision="fp32_refine")
        loss = 0.5 * ((u - ut) ** 2).sum()
        loss.backward()
        return y.grad, la.grad.item(), loss.item()

    t0 = time.time()
    grads()  # sets up (and caches) the 16 hierarchies and the batch graph
    setup_s = time.time() - t0
    K = 2
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        gy, gla, lval = grads()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K

    # Finite-difference check of instance 0's loss L_0 = 1/2 ||u_0 - u_target,0||^2:
    # its gradient through the same batched forward and adjoint solves (the
    # other instances' adjoint right-hand sides are then zero), against central
    # differences of FP64 solves of instance 0 alone.
    import paper_1502_03917_gb300.aaomg as mg

    y = yD.clone().requires_grad_(True)
    la = torch.tensor(np.log(alpha), dtype=torch.float64, requires_grad=True)
    u = control(y, la, L, tol=tol, precision="fp32_refine")
    (0.5 * ((u[0] - ut[0]) ** 2).sum()).backward()
    g0, gla0 = y.grad[0], la.grad.item()

    def loss0(y0, a):
        with mg.Solver(L, a, smoother="lsgs", precision="fp64", max_iter=200) as s:
            f = s.rhs_from_yd(y0.contiguous())
            x = torch.zeros_like(f)
            s.solve(f, x, tol=1e-12, raise_on_fail=False)
            return 0.5 * float(((s.control(x) - ut[0]) ** 2).sum())

    h = 1e-6
    v = torch.tensor(np.random.default_rng(8).standard_normal(N), dtype=torch.float64, device="cuda")
    fd_y = (loss0(yD[0] + h * v, alpha) - loss0(yD[0] - h * v, alpha)) / (2 * h)
    fd_a = (loss0(yD[0], alpha * np.exp(h)) - loss0(yD[0], alpha * np.exp(-h))) / (2 * h)
    an_y = float((g0 * v).sum())
    gla = gla0
    clear_cache()
    return {"metric": "gradients/s (dL/dy_D and dL/dlog alpha of 16 instances)", "value": B / (ms / 1e3),
            "unit": "instance gradients/s", "instances": B, "level": L, "alpha": alpha,
            "ms_per_step": ms, "steps": K, "setup_s": setup_s, "loss": lval,
            "fd_check": {"instance": 0, "step": h, "precision": "fp64", "dLdv_adjoint": an_y, "dLdv_fd": fd_y,
                         "rel_err_yD": abs(an_y - fd_y) / abs(fd_y), "dLdlogalpha_adjoint": gla,
                         "dLdlogalpha_fd": fd_a, "rel_err_log_alpha": abs(gla - fd_a) / abs(fd_a)},
            "config": "16 x h=2^-10, alpha=1e-2, y_D ~ U(-1,1) seed 4, u_target ~ N(0,1) seed 3, LSGS W(2,2), "
                      "FP32+FP64-refine forward and adjoint solves to 1e-10, one batch graph each"}


STOKES_GOLDEN = os.path.join(ROOT, "tests", "golden", "stokes_L{L}.json")


def run_stokes(args, peak, measured, flush, cpu=True):
    """The Stokes control problem (section 1, eq. (mp3); Taylor-Hood P2-P1):
    h = 2^-9 (4,712,454 unknowns), alpha = 1e-4, desired velocity the
    divergence-free vortex plus 0.1 N(0,1) noise (seed 1), LSGS W(2,2) in FP64
    from x = 0 to a relative residual of 1e-8; one solve at a time, L2 flushed
    before each.  The solution is checked at 256 sampled unknowns against the
    oracle's (tests/golden/stokes_L9.json, solved to 1e-10).  Roofline of the
    dominant kernel, the LSGS colour phases: one finest-level LSGS step (the
    residual and 90 colour launches) timed with CUDA events over ten steps;
    algorithmic bytes per step: the matrix once (column, A_ij, A_ij / L_jj:
    20 B per nonzero), the row data (index, length, start, 1 / N_ii: 24 B per
    unknown), x and r read and written once (32 B per unknown), and the
    residual's pass (12 B per nonzero, f read and r written: 16 B per
    unknown).  CPU baseline: a complete oracle solve of the same workload at
    h = 2^-7 (293,382 unknowns), timed on this host."""
    import numpy as np
    import torch

    from paper_1502_03917_gb300 import inputs
    from paper_1502_03917_gb300 import stokes

    L, a, tol = 9, 1e-4, 1e-8
    vD = torch.tensor(inputs.stokes_vd_vortex(L, 1), dtype=torch.float64, device="cuda")
    t0 = time.time()
    s = stokes.StokesSolver(L, a, smoother="lsgs", max_iter=100)
    setup_s = time.time() - t0
    f = s.rhs_from_vd(vD)
    x = torch.zeros_like(f)
    s.solve(f, x, tol=tol)
    K = 3
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    it = rr = None
    launches0 = s.kernel_launches()
    for k in range(K):
        flush.fill_(float(k))
        x.zero_()
        ev[k][0].record()
        it, rr, _ = s.solve(f, x, tol=tol)
        ev[k][1].record()
    torch.cuda.synchronize()
    launches = (s.kernel_launches() - launches0) // K
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / K
    err = None
    gpath = STOKES_GOLDEN.format(L=L)
    if os.path.exists(gpath):
        g = json.load(open(gpath))
        ref = next(r for r in g["runs"] if r["alpha"] == a)
        idx = np.array(g["sample"])
        s.normalize(x)
        xs = x.cpu().numpy()[idx]
        xo = np.array(ref["x"])
        nv, npn, _ = inputs.stokes_sizes(L)
        blk = np.searchsorted(np.array([nv, 2 * nv, 2 * nv + npn, 3 * nv + npn, 4 * nv + npn]), idx, side="right")
        err = max(float(np.abs(xs[blk == b] - xo[blk == b]).max() / np.abs(xo[blk == b]).max())
                  for b in np.unique(blk))
    # the finest-level LSGS step
    nnz, stored = s.operator_entries()
    steps = 10
    s.smooth(f, x, 2)
    flush.fill_(1.0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.smooth(f, x, steps)
    e1.record()
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / steps
    m = s.m
    phase_bytes = 20 * nnz + (24 + 32) * m
    resid_bytes = 12 * nnz + 16 * m
    achieved = (phase_bytes + resid_bytes / steps) / (step_ms / 1e3) / 1e9
    s.close()
    out = {"metric": "solved unknowns/s at 1e-8 rel. residual (FP64)", "value": m / (ms / 1e3),
           "unit": "unknowns/s", "ms_per_solve": ms, "solves_timed": K, "iterations": it, "relres": rr,
           "setup_s": setup_s, "gpu_launches_per_solve": launches, "error_vs_oracle": err,
           "config": {"workload": f"Stokes control (Taylor-Hood P2-P1), h=2^-{L} ({m} unknowns), alpha={a:g}, "
                                  f"v_D = vortex + 0.1 N(0,1) seed 1, LSGS W(2,2) to h=1/2 (levels <= 5 as one "
                                  f"dense map), FP64, tol {tol}", "l2": "flushed (256 MB write) before every solve"},
           "roofline": {"bound": "hbm", "kernel": "finest-level LSGS step (residual + 90 colour phases, k_st_phase)",
                        "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "peak_source": "measured" if measured else "fallback", "traffic": None,
                        "step_ms": step_ms, "nnz": nnz, "entries_held": stored,
                        "algorithmic_bytes_per_step": phase_bytes + resid_bytes}}
    if cpu:
        from oracle.stokes import StokesOracle

        Lc = 7
        o = StokesOracle(Lc, a, smoother="lsgs")
        fo = o.rhs(inputs.stokes_vd_vortex(Lc, 1))
        t1 = time.time()
        _, ito, _, _ = o.solve(fo, tol=tol, max_iter=100)
        sec = time.time() - t1
        mo = o.m()
        o.close()
        out["cpu_baseline"] = {"value": mo / sec, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                               "sample": f"one complete oracle solve of the same workload at h=2^-{Lc} ({mo} "
                                         f"unknowns, {ito} cycles, {sec:.1f} s), set-up excluded",
                               "host": host_cpu()}
    return out


def run_profile_stokes(args):
    """Profiling runs of the Stokes path (bench workload: alpha = 1e-4, LSGS,
    the vortex desired velocity of seed 1): one W-cycle, or one finest-level
    LSGS step of a hierarchy without the dense map (a small device footprint),
    between cudaProfilerStart and cudaProfilerStop."""
    import torch

    from paper_1502_03917_gb300 import inputs
    from paper_1502_03917_gb300 import stokes

    L = args.profile_stokes or args.profile_stokes_step
    step = not args.profile_stokes
    s = stokes.StokesSolver(L, 1e-4, smoother="lsgs", dense_level=-1 if step else 0)
    f = s.rhs_from_vd(torch.tensor(inputs.stokes_vd_vortex(L, 1), dtype=torch.float64, device="cuda"))
    x = torch.zeros_like(f)
    if not step:
        s.cycle(f, x)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    if step:
        s.smooth(f, x, 1)
    else:
        s.cycle(f, x)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profile": "stokes step" if step else "stokes cycle", "level": L, "unknowns": s.m,
                      "launches": s.kernel_launches()}))
    s.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.profile_stokes or args.profile_stokes_step:
        if rank == 0:
            run_profile_stokes(args)
    elif args.profile_band:
        if rank == 0:
            run_profile_band(args)
    elif args.batch:
        if rank == 0:
            run_batch(args)
    elif args.protocol:
        if rank == 0:
            run_protocol(args)
    elif args.protocol_stokes:
        if rank == 0:
            run_protocol_stokes(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
