"""Benchmark: cell-stage updates/s of the PP-WCNS-IS solver on one GB300.

Workload (the precision study): the 2D shock / air-bubble interaction in
water on a 2048 x 1024 grid ([0,2] x [0,1], symmetry at y = 0, transmissive
elsewhere, seed 2), SSPRK3 steps at CFL 0.5.  One bench step is one SSPRK3
step (three RHS evaluations, i.e. 3 x 2,097,152 cell-stage updates, all
directions fused per stage).  The headline value is the FP64 solver; the
mixed FP32/FP64 solver is the variant.  Both precisions' first step from
the initial state is compared with the FP64 oracle's step on the full grid
(L1 / Linf in rho, p, alpha1); that oracle step is also the timed CPU
baseline.  Inputs are synthetic and seeded (paper_2102_05287_gb300.problems).

Arms:
  default           this library (FP64 headline, mixed FP32/FP64 variant,
                    and both on the 1024 x 512 shock/bubble grid)
  --impl reference  the FP64 C++ oracle on the host cores (a deliberately
                    slow, plain reference; bounded sample of the same
                    workload)

Rooflines (the path has no dense contraction; it is ALU bound):
  roofline                  FP64 sweep: the oracle's op mix per cell and
                            direction (op-counting build, IS weights in their
                            one-division form; add, mul, min/max, division and
                            square root one flop each) over the live
                            CUDA-event time of the dominant sweep, against the
                            FP64 FMA peak measured live by csrc/peaks.cu
  variants.mixed.roofline   mixed sweep: the FP64 steps (node EOS, node
                            fluxes, update) at the FP64 peak plus all other
                            steps at the FP32 peak
  --workload riemann_batch  step-level fractions of the batched mode
  --workload bubble_3d      per-sweep fractions of the 3D solvers

Other workloads (--workload): convergence, riemann_batch, bubble_batch_2d,
bubble_3d, stress, full_runs, precision_2048 (the headline's workload with
more error statistics); each prints its own JSON line.

Multi-GPU (torchrun, one rank per GPU): independent replicas of the
workload, one per rank (weak scaling; no data-path collective).  Rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-stage updates/s per GB300 (FP64 vs mixed) at stated error; % of stencil roofline"
UNIT = "cell-stage updates/s"
WORKLOAD = "shock_bubble_2d_2048x1024"
SEED = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--n3d", type=int, default=384,
                    help="bubble_3d: cells an axis (384 is the workload; smaller grids for profiling)")
    ap.add_argument("--nprob", type=int, default=4096,
                    help="riemann_batch: number of problems (4096 is the workload; fewer for profiling)")
    ap.add_argument("--workload", default="shock_bubble",
                    choices=["shock_bubble", "precision_2048", "convergence", "riemann_batch", "bubble_batch_2d",
                             "bubble_3d", "stress", "full_runs"],
                    help="shock_bubble (default): the headline line; the others measure the remaining "
                         "workloads and print their own JSON line")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "gb300" else "gloo"
        if args.impl == "gb300":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier_and_max(world, value):
    """The maximum of a per-rank value over all ranks (NCCL on the GPUs,
    gloo on the host)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline inputs
# ---------------------------------------------------------------------------
def load_peaks():
    """Vector-pipe peaks: measured FP64/FP32 FMA and division/sqrt rates of
    this GPU (csrc/peaks.cu, run live), HBM copy from MEASURED_PEAKS.json
    when present."""
    out = {}
    exe = os.path.join(ROOT, "paper_2102_05287_gb300", "_build", "peaks")
    try:
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        out.update(json.loads(r.stdout.strip().splitlines()[-1]))
        out["source"] = "measured live (csrc/peaks.cu)"
    except Exception as e:  # keep the bench running
        out["error"] = "peaks microbenchmark failed: %s" % e
    mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(mp):
        try:
            out["measured_peaks_json"] = json.load(open(mp))
        except Exception:
            pass
    return out


OPCOUNTS = os.path.join(ROOT, "profiles", "opcounts.json")


def _opcount_table(name):
    """A stored algorithmic operation-count table (profiles/opcounts.json,
    written by oracle/opcount_table.py from the oracle's op-counting build
    and checked against it by tests/test_bench_roofline.py): per cell and
    direction, in total and per step of the method, the IS weights in their
    one-division form."""
    with open(OPCOUNTS) as f:
        t = json.load(f)[name]
    return t


def algorithmic_ops(nx, ny):
    """Per-cell, per-direction operation mix of one RHS evaluation of the 2D
    shock/bubble workload (measured on a 128 x 64 copy, the stored table;
    the mix is per cell, and the limiters idle on the initial state of
    every grid size)."""
    return _opcount_table("shock_bubble_2d")


# Steps the mixed-precision sweeps compute in FP64 on every cell (node
# pressure and sound speed from the conservative state, the stored node
# fluxes, the flux difference and the SSPRK3 state combination); all other steps run
# in FP32 (the limiters' FP32-certified path; their FP64 theta solves only
# run where certification fails, none on the bench workload).
MIXED_FP64_STEPS = ("node_eos", "node_flux", "update", "ssprk3_combine")
PROFILE_STEPS_MIXED = 5


def mixed_roofline(ops, peaks, avg_ms, ncell, fallbacks):
    """Roofline of the dominant mixed sweep: algorithmic FP64 flops at the
    FP64 FMA peak plus FP32 flops at the FP32 FMA peak (divisions and square
    roots as one flop each); the 'overlapped' form takes the larger of the
    two times instead of their sum."""
    f64 = f32 = 0.0
    for step, c in ops["per_step"].items():
        n = c["add"] + c["mul"] + c["div"] + c["sqrt"] + c["minmax"]
        if step in MIXED_FP64_STEPS:
            f64 += n
        else:
            f32 += n  # the wave-speed maximum included: reduced in FP32 in the combine epilogue
    p64 = peaks.get("fp64_fma_tflops", 1.25) * 1e12
    p32 = peaks.get("fp32_fma_tflops", 76.5) * 1e12
    t64 = f64 * ncell / p64
    t32 = f32 * ncell / p32
    t = avg_ms * 1e-3
    # achieved in FP64-equivalent flop/s: FP32 flops weighted by p64/p32
    achieved = (f64 + f32 * p64 / p32) * ncell / t / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": p64 / 1e12,
            "unit": "TFLOP/s (FP64-equivalent: FP32 flops weighted by the FP64:FP32 peak ratio)",
            "frac": (t64 + t32) / t, "frac_overlapped": max(t64, t32) / t,
            "fp64_flops_per_cell_dir": f64, "fp32_flops_per_cell_dir": f32,
            "roofline_us": (t64 + t32) * 1e6, "roofline_us_overlapped": max(t64, t32) * 1e6,
            "avg_launch_ms": avg_ms, "fp64_fallbacks": fallbacks, "traffic": None,
            "note": "mixed sweep: FP64 steps %s at the measured FP64 FMA peak plus the other steps at the "
                    "measured FP32 FMA peak, divisions and square roots as one flop (FP32 divisions and "
                    "square roots run on the multi-function unit, whose measured rates are in the line's "
                    "peaks: fp32_fdividef_gops, fp32_sqrt_gops), op mix per step from "
                    "the oracle's op-counting build (IS weights in one-division form); frac = roofline "
                    "time / CUDA-event time of one launch (of measured), from %d steps timed per kernel "
                    "right after the graph-replayed timed steps" % (MIXED_FP64_STEPS, PROFILE_STEPS_MIXED)}


def fp64_roofline(ops, peaks, avg_ms, ncell, kernel):
    """Roofline of one launch of an FP64 sweep (one direction over ncell
    cells): the oracle's op mix per cell and direction, every add, mul,
    min/max, division and square root one flop, over the launch time,
    against the measured FP64 FMA peak.  frac_div_sqrt_weighted counts each
    division and square root at its measured cost in FMA-flops instead."""
    p64 = peaks.get("fp64_fma_tflops", 1.25)
    div_eq = (p64 * 1e12) / (peaks.get("fp64_div_gops", 67.0) * 1e9)
    sqrt_eq = (p64 * 1e12) / (peaks.get("fp64_sqrt_gops", 58.5) * 1e9)
    plain = ops["add"] + ops["mul"] + ops["minmax"] + ops["div"] + ops["sqrt"]
    weighted = ops["add"] + ops["mul"] + ops["minmax"] + div_eq * ops["div"] + sqrt_eq * ops["sqrt"]
    t = avg_ms * 1e-3
    achieved = plain * ncell / t / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": p64, "unit": "TFLOP/s", "frac": achieved / p64,
            "traffic": None, "kernel": kernel, "avg_launch_ms": avg_ms,
            "flops_per_cell_dir": plain,
            "frac_div_sqrt_weighted": weighted * ncell / t / 1e12 / p64,
            "flop_eq_per_cell_dir_div_sqrt_weighted": weighted,
            "ops_per_cell_dir": {k: v for k, v in ops.items() if k != "per_step"},
            "peak_source": peaks.get("source", "nominal FP64 1.25 TFLOP/s (fallback)"),
            "note": "FP64-pipe roofline of the dominant sweep: algorithmic flops = the oracle's op mix per cell "
                    "and direction (op-counting build, IS weights in their one-division form), add, mul, "
                    "min/max, division and square root one flop each, x cells of one launch, over the launch's "
                    "live CUDA-event time; peak = the FP64 FMA rate of this GPU measured live (of measured). "
                    "frac_div_sqrt_weighted counts each division / square root at its measured cost in "
                    "FMA-flops (%.1f / %.1f)" % (div_eq, sqrt_eq)}


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def _cfl_dt(sm, pr):
    """dt = CFL / sum_d (max(|u_d| + c) / dx_d), CFL 0.5 (Sec. 3.3)."""
    return 0.5 / sum(sm[d] * pr.n[d] / (pr.hi[d] - pr.lo[d]) for d in range(pr.ndim))


def run_reference(args, world, rank):
    if rank != 0:
        return
    import numpy as np
    from oracle import Oracle
    from paper_2102_05287_gb300 import problems as P
    pr = P.shock_bubble_2d(args.nx, args.ny, seed=SEED)
    # each step is a bounded sample of the workload: one SSPRK3 step of its
    # lowest eighth of rows (the strip along the symmetry plane, with the
    # workload's initial state and boundary conditions), so that all of
    # --warmup W and --steps K run in well under a minute a step
    rows = max(1, pr.n[1] // 8)
    hi = (pr.hi[0], pr.lo[1] + (pr.hi[1] - pr.lo[1]) * rows / pr.n[1])
    o = Oracle((pr.n[0], rows), pr.lo, hi, pr.bcs, **pr.eos)
    W = np.ascontiguousarray(pr.W[:, :rows, :])
    ncell = pr.n[0] * rows

    def step(W):
        sm = o.max_wavespeed(W)
        dt = 0.5 / (sm[0] * pr.n[0] / (hi[0] - pr.lo[0]) + sm[1] * rows / (hi[1] - pr.lo[1]))
        return o.rk3_step(W, dt)

    for _ in range(args.warmup):
        W = step(W)
    steps = args.steps
    t0 = time.perf_counter()
    for _ in range(steps):
        W = step(W)
    el = time.perf_counter() - t0
    value = 3 * ncell * steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if (args.nx, args.ny) == (2048, 1024) else
                   "shock_bubble_2d_%dx%d" % (args.nx, args.ny),
                   "grid": [pr.n[0], pr.n[1]], "precision": "fp64",
                   "step": "one SSPRK3 step (3 RHS evaluations)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": "%d SSPRK3 steps, each of a %dx%d strip of the %dx%d workload (its "
                                   "lowest eighth of rows, initial state and boundary conditions), single "
                                   "thread" % (steps, pr.n[0], rows, pr.n[0], pr.n[1])},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def oracle_step(pr, dt):
    """CPU baseline leg: one SSPRK3 step of the FP64 oracle on the full grid
    from the initial state, single thread, timed.  Its result is also the
    reference of the GPU's first-step errors."""
    from oracle import Oracle
    o = Oracle(pr.n, pr.lo, pr.hi, pr.bcs, **pr.eos)
    t0 = time.perf_counter()
    W1 = o.rk3_step(pr.W, dt)
    el = time.perf_counter() - t0
    cpu = {"value": 3 * pr.ncells / el, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
           "sample": "one SSPRK3 step of the full %dx%d workload from its initial state, single thread "
                     "(the oracle is not threaded), %.1f s" % (pr.n[0], pr.n[1], el)}
    return cpu, W1


# ---------------------------------------------------------------------------
# this library
# ---------------------------------------------------------------------------
def timed_steps(torch, solver, W, steps, flush):
    """Per-step device time with CUDA events on the solver's stream; the L2
    is flushed (a 256 MiB write) between steps, outside the events."""
    stream = solver.stream
    times = []
    launches0 = solver.launches()
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.advance_steps(W, 1, cfl=0.5)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return times, solver.launches() - launches0


def kernel_time(torch, solver, W, flush, steps):
    """Per-direction launch count and summed CUDA-event time of the sweeps
    over `steps` steps, taken right after the graph-replayed timed steps
    (per-kernel events make every launch direct)."""
    solver.profile_enable(16 * steps + 16)
    solver.profile_read()
    timed_steps(torch, solver, W, steps, flush)
    prof = solver.profile_read()
    solver.profile_enable(0)
    return prof


def dominant(prof, ndim):
    d = max((d for d in range(ndim) if prof["launches"][d] > 0), key=lambda d: prof["ms"][d])
    return d, prof["ms"][d] / prof["launches"][d]


def all_sweeps(roof, prof, ndim):
    """Adds the fraction over every sweep launch of the profiled steps (the
    sum of their roofline times over the sum of their CUDA-event times),
    which does not depend on how the work splits between the directions,
    and each direction's own fraction."""
    per_launch_roofline_ms = roof["frac"] * roof["avg_launch_ms"]
    n = sum(prof["launches"][:ndim])
    ms = sum(prof["ms"][:ndim])
    roof["frac_all_sweeps"] = per_launch_roofline_ms * n / ms if ms > 0 else None
    roof["per_direction_avg_launch_ms"] = {"xyz"[d]: prof["ms"][d] / prof["launches"][d]
                                           for d in range(ndim) if prof["launches"][d] > 0}
    return roof


def run_gb300(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2102_05287_gb300 import problems as P
    from paper_2102_05287_gb300.wcns import Solver

    torch.cuda.set_device(local)
    pr = P.shock_bubble_2d(args.nx, args.ny, seed=SEED + rank)
    ncell = pr.ncells
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # ---------------- FP64 (the headline) ----------------------------------
    s64 = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision="fp64", stream=stream, **pr.eos)
    W64 = torch.from_numpy(pr.W).cuda()
    # the first step from the initial state, at the dt both precisions and
    # the oracle take, for the error report
    dt1 = _cfl_dt(s64.max_wavespeed(W64), pr)
    first = {"fp64": s64.rk3_step(W64.clone(), dt1)}
    for _ in range(args.warmup):
        s64.advance_steps(W64, 1, cfl=0.5)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        times64, launches = timed_steps(torch, s64, W64, args.steps, flush)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    clocks = clk.summary()
    ms64 = barrier_and_max(world, sum(times64)) / args.steps
    value = world * 3 * ncell / (ms64 * 1e-3)
    W64_after = W64.cpu()  # after warmup + steps, before the per-kernel timing advances it further
    prof64 = kernel_time(torch, s64, W64, flush, 3)
    stats64 = s64.stats()

    # ---------------- mixed FP32/FP64 variant -------------------------------
    mixed = None
    if not args.no_mixed:
        sm_ = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision="mixed", stream=stream, **pr.eos)
        Wm = torch.from_numpy(pr.W).cuda()
        first["mixed"] = sm_.rk3_step(Wm.clone(), dt1)
        for _ in range(args.warmup):
            sm_.advance_steps(Wm, 1, cfl=0.5)
        torch.cuda.synchronize()
        tm, _ = timed_steps(torch, sm_, Wm, args.steps, flush)
        msm = barrier_and_max(world, sum(tm)) / args.steps
        mixed = {"value": world * 3 * ncell / (msm * 1e-3), "ms_per_step": msm, "speedup_vs_fp64": ms64 / msm,
                 "error_vs_fp64_gpu_after_steps": dict(steps=args.warmup + args.steps,
                                                       **_errors(Wm.cpu(), W64_after, pr.eos, 2)),
                 "stats": sm_.stats()}
        mixed["profile"] = kernel_time(torch, sm_, Wm, flush, PROFILE_STEPS_MIXED)
        sm_.close()

    # ---------------- end to end through the host-buffer entry point --------
    Wh = torch.from_numpy(pr.W).pin_memory()
    s64.advance_steps_host(Wh, 1, cfl=0.5)
    e2e_steps = max(2, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s64.advance_steps_host(Wh, 1, cfl=0.5)
    e2e_el = barrier_and_max(world, time.perf_counter() - t0)
    nbytes = Wh.numel() * 8
    e2e = {"value": world * 3 * ncell * e2e_steps / e2e_el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
           "note": "wcns_advance_steps_host: pinned host state copied in, one SSPRK3 step, copied out"}

    # ---------------- the 1024 x 512 shock/bubble grid ------------------------
    small = {}
    if rank == 0 and (args.nx, args.ny) != (1024, 512):
        pc = P.shock_bubble_2d(1024, 512, seed=1)
        for prec in ("fp64", "mixed"):
            sc = Solver(pc.n, pc.lo, pc.hi, pc.bcs, precision=prec, stream=stream, **pc.eos)
            Wc = torch.from_numpy(pc.W).cuda()
            for _ in range(args.warmup):
                sc.advance_steps(Wc, 1, cfl=0.5)
            tc, _ = timed_steps(torch, sc, Wc, max(3, min(args.steps, 10)), flush)
            msc = sum(tc) / len(tc)
            small[prec] = {"value": 3 * pc.ncells / (msc * 1e-3), "ms_per_step": msc, "steps": len(tc)}
            sc.close()

    if rank != 0:
        s64.close()
        return

    # ---------------- CPU baseline and first-step errors vs the oracle -------
    cpu, W_or = (None, None) if args.no_cpu_baseline else oracle_step(pr, dt1)
    if W_or is not None:
        ref = torch.from_numpy(W_or)
        errs = {prec: _errors(first[prec].cpu(), ref, pr.eos, 2) for prec in first}
    else:
        errs = None

    # ---------------- rooflines of the dominant kernels ----------------------
    peaks = load_peaks()
    ops = algorithmic_ops(args.nx, args.ny)
    dom, avg_ms = dominant(prof64, 2)
    roofline = all_sweeps(fp64_roofline(ops, peaks, avg_ms, ncell,
                                        "sweep_kernel<2,%d,double> (%s sweep)" % (dom, "xy"[dom])), prof64, 2)
    src_hash = hashlib.sha256(open(os.path.join(ROOT, "paper_2102_05287_gb300", "csrc", "wcns_sweep.cuh"),
                                   "rb").read()).hexdigest()[:16]
    traffic_file = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if os.path.exists(traffic_file):
        try:
            tr = json.load(open(traffic_file))
            k = "fp64_dir%d" % dom
            # only counters taken on the current kernel source count; a
            # capture on a smaller grid is scaled by the cells of one launch
            if tr.get("kernel_source_sha256_16") == src_hash and k in tr:
                g = tr[k]["grid"]
                roofline["traffic"] = tr[k]["bytes_per_launch"] * ncell / float(g[0] * g[1])
                roofline["traffic_source"] = "ncu dram bytes of a %dx%d capture, scaled to %d cells" % (
                    g[0], g[1], ncell)
        except Exception:
            pass
    roofline["ops_per_step_per_cell_dir"] = ops["per_step"]
    if mixed:
        pm = mixed.pop("profile")
        dm, avg_m = dominant(pm, 2)
        mixed["roofline"] = mixed_roofline(ops, peaks, avg_m, ncell, mixed["stats"]["fp64_fallbacks"])
        mixed["roofline"]["kernel"] = "sweep_kernel_mixed<2,%d> (%s sweep)" % (dm, "xy"[dm])
        all_sweeps(mixed["roofline"], pm, 2)
        if errs:
            mixed["first_step_error_vs_fp64_oracle"] = errs["mixed"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if (args.nx, args.ny) == (2048, 1024) else
                   "shock_bubble_2d_%dx%d" % (args.nx, args.ny),
                   "grid": [args.nx, args.ny], "cells": ncell, "precision": "fp64", "seed": SEED,
                   "scheme": "PP-WCNS-IS + SSPRK3, CFL 0.5",
                   "step": "one SSPRK3 step = 3 RHS evaluations (x and y sweeps fused with the stage combine)",
                   "l2": "flushed between timed steps (256 MiB write outside the timed events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "wall_s_timed_region": wall,
        "first_step_error_vs_fp64_oracle": errs["fp64"] if errs else None,
        "variants": dict({"mixed": mixed} if mixed else {},
                         **({"shock_bubble_2d_1024x512": small} if small else {})),
        "stats_fp64": stats64,
        "peaks": {k: peaks.get(k) for k in ("fp64_fma_tflops", "fp32_fma_tflops", "fp64_div_gops",
                                           "fp64_sqrt_gops", "fp32_div_gops", "fp32_fdividef_gops",
                                           "fp32_sqrt_gops",
                                           "fp64_copy_gbs", "device")},
    }
    print(json.dumps(line), flush=True)
    s64.close()


# ---------------------------------------------------------------------------
# further workloads (one JSON line each)
# ---------------------------------------------------------------------------
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _pressure(W, eos, ndim):
    """Mixture pressure of a conservative state (Sec. 2), for error reports."""
    a1 = W[3 + ndim]
    rho = W[0] + W[1]
    ke = sum(W[2 + j] * W[2 + j] for j in range(ndim)) / rho
    G = a1 / (eos["gamma_l"] - 1) + (1 - a1) / (eos["gamma_g"] - 1)
    Pi = a1 * eos["gamma_l"] * eos["pinf_l"] / (eos["gamma_l"] - 1)
    return (W[2 + ndim] - 0.5 * ke - Pi) / G


def _errors(a, b, eos, ndim):
    """L1 / Linf errors of a against b, relative, in rho, p, alpha1."""
    out = {}
    for name, fa, fb in (("rho", a[0] + a[1], b[0] + b[1]), ("p", _pressure(a, eos, ndim), _pressure(b, eos, ndim)),
                         ("alpha1", a[3 + ndim], b[3 + ndim])):
        d = (fa - fb).abs()
        out[name] = {"l1": float(d.sum() / fb.abs().sum()), "linf": float(d.max() / fb.abs().max())}
    return out


def workload_precision(args):
    """2048x1024 shock/bubble: FP64 vs mixed on the GPU.  The workload's CPU
    baseline is one SSPRK3 step of the FP64 oracle on the full grid, timed
    on one host core; the GPU's first step of each precision is compared
    with that baseline's result."""
    import numpy as np
    import torch
    from oracle import Oracle
    from paper_2102_05287_gb300 import problems as P
    from paper_2102_05287_gb300.wcns import Solver
    pr = P.shock_bubble_2d(2048, 1024, seed=2)
    res = {}
    states = {}
    one = {}
    for prec in ("fp64", "mixed"):
        s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision=prec, **pr.eos)
        W = torch.from_numpy(pr.W).cuda()
        W1 = W.clone()
        s.advance_steps(W1, 1, cfl=0.5)
        one[prec] = W1
        s.advance_steps(W, args.warmup, cfl=0.5)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        s.advance_steps(W, args.steps, cfl=0.5)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[prec] = {"ms_per_step": ms, "cell_stage_updates_per_s": 3 * pr.ncells / (ms * 1e-3), "stats": s.stats()}
        states[prec] = W
        s.close()
    # CPU baseline leg: the oracle's step, timed; its result is also the
    # reference of the one-step errors below
    o = Oracle(pr.n, pr.lo, pr.hi, pr.bcs, **pr.eos)
    sm = o.max_wavespeed(pr.W)
    t0 = time.perf_counter()
    ref = o.rk3_step(pr.W, 0.5 / (sm[0] * pr.n[0] / 2.0 + sm[1] * pr.n[1]))
    t_or = time.perf_counter() - t0
    ref = torch.from_numpy(ref)
    cpu = {"value": 3 * pr.ncells / t_or, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
           "sample": "one SSPRK3 step of the full 2048x1024 grid, single thread, %.1f s" % t_or}
    line = {"workload": "precision_2048x1024", "metric": METRIC, "unit": UNIT,
            "steps": args.steps, "warmup": args.warmup, "results": res,
            "mixed_speedup_vs_fp64": res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"],
            "mixed_vs_fp64_after_steps": _errors(states["mixed"].cpu(), states["fp64"].cpu(), pr.eos, 2),
            "one_step_vs_cpu_baseline_result": {"fp64": _errors(one["fp64"].cpu(), ref, pr.eos, 2),
                                                "mixed": _errors(one["mixed"].cpu(), ref, pr.eos, 2)},
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


def workload_convergence(args):
    """Smooth 1D interface advection (periodic, alpha1 = 0.5 + 0.25 sin 2 pi x,
    rho1 = 1000, rho2 = 1, u = 1, p = 1e5, dt = 4e-5 dx, t_end = 1e-3) for
    N = 64..4096: L1 error of alpha1 against the exact solution and the
    observed order between successive N, FP64 and mixed.  Each precision's
    round-off floor is taken as its error at the finest grid (where the
    scheme's truncation error is below 1e-14); the order is fitted only over
    the N whose error exceeds 100x that floor (null if fewer than two)."""
    import numpy as np
    import torch
    from paper_2102_05287_gb300 import problems as P
    from paper_2102_05287_gb300.wcns import Solver
    rows = []
    for N in (64, 128, 256, 512, 1024, 2048, 4096):
        pr = P.advection_1d_smooth(N)
        steps = int(round(pr.t_end / pr.dt_fixed))
        row = {"N": N, "steps": steps}
        for prec in ("fp64", "mixed"):
            s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision=prec, **pr.eos)
            W = torch.from_numpy(pr.W).cuda()
            e0, e1 = _events(torch)
            e0.record()
            t = s.advance_steps(W, steps, dt_fixed=pr.dt_fixed)
            e1.record()
            torch.cuda.synchronize()
            a = W[-1].cpu().numpy()
            err = np.abs(a - pr.extra["exact"](t))
            row[prec] = {"l1_alpha1": float(err.mean()), "linf_alpha1": float(err.max()),
                         "ms": e0.elapsed_time(e1)}
            s.close()
        rows.append(row)
    fit = {}
    for prec in ("fp64", "mixed"):
        for a, b in zip(rows[:-1], rows[1:]):
            b[prec]["order"] = float(np.log2(a[prec]["l1_alpha1"] / b[prec]["l1_alpha1"]))
        floor = rows[-1][prec]["l1_alpha1"]
        use = [r for r in rows if r[prec]["l1_alpha1"] > 100.0 * floor]
        fit[prec] = {"floor": floor, "N": [r["N"] for r in use], "order": None}
        if len(use) >= 2:
            fit[prec]["order"] = float(-np.polyfit(np.log([r["N"] for r in use]),
                                                   np.log([r[prec]["l1_alpha1"] for r in use]), 1)[0])
    print(json.dumps({"workload": "convergence_1d_smooth", "t_end": 1e-3, "rows": rows, "fitted_order": fit}),
          flush=True)


def algorithmic_ops_1d(rb=None):
    """Per-cell operation mix of one 1D RHS evaluation, from 16 seeded
    problems of the 4096-problem batch (the stored table; the mix is per
    cell, so it serves smaller batches as well)."""
    return _opcount_table("riemann_batch")


def batch_roofline(ops, peaks, prec, ms_per_step, cells, ndim=1):
    """Step-level roofline fraction of the batched mode: the algorithmic
    work of three RHS evaluations over all cells and directions (every add,
    mul, min/max, division and square root one flop) at the FP64 pipe's
    measured rate (FP64) or at the two pipes' rates (mixed, as
    mixed_roofline), over the whole step's time (the per-problem dt kernel
    included)."""
    sweeps = 3 * ndim
    if prec == "mixed":
        r = mixed_roofline(ops, peaks, ms_per_step / sweeps, cells, fallbacks=None)
        r["note"] = "batched mixed step: " + r["note"] + "; time = the step over its %d sweeps" % sweeps
        return r
    r = fp64_roofline(ops, peaks, ms_per_step / sweeps, cells, "batched FP64 sweeps (the whole step)")
    r["note"] = ("batched FP64 step, time = the step over its %d sweeps (dt kernel included): " % sweeps) + r["note"]
    return r


def workload_batch(args):
    """Independent 1D two-phase Riemann problems (4096 by default;
    log-uniform sizes 128..8192, seed 3): one persistent launch per stage,
    CUDA-graph step, autotuned tiles; FP64 and mixed.  The timed steps of
    each precision run inside an NVTX range named batch_timed_<precision>
    (a profiler can select their launches after the autotuner's)."""
    import torch
    from paper_2102_05287_gb300 import problems as P
    from paper_2102_05287_gb300.wcns import Batch
    rb = P.riemann_batch(nprob=args.nprob)
    total = int(rb.offsets[-1])
    ops = algorithmic_ops_1d(rb)
    peaks = load_peaks()
    res, states = {}, {}
    for prec in ("fp64", "mixed"):
        b = Batch(rb.sizes, [0.0] * len(rb.sizes), [1.0] * len(rb.sizes), "transmissive", "transmissive",
                  precision=prec, **rb.eos)
        W = torch.from_numpy(rb.W).cuda()
        b.advance(W, args.warmup, cfl=0.5)  # includes the autotuning run
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        l0 = b.launches()
        with torch.cuda.nvtx.range("batch_timed_" + prec):
            e0.record()
            b.advance(W, args.steps, cfl=0.5)
            e1.record()
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[prec] = {"ms_per_step": ms, "cell_stage_updates_per_s": 3 * total / (ms * 1e-3),
                     "tuning": b.tuning(), "launches_per_step": (b.launches() - l0) / args.steps,
                     "stats": b.stats(), "roofline": batch_roofline(ops, peaks, prec, ms, total)}
        states[prec] = W
        b.close()
    a, bb = states["mixed"], states["fp64"]
    err = {"l1_rel_rho": float(((a[0] + a[1]) - (bb[0] + bb[1])).abs().sum() / (bb[0] + bb[1]).abs().sum()),
           "l1_rel_alpha1": float((a[4] - bb[4]).abs().sum() / bb[4].abs().sum())}
    # the oracle on the host: one CFL step of 32 seeded problems of the batch
    import numpy as np
    from oracle import Oracle
    picks = np.random.default_rng(0).choice(len(rb.sizes), 32, replace=False)
    cells, t0 = 0, time.perf_counter()
    for k in picks:
        n = int(rb.sizes[k])
        W0 = np.ascontiguousarray(rb.W[:, int(rb.offsets[k]):int(rb.offsets[k + 1])])
        o = Oracle((n,), (0.0,), (1.0,), (("transmissive", "transmissive"),), **rb.eos)
        o.rk3_step(W0, 0.5 / (o.max_wavespeed(W0)[0] * n))
        cells += n
    el = time.perf_counter() - t0
    cpu = {"value": 3 * cells / el, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
           "sample": "one SSPRK3 step of 32 seeded problems of the batch (%d cells), single thread, %.1f s"
                     % (cells, el)}
    print(json.dumps({"workload": "riemann_batch_%d" % len(rb.sizes), "problems": len(rb.sizes), "cells": total,
                      "steps": args.steps, "warmup": args.warmup, "results": res,
                      "mixed_speedup_vs_fp64": res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"],
                      "mixed_vs_fp64_after_steps": err, "cpu_baseline": cpu}), flush=True)


def workload_batch_2d(args):
    """Independent 2D shock / air-bubble problems of uneven sizes (1024 by
    default; 32..256 cells an axis, log-uniform, drawn separately, seed 5):
    one persistent launch per direction and stage, CUDA-graph step,
    autotuned persistent grid; FP64 and mixed."""
    import numpy as np
    import torch
    from oracle import Oracle
    from paper_2102_05287_gb300 import problems as P
    from paper_2102_05287_gb300.wcns import Batch
    nprob = args.nprob if args.nprob != 4096 else 1024
    gb = P.bubble_batch_2d(nprob=nprob, seed=5, nmin=32, nmax=256)
    total = int(gb.offsets[-1])
    ops = algorithmic_ops(0, 0)
    peaks = load_peaks()
    res, states = {}, {}
    for prec in ("fp64", "mixed"):
        b = Batch.grids(gb.sizes, gb.lo, gb.hi, gb.bcs, precision=prec, **gb.eos)
        W = torch.from_numpy(gb.W).cuda()
        b.advance(W, args.warmup, cfl=0.5)  # includes the autotuning run
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        l0 = b.launches()
        e0.record()
        b.advance(W, args.steps, cfl=0.5)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[prec] = {"ms_per_step": ms, "cell_stage_updates_per_s": 3 * total / (ms * 1e-3),
                     "tuning": b.tuning(), "launches_per_step": (b.launches() - l0) / args.steps,
                     "stats": b.stats(), "roofline": batch_roofline(ops, peaks, prec, ms, total, ndim=2)}
        states[prec] = W.cpu()
        b.close()
    err = _errors(states["mixed"], states["fp64"], gb.eos, 2)
    # the oracle on the host: one CFL step of 64 seeded problems of the batch
    picks = np.random.default_rng(0).choice(nprob, min(64, nprob), replace=False)
    cells, t0 = 0, time.perf_counter()
    for k in picks:
        nx, ny = (int(v) for v in gb.sizes[k])
        W0 = np.ascontiguousarray(gb.problem(k))
        o = Oracle((nx, ny), (0.0, 0.0), (1.0, 1.0), gb.bcs, **gb.eos)
        sm = o.max_wavespeed(W0)
        o.rk3_step(W0, 0.5 / (sm[0] * nx + sm[1] * ny))
        cells += nx * ny
    el = time.perf_counter() - t0
    cpu = {"value": 3 * cells / el, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
           "sample": "one SSPRK3 step of %d seeded problems of the batch (%d cells), single thread, %.1f s"
                     % (len(picks), cells, el)}
    print(json.dumps({"workload": "bubble_batch_2d_%d" % nprob, "problems": nprob, "cells": total,
                      "steps": args.steps, "warmup": args.warmup, "results": res,
                      "mixed_speedup_vs_fp64": res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"],
                      "mixed_vs_fp64_after_steps": err, "cpu_baseline": cpu}), flush=True)


def workload_3d(args):
    """3D air-bubble collapse in water, 384^3, 7 fields SoA: mixed (the
    workload's precision) and FP64, a few SSPRK3 steps each, then two more
    with per-sweep CUDA events for the rooflines of the x, y and z sweeps
    (FP64: the oracle's 3D op mix at the FP64 peak; mixed: the two-pipe
    roofline)."""
    import torch
    from paper_2102_05287_gb300 import problems as P
    from paper_2102_05287_gb300.wcns import Solver
    pr = P.bubble_collapse_3d(args.n3d)
    ops = _opcount_table("bubble_collapse_3d")
    peaks = load_peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    res, states = {}, {}
    for prec in ("mixed", "fp64"):
        s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision=prec, **pr.eos)
        W = torch.from_numpy(pr.W).cuda()
        s.advance_steps(W, 1, cfl=0.5)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        k = max(1, min(args.steps, 3))
        e0.record()
        s.advance_steps(W, k, cfl=0.5)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        prof = kernel_time(torch, s, W, flush, 2)
        sweeps = {}
        for d in range(3):
            avg = prof["ms"][d] / max(prof["launches"][d], 1)
            if prec == "fp64":
                r = fp64_roofline(ops, peaks, avg, pr.ncells, "sweep_kernel<3,%d,double>" % d)
            else:
                r = mixed_roofline(ops, peaks, avg, pr.ncells, fallbacks=None)
                r["kernel"] = "sweep_kernel_mixed<3,%d>" % d
            sweeps["xyz"[d]] = {"avg_launch_ms": avg, "frac": r["frac"]}
        dom, avg_dom = dominant(prof, 3)
        if prec == "fp64":
            roof = fp64_roofline(ops, peaks, avg_dom, pr.ncells, "sweep_kernel<3,%d,double>" % dom)
        else:
            roof = mixed_roofline(ops, peaks, avg_dom, pr.ncells, fallbacks=None)
            roof["kernel"] = "sweep_kernel_mixed<3,%d>" % dom
        all_sweeps(roof, prof, 3)
        roof.pop("ops_per_cell_dir", None)
        res[prec] = {"ms_per_step": ms, "steps": k, "cell_stage_updates_per_s": 3 * pr.ncells / (ms * 1e-3),
                     "stats": s.stats(), "roofline": roof, "sweeps": sweeps}
        states[prec] = W.cpu()
        del W
        s.close()
        torch.cuda.empty_cache()
    err = _errors(states["mixed"], states["fp64"], pr.eos, 3)
    del states
    # the oracle on the host: one CFL step of the same problem at 48^3,
    # a per-cell-stage rate extrapolated to 384^3
    from oracle import Oracle
    small = P.bubble_collapse_3d(48)
    o = Oracle(small.n, small.lo, small.hi, small.bcs, **small.eos)
    t0 = time.perf_counter()
    sm = o.max_wavespeed(small.W)
    o.rk3_step(small.W, 0.5 / (sum(sm) * 48))
    el = time.perf_counter() - t0
    cpu = {"value": 3 * small.ncells / el, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
           "kind": "oracle",
           "sample": "one SSPRK3 step of the same problem at 48^3 (single thread, %.1f s), "
                     "rate extrapolated to 384^3" % el}
    print(json.dumps({"workload": "bubble_collapse_3d_%d" % args.n3d, "cells": pr.ncells, "results": res,
                      "mixed_speedup_vs_fp64": res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"],
                      "mixed_vs_fp64_after_steps": err, "cpu_baseline": cpu}),
          flush=True)


def workload_stress(args):
    """Section 6 robustness problems at the paper's grids: Mach 10 shock /
    water cylinder 1152x768 and Mach 100 water jet 1024x512, CFL 0.5.
    PP-WCNS-IS in FP64 and mixed precision for a fixed number of steps
    (default 1000): admissibility counters, limiter activity, throughput and
    the minimum of every bounded quantity at the end; then the unlimited
    WCNS-IS ablation, stepped until the device counters report a state
    outside the admissible set (or the same number of steps)."""
    import numpy as np
    import torch
    from paper_2102_05287_gb300 import problems as P
    from paper_2102_05287_gb300.wcns import Solver
    nsteps = args.steps if args.steps != 20 else 1000
    out = []
    for pr in (P.mach10_water_cylinder(1152, 768), P.mach100_water_jet(1024, 512)):
        kw = {}
        if "dirichlet" in pr.extra:
            kw = dict(dirichlet=pr.extra["dirichlet"], dirichlet_face=pr.extra["dirichlet_face"])
        row = {"problem": pr.name, "grid": list(pr.n), "steps": nsteps}
        for prec in ("fp64", "mixed"):
            s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision=prec, **pr.eos, **kw)
            W = torch.from_numpy(pr.W).cuda()
            e0, e1 = _events(torch)
            e0.record()
            t = s.advance_steps(W, nsteps, cfl=0.5)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / nsteps
            Wc = W.cpu().numpy()
            a1 = Wc[-1]
            rho = Wc[0] + Wc[1]
            row[prec] = {"t": t, "ms_per_step": ms, "cell_stage_updates_per_s": 3 * pr.ncells / (ms * 1e-3),
                         "stats": s.stats(), "min_a1r1": float(Wc[0].min()), "min_a2r2": float(Wc[1].min()),
                         "min_alpha1": float(a1.min()), "min_1_minus_alpha1": float((1 - a1).min()),
                         "min_rho_ctilde2": float(_rho_ct2(Wc, pr.eos, 2).min()),
                         "max_rho": float(rho.max())}
            s.close()
        # mixed vs FP64 at the same time: the mixed run advanced to the FP64 run's end time
        s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision="mixed", **pr.eos, **kw)
        Wm = torch.from_numpy(pr.W).cuda()
        s.advance_to(Wm, 0.0, row["fp64"]["t"], cfl=0.5)
        s.close()
        W64 = torch.from_numpy(pr.W).cuda()
        s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision="fp64", **pr.eos, **kw)
        s.advance_to(W64, 0.0, row["fp64"]["t"], cfl=0.5)
        s.close()
        row["mixed_vs_fp64_same_time"] = _errors(Wm.cpu(), W64.cpu(), pr.eos, 2)
        # the problem's own sensitivity: FP64 from the initial state with
        # every value perturbed by a seeded relative 1e-15
        rng = np.random.default_rng(11)
        Wp = torch.from_numpy(pr.W * (1.0 + 1e-15 * rng.uniform(-1.0, 1.0, pr.W.shape))).cuda()
        s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision="fp64", **pr.eos, **kw)
        s.advance_to(Wp, 0.0, row["fp64"]["t"], cfl=0.5)
        s.close()
        row["fp64_vs_fp64_perturbed_1e-15_same_time"] = _errors(Wp.cpu(), W64.cpu(), pr.eos, 2)
        del Wm, W64, Wp
        s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, scheme="wcns-is", **pr.eos, **kw)
        W = torch.from_numpy(pr.W).cuda()
        failed_at = None
        from paper_2102_05287_gb300.wcns import WcnsError
        for k in range(nsteps):
            try:
                s.advance_steps(W, 1, cfl=0.5)
            except WcnsError as e:  # WCNS_E_INADMISSIBLE or WCNS_E_NONFINITE
                failed_at = k  # steps completed before the one whose call reported it
                failed_status = e.status
                break
        row["unlimited_wcns_is"] = {"flagged_after_steps": failed_at,
                                    "status": failed_status if failed_at is not None else 0, "stats": s.stats()}
        s.close()
        out.append(row)
    print(json.dumps({"workload": "stress_section6", "results": out}), flush=True)


def workload_full_runs(args):
    """The five configurations at their stated lengths, one JSON line:
    1D water-air shock tube to t = 2.4e-4 (FP64, next to its CPU baseline:
    the same run of the FP64 oracle on one host core), 2D shock/bubble
    1024x512 for 2000 steps (FP64 and mixed), the 4096-problem batch for 500
    steps (FP64 and mixed), 3D bubble collapse 384^3 for 500 steps (mixed).
    Device counters, wall time and the mixed-vs-FP64 difference at the end.
    (The shock tube against the exact two-stiffened-gas Riemann solution is
    checked in tests/test_gpu_parity.py.)"""
    import numpy as np
    import torch
    from oracle import Oracle
    from paper_2102_05287_gb300 import problems as P
    from paper_2102_05287_gb300.wcns import Batch, Solver
    out = {}
    # config 0
    pr = P.water_air_shock_tube(200)
    s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, **pr.eos)
    W = torch.from_numpy(pr.W).cuda()
    t, steps = s.advance_to(W, 0.0, pr.t_end, cfl=0.5)
    Wg = W.cpu().numpy()
    # CPU baseline leg: the same run of the oracle, timed; the GPU's end
    # state is compared with its result
    o = Oracle(pr.n, pr.lo, pr.hi, pr.bcs, **pr.eos)
    t0 = time.perf_counter()
    Wo, to, so = o.advance_to(pr.W, 0.0, pr.t_end, cfl=0.5)
    el = time.perf_counter() - t0
    out["config0_shock_tube_200"] = {
        "t": t, "steps": steps, "stats": s.stats(),
        "cpu_baseline": {"value": 3 * 200 * so / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "the full run (%d steps), single thread, %.2f s" % (so, el)},
        "l1_rho_gpu_vs_cpu_baseline_result": float(np.abs((Wg[0] + Wg[1]) - (Wo[0] + Wo[1])).sum() /
                                                   np.abs(Wo[0] + Wo[1]).sum())}
    s.close()
    # config 1
    pr = P.shock_bubble_2d(1024, 512)
    res, states = {}, {}
    for prec in ("fp64", "mixed"):
        s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision=prec, **pr.eos)
        W = torch.from_numpy(pr.W).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t = s.advance_steps(W, 2000, cfl=0.5)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        res[prec] = {"t": t, "wall_s": el, "cell_stage_updates_per_s": 3 * 2000 * pr.ncells / el, "stats": s.stats()}
        states[prec] = W.cpu()
        s.close()
    # compare at the same time: the mixed run advanced to the FP64 run's end time
    s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision="mixed", **pr.eos)
    Wm = torch.from_numpy(pr.W).cuda()
    s.advance_to(Wm, 0.0, res["fp64"]["t"], cfl=0.5)
    s.close()
    res["mixed_vs_fp64_same_time"] = _errors(Wm.cpu(), states["fp64"], pr.eos, 2)
    # the problem's own sensitivity after 2000 steps: FP64 from the initial
    # state perturbed by a seeded relative 1e-15
    rng = np.random.default_rng(11)
    Wp = torch.from_numpy(pr.W * (1.0 + 1e-15 * rng.uniform(-1.0, 1.0, pr.W.shape))).cuda()
    s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision="fp64", **pr.eos)
    s.advance_to(Wp, 0.0, res["fp64"]["t"], cfl=0.5)
    s.close()
    res["fp64_vs_fp64_perturbed_1e-15_same_time"] = _errors(Wp.cpu(), states["fp64"], pr.eos, 2)
    out["config1_shock_bubble_1024x512_2000_steps"] = res
    # config 3
    rb = P.riemann_batch()
    res = {}
    for prec in ("fp64", "mixed"):
        b = Batch(rb.sizes, np.zeros(len(rb.sizes)), np.ones(len(rb.sizes)), "transmissive", "transmissive",
                  precision=prec, **rb.eos)
        W = torch.from_numpy(rb.W).cuda()
        tt = torch.zeros(len(rb.sizes), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.advance(W, 500, cfl=0.5, t=tt)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        res[prec] = {"wall_s": el, "cell_stage_updates_per_s": 3 * 500 * int(rb.offsets[-1]) / el,
                     "stats": b.stats(), "tuning": b.tuning(), "t_min": float(tt.min()), "t_max": float(tt.max())}
        b.close()
    out["config3_riemann_batch_4096_500_steps"] = res
    # config 4
    pr = P.bubble_collapse_3d(384)
    s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision="mixed", **pr.eos)
    W = torch.from_numpy(pr.W).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t = s.advance_steps(W, 500, cfl=0.5)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    Wc = W.cpu().numpy()
    out["config4_bubble_collapse_384_500_steps_mixed"] = {
        "t": t, "wall_s": el, "cell_stage_updates_per_s": 3 * 500 * pr.ncells / el, "stats": s.stats(),
        "min_a1r1": float(Wc[0].min()), "min_a2r2": float(Wc[1].min()), "min_alpha1": float(Wc[-1].min()),
        "max_alpha1": float(Wc[-1].max()), "min_rho_ctilde2": float(_rho_ct2(Wc, pr.eos, 3).min())}
    s.close()
    print(json.dumps({"workload": "full_runs", "results": out}), flush=True)


def _rho_ct2(W, eos, ndim):
    """rho ctilde^2 = rho e - pbar of every cell (Sec. 2), for reports."""
    a1 = W[3 + ndim]
    rho = W[0] + W[1]
    rhoe = W[2 + ndim] - 0.5 * sum(W[2 + j] ** 2 for j in range(ndim)) / rho
    G = a1 / (eos["gamma_l"] - 1) + (1 - a1) / (eos["gamma_g"] - 1)
    Pi = a1 * eos["gamma_l"] * eos["pinf_l"] / (eos["gamma_l"] - 1)
    return rhoe - Pi / (G + 1)


def main():
    args = parse()
    if args.workload != "shock_bubble":
        {"precision_2048": workload_precision, "convergence": workload_convergence,
         "riemann_batch": workload_batch, "bubble_batch_2d": workload_batch_2d, "bubble_3d": workload_3d,
         "stress": workload_stress,
         "full_runs": workload_full_runs}[args.workload](args)
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gb300(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
