"""Benchmark of the Sakura all-pairs Kepler step on GB300.

Metric: pair-Kepler solves per second, counted as N^2 * steps / s (the
literal N^2 count; the kernel solves each of the N(N-1)/2 unordered pairs
once and applies it to both particles).

Default workload: equal-mass Plummer sphere, N = 1024, virial units,
dt = 2^-8, 256 steps (one N-body time unit), second-order map, FP64.  A
step is the pair kernel (every unordered pair's Kepler solve on systolic
32 x 32 tiles) and the apply kernel (Eqs. 27b-d), which also drifts for the
next step (Eq. 27a); a call's first step has a prep kernel for its drift.
The 256 steps are timed as 8 calls of ``sakura_evolve`` of 32 steps
(``--steps-per-call``; 1 times single ``sakura_step`` calls, each with its
own prep kernel), each call timed with CUDA events on the library stream.
The state (56 KB) fits in L2, so a 256 MB buffer is written between timed
calls to flush L2.  The pair kernel's own duration (the roofline's
denominator) is taken with CUDA events around each pair-kernel launch in a
second pass of the same calls, so that those events, which hold each launch
until the previous kernel has finished, do not add to the timed steps.  The
9-body planetary workload (72 pairs per step) runs in the single-block
kernel for small systems and is timed as calls of ``sakura_evolve`` of 100
steps each, one launch per call.

Printed JSON line (rank 0): value (device-resident throughput of the plain
FP64 form), e2e (the same through the host-buffer entry point
``sakura_evolve_host``, copies included), roofline of the pair kernel
against the FP64 ALU peak, variants.df64 (the same workload in the
double-word form: FP64-accurate pair solves on the FP32 pipe, against the
FP32 peak), cpu_baseline (the CPU oracle on the host cores), clocks sampled
during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload plummer1024|bh16384|binaries16384|planetary9|ensemble4096]
                    [--form fp64|mixed|df64] [--pairs symmetric|ordered]

Multi-GPU (torchrun, one process per GPU): every rank integrates its own
independently seeded replica; no data-path collective (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-Kepler solves/sec (N^2*steps/s)"
UNIT = "pair-solves/s"

# FP64 operations of one ordered pair in the pair kernel, counted by hand
# from paper_1402_3325_gb300/csrc/{step_fp64.cu,kepler_fp64.cuh}: FMA = 2,
# add/sub/mul = 1 (comparisons run on the integer pipe and are not counted).
#   C_FIX  = relative state and m_ij (7) + setup: backward drift, r0 and 1/r0
#            by seeded third-order refinement, eta0, v0^2, beta (2 m_ij by an
#            exponent add), zeta0 and the second-order guess (48) + Lagrange
#            epilogue (26) + m_j-weighted accumulation (12)
#   C_EVAL = one evaluation: beta s^2 (1), 3-term Stumpff series (12),
#            G-functions (5), F, F', F'' (13), 1/F' (6), Newton step and
#            convergence test (3)
#   C_STEP = one Laguerre correction (6)
# per pair: C_FIX + kbar * C_EVAL + (kbar - 1) * C_STEP, kbar = measured mean
# evaluations.  ncu cross-check (profiles/pair_step_fp64_plummer1024.md):
# 191 FP64 flops per pair executed, 4 % above this count.
C_FIX = 93
C_EVAL = 40
C_STEP = 6
# the symmetric mode adds the column accumulation (6 FMA) to every solve
C_SYM = 12
# a solve finished by the Taylor carry (single-precision seed): one more
# Laguerre correction (C_STEP) and the carry of G1..G3 and F' with a new
# 1/F' (28: h2 (1; the half by an exponent add), dF''/ds (4), three G's and
# F' (17), reciprocal (6))
C_CARRY = 28
# the seeded solve skips the standard (1) and second-order (4) guesses and
# the tolerance test's product (1), takes its near-root step in Halley form
# (the same count, less the half of q done by an exponent add: 1), scales
# the carry test by |s| (1) and forms the step's 1/F' by one quadratic
# refinement (2)
C_SEED_SAVED = 10
# FP32-class pair of the symmetric mixed form (see the roofline code below)
C_MIX32_FIX = 46 + 44 + 168
C_MIX32_ITER = 71

# FP64 ALU peak of one GB300: 152 SMs x 2 FP64 FMA units x 2 flop x 2.07 GHz
# (the unit count follows from the nominal 1.25 TFLOP/s at 2.07 GHz).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
# FP32 pipe peak of one GB300: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.07

# FP32 operations (FMA = 2) of one double-word pair solve, counted by running
# the library's double-word code on the host with an operation tally over the
# pairs of each workload's first step (tests/df64_flop_count.py; a CPU test
# checks these figures against the current code)
DF64_FLOPS_PER_SOLVE = {"plummer1024": 1922.0, "bh16384": 1922.0, "binaries16384": 1922.0}


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest of every rank's x (the timing rule: the slowest rank sets
    the job's time); x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, work_per_rank: float, ms_total: float) -> float:
    """Whole-job throughput of `world` replicas, each doing work_per_rank
    units (N^2 * steps), over the slowest rank's time in milliseconds."""
    return world * work_per_rank / (ms_total * 1e-3)


def _workload(name: str, seed: int):
    from paper_1402_3325_gb300 import ics
    if name == "plummer1024":
        return ics.plummer(1024, seed=seed), 256, (
            "plummer-N1024 equal-mass virial (E=-1/4), dt=2^-8, 256 steps = 1 N-body time unit,"
            " order 2")
    if name == "bh16384":
        return ics.bh_cluster(16384, seed=seed), 256, (
            "black hole (m=1) + 16383 stars (total 1e-2), Plummer a=1, circular velocities,"
            " dt=2^-10, order 2")
    if name == "binaries16384":
        return ics.plummer_binaries(16384, seed=seed), 64, (
            "Plummer N=16384 with 10% primordial binaries (a in [1e-4,1e-2], thermal e),"
            " dt=2^-10, order 2")
    if name == "ensemble4096":
        return ics.ensemble(4096, seed=seed), 1000, (
            "4096 independent planetary systems, N uniform in [3,64], per-system"
            " dt = P_inner/200, 1000 steps in one batched call (CUDA graph), order 2")
    if name == "planetary9":
        return ics.planetary(seed), 2000, (
            "planetary N=9 (central mass 1 + 8 planets), dt=P_inner/200, 2000 steps, order 2")
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if parts[3 + k].lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def _kernel_sources_hash(kernel: str = "pair_step_sym") -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1402_3325_gb300", "csrc")
    files = {"pair_step_sym": ["df64.cuh", "kepler_df64.cuh", "step_sym.cu"],
             "pair_step_fp64": ["step_fp64.cu"],
             "pair_step_sym_df64": ["df64.cuh", "kepler_df64.cuh", "step_df64.cu"],
             "small": ["df64.cuh", "kepler_df64.cuh", "step_small.cu", "step_small.cuh"],
             "batched": ["df64.cuh", "kepler_df64.cuh", "mlp_infer.cuh", "step_batched.cu",
                         "step_batched.cuh"]}.get(
                 kernel, ["step_fp64.cu"])
    for f in ["kepler_fp64.cuh", "pair_batch_fp64.cuh", "fp_bits.cuh", "step_common.cuh",
              "kepler_fp32.cuh"] + files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(workload: str, kernel: str):
    """DRAM bytes per pair-kernel launch from the committed ncu summary, or
    None when the summary is missing or the kernel changed since."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for ln in fh:
            if ":" in ln and ln.lstrip().startswith("- "):
                k, v = ln.lstrip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_sources_sha256_16") != _kernel_sources_hash(kernel):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _cpu_baseline(s, dt, budget_s=10.0, max_steps=256, min_s=2.0):
    """The oracle on the host cores: up to max_steps consecutive steps of the
    workload from its initial state, stopped after budget_s; a workload that
    takes less than min_s is run again from its initial state until min_s
    has passed (a few milliseconds cannot be timed reliably)."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.build()
    t0 = time.perf_counter()
    steps = passes = 0
    while True:
        r, v = s.r.copy(), s.v.copy()
        for _ in range(max_steps):
            rc, r, v = oracle.step(s.m, r, v, dt, 2, nthreads=cores)
            steps += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        passes += 1
        el = time.perf_counter() - t0
        if el >= min_s or el >= budget_s:
            break
    what = (f"{steps} consecutive steps" if passes == 1 else
            f"{passes} passes of {max_steps} consecutive steps")
    return {"value": s.n ** 2 * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what} of the same workload (N={s.n}) from its initial state,"
                      f" OpenMP over i on {cores} threads, {el:.1f} s"}


def run_reference(args, rank):
    """The reference arm: the CPU oracle as it stands on the host cores."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    s, _, desc = _workload(args.workload, 0)
    cores = os.cpu_count() or 1
    r, v = s.r.copy(), s.v.copy()
    for _ in range(args.warmup):
        rc, r, v = oracle.step(s.m, r, v, s.dt, 2, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rc, r, v = oracle.step(s.m, r, v, s.dt, 2, nthreads=cores)
    el = time.perf_counter() - t0
    value = s.n ** 2 * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "n": s.n, "dt": s.dt, "order": 2},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed steps after {args.warmup} warm-up"
                                       f" steps, full N={s.n}, OpenMP over i on {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ensemble(args, rank, world, device, stream, dist):
    """The batched ensemble: one sakura_step_batched call runs all K steps
    (state kept in shared memory), timed with CUDA events on the stream."""
    import numpy as np
    import torch

    from paper_1402_3325_gb300 import sakura as sk
    ens, _, desc = _workload(args.workload, seed=rank)
    guess = {"taylor": sk.GUESS_TAYLOR, "standard": sk.GUESS_STANDARD,
             "learned": sk.GUESS_LEARNED, "fp32": sk.GUESS_FP32}[args.guess]
    sizes = ens.offsets[1:] - ens.offsets[:-1]
    n2 = int((sizes * sizes).sum())
    st0 = torch.tensor(ens.state, device=device)  # initial state, kept for resets
    st = st0.clone()
    m = torch.tensor(ens.m, device=device)
    off = torch.tensor(ens.offsets, device=device)
    dt = torch.tensor(ens.dt, device=device)
    sk.init(device.index, stream=stream.cuda_stream, guess=guess, flags=sk.FLAG_STATS)
    if args.guess == "learned":
        from paper_1402_3325_gb300 import learned
        learned.load_default()
    sk.step_batched(st, m, off, ens.offsets, dt, 2, args.warmup)   # schedule, autotune
    sk.check()
    stt = sk.get_stats(reset=True)
    kbar = stt["iters"] / max(1, stt["solves"])
    carried = stt.get("carries", 0) / max(1, stt["solves"])
    lane_eff = stt["iters"] / max(1, stt["warp_slots"])
    warps, blocks, tune = sk.batched_tuning()
    sk.init(device.index, stream=stream.cuda_stream, guess=guess)
    st.copy_(st0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(device)
    with ClockSampler(device.index) as clocks:
        e0.record(stream)
        sk.step_batched(st, m, off, ens.offsets, dt, 2, args.steps)
        e1.record(stream)
        torch.cuda.synchronize(device)
    sk.check()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, device)
    value = whole_job_value(world, n2 * args.steps, ms)
    # end to end: host buffers copied in and out around the same call
    host = torch.empty(tuple(st.shape), dtype=torch.float64).pin_memory()
    host.copy_(torch.tensor(ens.state))
    t0 = time.perf_counter()
    st.copy_(host, non_blocking=True)
    sk.step_batched(st, m, off, ens.offsets, dt, 2, args.steps)
    host.copy_(st, non_blocking=True)
    torch.cuda.synchronize(device)
    el = time.perf_counter() - t0
    if rank != 0:
        return 0
    # every unordered pair is solved once and applied to both particles
    solves = int((sizes * (sizes - 1)).sum()) // 2
    flops_solve = (C_FIX + kbar * C_EVAL + (kbar - 1.0) * C_STEP + carried * (C_STEP + C_CARRY) +
                   C_SYM - (C_SEED_SAVED if args.guess == "fp32" else 0))
    achieved = solves * args.steps * flops_solve / (ms * 1e-3) / 1e12
    peak = FP64_PEAK_GFLOPS / 1e3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "nsys": ens.nsys, "particles": int(ens.offsets[-1]),
                       "n2_per_step": n2, "pairs_solved_per_step": solves, "order": 2,
                       "form": "batched",
                       "kepler_guess": args.guess,
                       "block_warps": warps, "blocks": blocks, "autotune_ms": tune,
                       "l2": "state (7.7 MB) stays in shared memory for the whole call"},
            "gpu_launches": 1,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         # a launch reads the state once, whatever its step count
                         "traffic": _profiled_traffic(args.workload, "batched"),
                         "kernel": "batched_kernel", "pipe": "fp64",
                         "flops_per_solve": flops_solve, "kepler_evals_per_solve": kbar,
                         "iteration_lane_efficiency": lane_eff},
            "clocks": clocks.summary(),
            "e2e": {"value": world * n2 * args.steps / el, "unit": UNIT,
                    "h2d_bytes_per_step": int(st.numel() * 8) // args.steps,
                    "d2h_bytes_per_step": int(st.numel() * 8) // args.steps,
                    "note": "state copied in and out once around the K-step call"}}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline_ensemble(ens)
    print(json.dumps(line))
    return 0


def _cpu_baseline_ensemble(ens, budget_s=10.0):
    """The oracle on the host cores over a bounded sample of the ensemble:
    whole systems in order, each for as many of its steps as the budget
    allows (at most 2000), N^2 * steps / s over the sample."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.build()
    t0 = time.perf_counter()
    work = 0
    nsys = 0
    for k in range(ens.nsys):
        s = ens.system(k)
        r, v = s.r.copy(), s.v.copy()
        for _ in range(2000):
            rc, r, v = oracle.step(s.m, r, v, s.dt, 2, nthreads=cores)
            work += s.n * s.n
            if time.perf_counter() - t0 >= budget_s:
                break
        nsys += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": work / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the first {nsys} system(s) of the same ensemble, consecutive steps from"
                      f" their initial states, OpenMP over i on {cores} threads, {el:.1f} s"}


def _pair_kernel_ms(args, sk, s, state, mass, device, stream, flush, guess, opts, per_call=1):
    """Mean duration of the pair kernel per step over a second pass of
    args.steps steps in calls of per_call steps, timed the same way as the
    timed steps (L2 flushed before each call), with CUDA events recorded by
    the library around each pair-kernel launch on its stream (for the
    single-block kernel of small systems: the launch that runs the call)."""
    import torch
    sk.init(device.index, stream=stream.cuda_stream, flags=sk.FLAG_TIMING, guess=guess, **opts)
    sk.get_stats(reset=True)
    torch.cuda.synchronize(device)
    for k in range(args.steps // per_call):
        flush.fill_(float(k))
        if per_call > 1:
            sk.evolve(state, mass, s.dt, 2, per_call)
        else:
            sk.step(state, mass, s.dt, 2)
    torch.cuda.synchronize(device)
    sk.check()
    st = sk.get_stats(reset=True)
    return st["pair_kernel_ms"] / max(1, args.steps)


def _variant_df64(args, sk, s, device, stream, flush, guess, per_call=1, small=False):
    """The same workload and step count in the double-word form (FP64-accurate
    pair solves on the FP32 pipe), timed the same way (calls of per_call
    steps); reported beside the plain FP64 headline."""
    import torch
    n = s.n
    opts = dict(pair_mode=sk.PAIRS_SYMMETRIC, precision=sk.PREC_DF64)
    mass = torch.tensor(s.m, device=device)
    state = torch.tensor(s.soa(), device=device)
    sk.init(device.index, stream=stream.cuda_stream, flags=sk.FLAG_STATS, guess=guess, **opts)
    sk.get_stats(reset=True)
    for _ in range(args.warmup):
        sk.step(state, mass, s.dt, 2)
    sk.check()
    st = sk.get_stats(reset=True)
    spp = st["solves"] / max(1, st["pairs"])
    share = st["fp32_pairs"] / max(1, st["solves"])
    sk.init(device.index, stream=stream.cuda_stream, guess=guess, **opts)
    state.copy_(torch.tensor(s.soa(), device=device))
    E0 = sk.energy(state, mass)
    nt = args.steps // per_call
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(nt)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(nt)]
    torch.cuda.synchronize(device)
    for k in range(nt):
        flush.fill_(float(k))
        starts[k].record(stream)
        if per_call > 1:
            sk.evolve(state, mass, s.dt, 2, per_call)
        else:
            sk.step(state, mass, s.dt, 2)
        ends[k].record(stream)
    torch.cuda.synchronize(device)
    sk.check()
    ms_total = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    dE = abs(sk.energy(state, mass) / E0 - 1.0)
    pair_ms = _pair_kernel_ms(args, sk, s, state, mass, device, stream, flush, guess, opts,
                              per_call)
    flops = DF64_FLOPS_PER_SOLVE.get(args.workload)
    solves = n * (n - 1) * spp
    achieved = solves * flops / (pair_ms * 1e-3) / 1e12 if flops else None
    peak = FP32_PEAK_GFLOPS / 1e3
    return {"value": n * n * args.steps / (ms_total * 1e-3), "unit": UNIT,
            "ms_per_step": ms_total / args.steps,
            "dtype": "f32 double-word (pair solves) + f64 (drift, sums, fallback pairs)",
            "parity": "same 1e-12 per-step bound against the FP64 oracle as the FP64 form",
            "double_word_solve_share": share,
            "energy_error": dE,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak if achieved else None,
                         "traffic": _profiled_traffic(
                             args.workload, "small" if small else "pair_step_sym_df64"),
                         "kernel": "small_kernel" if small else "pair_step_sym_df64_kernel",
                         "pipe": "fp32",
                         "flops_per_solve": flops, "pair_kernel_ms": pair_ms}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plummer1024",
                    choices=["plummer1024", "bh16384", "binaries16384", "planetary9",
                             "ensemble4096"])
    ap.add_argument("--guess", default="fp32",
                    choices=["standard", "taylor", "learned", "fp32"],
                    help="Kepler initial guess: t/r0, the second-order expansion, the"
                         " expansion refined by the trained network, or the root of a"
                         " single-precision solve of the pair (symmetric FP64 step)")
    ap.add_argument("--pairs", default="symmetric", choices=["symmetric", "ordered"],
                    help="symmetric: each unordered pair solved once (Newton's third law);"
                         " ordered: every ordered pair solved")
    ap.add_argument("--form", default="fp64", choices=["fp64", "mixed", "df64"],
                    help="fp64: every pair in FP64; mixed: FP32 solves for the pairs the"
                         " class rule admits, FP64 for the rest and all accumulation;"
                         " df64: every pair to FP64 accuracy in double-word arithmetic on"
                         " the FP32 pipe (symmetric pairs)")
    ap.add_argument("--mixed-rule", default="hyp", choices=["literal", "hyp"],
                    help="literal: FP32 iff r > 0.1 and e < 0.9; hyp: ... or e > 10")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the double-word form reported beside the FP64 headline")
    ap.add_argument("--steps-per-call", type=int, default=None,
                    help="time the steps as calls of sakura_evolve of this many steps"
                         " (default: 100 for planetary9, whose 72 pairs per step run in one"
                         " block for the whole call; 32 for plummer1024, whose steps after the"
                         " first in a call need no drift kernel; 1, i.e. sakura_step, for the"
                         " others)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.steps is None:
        args.steps = _workload(args.workload, 0)[1]
    args.warmup = max(3, args.warmup)

    if args.impl == "reference":
        return run_reference(args, rank)

    import numpy as np
    import torch

    from paper_1402_3325_gb300 import build as sk_build
    from paper_1402_3325_gb300 import ics
    from paper_1402_3325_gb300 import sakura as sk

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local_rank if world > 1 else 0)
    torch.cuda.set_device(device)
    if rank == 0:
        sk_build.build()
    if dist is not None:
        dist.barrier()
    stream = torch.cuda.current_stream(device)
    if args.workload == "ensemble4096":
        return run_ensemble(args, rank, world, device, stream, dist)
    s, _, desc = _workload(args.workload, seed=rank)
    n = s.n
    guess = {"taylor": sk.GUESS_TAYLOR, "standard": sk.GUESS_STANDARD,
             "learned": sk.GUESS_LEARNED, "fp32": sk.GUESS_FP32}[args.guess]
    form_opts = {"pair_mode": sk.PAIRS_SYMMETRIC if args.pairs == "symmetric"
                 else sk.PAIRS_ORDERED}
    if args.form == "df64":
        form_opts.update(precision=sk.PREC_DF64)
    if args.form == "mixed":
        form_opts.update(precision=sk.PREC_MIXED,
                         mixed_rule=sk.MIXED_RULE_HYP if args.mixed_rule == "hyp"
                         else sk.MIXED_RULE_LITERAL)
    sk.init(device.index, stream=stream.cuda_stream, guess=guess, **form_opts)
    if args.guess == "learned":
        from paper_1402_3325_gb300 import learned
        learned.load_default()

    state = torch.tensor(s.soa(), device=device)
    mass = torch.tensor(s.m, device=device)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)

    # warm-up, then the mean Kepler iteration count of this workload
    sk.init(device.index, stream=stream.cuda_stream, flags=sk.FLAG_STATS, guess=guess,
            **form_opts)
    for _ in range(args.warmup):
        sk.step(state, mass, s.dt, 2)
    sk.check()
    st = sk.get_stats(reset=True)
    kbar = st["iters"] / max(1, st["solves"])
    # share of warp iteration slots doing useful work: divergent iteration
    # counts leave lanes idle while the warp's slowest lane finishes
    lane_eff = st["iters"] / max(1, st["warp_slots"])
    st_iters_fp64 = float(st["iters"]) / max(1, args.warmup)
    carried = st.get("carries", 0) / max(1, st["solves"])
    solves_per_pair = st["solves"] / max(1, st["pairs"])
    fp32_share = st["fp32_pairs"] / max(1, st["pairs"])
    if args.steps_per_call is not None:
        per_call = args.steps_per_call
        if per_call < 1 or args.steps % per_call != 0:
            raise SystemExit("--steps must be a multiple of --steps-per-call")
    else:
        # the workload's call length, or the largest divisor of --steps below it
        cap = 100 if args.workload == "planetary9" else (32 if args.workload == "plummer1024"
                                                         else 1)
        per_call = max(d for d in range(1, min(cap, args.steps) + 1) if args.steps % d == 0)
    # the single-block kernel (csrc/step_small.cu) takes the FP64 and
    # double-word forms of small systems, each unordered pair once,
    # non-learned guesses
    small = (n <= sk.SMALL_MAX_N and args.form in ("fp64", "df64") and
             args.pairs == "symmetric" and args.guess != "learned")
    sk.init(device.index, stream=stream.cuda_stream, guess=guess, **form_opts)
    state.copy_(torch.tensor(s.soa(), device=device))
    E0 = sk.energy(state, mass)
    nt = args.steps // per_call
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(nt)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(nt)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(device)
    with ClockSampler(device.index) as clocks:
        for k in range(nt):
            flush.fill_(float(k))
            starts[k].record(stream)
            if per_call > 1:
                sk.evolve(state, mass, s.dt, 2, per_call)
            else:
                sk.step(state, mass, s.dt, 2)
            ends[k].record(stream)
        torch.cuda.synchronize(device)
    if dist is not None:
        dist.barrier()
    sk.check()
    ms_total = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    energy_error = abs(sk.energy(state, mass) / E0 - 1.0)  # outside the timed region
    pair_ms = _pair_kernel_ms(args, sk, s, state, mass, device, stream, flush, guess, form_opts,
                              per_call)
    ms_total = max_over_ranks(ms_total, dist, device)
    ms_step = ms_total / args.steps
    value = whole_job_value(world, n * n * args.steps, ms_total)

    # end to end through the host-buffer entry point, copies in the timed region
    e2e = None
    if not args.no_e2e:
        host_state = torch.empty((6, n), dtype=torch.float64).pin_memory().numpy()
        host_mass = torch.empty((n,), dtype=torch.float64).pin_memory().numpy()
        host_state[...] = s.soa()
        host_mass[...] = s.m
        sk.init(device.index, stream=stream.cuda_stream, guess=guess, **form_opts)
        for _ in range(2):
            sk.evolve_host(host_state, host_mass, s.dt, 2, 1)
        host_state[...] = s.soa()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sk.evolve_host(host_state, host_mass, s.dt, 2, 1)
        el = max_over_ranks(time.perf_counter() - t0, dist, device)
        e2e = {"value": whole_job_value(world, n * n * args.steps, el * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(host_state.nbytes + host_mass.nbytes),
               "d2h_bytes_per_step": int(host_state.nbytes)}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    symmetric = args.pairs == "symmetric" and args.form in ("fp64", "df64")
    solves = n * (n - 1) * solves_per_pair
    if args.form == "df64":
        flops_solve = DF64_FLOPS_PER_SOLVE.get(args.workload)
        peak = FP32_PEAK_GFLOPS / 1e3
        kname, pipe = ("small" if small else "pair_step_sym_df64"), "fp32"
        peak_source = ("152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz; flops per solve counted"
                       " by running the double-word code on the host with an operation tally")
    elif args.form == "mixed" and args.pairs == "symmetric" and fp32_share >= 0.5:
        # FP32 flops of an FP32-class unordered pair (hand count from
        # csrc/kepler_fp32.cuh and csrc/step_mixed.cu, FMA = 2): class test
        # 46, solve setup 12, epilogue with increments and finiteness test 32,
        # per Laguerre iteration 71 (evaluation 37, step 9, stopping test 2,
        # carry of G1..G3 and F' 23), double-word sums of m_j d and -m_i d
        # 168 (12 x (two_prod 3 + renormalised sum 11)); kbar =
        # single-precision iterations per solve.  ncu counts 354 for kbar = 1
        # (profiles/pair_step_sym_mixed_bh16384.md): the correctly rounded
        # divisions and square root of the class test take more than counted.
        flops_solve = fp32_share * (C_MIX32_FIX + kbar * C_MIX32_ITER)
        peak = FP32_PEAK_GFLOPS / 1e3
        kname, pipe = "pair_step_sym_mixed", "fp32"
        peak_source = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz; flops counted by hand"
    elif args.form == "mixed" and args.pairs == "symmetric":
        # mostly FP64-class pairs (through the FP64 queue): their FP64 solves
        flops_solve = (1.0 - fp32_share) * (C_FIX + kbar * C_EVAL + (kbar - 1.0) * C_STEP +
                                            C_SYM)
        peak = FP64_PEAK_GFLOPS / 1e3
        kname, pipe = "pair_step_sym_mixed", "fp64"
        peak_source = "152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"
    elif args.form == "mixed":
        # FP64 flops per ordered pair: the FP64 accumulation (6 FMA) of an
        # FP32-class pair, the full FP64 solve of the others (the FP32 solves
        # run on the FP32 pipe and are not counted here)
        k64 = st_iters_fp64 / max(1.0, solves_per_pair * n * (n - 1) * (1.0 - fp32_share))
        flops_solve = (fp32_share * 12.0 + (1.0 - fp32_share) *
                       (C_FIX + k64 * C_EVAL + max(0.0, k64 - 1.0) * C_STEP))
        peak = FP64_PEAK_GFLOPS / 1e3
        kname, pipe = "pair_step_mixed", "fp64 (FP32-class pairs: accumulation only)"
        peak_source = ("152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz; flops per pair counted"
                       " for the FP64 work only")
    else:
        flops_solve = (C_FIX + kbar * C_EVAL + (kbar - 1.0) * C_STEP +
                       carried * (C_STEP + C_CARRY) + (C_SYM if symmetric else 0) -
                       (C_SEED_SAVED if (args.guess == "fp32" and symmetric) else 0))
        peak = FP64_PEAK_GFLOPS / 1e3
        kname = "small" if small else ("pair_step_sym" if symmetric else (
            "pair_step_mixed" if args.form == "mixed" else "pair_step_fp64"))
        pipe = "fp64"
        peak_source = ("152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (derived from the nominal"
                       " 1.25 TFLOP/s; FMA probe measured 1.19)")
    achieved = (solves * flops_solve / (pair_ms * 1e-3) / 1e12) if flops_solve else None
    traffic = _profiled_traffic(args.workload, kname)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None, "traffic": traffic,
            "kernel": kname + "_kernel", "pipe": pipe, "peak_source": peak_source,
            "flops_per_solve": flops_solve, "kepler_evals_per_solve": kbar,
            "carried_share": carried,
            "iteration_lane_efficiency": lane_eff,
            "solves_per_step": solves,
            "pair_kernel_ms": pair_ms, "pair_kernel_share": pair_ms / ms_step,
            "pair_kernel_timing": ("CUDA events around each pair-kernel launch on the library"
                                   " stream, in a second pass of the same K steps with L2"
                                   " flushed before each step")}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32 double-word (pair solves) + f64 (drift, sums, fallback pairs)"
                      if args.form == "df64" else "f64"),
            "data": "synthetic",
            "config": {"workload": desc, "n": n, "dt": s.dt, "order": 2, "form": args.form,
                       "pairs": args.pairs,
                       "kepler_guess": args.guess,
                       "fp32_pair_share": fp32_share,
                       "pairs_solved_per_step": n * (n - 1),
                       "energy_error_over_timed_steps": energy_error,
                       "l2": ("256 MB buffer written between timed calls (state fits in L2)"
                              if per_call > 1 else
                              "256 MB buffer written between timed steps (state fits in L2)"),
                       "steps_per_call": per_call,
                       "timing": (f"{nt} calls of sakura_evolve of {per_call} steps, each"
                                  " timed with CUDA events" if per_call > 1 else
                                  "each sakura_step call timed with CUDA events"),
                       "kernels": ("single-block kernel for small systems, every step of a"
                                   " call in one launch" if small else
                                   "drift, pair and apply kernels per step"),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            # small systems: one launch per call; symmetric FP64 tiles: a
            # prep kernel per call, then a pair and an apply kernel per step
            # (each apply drifts for the next); otherwise prep, pair, apply
            "gpu_launches": (nt if small else
                             nt * (1 + 2 * per_call) if (args.form == "fp64" and
                                                         args.pairs == "symmetric")
                             else 3 * args.steps),
            "solves_per_pair": solves_per_pair,
            "roofline": roof, "clocks": clocks.summary()}
    if e2e is not None:
        line["e2e"] = e2e
    if (args.form == "fp64" and args.pairs == "symmetric" and not args.no_variants and
            args.workload in DF64_FLOPS_PER_SOLVE):
        line["variants"] = {"df64": _variant_df64(args, sk, s, device, stream, flush, guess,
                                                  per_call, n <= sk.SMALL_MAX_N)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(s, s.dt,
                                             max_steps=min(256, _workload(args.workload, 0)[1]))
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
