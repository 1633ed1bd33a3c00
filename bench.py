"""Benchmark of the Sakura all-pairs Kepler step on GB300.

Metric: pair-Kepler solves per second, counted as N^2 * steps / s (the
literal N^2 count; the kernel solves each of the N(N-1)/2 unordered pairs
once and applies it to both particles).

Default workload: black hole of mass 1 plus 16383 stars of total mass 1e-2
(Plummer scale 1, circular velocities), dt = 2^-10, second-order map, the
plain FP64 form (each unordered pair solved once on systolic 32 x 32 tiles,
single-precision seed, FP64 Kepler iteration and sums).  A step is the pair
kernel and the apply kernel (Eqs. 27b-d), which also drifts for the next
step (Eq. 27a); a call's first step has a prep kernel for its drift.  The
steps are timed as calls of ``sakura_evolve`` (up to 32 steps per call),
each call timed with CUDA events on the library stream, with a 256 MB buffer
written before every call to flush L2.  The pair kernel's own duration (the
roofline's denominator) comes from a second pass of the same calls with
CUDA events around each pair-kernel launch, so that those events, which
hold each launch until the previous kernel has finished, do not add to the
timed steps.

Beside the headline the JSON line carries ``variants``: the same workload
and step count in the other forms the metric compares with the plain FP64
one, each with its own roofline: the mixed form under the literal class rule
(FP32 iff r > 0.1 and e < 0.9) and under the hyperbolic reading (... or
e > 10), the learned initial guess, the standard guess t/r0 (the method
without a seed or a network), and the double-word form.  Each reports its
energy error over the timed steps, next to the FP64 form's.

Printed JSON line (rank 0): value (device-resident throughput of the plain
FP64 form), e2e (the same through the host-buffer entry point
``sakura_evolve_host``, one step per call, copies included), roofline of the
pair kernel against the FP64 ALU peak, variants, cpu_baseline (the CPU
oracle on the host cores over a bounded sample), clocks sampled during the
timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload bh16384|binaries16384|plummer1024|planetary9|ensemble4096]
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
import re
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
# evaluations.  ncu cross-check on the ordered kernel (Plummer N = 1024):
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
# FP64 multiplies per solve that the FP64 kernels form on the integer pipes
# instead (csrc/fp64_emu.cuh; the same IEEE results, counted in the flops
# above all the same), per kernel and guess (the EMU sets of step_grp.cu,
# step_sym.cu and step_batched.cu): the increments' 10, the setup's 6, the
# carry's 4 and the 10 of each Laguerre evaluation
EMU_INC_MULS = 10
EMU_SETUP_MULS = 6
EMU_CARRY_MULS = 4
EMU_ITER_MULS = 10


def _integer_pipe_flops(kernel, guess, kbar, mixed=False):
    if kernel not in ("pair_step_grp", "pair_step_sym", "batched"):
        return 0
    if mixed:  # the inline class test: row groups only
        return (EMU_INC_MULS + EMU_SETUP_MULS + EMU_CARRY_MULS) if kernel == "pair_step_grp" else 0
    if guess == "fp32":
        return EMU_INC_MULS + EMU_SETUP_MULS + kbar * EMU_ITER_MULS
    if guess in ("standard", "taylor"):
        return EMU_INC_MULS + kbar * EMU_ITER_MULS
    return EMU_INC_MULS if kernel == "pair_step_grp" else 0


# FP32-class pair of the symmetric mixed form (see the roofline code below)
C_MIX32_FIX = 44 + 44 + 168
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


# the source file of each profiled kernel
KERNEL_SOURCES = {"pair_step_sym": "step_sym.cu", "pair_step_grp": "step_grp.cu",
                  "pair_step_fp64": "step_fp64.cu", "pair_step_sym_df64": "step_df64.cu",
                  "pair_step_grp_df64": "step_df64.cu",
                  "pair_step_grp_mixed": "step_mixed.cu", "pair_step_mixed": "step_mixed.cu",
                  "small": "step_small.cu", "batched": "step_batched.cu"}


def _kernel_sources_hash(kernel: str = "pair_step_sym") -> str:
    """SHA-256 (first 16 hex digits) of the kernel's source file and of every
    header it includes from csrc/, directly or through other headers."""
    csrc = os.path.join(ROOT, "paper_1402_3325_gb300", "csrc")
    seen, todo = set(), [KERNEL_SOURCES.get(kernel, "step_fp64.cu")]
    while todo:
        f = todo.pop()
        if f in seen:
            continue
        seen.add(f)
        with open(os.path.join(csrc, f)) as fh:
            for inc in re.findall(r'#include\s+"([^"]+)"', fh.read()):
                if os.path.exists(os.path.join(csrc, inc)):
                    todo.append(inc)
    h = hashlib.sha256()
    for f in sorted(seen):
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(workload: str, kernel: str):
    """DRAM bytes per pair-kernel launch from the committed ncu summary of
    this kernel on this workload, or None when there is none or the kernel's
    sources changed since it was taken."""
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
    out = {"value": s.n ** 2 * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{what} of the same workload (N={s.n}) from its initial state,"
                     f" OpenMP over i on {cores} threads, {el:.1f} s"}
    # the same oracle on one core: rows of the first step (each summing over
    # all n columns), about a second of work
    import numpy as np
    rows = max(1, min(s.n, int(4e6 // s.n)))
    t1 = time.perf_counter()
    oracle.step_sample(s.m, s.r, s.v, dt, np.arange(rows), 2, nthreads=1)
    el1 = time.perf_counter() - t1
    out["one_core"] = {"value": rows * s.n / el1, "unit": UNIT,
                       "sample": f"{rows} rows of the first step (oracle.step_sample),"
                                 f" {rows * s.n} ordered pairs, 1 thread, {el1:.2f} s"}
    return out


# the reference arm's steps on large workloads: this many rows of the
# step (oracle.step_sample, each row summing over all n columns), so that a
# run of --steps K --warmup W takes seconds per step on the host cores
REFERENCE_ROWS = 2048


def run_reference(args, rank):
    """The reference arm: the CPU oracle as it stands on the host cores.
    Workloads of up to REFERENCE_ROWS particles run whole oracle steps;
    larger ones run, per step, REFERENCE_ROWS consecutive rows of the step
    (the rows rotate from step to step, all from the initial state), whose
    REFERENCE_ROWS * n ordered pairs are the step's work in the metric's
    count."""
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    oracle.build()
    s, _, desc = _workload(args.workload, 0)
    cores = os.cpu_count() or 1
    sampled = s.n > REFERENCE_ROWS
    r, v = s.r.copy(), s.v.copy()

    def one(k):
        nonlocal r, v
        if sampled:
            rows = (np.arange(REFERENCE_ROWS) + k * REFERENCE_ROWS) % s.n
            oracle.step_sample(s.m, s.r, s.v, s.dt, rows, 2, nthreads=cores)
        else:
            _, r, v = oracle.step(s.m, r, v, s.dt, 2, nthreads=cores)

    for k in range(args.warmup):
        one(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        one(args.warmup + k)
    el = time.perf_counter() - t0
    work = (REFERENCE_ROWS * s.n if sampled else s.n ** 2) * args.steps
    value = work / el
    sample = (f"{args.steps} timed steps after {args.warmup} warm-up steps, each"
              f" {REFERENCE_ROWS} of the {s.n} rows of the step (oracle.step_sample;"
              f" {REFERENCE_ROWS} x {s.n} ordered pairs), OpenMP over rows on {cores} threads"
              if sampled else
              f"{args.steps} timed steps after {args.warmup} warm-up steps, full N={s.n},"
              f" OpenMP over i on {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "n": s.n, "dt": s.dt, "order": 2},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _batched_flops(kbar, carried, guess):
    """FP64 flops per solve of the batched kernel (the symmetric FP64 count)."""
    return (C_FIX + kbar * C_EVAL + (kbar - 1.0) * C_STEP + carried * (C_STEP + C_CARRY) +
            C_SYM - (C_SEED_SAVED if guess == "fp32" else 0))


def _measure_batched(args, sk, ens, device, stream, guess, clocks=None, dist=None):
    """sakura_step_batched over the ensemble: args.warmup steps with
    statistics (and the schedule and autotuner), then one call of
    args.steps steps timed with CUDA events on the stream."""
    import torch
    st0 = torch.tensor(ens.state, device=device)
    st = st0.clone()
    m = torch.tensor(ens.m, device=device)
    off = torch.tensor(ens.offsets, device=device)
    dt = torch.tensor(ens.dt, device=device)
    gcode = _guess_code(sk, guess)
    sk.init(device.index, stream=stream.cuda_stream, guess=gcode, flags=sk.FLAG_STATS)
    sk.get_stats(reset=True)  # counters of earlier calls
    sk.step_batched(st, m, off, ens.offsets, dt, 2, args.warmup)   # schedule, autotune
    sk.check()
    stt = sk.get_stats(reset=True)
    out = {"kepler_evals_per_solve": stt["iters"] / max(1, stt["solves"]),
           "carried_share": stt.get("carries", 0) / max(1, stt["solves"]),
           "iteration_lane_efficiency": stt["iters"] / max(1, stt["warp_slots"])}
    out["tuning"] = sk.batched_tuning()
    sk.init(device.index, stream=stream.cuda_stream, guess=gcode)
    st.copy_(st0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(device)
    if clocks is not None:
        clocks.__enter__()
    try:
        e0.record(stream)
        sk.step_batched(st, m, off, ens.offsets, dt, 2, args.steps)
        e1.record(stream)
        torch.cuda.synchronize(device)
    finally:
        if clocks is not None:
            clocks.__exit__(None, None, None)
    sk.check()
    out["ms"] = e0.elapsed_time(e1)
    out["bufs"] = (st, m, off, dt)
    return out


def _per_system_launches(args, sk, ens, device, stream, steps):
    """The same systems without batching: one sakura_evolve call of `steps`
    steps per system, one after another on the library stream (systems of
    up to 20 particles in one launch of the single-block kernel, larger ones
    as drift, pair and apply kernels per step), timed with CUDA events
    around the whole sequence."""
    import torch
    sk.init(device.index, stream=stream.cuda_stream, guess=sk.GUESS_FP32)
    states, masses = [], []
    for k in range(ens.nsys):
        sysk = ens.system(k)
        states.append(torch.tensor(sysk.soa(), device=device))
        masses.append(torch.tensor(sysk.m, device=device))
    for k in range(ens.nsys):  # warm-up: one step each (sizes the scratch)
        sk.evolve(states[k], masses[k], float(ens.dt[k]), 2, 1)
    sk.check()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    e0.record(stream)
    for k in range(ens.nsys):
        sk.evolve(states[k], masses[k], float(ens.dt[k]), 2, steps)
    e1.record(stream)
    torch.cuda.synchronize(device)
    sk.check()
    return e0.elapsed_time(e1)


def run_ensemble(args, rank, world, device, stream, dist):
    """The batched ensemble: one sakura_step_batched call runs all K steps
    (state kept in shared memory), timed with CUDA events on the stream.
    Variants: the same call with the learned initial guess, and the same
    systems as one sakura_evolve call per system (a bounded number of steps
    each)."""
    import torch

    from paper_1402_3325_gb300 import sakura as sk
    ens, _, desc = _workload(args.workload, seed=rank)
    sizes = ens.offsets[1:] - ens.offsets[:-1]
    n2 = int((sizes * sizes).sum())
    # every unordered pair is solved once and applied to both particles
    solves = int((sizes * (sizes - 1)).sum()) // 2
    sk.init(device.index, stream=stream.cuda_stream)
    from paper_1402_3325_gb300 import learned
    learned.load_default()
    clocks = ClockSampler(device.index)
    h = _measure_batched(args, sk, ens, device, stream, args.guess, clocks, dist)
    ms = max_over_ranks(h["ms"], dist, device)
    value = whole_job_value(world, n2 * args.steps, ms)
    # end to end: host buffers copied in and out around the same call
    st, m, off, dt = h["bufs"]
    host = torch.empty(tuple(st.shape), dtype=torch.float64).pin_memory()
    host.copy_(torch.tensor(ens.state))
    t0 = time.perf_counter()
    st.copy_(host, non_blocking=True)
    sk.step_batched(st, m, off, ens.offsets, dt, 2, args.steps)
    host.copy_(st, non_blocking=True)
    torch.cuda.synchronize(device)
    el = time.perf_counter() - t0
    variants = None
    if not args.no_variants:
        hl = _measure_batched(args, sk, ens, device, stream, "learned")
        fl = _batched_flops(hl["kepler_evals_per_solve"], hl["carried_share"], "learned")
        ach = solves * args.steps * fl / (hl["ms"] * 1e-3) / 1e12
        variants = {"batched_learned_guess": {
            "value": n2 * args.steps / (hl["ms"] * 1e-3), "unit": UNIT,
            "ms_per_step": hl["ms"] / args.steps, "kepler_guess": "learned",
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_GFLOPS / 1e3,
                         "unit": "TFLOP/s", "frac": ach / (FP64_PEAK_GFLOPS / 1e3),
                         "traffic": None, "kernel": "batched_kernel (learned guess)",
                         "pipe": "fp64", "flops_per_solve": fl,
                         "integer_pipe_flops_per_solve": _integer_pipe_flops(
                             "batched", "learned", hl["kepler_evals_per_solve"]),
                         "kepler_evals_per_solve": hl["kepler_evals_per_solve"],
                         "iteration_lane_efficiency": hl["iteration_lane_efficiency"]}}}
        ps_steps = min(args.steps, 10)
        ms_ps = _per_system_launches(args, sk, ens, device, stream, ps_steps)
        v_ps = n2 * ps_steps / (ms_ps * 1e-3)
        variants["per_system_launches"] = {
            "value": v_ps, "unit": UNIT, "ms_per_step": ms_ps / ps_steps,
            "steps": ps_steps,
            "note": (f"one sakura_evolve call of {ps_steps} steps per system, {ens.nsys}"
                     " calls in sequence on one stream (systems of up to 20 particles in"
                     " one single-block launch, larger ones three kernels per step),"
                     " FP32 seed"),
            "batched_over_per_system": value / world / v_ps}
    if rank != 0:
        return 0
    kbar, carried = h["kepler_evals_per_solve"], h["carried_share"]
    flops_solve = _batched_flops(kbar, carried, args.guess)
    achieved = solves * args.steps * flops_solve / (ms * 1e-3) / 1e12
    peak = FP64_PEAK_GFLOPS / 1e3
    warps, blocks, tune = h["tuning"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "nsys": ens.nsys, "particles": int(ens.offsets[-1]),
                       "pairs_counted_per_step": n2, "kepler_solves_per_step": solves,
                       "order": 2, "form": "batched",
                       "kepler_guess": args.guess,
                       "block_warps": warps, "blocks": blocks, "autotune_ms": tune,
                       "l2": "state (7.7 MB) stays in shared memory for the whole call"},
            "gpu_launches": 1,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         # a launch reads the state once, whatever its step count
                         "traffic": _profiled_traffic(args.workload, "batched"),
                         "kernel": "batched_kernel", "pipe": "fp64",
                         "flops_per_solve": flops_solve,
                         "integer_pipe_flops_per_solve": _integer_pipe_flops("batched", args.guess,
                                                                             kbar),
                         "kepler_evals_per_solve": kbar,
                         "iteration_lane_efficiency": h["iteration_lane_efficiency"]},
            "clocks": clocks.summary(),
            "e2e": {"value": world * n2 * args.steps / el, "unit": UNIT,
                    "h2d_bytes_per_step": int(st.numel() * 8) // args.steps,
                    "d2h_bytes_per_step": int(st.numel() * 8) // args.steps,
                    "note": "state copied in and out once around the K-step call"}}
    if variants is not None:
        line["variants"] = variants
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
    sk.init(device.index, stream=stream.cuda_stream, flags=sk.FLAG_TIMING | EXTRA_FLAGS,
            guess=guess, **opts)
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


GUESSES = ("standard", "taylor", "learned", "fp32")


def _guess_code(sk, name):
    return {"taylor": sk.GUESS_TAYLOR, "standard": sk.GUESS_STANDARD,
            "learned": sk.GUESS_LEARNED, "fp32": sk.GUESS_FP32}[name]


KERNEL_FLAG = {"auto": 0, "tiles": 32, "groups": 64}  # SAKURA_FLAG_TILES / _GROUPS
EXTRA_FLAGS = 0  # library flags of --kernel, added to every measured configuration


def _form_options(sk, form, pairs, mixed_rule):
    opts = {"pair_mode": sk.PAIRS_SYMMETRIC if pairs == "symmetric" else sk.PAIRS_ORDERED}
    if form == "df64":
        opts.update(precision=sk.PREC_DF64)
    if form == "mixed":
        opts.update(precision=sk.PREC_MIXED,
                    mixed_rule=sk.MIXED_RULE_HYP if mixed_rule == "hyp"
                    else sk.MIXED_RULE_LITERAL)
    return opts


def _roofline(workload, form, pairs, guess, n, small, m):
    """Roofline of the pair kernel of one measured form: algorithmic flops
    per Kepler solve (hand counts above, with the measured evaluation and
    carry shares) times the solves per step, over the pair kernel's mean
    duration, against the pipe that bounds it."""
    kbar, carried, share = m["kepler_evals_per_solve"], m["carried_share"], m["fp32_pair_share"]
    symmetric = pairs == "symmetric" and form in ("fp64", "df64")
    fp64_peak_src = ("152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (derived from the nominal"
                     " 1.25 TFLOP/s; an FP64 FMA probe on this GPU sustains 1.06 TFLOP/s)")
    fp32_peak_src = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
    if form == "df64":
        flops = DF64_FLOPS_PER_SOLVE.get(workload)
        peak, pipe, src = FP32_PEAK_GFLOPS / 1e3, "fp32", fp32_peak_src + (
            "; flops per solve counted by running the double-word code on the host with an"
            " operation tally")
        kname = "small" if small else (
            "pair_step_grp_df64" if m["row_groups"] else "pair_step_sym_df64")
    elif form == "mixed" and pairs == "symmetric" and share >= 0.5:
        # FP32 flops of an FP32-class unordered pair (hand count from
        # csrc/kepler_fp32.cuh and csrc/step_mixed.cu, FMA = 2): class test
        # 44, solve setup 12, epilogue with increments and finiteness test
        # 32, per Laguerre iteration 71 (evaluation 37, step 9, stopping
        # test 2, carry of G1..G3 and F' 23), double-word sums of m_j d and
        # -m_i d 168 (12 x (two_prod 3 + renormalised sum 11)); kbar =
        # single-precision iterations per solve
        flops = share * (C_MIX32_FIX + kbar * C_MIX32_ITER)
        peak, pipe, src = FP32_PEAK_GFLOPS / 1e3, "fp32", fp32_peak_src + "; flops counted by hand"
        kname = "pair_step_grp_mixed" if m["row_groups"] else "pair_step_sym"
    elif form == "mixed" and pairs == "symmetric":
        # mostly FP64-class pairs (the literal rule: the FP64 tile kernel with
        # an inline class test): their FP64 solves, counted as in the
        # symmetric FP64 kernel (single-precision seed and Taylor carry with
        # guess fp32)
        flops = (1.0 - share) * (C_FIX + kbar * C_EVAL + (kbar - 1.0) * C_STEP +
                                 carried * (C_STEP + C_CARRY) + C_SYM -
                                 (C_SEED_SAVED if guess == "fp32" else 0))
        peak, pipe, src = FP64_PEAK_GFLOPS / 1e3, "fp64", fp64_peak_src
        # the FP64 kernels with the inline class test (literal rule): in row
        # groups or on tiles
        kname = "pair_step_grp" if m["row_groups"] else "pair_step_sym"
    elif form == "mixed":
        # FP64 flops per ordered pair: the FP64 accumulation (6 FMA) of an
        # FP32-class pair, the full FP64 solve of the others
        k64 = m["fp64_evals_per_fp64_pair"]
        flops = (share * 12.0 + (1.0 - share) *
                 (C_FIX + k64 * C_EVAL + max(0.0, k64 - 1.0) * C_STEP))
        peak, pipe, src = FP64_PEAK_GFLOPS / 1e3, "fp64 (FP32-class pairs: accumulation only)", (
            fp64_peak_src + "; flops per pair counted for the FP64 work only")
        kname = "pair_step_mixed"
    else:
        flops = (C_FIX + kbar * C_EVAL + (kbar - 1.0) * C_STEP + carried * (C_STEP + C_CARRY) +
                 (C_SYM if symmetric else 0) -
                 (C_SEED_SAVED if (guess == "fp32" and symmetric) else 0))
        peak, pipe, src = FP64_PEAK_GFLOPS / 1e3, "fp64", fp64_peak_src
        kname = "small" if small else (
            ("pair_step_grp" if m["row_groups"] else "pair_step_sym")
            if symmetric else "pair_step_fp64")
    solves = n * (n - 1) * m["solves_per_pair"]
    pair_ms = m["pair_kernel_ms"]
    achieved = solves * flops / (pair_ms * 1e-3) / 1e12 if flops and pair_ms > 0 else None
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None,
            "traffic": _profiled_traffic(workload, kname),
            "kernel": kname + "_kernel", "pipe": pipe, "peak_source": src,
            "flops_per_solve": flops,
            "integer_pipe_flops_per_solve": (
                (1.0 - share if form == "mixed" else 1.0) *
                _integer_pipe_flops(kname, guess, kbar, mixed=form == "mixed")
                if form in ("fp64", "mixed") and pipe.startswith("fp64") and not small else 0.0),
            "kepler_evals_per_solve": kbar,
            "carried_share": carried, "iteration_lane_efficiency": m["iteration_lane_efficiency"],
            "solves_per_step": solves, "pair_kernel_ms": pair_ms,
            "pair_kernel_share": pair_ms / m["ms_per_step"],
            "pair_kernel_timing": ("CUDA events around each pair-kernel launch on the library"
                                   " stream, in a second pass of the same K steps with L2"
                                   " flushed before each call")}


def _measure(args, sk, s, device, stream, flush, guess, opts, per_call, clocks=None,
             dist=None):
    """One form on one workload: args.warmup steps with statistics (Kepler
    evaluations, carries, FP32 share), then args.steps steps in calls of
    per_call steps, each call timed with CUDA events on the library stream
    after an L2 flush, then the pair kernel's own duration from a second
    pass.  The energy error is taken over the timed steps."""
    import torch
    n = s.n
    mass = torch.tensor(s.m, device=device)
    state0 = torch.tensor(s.soa(), device=device)
    state = state0.clone()
    gcode = _guess_code(sk, guess)
    sk.init(device.index, stream=stream.cuda_stream, flags=sk.FLAG_STATS | EXTRA_FLAGS,
            guess=gcode, **opts)
    sk.get_stats(reset=True)  # counters of earlier calls
    for _ in range(args.warmup):
        sk.step(state, mass, s.dt, 2)
    sk.check()
    st = sk.get_stats(reset=True)
    m = {"kepler_evals_per_solve": st["iters"] / max(1, st["solves"]),
         # share of warp iteration slots doing useful work: divergent
         # iteration counts leave lanes idle while the slowest lane finishes
         "iteration_lane_efficiency": st["iters"] / max(1, st["warp_slots"]),
         "carried_share": st.get("carries", 0) / max(1, st["solves"]),
         "solves_per_pair": st["solves"] / max(1, st["pairs"]),
         "fp32_pair_share": st["fp32_pairs"] / max(1, st["pairs"]),
         # the pair kernel the library chose: the row-group layout or not
         "row_groups": st.get("group_launches", 0) > 0}
    m["fp64_evals_per_fp64_pair"] = (float(st["iters"]) / max(
        1.0, st["solves"] * (1.0 - m["fp32_pair_share"])))
    sk.init(device.index, stream=stream.cuda_stream, flags=EXTRA_FLAGS, guess=gcode, **opts)
    state.copy_(state0)
    E0 = sk.energy(state, mass)
    nt = args.steps // per_call
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(nt)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(nt)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(device)
    if clocks is not None:
        clocks.__enter__()
    try:
        for k in range(nt):
            flush.fill_(float(k))
            starts[k].record(stream)
            if per_call > 1:
                sk.evolve(state, mass, s.dt, 2, per_call)
            else:
                sk.step(state, mass, s.dt, 2)
            ends[k].record(stream)
        torch.cuda.synchronize(device)
    finally:
        if clocks is not None:
            clocks.__exit__(None, None, None)
    if dist is not None:
        dist.barrier()
    sk.check()
    ms_total = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    m["energy_error"] = abs(sk.energy(state, mass) / E0 - 1.0)  # outside the timed region
    m["pair_kernel_ms"] = _pair_kernel_ms(args, sk, s, state, mass, device, stream, flush,
                                          gcode, opts, per_call)
    m["ms_total"] = ms_total
    m["ms_per_step"] = ms_total / args.steps
    m["value"] = n * n * args.steps / (ms_total * 1e-3)
    return m


def _variant(args, sk, s, device, stream, flush, per_call, small, form, pairs, guess,
             mixed_rule="literal", note=""):
    """A form other than the headline, on the same workload and step count,
    timed the same way; its roofline is its own pair kernel's."""
    opts = _form_options(sk, form, pairs, mixed_rule)
    small = small and form in ("fp64", "df64") and pairs == "symmetric" and guess != "learned"
    m = _measure(args, sk, s, device, stream, flush, guess, opts, per_call)
    out = {"value": m["value"], "unit": UNIT, "ms_per_step": m["ms_per_step"],
           "form": form, "pairs": pairs, "kepler_guess": guess,
           "dtype": {"fp64": "f64", "mixed": "f32 (FP32-class pair solves) + f64 (other pairs,"
                     " accumulation)", "df64": "f32 double-word (pair solves) + f64 (drift,"
                     " sums, fallback pairs)"}[form],
           "energy_error_over_timed_steps": m["energy_error"],
           "fp32_pair_share": m["fp32_pair_share"],
           "roofline": _roofline(args.workload, form, pairs, guess, s.n, small, m)}
    if form == "mixed":
        out["class_rule"] = ("FP32 iff r > 0.1 and e < 0.9" if mixed_rule == "literal" else
                             "FP32 iff r > 0.1 and (e < 0.9 or e > 10)")
    if note:
        out["note"] = note
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bh16384",
                    choices=["bh16384", "binaries16384", "plummer1024", "planetary9",
                             "ensemble4096"])
    ap.add_argument("--guess", default="fp32", choices=list(GUESSES),
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
    ap.add_argument("--kernel", default="auto", choices=["auto", "tiles", "groups"],
                    help="symmetric FP64 and mixed forms: the library's choice, or force the"
                         " systolic-tile or the row-group kernel")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the other forms reported beside the FP64 headline")
    ap.add_argument("--steps-per-call", type=int, default=None,
                    help="time the steps as calls of sakura_evolve of this many steps"
                         " (default: the largest divisor of --steps up to 100 for planetary9,"
                         " whose steps run in one block for the whole call, and up to 32"
                         " otherwise; in the FP64 form the steps after a call's first need"
                         " no drift kernel)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.steps is None:
        args.steps = _workload(args.workload, 0)[1]
    args.warmup = max(3, args.warmup)
    global EXTRA_FLAGS
    EXTRA_FLAGS = KERNEL_FLAG[args.kernel]

    if args.impl == "reference":
        return run_reference(args, rank)

    import torch

    from paper_1402_3325_gb300 import build as sk_build
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
    sk.init(device.index, stream=stream.cuda_stream)
    if args.guess == "learned" or not args.no_variants:
        from paper_1402_3325_gb300 import learned
        learned.load_default()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    if args.steps_per_call is not None:
        per_call = args.steps_per_call
        if per_call < 1 or args.steps % per_call != 0:
            raise SystemExit("--steps must be a multiple of --steps-per-call")
    else:
        cap = 100 if args.workload == "planetary9" else 32
        per_call = max(d for d in range(1, min(cap, args.steps) + 1) if args.steps % d == 0)
    # the single-block kernel (csrc/step_small.cu) takes the FP64 and
    # double-word forms of small systems, each unordered pair once,
    # non-learned guesses
    small = (n <= sk.SMALL_MAX_N and args.form in ("fp64", "df64") and
             args.pairs == "symmetric" and args.guess != "learned")
    opts = _form_options(sk, args.form, args.pairs, args.mixed_rule)
    clocks = ClockSampler(device.index)
    m = _measure(args, sk, s, device, stream, flush, args.guess, opts, per_call, clocks, dist)
    ms_total = max_over_ranks(m["ms_total"], dist, device)
    ms_step = ms_total / args.steps
    value = whole_job_value(world, n * n * args.steps, ms_total)

    # end to end through the host-buffer entry point, copies in the timed
    # region, one call (one step) at a time
    e2e = None
    if not args.no_e2e:
        host_state = torch.empty((6, n), dtype=torch.float64).pin_memory().numpy()
        host_mass = torch.empty((n,), dtype=torch.float64).pin_memory().numpy()
        host_state[...] = s.soa()
        host_mass[...] = s.m
        sk.init(device.index, stream=stream.cuda_stream, flags=EXTRA_FLAGS,
                guess=_guess_code(sk, args.guess), **opts)
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
               "d2h_bytes_per_step": int(host_state.nbytes),
               "timing": "one sakura_evolve_host call per step on page-locked host buffers,"
                         " wall clock"}

    variants = None
    if (not args.no_variants and args.form == "fp64" and args.pairs == "symmetric" and
            args.guess == "fp32" and n > sk.SMALL_MAX_N):
        V = lambda *a, **k: _variant(args, sk, s, device, stream, flush, per_call, small,  # noqa
                                     *a, **k)
        variants = {
            "mixed_literal": V("mixed", "symmetric", "fp32", "literal",
                               "the class rule as stated for this workload"),
            "mixed_hyp": V("mixed", "symmetric", "fp32", "hyp",
                           "the class rule with strong hyperbolae (e > 10) also in FP32"),
            "fp64_learned_guess": V("fp64", "symmetric", "learned",
                                    note="FP64 form, second-order guess refined by the"
                                         " trained network (BF16 mma.sync in the pair kernel)"),
            "fp64_standard_guess": V("fp64", "symmetric", "standard",
                                     note="FP64 form, standard guess t/r0: the method without"
                                          " a seed or a network"),
            "df64": V("df64", "symmetric", "fp32",
                      note="every pair to FP64 accuracy in double-word arithmetic on the FP32"
                           " pipe; same 1e-12 per-step parity bound as the FP64 form"),
        }
    elif (not args.no_variants and args.form == "fp64" and args.pairs == "symmetric" and
          args.workload in DF64_FLOPS_PER_SOLVE):
        variants = {"df64": _variant(args, sk, s, device, stream, flush, per_call, small,
                                     "df64", "symmetric", args.guess)}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    symmetric = args.pairs == "symmetric" and args.form in ("fp64", "df64")
    roof = _roofline(args.workload, args.form, args.pairs, args.guess, n, small, m)
    solves = n * (n - 1) * m["solves_per_pair"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32 double-word (pair solves) + f64 (drift, sums, fallback pairs)"
                      if args.form == "df64" else
                      "f32 (FP32-class pair solves) + f64 (other pairs, accumulation)"
                      if args.form == "mixed" else "f64"),
            "data": "synthetic",
            "config": {"workload": desc, "n": n, "dt": s.dt, "order": 2, "form": args.form,
                       "pairs": args.pairs, "kernel_choice": args.kernel,
                       "kepler_guess": args.guess,
                       "fp32_pair_share": m["fp32_pair_share"],
                       "pairs_counted_per_step": n * n,
                       "kepler_solves_per_step": solves,
                       "energy_error_over_timed_steps": m["energy_error"],
                       "l2": "256 MB buffer written before every timed call",
                       "steps_per_call": per_call,
                       "timing": (f"{args.steps // per_call} calls of sakura_evolve of"
                                  f" {per_call} steps, each timed with CUDA events"
                                  if per_call > 1 else
                                  "each sakura_step call timed with CUDA events"),
                       "kernels": ("single-block kernel for small systems, every step of a"
                                   " call in one launch" if small else
                                   "drift, pair and apply kernels per step"),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            # small systems: one launch per call; symmetric FP64 tiles: a
            # prep kernel per call, then a pair and an apply kernel per step
            # (each apply drifts for the next); otherwise prep, pair, apply
            "gpu_launches": ((args.steps // per_call) if small else
                             (args.steps // per_call) * (1 + 2 * per_call)
                             if (args.form == "fp64" and symmetric) else 3 * args.steps),
            "solves_per_pair": m["solves_per_pair"],
            "roofline": roof, "clocks": clocks.summary()}
    if e2e is not None:
        line["e2e"] = e2e
    if variants is not None:
        line["variants"] = variants
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(s, s.dt,
                                             max_steps=min(256, _workload(args.workload, 0)[1]))
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
