"""Algorithmic FP32 work of one double-word pair solve, for the roofline of
the double-word form in bench.py.

The library's double-word code (csrc/df64.cuh, csrc/kepler_df64.cuh) is
compiled as host C++ with an operation tally (tests/df64_host.cpp,
-DSAKURA_DW_COUNT): every pair of a workload's first step is taken through
the six exact three-float differences, the FP32 phase, the double-word
phase and the two weighted double-word accumulations, and its floating-point
operations are counted (add, subtract, multiply = 1, fused multiply-add = 2;
special-function approximations counted apart).  The mean over the admitted
pairs is the per-solve figure.

    python tests/df64_flop_count.py            # prints the figures bench.py uses
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

# pairs counted per workload: every unordered pair up to this many, else a
# seeded uniform sample of unordered pairs
MAX_PAIRS = 400_000


def build(out_dir: str) -> ctypes.CDLL:
    out = os.path.join(out_dir, "libdf64count.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                    "-DSAKURA_DW_COUNT", "-shared", "-fPIC",
                    os.path.join(HERE, "df64_host.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    D = ctypes.POINTER(ctypes.c_double)
    lib.dw_count_pairs.argtypes = [ctypes.c_long, D, D, D, D, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, D, D,
                                   ctypes.POINTER(ctypes.c_long)]
    return lib


def count(lib, system, guess: int = 2):
    """(flops per admitted solve, approximations per solve, admitted share)
    for the pairs of the first order-2 step of `system`."""
    X = np.concatenate([system.r + 0.5 * system.dt * system.v, system.v], axis=1)
    n = system.n
    if n * (n - 1) // 2 <= MAX_PAIRS:
        i, j = np.triu_indices(n, 1)
    else:
        rng = np.random.default_rng(0)
        i = rng.integers(0, n, MAX_PAIRS)
        j = (i + rng.integers(1, n, MAX_PAIRS)) % n
    D = ctypes.POINTER(ctypes.c_double)
    dp = lambda a: np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(D)
    fl, mu, ad = ctypes.c_double(), ctypes.c_double(), ctypes.c_long()
    lib.dw_count_pairs(len(i), dp(X[i]), dp(X[j]), dp(system.m[i]), dp(system.m[j]),
                       system.dt, 0.5, 0.5, guess, ctypes.byref(fl), ctypes.byref(mu),
                       ctypes.byref(ad))
    return fl.value / ad.value, mu.value / ad.value, ad.value / len(i)


def workloads():
    from paper_1402_3325_gb300 import ics
    return {"plummer1024": ics.plummer(1024, seed=0),
            "bh16384": ics.bh_cluster(16384, seed=0),
            "binaries16384": ics.plummer_binaries(16384, seed=0)}


def main():
    with tempfile.TemporaryDirectory() as tmp:
        lib = build(tmp)
        for name, s in workloads().items():
            f, m, a = count(lib, s)
            print(f"{name}: {f:.1f} flops per solve, {m:.2f} approximations, admitted {a:.4f}")


if __name__ == "__main__":
    main()
