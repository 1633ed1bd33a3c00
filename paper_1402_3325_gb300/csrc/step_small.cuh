// step_small.cuh -- interface of the single-block kernel for small systems.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "step_batched.cuh"

namespace sakura {

// Measured on GB300 (steps of 100 per call, random systems): this kernel
// takes 6.5 us per step at n = 2, 8.6 at 9, 8.9 at 16, 11.9 at 20, 17.8 at
// 24 and 22.5 at 32, the multi-kernel step 16.4-18.4 us throughout: past
// about 22 particles the pairs' FP64 work on one SM outweighs the launch
// and kernel-boundary latency that the single block saves.
constexpr int kSmallMaxN = 20;                                 // particles
constexpr int kSmallMaxPairs = kSmallMaxN * (kSmallMaxN - 1) / 2;
constexpr int kSmallMaxWarps = (kSmallMaxPairs + 31) / 32;     // one per 32 pairs (6)

struct SmallArgs {
    const double *src;        // [6][n] state read at the start (device or mapped host)
    double *dst;              // [6][n] state written at the end (may equal src)
    const double *mass;       // [n]
    int n;
    int nsteps;
    int nsub;                 // sub-steps per step: 1, or 3 / 9 / 27 for orders 4 / 6 / 8
    double sub[kMaxSubsteps]; // time weight of each sub-step (the composition)
    double dt;                // step
    double drift_frac;        // first drift / tau (order 2: 1/2, 1: 0, -1: 1)
    double post_drift_frac;   // last drift / tau (order 2: 1/2, 1: 1, -1: 0)
    double pre, post;         // backward-drift fractions of the pair map
    double tol;
    int max_iter;
    int bisection;
    int guess;                // initial guess of pair_setup (and of the FP32 phase of
                              // the double-word form) when not seeded
    unsigned *status;
    unsigned long long *stats;
};

// Warps of the block for n particles: one per 32 pairs, at least 4 (one per
// SM sub-partition), at most kSmallMaxWarps.
int small_warps(int n);
// One launch of one block running a.nsteps steps; seed: the single-precision
// seed and Taylor carry of the FP64 kernels; dw: the double-word form (pair
// solves on the FP32 pipe, FP64 solves for the pairs it does not admit).
void launch_small(const SmallArgs &a, bool stats, bool seed, bool dw, cudaStream_t s);

}  // namespace sakura
