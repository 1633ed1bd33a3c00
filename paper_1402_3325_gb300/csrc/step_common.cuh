// step_common.cuh -- arguments and launchers shared by the step kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace sakura {

// indices into the device statistics counters
constexpr int kStatIters = 0;
constexpr int kStatMaxIters = 1;
constexpr int kStatSlots = 2;
constexpr int kStatFallbacks = 3;
constexpr int kStatFp32Pairs = 4;
constexpr int kStatCount = 8;

struct StepArgs {
    const double *state;  // [6][n] pre-step state (read only)
    const double *mass;   // [n]
    double *partial;      // [nsplit][6][n] per-segment row sums of mu * delta
    int64_t n;
    int64_t jchunk;       // j segment length
    double tau;
    double drift;         // one-subscript drift applied to loaded positions
    double pre, post;     // backward-drift fractions of the pair map
    double tol;           // Kepler tolerance (x DBL_EPSILON)
    int max_iter;
    int bisection;
    unsigned *status;
    unsigned long long *stats;
};

void launch_pair_step_fp64(const StepArgs &a, int warps, int nsplit, bool stats,
                           cudaStream_t s);
void launch_apply_step(double *state, const double *mass, const double *partial, int64_t n,
                       int nsplit, double tau, int order, unsigned *status, cudaStream_t s);
void launch_energy(const double *state, const double *mass, int64_t n, double *work,
                   int nwork, double *out, unsigned *status, cudaStream_t s);
int energy_work_size(int64_t n);

}  // namespace sakura
