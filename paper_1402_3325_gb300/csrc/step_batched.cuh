// step_batched.cuh -- interface of the batched ensemble kernel.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace sakura {

struct MlpWeights;

constexpr int kMaxSubsteps = 27;

struct BatchArgs {
    double *state;            // [6][total] SoA of all systems, updated in place
    const double *mass;       // [total]
    const int64_t *offsets;   // [nsys + 1]
    const double *dt;         // [nsys]
    const int *task_begin;    // [ntasks + 1] ranges into task_sys
    const int *task_sys;      // systems of each task
    int ntasks;
    int *counter;             // work counter, zeroed before the launch
    int64_t total;            // particles in all systems (row stride of state)
    int nsteps;
    int nsub;                 // sub-steps per step: 1, or 3 / 9 / 27 for orders 4 / 6 / 8
    double sub[kMaxSubsteps]; // time weight of each sub-step (the composition)
    double drift_frac;        // first drift / tau (order 2: 1/2, 1: 0, -1: 1)
    double post_drift_frac;   // last drift / tau (order 2: 1/2, 1: 1, -1: 0)
    double pre, post;         // backward-drift fractions of the pair map
    double tol;
    int max_iter;
    int bisection;
    int guess;
    int seed;                 // 1: single-precision seed and Taylor carry
    const MlpWeights *mlp;    // learned guess network, or nullptr
    unsigned *status;
    unsigned long long *stats;
};

int batched_blocks_per_sm(int warps, bool stats, bool learned = false, bool seed = false);
void build_batch_schedule(const int64_t *offsets, int nsys, std::vector<int> &task_begin,
                          std::vector<int> &task_sys);
void launch_batched(const BatchArgs &a, int warps, int blocks, bool stats, cudaStream_t s);
cudaError_t build_batched_graph(const BatchArgs &a, int warps, int blocks, bool stats,
                                cudaGraphExec_t *exec);

}  // namespace sakura
