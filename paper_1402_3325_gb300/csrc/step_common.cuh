// step_common.cuh -- arguments and launchers shared by the step kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "df64.cuh"
#include "kepler_fp32.cuh"

namespace sakura {

struct MlpWeights;

// Programmatic dependent launch (sm_90 and later).  A kernel launched by
// launch_pdl may begin while the kernel before it in the stream is still
// running: griddep_wait() returns once that kernel has completed and its
// writes are visible (a hardware dependency, not a polling loop), so every
// such kernel calls it before it reads what its predecessor wrote.
// griddep_launch() lets the next kernel in the stream begin its launch.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

inline cudaError_t launch_pdl(const void *fn, dim3 grid, dim3 block, void **args, size_t smem,
                              cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// indices into the device statistics counters
constexpr int kStatIters = 0;
constexpr int kStatMaxIters = 1;
constexpr int kStatSlots = 2;
constexpr int kStatFallbacks = 3;
constexpr int kStatFp32Pairs = 4;
constexpr int kStatCarries = 5;
constexpr int kStatCount = 8;

struct StepArgs {
    const double *X;      // [7][n] drifted positions, velocities, masses (prep kernel)
    double *partial;      // [slots][6][n] row sums of mu_ij delta / m_i, split by warp
    int64_t n;
    double tau;
    double pre, post;     // backward-drift fractions of the pair map
    double tol;           // Kepler tolerance (x DBL_EPSILON)
    int max_iter;
    int bisection;
    int guess;            // 0 standard, 2 second-order analytic
    const MlpWeights *mlp; // learned guess network (device), or nullptr
    const float *X32;      // [10][n] float copy for the single-precision seed
                           // (hi xyz, lo xyz, v xyz, m), or nullptr
    float ptau32, t32;     // (float)(pre tau), (float)tau for the seed
    unsigned *status;
    unsigned long long *stats;
    // mixed form in the FP64 tile kernel (mixed = 1; 2 with the FP64-class
    // pairs seeded): pairs the class rule admits are solved in FP32 (t32,
    // post32) and accumulated in FP64
    int mixed;
    ClassRule rule;
    float post32;
};

// extra arguments of the mixed-precision pair kernel
struct MixedArgs {
    const float *X32;     // [10][n] hi xyz, lo xyz, v xyz, m (floats)
    ClassRule rule;       // FP32 class rule (kepler_fp32.cuh)
    float tau32, post32;  // tau and the post-drift fraction in FP32
};

void launch_prep_mixed(const double *state, const double *mass, double *X, float *X32,
                       int64_t n, double drift, unsigned *status, cudaStream_t s);
void launch_pair_step_mixed(const StepArgs &a, const MixedArgs &ma, int blocks, bool stats,
                            cudaStream_t s);
int pair_step_mixed_blocks_per_sm(bool stats);
// The row-group kernels' declarations: step_grp.cuh.
// the FP32 class of every ordered pair as the mixed kernels decide it
// (out: n x n bytes), from the float copy that launch_prep_mixed writes
void launch_pair_classes(const float *X32, int64_t n, const ClassRule &rule, unsigned char *out,
                         cudaStream_t s);

// Tiling of the symmetric (Newton's third law) kernels, step_sym.cu and
// step_df64.cu.  Tile t = J (J + 1) / 2 + I covers row block I and column
// block J, I <= J < nb; its 32 systolic steps are the tile-steps
// 32 t .. 32 t + 31 of T = 32 tiles.  Warp w of W takes the contiguous
// tile-steps [w T / W, (w + 1) T / W) (W <= T, so no range is empty), so every
// warp gets T / W steps to within one.  The warp's piece of a tile is that
// tile's segment number w - sym_owner(32 t); its row sums go to slot
// J Smax + segment of the rows' particles and its column sums to slot
// I Smax + segment of the columns' particles; Smax = ceil(32 W / T) + 1 bounds
// the segments of any tile (32 consecutive tile-steps meet at most
// ceil(31 W / T) + 1 ranges).  The apply kernels read exactly the slots that
// exist (sym_segments), in a fixed order.
__device__ __forceinline__ int64_t sym_owner(int64_t p, int64_t W, int64_t T)
{
    return ((p + 1) * W - 1) / T;
}

__device__ __forceinline__ void sym_tile_of(int64_t t, int64_t &I, int64_t &J)
{
    int64_t j = (int64_t)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((j + 1) * (j + 2) / 2 <= t) ++j;
    while (j * (j + 1) / 2 > t) --j;
    J = j;
    I = t - j * (j + 1) / 2;
}

__device__ __forceinline__ int sym_segments(int64_t t, int64_t W, int64_t T)
{
    return (int)(sym_owner(32 * t + 31, W, T) - sym_owner(32 * t, W, T)) + 1;
}

// extra arguments of the double-word pair kernel
struct DwArgs {
    const float *X3;      // [20][n] three-float drifted state, double-word masses
    float ptau32, t32;    // (float)(pre tau), (float)tau for the FP32 phase
    dw ptau, t, qtau;     // pre tau, tau and post tau as double-words
};

void launch_prep_df64(const double *state, const double *mass, double *X, float *X3, int64_t n,
                      double drift, unsigned *status, cudaStream_t s);
void launch_pair_step_df64(const StepArgs &a, const DwArgs &da, int Smax, int64_t T, int blocks,
                           bool stats, cudaStream_t s);
void launch_apply_df64(double *state, const double *X, const void *partial, int64_t n, int Smax,
                       int64_t W, int64_t T, double post_drift, unsigned *status,
                       cudaStream_t s);
int pair_step_df64_blocks_per_sm(bool stats);

// pair kernel: one persistent wave of `blocks` blocks of `warps` warps
void launch_pair_step_fp64(const StepArgs &a, int warps, int blocks, bool stats,
                           cudaStream_t s);
int pair_step_fp64_blocks_per_sm(int warps, bool stats, bool learned = false);

// learned-guess network: data, training and evaluation (mlp.cu)
void launch_sample_pairs(const double *X, int64_t n, double tau, double pre, const int64_t *ids,
                         int64_t count, float *feat, float *target, int *iters, double tol,
                         unsigned *status, cudaStream_t s);
void launch_mlp_grad(const float *P, const float *norm, const float *feat, const float *target,
                     int64_t B, float *scratch, float *grad, float *loss, cudaStream_t s);
size_t mlp_grad_scratch_floats(int64_t B);
void launch_adam(float *P, float *m, float *v, const float *g, float lr, float b1t, float b2t,
                 cudaStream_t s);
void launch_mlp_pack(const float *blob, MlpWeights *W, cudaStream_t s);
void launch_mlp_eval(const MlpWeights *W, const float *feat, int64_t count, float *out,
                     cudaStream_t s);
// symmetric (Newton's third law) pair kernel: items = tiles * S
int pair_step_sym_blocks_per_sm(bool stats, bool learned, bool seed = false,
                                bool mixed = false);
void launch_pair_step_sym(const StepArgs &a, int Smax, int64_t T, int blocks, bool stats,
                          cudaStream_t s);
// fuse: also apply the next sub-step's drift next_drift and write its
// drifted copy to X (and X32, if not null), replacing the next prep kernel
void launch_apply_sym(double *state, double *X, float *X32, const double *partial, int64_t n,
                      int Smax, int64_t W, int64_t T, double post_drift, bool fuse,
                      double next_drift, unsigned *status, cudaStream_t s);

// number of partial-sum slots per row for W warps
int pair_step_slots(int64_t n, int64_t W);
// X32 (optional): float copy for the single-precision seed, [10][n]
void launch_prep_step(const double *state, const double *mass, double *X, float *X32, int64_t n,
                      double drift, unsigned *status, cudaStream_t s);
// W = 0: no pair sums (n = 1)
void launch_apply_step(double *state, const double *X, const double *partial, int64_t n,
                       int64_t W, double post_drift, unsigned *status, cudaStream_t s);
void launch_energy(const double *state, const double *mass, int64_t n, double *work,
                   int nwork, double *out, unsigned *status, cudaStream_t s);
int energy_work_size(int64_t n);

}  // namespace sakura
