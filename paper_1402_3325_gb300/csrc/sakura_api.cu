// sakura_api.cu -- the extern "C" boundary declared in include/sakura.h.
//
// Holds the process-wide context (device, stream, configuration, library-owned
// scratch), validates arguments, sizes the launches and maps the device status
// word to return codes.  All arithmetic of the method runs in the kernels.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <algorithm>
#include <cstring>
#include <vector>

#include "sakura.h"
#include "kepler_fp64.cuh"
#include "mlp_infer.cuh"
#include "step_batched.cuh"
#include "step_common.cuh"
#include "step_grp.cuh"
#include "step_small.cuh"

namespace {

struct Buffer {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Cached state of the batched ensemble path.
struct BatchCache {
    std::vector<int64_t> host_offsets;  // schedule key
    Buffer task_begin, task_sys, counter, tune_state;
    int ntasks = 0;
    int warps = 4;
    int blocks = 0;
    bool tuned = false;
    cudaGraphExec_t exec = nullptr;
    sakura::BatchArgs graph_args{};
    int graph_warps = 0, graph_blocks = 0;
    bool graph_stats = false;
    double tuned_ms[4] = {0, 0, 0, 0};
};

struct Context {
    bool init = false;
    sakura_config cfg{};
    cudaStream_t stream = nullptr;
    unsigned *d_status = nullptr;
    unsigned long long *d_stats = nullptr;
    double *d_energy = nullptr;  // [3] E, T, U
    unsigned *h_status = nullptr;      // page-locked host copy of the status word
    unsigned *h_status_dev = nullptr;  // its address on the device
    Buffer partial;              // pair-kernel segment sums
    Buffer energy_work;
    Buffer host_state, host_mass;  // device copies for sakura_evolve_host
    int64_t steps = 0;
    int64_t pairs = 0;
    int64_t solves = 0;
    int sm_count = 152;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> timers;  // pending pair-kernel timings
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spare;
    double timed_ms = 0.0;
    int64_t timed_launches = 0;
    int64_t group_launches = 0;
    BatchCache batch;
    Buffer mlp, mlp_blob, mlp_scratch, mlp_adam;  // learned-guess network and training
    bool mlp_loaded = false;
};

Context g;

int grow(Buffer &b, size_t bytes)
{
    if (b.bytes >= bytes) return SAKURA_OK;
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SAKURA_E_NOMEM;
    }
    b.bytes = bytes;
    return SAKURA_OK;
}

int status_to_code(unsigned st)
{
    if (st & sakura::kStatusMass) return SAKURA_E_MASS;
    if (st & sakura::kStatusNonfinite) return SAKURA_E_NONFINITE;
    if (st & sakura::kStatusCoincident) return SAKURA_E_COINCIDENT;
    if (st & sakura::kStatusKepler) return SAKURA_E_KEPLER;
    if (st & sakura::kStatusTimeout) return SAKURA_E_TIMEOUT;
    return SAKURA_OK;
}

// Event pair for one timed launch (reused across calls).
std::pair<cudaEvent_t, cudaEvent_t> take_timer()
{
    if (!g.spare.empty()) {
        auto p = g.spare.back();
        g.spare.pop_back();
        return p;
    }
    std::pair<cudaEvent_t, cudaEvent_t> p{nullptr, nullptr};
    cudaEventCreate(&p.first);
    cudaEventCreate(&p.second);
    return p;
}

// Fold completed timings into the totals (the caller has synchronised).
void collect_timers()
{
    for (auto &p : g.timers) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) {
            g.timed_ms += ms;
            g.timed_launches += 1;
        }
        g.spare.push_back(p);
    }
    g.timers.clear();
    cudaGetLastError();
}

int launch_error()
{
    return cudaGetLastError() == cudaSuccess ? SAKURA_OK : SAKURA_E_CUDA;
}

// Synchronise, read and clear the status word.
// Copies the status word into page-locked host memory and clears it (one
// thread, after every earlier kernel on the stream): one launch instead of a
// copy-engine transfer, whose fixed latency is several times larger.  It is
// launched as a programmatic dependent; griddep_wait returns once the kernel
// before it has completed and its writes are visible.
__global__ void publish_status_kernel(unsigned *status, unsigned *host_status)
{
    sakura::griddep_wait();
    const unsigned st = *status;
    *host_status = st;
    if (st) *status = 0u;
}

int drain_status()
{
    void *args[] = {(void *)&g.d_status, (void *)&g.h_status_dev};
    if (sakura::launch_pdl((const void *)publish_status_kernel, dim3(1), dim3(1), args, 0,
                           g.stream) != cudaSuccess) {
        cudaGetLastError();
        return SAKURA_E_CUDA;
    }
    if (cudaStreamSynchronize(g.stream) != cudaSuccess) return SAKURA_E_CUDA;
    return status_to_code(*(volatile unsigned *)g.h_status);
}

struct Plan {
    int warps;
    int blocks;
    int64_t W;  // warps in the persistent pair-kernel grid
};

// Launch shape of the persistent pair kernel: one wave of resident blocks
// (or grid_blocks), never more warps than 32-pair batches: with W <= B every
// warp owns at least one batch, so the slots of a row are all written.  (For
// n <= 32 a row is a single batch and W may exceed B harmlessly.)
Plan plan_step(int64_t n)
{
    Plan p;
    const bool mixed = g.cfg.precision == SAKURA_PREC_MIXED;
    p.warps = g.cfg.block_warps > 0 ? g.cfg.block_warps : 4;
    if (p.warps != 4 && p.warps != 8 && p.warps != 16) p.warps = 4;
    if (mixed) p.warps = 4;
    const int64_t nb = (n + 31) / 32;
    const int64_t B = n * nb;
    int64_t blocks = g.cfg.grid_blocks;
    if (blocks <= 0) {
        const bool st = (g.cfg.flags & SAKURA_FLAG_STATS) != 0;
        const bool learned = g.cfg.guess == SAKURA_GUESS_LEARNED;
        const int bps = mixed ? sakura::pair_step_mixed_blocks_per_sm(st)
                              : sakura::pair_step_fp64_blocks_per_sm(p.warps, st, learned);
        blocks = (int64_t)g.sm_count * bps;
    }
    blocks = std::min<int64_t>(blocks, std::max<int64_t>(1, B / p.warps));
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, 1 << 20));
    p.blocks = (int)blocks;
    p.W = blocks * p.warps;
    return p;
}

// The mixed form's class rule with the configured thresholds, for a step
// whose backward drift is ptau = pre * tau (kepler_fp32.cuh).
sakura::ClassRule class_rule(double ptau)
{
    sakura::ClassRule r;
    r.ptau = (float)ptau;
    r.rmin2 = (float)(g.cfg.mixed_r_min * g.cfg.mixed_r_min);
    r.emax2m1 = (float)(g.cfg.mixed_e_max * g.cfg.mixed_e_max - 1.0);
    r.ehyp2m1 = (float)(g.cfg.mixed_e_hyp * g.cfg.mixed_e_hyp - 1.0);
    r.rule = g.cfg.mixed_rule;
    return r;
}

sakura::dw split_dw(double d)
{
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}

// The mixed form with each unordered pair once, in row-group phases
// (step_mixed.cu): prep (drift and float copy), pair and apply kernels.
int step_device_mixed_grp(const double *src, double *dst, const double *masses, int64_t n,
                          double dt, int order)
{
    const bool stats = (g.cfg.flags & SAKURA_FLAG_STATS) != 0;
    const bool seed = g.cfg.guess == SAKURA_GUESS_FP32;
    int64_t blocks =
        g.cfg.grid_blocks > 0
            ? g.cfg.grid_blocks
            : (int64_t)g.sm_count * sakura::pair_step_grp_mixed_blocks_per_sm(stats, seed);
    const sakura::GrpLayout L = sakura::make_grp_layout(n, sakura::kMixedGrpShape, blocks);
    // scratch: X[7][n] doubles, row partials [Hmax][6][n], column partials
    // [ng][6][n] and [blocks][6][32], then X32[10][n] floats
    int rc = grow(g.partial, (size_t)(7 * n + (int64_t)(L.Hmax + L.ng) * 6 * n + blocks * 192 +
                                      5 * n) *
                                 sizeof(double));
    if (rc) return rc;
    double *X = (double *)g.partial.ptr;
    sakura::GrpParts parts;
    parts.row = X + 7 * n;
    parts.col = parts.row + (int64_t)L.Hmax * 6 * n;
    parts.colx = parts.col + (int64_t)L.ng * 6 * n;
    float *X32 = (float *)(parts.colx + blocks * 192);
    const double drift = order == 2 ? 0.5 * dt : (order == 1 ? 0.0 : dt);
    const double post_drift = order == 2 ? 0.5 * dt : (order == 1 ? dt : 0.0);
    sakura::launch_prep_mixed(src, masses, X, X32, n, drift, g.d_status, g.stream);
    sakura::StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.X = X;
    a.n = n;
    a.tau = dt;
    a.pre = order == 2 ? 0.5 : (order == 1 ? 0.0 : 1.0);
    a.post = 1.0 - a.pre;
    a.tol = g.cfg.kepler_tol * DBL_EPSILON;
    a.max_iter = g.cfg.kepler_max_iter;
    a.bisection = g.cfg.kepler_bisection;
    a.guess = (g.cfg.guess == SAKURA_GUESS_TAYLOR || g.cfg.guess == SAKURA_GUESS_FP32) ? 2 : 0;
    a.X32 = seed ? X32 : nullptr;
    a.ptau32 = (float)(a.pre * dt);
    a.t32 = (float)dt;
    a.status = g.d_status;
    a.stats = g.d_stats;
    sakura::MixedArgs ma;
    ma.X32 = X32;
    ma.rule = class_rule(a.pre * dt);
    ma.tau32 = (float)dt;
    ma.post32 = (float)a.post;
    const bool timing = (g.cfg.flags & SAKURA_FLAG_TIMING) != 0;
    std::pair<cudaEvent_t, cudaEvent_t> tm{nullptr, nullptr};
    if (timing) {
        tm = take_timer();
        cudaEventRecord(tm.first, g.stream);
    }
    sakura::launch_pair_step_grp_mixed(a, ma, L, parts, (int)blocks, stats, g.stream);
    g.group_launches += 1;
    if (timing) {
        cudaEventRecord(tm.second, g.stream);
        g.timers.push_back(tm);
    }
    sakura::launch_apply_grp(dst, X, nullptr, parts, n, L, blocks, post_drift, false, 0.0,
                             g.d_status, g.stream);
    rc = launch_error();
    if (rc) return rc;
    g.steps += 1;
    g.pairs += n * (n - 1);
    int64_t diag = 0;  // ordered pairs inside diagonal tiles
    for (int64_t b = 0; b < L.nb; ++b) {
        const int64_t nbk = std::min<int64_t>(32, n - 32 * b);
        diag += nbk * (nbk - 1);
    }
    g.solves += (n * (n - 1) - diag) / 2 + diag;
    return SAKURA_OK;
}

// Scratch of the two symmetric layouts: the systolic tile kernels keep
// 6 doubles per particle per (other block, tile segment) slot, at most
// 8 nb n of them; the row-group kernels one 6-vector per particle per group
// (nb / G groups) plus a few row pieces.
double tile_partial_bytes(int64_t n) { return 8.0 * 6.0 * 8.0 * (double)((n + 31) / 32) * n; }
double group_partial_bytes(int64_t n, int G)
{
    return 48.0 * (double)n * (double)(((n + 31) / 32 + G - 1) / G + 16);
}

// The symmetric FP64 form runs on systolic tiles (step_sym.cu) below
// kFp64GroupsMinN bodies and in row-group phases (step_grp.cu) from there,
// where the row groups are level or faster and write about a hundredth of
// the tile kernel's partial traffic (measured with the single-precision
// seed, ms per step, tiles / row groups: black hole + 2047 stars 0.380 /
// 0.412, + 4095 stars 1.376 / 1.351, + 8191 stars 5.378 / 5.182, + 12287
// stars 12.07 / 11.54, + 16383 stars 21.58 / 20.41; Plummer 2048 bodies
// 0.358 / 0.393, 4096 1.354 / 1.357, 8192 5.350 / 5.262, 12288 12.02 /
// 11.71, 16384 21.47 / 20.73).  The flags force either kernel.
constexpr int64_t kFp64GroupsMinN = 4096;
bool fp64_groups(int64_t n)
{
    if (g.cfg.flags & SAKURA_FLAG_GROUPS) return true;
    if (g.cfg.flags & SAKURA_FLAG_TILES) return false;
    return n >= kFp64GroupsMinN;
}

// The mixed form's kernels.  Under the literal rule, which admits few pairs
// in clusters (the black-hole cluster: 0.01 % of them), the FP64 kernels
// with an inline class test: on tiles (step_sym.cu) or in row groups
// (step_grp.cu) as for the FP64 form.  Under the hyperbolic rule the
// row-group mixed kernel (step_mixed.cu), or the tile kernel with the inline
// test when SAKURA_FLAG_TILES forces it.
enum class MixedKernel { Tiles, Fp64Groups, MixedGroups };

MixedKernel mixed_kernel(int64_t n)
{
    if (g.cfg.mixed_rule == SAKURA_MIXED_RULE_LITERAL)
        return fp64_groups(n) ? MixedKernel::Fp64Groups : MixedKernel::Tiles;
    if (g.cfg.flags & SAKURA_FLAG_TILES) return MixedKernel::Tiles;
    return MixedKernel::MixedGroups;
}

// The double-word form: tiles while their partials take at most
// kDf64TileMaxBytes (about 13400 bodies; at 8192 bodies the tiles measured
// 2.15 ms per step against 2.24 in row groups), row groups beyond; the
// flags force either.
constexpr double kDf64TileMaxBytes = 2.0 * 1024 * 1024 * 1024;
bool df64_groups(int64_t n)
{
    if (g.cfg.flags & SAKURA_FLAG_GROUPS) return true;
    if (g.cfg.flags & SAKURA_FLAG_TILES) return false;
    return tile_partial_bytes(n) > kDf64TileMaxBytes;
}

// The double-word form in row-group phases (step_df64.cu): prep (drift and
// three-float copy), pair and apply kernels.
int step_device_df64_grp(const double *src, double *dst, const double *masses, int64_t n,
                         double dt, int order)
{
    const bool stats = (g.cfg.flags & SAKURA_FLAG_STATS) != 0;
    int64_t blocks = g.cfg.grid_blocks > 0
                         ? g.cfg.grid_blocks
                         : (int64_t)g.sm_count * sakura::pair_step_grp_df64_blocks_per_sm(stats);
    const sakura::GrpLayout L = sakura::make_grp_layout(n, sakura::kDf64GrpShape, blocks);
    // scratch: X[7][n] doubles, row partials [Hmax][6][n], column partials
    // [ng][6][n] and [blocks][6][32], then X3[20][n] floats
    int rc = grow(g.partial, (size_t)(7 * n + (int64_t)(L.Hmax + L.ng) * 6 * n + blocks * 192 +
                                      10 * n) *
                                 sizeof(double));
    if (rc) return rc;
    double *X = (double *)g.partial.ptr;
    sakura::GrpParts parts;
    parts.row = X + 7 * n;
    parts.col = parts.row + (int64_t)L.Hmax * 6 * n;
    parts.colx = parts.col + (int64_t)L.ng * 6 * n;
    float *X3 = (float *)(parts.colx + blocks * 192);
    const double drift = order == 2 ? 0.5 * dt : (order == 1 ? 0.0 : dt);
    const double post_drift = order == 2 ? 0.5 * dt : (order == 1 ? dt : 0.0);
    sakura::launch_prep_df64(src, masses, X, X3, n, drift, g.d_status, g.stream);
    sakura::StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.X = X;
    a.n = n;
    a.tau = dt;
    a.pre = order == 2 ? 0.5 : (order == 1 ? 0.0 : 1.0);
    a.post = 1.0 - a.pre;
    a.tol = g.cfg.kepler_tol * DBL_EPSILON;
    a.max_iter = g.cfg.kepler_max_iter;
    a.bisection = g.cfg.kepler_bisection;
    a.guess = (g.cfg.guess == SAKURA_GUESS_TAYLOR || g.cfg.guess == SAKURA_GUESS_FP32) ? 2 : 0;
    a.status = g.d_status;
    a.stats = g.d_stats;
    sakura::DwArgs da;
    da.X3 = X3;
    da.ptau32 = (float)(a.pre * dt);
    da.t32 = (float)dt;
    da.ptau = split_dw(a.pre * dt);
    da.t = split_dw(dt);
    da.qtau = split_dw(a.post * dt);
    const bool timing = (g.cfg.flags & SAKURA_FLAG_TIMING) != 0;
    std::pair<cudaEvent_t, cudaEvent_t> tm{nullptr, nullptr};
    if (timing) {
        tm = take_timer();
        cudaEventRecord(tm.first, g.stream);
    }
    sakura::launch_pair_step_grp_df64(a, da, L, parts, (int)blocks, stats, g.stream);
    g.group_launches += 1;
    if (timing) {
        cudaEventRecord(tm.second, g.stream);
        g.timers.push_back(tm);
    }
    sakura::launch_apply_grp(dst, X, nullptr, parts, n, L, blocks, post_drift, false, 0.0,
                             g.d_status, g.stream);
    rc = launch_error();
    if (rc) return rc;
    g.steps += 1;
    g.pairs += n * (n - 1);
    int64_t diag = 0;  // ordered pairs inside diagonal tiles
    for (int64_t b = 0; b < L.nb; ++b) {
        const int64_t nbk = std::min<int64_t>(32, n - 32 * b);
        diag += nbk * (nbk - 1);
    }
    g.solves += (n * (n - 1) - diag) / 2 + diag;
    return SAKURA_OK;
}

// The FP64 form with each unordered pair once, in row-group phases
// (step_grp.cu).  prepped: X (and X32) already hold this sub-step's drifted
// state, written by the previous apply kernel; fuse: the apply kernel also
// applies the next sub-step's drift next_drift and writes its X (and X32).
int step_device_fp64_grp(const double *src, double *dst, const double *masses, int64_t n,
                         double dt, int order, bool prepped, bool fuse, double next_drift,
                         bool mixed = false)
{
    const bool stats = (g.cfg.flags & SAKURA_FLAG_STATS) != 0;
    const bool learned = !mixed && g.cfg.guess == SAKURA_GUESS_LEARNED;
    const bool seed = g.cfg.guess == SAKURA_GUESS_FP32;
    int64_t blocks = g.cfg.grid_blocks > 0
                         ? g.cfg.grid_blocks
                         : (int64_t)g.sm_count *
                               sakura::pair_step_grp_blocks_per_sm(stats, learned, seed, mixed);
    const sakura::GrpLayout L = sakura::make_grp_layout(n, sakura::kFp64GrpShape, blocks);
    // scratch: X[7][n] doubles, row partials [Hmax][6][n], column partials
    // [ng][6][n] and [blocks][6][32], then X32[10][n] floats (single-precision
    // seed)
    int rc = grow(g.partial, (size_t)(7 * n + (int64_t)(L.Hmax + L.ng) * 6 * n + blocks * 192 +
                                      5 * n) *
                                 sizeof(double));
    if (rc) return rc;
    double *X = (double *)g.partial.ptr;
    sakura::GrpParts parts;
    parts.row = X + 7 * n;
    parts.col = parts.row + (int64_t)L.Hmax * 6 * n;
    parts.colx = parts.col + (int64_t)L.ng * 6 * n;
    float *X32 = (seed || mixed) ? (float *)(parts.colx + blocks * 192) : nullptr;
    const double drift = order == 2 ? 0.5 * dt : (order == 1 ? 0.0 : dt);
    const double post_drift = order == 2 ? 0.5 * dt : (order == 1 ? dt : 0.0);
    if (!prepped) sakura::launch_prep_step(src, masses, X, X32, n, drift, g.d_status, g.stream);
    sakura::StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.X = X;
    a.X32 = X32;
    a.n = n;
    a.tau = dt;
    a.pre = order == 2 ? 0.5 : (order == 1 ? 0.0 : 1.0);
    a.post = 1.0 - a.pre;
    a.ptau32 = (float)(a.pre * dt);
    a.t32 = (float)dt;
    a.tol = g.cfg.kepler_tol * DBL_EPSILON;
    a.max_iter = g.cfg.kepler_max_iter;
    a.bisection = g.cfg.kepler_bisection;
    a.guess = (g.cfg.guess == SAKURA_GUESS_TAYLOR || g.cfg.guess == SAKURA_GUESS_FP32) ? 2 : 0;
    a.mlp = learned ? (const sakura::MlpWeights *)g.mlp.ptr : nullptr;
    a.status = g.d_status;
    a.stats = g.d_stats;
    if (mixed) {
        a.mixed = seed ? 2 : 1;
        a.rule = class_rule(a.pre * dt);
        a.post32 = (float)a.post;
    }
    const bool timing = (g.cfg.flags & SAKURA_FLAG_TIMING) != 0;
    std::pair<cudaEvent_t, cudaEvent_t> tm{nullptr, nullptr};
    if (timing) {
        tm = take_timer();
        cudaEventRecord(tm.first, g.stream);
    }
    sakura::launch_pair_step_grp(a, L, parts, (int)blocks, stats, g.stream);
    g.group_launches += 1;
    if (timing) {
        cudaEventRecord(tm.second, g.stream);
        g.timers.push_back(tm);
    }
    sakura::launch_apply_grp(dst, X, X32, parts, n, L, blocks, post_drift, fuse, next_drift,
                             g.d_status, g.stream);
    rc = launch_error();
    if (rc) return rc;
    g.steps += 1;
    g.pairs += n * (n - 1);
    int64_t diag = 0;  // ordered pairs inside diagonal tiles
    for (int64_t b = 0; b < L.nb; ++b) {
        const int64_t nbk = std::min<int64_t>(32, n - 32 * b);
        diag += nbk * (nbk - 1);
    }
    g.solves += (n * (n - 1) - diag) / 2 + diag;
    return SAKURA_OK;
}

// Unordered pairs once (Newton's third law): systolic 32 x 32 tiles; df64:
// the pair solves in double-word arithmetic (step_df64.cu).
// prepped: X (and X32) already hold this sub-step's drifted state, written
// by the previous apply kernel (FP64 form only); fuse: the apply kernel also
// applies the next sub-step's drift next_drift and writes its X (and X32).
int step_device_sym(const double *src, double *dst, const double *masses, int64_t n, double dt,
                    int order, bool df64, bool mixed, bool prepped = false, bool fuse = false,
                    double next_drift = 0.0)
{
    if (mixed) {
        const MixedKernel k = mixed_kernel(n);
        if (k == MixedKernel::MixedGroups)
            return step_device_mixed_grp(src, dst, masses, n, dt, order);
        if (k == MixedKernel::Fp64Groups)
            return step_device_fp64_grp(src, dst, masses, n, dt, order, false, false, 0.0, true);
    }
    if (df64 && df64_groups(n)) return step_device_df64_grp(src, dst, masses, n, dt, order);
    if (!df64 && !mixed && fp64_groups(n))
        return step_device_fp64_grp(src, dst, masses, n, dt, order, prepped, fuse, next_drift);
    const bool stats = (g.cfg.flags & SAKURA_FLAG_STATS) != 0;
    const bool learned = !df64 && !mixed && g.cfg.guess == SAKURA_GUESS_LEARNED;
    const bool seed = !df64 && g.cfg.guess == SAKURA_GUESS_FP32;
    const int64_t nb = (n + 31) / 32;
    const int64_t tiles = nb * (nb + 1) / 2;
    const int bps = df64 ? sakura::pair_step_df64_blocks_per_sm(stats)
                         : sakura::pair_step_sym_blocks_per_sm(stats, learned, seed, mixed);
    // contiguous tile-step ranges for W <= T warps (step_common.cuh)
    const int64_t T = tiles * 32;
    int64_t blocks = g.cfg.grid_blocks > 0 ? g.cfg.grid_blocks : (int64_t)g.sm_count * bps;
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, T / 4));
    const int64_t W = blocks * 4;
    const int Smax = (int)((32 * W + T - 1) / T + 1);
    const int64_t nslots = nb * Smax;
    // scratch: X[7][n] doubles, tile partials [nslots][6][n] (doubles, or
    // double-words of two floats), then (df64) X3[20][n] or (seed) X32[10][n]
    // floats
    int rc = grow(g.partial, (size_t)(7 * n + nslots * 6 * n + (df64 ? 10 * n : 5 * n)) *
                                 sizeof(double));
    if (rc) return rc;
    double *X = (double *)g.partial.ptr;
    double *partial = X + 7 * n;
    float *X3 = (float *)(partial + nslots * 6 * n);
    float *X32 = (seed || mixed) ? X3 : nullptr;
    const double drift = order == 2 ? 0.5 * dt : (order == 1 ? 0.0 : dt);
    const double post_drift = order == 2 ? 0.5 * dt : (order == 1 ? dt : 0.0);
    if (df64)
        sakura::launch_prep_df64(src, masses, X, X3, n, drift, g.d_status, g.stream);
    else if (!prepped)
        sakura::launch_prep_step(src, masses, X, X32, n, drift, g.d_status, g.stream);
    sakura::StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.X = X;
    a.X32 = X32;
    a.partial = partial;
    a.n = n;
    a.tau = dt;
    a.pre = order == 2 ? 0.5 : (order == 1 ? 0.0 : 1.0);
    a.post = 1.0 - a.pre;
    a.ptau32 = (float)(a.pre * dt);
    a.t32 = (float)dt;
    a.tol = g.cfg.kepler_tol * DBL_EPSILON;
    a.max_iter = g.cfg.kepler_max_iter;
    a.bisection = g.cfg.kepler_bisection;
    a.guess = (g.cfg.guess == SAKURA_GUESS_TAYLOR || g.cfg.guess == SAKURA_GUESS_FP32) ? 2 : 0;
    a.mlp = learned ? (const sakura::MlpWeights *)g.mlp.ptr : nullptr;
    a.status = g.d_status;
    a.stats = g.d_stats;
    if (mixed) {
        a.mixed = seed ? 2 : 1;
        a.rule = class_rule(a.pre * dt);
        a.post32 = (float)a.post;
    }
    const bool timing = (g.cfg.flags & SAKURA_FLAG_TIMING) != 0;
    std::pair<cudaEvent_t, cudaEvent_t> tm{nullptr, nullptr};
    if (timing) {
        tm = take_timer();
        cudaEventRecord(tm.first, g.stream);
    }
    if (df64) {
        sakura::DwArgs da;
        da.X3 = X3;
        da.ptau32 = (float)(a.pre * dt);
        da.t32 = (float)dt;
        da.ptau = split_dw(a.pre * dt);
        da.t = split_dw(dt);
        da.qtau = split_dw(a.post * dt);
        sakura::launch_pair_step_df64(a, da, Smax, T, (int)blocks, stats, g.stream);
    } else {
        sakura::launch_pair_step_sym(a, Smax, T, (int)blocks, stats, g.stream);
    }
    if (timing) {
        cudaEventRecord(tm.second, g.stream);
        g.timers.push_back(tm);
    }
    if (df64)
        sakura::launch_apply_df64(dst, X, partial, n, Smax, W, T, post_drift, g.d_status,
                                  g.stream);
    else
        sakura::launch_apply_sym(dst, X, X32, partial, n, Smax, W, T, post_drift,
                                 fuse && !mixed, next_drift, g.d_status, g.stream);
    rc = launch_error();
    if (rc) return rc;
    g.steps += 1;
    g.pairs += n * (n - 1);
    int64_t diag = 0;  // ordered pairs inside diagonal tiles
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t nbk = std::min<int64_t>(32, n - 32 * b);
        diag += nbk * (nbk - 1);
    }
    g.solves += (n * (n - 1) - diag) / 2 + diag;
    return SAKURA_OK;
}

// The symmetric mode keeps O(n^2 / 32) partial sums; beyond kSymMaxBytes the
// ordered-pair kernel (O(n) scratch) is used instead.
constexpr double kSymMaxBytes = 16.0 * 1024 * 1024 * 1024;

// One step of the given order from src to dst (the same buffer, or two
// buffers that do not overlap): the drift kernel reads src and masses, the
// apply kernel writes dst.  Either kernel copies the masses into row 6 of the
// drifted state X[7][n] at the start of the scratch buffer (step_masses).
bool sym_path(int64_t n)
{
    if (g.cfg.pair_mode != SAKURA_PAIRS_SYMMETRIC || n < 2) return false;
    if (g.cfg.precision == SAKURA_PREC_DF64)
        return (df64_groups(n) ? group_partial_bytes(n, sakura::kDf64GrpWarps)
                               : tile_partial_bytes(n)) <= kSymMaxBytes;
    if (g.cfg.precision == SAKURA_PREC_MIXED)
        switch (mixed_kernel(n)) {
        case MixedKernel::Tiles: return tile_partial_bytes(n) <= kSymMaxBytes;
        case MixedKernel::Fp64Groups:
            return group_partial_bytes(n, sakura::kFp64GrpWarps) <= kSymMaxBytes;
        default: return group_partial_bytes(n, sakura::kMixedGrpWarps) <= kSymMaxBytes;
        }
    return (fp64_groups(n) ? group_partial_bytes(n, sakura::kFp64GrpWarps)
                           : tile_partial_bytes(n)) <= kSymMaxBytes;
}

// Sub-steps whose apply kernel can also drift for the next one: the FP64
// form on symmetric tiles.
bool fusable(int64_t n) { return sym_path(n) && g.cfg.precision == SAKURA_PREC_FP64; }

int step_device(const double *src, double *dst, const double *masses, int64_t n, double dt,
                int order, bool prepped = false, bool fuse = false, double next_drift = 0.0)
{
    if (sym_path(n))
        return step_device_sym(src, dst, masses, n, dt, order,
                               g.cfg.precision == SAKURA_PREC_DF64,
                               g.cfg.precision == SAKURA_PREC_MIXED, prepped, fuse, next_drift);
    const Plan p = plan_step(n);
    const int64_t slots = sakura::pair_step_slots(n, p.W);
    const bool mixed = g.cfg.precision == SAKURA_PREC_MIXED;
    // scratch: X[7][n] doubles, row partials [slots][6][n], then (mixed)
    // X32[10][n] floats
    const size_t doubles = (size_t)(7 * n + slots * 6 * n) + (mixed ? (size_t)(5 * n) : 0);
    int rc = grow(g.partial, doubles * sizeof(double));
    if (rc) return rc;
    double *X = (double *)g.partial.ptr;
    double *partial = X + 7 * n;
    float *X32 = (float *)(partial + slots * 6 * n);
    const double drift = order == 2 ? 0.5 * dt : (order == 1 ? 0.0 : dt);
    const double post_drift = order == 2 ? 0.5 * dt : (order == 1 ? dt : 0.0);
    if (mixed)
        sakura::launch_prep_mixed(src, masses, X, X32, n, drift, g.d_status, g.stream);
    else
        sakura::launch_prep_step(src, masses, X, nullptr, n, drift, g.d_status, g.stream);
    sakura::StepArgs a;
    a.X = X;
    a.partial = partial;
    a.n = n;
    a.tau = dt;
    a.pre = order == 2 ? 0.5 : (order == 1 ? 0.0 : 1.0);
    a.post = 1.0 - a.pre;
    a.ptau32 = (float)(a.pre * dt);
    a.t32 = (float)dt;
    a.tol = g.cfg.kepler_tol * DBL_EPSILON;
    a.max_iter = g.cfg.kepler_max_iter;
    a.bisection = g.cfg.kepler_bisection;
    a.guess = (g.cfg.guess == SAKURA_GUESS_TAYLOR || g.cfg.guess == SAKURA_GUESS_FP32) ? 2 : 0;
    a.mlp = (g.cfg.guess == SAKURA_GUESS_LEARNED && !mixed)
                ? (const sakura::MlpWeights *)g.mlp.ptr
                : nullptr;
    a.status = g.d_status;
    a.stats = g.d_stats;
    const bool stats = (g.cfg.flags & SAKURA_FLAG_STATS) != 0;
    int64_t W = p.W;
    if (n > 1) {
        const bool timing = (g.cfg.flags & SAKURA_FLAG_TIMING) != 0;
        std::pair<cudaEvent_t, cudaEvent_t> tm{nullptr, nullptr};
        if (timing) {
            tm = take_timer();
            cudaEventRecord(tm.first, g.stream);
        }
        if (mixed) {
            sakura::MixedArgs ma;
            ma.X32 = X32;
            ma.rule = class_rule(a.pre * dt);
            ma.tau32 = (float)dt;
            ma.post32 = (float)a.post;
            sakura::launch_pair_step_mixed(a, ma, p.blocks, stats, g.stream);
        } else {
            sakura::launch_pair_step_fp64(a, p.warps, p.blocks, stats, g.stream);
        }
        if (timing) {
            cudaEventRecord(tm.second, g.stream);
            g.timers.push_back(tm);
        }
    } else {
        W = 0;  // a single particle only drifts
    }
    sakura::launch_apply_step(dst, X, partial, n, W, post_drift, g.d_status, g.stream);
    rc = launch_error();
    if (rc) return rc;
    g.steps += 1;
    g.pairs += n * (n - 1);
    g.solves += n * (n - 1);
    return SAKURA_OK;
}

bool valid_order(int order) { return order == 2 || order == 1 || order == -1; }

bool valid_step_order(int order)
{
    return valid_order(order) || order == 4 || order == 6 || order == 8;
}

// Sub-steps of one step of the given order: the map itself for orders 2, 1
// and -1; for orders 4, 6 and 8 Yoshida's triple jump applied to the order
// below, S_2k(t) = S_2k-2(x1 t) S_2k-2(x0 t) S_2k-2(x1 t) with
// x1 = 1 / (2 - 2^(1/(2k-1))) and x0 = 1 - 2 x1, down to second-order steps
// (the paper's route to higher orders, Sec. 2.2).  Writes the time weights
// (3, 9 or 27 of them) and the order of each sub-step; returns the count.
int substeps(int order, double *w, int *sub_order)
{
    int cnt = 1;
    w[0] = 1.0;
    *sub_order = order;
    if (!(order == 4 || order == 6 || order == 8)) return cnt;
    *sub_order = 2;
    for (int k = 4; k <= order; k += 2) {
        const double c = std::pow(2.0, 1.0 / (double)(k - 1));
        const double x1 = 1.0 / (2.0 - c);
        const double x[3] = {x1, 1.0 - 2.0 * x1, x1};
        double nw[sakura::kMaxSubsteps];
        int m = 0;
        for (int q = 0; q < 3; ++q)
            for (int i = 0; i < cnt; ++i) nw[m++] = x[q] * w[i];
        cnt = m;
        std::memcpy(w, nw, cnt * sizeof(double));
    }
    return cnt;
}

// The device copy of the masses that the last step's drift kernel wrote.
const double *step_masses(int64_t n) { return (const double *)g.partial.ptr + 6 * n; }

// nsteps steps of the given order as one run of sub-steps: the first reads
// src, the last writes dst, the others read and write mid (src, mid and dst
// may be the same buffer).  From the second sub-step on, the masses come
// from the copy that the first drift kernel left in the scratch (same n, so
// the scratch is not reallocated).  On symmetric FP64 tiles every apply
// kernel but the last also drifts for the next sub-step, so only the first
// sub-step runs a prep kernel (the same arithmetic: results are unchanged).
int run_substeps(const double *src, double *mid, double *dst, const double *masses, int64_t n,
                 double dt, int order, int nsteps)
{
    double w[sakura::kMaxSubsteps];
    int so;
    const int cnt = substeps(order, w, &so);
    const int64_t total = (int64_t)cnt * nsteps;
    const bool fuse = fusable(n);
    for (int64_t k = 0; k < total; ++k) {
        const bool last = k == total - 1;
        const double tn = last ? 0.0 : w[(k + 1) % cnt] * dt;
        const double next_drift = so == 2 ? 0.5 * tn : (so == 1 ? 0.0 : tn);  // as the prep
        const int rc = step_device(k == 0 ? src : mid, last ? dst : mid,
                                   k == 0 ? masses : step_masses(n), n, w[k % cnt] * dt, so,
                                   fuse && k > 0, fuse && !last, next_drift);
        if (rc) return rc;
    }
    return SAKURA_OK;
}

// Systems small enough for the single-block kernel (step_small.cu): the FP64
// or double-word form with each unordered pair once and a non-learned guess.
bool small_path(int64_t n)
{
    return n >= 2 && n <= sakura::kSmallMaxN &&
           (g.cfg.precision == SAKURA_PREC_FP64 || g.cfg.precision == SAKURA_PREC_DF64) &&
           g.cfg.pair_mode == SAKURA_PAIRS_SYMMETRIC && g.cfg.guess != SAKURA_GUESS_LEARNED &&
           !(g.cfg.flags & SAKURA_FLAG_NO_SMALL);
}

// nsteps steps of the given order from src to dst in one launch of the
// single-block kernel (src and dst device or mapped host memory).
int step_small(const double *src, double *dst, const double *masses, int64_t n, double dt,
               int order, int nsteps)
{
    sakura::SmallArgs a;
    std::memset(&a, 0, sizeof(a));
    a.src = src;
    a.dst = dst;
    a.mass = masses;
    a.n = (int)n;
    a.nsteps = nsteps;
    int so;
    a.nsub = substeps(order, a.sub, &so);
    a.dt = dt;
    a.drift_frac = so == 2 ? 0.5 : (so == 1 ? 0.0 : 1.0);
    a.post_drift_frac = so == 2 ? 0.5 : (so == 1 ? 1.0 : 0.0);
    a.pre = a.drift_frac;
    a.post = 1.0 - a.pre;
    a.tol = g.cfg.kepler_tol * DBL_EPSILON;
    a.max_iter = g.cfg.kepler_max_iter;
    a.bisection = g.cfg.kepler_bisection;
    const bool dw = g.cfg.precision == SAKURA_PREC_DF64;
    // the double-word form's FP32 phase seeds its own evaluations; its FP64
    // solves (pairs it does not admit) start from the second-order guess
    a.guess = (g.cfg.guess == SAKURA_GUESS_TAYLOR || (dw && g.cfg.guess == SAKURA_GUESS_FP32))
                  ? 2
                  : 0;
    a.status = g.d_status;
    a.stats = g.d_stats;
    const bool timing = (g.cfg.flags & SAKURA_FLAG_TIMING) != 0;
    std::pair<cudaEvent_t, cudaEvent_t> tm{nullptr, nullptr};
    if (timing) {
        tm = take_timer();
        cudaEventRecord(tm.first, g.stream);
    }
    sakura::launch_small(a, (g.cfg.flags & SAKURA_FLAG_STATS) != 0,
                         !dw && g.cfg.guess == SAKURA_GUESS_FP32, dw, g.stream);
    if (timing) {
        cudaEventRecord(tm.second, g.stream);
        g.timers.push_back(tm);
    }
    const int rc = launch_error();
    if (rc) return rc;
    const int64_t subs = (int64_t)nsteps * a.nsub;
    g.steps += subs;
    g.pairs += n * (n - 1) * subs;
    g.solves += n * (n - 1) / 2 * subs;
    return SAKURA_OK;
}

// Device address of a host buffer of `bytes` bytes that is page-locked and
// mapped into the device's address space (cudaHostAlloc, cudaMallocHost or
// cudaHostRegister under unified addressing), checked at its first and last
// byte; null otherwise.
const void *mapped_host(const void *p, size_t bytes)
{
    cudaPointerAttributes a, b;
    const char *last = (const char *)p + bytes - 1;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
        cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer ||
        (const char *)b.devicePointer != (const char *)a.devicePointer + bytes - 1)
        return nullptr;
    return a.devicePointer;
}

}  // namespace

extern "C" {

void sakura_default_config(sakura_config *cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->device = 0;
    cfg->stream = nullptr;
    cfg->precision = SAKURA_PREC_FP64;
    cfg->mixed_rule = SAKURA_MIXED_RULE_LITERAL;
    cfg->mixed_r_min = 0.1;
    cfg->mixed_e_max = 0.9;
    cfg->mixed_e_hyp = 10.0;
    cfg->guess = SAKURA_GUESS_STANDARD;
    cfg->kepler_tol = 4.0;
    cfg->kepler_max_iter = 50;
    cfg->kepler_bisection = 1;
    cfg->flags = 0;
    cfg->block_warps = 0;
    cfg->grid_blocks = 0;
    cfg->pair_mode = SAKURA_PAIRS_SYMMETRIC;
}

int sakura_init(const sakura_config *cfg)
{
    sakura_config c;
    if (cfg)
        c = *cfg;
    else
        sakura_default_config(&c);
    if (c.kepler_max_iter < 1 || c.kepler_max_iter > 10000 || !(c.kepler_tol > 0.0))
        return SAKURA_E_ARG;
    if (c.precision != SAKURA_PREC_FP64 && c.precision != SAKURA_PREC_MIXED &&
        c.precision != SAKURA_PREC_DF64)
        return SAKURA_E_ARG;
    if (c.mixed_rule != SAKURA_MIXED_RULE_LITERAL && c.mixed_rule != SAKURA_MIXED_RULE_HYP)
        return SAKURA_E_ARG;
    if (c.pair_mode != SAKURA_PAIRS_ORDERED && c.pair_mode != SAKURA_PAIRS_SYMMETRIC)
        return SAKURA_E_ARG;
    if (c.guess != SAKURA_GUESS_STANDARD && c.guess != SAKURA_GUESS_LEARNED &&
        c.guess != SAKURA_GUESS_TAYLOR && c.guess != SAKURA_GUESS_FP32)
        return SAKURA_E_ARG;
    if (cudaSetDevice(c.device) != cudaSuccess) {
        cudaGetLastError();
        return SAKURA_E_CUDA;
    }
    if (g.init && g.cfg.device != c.device) sakura_finalize();
    if (!g.init) {
        if (cudaMalloc(&g.d_status, sizeof(unsigned)) != cudaSuccess) return SAKURA_E_NOMEM;
        if (cudaMalloc(&g.d_stats, sakura::kStatCount * sizeof(unsigned long long)) !=
            cudaSuccess)
            return SAKURA_E_NOMEM;
        if (cudaMalloc(&g.d_energy, 3 * sizeof(double)) != cudaSuccess) return SAKURA_E_NOMEM;
        if (cudaMemset(g.d_status, 0, sizeof(unsigned)) != cudaSuccess) return SAKURA_E_CUDA;
        if (cudaHostAlloc(&g.h_status, sizeof(unsigned), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer(&g.h_status_dev, g.h_status, 0) != cudaSuccess)
            return SAKURA_E_NOMEM;
        *g.h_status = 0u;
        if (cudaMemset(g.d_stats, 0, sakura::kStatCount * sizeof(unsigned long long)) !=
            cudaSuccess)
            return SAKURA_E_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device) ==
                cudaSuccess &&
            sms > 0)
            g.sm_count = sms;
        g.steps = g.pairs = g.solves = 0;
    }
    g.cfg = c;
    g.stream = (cudaStream_t)c.stream;
    g.init = true;
    return SAKURA_OK;
}

int sakura_finalize(void)
{
    if (!g.init) return SAKURA_OK;
    cudaStreamSynchronize(g.stream);
    if (g.batch.exec) cudaGraphExecDestroy(g.batch.exec);
    Buffer *bufs[] = {&g.partial,          &g.energy_work,      &g.host_state,
                      &g.host_mass,        &g.batch.task_begin, &g.batch.task_sys,
                      &g.batch.counter,    &g.batch.tune_state, &g.mlp,
                      &g.mlp_blob,         &g.mlp_scratch,      &g.mlp_adam};
    for (Buffer *b : bufs) {
        if (b->ptr) cudaFree(b->ptr);
        b->ptr = nullptr;
        b->bytes = 0;
    }
    cudaFree(g.d_status);
    cudaFree(g.d_stats);
    cudaFree(g.d_energy);
    if (g.h_status) cudaFreeHost(g.h_status);
    for (auto &p : g.timers) g.spare.push_back(p);
    for (auto &p : g.spare) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    g = Context();
    return SAKURA_OK;
}

int sakura_set_stream(void *stream)
{
    if (!g.init) return SAKURA_E_NOINIT;
    g.stream = (cudaStream_t)stream;
    g.cfg.stream = stream;
    return SAKURA_OK;
}

int sakura_step(double *state, const double *masses, int64_t n, double dt, int order)
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (!state || !masses || n < 1 || !valid_step_order(order) || !std::isfinite(dt))
        return SAKURA_E_ARG;
    if (g.cfg.guess == SAKURA_GUESS_LEARNED && !g.mlp_loaded) return SAKURA_E_ARG;
    int rc = small_path(n) ? step_small(state, state, masses, n, dt, order, 1)
                           : run_substeps(state, state, state, masses, n, dt, order, 1);
    if (rc) return rc;
    if (g.cfg.flags & SAKURA_FLAG_SYNC_CHECK) return drain_status();
    return SAKURA_OK;
}

int sakura_evolve(double *state, const double *masses, int64_t n, double dt, int order,
                  int nsteps)
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (!state || !masses || n < 1 || !valid_step_order(order) || !std::isfinite(dt) ||
        nsteps < 0)
        return SAKURA_E_ARG;
    if (g.cfg.guess == SAKURA_GUESS_LEARNED && !g.mlp_loaded) return SAKURA_E_ARG;
    int rc = SAKURA_OK;
    if (nsteps > 0)
        rc = small_path(n) ? step_small(state, state, masses, n, dt, order, nsteps)
                           : run_substeps(state, state, state, masses, n, dt, order, nsteps);
    if (rc) return rc;
    if (g.cfg.flags & SAKURA_FLAG_SYNC_CHECK) return drain_status();
    return SAKURA_OK;
}

int sakura_evolve_host(double *state, const double *masses, int64_t n, double dt, int order,
                       int nsteps)
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (g.cfg.guess == SAKURA_GUESS_LEARNED && !g.mlp_loaded) return SAKURA_E_ARG;
    if (!state || !masses || n < 1 || !valid_step_order(order) || !std::isfinite(dt) ||
        nsteps < 0)
        return SAKURA_E_ARG;
    const size_t sbytes = 6 * (size_t)n * sizeof(double), mbytes = (size_t)n * sizeof(double);
    int rc;
    // page-locked, mapped buffers: the first drift kernel reads the host
    // state and masses and the last apply kernel writes the host state
    // (NVLink-C2C loads and stores), in place of copy-engine transfers
    double *hs = nsteps > 0 ? (double *)mapped_host(state, sbytes) : nullptr;
    const double *hm = hs ? (const double *)mapped_host(masses, mbytes) : nullptr;
    if (hs && hm && small_path(n)) {
        rc = step_small(hs, hs, hm, n, dt, order, nsteps);
        if (rc) return rc;
        return drain_status();
    }
    if (hs && hm) {
        // sub-steps between the first and the last run in library memory
        double w[sakura::kMaxSubsteps];
        int so;
        double *ds = nullptr;
        if ((int64_t)substeps(order, w, &so) * nsteps > 1) {
            rc = grow(g.host_state, sbytes);
            if (rc) return rc;
            ds = (double *)g.host_state.ptr;
        }
        rc = run_substeps(hs, ds, hs, hm, n, dt, order, nsteps);
        if (rc) return rc;
        return drain_status();
    }
    rc = grow(g.host_state, sbytes);
    if (rc) return rc;
    rc = grow(g.host_mass, mbytes);
    if (rc) return rc;
    double *ds = (double *)g.host_state.ptr;
    double *dm = (double *)g.host_mass.ptr;
    if (cudaMemcpyAsync(ds, state, sbytes, cudaMemcpyHostToDevice, g.stream) != cudaSuccess ||
        cudaMemcpyAsync(dm, masses, mbytes, cudaMemcpyHostToDevice, g.stream) != cudaSuccess)
        return SAKURA_E_CUDA;
    if (nsteps > 0) {
        rc = small_path(n) ? step_small(ds, ds, dm, n, dt, order, nsteps)
                           : run_substeps(ds, ds, ds, dm, n, dt, order, nsteps);
        if (rc) return rc;
    }
    if (cudaMemcpyAsync(state, ds, sbytes, cudaMemcpyDeviceToHost, g.stream) != cudaSuccess)
        return SAKURA_E_CUDA;
    return drain_status();
}

int sakura_energy(const double *state, const double *masses, int64_t n, double *E_out)
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (!state || !masses || n < 1 || !E_out) return SAKURA_E_ARG;
    const int nwork = sakura::energy_work_size(n);
    int rc = grow(g.energy_work, (size_t)nwork * sizeof(double));
    if (rc) return rc;
    sakura::launch_energy(state, masses, n, (double *)g.energy_work.ptr, nwork, g.d_energy,
                          g.d_status, g.stream);
    rc = launch_error();
    if (rc) return rc;
    double out[3];
    if (cudaMemcpyAsync(out, g.d_energy, sizeof(out), cudaMemcpyDeviceToHost, g.stream) !=
        cudaSuccess)
        return SAKURA_E_CUDA;
    rc = drain_status();
    *E_out = out[0];
    return rc;
}

int sakura_step_batched(double *state, const double *masses, const int64_t *offsets,
                        const int64_t *host_offsets, int nsys, const double *dt, int order,
                        int nsteps)
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (!state || !masses || !offsets || !host_offsets || !dt || nsys < 1 || nsteps < 0 ||
        !valid_step_order(order))
        return SAKURA_E_ARG;
    if (host_offsets[0] != 0) return SAKURA_E_ARG;
    for (int k = 0; k < nsys; ++k) {
        const int64_t nk = host_offsets[k + 1] - host_offsets[k];
        if (nk < 1 || nk > SAKURA_BATCH_MAX_N) return SAKURA_E_ARG;
    }
    if (nsteps == 0) return SAKURA_OK;
    if (g.cfg.guess == SAKURA_GUESS_LEARNED && !g.mlp_loaded) return SAKURA_E_ARG;
    BatchCache &bc = g.batch;
    int rc;
    const bool new_schedule =
        bc.host_offsets.size() != (size_t)nsys + 1 ||
        !std::equal(bc.host_offsets.begin(), bc.host_offsets.end(), host_offsets);
    if (new_schedule) {
        std::vector<int> tb, ts;
        sakura::build_batch_schedule(host_offsets, nsys, tb, ts);
        if ((rc = grow(bc.task_begin, tb.size() * sizeof(int)))) return rc;
        if ((rc = grow(bc.task_sys, ts.size() * sizeof(int)))) return rc;
        if ((rc = grow(bc.counter, sizeof(int)))) return rc;
        if (cudaMemcpyAsync(bc.task_begin.ptr, tb.data(), tb.size() * sizeof(int),
                            cudaMemcpyHostToDevice, g.stream) != cudaSuccess ||
            cudaMemcpyAsync(bc.task_sys.ptr, ts.data(), ts.size() * sizeof(int),
                            cudaMemcpyHostToDevice, g.stream) != cudaSuccess ||
            cudaStreamSynchronize(g.stream) != cudaSuccess)
            return SAKURA_E_CUDA;
        bc.host_offsets.assign(host_offsets, host_offsets + nsys + 1);
        bc.ntasks = (int)tb.size() - 1;
        bc.tuned = false;
        if (bc.exec) cudaGraphExecDestroy(bc.exec);
        bc.exec = nullptr;
    }
    const int64_t total = host_offsets[nsys];
    const bool stats = (g.cfg.flags & SAKURA_FLAG_STATS) != 0;
    sakura::BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.state = state;
    a.mass = masses;
    a.offsets = offsets;
    a.dt = dt;
    a.task_begin = (const int *)bc.task_begin.ptr;
    a.task_sys = (const int *)bc.task_sys.ptr;
    a.ntasks = bc.ntasks;
    a.counter = (int *)bc.counter.ptr;
    a.total = total;
    a.nsteps = nsteps;
    int so;
    a.nsub = substeps(order, a.sub, &so);
    a.drift_frac = so == 2 ? 0.5 : (so == 1 ? 0.0 : 1.0);
    a.post_drift_frac = so == 2 ? 0.5 : (so == 1 ? 1.0 : 0.0);
    a.pre = a.drift_frac;
    a.post = 1.0 - a.pre;
    a.tol = g.cfg.kepler_tol * DBL_EPSILON;
    a.max_iter = g.cfg.kepler_max_iter;
    a.bisection = g.cfg.kepler_bisection;
    a.guess = (g.cfg.guess == SAKURA_GUESS_TAYLOR || g.cfg.guess == SAKURA_GUESS_FP32) ? 2 : 0;
    a.mlp = g.cfg.guess == SAKURA_GUESS_LEARNED ? (const sakura::MlpWeights *)g.mlp.ptr : nullptr;
    a.seed = g.cfg.guess == SAKURA_GUESS_FP32 ? 1 : 0;
    a.status = g.d_status;
    a.stats = g.d_stats;
    const bool learned = a.mlp != nullptr;
    const bool seed = a.seed != 0;

    // autotune the block shape once per schedule, on a scratch copy
    static const int kCand[4] = {1, 2, 4, 8};
    if (!bc.tuned) {
        bc.warps = g.cfg.block_warps > 0 ? g.cfg.block_warps : 4;
        if (bc.warps != 1 && bc.warps != 2 && bc.warps != 4 && bc.warps != 8) bc.warps = 4;
        bc.blocks = g.cfg.grid_blocks > 0
                        ? g.cfg.grid_blocks
                        : g.sm_count * sakura::batched_blocks_per_sm(bc.warps, stats, learned, seed);
        if (!(g.cfg.flags & SAKURA_FLAG_NO_AUTOTUNE) && g.cfg.block_warps <= 0 &&
            g.cfg.grid_blocks <= 0) {
            if ((rc = grow(bc.tune_state, 6 * (size_t)total * sizeof(double)))) return rc;
            sakura::BatchArgs t = a;
            t.state = (double *)bc.tune_state.ptr;
            t.nsteps = 1;
            t.stats = g.d_stats;
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            double best = 1e300;
            for (int c = 0; c < 4; ++c) {
                const int w = kCand[c];
                const int blocks = g.sm_count * sakura::batched_blocks_per_sm(w, false, learned, seed);
                float ms = 0.f;
                for (int rep = 0; rep < 2; ++rep) {  // first launch warms up
                    cudaMemcpyAsync(t.state, state, 6 * (size_t)total * sizeof(double),
                                    cudaMemcpyDeviceToDevice, g.stream);
                    cudaMemsetAsync(t.counter, 0, sizeof(int), g.stream);
                    cudaEventRecord(e0, g.stream);
                    sakura::launch_batched(t, w, blocks, false, g.stream);
                    cudaEventRecord(e1, g.stream);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&ms, e0, e1);
                }
                bc.tuned_ms[c] = ms;
                if (ms < best) {
                    best = ms;
                    bc.warps = w;
                    bc.blocks = blocks;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (cudaGetLastError() != cudaSuccess) return SAKURA_E_CUDA;
            // the tuning launches touched only the scratch copy; clear their
            // status bits and statistics
            cudaMemsetAsync(g.d_status, 0, sizeof(unsigned), g.stream);
            cudaMemsetAsync(g.d_stats, 0, sakura::kStatCount * sizeof(unsigned long long),
                            g.stream);
        }
        bc.tuned = true;
    }
    // one wave of the kernel variant this call runs (statistics, the network
    // and the float copies change its occupancy), not of the variant that
    // happened to be running when the shape was tuned
    bc.blocks = g.cfg.grid_blocks > 0
                    ? g.cfg.grid_blocks
                    : g.sm_count * sakura::batched_blocks_per_sm(bc.warps, stats, learned, seed);
    // (re)build the graph when anything it captured changed
    const bool same = bc.exec && bc.graph_warps == bc.warps && bc.graph_blocks == bc.blocks &&
                      bc.graph_stats == stats &&
                      std::memcmp(&bc.graph_args, &a, sizeof(a)) == 0;
    if (!same) {
        if (bc.exec) cudaGraphExecDestroy(bc.exec);
        bc.exec = nullptr;
        if (sakura::build_batched_graph(a, bc.warps, bc.blocks, stats, &bc.exec) != cudaSuccess) {
            cudaGetLastError();
            return SAKURA_E_CUDA;
        }
        bc.graph_args = a;
        bc.graph_warps = bc.warps;
        bc.graph_blocks = bc.blocks;
        bc.graph_stats = stats;
    }
    if (cudaGraphLaunch(bc.exec, g.stream) != cudaSuccess) {
        cudaGetLastError();
        return SAKURA_E_CUDA;
    }
    g.steps += (int64_t)nsteps * a.nsub;
    int64_t pairs = 0;
    for (int k = 0; k < nsys; ++k) {
        const int64_t nk = host_offsets[k + 1] - host_offsets[k];
        pairs += nk * (nk - 1);
    }
    // every unordered pair is solved once
    g.pairs += pairs * nsteps * a.nsub;
    g.solves += pairs / 2 * nsteps * a.nsub;
    if (g.cfg.flags & SAKURA_FLAG_SYNC_CHECK) return drain_status();
    return SAKURA_OK;
}

int sakura_batched_tuning(int *warps, int *blocks, double times_ms[4])
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (!g.batch.tuned) return SAKURA_E_ARG;
    if (warps) *warps = g.batch.warps;
    if (blocks) *blocks = g.batch.blocks;
    if (times_ms)
        for (int c = 0; c < 4; ++c) times_ms[c] = g.batch.tuned_ms[c];
    return SAKURA_OK;
}

int sakura_batched_schedule(const int64_t *host_offsets, int nsys, int *task_begin,
                            int *task_sys, int *ntasks)
{
    if (!host_offsets || nsys < 1 || !task_begin || !task_sys || !ntasks) return SAKURA_E_ARG;
    if (host_offsets[0] != 0) return SAKURA_E_ARG;
    for (int k = 0; k < nsys; ++k) {
        const int64_t nk = host_offsets[k + 1] - host_offsets[k];
        if (nk < 1 || nk > SAKURA_BATCH_MAX_N) return SAKURA_E_ARG;
    }
    std::vector<int> tb, ts;
    sakura::build_batch_schedule(host_offsets, nsys, tb, ts);
    *ntasks = (int)tb.size() - 1;
    std::memcpy(task_begin, tb.data(), tb.size() * sizeof(int));
    std::memcpy(task_sys, ts.data(), ts.size() * sizeof(int));
    return SAKURA_OK;
}

int sakura_load_mlp(const void *weights, size_t bytes)
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (!weights || bytes != (size_t)sakura::kMlpBlob * sizeof(float)) return SAKURA_E_ARG;
    const float *w = (const float *)weights;
    for (int k = 0; k < sakura::kMlpBlob; ++k)
        if (!std::isfinite(w[k])) return SAKURA_E_ARG;
    for (int k = 0; k < 6; ++k)
        if (!(w[sakura::kMlpParams + 6 + k] > 0.0f)) return SAKURA_E_ARG;  // input scales
    int rc;
    if ((rc = grow(g.mlp, sizeof(sakura::MlpWeights)))) return rc;
    if ((rc = grow(g.mlp_blob, bytes))) return rc;
    if (cudaMemcpyAsync(g.mlp_blob.ptr, weights, bytes, cudaMemcpyHostToDevice, g.stream) !=
        cudaSuccess)
        return SAKURA_E_CUDA;
    sakura::launch_mlp_pack((const float *)g.mlp_blob.ptr, (sakura::MlpWeights *)g.mlp.ptr,
                            g.stream);
    if (cudaStreamSynchronize(g.stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return SAKURA_E_CUDA;
    g.mlp_loaded = true;
    return SAKURA_OK;
}

int sakura_sample_pairs(const double *state, const double *masses, int64_t n, double dt,
                        int order, const int64_t *pair_ids, int64_t count, float *features,
                        float *targets, int *iters)
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (!state || !masses || !pair_ids || !features || !targets || n < 2 || count < 0 ||
        !valid_order(order) || !std::isfinite(dt))
        return SAKURA_E_ARG;
    if (count == 0) return SAKURA_OK;
    // the drifted state X[7][n] in the head of the step scratch
    int rc = grow(g.partial, (size_t)7 * n * sizeof(double));
    if (rc) return rc;
    double *X = (double *)g.partial.ptr;
    const double drift = order == 2 ? 0.5 * dt : (order == 1 ? 0.0 : dt);
    const double pre = order == 2 ? 0.5 : (order == 1 ? 0.0 : 1.0);
    sakura::launch_prep_step(state, masses, X, nullptr, n, drift, g.d_status, g.stream);
    sakura::launch_sample_pairs(X, n, dt, pre, pair_ids, count, features, targets, iters,
                                g.cfg.kepler_tol * DBL_EPSILON, g.d_status, g.stream);
    if (launch_error()) return SAKURA_E_CUDA;
    return drain_status();
}

int sakura_pair_classes(const double *state, const double *masses, int64_t n, double dt,
                        int order, unsigned char *classes)
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (!state || !masses || !classes || n < 1 || !valid_order(order) || !std::isfinite(dt) ||
        n > (int64_t)1 << 20)
        return SAKURA_E_ARG;
    // X[7][n] doubles and X32[10][n] floats in the head of the step scratch
    int rc = grow(g.partial, (size_t)12 * n * sizeof(double));
    if (rc) return rc;
    double *X = (double *)g.partial.ptr;
    float *X32 = (float *)(X + 7 * n);
    const double drift = order == 2 ? 0.5 * dt : (order == 1 ? 0.0 : dt);
    const double pre = order == 2 ? 0.5 : (order == 1 ? 0.0 : 1.0);
    sakura::launch_prep_mixed(state, masses, X, X32, n, drift, g.d_status, g.stream);
    sakura::launch_pair_classes(X32, n, class_rule(pre * dt), classes, g.stream);
    if (launch_error()) return SAKURA_E_CUDA;
    return drain_status();
}

int sakura_mlp_grad(const float *params, const float *norm, const float *features,
                    const float *targets, int64_t batch, float *grad, float *loss)
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (!params || !norm || !features || !targets || !grad || !loss || batch < 1)
        return SAKURA_E_ARG;
    int rc = grow(g.mlp_scratch, sakura::mlp_grad_scratch_floats(batch) * sizeof(float));
    if (rc) return rc;
    sakura::launch_mlp_grad(params, norm, features, targets, batch, (float *)g.mlp_scratch.ptr,
                            grad, loss, g.stream);
    if (launch_error()) return SAKURA_E_CUDA;
    return cudaStreamSynchronize(g.stream) == cudaSuccess ? SAKURA_OK : SAKURA_E_CUDA;
}

int sakura_mlp_train(float *params, const float *norm, const float *features,
                     const float *targets, int64_t nsamples, int64_t batch, int epochs, float lr,
                     float *losses)
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (!params || !norm || !features || !targets || nsamples < 1 || batch < 1 || epochs < 0 ||
        !(lr > 0.0f))
        return SAKURA_E_ARG;
    batch = std::min(batch, nsamples);
    const int P = sakura::kMlpParams;
    int rc = grow(g.mlp_scratch, sakura::mlp_grad_scratch_floats(batch) * sizeof(float));
    if (rc) return rc;
    if ((rc = grow(g.mlp_adam, (size_t)(3 * P + 1) * sizeof(float)))) return rc;
    float *m = (float *)g.mlp_adam.ptr, *v = m + P, *gr = v + P, *lossbuf = gr + P;
    if (cudaMemsetAsync(m, 0, 2 * P * sizeof(float), g.stream) != cudaSuccess)
        return SAKURA_E_CUDA;
    const int64_t per_epoch = nsamples / batch;
    int64_t t = 0;
    double b1t = 1.0, b2t = 1.0;
    for (int e = 0; e < epochs; ++e) {
        for (int64_t k = 0; k < per_epoch; ++k) {
            const int64_t off = k * batch;
            float *lp = losses ? losses + t : lossbuf;
            sakura::launch_mlp_grad(params, norm, features + off * 6, targets + off, batch,
                                    (float *)g.mlp_scratch.ptr, gr, lp, g.stream);
            ++t;
            b1t *= 0.9;
            b2t *= 0.999;
            sakura::launch_adam(params, m, v, gr, lr, (float)b1t, (float)b2t, g.stream);
        }
    }
    if (launch_error()) return SAKURA_E_CUDA;
    return cudaStreamSynchronize(g.stream) == cudaSuccess ? SAKURA_OK : SAKURA_E_CUDA;
}

int sakura_mlp_eval(const float *features, int64_t count, float *out)
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (!g.mlp_loaded) return SAKURA_E_ARG;
    if (!features || !out || count < 0) return SAKURA_E_ARG;
    if (count == 0) return SAKURA_OK;
    sakura::launch_mlp_eval((const sakura::MlpWeights *)g.mlp.ptr, features, count, out,
                            g.stream);
    if (launch_error()) return SAKURA_E_CUDA;
    return cudaStreamSynchronize(g.stream) == cudaSuccess ? SAKURA_OK : SAKURA_E_CUDA;
}

int sakura_get_stats(sakura_stats *out, int reset)
{
    if (!g.init) return SAKURA_E_NOINIT;
    if (!out) return SAKURA_E_ARG;
    unsigned long long h[sakura::kStatCount];
    if (cudaMemcpyAsync(h, g.d_stats, sizeof(h), cudaMemcpyDeviceToHost, g.stream) !=
        cudaSuccess)
        return SAKURA_E_CUDA;
    if (cudaStreamSynchronize(g.stream) != cudaSuccess) return SAKURA_E_CUDA;
    out->steps = g.steps;
    out->pairs = g.pairs;
    out->solves = g.solves;
    out->iters = (int64_t)h[sakura::kStatIters];
    out->max_iters = (int64_t)h[sakura::kStatMaxIters];
    out->warp_slots = (int64_t)h[sakura::kStatSlots];
    out->fallbacks = (int64_t)h[sakura::kStatFallbacks];
    out->fp32_pairs = (int64_t)h[sakura::kStatFp32Pairs];
    out->carries = (int64_t)h[sakura::kStatCarries];
    collect_timers();
    out->timed_launches = g.timed_launches;
    out->pair_kernel_ms = g.timed_ms;
    out->group_launches = g.group_launches;
    if (reset) {
        if (cudaMemsetAsync(g.d_stats, 0, sizeof(h), g.stream) != cudaSuccess)
            return SAKURA_E_CUDA;
        g.steps = g.pairs = g.solves = 0;
        g.timed_ms = 0.0;
        g.timed_launches = 0;
        g.group_launches = 0;
    }
    return SAKURA_OK;
}

int sakura_check(void)
{
    if (!g.init) return SAKURA_E_NOINIT;
    return drain_status();
}

const char *sakura_strerror(int code)
{
    switch (code) {
    case SAKURA_OK: return "ok";
    case SAKURA_E_NOINIT: return "sakura_init has not been called";
    case SAKURA_E_ARG: return "invalid argument";
    case SAKURA_E_MASS: return "a mass is not positive";
    case SAKURA_E_COINCIDENT: return "two particles coincide (r_ij = 0)";
    case SAKURA_E_NONFINITE: return "non-finite state";
    case SAKURA_E_KEPLER: return "Kepler solver did not converge";
    case SAKURA_E_CUDA: return "CUDA runtime error";
    case SAKURA_E_TIMEOUT: return "bounded device wait ran out";
    case SAKURA_E_NOMEM: return "device allocation failed";
    default: return "unknown error";
    }
}

}  // extern "C"
