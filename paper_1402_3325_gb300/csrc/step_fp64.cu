// step_fp64.cu -- FP64 W-step kernels of the Sakura integrator.
//
// One step = prep kernel + pair kernel + apply kernel, on the library stream.
//
// prep kernel: writes the drifted structure-of-arrays X[7][n] = (x, y, z
//   after the one-subscript drift, vx, vy, vz, m) once per step (Eq. 27a or
//   the order-1 forms), so no pair recomputes a drift.
// pair kernel: a persistent launch of one wave of resident warps.  The
//   ordered pairs are cut into B = n * ceil(n/32) batches (row i, 32
//   consecutive j); warp w owns the contiguous batch range [w B / W,
//   (w+1) B / W), so every warp gets the same number of batches (+-1) and
//   crosses a row boundary about ceil(W/n) times at most.  Lane l of a batch
//   solves the pair (i, j = 32 jb + l).  The Laguerre iterations of a batch
//   run warp-synchronously (converged lanes idle; the Stumpff term count is
//   chosen per warp).  Each lane keeps six FP64 accumulators of
//   m_j (delta_r, delta_v) / m_ij = mu_ij (delta_r, delta_v) / m_i (Eq. 23);
//   when the warp leaves a row it reduces them with xor shuffles and lane 0
//   stores the row partial in slot k = w - owner(first batch of row i).  No
//   atomics touch FP64 data.
// apply kernel: sums a row's slots in slot order (deterministic for a given
//   grid) and applies Eqs. 27b-d, or the order-1 forms, in place.
#include <cuda_runtime.h>

#include "kepler_fp64.cuh"
#include "mlp_infer.cuh"
#include "pair_batch_fp64.cuh"
#include "step_common.cuh"

namespace sakura {

// Warp that owns batch b when B batches are split over W warps as
// [w B / W, (w+1) B / W).
__device__ __host__ __forceinline__ int64_t batch_owner(int64_t b, int64_t B, int64_t W)
{
    return ((b + 1) * W - 1) / B;
}

// X[7][n]: drifted positions, velocities, masses.
// X32 (optional): float copy of the drifted state for the single-precision
// seed, positions split x = hi + lo (hi = fl32(x), lo = fl32(x - hi)) so that
// float differences keep the accuracy of the separation
__global__ void prep_step_kernel(const double *state, const double *mass, double *X, float *X32,
                                 int64_t n, double drift, unsigned *status)
{
    griddep_launch();  // the pair kernel may begin launching
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double m = mass[i];
    if (!(m > 0.0)) atomicOr(status, kStatusMass);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double v = state[(3 + q) * n + i];
        const double x = fma(v, drift, state[q * n + i]);
        X[q * n + i] = x;
        X[(3 + q) * n + i] = v;
        if (X32) {
            const float hi = __double2float_rn(x);
            X32[q * n + i] = hi;
            X32[(3 + q) * n + i] = __double2float_rn(x - (double)hi);
            X32[(6 + q) * n + i] = __double2float_rn(v);
        }
    }
    X[6 * n + i] = m;
    if (X32) X32[9 * n + i] = __double2float_rn(m);
}

template <int WARPS, bool STATS, bool LEARNED>
__global__ void __launch_bounds__(WARPS * 32)
    pair_step_fp64_kernel(StepArgs a)
{
    // learned guess: network and per-warp staging in dynamic shared memory
    extern __shared__ __align__(16) unsigned char dsm[];
    MlpWeights *mlpW = reinterpret_cast<MlpWeights *>(dsm);
    __nv_bfloat16 *mlpStage = reinterpret_cast<__nv_bfloat16 *>(dsm + sizeof(MlpWeights));
    if (LEARNED) mlp_load_shared(*mlpW, a.mlp);
    const int lane = threadIdx.x & 31;
    const int64_t n = a.n;
    const int64_t nb = (n + 31) >> 5;
    const int64_t B = n * nb;
    const int64_t W = (int64_t)gridDim.x * WARPS;
    const int64_t w = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    const int64_t b0 = w * B / W;
    const int64_t b1 = (w + 1) * B / W;
    const double *X = a.X;
    const KeplerParams kp{a.tol, a.max_iter, a.bisection};

    unsigned status = 0;
    long long it_sum = 0, slots = 0, fallbacks = 0;
    int it_max = 0;

    int64_t i = b0 / nb;
    int64_t jb = b0 - i * nb;
    double xi = 0, yi = 0, zi = 0, vxi = 0, vyi = 0, vzi = 0, mi = 1;
    if (b0 < b1) {
        xi = X[i];
        yi = X[n + i];
        zi = X[2 * n + i];
        vxi = X[3 * n + i];
        vyi = X[4 * n + i];
        vzi = X[5 * n + i];
        mi = X[6 * n + i];
    }
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t b = b0; b < b1; ++b) {
        const int64_t j = (jb << 5) + lane;
        const bool valid = (j < n) && (j != i);
        int iters = 0, fb = 0;
        if (LEARNED)
            fp64_pair_batch<true>(X, n, j, valid, xi, yi, zi, vxi, vyi, vzi, mi, a, kp, acc,
                                  status, iters, fb, mlpW,
                                  mlpStage + (threadIdx.x >> 5) * 32 * 16);
        else
            fp64_pair_batch<false>(X, n, j, valid, xi, yi, zi, vxi, vyi, vzi, mi, a, kp, acc,
                                   status, iters, fb);
        if (STATS) {
            it_sum += iters;
            fallbacks += fb;
            it_max = max(it_max, iters);
            const int wmax = __reduce_max_sync(0xffffffffu, iters);
            if (lane == 0) slots += 32LL * wmax;
        }
        // leaving row i: reduce and store its partial
        if (++jb == nb || b + 1 == b1) {
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                double v = acc[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                acc[q] = 0.0;
                if (lane == 0) {
                    const int64_t k = w - batch_owner(i * nb, B, W);
                    a.partial[(k * 6 + q) * n + i] = v;
                }
            }
            if (b + 1 < b1) {
                ++i;
                jb = 0;
                xi = X[i];
                yi = X[n + i];
                zi = X[2 * n + i];
                vxi = X[3 * n + i];
                vyi = X[4 * n + i];
                vzi = X[5 * n + i];
                mi = X[6 * n + i];
            }
        }
    }
    status = __reduce_or_sync(0xffffffffu, status);
    if (lane == 0 && status) atomicOr(a.status, status);
    if (STATS) {
        long long s1 = it_sum, s2 = slots, s3 = fallbacks;
        int mx = it_max;
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            s3 += __shfl_xor_sync(0xffffffffu, s3, o);
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            atomicAdd(&a.stats[kStatIters], (unsigned long long)s1);
            atomicAdd(&a.stats[kStatSlots], (unsigned long long)s2);
            atomicAdd(&a.stats[kStatFallbacks], (unsigned long long)s3);
            atomicMax(&a.stats[kStatMaxIters], (unsigned long long)mx);
        }
    }
}

// Eqs. 27b-d (order 2) and the first-order forms.  The slots of row i hold
// sum_j m_j delta_ij / m_ij = sum_j mu_ij delta_ij / m_i (Eq. 23) split by
// warp; they are added in slot order.  Positions come from X (after the
// first drift), so  x_new = X_pos + dr + post_drift * v_new.
__global__ void apply_step_kernel(double *state, const double *X, const double *partial,
                                  int64_t n, int64_t W, double post_drift, unsigned *status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d[6] = {0, 0, 0, 0, 0, 0};
    if (W > 0) {
        const int64_t nb = (n + 31) >> 5;
        const int64_t B = n * nb;
        const int64_t k1 = batch_owner((i + 1) * nb - 1, B, W) - batch_owner(i * nb, B, W);
        for (int64_t k = 0; k <= k1; ++k) {
#pragma unroll
            for (int q = 0; q < 6; ++q) d[q] += partial[(k * 6 + q) * n + i];
        }
    }
    unsigned st = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double v1 = X[(3 + q) * n + i] + d[3 + q];   // 27c
        const double xt = X[q * n + i] + d[q];             // 27b
        const double x1 = fma(v1, post_drift, xt);         // 27d
        if (!isfinite(x1) || !isfinite(v1)) st |= kStatusNonfinite;
        state[q * n + i] = x1;
        state[(3 + q) * n + i] = v1;
    }
    if (st) atomicOr(status, st);
}

int pair_step_slots(int64_t n, int64_t W)
{
    return (int)((W + n - 1) / n + 1);
}

void launch_prep_step(const double *state, const double *mass, double *X, float *X32, int64_t n,
                      double drift, unsigned *status, cudaStream_t s)
{
    const int threads = 64;  // small blocks spread a small n over many SMs
    prep_step_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(
        state, mass, X, X32, n, drift, status);
}

namespace {

template <int W>
const void *fp64_kernel_ptr(bool stats, bool learned)
{
    if (learned)
        return stats ? (const void *)pair_step_fp64_kernel<W, true, true>
                     : (const void *)pair_step_fp64_kernel<W, false, true>;
    return stats ? (const void *)pair_step_fp64_kernel<W, true, false>
                 : (const void *)pair_step_fp64_kernel<W, false, false>;
}

const void *fp64_kernel(int warps, bool stats, bool learned)
{
    switch (warps) {
    case 8: return fp64_kernel_ptr<8>(stats, learned);
    case 16: return fp64_kernel_ptr<16>(stats, learned);
    default: return fp64_kernel_ptr<4>(stats, learned);
    }
}

}  // namespace

size_t learned_smem(int warps) { return sizeof(MlpWeights) + (size_t)warps * 32 * 16 * 2; }

void launch_pair_step_fp64(const StepArgs &a, int warps, int blocks, bool stats,
                           cudaStream_t s)
{
    if (warps != 8 && warps != 16) warps = 4;
    const bool learned = a.mlp != nullptr;
    void *args[] = {(void *)&a};
    cudaLaunchKernel(fp64_kernel(warps, stats, learned), dim3(blocks), dim3(warps * 32), args,
                     learned ? learned_smem(warps) : 0, s);
}

int pair_step_fp64_blocks_per_sm(int warps, bool stats, bool learned)
{
    if (warps != 8 && warps != 16) warps = 4;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fp64_kernel(warps, stats, learned),
                                                      warps * 32,
                                                      learned ? learned_smem(warps) : 0) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return b > 0 ? b : 1;
}

void launch_apply_step(double *state, const double *X, const double *partial, int64_t n,
                       int64_t W, double post_drift, unsigned *status, cudaStream_t s)
{
    const int threads = 256;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    apply_step_kernel<<<blocks, threads, 0, s>>>(state, X, partial, n, W, post_drift, status);
}

}  // namespace sakura
