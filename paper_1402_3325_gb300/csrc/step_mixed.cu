// step_mixed.cu -- mixed-precision W step: distant, weakly perturbing pairs in
// FP32, everything else in FP64, all increments accumulated in FP64.
//
// prep kernel: the drift in FP64 (x + v drift, rounded twice, as a plain CPU
//   loop computes it), the FP64 drifted state X[7][n], and a float copy
//   X32[10][n] = (hi x, y, z, lo x, y, z, vx, vy, vz, m) with x = hi + lo,
//   hi = fl32(x), lo = fl32(x - hi), so FP32 pair differences keep the
//   accuracy of the separation rather than of the coordinate.
// pair kernel: the persistent batch partition of the FP64 kernel.  For each
//   batch every lane forms its pair's FP32 Kepler input and class (class rule
//   in kepler_fp32.cuh); FP32-class lanes solve in FP32 and add
//   m_j * delta/m_ij to the FP64 row accumulators; the other pairs are
//   compacted into a per-warp shared-memory queue and solved 32 at a time by
//   the FP64 batch solver, so a few close pairs never make a whole warp run
//   the FP64 path half-empty.  The queue is drained at every row end.
#include <cuda_runtime.h>

#include "df64.cuh"
#include "kepler_df64.cuh"
#include "kepler_fp32.cuh"
#include "kepler_fp64.cuh"
#include "pair_batch_fp64.cuh"
#include "step_common.cuh"

namespace sakura {

__device__ __host__ __forceinline__ int64_t mixed_owner(int64_t b, int64_t B, int64_t W)
{
    return ((b + 1) * W - 1) / B;
}

__global__ void prep_mixed_kernel(const double *state, const double *mass, double *X, float *X32,
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
        const double x = __dadd_rn(state[q * n + i], __dmul_rn(v, drift));
        const float hi = __double2float_rn(x);
        const float lo = __double2float_rn(__dsub_rn(x, (double)hi));
        X[q * n + i] = x;
        X[(3 + q) * n + i] = v;
        X32[q * n + i] = hi;
        X32[(3 + q) * n + i] = lo;
        X32[(6 + q) * n + i] = __double2float_rn(v);
    }
    X[6 * n + i] = m;
    X32[9 * n + i] = __double2float_rn(m);
}

template <int WARPS, bool STATS>
__global__ void __launch_bounds__(WARPS * 32)
    pair_step_mixed_kernel(StepArgs a, MixedArgs ma)
{
    __shared__ int queue[WARPS][64];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int *qw = queue[wib];
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n = a.n;
    const int64_t nb = (n + 31) >> 5;
    const int64_t B = n * nb;
    const int64_t W = (int64_t)gridDim.x * WARPS;
    const int64_t w = (int64_t)blockIdx.x * WARPS + wib;
    const int64_t b0 = w * B / W;
    const int64_t b1 = (w + 1) * B / W;
    const double *X = a.X;
    const float *X32 = ma.X32;
    const KeplerParams kp{a.tol, a.max_iter, a.bisection};

    unsigned status = 0;
    long long it_sum = 0, slots = 0, fallbacks = 0, n32 = 0;
    int it_max = 0;
    int tail = 0;  // warp-uniform queue length

    int64_t i = b0 / nb;
    int64_t jb = b0 - i * nb;
    double xi = 0, yi = 0, zi = 0, vxi = 0, vyi = 0, vzi = 0, mi = 1;
    float hi_i[3] = {0, 0, 0}, lo_i[3] = {0, 0, 0}, v_i[3] = {0, 0, 0}, mfi = 1.0f;
    auto load_row = [&](int64_t r) {
        xi = X[r];
        yi = X[n + r];
        zi = X[2 * n + r];
        vxi = X[3 * n + r];
        vyi = X[4 * n + r];
        vzi = X[5 * n + r];
        mi = X[6 * n + r];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            hi_i[q] = X32[q * n + r];
            lo_i[q] = X32[(3 + q) * n + r];
            v_i[q] = X32[(6 + q) * n + r];
        }
        mfi = X32[9 * n + r];
    };
    if (b0 < b1) load_row(i);
    double acc[6] = {0, 0, 0, 0, 0, 0};

    auto run_fp64 = [&](int64_t jq, bool vq) {
        int iters = 0, fb = 0;
        fp64_pair_batch(X, n, jq, vq, xi, yi, zi, vxi, vyi, vzi, mi, a, kp, acc, status, iters,
                        fb);
        if (STATS) {
            it_sum += iters;
            fallbacks += fb;
            it_max = max(it_max, iters);
            const int wmax = __reduce_max_sync(0xffffffffu, iters);
            if (lane == 0) slots += 32LL * wmax;
        }
    };

    for (int64_t b = b0; b < b1; ++b) {
        const int64_t j = (jb << 5) + lane;
        const bool valid = (j < n) && (j != i);
        bool solved32 = false;
        if (valid) {
            float hi_j[3], lo_j[3], v_j[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                hi_j[q] = X32[q * n + j];
                lo_j[q] = X32[(3 + q) * n + j];
                v_j[q] = X32[(6 + q) * n + j];
            }
            Pair32 p;
            pair32_setup(p, hi_i, lo_i, v_i, mfi, hi_j, lo_j, v_j, X32[9 * n + j], ma.rule);
            if (p.fp32) {
                float d[6];
                int it32 = 0;
                solved32 = pair32_solve(p, ma.tau32, ma.post32, a.guess, d, it32);
                if (solved32) {
                    const double mj = X[6 * n + j];
#pragma unroll
                    for (int q = 0; q < 6; ++q) acc[q] = fma(mj, (double)d[q], acc[q]);
                }
            }
        }
        if (STATS) n32 += solved32 ? 1 : 0;
        // every other valid pair joins the warp's FP64 queue
        const bool need64 = valid && !solved32;
        const unsigned mask = __ballot_sync(0xffffffffu, need64);
        if (need64) qw[tail + __popc(mask & lt_mask)] = (int)j;
        tail += __popc(mask);
        __syncwarp();
        if (tail >= 32) {
            run_fp64(qw[lane], true);
            __syncwarp();
            if (lane < tail - 32) qw[lane] = qw[32 + lane];
            __syncwarp();
            tail -= 32;
        }
        // leaving row i: drain the queue, reduce and store the row partial
        if (++jb == nb || b + 1 == b1) {
            if (tail > 0) {
                const bool vq = lane < tail;
                run_fp64(vq ? qw[lane] : 0, vq);
                __syncwarp();
                tail = 0;
            }
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                double v = acc[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                acc[q] = 0.0;
                if (lane == 0) {
                    const int64_t k = w - mixed_owner(i * nb, B, W);
                    a.partial[(k * 6 + q) * n + i] = v;
                }
            }
            if (b + 1 < b1) {
                ++i;
                jb = 0;
                load_row(i);
            }
        }
    }
    status = __reduce_or_sync(0xffffffffu, status);
    if (lane == 0 && status) atomicOr(a.status, status);
    if (STATS) {
        long long s1 = it_sum, s2 = slots, s3 = fallbacks, s4 = n32;
        int mx = it_max;
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            s3 += __shfl_xor_sync(0xffffffffu, s3, o);
            s4 += __shfl_xor_sync(0xffffffffu, s4, o);
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            atomicAdd(&a.stats[kStatIters], (unsigned long long)s1);
            atomicAdd(&a.stats[kStatSlots], (unsigned long long)s2);
            atomicAdd(&a.stats[kStatFallbacks], (unsigned long long)s3);
            atomicAdd(&a.stats[kStatFp32Pairs], (unsigned long long)s4);
            atomicMax(&a.stats[kStatMaxIters], (unsigned long long)mx);
        }
    }
}

// Symmetric form: every unordered pair once, on the systolic tiles and
// contiguous tile-step ranges of step_sym.cu (step_common.cuh).  The class
// rule is symmetric in (i, j) (float negation and round-to-nearest are), so
// one decision serves both ordered pairs.  An FP32-class pair's increments
// m_j d and -m_i d (float products, formed exactly by two_prod) are summed in
// double-word form within the tile segment (at most 32 terms, exact to
// 2^-48) and the segment sums go out in FP64, where the apply kernel adds
// them; every other pair joins the per-warp FP64 queue of step_df64.cu.
// 4 blocks per SM (120 registers, no spills): 8.5 % faster on GB300 than the
// 3 that 150 registers allowed
template <bool STATS>
__global__ void __launch_bounds__(128, 4)
    pair_step_sym_mixed_kernel(StepArgs a, MixedArgs ma, int Smax, int64_t T)
{
    // FP64-class pairs wait in a per-warp queue (global i, j) until 32 have
    // collected or the warp's range ends, so that the FP64 solves run with
    // every lane busy: a queue flushed at every segment end ran mostly
    // single-lane solves (13 % of the kernel on GB300).  (Flushing queues of
    // 8 or more at segment ends was slower under both class rules.)
    __shared__ int queue_i[4][64], queue_j[4][64];
    __shared__ float2 qres[4][32][12];  // queued results as double-words
    griddep_wait();    // X and X32 from the prep kernel
    griddep_launch();  // the apply kernel may begin launching
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int *qi = queue_i[wib], *qj = queue_j[wib];
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n = a.n;
    const int64_t W = (int64_t)gridDim.x * 4;
    const int64_t w = (int64_t)blockIdx.x * 4 + wib;
    const float *X32 = ma.X32;
    const KeplerParams kp{a.tol, a.max_iter, a.bisection};
    unsigned status = 0;
    long long it_sum = 0, slots = 0, fallbacks = 0, n32 = 0;
    int it_max = 0;
    int tail = 0;  // queued pairs

    // FP64 solve of queue entries 0..cnt-1.  Entries of the current tile
    // (I, J) at step kc are added to the row owners' and column holders'
    // double-word sums, in queue order; entries of the warp's earlier
    // segments are added to those segments' FP64 partials, which this warp
    // wrote and no other warp touches, in queue order where two entries meet
    // the same element (passes by rank among equal targets).
    auto flush = [&](int64_t I, int64_t J, bool diag, int kc, int cnt, dw racc[6], dw cacc[6]) {
        const bool vq = lane < cnt;
        const int64_t iq = vq ? qi[lane] : 0, jq = vq ? qj[lane] : 0;
        const bool cur = vq && (iq >> 5) == I && (jq >> 5) == J;
        PairSolve p;
        double miq = 0.0, mjq = 0.0;
        if (vq) {
            const double *X = a.X;
            miq = X[6 * n + iq];
            mjq = X[6 * n + jq];
            pair_setup(p, a.tau, miq + mjq, X[iq] - X[jq], X[n + iq] - X[n + jq],
                       X[2 * n + iq] - X[2 * n + jq], X[3 * n + iq] - X[3 * n + jq],
                       X[4 * n + iq] - X[4 * n + jq], X[5 * n + iq] - X[5 * n + jq], a.pre,
                       a.guess);
        } else {
            p.done = true;
            p.beta = p.s = 0.0;
            p.iters = 0;
            p.status = 0;
        }
        double d[6];
        int iters = 0, fb = 0;
        fp64_solve_warp(p, vq, a.tau, a.post * a.tau, kp, d, iters, fb);
        double xr[6], xc[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            xr[q] = mjq * d[q];
            xc[q] = -miq * d[q];
        }
        if (vq) status |= p.status;
        if (cur) {
            // converted to double-words here, with every lane active (the
            // owners below add them one lane at a time)
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const float rh = __double2float_rn(xr[q]), ch = __double2float_rn(xc[q]);
                qres[wib][lane][q] = make_float2(rh, __double2float_rn(xr[q] - (double)rh));
                qres[wib][lane][6 + q] = make_float2(ch, __double2float_rn(xc[q] - (double)ch));
            }
        }
        if (STATS) {
            it_sum += iters;
            fallbacks += fb;
            it_max = max(it_max, iters);
            const int wmax = __reduce_max_sync(0xffffffffu, iters);
            if (lane == 0) slots += 32LL * wmax;
        }
        __syncwarp();
        if (__any_sync(0xffffffffu, cur)) {
            const int mycol = (lane + kc) & 31;
            for (int q = 0; q < cnt; ++q) {
                const int ie = qi[q], je = qj[q];
                if ((ie >> 5) != I || (je >> 5) != J) continue;
                if ((ie & 31) == lane) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        const float2 x = qres[wib][q][c];
                        dw_acc(racc[c], dw{x.x, x.y});
                    }
                }
                if (!diag && (je & 31) == mycol) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        const float2 x = qres[wib][q][6 + c];
                        dw_acc(cacc[c], dw{x.x, x.y});
                    }
                }
            }
        }
        const bool old = vq && !cur;
        if (__any_sync(0xffffffffu, old)) {
            // the entry's tile and this warp's segment of it
            const int64_t Iq = iq >> 5, Jq = jq >> 5;
            const int64_t tq = Jq * (Jq + 1) / 2 + Iq;
            const int64_t hq = old ? w - sym_owner(32 * tq, W, T) : 0;
            const bool dq = Iq == Jq;
            for (int side = 0; side < 2; ++side) {
                const bool act = old && (side == 0 || !dq);
                // target element: slot (other block, segment) of particle
                const int64_t slot = side == 0 ? Jq * Smax + hq : Iq * Smax + hq;
                const int64_t part = side == 0 ? iq : jq;
                const long long key = act ? (long long)(slot * n + part) : -1 - (long long)lane;
                const unsigned same = __match_any_sync(0xffffffffu, key);
                const int rank = __popc(same & lt_mask);
                const int passes = __reduce_max_sync(0xffffffffu, act ? rank : 0);
                for (int pass = 0; pass <= passes; ++pass) {
                    if (act && rank == pass) {
                        double *dst = a.partial + slot * 6 * n + part;
#pragma unroll
                        for (int c = 0; c < 6; ++c)
                            dst[c * n] += side == 0 ? xr[c] : xc[c];
                    }
                    __syncwarp();
                }
            }
        }
        __syncwarp();
    };

    const int64_t p1 = (w + 1) * T / W;
    for (int64_t pos = w * T / W; pos < p1;) {
        const int64_t tile = pos >> 5;
        const int k0 = (int)(pos & 31);
        const int k1 = p1 - pos < 32 - k0 ? k0 + (int)(p1 - pos) : 32;
        const int h = (int)(w - sym_owner(32 * tile, W, T));  // segment of the tile
        pos += k1 - k0;
        int64_t I, J;
        sym_tile_of(tile, I, J);
        const bool diag = I == J;
        const int64_t i = 32 * I + lane;
        const bool irow = i < n;
        float hi_i[3] = {0, 0, 0}, lo_i[3] = {0, 0, 0}, v_i[3] = {0, 0, 0}, mfi = 1.0f;
        if (irow) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                hi_i[q] = X32[q * n + i];
                lo_i[q] = X32[(3 + q) * n + i];
                v_i[q] = X32[(6 + q) * n + i];
            }
            mfi = X32[9 * n + i];
        }
        dw racc[6], cacc[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) racc[q] = cacc[q] = dw{0.0f, 0.0f};

        for (int k = k0; k < k1; ++k) {
            const int c = (lane + k) & 31;
            const int64_t j = 32 * J + c;
            const bool valid = irow && j < n && (!diag || c != lane);
            bool solved32 = false;
            int it32 = 0;
            if (valid) {
                float hi_j[3], lo_j[3], v_j[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    hi_j[q] = X32[q * n + j];
                    lo_j[q] = X32[(3 + q) * n + j];
                    v_j[q] = X32[(6 + q) * n + j];
                }
                const float mfj = X32[9 * n + j];
                Pair32 p;
                pair32_setup(p, hi_i, lo_i, v_i, mfi, hi_j, lo_j, v_j, mfj, ma.rule);
                if (p.fp32) {
                    float d[6];
                    solved32 = pair32_solve(p, ma.tau32, ma.post32, a.guess, d, it32);
                    if (solved32) {
#pragma unroll
                        for (int q = 0; q < 6; ++q) {
                            dw_acc(racc[q], two_prod(mfj, d[q]));
                            dw_acc(cacc[q], two_prod(-mfi, d[q]));
                        }
                    }
                }
            }
            if (STATS) {
                n32 += solved32 ? (diag ? 1 : 2) : 0;  // in ordered pairs
                // single-precision iterations of the FP32-class solves
                const int its = solved32 ? it32 : 0;
                it_sum += its;
                it_max = max(it_max, its);
                const int wmax = __reduce_max_sync(0xffffffffu, its);
                if (lane == 0) slots += 32LL * wmax;
            }
            const bool need64 = valid && !solved32;
            const unsigned mask = __ballot_sync(0xffffffffu, need64);
            if (need64) {
                qi[tail + __popc(mask & lt_mask)] = (int)i;
                qj[tail + __popc(mask & lt_mask)] = (int)j;
            }
            tail += __popc(mask);
            __syncwarp();
            if (tail >= 32) {
                flush(I, J, diag, k, 32, racc, cacc);
                if (lane < tail - 32) {
                    qi[lane] = qi[32 + lane];
                    qj[lane] = qj[32 + lane];
                }
                __syncwarp();
                tail -= 32;
            }
            if (!diag && k + 1 < k1) {
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    cacc[q].h = __shfl_sync(0xffffffffu, cacc[q].h, (lane + 1) & 31);
                    cacc[q].l = __shfl_sync(0xffffffffu, cacc[q].l, (lane + 1) & 31);
                }
            }
        }
        // segment sums in FP64: rows of i to slot (J, h), columns to slot (I, h)
        if (irow) {
            double *dst = a.partial + (J * Smax + h) * 6 * n;
#pragma unroll
            for (int q = 0; q < 6; ++q) dst[q * n + i] = (double)racc[q].h + (double)racc[q].l;
        }
        if (!diag) {
            const int64_t jc = 32 * J + ((lane + k1 - 1) & 31);
            if (jc < n) {
                double *dst = a.partial + (I * Smax + h) * 6 * n;
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    dst[q * n + jc] = (double)cacc[q].h + (double)cacc[q].l;
            }
        }
        __syncwarp();
    }
    // the pairs still queued belong to written segments
    if (tail > 0) {
        dw none[6];
        flush(-1, -1, false, 0, tail, none, none);
    }
    status = __reduce_or_sync(0xffffffffu, status);
    if (lane == 0 && status) atomicOr(a.status, status);
    if (STATS) {
        long long s1 = it_sum, s2 = slots, s3 = fallbacks, s4 = n32;
        int mx = it_max;
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            s3 += __shfl_xor_sync(0xffffffffu, s3, o);
            s4 += __shfl_xor_sync(0xffffffffu, s4, o);
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            atomicAdd(&a.stats[kStatIters], (unsigned long long)s1);
            atomicAdd(&a.stats[kStatSlots], (unsigned long long)s2);
            atomicAdd(&a.stats[kStatFallbacks], (unsigned long long)s3);
            atomicAdd(&a.stats[kStatFp32Pairs], (unsigned long long)s4);
            atomicMax(&a.stats[kStatMaxIters], (unsigned long long)mx);
        }
    }
}

// The class of every ordered pair (i, j) as the mixed kernels decide it
// (pair32_setup on the float copy X32 that prep_mixed_kernel writes): one
// byte per pair, row i, column j, 1 = single precision, diagonal 0.  One
// thread per pair; consecutive threads take consecutive j.
__global__ void pair_class_kernel(const float *X32, int64_t n, ClassRule rule,
                                  unsigned char *out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * n) return;
    const int64_t i = k / n, j = k - i * n;
    unsigned char c = 0;
    if (i != j) {
        float hi_i[3], lo_i[3], v_i[3], hi_j[3], lo_j[3], v_j[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            hi_i[q] = X32[q * n + i];
            lo_i[q] = X32[(3 + q) * n + i];
            v_i[q] = X32[(6 + q) * n + i];
            hi_j[q] = X32[q * n + j];
            lo_j[q] = X32[(3 + q) * n + j];
            v_j[q] = X32[(6 + q) * n + j];
        }
        Pair32 p;
        pair32_setup(p, hi_i, lo_i, v_i, X32[9 * n + i], hi_j, lo_j, v_j, X32[9 * n + j], rule);
        c = p.fp32 ? 1 : 0;
    }
    out[k] = c;
}

void launch_pair_classes(const float *X32, int64_t n, const ClassRule &rule, unsigned char *out,
                         cudaStream_t s)
{
    const int threads = 256;
    const int64_t total = n * n;
    pair_class_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, s>>>(
        X32, n, rule, out);
}

void launch_pair_step_sym_mixed(const StepArgs &a, const MixedArgs &ma, int Smax, int64_t T,
                                int blocks, bool stats, cudaStream_t s)
{
    int Sv = Smax;
    int64_t it = T;
    void *args[] = {(void *)&a, (void *)&ma, (void *)&Sv, (void *)&it};
    launch_pdl(stats ? (const void *)pair_step_sym_mixed_kernel<true>
                     : (const void *)pair_step_sym_mixed_kernel<false>,
               dim3(blocks), dim3(128), args, 0, s);
}

int pair_step_sym_mixed_blocks_per_sm(bool stats)
{
    int b = 0;
    const cudaError_t e =
        stats ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &b, pair_step_sym_mixed_kernel<true>, 128, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &b, pair_step_sym_mixed_kernel<false>, 128, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return b > 0 ? b : 1;
}

void launch_prep_mixed(const double *state, const double *mass, double *X, float *X32,
                       int64_t n, double drift, unsigned *status, cudaStream_t s)
{
    const int threads = 256;
    prep_mixed_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(
        state, mass, X, X32, n, drift, status);
}

void launch_pair_step_mixed(const StepArgs &a, const MixedArgs &ma, int blocks, bool stats,
                            cudaStream_t s)
{
    if (stats)
        pair_step_mixed_kernel<4, true><<<blocks, 128, 0, s>>>(a, ma);
    else
        pair_step_mixed_kernel<4, false><<<blocks, 128, 0, s>>>(a, ma);
}

int pair_step_mixed_blocks_per_sm(bool stats)
{
    int b = 0;
    const cudaError_t e =
        stats ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pair_step_mixed_kernel<4, true>,
                                                              128, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &b, pair_step_mixed_kernel<4, false>, 128, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return b > 0 ? b : 1;
}

}  // namespace sakura
