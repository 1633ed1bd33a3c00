// step_df64.cu -- the W step with every unordered pair solved once (Newton's
// third law, as step_sym.cu) and the Kepler solves done in double-word
// arithmetic on the FP32 pipe (kepler_df64.cuh), to FP64 accuracy.
//
// prep kernel: the FP64 drift of Eq. 27a (as prep_step_kernel), the FP64
//   drifted state X[7][n] and its exact three-float form X3[20][n]
//   (rows 3q..3q+2: component q of x, y, z, vx, vy, vz split as d0 + d1 + d2;
//   rows 18, 19: the mass as a double-word).
// pair kernel: the systolic 32 x 32 tiles of step_sym.cu.  Each lane forms
//   its pair's exact double-word differences (tf_diff), runs the FP32 phase
//   and class test, and the admitted lanes run the double-word phase; the
//   row and column sums are kept as renormalised double-words.  A pair the
//   class test rejects (or whose double-word phase does not converge) joins
//   a per-warp shared-memory queue that is solved 32 at a time by the FP64
//   batch solver; each result is added to its row owner and to the lane that
//   holds its column at that moment, in queue order (deterministic).
//   Partial sums go out as double-words (float2) to the slots of step_sym.cu
//   (contiguous tile-step ranges per warp, step_common.cuh).
// apply kernel: Eqs. 27b-d with the slots added in double-word arithmetic
//   and converted to FP64 once per particle.
#include <cuda_runtime.h>

#include "df64.cuh"
#include "kepler_df64.cuh"
#include "kepler_fp64.cuh"
#include "pair_batch_fp64.cuh"
#include "step_common.cuh"

namespace sakura {

// one thread per (particle, component): blockIdx.y = 0..5 for x, y, z, vx,
// vy, vz, 6 for the mass
__global__ void prep_df64_kernel(const double *state, const double *mass, double *X, float *X3,
                                 int64_t n, double drift, unsigned *status)
{
    griddep_launch();  // the pair kernel may begin launching
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (i >= n) return;
    if (q == 6) {
        const double m = mass[i];
        if (!(m > 0.0)) atomicOr(status, kStatusMass);
        X[6 * n + i] = m;
        const float mh = __double2float_rn(m);
        X3[18 * n + i] = mh;
        X3[19 * n + i] = __double2float_rn(m - (double)mh);
        return;
    }
    const double x = q < 3 ? fma(state[(3 + q) * n + i], drift, state[q * n + i])
                           : state[q * n + i];
    X[q * n + i] = x;
    float d0, d1, d2;
    tf_split(x, d0, d1, d2);
    X3[(3 * q) * n + i] = d0;
    X3[(3 * q + 1) * n + i] = d1;
    X3[(3 * q + 2) * n + i] = d2;
}

// FP64 solve of queue entries 0..cnt-1 of tile (I, J): the results are
// converted to double-words here, with every lane active, into qres[lane]
// (the owners then add them one lane at a time).  Kept out of line so that
// the double-word hot loop's code stays small: 1.6-2.7 % faster on GB300.
__device__ __noinline__ void df64_queue_solve(const StepArgs &a, const int *qw, int cnt,
                                              int64_t I, int64_t J, int guess,
                                              float2 (*qres)[12], unsigned *status,
                                              int *iters_out, int *fb_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t n = a.n;
    const KeplerParams kp{a.tol, a.max_iter, a.bisection};
    const bool vq = lane < cnt;
    const int e = vq ? qw[lane] : 0;
    const int64_t iq = 32 * I + (e & 31), jq = 32 * J + (e >> 5);
    PairSolve p;
    double miq = 0.0, mjq = 0.0;
    if (vq) {
        const double *X = a.X;
        miq = X[6 * n + iq];
        mjq = X[6 * n + jq];
        pair_setup(p, a.tau, miq + mjq, X[iq] - X[jq], X[n + iq] - X[n + jq],
                   X[2 * n + iq] - X[2 * n + jq], X[3 * n + iq] - X[3 * n + jq],
                   X[4 * n + iq] - X[4 * n + jq], X[5 * n + iq] - X[5 * n + jq], a.pre, guess);
    } else {
        p.done = true;
        p.beta = p.s = 0.0;
        p.iters = 0;
        p.status = 0;
    }
    double d[6];
    int iters = 0, fb = 0;
    fp64_solve_warp(p, vq, a.tau, a.post * a.tau, kp, d, iters, fb);
    if (vq) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const double xr = mjq * d[q], xc = -miq * d[q];
            const float rh = __double2float_rn(xr), ch = __double2float_rn(xc);
            qres[lane][q] = make_float2(rh, __double2float_rn(xr - (double)rh));
            qres[lane][6 + q] = make_float2(ch, __double2float_rn(xc - (double)ch));
        }
        *status |= p.status;
    }
    *iters_out = iters;
    *fb_out = fb;
}

template <bool STATS>
__global__ void __launch_bounds__(128)
    pair_step_sym_df64_kernel(StepArgs a, DwArgs da, int Smax, int64_t T)
{
    __shared__ int queue[4][64];
    __shared__ float2 qres[4][32][12];  // queued results as double-words
    griddep_wait();    // X and X3 from the prep kernel
    griddep_launch();  // the apply kernel may begin launching
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int *qw = queue[wib];
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n = a.n;
    const int64_t W = (int64_t)gridDim.x * 4;
    const int64_t w = (int64_t)blockIdx.x * 4 + wib;
    const float *X3 = da.X3;
    const int guess = a.guess == 1 ? 2 : a.guess;
    unsigned status = 0;
    long long it_sum = 0, slots = 0, fallbacks = 0, ndw = 0;
    int it_max = 0;

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
        float xi[18];
        dw mi = {1.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < 18; ++q) xi[q] = irow ? X3[q * n + i] : 0.0f;
        if (irow) mi = {X3[18 * n + i], X3[19 * n + i]};
        dw racc[6], cacc[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) racc[q] = cacc[q] = dw{0.0f, 0.0f};
        int tail = 0;

        // FP64 solve of queue entries 0..cnt-1 at step kc, results added to
        // the row owners and the lanes holding the columns, in queue order
        auto flush = [&](int kc, int cnt) {
            int iters = 0, fb = 0;
            df64_queue_solve(a, qw, cnt, I, J, guess, qres[wib], &status, &iters, &fb);
            if (STATS) {
                it_sum += iters;
                fallbacks += fb;
                it_max = max(it_max, iters);
                const int wmax = __reduce_max_sync(0xffffffffu, iters);
                if (lane == 0) slots += 32LL * wmax;
            }
            __syncwarp();
            const int mycol = (lane + kc) & 31;
            for (int q = 0; q < cnt; ++q) {
                const int eq = qw[q];
                if ((eq & 31) == lane) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        const float2 x = qres[wib][q][c];
                        dw_acc(racc[c], dw{x.x, x.y});
                    }
                }
                if (!diag && (eq >> 5) == mycol) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        const float2 x = qres[wib][q][6 + c];
                        dw_acc(cacc[c], dw{x.x, x.y});
                    }
                }
            }
            __syncwarp();
        };

        for (int k = k0; k < k1; ++k) {
            const int c = (lane + k) & 31;
            const int64_t j = 32 * J + c;
            const bool valid = irow && j < n && (!diag || c != lane);
            dw rr[3], vv[3], mj = {0.0f, 0.0f};
            K32 o;
            o.ok = false;
            o.x = 0.0f;
            o.s = 0.0f;
            o.iters = 0;
            if (valid) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    rr[q] = tf_diff(xi[3 * q], xi[3 * q + 1], xi[3 * q + 2], X3[(3 * q) * n + j],
                                    X3[(3 * q + 1) * n + j], X3[(3 * q + 2) * n + j]);
                    vv[q] = tf_diff(xi[9 + 3 * q], xi[10 + 3 * q], xi[11 + 3 * q],
                                    X3[(9 + 3 * q) * n + j], X3[(10 + 3 * q) * n + j],
                                    X3[(11 + 3 * q) * n + j]);
                }
                mj = {X3[18 * n + j], X3[19 * n + j]};
                o = dw_phase1(rr, vv, dw_add(mi, mj), da.ptau32, da.t32, guess);
            }
            const bool big = __any_sync(0xffffffffu, o.ok && fabsf(o.x) > 0x1p-8f);
            bool solved = false;
            int evals = 0;
            dw d[6];
            if (o.ok)
                solved = dw_phase2(rr, vv, dw_add(mi, mj), da.ptau, da.t, da.qtau, o.s, big, d,
                                   evals);
            if (solved) {
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    dw_acc(racc[q], dw_mul(mj, d[q]));
                    dw_acc(cacc[q], dw_mul(dw_neg(mi), d[q]));
                }
            }
            if (STATS) {
                const int it = o.iters + evals;
                it_sum += it;
                it_max = max(it_max, it);
                ndw += solved ? 1 : 0;
                const int wmax = __reduce_max_sync(0xffffffffu, it);
                if (lane == 0) slots += 32LL * wmax;
            }
            const bool need64 = valid && !solved;
            const unsigned mask = __ballot_sync(0xffffffffu, need64);
            if (need64) qw[tail + __popc(mask & lt_mask)] = lane | (c << 5);
            tail += __popc(mask);
            __syncwarp();
            // solve the queue 32 at a time, and drain it at the item's last
            // step (one call site keeps the FP64 solver's code single)
            while (tail >= 32 || (k + 1 == k1 && tail > 0)) {
                const int cnt = min(tail, 32);
                flush(k, cnt);
                if (lane < tail - cnt) qw[lane] = qw[cnt + lane];
                __syncwarp();
                tail -= cnt;
            }
            if (!diag && k + 1 < k1) {
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    cacc[q].h = __shfl_sync(0xffffffffu, cacc[q].h, (lane + 1) & 31);
                    cacc[q].l = __shfl_sync(0xffffffffu, cacc[q].l, (lane + 1) & 31);
                }
            }
        }
        // row sums of rows i to slot (J, h); column sums to slot (I, h)
        float2 *part = reinterpret_cast<float2 *>(a.partial);
        if (irow) {
            float2 *dst = part + (J * Smax + h) * 6 * n;
#pragma unroll
            for (int q = 0; q < 6; ++q) dst[q * n + i] = make_float2(racc[q].h, racc[q].l);
        }
        if (!diag) {
            const int64_t jc = 32 * J + ((lane + k1 - 1) & 31);
            if (jc < n) {
                float2 *dst = part + (I * Smax + h) * 6 * n;
#pragma unroll
                for (int q = 0; q < 6; ++q) dst[q * n + jc] = make_float2(cacc[q].h, cacc[q].l);
            }
        }
    }
    status = __reduce_or_sync(0xffffffffu, status);
    if (lane == 0 && status) atomicOr(a.status, status);
    if (STATS) {
        long long s1 = it_sum, s2 = slots, s3 = fallbacks, s4 = ndw;
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

// Eqs. 27b-d: block (x, y) takes 32 particles (one per lane) and the
// component pair (y, 3 + y); its kApplyDwWarps warps add the existing
// double-word slots of the other blocks Q = w, w + kApplyDwWarps, ... of
// those particles, warp 0 adds the warps' sums in warp order, converts to
// FP64 and applies the update.
constexpr int kApplyDwWarps = 16;

__global__ void __launch_bounds__(32 * kApplyDwWarps)
    apply_df64_kernel(double *state, const double *X, const float2 *partial, int64_t n, int Smax,
                      int64_t W, int64_t T, double post_drift, unsigned *status)
{
    __shared__ float2 red[kApplyDwWarps][2][32];
    griddep_wait();  // the pair kernel's partials
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int q = blockIdx.y;
    const int64_t P = blockIdx.x;
    const int64_t i = P * 32 + lane;
    const int64_t nb = (n + 31) >> 5;
    dw dr = {0.0f, 0.0f}, dv = {0.0f, 0.0f};
    if (i < n) {
        // slot k = Q Smax + o holds the segment o of the tile of blocks P, Q
        for (int64_t Q = wid; Q < nb; Q += kApplyDwWarps) {
            const int64_t tile = P <= Q ? Q * (Q + 1) / 2 + P : P * (P + 1) / 2 + Q;
            const int segs = sym_segments(tile, W, T);
            for (int o = 0; o < segs; ++o) {
                const int64_t k = Q * Smax + o;
                const float2 a0 = partial[(k * 6 + q) * n + i];
                const float2 b0 = partial[(k * 6 + 3 + q) * n + i];
                dw_acc(dr, dw{a0.x, a0.y});
                dw_acc(dv, dw{b0.x, b0.y});
            }
        }
    }
    red[wid][0][lane] = make_float2(dr.h, dr.l);
    red[wid][1][lane] = make_float2(dv.h, dv.l);
    __syncthreads();
    if (wid != 0 || i >= n) return;
    dw tr = {red[0][0][lane].x, red[0][0][lane].y};
    dw tv = {red[0][1][lane].x, red[0][1][lane].y};
    for (int w = 1; w < kApplyDwWarps; ++w) {
        tr = dw_add(tr, dw{red[w][0][lane].x, red[w][0][lane].y});
        tv = dw_add(tv, dw{red[w][1][lane].x, red[w][1][lane].y});
    }
    const double v1 = X[(3 + q) * n + i] + ((double)tv.h + (double)tv.l);
    const double x1 = fma(v1, post_drift, X[q * n + i] + ((double)tr.h + (double)tr.l));
    if (!isfinite(x1) || !isfinite(v1)) atomicOr(status, kStatusNonfinite);
    state[q * n + i] = x1;
    state[(3 + q) * n + i] = v1;
}

namespace {

const void *df64_kernel(bool stats)
{
    return stats ? (const void *)pair_step_sym_df64_kernel<true>
                 : (const void *)pair_step_sym_df64_kernel<false>;
}

}  // namespace

int pair_step_df64_blocks_per_sm(bool stats)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, df64_kernel(stats), 128, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return b > 0 ? b : 1;
}

void launch_prep_df64(const double *state, const double *mass, double *X, float *X3, int64_t n,
                      double drift, unsigned *status, cudaStream_t s)
{
    const int threads = 64;
    prep_df64_kernel<<<dim3((unsigned)((n + threads - 1) / threads), 7), threads, 0, s>>>(
        state, mass, X, X3, n, drift, status);
}

void launch_pair_step_df64(const StepArgs &a, const DwArgs &da, int Smax, int64_t T, int blocks,
                           bool stats, cudaStream_t s)
{
    int Sv = Smax;
    int64_t it = T;
    void *args[] = {(void *)&a, (void *)&da, (void *)&Sv, (void *)&it};
    launch_pdl(df64_kernel(stats), dim3(blocks), dim3(128), args, 0, s);
}

void launch_apply_df64(double *state, const double *X, const void *partial, int64_t n, int Smax,
                       int64_t W, int64_t T, double post_drift, unsigned *status, cudaStream_t s)
{
    const float2 *part = reinterpret_cast<const float2 *>(partial);
    void *args[] = {(void *)&state, (void *)&X,    (void *)&part,       (void *)&n,
                    (void *)&Smax,  (void *)&W,    (void *)&T,          (void *)&post_drift,
                    (void *)&status};
    launch_pdl((const void *)apply_df64_kernel, dim3((unsigned)((n + 31) / 32), 3),
               dim3(32 * kApplyDwWarps), args, 0, s);
}

}  // namespace sakura
