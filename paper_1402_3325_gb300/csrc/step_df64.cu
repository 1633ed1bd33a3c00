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
// Row-group form (pair_step_grp_df64_kernel, the default where the tile
//   partials would pass 2 GB): the same pair solves in the row-group phases
//   of the mixed kernel (step_mixed.cu): one block of 12 warps per SM,
//   column sums as double-words in shared memory reduced per window, row
//   sums in registers;
//   the partial sums go out in FP64 (a double-word is a double exactly) to
//   the row-group apply kernel (step_grp.cu).
#include <cuda_runtime.h>

#include "df64.cuh"
#include "kepler_df64.cuh"
#include "kepler_fp64.cuh"
#include "pair_batch_fp64.cuh"
#include "step_common.cuh"
#include "step_grp.cuh"

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

// Row-group form.  A block of kDf64GrpWarps warps takes a group of as many
// row blocks (warp w: row block I = g G + w in layout order, particle
// grp_particle(i)) and sweeps the column blocks J >= g G with them, one
// phase per J, in windows of up to kGrpWindow phases of one group (whole
// phases, grp_layout.cuh).  Column blocks of a window are staged in shared
// memory (20 floats per particle, double buffered); each warp adds its column
// sums of the window as double-words into its own shared-memory
// accumulators, which the block adds in warp order after the window's
// barrier; row sums stay in registers for the whole group.  Pairs the
// double-word solve rejects join the warp's FP64 queue, solved 32 at a time
// and drained at the end of each window.
constexpr int kDf64GrpWin = kGrpWindow;
constexpr size_t kDf64GrpSmem = sizeof(float4) * (kDf64GrpWarps * 3 + 2 * 5) * kDf64GrpWin * 32 +
                                sizeof(int) * 2 * kDf64GrpWarps * 64 +
                                sizeof(float2) * kDf64GrpWarps * 32 * 12;

template <bool STATS>
__global__ void __launch_bounds__(kDf64GrpWarps * 32, 1)
    pair_step_grp_df64_kernel(StepArgs a, DwArgs da, GrpLayout L, GrpParts parts)
{
    constexpr int G = kDf64GrpWarps;
    constexpr int WIN = kDf64GrpWin;
    // dynamic shared memory: the warps' column sums of the window (float4
    // q2 of column block slot cb: components 2 q2 and 2 q2 + 1 as
    // double-words h, l, h, l); the window's column blocks, double buffered
    // (rows 0..19 of X3 as five float4); the FP64 queues and their results
    extern __shared__ __align__(16) unsigned char gsm[];
    float4(*cacc)[WIN][3][32] = reinterpret_cast<float4(*)[WIN][3][32]>(gsm);
    float4(*cx)[WIN][5][32] =
        reinterpret_cast<float4(*)[WIN][5][32]>(gsm + sizeof(float4) * G * WIN * 3 * 32);
    int(*queue_i)[64] =
        reinterpret_cast<int(*)[64]>(gsm + sizeof(float4) * (G * 3 + 2 * 5) * WIN * 32);
    int(*queue_j)[64] = queue_i + G;
    float2(*qres)[32][12] = reinterpret_cast<float2(*)[32][12]>(queue_j + G);
    griddep_wait();    // X and X3 from the prep kernel
    griddep_launch();  // the apply kernel may begin launching
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int tid = threadIdx.x;
    int *qi = queue_i[wib], *qj = queue_j[wib];
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n = a.n;
    const int64_t nb = L.nb;
    const int64_t B = gridDim.x;
    const int64_t b = blockIdx.x;
    const float *X3 = da.X3;
    const KeplerParams kp{a.tol, a.max_iter, a.bisection};
    const int guess = a.guess == 1 ? 2 : a.guess;
    unsigned status = 0;
    long long it_sum = 0, slots = 0, fallbacks = 0, ndw = 0;
    int it_max = 0;

    // the range: whole phases (L.S = 32); its end is block-uniform and kept
    // in shared memory
    GrpPos cur = grp_block_start(L, b, B);
    __shared__ GrpPos s_end;
    if (tid == 0) s_end = grp_block_start(L, b + 1, B);
    __syncthreads();
    auto in_range = [&](const GrpPos &p) {
        const GrpPos e = s_end;
        return p.g < e.g || (p.g == e.g && p.t < e.t);
    };
    auto window_len = [&](const GrpPos &p) {
        const GrpPos e = s_end;
        const int64_t m = p.g < e.g ? nb - p.g * G - p.t : e.t - p.t;
        return (int)(m < WIN ? m : WIN);
    };
    // the window's column blocks Jw .. Jw + len - 1 into cx[buf]
    auto load_cols = [&](int buf, int64_t Jw, int len) {
        for (int e = tid; e < len * 160; e += G * 32) {
            const int cb = e / 160, r = (e >> 5) % 5, c = e & 31;
            const int64_t j = 32 * (Jw + cb) + c;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < n) {
                const int64_t jp = grp_particle(L, n, j);
                v = make_float4(X3[(4 * r) * n + jp], X3[(4 * r + 1) * n + jp],
                                X3[(4 * r + 2) * n + jp], X3[(4 * r + 3) * n + jp]);
            }
            cx[buf][cb][r][c] = v;
        }
    };
    int wl = in_range(cur) ? window_len(cur) : 0;
    if (wl > 0) load_cols(0, cur.g * G + cur.t, wl);
    __syncthreads();

    float xi[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) xi[q] = 0.0f;
    dw mi = {1.0f, 0.0f};
    dw racc[6];
    bool new_group = true;
    int buf = 0;

    // FP64 solve of queue entries 0..cnt-1 (layout indices), all of the
    // current window (column blocks Jw ..); their increments are added in
    // queue order to the row owners' sums and the warp's column sums
    auto flush = [&](int64_t Jw, int cnt) {
        const bool vq = lane < cnt;
        const int64_t iq = vq ? qi[lane] : 0, jq = vq ? qj[lane] : 0;
        PairSolve ps;
        double miq = 0.0, mjq = 0.0;
        if (vq) {
            const double *X = a.X;
            const int64_t ip = grp_particle(L, n, iq), jp = grp_particle(L, n, jq);
            miq = X[6 * n + ip];
            mjq = X[6 * n + jp];
            pair_setup(ps, a.tau, miq + mjq, X[ip] - X[jp], X[n + ip] - X[n + jp],
                       X[2 * n + ip] - X[2 * n + jp], X[3 * n + ip] - X[3 * n + jp],
                       X[4 * n + ip] - X[4 * n + jp], X[5 * n + ip] - X[5 * n + jp], a.pre,
                       guess);
        } else {
            ps.done = true;
            ps.beta = ps.s = 0.0;
            ps.iters = 0;
            ps.status = 0;
        }
        double d[6];
        int iters = 0, fb = 0;
        fp64_solve_warp(ps, vq, a.tau, a.post * a.tau, kp, d, iters, fb);
        if (vq) {
            status |= ps.status;
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const double xr = mjq * d[q], xc = -miq * d[q];
                const float rh = __double2float_rn(xr), ch = __double2float_rn(xc);
                qres[wib][lane][q] = make_float2(rh, __double2float_rn(xr - (double)rh));
                qres[wib][lane][6 + q] = make_float2(ch, __double2float_rn(xc - (double)ch));
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
        for (int e = 0; e < cnt; ++e) {
            const int ie = qi[e], je = qj[e];
            if ((ie & 31) == lane) {
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const float2 x = qres[wib][e][q];
                    dw_acc(racc[q], dw{x.x, x.y});
                }
            }
            // the diagonal tile keeps row sums only
            if ((ie >> 5) != (je >> 5) && (je & 31) == lane) {
                const int cb = (int)((je >> 5) - Jw);
#pragma unroll
                for (int q2 = 0; q2 < 3; ++q2) {
                    const float4 x = cacc[wib][cb][q2][lane];
                    dw a0{x.x, x.y}, a1{x.z, x.w};
                    const float2 y0 = qres[wib][e][6 + 2 * q2], y1 = qres[wib][e][7 + 2 * q2];
                    dw_acc(a0, dw{y0.x, y0.y});
                    dw_acc(a1, dw{y1.x, y1.y});
                    cacc[wib][cb][q2][lane] = make_float4(a0.h, a0.l, a1.h, a1.l);
                }
            }
        }
        __syncwarp();
    };

    while (wl > 0) {
        const int64_t g = cur.g, J = g * G + cur.t;
        const int64_t I = g * G + wib;
        const int64_t i = 32 * I + lane;
        const bool irow = I < nb && i < n;
        if (new_group) {
#pragma unroll
            for (int q = 0; q < 6; ++q) racc[q] = dw{0.0f, 0.0f};
            if (irow) {
                const int64_t ip = grp_particle(L, n, i);
#pragma unroll
                for (int q = 0; q < 18; ++q) xi[q] = X3[q * n + ip];
                mi = {X3[18 * n + ip], X3[19 * n + ip]};
            }
            new_group = false;
        }
        for (int cb = 0; cb < wl; ++cb) {
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2)
                cacc[wib][cb][q2][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        int tail = 0;
        for (int cb = 0; cb < wl; ++cb) {
            const int64_t Jt = J + cb;
            if (!(I <= Jt && I < nb)) continue;  // warp-uniform: no tile (I, Jt)
            const bool diag = I == Jt;
            for (int k = 0; k < 32; ++k) {
                const int c = (lane + k) & 31;
                const int64_t j = 32 * Jt + c;
                const bool valid = irow && j < n && (!diag || c != lane);
                dw rr[3], vv[3], mj = {0.0f, 0.0f};
                K32 o;
                o.ok = false;
                o.x = 0.0f;
                o.s = 0.0f;
                o.iters = 0;
                if (valid) {
                    const float4 c0 = cx[buf][cb][0][c], c1 = cx[buf][cb][1][c],
                                 c2 = cx[buf][cb][2][c], c3 = cx[buf][cb][3][c],
                                 c4 = cx[buf][cb][4][c];
                    const float cj[20] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z,
                                          c1.w, c2.x, c2.y, c2.z, c2.w, c3.x, c3.y,
                                          c3.z, c3.w, c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        rr[q] = tf_diff(xi[3 * q], xi[3 * q + 1], xi[3 * q + 2], cj[3 * q],
                                        cj[3 * q + 1], cj[3 * q + 2]);
                        vv[q] = tf_diff(xi[9 + 3 * q], xi[10 + 3 * q], xi[11 + 3 * q],
                                        cj[9 + 3 * q], cj[10 + 3 * q], cj[11 + 3 * q]);
                    }
                    mj = {cj[18], cj[19]};
                    o = dw_phase1(rr, vv, dw_add(mi, mj), da.ptau32, da.t32, guess);
                }
                const bool big = __any_sync(0xffffffffu, o.ok && fabsf(o.x) > 0x1p-8f);
                bool solved = false;
                int evals = 0;
                dw d[6];
                if (o.ok)
                    solved = dw_phase2(rr, vv, dw_add(mi, mj), da.ptau, da.t, da.qtau, o.s, big,
                                       d, evals);
                if (solved) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) dw_acc(racc[q], dw_mul(mj, d[q]));
                    if (!diag) {
                        const dw nmi = dw_neg(mi);
#pragma unroll
                        for (int q2 = 0; q2 < 3; ++q2) {
                            const float4 x = cacc[wib][cb][q2][c];
                            dw a0{x.x, x.y}, a1{x.z, x.w};
                            dw_acc(a0, dw_mul(nmi, d[2 * q2]));
                            dw_acc(a1, dw_mul(nmi, d[2 * q2 + 1]));
                            cacc[wib][cb][q2][c] = make_float4(a0.h, a0.l, a1.h, a1.l);
                        }
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
                if (need64) {
                    qi[tail + __popc(mask & lt_mask)] = (int)i;
                    qj[tail + __popc(mask & lt_mask)] = (int)j;
                }
                tail += __popc(mask);
                __syncwarp();
                if (tail >= 32) {
                    flush(J, 32);
                    if (lane < tail - 32) {
                        qi[lane] = qi[32 + lane];
                        qj[lane] = qj[32 + lane];
                    }
                    __syncwarp();
                    tail -= 32;
                }
            }
        }
        if (tail > 0) flush(J, tail);
        __syncthreads();  // every warp's column sums of the window are complete
        // the next window; its column blocks are loaded now
        GrpPos nxt{g, cur.t + wl, 0};
        if (nxt.t == nb - g * G) {
            nxt.g = g + 1;
            nxt.t = 0;
        }
        const int wln = in_range(nxt) ? window_len(nxt) : 0;
        if (wln > 0) load_cols(buf ^ 1, nxt.g * G + nxt.t, wln);
        // the window's column partials: the warps' double-words added in
        // warp order, in FP64
        for (int e = tid; e < wl * 192; e += G * 32) {
            const int cb = e / 192, rem = e - cb * 192, c = rem & 31, q = rem >> 5;
            const int64_t j = 32 * (J + cb) + c;
            if (j < n) {
                double sum = 0.0;
#pragma unroll
                for (int w = 0; w < G; ++w) {
                    const float4 x = cacc[w][cb][q >> 1][c];
                    sum += (q & 1) ? ((double)x.z + (double)x.w) : ((double)x.x + (double)x.y);
                }
                parts.col[(g * 6 + q) * n + j] = sum;
            }
        }
        // leaving the group (or the block's range): this piece's row partial
        if (nxt.g != g || wln == 0) {
            if (irow) {
                const int64_t h = b - grp_owner(grp_phase_x(L, g, 0), B, L);
                double *dst = parts.row + h * 6 * n;
#pragma unroll
                for (int q = 0; q < 6; ++q) dst[q * n + i] = (double)racc[q].h + (double)racc[q].l;
            }
            new_group = true;
        }
        __syncthreads();  // the sums are read and the next column blocks stored
        cur = nxt;
        wl = wln;
        buf ^= 1;
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

namespace {

const void *grp_df64_kernel(bool stats)
{
    return stats ? (const void *)pair_step_grp_df64_kernel<true>
                 : (const void *)pair_step_grp_df64_kernel<false>;
}

}  // namespace

int pair_step_grp_df64_blocks_per_sm(bool stats)
{
    const void *fn = grp_df64_kernel(stats);
    int b = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDf64GrpSmem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kDf64GrpWarps * 32, kDf64GrpSmem) !=
            cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return b > 0 ? b : 1;
}

void launch_pair_step_grp_df64(const StepArgs &a, const DwArgs &da, const GrpLayout &L,
                               const GrpParts &parts, int blocks, bool stats, cudaStream_t s)
{
    const void *fn = grp_df64_kernel(stats);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDf64GrpSmem);
    GrpLayout Lv = L;
    GrpParts pv = parts;
    void *args[] = {(void *)&a, (void *)&da, (void *)&Lv, (void *)&pv};
    launch_pdl(fn, dim3(blocks), dim3(kDf64GrpWarps * 32), args, kDf64GrpSmem, s);
}

}  // namespace sakura
