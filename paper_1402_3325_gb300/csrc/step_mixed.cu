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

#include <algorithm>

#include "df64.cuh"
#include "kepler_df64.cuh"
#include "kepler_fp32.cuh"
#include "kepler_fp64.cuh"
#include "pair_batch_fp64.cuh"
#include "step_common.cuh"
#include "step_grp.cuh"

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

// Symmetric form: every unordered pair once, in row-group phases.
//
// A block of kGrpWarps warps owns a group of kGrpWarps consecutive row blocks
// of 32 particles (warp w: row block I = g kGrpWarps + w).  The block's warps
// sweep the column blocks J >= g kGrpWarps together, one phase per J: in the
// phase, warp w solves the 32 x 32 tile (I, J) (nothing when I > J; the
// ordered pairs of the diagonal tile when I = J) on the systolic schedule of
// step_sym.cu, lane l owning row i = 32 I + l and solving column
// (l + k) mod 32 at step k.  Row sums stay in the lane's registers for the
// whole group; column sums go to the warp's shared-memory accumulators of
// the phase.  The phases of all groups are split into contiguous, equal
// ranges of whole phases over the persistent grid (grp_layout.cuh,
// kMixedGrpShape: whole phases, each of the same cost).  A block takes its
// phases in windows of up to kGrpWindow phases of one group: after each
// window a block barrier, then the block adds the warps' column sums of each
// phase in warp order and writes one column partial per particle of each
// block J; a block writes one row partial per group it meets.  So the
// partial sums written per step are one 6-vector per
// particle per group that covers its column block, plus one per row piece:
// about 30 MB at n = 16384, which stays in L2, against a 6-vector per
// particle per tile segment in the earlier contiguous-range kernel (369 MB).
//
// The class rule is symmetric in (i, j) (float negation and round-to-nearest
// are), so one decision serves both ordered pairs.  An FP32-class pair's
// increments m_j d and -m_i d (float products, formed exactly by two_prod)
// are summed in double-word form within the window (at most 32 terms per
// accumulator and phase, exact to 2^-48); the block's column reduction and
// the row partials go out in FP64, where the apply kernel adds them.  Every
// other pair joins the warp's FP64 queue, solved 32 at a time and drained at
// the end of each window, so every queued pair belongs to the current
// window (drained at every phase, the lone-lane solves before each barrier
// cost 12 % on GB300).

// SEED: the FP64-class pairs start their FP64 iteration from the root of a
// single-precision solve of the same pair and finish by the Taylor carry, as
// in the symmetric FP64 kernel (step_sym.cu); otherwise from a.guess.
constexpr int kGrpWarps = kMixedGrpWarps;

template <bool STATS, bool SEED>
__global__ void __launch_bounds__(kGrpWarps * 32, 2)
    pair_step_grp_mixed_kernel(StepArgs a, MixedArgs ma, GrpLayout L, GrpParts parts)
{
    // dynamic shared memory (grp_smem_bytes): the warps' column sums of the
    // window, float4 q2 of column block slot cb holding components 2 q2 and
    // 2 q2 + 1 as double-words (h, l, h, l); the window's column blocks
    // (double buffered): (hi xyz, m), (lo xyz, 0), (v xyz, 0); the FP64
    // queues and their results
    extern __shared__ __align__(16) unsigned char gsm[];
    float4(*cacc)[kGrpWindow][3][32] = reinterpret_cast<float4(*)[kGrpWindow][3][32]>(gsm);
    float4(*cx)[kGrpWindow][3][32] = reinterpret_cast<float4(*)[kGrpWindow][3][32]>(
        gsm + sizeof(float4) * kGrpWarps * kGrpWindow * 3 * 32);
    int(*queue_i)[64] = reinterpret_cast<int(*)[64]>(
        gsm + sizeof(float4) * (kGrpWarps + 2) * kGrpWindow * 3 * 32);
    int(*queue_j)[64] = queue_i + kGrpWarps;
    float2(*qres)[32][12] = reinterpret_cast<float2(*)[32][12]>(queue_j + kGrpWarps);
    griddep_wait();    // X and X32 from the prep kernel
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
    const float *X32 = ma.X32;
    const KeplerParams kp{a.tol, a.max_iter, a.bisection};
    unsigned status = 0;
    long long it_sum = 0, slots = 0, fallbacks = 0, n32 = 0, carries = 0;
    int it_max = 0;

    // the layout is made with the particles in array order (L.rev = 0):
    // layout indices are particle indices throughout this kernel.
    // the range: whole phases (L.S = 32), so every position has k = 0; its
    // end is block-uniform and kept in shared memory (read once per window)
    // rather than in registers
    GrpPos cur = grp_block_start(L, b, B);
    __shared__ GrpPos s_end;
    if (tid == 0) s_end = grp_block_start(L, b + 1, B);
    __syncthreads();
    auto in_range = [&](const GrpPos &p) {
        const GrpPos e = s_end;
        return p.g < e.g || (p.g == e.g && p.t < e.t);
    };
    // a window: up to kGrpWindow consecutive phases of one group within the
    // block's range
    auto window_len = [&](const GrpPos &p) {
        const GrpPos e = s_end;
        const int64_t m = p.g < e.g ? nb - p.g * kGrpWarps - p.t : e.t - p.t;
        return (int)(m < kGrpWindow ? m : kGrpWindow);
    };
    // the window's column blocks Jw .. Jw + len - 1 into cx[buf]
    auto load_cols = [&](int buf, int64_t Jw, int len) {
        for (int e = tid; e < len * 96; e += kGrpWarps * 32) {
            const int cb = e / 96, r = (e >> 5) % 3, c = e & 31;
            const int64_t j = 32 * (Jw + cb) + c;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < n) {
                if (r == 0)
                    v = make_float4(X32[j], X32[n + j], X32[2 * n + j], X32[9 * n + j]);
                else if (r == 1)
                    v = make_float4(X32[3 * n + j], X32[4 * n + j], X32[5 * n + j], 0.f);
                else
                    v = make_float4(X32[6 * n + j], X32[7 * n + j], X32[8 * n + j], 0.f);
            }
            cx[buf][cb][r][c] = v;
        }
    };
    int wl = in_range(cur) ? window_len(cur) : 0;
    if (wl > 0) load_cols(0, cur.g * kGrpWarps + cur.t, wl);
    __syncthreads();

    float hi_i[3] = {0, 0, 0}, lo_i[3] = {0, 0, 0}, v_i[3] = {0, 0, 0}, mfi = 1.0f;
    dw racc[6];
    bool new_group = true;
    int buf = 0;

    // FP64 solve of queue entries 0..cnt-1, all of the current window (column
    // blocks Jw ..); their increments are added in queue order to the row
    // owners' sums and to the warp's column accumulators of the window
    auto flush = [&](int64_t Jw, int cnt) {
        const bool vq = lane < cnt;
        const int64_t iq = vq ? qi[lane] : 0, jq = vq ? qj[lane] : 0;
        PairSolve ps;
        double miq = 0.0, mjq = 0.0;
        if (vq) {
            const double *X = a.X;
            miq = X[6 * n + iq];
            mjq = X[6 * n + jq];
            pair_setup(ps, a.tau, miq + mjq, X[iq] - X[jq], X[n + iq] - X[n + jq],
                       X[2 * n + iq] - X[2 * n + jq], X[3 * n + iq] - X[3 * n + jq],
                       X[4 * n + iq] - X[4 * n + jq], X[5 * n + iq] - X[5 * n + jq], a.pre,
                       SEED ? -1 : a.guess);
            if (SEED) {
                // the root of the single-precision solve of the pair (unless
                // t was reduced modulo the period), else the second-order guess
                float dr[3], dv[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    dr[q] = __fadd_rn(__fsub_rn(X32[q * n + iq], X32[q * n + jq]),
                                      __fsub_rn(X32[(3 + q) * n + iq], X32[(3 + q) * n + jq]));
                    dv[q] = __fsub_rn(X32[(6 + q) * n + iq], X32[(6 + q) * n + jq]);
                }
                const K32 o = k32_phase1(dr, dv, X32[9 * n + iq] + X32[9 * n + jq], a.ptau32,
                                         a.t32, 2);
                if (o.ok && __double_as_longlong(ps.t) == __double_as_longlong(a.tau) &&
                    !ps.done) {
                    ps.s = f2d(o.s);
                } else if (!ps.done) {
                    ps.s = ps.t * ps.ir0;
                    const double cq = 0.5 * ps.s * (ps.eta0 * ps.ir0);
                    if (magbits(cq) < 0x3fe0000000000000LL) ps.s = fma(-cq, ps.s, ps.s);
                }
            }
        } else {
            ps.done = true;
            ps.beta = ps.s = 0.0;
            ps.iters = 0;
            ps.status = 0;
        }
        double d[6];
        int iters = 0, fb = 0;
        fp64_solve_warp<SEED>(ps, vq, a.tau, a.post * a.tau, kp, d, iters, fb);
        if (vq) {
            status |= ps.status;
            // converted to double-words here, with every lane active
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const double xr = mjq * d[q], xc = -miq * d[q];
                const float rh = __double2float_rn(xr), ch = __double2float_rn(xc);
                qres[wib][lane][q] = make_float2(rh, __double2float_rn(xr - (double)rh));
                qres[wib][lane][6 + q] = make_float2(ch, __double2float_rn(xc - (double)ch));
            }
        }
        if (STATS) {
            carries += (vq && ps.carried) ? 1 : 0;
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
            const bool dg = (ie >> 5) == (je >> 5);
            if (!dg && (je & 31) == lane) {
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
        const int64_t g = cur.g, J = g * kGrpWarps + cur.t;
        const int64_t I = g * kGrpWarps + wib;
        const int64_t i = 32 * I + lane;
        const bool irow = I < nb && i < n;
        if (new_group) {
#pragma unroll
            for (int q = 0; q < 6; ++q) racc[q] = dw{0.0f, 0.0f};
            if (irow) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    hi_i[q] = X32[q * n + i];
                    lo_i[q] = X32[(3 + q) * n + i];
                    v_i[q] = X32[(6 + q) * n + i];
                }
                mfi = X32[9 * n + i];
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
                bool solved32 = false;
                int it32 = 0;
                if (valid) {
                    const float4 c0 = cx[buf][cb][0][c], c1 = cx[buf][cb][1][c],
                                 c2 = cx[buf][cb][2][c];
                    const float hi_j[3] = {c0.x, c0.y, c0.z}, lo_j[3] = {c1.x, c1.y, c1.z},
                                v_j[3] = {c2.x, c2.y, c2.z};
                    const float mfj = c0.w;
                    Pair32 pr;
                    pair32_setup(pr, hi_i, lo_i, v_i, mfi, hi_j, lo_j, v_j, mfj, ma.rule);
                    if (pr.fp32) {
                        float d[6];
                        solved32 = pair32_solve(pr, ma.tau32, ma.post32, a.guess, d, it32);
                        if (solved32) {
#pragma unroll
                            for (int q = 0; q < 6; ++q) dw_acc(racc[q], two_prod(mfj, d[q]));
                            if (!diag) {
#pragma unroll
                                for (int q2 = 0; q2 < 3; ++q2) {
                                    const float4 x = cacc[wib][cb][q2][c];
                                    dw a0{x.x, x.y}, a1{x.z, x.w};
                                    dw_acc(a0, two_prod(-mfi, d[2 * q2]));
                                    dw_acc(a1, two_prod(-mfi, d[2 * q2 + 1]));
                                    cacc[wib][cb][q2][c] = make_float4(a0.h, a0.l, a1.h, a1.l);
                                }
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
        if (nxt.t == nb - g * kGrpWarps) {
            nxt.g = g + 1;
            nxt.t = 0;
        }
        const int wln = in_range(nxt) ? window_len(nxt) : 0;
        if (wln > 0) load_cols(buf ^ 1, nxt.g * kGrpWarps + nxt.t, wln);
        // the window's column partials: the warps' sums added in warp order
        for (int e = tid; e < wl * 192; e += kGrpWarps * 32) {
            const int cb = e / 192, rem = e - cb * 192, c = rem & 31, q = rem >> 5;
            const int64_t j = 32 * (J + cb) + c;
            if (j < n) {
                double sum = 0.0;
#pragma unroll
                for (int w = 0; w < kGrpWarps; ++w) {
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
        long long s1 = it_sum, s2 = slots, s3 = fallbacks, s4 = n32, s5 = carries;
        int mx = it_max;
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            s3 += __shfl_xor_sync(0xffffffffu, s3, o);
            s4 += __shfl_xor_sync(0xffffffffu, s4, o);
            s5 += __shfl_xor_sync(0xffffffffu, s5, o);
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            atomicAdd(&a.stats[kStatIters], (unsigned long long)s1);
            atomicAdd(&a.stats[kStatSlots], (unsigned long long)s2);
            atomicAdd(&a.stats[kStatFallbacks], (unsigned long long)s3);
            atomicAdd(&a.stats[kStatFp32Pairs], (unsigned long long)s4);
            atomicAdd(&a.stats[kStatCarries], (unsigned long long)s5);
            atomicMax(&a.stats[kStatMaxIters], (unsigned long long)mx);
        }
    }
}

// dynamic shared memory of the row-group kernel
constexpr size_t kGrpSmem = sizeof(float4) * (kGrpWarps + 2) * kGrpWindow * 3 * 32 +
                            sizeof(int) * 2 * kGrpWarps * 64 + sizeof(float2) * kGrpWarps * 32 * 12;

const void *grp_kernel(bool stats, bool seed)
{
    if (seed)
        return stats ? (const void *)pair_step_grp_mixed_kernel<true, true>
                     : (const void *)pair_step_grp_mixed_kernel<false, true>;
    return stats ? (const void *)pair_step_grp_mixed_kernel<true, false>
                 : (const void *)pair_step_grp_mixed_kernel<false, false>;
}

void launch_pair_step_grp_mixed(const StepArgs &a, const MixedArgs &ma, const GrpLayout &L,
                                const GrpParts &parts, int blocks, bool stats, cudaStream_t s)
{
    GrpLayout Lv = L;
    GrpParts pv = parts;
    void *args[] = {(void *)&a, (void *)&ma, (void *)&Lv, (void *)&pv};
    const void *fn = grp_kernel(stats, a.X32 != nullptr);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGrpSmem);
    launch_pdl(fn, dim3(blocks), dim3(kGrpWarps * 32), args, kGrpSmem, s);
}

int pair_step_grp_mixed_blocks_per_sm(bool stats, bool seed)
{
    int b = 0;
    const void *fn = grp_kernel(stats, seed);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGrpSmem);
    const cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kGrpWarps * 32, kGrpSmem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return b > 0 ? b : 1;
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
