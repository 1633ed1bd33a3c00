// step_small.cu -- one small system, every step of a call in one block.
//
// For n <= kSmallMaxN particles the whole system lives in the shared memory
// of one block, which runs all the steps (and sub-steps) of a call in one
// launch: no kernel boundary, no global-memory round trip between steps.
//
// Each unordered pair is solved once (Newton's third law, as in step_sym.cu):
// the increments of the ordered pairs (i, j) and (j, i) are exact negatives.
// The P = n (n - 1) / 2 pairs (a, b), a < b, are numbered row by row,
//   p(a, b) = a n - a (a + 1) / 2 + b - a - 1,
// and packed densely over the lanes: lane l of chunk c solves pair 32 c + l,
// so a step costs ceil(P / 32) warp-wide solves.  (The FP64 pipe charges a
// warp instruction the same however many lanes are active, so the dense
// packing matters: a round-robin order needs n or n - 1 warp-wide rounds of
// n / 2 active lanes.)  Each lane writes its
// increments divided by m_ab to shared memory; after a block barrier thread
// (i, c) adds particle i's increments in ascending j (+m_j d for the pair
// (i, j), -m_j d for the pair (j, i); Eq. 23 with 1/m_i folded in), a fixed
// order, so the result is deterministic, and applies Eqs. 27b-d.
//
// The block is bound by latency, and an FP64 warp instruction costs about 64
// cycles of issue on GB300 however many of its lanes are active (each of an
// SM's four sub-partitions has a quarter of its FP64 rate; measured: a warp
// running 8 independent chains of FP64 FMAs issues one per 64 cycles).  So
// the block has at least four warps, one per sub-partition, and the
// per-particle work of the drift and the sums is dealt out over all of them
// (element e to lane e / nw of warp e % nw): what counts is the number of
// FP64 instructions each warp issues, not the number of threads.
//
// DW: the double-word form of step_df64.cu for the pair solves (FP32 phase,
// double-word evaluations and carry from the pair's exact double-word
// differences of the three-float split state), with the FP64 solve for the
// lanes whose pair it does not admit.  Its increments are stored as doubles
// (h + l, rounded once), and the sums stay in FP64.  A
// dependent FP32 instruction waits a few cycles where an FP64 one waits
// tens, so the latency of a step, which bounds this kernel, is shorter.
#include <cuda_runtime.h>

#include "kepler_df64.cuh"
#include "kepler_fp64.cuh"
#include "pair_batch_fp64.cuh"
#include "step_common.cuh"
#include "step_small.cuh"

namespace sakura {

// the sign bit of a double, flipped by an integer XOR
constexpr long long kSignBit = (long long)0x8000000000000000ULL;

namespace {

__device__ __forceinline__ dw split_dw(double x)
{
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}

}  // namespace

template <bool STATS, bool SEED, bool DW>
__global__ void __launch_bounds__(32 * kSmallMaxWarps, 1) small_kernel(SmallArgs a)
{
    __shared__ double S[7][kSmallMaxN];
    __shared__ float S32[SEED ? 10 : 1][kSmallMaxN];
    __shared__ float S3[DW ? 20 : 1][kSmallMaxN];  // three-float state, double-word masses
    __shared__ double D[6][kSmallMaxPairs];
    __shared__ unsigned char PA[kSmallMaxPairs], PB[kSmallMaxPairs];
    const int n = a.n;
    const int P = n * (n - 1) / 2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, wib = tid >> 5, nw = nthr >> 5;
    const int ew = lane * nw + wib;  // first per-particle element of this thread
    const KeplerParams kp{a.tol, a.max_iter, a.bisection};
    unsigned status = 0;
    long long it_sum = 0, slots = 0, fallbacks = 0, carries = 0, ndw = 0;
    int it_max = 0;

    for (int i = tid; i < n; i += nthr) {
#pragma unroll
        for (int c = 0; c < 6; ++c) S[c][i] = a.src[c * n + i];
        const double m = a.mass[i];
        if (!(m > 0.0)) status |= kStatusMass;
        S[6][i] = m;
        if (DW) {
            const dw md = split_dw(m);
            S3[18][i] = md.h;
            S3[19][i] = md.l;
        }
        int p = i * n - i * (i + 1) / 2;  // the pairs (i, b), b > i
        for (int b = i + 1; b < n; ++b, ++p) {
            PA[p] = (unsigned char)i;
            PB[p] = (unsigned char)b;
        }
    }
    const double dt = a.dt;
    __syncthreads();
    const int chunks = (P + 31) >> 5;
    for (int64_t sub = 0; sub < (int64_t)a.nsteps * a.nsub; ++sub) {
        // sub-step sub % nsub of the composition (one sub-step for orders 2, 1, -1)
        const double tau = dt * a.sub[(int)(sub % a.nsub)];
        const double drift = a.drift_frac * tau;
        const double post_drift = a.post_drift_frac * tau;
        const double qtau = a.post * tau;
        for (int e = ew; e < 3 * n; e += nthr) {  // Eq. 27a, element (i, c)
            const int c = e / n, i = e - c * n;
            const double x = fma(S[3 + c][i], drift, S[c][i]);
            S[c][i] = x;
            if (SEED) {
                const float hi = __double2float_rn(x);
                S32[c][i] = hi;
                S32[3 + c][i] = __double2float_rn(x - (double)hi);
                S32[6 + c][i] = __double2float_rn(S[3 + c][i]);
                if (c == 0) S32[9][i] = __double2float_rn(S[6][i]);
            }
            if (DW) {
                tf_split(x, S3[3 * c][i], S3[3 * c + 1][i], S3[3 * c + 2][i]);
                tf_split(S[3 + c][i], S3[9 + 3 * c][i], S3[10 + 3 * c][i], S3[11 + 3 * c][i]);
            }
        }
        __syncthreads();
        const float ptau32 = (float)(a.pre * tau), t32 = (float)tau;
        for (int ch = wib; ch < chunks; ch += nw) {
            const int p = 32 * ch + lane;
            const bool valid = p < P;
            const int i = valid ? PA[p] : 0, j = valid ? PB[p] : 0;
            bool need64 = valid;
            if (DW) {
                // the double-word solve of the admitted pairs
                dw rr[3], vv[3], m = {0.0f, 0.0f};
                K32 o;
                o.ok = false;
                o.x = o.s = 0.0f;
                o.iters = 0;
                if (valid) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        rr[q] = tf_diff(S3[3 * q][i], S3[3 * q + 1][i], S3[3 * q + 2][i],
                                        S3[3 * q][j], S3[3 * q + 1][j], S3[3 * q + 2][j]);
                        vv[q] = tf_diff(S3[9 + 3 * q][i], S3[10 + 3 * q][i], S3[11 + 3 * q][i],
                                        S3[9 + 3 * q][j], S3[10 + 3 * q][j], S3[11 + 3 * q][j]);
                    }
                    m = dw_add(dw{S3[18][i], S3[19][i]}, dw{S3[18][j], S3[19][j]});
                    o = dw_phase1(rr, vv, m, ptau32, t32, a.guess);
                }
                const bool big = __any_sync(0xffffffffu, o.ok && fabsf(o.x) > 0x1p-8f);
                dw d[6];
                int evals = 0;
                const bool solved =
                    o.ok && dw_phase2(rr, vv, m, split_dw(a.pre * tau), split_dw(tau),
                                      split_dw(qtau), o.s, big, d, evals);
                if (solved) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) D[q][p] = (double)d[q].h + (double)d[q].l;
                }
                need64 = valid && !solved;
                if (STATS) {
                    const int it = o.iters + evals;
                    it_sum += it;
                    it_max = max(it_max, it);
                    ndw += solved ? 1 : 0;
                    const int wmax = __reduce_max_sync(0xffffffffu, it);
                    if (lane == 0) slots += 32LL * wmax;
                }
                if (!__any_sync(0xffffffffu, need64)) continue;
            }
            PairSolve ps;
            if (need64) {
                K32 o;
                if (SEED) {
                    // single-precision seed: the root of the FP32 solve of the
                    // same pair (unless t is reduced modulo the period)
                    float dr[3], dv[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        dr[c] = __fadd_rn(__fsub_rn(S32[c][i], S32[c][j]),
                                          __fsub_rn(S32[3 + c][i], S32[3 + c][j]));
                        dv[c] = __fsub_rn(S32[6 + c][i], S32[6 + c][j]);
                    }
                    o = k32_phase1(dr, dv, S32[9][i] + S32[9][j], ptau32, t32, 2);
                }
                pair_setup(ps, tau, S[6][i] + S[6][j], S[0][i] - S[0][j], S[1][i] - S[1][j],
                           S[2][i] - S[2][j], S[3][i] - S[3][j], S[4][i] - S[4][j],
                           S[5][i] - S[5][j], a.pre, SEED ? -1 : a.guess);
                if (SEED) {
                    if (o.ok && dbits(ps.t) == dbits(tau) &&
                        !ps.done) {
                        ps.s = f2d(o.s);
                    } else if (!ps.done) {
                        // no usable seed: the second-order guess, as pair_setup
                        // computes it
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
            fp64_solve_warp<SEED>(ps, need64, tau, qtau, kp, d, iters, fb);
            if (need64) {
#pragma unroll
                for (int q = 0; q < 6; ++q) D[q][p] = d[q];
                status |= ps.status;
            }
            if (STATS) {
                carries += (need64 && ps.carried) ? 1 : 0;
                it_sum += iters;
                fallbacks += fb;
                it_max = max(it_max, iters);
                const int wmax = __reduce_max_sync(0xffffffffu, iters);
                if (lane == 0) slots += 32LL * wmax;
            }
        }
        __syncthreads();
        // Eqs. 23 and 27b-d: element (i, c) sums particle i's increments of
        // component c in ascending j (one loop, so the lanes of a warp do not
        // diverge) and updates v_c and x_c
        for (int e = ew; e < 3 * n; e += nthr) {
            const int c = e / n, i = e - c * n;
            double sr = 0.0, sv = 0.0;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                // the pair (j, i) for j < i gives -m_j d, the pair (i, j) +m_j d
                const int lo = min(i, j), hi = max(i, j);
                const int p = lo * n - lo * (lo + 1) / 2 + hi - lo - 1;
                // -m_j as the same bits by an integer XOR of the sign bit
                // (no FP64 instruction)
                const double w = __longlong_as_double(dbits(S[6][j]) ^
                                                      (j < i ? kSignBit : 0LL));
                sr = fma(w, D[c][p], sr);
                sv = fma(w, D[3 + c][p], sv);
            }
            const double v1 = S[3 + c][i] + sv;
            S[c][i] = fma(v1, post_drift, S[c][i] + sr);
            S[3 + c][i] = v1;
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += nthr) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double x = S[c][i];
            if (!isfinite(x)) status |= kStatusNonfinite;
            a.dst[c * n + i] = x;
        }
    }
    status = __reduce_or_sync(0xffffffffu, status);
    if (lane == 0 && status) atomicOr(a.status, status);
    if (STATS) {
        long long s1 = it_sum, s2 = slots, s3 = fallbacks, s4 = carries;
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
            atomicAdd(&a.stats[kStatCarries], (unsigned long long)s4);
            atomicMax(&a.stats[kStatMaxIters], (unsigned long long)mx);
        }
        if (DW) {
            long long s5 = ndw;
            for (int o = 16; o > 0; o >>= 1) s5 += __shfl_xor_sync(0xffffffffu, s5, o);
            if (lane == 0) atomicAdd(&a.stats[kStatFp32Pairs], (unsigned long long)s5);
        }
    }
}

int small_warps(int n)
{
    const int chunks = (n * (n - 1) / 2 + 31) / 32;
    return chunks < 4 ? 4 : (chunks > kSmallMaxWarps ? kSmallMaxWarps : chunks);
}

void launch_small(const SmallArgs &a, bool stats, bool seed, bool dw, cudaStream_t s)
{
    const int threads = 32 * small_warps(a.n);
    if (dw) {
        if (stats)
            small_kernel<true, false, true><<<1, threads, 0, s>>>(a);
        else
            small_kernel<false, false, true><<<1, threads, 0, s>>>(a);
    } else if (seed) {
        if (stats)
            small_kernel<true, true, false><<<1, threads, 0, s>>>(a);
        else
            small_kernel<false, true, false><<<1, threads, 0, s>>>(a);
    } else {
        if (stats)
            small_kernel<true, false, false><<<1, threads, 0, s>>>(a);
        else
            small_kernel<false, false, false><<<1, threads, 0, s>>>(a);
    }
}

}  // namespace sakura
