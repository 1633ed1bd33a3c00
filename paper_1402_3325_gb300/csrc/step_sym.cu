// step_sym.cu -- FP64 W step solving every unordered pair once (Newton's third
// law, which the paper leaves to future implementations, Sec. 2.1).
//
// The increments of the ordered pairs (i, j) and (j, i) are exact negatives
// of each other: every scalar of the solve (r0^2, eta0 = r0.v0, v0^2, beta,
// zeta0, s, G_k) is unchanged when (r0, v0) -> (-r0, -v0), IEEE negation and
// round-to-nearest are symmetric, and the increments are linear in (r0, v0).
// So each pair is solved once and adds  m_j delta/m_ij  to particle i and
// -m_i delta/m_ij  to particle j (Eq. 23 with 1/m_i folded in).
//
// Work: 32 x 32 tiles (row block I, column block J), I <= J; each warp takes
// a contiguous range of tile-steps (step_common.cuh).  Lane l owns row
// i = 32 I + l; at step k it solves the pair with column c = (l + k) mod 32,
// so the 32 lanes always hold 32 different columns.  Row sums stay in the
// lane; column sums travel with their column: after each step every lane
// takes the column accumulator of lane l + 1 (warp shuffle), so the
// accumulator of column (l + k) mod 32 is in lane l at step k.  Diagonal tiles
// (I = J) solve their ordered pairs (i != j) and keep only row sums.
// Partials go to part[slot][6][n] with slot = other_block * Smax + segment:
// the row sums of tile (I, J) to slot (J, h) of the rows, the column sums to
// slot (I, h) of the columns.  Every existing (slot, particle) is written
// exactly once and the apply kernel adds a particle's existing slots in a
// fixed order (deterministic, no atomics).
#include <cuda_runtime.h>

#include "kepler_df64.cuh"
#include "kepler_fp64.cuh"
#include "mlp_infer.cuh"
#include "pair_batch_fp64.cuh"
#include "step_common.cuh"

namespace sakura {

// The FP64 operations formed on the integer pipes (kepler_fp64.cuh), per
// initial guess, as measured on Plummer spheres of 1024 to 8192 bodies and
// the black-hole cluster of 12288: with the seed, 3 blocks per SM (ptxas
// fits the kernel in 143 registers) and the increments', the setup's and
// the iterations' multiplies (3 % faster at 1024 bodies, 13-15 % from 2048
// up, against 2 blocks and none; 3 blocks and none alone were 1 % slower);
// with the learned guess 3 blocks and none (2 % faster at 4096; the
// increments' multiplies were 5 % slower); with the standard guess the
// increments' and the iterations' multiplies (13 % and 16 % faster at 1024
// and 4096 bodies).  The inline class test (2 blocks per SM) moves none: with
// the seed's set its Plummer-1024 line fell from 8.62e9 to 8.16e9.
constexpr int kSymEmuSeed = kEmuIncMul | kEmuSetupMul | kEmuIterMul;
constexpr int kSymEmuMixed = 0;
constexpr int kSymEmuLearned = 0;
constexpr int kSymEmuStandard = kEmuIncMul | kEmuIterMul;

// MIXED: the mixed form for class rules that admit few pairs (the literal
// rule): each pair's class is decided as in the row-group mixed kernel
// (kepler_fp32.cuh); a pair the rule admits is solved in FP32 and its
// increments, converted to double, are accumulated in FP64 with the rest;
// every other pair takes the FP64 solve (seeded with SEED).
template <bool STATS, bool LEARNED, bool SEED, bool MIXED>
__global__ void __launch_bounds__(128, MIXED ? 2 : ((SEED || LEARNED) ? 3 : 4))
    pair_step_sym_kernel(StepArgs a, int Smax, int64_t T)
{
    constexpr int kSymEmu =
        MIXED ? kSymEmuMixed : (SEED ? kSymEmuSeed : (LEARNED ? kSymEmuLearned : kSymEmuStandard));
    extern __shared__ __align__(16) unsigned char dsm[];
    MlpWeights *mlpW = reinterpret_cast<MlpWeights *>(dsm);
    __nv_bfloat16 *mlpStage = reinterpret_cast<__nv_bfloat16 *>(dsm + sizeof(MlpWeights));
    griddep_wait();    // X from the prep kernel
    griddep_launch();  // the apply kernel may begin launching
    if (LEARNED) mlp_load_shared(*mlpW, a.mlp);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t n = a.n;
    const int64_t W = (int64_t)gridDim.x * 4;
    const int64_t w = (int64_t)blockIdx.x * 4 + wib;
    const double *X = a.X;
    const KeplerParams kp{a.tol, a.max_iter, a.bisection};
    unsigned status = 0;
    long long it_sum = 0, slots = 0, fallbacks = 0, carries = 0, n32 = 0;
    int it_max = 0;
    const float *X32 = a.X32;

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
        double xi = 0, yi = 0, zi = 0, vxi = 0, vyi = 0, vzi = 0, mi = 1;
        if (irow) {
            xi = X[i];
            yi = X[n + i];
            zi = X[2 * n + i];
            vxi = X[3 * n + i];
            vyi = X[4 * n + i];
            vzi = X[5 * n + i];
            mi = X[6 * n + i];
        }
        float hi_i[3] = {0, 0, 0}, lo_i[3] = {0, 0, 0}, v_i[3] = {0, 0, 0}, m32i = 0.0f;
        if ((SEED || MIXED) && irow) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                hi_i[q] = X32[q * n + i];
                lo_i[q] = X32[(3 + q) * n + i];
                v_i[q] = X32[(6 + q) * n + i];
            }
            m32i = X32[9 * n + i];
        }
        double racc[6] = {0, 0, 0, 0, 0, 0}, cacc[6] = {0, 0, 0, 0, 0, 0};
        for (int k = k0; k < k1; ++k) {
            const int c = (lane + k) & 31;
            const int64_t j = 32 * J + c;
            const bool valid = irow && j < n && (!diag || c != lane);
            PairSolve p;
            double mj = 0.0;
            bool lane32 = false;  // MIXED: solved in FP32
            float d32[6];
            if (valid) {
                mj = X[6 * n + j];
                if (MIXED) {
                    float hi_j[3], lo_j[3], v_j[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        hi_j[q] = X32[q * n + j];
                        lo_j[q] = X32[(3 + q) * n + j];
                        v_j[q] = X32[(6 + q) * n + j];
                    }
                    Pair32 pr;
                    pair32_setup(pr, hi_i, lo_i, v_i, m32i, hi_j, lo_j, v_j, X32[9 * n + j],
                                 a.rule);
                    if (pr.fp32) {
                        int it32 = 0;
                        lane32 = pair32_solve(pr, a.t32, a.post32, a.guess, d32, it32);
                    }
                }
                if (!lane32)
                    pair_setup<kSymEmu>(p, a.tau, mi + mj, xi - X[j], yi - X[n + j],
                                        zi - X[2 * n + j], vxi - X[3 * n + j], vyi - X[4 * n + j],
                                        vzi - X[5 * n + j], a.pre,
                                        LEARNED ? 2 : (SEED ? -1 : a.guess));
                if (SEED && !lane32) {
                    // single-precision seed: the root of the FP32 solve of the
                    // same pair (unless t was reduced modulo the period)
                    float dr[3], dv[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        dr[q] = __fadd_rn(__fsub_rn(hi_i[q], X32[q * n + j]),
                                          __fsub_rn(lo_i[q], X32[(3 + q) * n + j]));
                        dv[q] = __fsub_rn(v_i[q], X32[(6 + q) * n + j]);
                    }
                    const K32 o = k32_phase1(dr, dv, m32i + X32[9 * n + j], a.ptau32, a.t32, 2);
                    if (o.ok && dbits(p.t) == dbits(a.tau) &&
                        !p.done) {
                        p.s = f2d(o.s);
                    } else if (!p.done) {
                        // no usable seed: the second-order guess, as pair_setup
                        // computes it
                        p.s = p.t * p.ir0;
                        const double cq = 0.5 * p.s * (p.eta0 * p.ir0);
                        if (magbits(cq) < 0x3fe0000000000000LL) p.s = fma(-cq, p.s, p.s);
                    }
                }
            }
            if (!valid || lane32) {
                p.done = true;
                p.beta = p.s = 0.0;
                p.iters = 0;
                p.status = 0;
            }
            if (LEARNED) learned_guess_warp(p, valid, *mlpW, mlpStage + wib * 32 * 16);
            double d[6];
            int iters = 0, fb = 0;
            fp64_solve_warp<SEED, kSymEmu>(p, valid && !lane32, a.tau, a.post * a.tau, kp, d, iters,
                                           fb);
            if (MIXED && lane32) {
                // exact conversions on the integer pipe
#pragma unroll
                for (int q = 0; q < 6; ++q) d[q] = f2d(d32[q]);
            }
            if (valid) {
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    racc[q] = fma(mj, d[q], racc[q]);
                    cacc[q] = fma(-mi, d[q], cacc[q]);
                }
                status |= p.status;
            }
            if (STATS) {
                carries += (valid && p.carried) ? 1 : 0;
                n32 += lane32 ? (diag ? 1 : 2) : 0;  // in ordered pairs
                it_sum += iters;
                fallbacks += fb;
                it_max = max(it_max, iters);
                const int wmax = __reduce_max_sync(0xffffffffu, iters);
                if (lane == 0) slots += 32LL * wmax;
            }
            if (!diag && k + 1 < k1) {
#pragma unroll
                for (int q = 0; q < 6; ++q) cacc[q] = __shfl_sync(0xffffffffu, cacc[q], (lane + 1) & 31);
            }
        }
        // row sums of rows i to slot (J, h); column sums to slot (I, h)
        if (irow) {
            double *dst = a.partial + (J * Smax + h) * 6 * n;
#pragma unroll
            for (int q = 0; q < 6; ++q) dst[q * n + i] = racc[q];
        }
        if (!diag) {
            const int64_t j = 32 * J + ((lane + k1 - 1) & 31);
            if (j < n) {
                double *dst = a.partial + (I * Smax + h) * 6 * n;
#pragma unroll
                for (int q = 0; q < 6; ++q) dst[q * n + j] = cacc[q];
            }
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
        if (MIXED) {
            long long s5 = n32;
            for (int o = 16; o > 0; o >>= 1) s5 += __shfl_xor_sync(0xffffffffu, s5, o);
            if (lane == 0) atomicAdd(&a.stats[kStatFp32Pairs], (unsigned long long)s5);
        }
    }
}

// Eqs. 27b-d with the existing slots of each particle added in a fixed
// order.  Block (x, y) takes 32 particles (one per lane) and the component
// pair (y, 3 + y), so that a step's partials are read by 3 n / 32 blocks; its
// kApplyWarps warps sum the slots of the other blocks Q = w, w + kApplyWarps,
// ... (coalesced loads, two interleaved sums each) and warp 0 adds the warps'
// sums in warp order and applies the update of x_y and v_y.
// fuse: the next sub-step's drift (Eq. 27a, next_drift) is applied too and
// its drifted copy written to X (and X32), as the prep kernel would write it
// from the new state, so that a run of steps needs no prep kernel after its
// first; the next pair kernel may then begin launching at once.
constexpr int kApplyWarps = 16;

__global__ void __launch_bounds__(32 * kApplyWarps)
    apply_sym_kernel(double *state, double *X, float *X32, const double *partial, int64_t n,
                     int Smax, int64_t W, int64_t T, double post_drift, int fuse,
                     double next_drift, unsigned *status)
{
    __shared__ double red[kApplyWarps][2][32];
    griddep_wait();  // the pair kernel's partials
    // Without fuse, a kernel that follows reads this one's output only after
    // its own griddep_wait or is launched plainly, so it may begin launching
    // now.  With fuse the next kernel is a persistent pair kernel whose
    // blocks must be spread evenly over the SMs: launched while this grid's
    // blocks still hold SM resources, some SMs would receive an extra block
    // (the seeded kernel is sized below its occupancy limit), and its static
    // work partition would then run those SMs' warps a third slower (a
    // 16384-body step measured 40.4 ms against 27.4 ms); it waits for this
    // grid to complete instead.
    if (!fuse) griddep_launch();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int q = blockIdx.y;
    const int64_t P = blockIdx.x;
    const int64_t i = P * 32 + lane;
    const int64_t nb = (n + 31) >> 5;
    double dr = 0.0, dv = 0.0;
    if (i < n) {
        // slot k = Q Smax + o holds the segment o of the tile of blocks P, Q
        double er[2] = {0, 0}, ev[2] = {0, 0};
        int u = 0;
        for (int64_t Q = wid; Q < nb; Q += kApplyWarps) {
            const int64_t tile = P <= Q ? Q * (Q + 1) / 2 + P : P * (P + 1) / 2 + Q;
            const int segs = sym_segments(tile, W, T);
            for (int o = 0; o < segs; ++o) {
                const int64_t k = Q * Smax + o;
                er[u] += partial[(k * 6 + q) * n + i];
                ev[u] += partial[(k * 6 + 3 + q) * n + i];
                u ^= 1;
            }
        }
        dr = er[0] + er[1];
        dv = ev[0] + ev[1];
    }
    red[wid][0][lane] = dr;
    red[wid][1][lane] = dv;
    __syncthreads();
    if (wid != 0 || i >= n) return;
    double tr = red[0][0][lane], tv = red[0][1][lane];
    for (int w = 1; w < kApplyWarps; ++w) {
        tr += red[w][0][lane];
        tv += red[w][1][lane];
    }
    const double v1 = X[(3 + q) * n + i] + tv;
    const double x1 = fma(v1, post_drift, X[q * n + i] + tr);
    if (!isfinite(x1) || !isfinite(v1)) atomicOr(status, kStatusNonfinite);
    state[q * n + i] = x1;
    state[(3 + q) * n + i] = v1;
    if (fuse) {
        const double x = fma(v1, next_drift, x1);
        X[q * n + i] = x;
        X[(3 + q) * n + i] = v1;
        if (X32) {
            const float hi = __double2float_rn(x);
            X32[q * n + i] = hi;
            X32[(3 + q) * n + i] = __double2float_rn(x - (double)hi);
            X32[(6 + q) * n + i] = __double2float_rn(v1);
        }
    }
}

namespace {

const void *sym_kernel(bool stats, bool learned, bool seed, bool mixed)
{
    if (mixed) {
        if (seed)
            return stats ? (const void *)pair_step_sym_kernel<true, false, true, true>
                         : (const void *)pair_step_sym_kernel<false, false, true, true>;
        return stats ? (const void *)pair_step_sym_kernel<true, false, false, true>
                     : (const void *)pair_step_sym_kernel<false, false, false, true>;
    }
    if (learned)
        return stats ? (const void *)pair_step_sym_kernel<true, true, false, false>
                     : (const void *)pair_step_sym_kernel<false, true, false, false>;
    if (seed)
        return stats ? (const void *)pair_step_sym_kernel<true, false, true, false>
                     : (const void *)pair_step_sym_kernel<false, false, true, false>;
    return stats ? (const void *)pair_step_sym_kernel<true, false, false, false>
                 : (const void *)pair_step_sym_kernel<false, false, false, false>;
}

size_t sym_smem(bool learned) { return learned ? sizeof(MlpWeights) + 4 * 32 * 16 * 2 : 0; }

}  // namespace

int pair_step_sym_blocks_per_sm(bool stats, bool learned, bool seed, bool mixed)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sym_kernel(stats, learned, seed, mixed),
                                                      128, sym_smem(learned)) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    // the seeded kernel runs fastest with 3 blocks per SM since part of its
    // multiplies moved to the integer pipes (before that, 2: 120.8 us against
    // 123.1 at 3, Plummer N = 1024); the mixed form's with 2; the others with
    // as many as fit
    if (mixed && b > 2) b = 2;
    if (seed && b > 3) b = 3;
    return b > 0 ? b : 1;
}

void launch_pair_step_sym(const StepArgs &a, int Smax, int64_t T, int blocks, bool stats,
                          cudaStream_t s)
{
    const bool learned = a.mlp != nullptr;
    const bool mixed = a.mixed != 0;
    const bool seed = !learned && a.X32 != nullptr && (!mixed || a.mixed == 2);
    int Sv = Smax;
    int64_t it = T;
    void *args[] = {(void *)&a, (void *)&Sv, (void *)&it};
    launch_pdl(sym_kernel(stats, learned, seed, mixed), dim3(blocks), dim3(128), args,
               sym_smem(learned), s);
}

void launch_apply_sym(double *state, double *X, float *X32, const double *partial, int64_t n,
                      int Smax, int64_t W, int64_t T, double post_drift, bool fuse,
                      double next_drift, unsigned *status, cudaStream_t s)
{
    int f = fuse ? 1 : 0;
    void *args[] = {(void *)&state,      (void *)&X, (void *)&X32, (void *)&partial,
                    (void *)&n,          (void *)&Smax, (void *)&W, (void *)&T,
                    (void *)&post_drift, (void *)&f, (void *)&next_drift, (void *)&status};
    launch_pdl((const void *)apply_sym_kernel, dim3((unsigned)((n + 31) / 32), 3),
               dim3(32 * kApplyWarps), args, 0, s);
}

}  // namespace sakura
