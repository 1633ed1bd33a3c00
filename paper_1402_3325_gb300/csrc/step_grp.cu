// step_grp.cu -- FP64 W step solving every unordered pair once (Newton's
// third law, which the paper leaves to future implementations, Sec. 2.1), in
// row-group phases, and the apply kernel of the row-group layout.
//
// The increments of the ordered pairs (i, j) and (j, i) are exact negatives
// of each other: every scalar of the solve (r0^2, eta0 = r0.v0, v0^2, beta,
// zeta0, s, G_k) is unchanged when (r0, v0) -> (-r0, -v0), IEEE negation and
// round-to-nearest are symmetric, and the increments are linear in (r0, v0).
// So each pair is solved once and adds  m_j delta/m_ij  to particle i and
// -m_i delta/m_ij  to particle j (Eq. 23 with 1/m_i folded in).
//
// Work (step_common.cuh): a block of kFp64GrpWarps warps owns a group of as
// many row blocks of 32 particles, warp w the row block I = g G + w, and its
// warps sweep the column blocks J >= g G together.  In phase J warp w solves the 32 x 32 tile (I, J) (nothing when
// I > J; the ordered pairs of the diagonal tile when I = J) on a systolic
// schedule: lane l owns row i = 32 I + l and at step k solves column
// c = (l + k) mod 32, so the 32 lanes always hold 32 different columns.  The
// column blocks of a window of up to 8 (or 4) phases are staged in shared
// memory for all warps.  Row sums stay in the lane's registers for the whole
// group; each warp adds its column sums into its own shared-memory
// accumulators of the window, and after the window's block barrier the
// block adds the warps' accumulators in warp order and writes one column
// partial per particle.  Every (slot, particle) is written exactly once and
// the apply kernel adds a particle's slots in a fixed order (deterministic,
// no atomics).  Partials per step: about 30 MB at n = 16384, which stay in
// L2 (the earlier per-tile-segment slots were 0.4 GB).
#include <cuda_runtime.h>

#include <algorithm>

#include "kepler_df64.cuh"
#include "kepler_fp64.cuh"
#include "mlp_infer.cuh"
#include "pair_batch_fp64.cuh"
#include "step_common.cuh"

namespace sakura {

GrpLayout make_grp_layout(int64_t n, int G, int64_t &blocks)
{
    GrpLayout L;
    L.nb = (n + 31) / 32;
    L.G = G;
    L.ng = (int)((L.nb + G - 1) / G);
    L.P = grp_start(L.ng, L.nb, G);
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, L.P));
    L.Hmax = 1;
    for (int64_t g = 0; g < L.ng; ++g) {
        const int64_t s0 = grp_start(g, L.nb, G), s1 = grp_start(g + 1, L.nb, G);
        const int64_t h = grp_owner(s1 - 1, blocks, L.P) - grp_owner(s0, blocks, L.P) + 1;
        L.Hmax = std::max<int>(L.Hmax, (int)h);
    }
    return L;
}

// Eqs. 27b-d for the row-group layout.  Particle i of row block I (group
// gi = I / G) adds its group's row pieces h = 0 .. npieces - 1 and the
// column partials of groups g = 0 .. gi (the phases (g, I)), in that fixed
// order, spread over the block's warps (slot s to warp s mod
// kGrpApplyWarps, alternately into two sums) and then added in warp order.
// Block (x, y) takes 32 particles and the component pair (y, 3 + y).
// fuse: the next sub-step's drift (Eq. 27a, next_drift) is applied too and
// its drifted copy written to X (and X32), as the prep kernel would write it
// from the new state.
constexpr int kGrpApplyWarps = 8;

__global__ void __launch_bounds__(32 * kGrpApplyWarps)
    apply_grp_kernel(double *state, double *X, float *X32, const double *rowpart,
                     const double *colpart, int64_t n, GrpLayout L, int64_t B,
                     double post_drift, int fuse, double next_drift, unsigned *status)
{
    __shared__ double red[kGrpApplyWarps][2][32];
    griddep_wait();  // the pair kernel's partials
    // Without fuse, a kernel that follows reads this one's output only after
    // its own griddep_wait or is launched plainly, so it may begin launching
    // now.  With fuse the next kernel is a persistent pair kernel whose
    // blocks must be spread evenly over the SMs: launched while this grid's
    // blocks still hold SM resources, some SMs could receive an extra block
    // and the static phase ranges would then run slower there; it waits for
    // this grid to complete instead.
    if (!fuse) griddep_launch();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int q = blockIdx.y;
    const int64_t Ib = blockIdx.x;
    const int64_t i = Ib * 32 + lane;
    const int64_t gi = Ib / L.G;
    const int64_t s0 = grp_start(gi, L.nb, L.G), s1 = grp_start(gi + 1, L.nb, L.G);
    const int npieces = (int)(grp_owner(s1 - 1, B, L.P) - grp_owner(s0, B, L.P)) + 1;
    const int nslots = npieces + (int)gi + 1;
    double dr = 0.0, dv = 0.0;
    if (i < n) {
        auto slot = [&](int sl) {
            return sl < npieces ? rowpart + (int64_t)sl * 6 * n
                                : colpart + (int64_t)(sl - npieces) * 6 * n;
        };
        double er0 = 0, er1 = 0, ev0 = 0, ev1 = 0;
        int sl = wid;
        for (; sl + kGrpApplyWarps < nslots; sl += 2 * kGrpApplyWarps) {
            const double *b0 = slot(sl), *b1 = slot(sl + kGrpApplyWarps);
            er0 += b0[q * n + i];
            ev0 += b0[(3 + q) * n + i];
            er1 += b1[q * n + i];
            ev1 += b1[(3 + q) * n + i];
        }
        if (sl < nslots) {
            const double *b0 = slot(sl);
            er0 += b0[q * n + i];
            ev0 += b0[(3 + q) * n + i];
        }
        dr = er0 + er1;
        dv = ev0 + ev1;
    }
    red[wid][0][lane] = dr;
    red[wid][1][lane] = dv;
    __syncthreads();
    if (wid != 0 || i >= n) return;
    double tr = red[0][0][lane], tv = red[0][1][lane];
    for (int w = 1; w < kGrpApplyWarps; ++w) {
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

void launch_apply_grp(double *state, double *X, float *X32, const double *rowpart,
                      const double *colpart, int64_t n, const GrpLayout &L, int64_t blocks,
                      double post_drift, bool fuse, double next_drift, unsigned *status,
                      cudaStream_t s)
{
    GrpLayout Lv = L;
    int64_t B = blocks;
    int f = fuse ? 1 : 0;
    void *args[] = {(void *)&state,      (void *)&X,    (void *)&X32,       (void *)&rowpart,
                    (void *)&colpart,    (void *)&n,    (void *)&Lv,        (void *)&B,
                    (void *)&post_drift, (void *)&f,    (void *)&next_drift, (void *)&status};
    launch_pdl((const void *)apply_grp_kernel, dim3((unsigned)((n + 31) / 32), 3),
               dim3(32 * kGrpApplyWarps), args, 0, s);
}

// shared memory of the pair kernel: the warps' column sums of the window
// (double [kFp64GrpWarps][WIN][6][32]), the window's column blocks double
// buffered (double [2][WIN][7][32]: x, y, z, vx, vy, vz, m of the drifted
// state; float [2][WIN][10][32]: the float copy for the seed), then (learned
// guess) the network and the warps' staging
// (kFp64GrpWarps = 4 warps per block and two blocks per SM: one block's
// warps keep the SM's FP64 pipes busy while the other block waits at a
// window barrier)
// The window: 8 phases with the seed (two blocks of 4 warps per SM), 4
// otherwise (the network's weights take shared memory; without either, four
// blocks per SM fit).
__host__ __device__ constexpr int grp_window(bool seed) { return seed ? 8 : 4; }
__host__ __device__ constexpr size_t grp_cs_bytes(int win)
{
    return sizeof(double) * kFp64GrpWarps * win * 6 * 32;
}
__host__ __device__ constexpr size_t grp_cd_bytes(int win) { return sizeof(double) * 2 * win * 7 * 32; }
__host__ __device__ constexpr size_t grp_cf_bytes(int win, bool seed)
{
    return seed ? sizeof(float) * 2 * win * 10 * 32 : 0;
}
__host__ __device__ constexpr size_t grp_base_smem(int win, bool seed)
{
    return grp_cs_bytes(win) + grp_cd_bytes(win) + grp_cf_bytes(win, seed);
}

size_t grp_smem(bool learned, bool seed)
{
    const int win = grp_window(seed);
    return grp_base_smem(win, seed) +
           (learned ? sizeof(MlpWeights) + kFp64GrpWarps * 32 * 16 * 2 : 0);
}

template <bool STATS, bool LEARNED, bool SEED>
__global__ void __launch_bounds__(kFp64GrpWarps * 32, (LEARNED || SEED) ? 2 : 4)
    pair_step_grp_kernel(StepArgs a, GrpLayout L, double *rowpart, double *colpart)
{
    constexpr int WIN = grp_window(SEED);
    extern __shared__ __align__(16) unsigned char gsm[];
    double(*cs)[WIN][6][32] = reinterpret_cast<double(*)[WIN][6][32]>(gsm);
    double(*cd)[WIN][7][32] = reinterpret_cast<double(*)[WIN][7][32]>(gsm + grp_cs_bytes(WIN));
    float(*cf)[WIN][10][32] =
        reinterpret_cast<float(*)[WIN][10][32]>(gsm + grp_cs_bytes(WIN) + grp_cd_bytes(WIN));
    MlpWeights *mlpW = reinterpret_cast<MlpWeights *>(gsm + grp_base_smem(WIN, SEED));
    __nv_bfloat16 *mlpStage =
        reinterpret_cast<__nv_bfloat16 *>(gsm + grp_base_smem(WIN, SEED) + sizeof(MlpWeights));
    griddep_wait();    // X (and X32) from the prep kernel or the previous apply kernel
    griddep_launch();  // the apply kernel may begin launching
    if (LEARNED) mlp_load_shared(*mlpW, a.mlp);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int tid = threadIdx.x;
    const int64_t n = a.n;
    const int64_t nb = L.nb;
    const int64_t P = L.P;
    const int64_t B = gridDim.x;
    const int64_t b = blockIdx.x;
    const double *X = a.X;
    const float *X32 = a.X32;
    const KeplerParams kp{a.tol, a.max_iter, a.bisection};
    unsigned status = 0;
    long long it_sum = 0, slots = 0, fallbacks = 0, carries = 0;
    int it_max = 0;

    const int64_t p0 = b * P / B, p1 = (b + 1) * P / B;
    int64_t g = 0;
    while (g + 1 < L.ng && grp_start(g + 1, nb, kFp64GrpWarps) <= p0) ++g;
    int64_t J = g * kFp64GrpWarps + (p0 - grp_start(g, nb, kFp64GrpWarps));
    int64_t p = p0;
    // a window: up to WIN consecutive phases of one group within the
    // block's range
    auto window_len = [&](int64_t pw, int64_t Jw) {
        const int64_t m = nb - Jw < p1 - pw ? nb - Jw : p1 - pw;
        return (int)(m < WIN ? m : WIN);
    };
    // the window's column blocks Jw .. Jw + len - 1 into buffer buf
    auto load_cols = [&](int buf, int64_t Jw, int len) {
        for (int e = tid; e < len * 32; e += kFp64GrpWarps * 32) {
            const int cb = e >> 5, c = e & 31;
            const int64_t j = 32 * (Jw + cb) + c;
            const bool ok = j < n;
#pragma unroll
            for (int f = 0; f < 7; ++f) cd[buf][cb][f][c] = ok ? X[f * n + j] : 0.0;
            if (SEED) {
#pragma unroll
                for (int f = 0; f < 10; ++f) cf[buf][cb][f][c] = ok ? X32[f * n + j] : 0.0f;
            }
        }
    };
    int wl = p < p1 ? window_len(p, J) : 0;
    if (wl > 0) load_cols(0, J, wl);
    __syncthreads();

    double xi = 0, yi = 0, zi = 0, vxi = 0, vyi = 0, vzi = 0, mi = 1;
    float hi_i[3] = {0, 0, 0}, lo_i[3] = {0, 0, 0}, v_i[3] = {0, 0, 0}, m32i = 0.0f;
    double racc[6];
    bool new_group = true;
    int buf = 0;
    while (wl > 0) {
        const int64_t I = g * kFp64GrpWarps + wib;
        const int64_t i = 32 * I + lane;
        const bool irow = I < nb && i < n;
        if (new_group) {
#pragma unroll
            for (int q = 0; q < 6; ++q) racc[q] = 0.0;
            if (irow) {
                xi = X[i];
                yi = X[n + i];
                zi = X[2 * n + i];
                vxi = X[3 * n + i];
                vyi = X[4 * n + i];
                vzi = X[5 * n + i];
                mi = X[6 * n + i];
                if (SEED) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        hi_i[q] = X32[q * n + i];
                        lo_i[q] = X32[(3 + q) * n + i];
                        v_i[q] = X32[(6 + q) * n + i];
                    }
                    m32i = X32[9 * n + i];
                }
            }
            new_group = false;
        }
        for (int cb = 0; cb < wl; ++cb) {
#pragma unroll
            for (int q = 0; q < 6; ++q) cs[wib][cb][q][lane] = 0.0;
        }
        __syncwarp();
        for (int cb = 0; cb < wl; ++cb) {
            const int64_t Jt = J + cb;
            if (!(I <= Jt && I < nb)) continue;  // warp-uniform: no tile (I, Jt)
            const bool diag = I == Jt;
            for (int k = 0; k < 32; ++k) {
                const int c = (lane + k) & 31;
                const int64_t j = 32 * Jt + c;
                const bool valid = irow && j < n && (!diag || c != lane);
                PairSolve ps;
                double mj = 0.0;
                if (valid) {
                    mj = cd[buf][cb][6][c];
                    pair_setup(ps, a.tau, mi + mj, xi - cd[buf][cb][0][c], yi - cd[buf][cb][1][c],
                               zi - cd[buf][cb][2][c], vxi - cd[buf][cb][3][c],
                               vyi - cd[buf][cb][4][c], vzi - cd[buf][cb][5][c], a.pre,
                               LEARNED ? 2 : (SEED ? -1 : a.guess));
                    if (SEED) {
                        // single-precision seed: the root of the FP32 solve of
                        // the same pair (unless t was reduced modulo the period)
                        float dr[3], dv[3];
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            dr[q] = __fadd_rn(__fsub_rn(hi_i[q], cf[buf][cb][q][c]),
                                              __fsub_rn(lo_i[q], cf[buf][cb][3 + q][c]));
                            dv[q] = __fsub_rn(v_i[q], cf[buf][cb][6 + q][c]);
                        }
                        const K32 o = k32_phase1(dr, dv, m32i + cf[buf][cb][9][c], a.ptau32,
                                                 a.t32, 2);
                        if (o.ok && __double_as_longlong(ps.t) == __double_as_longlong(a.tau) &&
                            !ps.done) {
                            ps.s = f2d(o.s);
                        } else if (!ps.done) {
                            // no usable seed: the second-order guess, as
                            // pair_setup computes it
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
                if (LEARNED) learned_guess_warp(ps, valid, *mlpW, mlpStage + wib * 32 * 16);
                double d[6];
                int iters = 0, fb = 0;
                fp64_solve_warp<SEED>(ps, valid, a.tau, a.post * a.tau, kp, d, iters, fb);
                if (valid) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) racc[q] = fma(mj, d[q], racc[q]);
                    if (!diag) {
#pragma unroll
                        for (int q = 0; q < 6; ++q) cs[wib][cb][q][c] = fma(-mi, d[q], cs[wib][cb][q][c]);
                    }
                    status |= ps.status;
                }
                if (STATS) {
                    carries += (valid && ps.carried) ? 1 : 0;
                    it_sum += iters;
                    fallbacks += fb;
                    it_max = max(it_max, iters);
                    const int wmax = __reduce_max_sync(0xffffffffu, iters);
                    if (lane == 0) slots += 32LL * wmax;
                }
            }
        }
        __syncthreads();  // every warp's column sums of the window are complete
        // the next window; its column blocks are loaded now
        const int64_t pn = p + wl;
        int64_t gn = g, Jn = J + wl;
        if (Jn == nb) {
            gn = g + 1;
            Jn = gn * kFp64GrpWarps;
        }
        const int wln = pn < p1 ? window_len(pn, Jn) : 0;
        if (wln > 0) load_cols(buf ^ 1, Jn, wln);
        // the window's column partials: the warps' sums added in warp order
        for (int e = tid; e < wl * 192; e += kFp64GrpWarps * 32) {
            const int cb = e / 192, rem = e - cb * 192, c = rem & 31, q = rem >> 5;
            const int64_t j = 32 * (J + cb) + c;
            if (j < n) {
                double sum = cs[0][cb][q][c];
#pragma unroll
                for (int w = 1; w < kFp64GrpWarps; ++w) sum += cs[w][cb][q][c];
                colpart[(g * 6 + q) * n + j] = sum;
            }
        }
        // leaving the group (or the block's range): this piece's row partial
        if (gn != g || pn == p1) {
            if (irow) {
                const int64_t h = b - grp_owner(grp_start(g, nb, kFp64GrpWarps), B, P);
                double *dst = rowpart + h * 6 * n;
#pragma unroll
                for (int q = 0; q < 6; ++q) dst[q * n + i] = racc[q];
            }
            new_group = true;
        }
        __syncthreads();  // the sums are read and the next column blocks stored
        p = pn;
        g = gn;
        J = Jn;
        wl = wln;
        buf ^= 1;
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
    }
}

namespace {

const void *grp_fp64_kernel(bool stats, bool learned, bool seed)
{
    if (learned)
        return stats ? (const void *)pair_step_grp_kernel<true, true, false>
                     : (const void *)pair_step_grp_kernel<false, true, false>;
    if (seed)
        return stats ? (const void *)pair_step_grp_kernel<true, false, true>
                     : (const void *)pair_step_grp_kernel<false, false, true>;
    return stats ? (const void *)pair_step_grp_kernel<true, false, false>
                 : (const void *)pair_step_grp_kernel<false, false, false>;
}

}  // namespace

int pair_step_grp_blocks_per_sm(bool stats, bool learned, bool seed)
{
    const void *fn = grp_fp64_kernel(stats, learned, seed);
    const size_t smem = grp_smem(learned, seed && !learned);
    int b = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kFp64GrpWarps * 32, smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return b > 0 ? b : 1;
}

void launch_pair_step_grp(const StepArgs &a, const GrpLayout &L, double *rowpart,
                          double *colpart, int blocks, bool stats, cudaStream_t s)
{
    const bool learned = a.mlp != nullptr;
    const bool seed = !learned && a.X32 != nullptr;
    const void *fn = grp_fp64_kernel(stats, learned, seed);
    const size_t smem = grp_smem(learned, seed);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    GrpLayout Lv = L;
    void *args[] = {(void *)&a, (void *)&Lv, (void *)&rowpart, (void *)&colpart};
    launch_pdl(fn, dim3(blocks), dim3(kFp64GrpWarps * 32), args, smem, s);
}

}  // namespace sakura
