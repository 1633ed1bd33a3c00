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
// Work (step_common.cuh): a block of kFp64GrpWarps = G warps takes the
// tile-steps of a group of G row blocks, which meets the column blocks
// J >= g G one phase per J, and the grid's blocks take equal contiguous
// ranges of all groups' tile-steps.  In phase J the tiles (g G + r, J),
// r <= J - g G, are solved one per warp, warp w taking row block
// r = (w + J) mod G: the row blocks rotate over the warps from phase to phase,
// so a row whose pairs cost more (a black hole's, whose orbits take more
// series terms and seed iterations) slows each warp in turn rather than one
// warp of the block, which the others would wait for at every window
// barrier.  A tile is solved on a systolic schedule: lane l owns row
// i = 32 I + l and at step k solves column c = (l + k) mod 32, so the 32
// lanes always hold 32 different columns.  The column blocks of a window of
// up to 8 (or 4) phases are staged in shared memory for all warps.  Each
// warp sums a phase's row sums in registers and adds them to its own
// shared-memory row sums of the group, and adds its column sums into its own
// shared-memory accumulators of the window; after the window's block barrier
// the block adds the warps' column sums in warp order and writes one column
// partial per particle (colpart, or colx for a phase the block entered after
// its step 0), and on leaving the group the warps' row sums in warp order
// (one row piece).  Every slot is written exactly once and the apply kernel
// adds a particle's slots in a fixed order (deterministic, no atomics).
// Partials per step: about 30 MB at n = 16384, which stay in L2 (the
// systolic tile kernel's per-tile-segment slots are 0.4 GB).
#include <cuda_runtime.h>

#include <algorithm>

#include "kepler_df64.cuh"
#include "kepler_fp32.cuh"
#include "kepler_fp64.cuh"
#include "mlp_infer.cuh"
#include "pair_batch_fp64.cuh"
#include "step_common.cuh"
#include "step_grp.cuh"

namespace sakura {

// The FP64 operations formed on the integer pipes (kepler_fp64.cuh) and the
// blocks of 4 warps per SM, per kernel, as measured at 16384 bodies (ms per
// step).  The emulated multiplies lengthen each warp's dependency chains, so
// they pay only with enough warps per SM to hide them:
//   seed: 4 blocks (ptxas fits the kernel in 128 registers, spilling 52
//     bytes), windows of 2
//     phases, the increments', the setup's and the iterations' multiplies:
//     20.43 (20.72 with the steps weighted 3 + tiles in the layout), against
//     24.03 with 2 blocks and the increments' multiplies only, 22.15 with 3
//     blocks and those, 20.85-21.72 with other sets;
//   mixed form under the literal rule (inline class test): 3 blocks, windows
//     of 2, the increments', the setup's and the carry's multiplies: 21.57
//     against 25.43 with 2 blocks;
//   learned guess (255 registers at 2 blocks, 168 with some spills at 3):
//     3 blocks, the increments' multiplies: 27.74 against 29.02 with 2
//     blocks and 35.36 with the iterations' and the setup's too;
//   standard guess (4 blocks of 128 registers): the increments' and the
//     iterations' multiplies: 26.47, against 27.09 with the setup's too.
constexpr int kGrpLearnedBlocks = 3;
constexpr int kGrpEmuSeed = kEmuIncMul | kEmuSetupMul | kEmuIterMul;
constexpr int kGrpEmuMixed = kEmuIncMul | kEmuSetupMul | kEmuCarryMul;
constexpr int kGrpEmuLearned = kEmuIncMul;
constexpr int kGrpEmuStandard = kEmuIncMul | kEmuIterMul;

// Eqs. 27b-d for the row-group layout.  Layout index i (particle
// grp_particle(i)) of row block I (group gi = I / G) adds its group's row
// pieces h = 0 .. npieces - 1 and the
// column sums of the phases (g, I), g = 0 .. gi (colpart[g], then the colx
// slots of the blocks that start inside that phase), in that fixed order,
// spread over the block's warps (slot s to warp s mod kGrpApplyWarps,
// alternately into two sums) and then added in warp order.  Block (x, y)
// takes 32 particles and the component pair (y, 3 + y).
// fuse: the next sub-step's drift (Eq. 27a, next_drift) is applied too and
// its drifted copy written to X (and X32), as the prep kernel would write it
// from the new state.
constexpr int kGrpApplyWarps = 8;

__global__ void __launch_bounds__(32 * kGrpApplyWarps)
    apply_grp_kernel(double *state, double *X, float *X32, GrpParts parts, int64_t n,
                     GrpLayout L, int64_t B, double post_drift, int fuse, double next_drift,
                     unsigned *status)
{
    __shared__ double red[kGrpApplyWarps][2][32];
    griddep_wait();  // the pair kernel's partials
    // Without fuse, a kernel that follows reads this one's output only after
    // its own griddep_wait or is launched plainly, so it may begin launching
    // now.  With fuse the next kernel is a persistent pair kernel whose
    // blocks must be spread evenly over the SMs: launched while this grid's
    // blocks still hold SM resources, some SMs could receive an extra block
    // and the static ranges would then run slower there; it waits for this
    // grid to complete instead.
    if (!fuse) griddep_launch();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int q = blockIdx.y;
    const int64_t Ib = blockIdx.x;
    const int64_t i = Ib * 32 + lane;
    const int64_t gi = Ib / L.G;
    const int64_t x0 = grp_phase_x(L, gi, 0), x1 = grp_phase_last_x(L, gi, L.nb - gi * L.G - 1);
    const int npieces = (int)(grp_owner(x1, B, L) - grp_owner(x0, B, L)) + 1;
    const int nslots = npieces + (int)gi + 1;
    double dr = 0.0, dv = 0.0;
    if (i < n) {
        // slot sl: row piece sl, or the column sums of phase (sl - npieces, Ib)
        auto add = [&](int sl, double &er, double &ev) {
            if (sl < npieces) {
                const double *p = parts.row + (int64_t)sl * 6 * n;
                er += p[q * n + i];
                ev += p[(3 + q) * n + i];
                return;
            }
            const int64_t gg = sl - npieces;
            const double *p = parts.col + gg * 6 * n;
            er += p[q * n + i];
            ev += p[(3 + q) * n + i];
            if (L.S == 32) return;  // whole phases: no phase is split
            const int64_t t = Ib - gg * L.G;
            const int64_t bl = grp_owner(grp_phase_last_x(L, gg, t), B, L);
            for (int64_t bb = grp_owner(grp_phase_x(L, gg, t), B, L) + 1; bb <= bl; ++bb) {
                er += parts.colx[(bb * 6 + q) * 32 + lane];
                ev += parts.colx[(bb * 6 + 3 + q) * 32 + lane];
            }
        };
        double er0 = 0, er1 = 0, ev0 = 0, ev1 = 0;
        int sl = wid;
        for (; sl + kGrpApplyWarps < nslots; sl += 2 * kGrpApplyWarps) {
            add(sl, er0, ev0);
            add(sl + kGrpApplyWarps, er1, ev1);
        }
        if (sl < nslots) add(sl, er0, ev0);
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
    const int64_t ip = grp_particle(L, n, i);  // the particle of layout index i
    const double v1 = X[(3 + q) * n + ip] + tv;
    const double x1n = fma(v1, post_drift, X[q * n + ip] + tr);
    if (!isfinite(x1n) || !isfinite(v1)) atomicOr(status, kStatusNonfinite);
    state[q * n + ip] = x1n;
    state[(3 + q) * n + ip] = v1;
    if (fuse) {
        const double x = fma(v1, next_drift, x1n);
        X[q * n + ip] = x;
        X[(3 + q) * n + ip] = v1;
        if (X32) {
            const float hi = __double2float_rn(x);
            X32[q * n + ip] = hi;
            X32[(3 + q) * n + ip] = __double2float_rn(x - (double)hi);
            X32[(6 + q) * n + ip] = __double2float_rn(v1);
        }
    }
}

void launch_apply_grp(double *state, double *X, float *X32, const GrpParts &parts, int64_t n,
                      const GrpLayout &L, int64_t blocks, double post_drift, bool fuse,
                      double next_drift, unsigned *status, cudaStream_t s)
{
    GrpParts pv = parts;
    GrpLayout Lv = L;
    int64_t B = blocks;
    int f = fuse ? 1 : 0;
    void *args[] = {(void *)&state,      (void *)&X, (void *)&X32,        (void *)&pv,
                    (void *)&n,          (void *)&Lv, (void *)&B,         (void *)&post_drift,
                    (void *)&f,          (void *)&next_drift, (void *)&status};
    launch_pdl((const void *)apply_grp_kernel, dim3((unsigned)((n + 31) / 32), 3),
               dim3(32 * kGrpApplyWarps), args, 0, s);
}

// shared memory of the pair kernel: the warps' column sums of the window
// (double [G][WIN][6][32]), the window's column blocks (double [WIN][7][32]:
// x, y, z, vx, vy, vz, m of the drifted state; float [WIN][10][32]: the float
// copy for the seed), the warps' row sums of the group (double [G][G][6][32]:
// warp, row block of the group), then (learned guess) the network and the
// warps' staging.  G = kFp64GrpWarps = 4 warps per block and several blocks
// per SM: one block's warps keep the SM's FP64 pipes busy while another
// waits at a window barrier.  The window: 2 phases with the seed or the
// inline class test (their 4 and 3 blocks per SM must fit in shared memory),
// 4 otherwise.  The column blocks are loaded between the window's two
// barriers, after every warp has finished with the previous ones, so one
// buffer serves.
constexpr int kGrpSeedBlocks = 4, kGrpSeedWindow = 2;
constexpr int kGrpMixedBlocks = 3, kGrpMixedWindow = 2;
__host__ __device__ constexpr int grp_window(bool seed, bool mixed)
{
    return mixed ? kGrpMixedWindow : (seed ? kGrpSeedWindow : 4);
}
__host__ __device__ constexpr size_t grp_cs_bytes(int win)
{
    return sizeof(double) * kFp64GrpWarps * win * 6 * 32;
}
__host__ __device__ constexpr size_t grp_cd_bytes(int win) { return sizeof(double) * win * 7 * 32; }
__host__ __device__ constexpr size_t grp_cf_bytes(int win, bool seed)
{
    return seed ? sizeof(float) * win * 10 * 32 : 0;
}
__host__ __device__ constexpr size_t grp_rs_bytes()
{
    return sizeof(double) * kFp64GrpWarps * kFp64GrpWarps * 6 * 32;
}
__host__ __device__ constexpr size_t grp_base_smem(int win, bool seed)
{
    return grp_cs_bytes(win) + grp_cd_bytes(win) + grp_cf_bytes(win, seed) + grp_rs_bytes();
}

// f32: the float copy is staged (the seed, or the inline class test)
size_t grp_smem(bool learned, bool seed, bool mixed)
{
    const int win = grp_window(seed, mixed);
    const bool f32 = seed || mixed;
    return grp_base_smem(win, f32) +
           (learned ? sizeof(MlpWeights) + kFp64GrpWarps * 32 * 16 * 2 : 0);
}

// MIXED: the mixed form for class rules that admit few pairs (the literal
// rule), as in the tile kernel (step_sym.cu): each pair's class is decided
// from the float copy (kepler_fp32.cuh); a pair the rule admits is solved in
// FP32 and its increments, converted to double, are accumulated in FP64 with
// the rest; every other pair takes the FP64 solve (seeded with SEED).
template <bool STATS, bool LEARNED, bool SEED, bool MIXED>
__global__ void __launch_bounds__(kFp64GrpWarps * 32,
                                  LEARNED ? kGrpLearnedBlocks
                                          : (MIXED ? kGrpMixedBlocks : (SEED ? kGrpSeedBlocks : 4)))
    pair_step_grp_kernel(StepArgs a, GrpLayout L, GrpParts parts)
{
    constexpr int G = kFp64GrpWarps;
    constexpr bool F32 = SEED || MIXED;  // the float copy is staged
    constexpr int kGrpEmu =
        MIXED ? kGrpEmuMixed : (SEED ? kGrpEmuSeed : (LEARNED ? kGrpEmuLearned : kGrpEmuStandard));
    constexpr int WIN = grp_window(SEED, MIXED);
    extern __shared__ __align__(16) unsigned char gsm[];
    double(*cs)[WIN][6][32] = reinterpret_cast<double(*)[WIN][6][32]>(gsm);
    double(*cd)[7][32] = reinterpret_cast<double(*)[7][32]>(gsm + grp_cs_bytes(WIN));
    float(*cf)[10][32] =
        reinterpret_cast<float(*)[10][32]>(gsm + grp_cs_bytes(WIN) + grp_cd_bytes(WIN));
    double(*rs)[G][6][32] = reinterpret_cast<double(*)[G][6][32]>(
        gsm + grp_cs_bytes(WIN) + grp_cd_bytes(WIN) + grp_cf_bytes(WIN, F32));
    MlpWeights *mlpW = reinterpret_cast<MlpWeights *>(gsm + grp_base_smem(WIN, F32));
    __nv_bfloat16 *mlpStage =
        reinterpret_cast<__nv_bfloat16 *>(gsm + grp_base_smem(WIN, F32) + sizeof(MlpWeights));
    griddep_wait();    // X (and X32) from the prep kernel or the previous apply kernel
    griddep_launch();  // the apply kernel may begin launching
    if (LEARNED) mlp_load_shared(*mlpW, a.mlp);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int tid = threadIdx.x;
    const int64_t n = a.n;
    const int64_t nb = L.nb;
    const int64_t B = gridDim.x;
    const int64_t b = blockIdx.x;
    const double *X = a.X;
    const float *X32 = a.X32;
    const KeplerParams kp{a.tol, a.max_iter, a.bisection};
    unsigned status = 0;
    long long it_sum = 0, slots = 0, fallbacks = 0, carries = 0, n32 = 0;
    int it_max = 0;

    GrpPos cur = grp_block_start(L, b, B);
    // the range's end, block-uniform, kept in shared memory (read once per
    // window) rather than in registers
    __shared__ GrpPos s_end;
    if (tid == 0) s_end = grp_block_start(L, b + 1, B);
    __syncthreads();
    auto in_range = [&](const GrpPos &p) {
        const GrpPos e = s_end;
        return p.g < e.g || (p.g == e.g && (p.t < e.t || (p.t == e.t && p.k < e.k)));
    };
    // a window: up to WIN consecutive phases of one group within the range
    auto window_len = [&](const GrpPos &p) {
        const GrpPos e = s_end;
        const int64_t m = p.g < e.g ? nb - p.g * G - p.t : e.t - p.t + (e.k > 0 ? 1 : 0);
        return (int)(m < WIN ? m : WIN);
    };
    // the window's column blocks Jw .. Jw + len - 1
    auto load_cols = [&](int64_t Jw, int len) {
        for (int e = tid; e < len * 32; e += G * 32) {
            const int cb = e >> 5, c = e & 31;
            const int64_t j = 32 * (Jw + cb) + c;
            const bool ok = j < n;
            const int64_t jp = ok ? grp_particle(L, n, j) : 0;
#pragma unroll
            for (int f = 0; f < 7; ++f) cd[cb][f][c] = ok ? X[f * n + jp] : 0.0;
            if (F32) {
#pragma unroll
                for (int f = 0; f < 10; ++f) cf[cb][f][c] = ok ? X32[f * n + jp] : 0.0f;
            }
        }
    };
    for (int e = tid; e < G * G * 6 * 32; e += G * 32) (&rs[0][0][0][0])[e] = 0.0;
    int wl = in_range(cur) ? window_len(cur) : 0;
    if (wl > 0) load_cols(cur.g * G + cur.t, wl);
    __syncthreads();

    while (wl > 0) {
        const int64_t g = cur.g, R = grp_rows(L, g), J0 = g * G + cur.t;
        // the steps of the window's first and last phases
        const int kfirst = cur.k;
        const int klast = (g == s_end.g && cur.t + wl - 1 == s_end.t) ? s_end.k : 32;
        for (int cb = 0; cb < wl; ++cb) {
#pragma unroll
            for (int q = 0; q < 6; ++q) cs[wib][cb][q][lane] = 0.0;
        }
        __syncwarp();
        for (int cb = 0; cb < wl; ++cb) {
            const int64_t t = cur.t + cb;
            const int r = (int)((wib + t) % G);  // this warp's row block of the phase
            if (!(r <= t && r < R)) continue;     // warp-uniform: no tile
            const int64_t I = g * G + r, Jt = J0 + cb;
            const bool diag = I == Jt;
            const int64_t i = 32 * I + lane;
            const bool irow = i < n;
            const int kb = cb == 0 ? kfirst : 0;
            const int ke = cb == wl - 1 ? klast : 32;
            double xi = 0, yi = 0, zi = 0, vxi = 0, vyi = 0, vzi = 0, mi = 1;
            float hi_i[3] = {0, 0, 0}, lo_i[3] = {0, 0, 0}, v_i[3] = {0, 0, 0}, m32i = 0.0f;
            if (irow) {
                const int64_t ip = grp_particle(L, n, i);
                xi = X[ip];
                yi = X[n + ip];
                zi = X[2 * n + ip];
                vxi = X[3 * n + ip];
                vyi = X[4 * n + ip];
                vzi = X[5 * n + ip];
                mi = X[6 * n + ip];
                if (F32) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        hi_i[q] = X32[q * n + ip];
                        lo_i[q] = X32[(3 + q) * n + ip];
                        v_i[q] = X32[(6 + q) * n + ip];
                    }
                    m32i = X32[9 * n + ip];
                }
            }
            double racc[6] = {0, 0, 0, 0, 0, 0};
            for (int k = kb; k < ke; ++k) {
                const int c = (lane + k) & 31;
                const int64_t j = 32 * Jt + c;
                const bool valid = irow && j < n && (!diag || c != lane);
                PairSolve ps;
                double mj = 0.0;
                bool lane32 = false;  // MIXED: solved in FP32
                float d32[6];
                if (valid) {
                    mj = cd[cb][6][c];
                    if (MIXED) {
                        const float hi_j[3] = {cf[cb][0][c], cf[cb][1][c], cf[cb][2][c]};
                        const float lo_j[3] = {cf[cb][3][c], cf[cb][4][c], cf[cb][5][c]};
                        const float v_j[3] = {cf[cb][6][c], cf[cb][7][c], cf[cb][8][c]};
                        Pair32 pr;
                        pair32_setup(pr, hi_i, lo_i, v_i, m32i, hi_j, lo_j, v_j, cf[cb][9][c],
                                     a.rule);
                        if (pr.fp32) {
                            int it32 = 0;
                            lane32 = pair32_solve(pr, a.t32, a.post32, a.guess, d32, it32);
                        }
                    }
                    if (!lane32)
                        pair_setup<kGrpEmu>(ps, a.tau, mi + mj, xi - cd[cb][0][c],
                                            yi - cd[cb][1][c], zi - cd[cb][2][c],
                                            vxi - cd[cb][3][c], vyi - cd[cb][4][c],
                                            vzi - cd[cb][5][c], a.pre,
                                            LEARNED ? 2 : (SEED ? -1 : a.guess));
                    if (SEED && !lane32) {
                        // single-precision seed: the root of the FP32 solve of
                        // the same pair (unless t was reduced modulo the period)
                        float dr[3], dv[3];
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            dr[q] = __fadd_rn(__fsub_rn(hi_i[q], cf[cb][q][c]),
                                              __fsub_rn(lo_i[q], cf[cb][3 + q][c]));
                            dv[q] = __fsub_rn(v_i[q], cf[cb][6 + q][c]);
                        }
                        const K32 o =
                            k32_phase1(dr, dv, m32i + cf[cb][9][c], a.ptau32, a.t32, 2);
                        if (o.ok && dbits(ps.t) == dbits(a.tau) &&
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
                }
                if (!valid || lane32) {
                    ps.done = true;
                    ps.beta = ps.s = 0.0;
                    ps.iters = 0;
                    ps.status = 0;
                }
                if (LEARNED) learned_guess_warp(ps, valid, *mlpW, mlpStage + wib * 32 * 16);
                double d[6];
                int iters = 0, fb = 0;
                fp64_solve_warp<SEED, kGrpEmu>(ps, valid && !lane32, a.tau, a.post * a.tau, kp,
                                               d, iters, fb);
                if (MIXED && lane32) {
                    // exact conversions on the integer pipe
#pragma unroll
                    for (int q = 0; q < 6; ++q) d[q] = f2d(d32[q]);
                }
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
                    n32 += lane32 ? (diag ? 1 : 2) : 0;  // in ordered pairs
                    it_sum += iters;
                    fallbacks += fb;
                    it_max = max(it_max, iters);
                    const int wmax = __reduce_max_sync(0xffffffffu, iters);
                    if (lane == 0) slots += 32LL * wmax;
                }
            }
            // the phase's row sums into the warp's row sums of the group
#pragma unroll
            for (int q = 0; q < 6; ++q) rs[wib][r][q][lane] += racc[q];
        }
        __syncthreads();  // every warp's sums of the window are complete
        GrpPos nxt{g, cur.t + wl, 0};
        if (nxt.t == nb - g * G) {
            nxt.g = g + 1;
            nxt.t = 0;
        }
        const int wln = in_range(nxt) ? window_len(nxt) : 0;
        // the window's column partials: the warps' sums added in warp order;
        // a phase entered after its step 0 goes to the block's colx slot
        for (int e = tid; e < wl * 192; e += G * 32) {
            const int cb = e / 192, rem = e - cb * 192, c = rem & 31, q = rem >> 5;
            double sum = cs[0][cb][q][c];
#pragma unroll
            for (int w = 1; w < G; ++w) sum += cs[w][cb][q][c];
            if (cb == 0 && kfirst > 0) {
                parts.colx[(b * 6 + q) * 32 + c] = sum;
            } else {
                const int64_t j = 32 * (J0 + cb) + c;
                if (j < n) parts.col[(g * 6 + q) * n + j] = sum;
            }
        }
        // leaving the group (or the range): the block's row piece of the
        // group, the warps' sums added in warp order (and cleared)
        if (nxt.g != g || wln == 0) {
            const int64_t h = b - grp_owner(grp_phase_x(L, g, 0), B, L);
            double *dst = parts.row + h * 6 * n;
            for (int e = tid; e < R * 192; e += G * 32) {
                const int r = e / 192, rem = e - r * 192, l = rem & 31, q = rem >> 5;
                const int64_t i = 32 * (g * G + r) + l;
                double sum = rs[0][r][q][l];
                rs[0][r][q][l] = 0.0;
#pragma unroll
                for (int w = 1; w < G; ++w) {
                    sum += rs[w][r][q][l];
                    rs[w][r][q][l] = 0.0;
                }
                if (i < n) dst[q * n + i] = sum;
            }
        }
        if (wln > 0) load_cols(nxt.g * G + nxt.t, wln);
        __syncthreads();  // the sums are read and the next column blocks stored
        cur = nxt;
        wl = wln;
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

namespace {

const void *grp_fp64_kernel(bool stats, bool learned, bool seed, bool mixed)
{
    if (mixed) {
        if (seed)
            return stats ? (const void *)pair_step_grp_kernel<true, false, true, true>
                         : (const void *)pair_step_grp_kernel<false, false, true, true>;
        return stats ? (const void *)pair_step_grp_kernel<true, false, false, true>
                     : (const void *)pair_step_grp_kernel<false, false, false, true>;
    }
    if (learned)
        return stats ? (const void *)pair_step_grp_kernel<true, true, false, false>
                     : (const void *)pair_step_grp_kernel<false, true, false, false>;
    if (seed)
        return stats ? (const void *)pair_step_grp_kernel<true, false, true, false>
                     : (const void *)pair_step_grp_kernel<false, false, true, false>;
    return stats ? (const void *)pair_step_grp_kernel<true, false, false, false>
                 : (const void *)pair_step_grp_kernel<false, false, false, false>;
}

}  // namespace

int pair_step_grp_blocks_per_sm(bool stats, bool learned, bool seed, bool mixed)
{
    learned = learned && !mixed;
    seed = seed && !learned;
    const void *fn = grp_fp64_kernel(stats, learned, seed, mixed);
    const size_t smem = grp_smem(learned, seed, mixed);
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

void launch_pair_step_grp(const StepArgs &a, const GrpLayout &L, const GrpParts &parts,
                          int blocks, bool stats, cudaStream_t s)
{
    const bool mixed = a.mixed != 0;
    const bool learned = !mixed && a.mlp != nullptr;
    const bool seed = !learned && a.X32 != nullptr && (!mixed || a.mixed == 2);
    const void *fn = grp_fp64_kernel(stats, learned, seed, mixed);
    const size_t smem = grp_smem(learned, seed, mixed);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    GrpLayout Lv = L;
    GrpParts pv = parts;
    void *args[] = {(void *)&a, (void *)&Lv, (void *)&pv};
    launch_pdl(fn, dim3(blocks), dim3(kFp64GrpWarps * 32), args, smem, s);
}

}  // namespace sakura
