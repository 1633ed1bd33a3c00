// pair_batch_fp64.cuh -- one warp-wide batch of FP64 pair solves.
#pragma once

#include "kepler_fp64.cuh"
#include "mlp_infer.cuh"
#include "step_common.cuh"

namespace sakura {

// Warp-synchronous FP64 solve of 32 pairs, one per lane, whose setup is
// done (lanes with p.done == true at entry idle).  Every lane of the warp must
// call this.  tau, qtau: this lane's step and post-drift time (post * tau).  Writes
// the increments divided by m_ij to d (only meaningful when valid), returns
// the lane's evaluation count and whether it needed bisection.
template <bool CARRY = false, int EMU = 0>
__device__ __forceinline__ void fp64_solve_warp(PairSolve &p, bool valid, double tau,
                                                double qtau, const KeplerParams &kp,
                                                double d[6], int &iters, int &fb)
{
    for (int it = 0; it < kp.max_iter; ++it) {
        if (__all_sync(0xffffffffu, p.done)) break;
        const double s2 = xmul<EMU, kEmuIterMul>(p.s, p.s);
        const double x = xmul<EMU, kEmuIterMul>(p.beta, s2);
        const unsigned hx = p.done ? 0u : abs_hiword(x);
        const int nt = stumpff_terms(__reduce_max_sync(0xffffffffu, hx));
        bool oob = false;
        if (!p.done) oob = pair_iterate<CARRY, EMU>(p, x, s2, nt, kp);
        if (__any_sync(0xffffffffu, oob)) {
            if (oob) pair_safeguard(p);
        }
    }
    fb = 0;
    if (!p.done) {
        if (kp.bisection) {
            pair_bisect(p);
            fb = 1;
        } else {
            p.status |= kStatusKepler;
        }
    }
    iters = valid ? p.iters : 0;
    if (valid) pair_increment_over_m<EMU>(p, tau, qtau, d);
}

// Learned initial guess for the 32 lanes (every lane calls): replaces the
// second-order guess p.s of valid, unfinished lanes by s_T2 exp(w g(x))
// (mlp_infer.cuh).  The sign of s is kept, so the bracket stays valid.  The
// network changes log s by at most 4w, and where every lane of the warp has
// w <= kLearnedMinGate the second-order guess is already accurate to about w
// (one Laguerre step then reaches the FP64 root), so the warp skips the
// network.
constexpr float kLearnedMinGate = 1e-4f;

__device__ __forceinline__ void learned_guess_warp(PairSolve &p, bool valid, const MlpWeights &W,
                                                   __nv_bfloat16 *stage)
{
    GuessVars gv;
    gv.w = 0.0f;
    bool use = false;
    if (valid && !p.done) use = guess_gate(p.t, p.m, p.r0, p.ir0, p.eta0, p.beta, gv);
    if (!__any_sync(0xffffffffu, use && gv.w > kLearnedMinGate)) return;
    float f[6] = {0, 0, 0, 0, 0, 0};
    if (use) guess_features_from(gv, f);
    const float g = mlp_eval_warp(W, stage, f);
    if (use) p.s *= (double)__expf(gv.w * g);
}

// 32 ordered pairs (i, j_lane) of one row, one per lane; every lane of the
// warp must call this (invalid lanes idle).  X is the drifted state
// [7][n].  Adds m_j (delta_r, delta_v) / m_ij to acc (Eq. 23 with the
// 1/m_i folded in), ORs device faults into status, and returns the lane's
// Kepler evaluation count and whether it needed bisection.  With LEARNED the
// setup uses the second-order guess refined by the network in W.
template <bool LEARNED = false>
__device__ __forceinline__ void fp64_pair_batch(const double *X, int64_t n, int64_t j, bool valid,
                                                double xi, double yi, double zi, double vxi,
                                                double vyi, double vzi, double mi,
                                                const StepArgs &a, const KeplerParams &kp,
                                                double acc[6], unsigned &status, int &iters,
                                                int &fb, const MlpWeights *W = nullptr,
                                                __nv_bfloat16 *stage = nullptr)
{
    PairSolve p;
    double mj = 0.0;
    if (valid) {
        mj = X[6 * n + j];
        pair_setup(p, a.tau, mi + mj, xi - X[j], yi - X[n + j], zi - X[2 * n + j],
                   vxi - X[3 * n + j], vyi - X[4 * n + j], vzi - X[5 * n + j], a.pre,
                   LEARNED ? 2 : a.guess);
    } else {
        p.done = true;
        p.beta = p.s = 0.0;
        p.iters = 0;
        p.status = 0;
    }
    if (LEARNED) learned_guess_warp(p, valid, *W, stage);
    double d[6];
    fp64_solve_warp(p, valid, a.tau, a.post * a.tau, kp, d, iters, fb);
    if (valid) {
#pragma unroll
        for (int q = 0; q < 6; ++q) acc[q] = fma(mj, d[q], acc[q]);
        status |= p.status;
    }
}

}  // namespace sakura
