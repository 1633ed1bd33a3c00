// kepler_df64.cuh -- the pair map of Eq. 26 with the Kepler flow of Eq. 18
// computed on the FP32 pipe to FP64 accuracy.
//
// Same method as kepler_fp64.cuh (universal variable s, F(s) = r0 s +
// eta0 G2 + zeta0 G3 - t, Stumpff functions by series with quartering and
// doubling, Laguerre steps of order 5 (Conway 1986), increments divided by
// m = m_i + m_j), organised in two phases:
//
//   1. FP32: the Kepler input from the leading float of each exact
//      double-word difference, then Laguerre iterations in single precision
//      until a step falls below 2^-8 of max(|s|, |t/F'|) (k32_solve).  This
//      finds the root to about 1e-7.
//   2. Double-word (df64.cuh): the Kepler input (backward drift, r0, 1/r0,
//      eta0, beta, zeta0), F, F' and F'' at s in double-word arithmetic and
//      one Laguerre correction ds = q (1 + k), q = F / F' in double-word form
//      and the small Laguerre factor k in float.  When |ds| <= 2^-20
//      max(|s|, |t/F'|) the truncation error of the cubically convergent
//      step is far below 2^-48 and G1..G3 and F' are carried to s - ds by their
//      Taylor series (dG_k/ds = G_{k-1}, G_0 = c0, dG_0/ds = -beta G1), with
//      first-order terms in double-word form; otherwise s - ds is evaluated
//      again (at most kDwMaxEval evaluations).
//
// A pair is solved this way only where single precision has the range for
// it (class test in dw_admit): 1e-30 < r0^2, v^2, m < 1e30, a bound orbit
// whose step is below 0.9 of its period (no reduction of t modulo the
// period), a converged FP32 phase and |beta s^2| <= 256 (hyperbolic G
// functions below e^16).  The caller solves every other pair with the FP64
// solver.  Every admitted increment is accurate to a few units of 2^-48
// relative, so the results match the FP64 solver within the per-step parity
// bound.
#pragma once

#include <cmath>

#include "df64.cuh"

namespace sakura {

constexpr int kDwMaxEval = 3;
constexpr int kDwFp32MaxIter = 12;

// double-word 1/(2n+2)! and 1/(2n+3)! (hi, lo), split from the exact values
#define SAKURA_DW_INV6 dw{0x1.555556p-3f, -0x1.555556p-28f}
#define SAKURA_DW_INV24 dw{0x1.555556p-5f, -0x1.555556p-30f}
#define SAKURA_DW_INV720 dw{0x1.6c16c2p-10f, -0x1.27d27ep-35f}
#define SAKURA_DW_INV120 dw{0x1.111112p-7f, -0x1.dddddep-32f}
#define SAKURA_DW_INV5040 dw{0x1.a01a02p-13f, -0x1.7f97fap-39f}

// --------------------------------------------------------------------------
// phase 1: single precision

struct K32 {
    float s;      // root estimate
    float x;      // beta s^2 at the estimate
    float beta;
    bool ok;      // converged (and finite)
    int iters;
};

DW_HD float stumpff32_terms(float x, float &c0, float &c1, float &c2)
{
    int k = 0;
    while (fabsf(x) > 0.1f && k < 40) {
        x = fmul(x, 0.25f);
        ++k;
    }
    const float y = -x;
    float s2 = ffma(ffma(ffma(1.0f / 40320.0f, y, 1.0f / 720.0f), y, 1.0f / 24.0f), y, 0.5f);
    float s3 = ffma(ffma(ffma(1.0f / 362880.0f, y, 1.0f / 5040.0f), y, 1.0f / 120.0f), y,
                    1.0f / 6.0f);
    float s0 = ffma(y, s2, 1.0f);
    float s1 = ffma(y, s3, 1.0f);
    for (; k > 0; --k) {
        const float n3 = fmul(0.25f, ffma(s0, s3, s2));
        const float n2 = fmul(fmul(0.5f, s1), s1);
        const float n1 = fmul(s0, s1);
        x = fmul(x, 4.0f);
        s0 = ffma(-x, n2, 1.0f);
        s1 = n1;
        s2 = n2;
        s3 = n3;
    }
    c0 = s0;
    c1 = s1;
    c2 = s2;
    return s3;
}

// Laguerre iterations in FP32 from the standard (guess 0) or second-order
// (guess 2) initial value (approximate reciprocals: this phase only needs
// the root to about 1e-7).  It stops after a Laguerre step below 2^-8 of
// the scale (the step taken), so a lane close to its root takes one
// evaluation and the warp seldom waits for a second.
DW_HD K32 k32_solve(float r0, float ir0, float eta, float beta, float zeta, float t, int guess)
{
    K32 o;
    o.beta = beta;
    float s = fmul(t, ir0);
    if (guess == 2) {
        const float c = fmul(fmul(0.5f, s), fmul(eta, ir0));
        if (fabsf(c) < 0.5f) s = ffma(-c, s, s);
    }
    o.ok = false;
    o.iters = 0;
    for (int it = 0; it < kDwFp32MaxIter; ++it) {
        float c0, c1, c2;
        const float s2 = fmul(s, s);
        const float c3 = stumpff32_terms(fmul(beta, s2), c0, c1, c2);
        const float G1 = fmul(s, c1), G2 = fmul(s2, c2), G3 = fmul(fmul(s2, s), c3);
        const float F = ffma(r0, s, ffma(eta, G2, ffma(zeta, G3, -t)));
        const float Fp = ffma(eta, G1, ffma(zeta, G2, r0));
        const float Fpp = ffma(eta, c0, fmul(zeta, G1));
        const float ir = rcp_approx(Fp);
        const float q = fmul(F, ir);
        ++o.iters;
        if (!(fabsf(q) <= 1e30f)) break;  // overflow or NaN
        // (no separate |q| test: a lane at its root takes a step of a few
        // ulps and stops below, so every lane follows one path)
        const float u = fmul(fmul(1.25f, q), fmul(Fpp, ir));
        const float den = ffma(4.0f, fsqrt_approx(fabsf(fsub(1.0f, u))), 1.0f);
        const float step = fmul(fmul(5.0f, q), rcp_approx(den));
        s = fsub(s, step);
        // a step below 2^-8 of the scale leaves the cubically convergent
        // iteration at single-precision round-off: accept without evaluating
        // again (only s is needed from this phase)
        if (fabsf(step) <= fmul(0x1p-8f, fmaxf(fabsf(s), fabsf(fmul(t, ir))))) {
            o.ok = true;
            break;
        }
    }
    o.s = s;
    o.x = fmul(fmul(beta, s), s);
    o.ok = o.ok && (fabsf(o.x) <= 256.0f) && fabsf(s) <= 3.0e38f;
    return o;
}

// --------------------------------------------------------------------------
// phase 2: double-word

struct PairDW {
    dw x0, y0, z0;   // backward-drifted relative position (Kepler input)
    dw vx, vy, vz;   // relative velocity
    dw m;            // m_i + m_j
    dw r0, ir0, eta0, beta, zeta0;
};

// Relative state from exact double-word differences rr, vv; ptau = pre tau.
DW_HD void dw_setup(PairDW &p, const dw rr[3], const dw vv[3], dw m, dw ptau)
{
    p.vx = vv[0];
    p.vy = vv[1];
    p.vz = vv[2];
    p.x0 = dw_sub(rr[0], dw_mul(ptau, vv[0]));
    p.y0 = dw_sub(rr[1], dw_mul(ptau, vv[1]));
    p.z0 = dw_sub(rr[2], dw_mul(ptau, vv[2]));
    p.m = m;
    const dw r2 = dw_add_nc(dw_add_nc(dw_sqr(p.x0), dw_sqr(p.y0)), dw_sqr(p.z0));
    p.ir0 = dw_rsqrt(r2);
    p.r0 = dw_mul(r2, p.ir0);
    p.eta0 = dw_add(dw_add(dw_mul(p.x0, p.vx), dw_mul(p.y0, p.vy)), dw_mul(p.z0, p.vz));
    const dw v2 = dw_add_nc(dw_add_nc(dw_sqr(p.vx), dw_sqr(p.vy)), dw_sqr(p.vz));
    p.beta = dw_sub(dw_scale(dw_mul(m, p.ir0), 2.0f), v2);
    p.zeta0 = dw_sub(m, dw_mul(p.beta, p.r0));
}

// c0..c3 at x in double-word form.  big (warp-uniform): some |x| of the warp
// exceeds 2^-8, so three double-word Horner steps are used (else two, which
// keep the float tail's error below 2^-49 for |x| < 2^-8); arguments above
// 0.1 are quartered first and doubled back.
struct StumpffDW {
    dw c0, c1, c2, c3;
};

DW_HD StumpffDW stumpff_dw(dw x, bool big)
{
    int k = 0;
    while (fabsf(x.h) > 0.1f && k < 16) {
        x = dw_scale(x, 0.25f);
        ++k;
    }
    const dw y = dw_neg(x);
    const float yf = y.h;
    // c2 = 1/2 + y (1/24 + y (1/720 + y (1/40320 + ...))), c3 likewise from
    // 1/6: the inner terms in float, the outer two or three in double-word;
    // |y| <= 0.1, so each constant outweighs the term added to it (no
    // cancellation)
    dw c2, c3;
    if (big) {
        const float t2 = ffma(ffma(1.0f / 479001600.0f, yf, 1.0f / 3628800.0f), yf,
                              1.0f / 40320.0f);
        const float t3 = ffma(ffma(1.0f / 6227020800.0f, yf, 1.0f / 39916800.0f), yf,
                              1.0f / 362880.0f);
        c2 = dw_add_nc(dw_mul(y, dw_add_nc(SAKURA_DW_INV720, dw_mul_f(y, t2))), SAKURA_DW_INV24);
        c3 = dw_add_nc(dw_mul(y, dw_add_nc(SAKURA_DW_INV5040, dw_mul_f(y, t3))),
                       SAKURA_DW_INV120);
    } else {
        const float t2 = ffma(ffma(1.0f / 3628800.0f, yf, 1.0f / 40320.0f), yf, 1.0f / 720.0f);
        const float t3 = ffma(ffma(1.0f / 39916800.0f, yf, 1.0f / 362880.0f), yf,
                              1.0f / 5040.0f);
        c2 = dw_add_nc(dw_mul_f(y, t2), SAKURA_DW_INV24);
        c3 = dw_add_nc(dw_mul_f(y, t3), SAKURA_DW_INV120);
    }
    c2 = dw_add_f(dw_mul(y, c2), 0.5f);
    c3 = dw_add_nc(dw_mul(y, c3), SAKURA_DW_INV6);
    dw c0 = dw_add_f(dw_mul(y, c2), 1.0f);
    dw c1 = dw_add_f(dw_mul(y, c3), 1.0f);
    for (; k > 0; --k) {
        const dw n3 = dw_scale(dw_add(dw_mul(c0, c3), c2), 0.25f);
        const dw n2 = dw_scale(dw_sqr(c1), 0.5f);
        const dw n1 = dw_mul(c0, c1);
        x = dw_scale(x, 4.0f);
        c0 = dw_add_f(dw_neg(dw_mul(x, n2)), 1.0f);
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    return {c0, c1, c2, c3};
}

struct EvalDW {
    dw G1, G2, G3, c0, Fp, Fpp;
    dw ds;         // Laguerre correction: the root is s - ds
    bool conv;     // |ds| small enough for the Taylor carry
};

DW_HD EvalDW dw_eval(const PairDW &p, dw s, dw t, bool big)
{
    EvalDW e;
    const dw s2 = dw_sqr(s);
    const StumpffDW c = stumpff_dw(dw_mul(p.beta, s2), big);
    e.c0 = c.c0;
    e.G1 = dw_mul(s, c.c1);
    e.G2 = dw_mul(s2, c.c2);
    e.G3 = dw_mul(dw_mul(s2, s), c.c3);
    const dw F = dw_sub(dw_add(dw_add(dw_mul(p.r0, s), dw_mul(p.eta0, e.G2)),
                               dw_mul(p.zeta0, e.G3)),
                        t);
    e.Fp = dw_add(dw_add(p.r0, dw_mul(p.eta0, e.G1)), dw_mul(p.zeta0, e.G2));
    e.Fpp = dw_add(dw_mul(p.eta0, c.c0), dw_mul(p.zeta0, e.G1));
    const dw ir = dw_rcp(e.Fp);
    const dw q = dw_mul(F, ir);
    // Laguerre factor of order 5 in float: ds = q (1 + k)
    const float u = fmul(fmul(1.25f, q.h), fmul(e.Fpp.h, ir.h));
    const float r = fsqrt_approx(fabsf(fsub(1.0f, u)));
    const float cf = fmul(fmul(0.8f, u), rcp_approx(fadd(1.0f, r)));
    const float k = fabsf(u) < 0.5f ? fmul(cf, rcp_approx(fsub(1.0f, cf)))
                                    : fsub(fmul(5.0f, rcp_approx(ffma(4.0f, r, 1.0f))), 1.0f);
    e.ds = dw_add_f(q, fmul(q.h, k));
    const float sc = fmaxf(fabsf(s.h), fabsf(fmul(t.h, ir.h)));
    e.conv = fabsf(e.ds.h) <= fmul(0x1p-20f, sc);
    return e;
}

// Carry G1..G3 and F' = r from s to s - ds (|ds| <= 2^-20 |s|): first-order
// terms in double-word form, second-order terms in float.  (The first-order
// terms are small next to the values, which keeps the sums free of
// cancellation.)
DW_HD void dw_carry(EvalDW &e, const PairDW &p)
{
    const dw d = e.ds;
    const float h2 = fmul(fmul(0.5f, d.h), d.h);
    const dw G0 = e.c0;
    const float Gm1 = fmul(-p.beta.h, e.G1.h);  // dG0/ds
    const float F3 = ffma(fmul(-p.eta0.h, p.beta.h), e.G1.h, fmul(p.zeta0.h, G0.h));  // dF''/ds
    // each first-order term is at most about 2^-18 of the value it corrects
    // (|ds| <= 2^-20 |s|), so an unnormalised product suffices and the
    // subtraction cannot cancel
    e.G3 = dw_add_f(dw_add_nc(e.G3, dw_neg(dw_mul(d, e.G2))), fmul(h2, e.G1.h));
    e.G2 = dw_add_f(dw_add_nc(e.G2, dw_neg(dw_mul(d, e.G1))), fmul(h2, G0.h));
    e.G1 = dw_add_f(dw_add_nc(e.G1, dw_neg(dw_mul(d, G0))), fmul(h2, Gm1));
    e.Fp = dw_add_f(dw_add_nc(e.Fp, dw_neg(dw_mul(d, e.Fpp))), fmul(h2, F3));
}

// Increments of the pair map (Eq. 26, increment form) divided by m, from
// the G functions and r = F' at the root; qtau = post tau.
DW_HD void dw_increment_over_m(const PairDW &p, const EvalDW &e, dw qtau,
                                                    dw out[6])
{
    const dw ir = dw_rcp(e.Fp);
    const dw fm1 = dw_neg(dw_mul(e.G2, p.ir0));
    const dw gmt = dw_neg(e.G3);
    const dw fd = dw_neg(dw_mul(dw_mul(e.G1, p.ir0), ir));
    const dw gdm1 = dw_neg(dw_mul(e.G2, ir));
    const dw A = dw_sub(fm1, dw_mul(qtau, fd));
    const dw B = dw_sub(gmt, dw_mul(qtau, gdm1));
    out[3] = dw_add(dw_mul(fd, p.x0), dw_mul(gdm1, p.vx));
    out[4] = dw_add(dw_mul(fd, p.y0), dw_mul(gdm1, p.vy));
    out[5] = dw_add(dw_mul(fd, p.z0), dw_mul(gdm1, p.vz));
    out[0] = dw_add(dw_mul(A, p.x0), dw_mul(B, p.vx));
    out[1] = dw_add(dw_mul(A, p.y0), dw_mul(B, p.vy));
    out[2] = dw_add(dw_mul(A, p.z0), dw_mul(B, p.vz));
}

// Phase 1 with the class test from float relative coordinates dr, dv (after
// the one-subscript drift), float m = m_i + m_j, ptau32 = (float)(pre tau),
// t32 = (float)tau: the backward drift, the range and period conditions and
// the FP32 solve.  Also the single-precision seed of the FP64 solver.
DW_HD K32 k32_phase1(const float dr[3], const float dv[3], float m, float ptau32, float t32,
                     int guess)
{
    float x[3];
    for (int q = 0; q < 3; ++q) x[q] = ffma(-ptau32, dv[q], dr[q]);
    const float r2 = ffma(x[0], x[0], ffma(x[1], x[1], fmul(x[2], x[2])));
    const float v2 = ffma(dv[0], dv[0], ffma(dv[1], dv[1], fmul(dv[2], dv[2])));
    const float eta = ffma(x[0], dv[0], ffma(x[1], dv[1], fmul(x[2], dv[2])));
    const bool range = r2 > 1e-30f && r2 < 1e30f && v2 < 1e30f && m > 1e-30f && m < 1e30f;
    K32 o;
    o.ok = false;
    o.iters = 0;
    o.s = 0.0f;
    o.x = 0.0f;
    o.beta = 0.0f;
    if (!range) return o;
    const float ir0 = rsqrt_approx(r2);
    const float r0 = fmul(r2, ir0);
    const float beta = ffma(fmul(2.0f, m), ir0, -v2);
    const float zeta = ffma(-beta, r0, m);
    // a bound orbit whose step exceeds 0.9 of its period needs t reduced
    // modulo the period: FP64 solver
    if (beta > 0.0f) {
        const float b3 = fmul(fmul(beta, beta), beta);
        const float tm = fmul(6.2831853f * 0.9f, m);
        if (fmul(fmul(t32, t32), b3) >= fmul(tm, tm)) return o;
    }
    return k32_solve(r0, ir0, eta, beta, zeta, t32, guess);
}

// Phase 1 for the double-word form: the leading floats of the exact
// double-word differences rr, vv and of m.
DW_HD K32 dw_phase1(const dw rr[3], const dw vv[3], dw m, float ptau32, float t32, int guess)
{
    const float dr[3] = {rr[0].h, rr[1].h, rr[2].h};
    const float dv[3] = {vv[0].h, vv[1].h, vv[2].h};
    return k32_phase1(dr, dv, m.h, ptau32, t32, guess);
}

// Phase 2 for an admitted pair: setup, evaluations from s32, Taylor carry
// and increments over m.  Returns false when kDwMaxEval evaluations did not
// reach the carry condition (the caller then uses the FP64 solver).
DW_HD bool dw_phase2(const dw rr[3], const dw vv[3], dw m, dw ptau, dw t, dw qtau, float s32,
                     bool big, dw out[6], int &evals)
{
    PairDW p;
    dw_setup(p, rr, vv, m, ptau);
    dw s = dw_from(s32);
    EvalDW e;
    evals = 0;
    for (;;) {
        e = dw_eval(p, s, t, big);
        ++evals;
        if (e.conv) break;
        if (evals >= kDwMaxEval) return false;
        s = dw_sub(s, e.ds);
    }
    dw_carry(e, p);
    dw_increment_over_m(p, e, qtau, out);
    return true;
}

// acc += p with renormalisation
DW_HD void dw_acc(dw &acc, dw p)
{
    const dw s = two_sum(acc.h, p.h);
    acc = fast_two_sum(s.h, fadd(s.l, fadd(acc.l, p.l)));
}

}  // namespace sakura
