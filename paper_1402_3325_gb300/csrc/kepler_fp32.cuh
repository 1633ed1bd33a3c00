// kepler_fp32.cuh -- single-precision pair solve of the mixed-precision form.
//
// Same method as kepler_fp64.cuh (universal variable, Stumpff functions by
// quartering and doubling, Laguerre n = 5 with the Newton-step convergence
// test, increment form of the Eq. 26 pair map divided by m = m_i + m_j), in
// FP32 throughout.  A lane stops after a Laguerre step below 2^-11 of the
// scale max(|s|, |t| |1/F'|): the step is taken and G1..G3 and F' carried to
// it by a Taylor series (a lane already at its root takes a step of a few
// ulps or zero).  One stopping rule for every lane keeps the warp on one
// path; a separate |F/F'| test for lanes already at the root split the warp
// and made the symmetric mixed kernel 25 % slower on GB300.  A lane that has
// not converged after kFp32MaxIter steps is handed to the FP64 solver.  The solve's
// reciprocals and square root are the hardware approximations (about 1 ulp).
// Only pairs that the FP32 class rule admits (distant, low- or
// very-high-eccentricity pairs, whose increments are small next to the state)
// come here; the caller accumulates their increments (in FP64, or as exact
// double-word sums of the float products, step_mixed.cu).
//
// The class rule is stated on the pair's Kepler input (r0, v0) of Eq. 26
// with m = m_i + m_j: r = |r0|, e^2 = 1 + 2 E h^2 / m^2, E = v0^2/2 - m/r,
// h^2 = r^2 v0^2 - (r0.v0)^2.  It is decided in single precision on the
// hi/lo float split of the drifted positions, multiplied through by m^2 > 0
// so that no division or square root is needed:
//   e < e_max  <=>  (v0^2 - 2m/r) h^2 < (e_max^2 - 1) m^2,  likewise e > e_hyp,
// with 1/r from the hardware reciprocal square root.  Pairs next to a
// threshold may fall either way (a pair of either class is solved
// correctly); away from the thresholds' rounding band the decision equals the
// double-precision rule's (tested against the oracle pair by pair).
#pragma once

#include <cstdint>

#include "df64.cuh"

namespace sakura {

constexpr int kFp32MaxIter = 12;

// Relative Kepler input of a pair in FP32 and the class decision.
struct Pair32 {
    float x0, y0, z0, vx, vy, vz;  // r0 (backward-drifted) and v0
    float r2, v2, eta, m;
    bool fp32;                      // admitted by the FP32 class rule
};

struct ClassRule {
    float ptau;     // (float)(pre * tau)
    float rmin2;    // (float)(r_min^2)
    float emax2m1;  // (float)(e_max^2 - 1)
    float ehyp2m1;  // (float)(e_hyp^2 - 1)
    int rule;       // 0: r > r_min and e < e_max; 1: ... or e > e_hyp
};

// dx = (hi_i - hi_j) + (lo_i - lo_j) for each coordinate (the separation to
// the accuracy of the separation), dv in float, r0 = dx - ptau dv, then the
// class.  The decision is symmetric in (i, j): every quantity it uses is
// even under (r0, v0) -> (-r0, -v0), and negation commutes with rounding.
// Pair masses with m^2 below 2^-120 (out of single precision's normal
// range) stay in FP64.
__device__ __forceinline__ void pair32_setup(Pair32 &p, const float hi_i[3], const float lo_i[3],
                                             const float v_i[3], float m_i, const float hi_j[3],
                                             const float lo_j[3], const float v_j[3], float m_j,
                                             const ClassRule &cr)
{
    float x[3], u[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float d = (hi_i[q] - hi_j[q]) + (lo_i[q] - lo_j[q]);
        u[q] = v_i[q] - v_j[q];
        x[q] = fmaf(-cr.ptau, u[q], d);
    }
    p.x0 = x[0];
    p.y0 = x[1];
    p.z0 = x[2];
    p.vx = u[0];
    p.vy = u[1];
    p.vz = u[2];
    p.r2 = fmaf(x[0], x[0], fmaf(x[1], x[1], x[2] * x[2]));
    p.v2 = fmaf(u[0], u[0], fmaf(u[1], u[1], u[2] * u[2]));
    p.eta = fmaf(x[0], u[0], fmaf(x[1], u[1], x[2] * u[2]));
    p.m = m_i + m_j;
    const float h2 = fmaf(p.r2, p.v2, -(p.eta * p.eta));
    const float twoE = fmaf(-2.0f * p.m, rsqrtf(p.r2), p.v2);
    const float lhs = twoE * h2;
    const float m2 = p.m * p.m;
    const bool far = p.r2 > cr.rmin2;
    const bool lowe = lhs < cr.emax2m1 * m2;
    const bool hyp = (cr.rule == 1) && (lhs > cr.ehyp2m1 * m2);
    p.fp32 = far && m2 >= 0x1p-120f && (lowe || hyp);
}

struct Stumpff32 {
    float c0, c1, c2, c3;
};

__device__ __forceinline__ Stumpff32 stumpff_fp32(float x)
{
    int k = 0;
    while (fabsf(x) > 0.1f && k < 40) {
        x *= 0.25f;
        ++k;
    }
    const float y = -x;
    // 1/(2n+2)!, 1/(2n+3)!, n = 0..3 (first omitted term < 3e-11 relative)
    float c2 = fmaf(fmaf(fmaf(1.0f / 40320.0f, y, 1.0f / 720.0f), y, 1.0f / 24.0f), y, 0.5f);
    float c3 = fmaf(fmaf(fmaf(1.0f / 362880.0f, y, 1.0f / 5040.0f), y, 1.0f / 120.0f), y,
                    1.0f / 6.0f);
    float c0 = fmaf(y, c2, 1.0f);
    float c1 = fmaf(y, c3, 1.0f);
    for (; k > 0; --k) {
        const float n3 = 0.25f * fmaf(c0, c3, c2);
        const float n2 = 0.5f * c1 * c1;
        const float n1 = c0 * c1;
        x *= 4.0f;
        c0 = fmaf(-x, n2, 1.0f);
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    return {c0, c1, c2, c3};
}

// FP32 Kepler solve and increments divided by m; returns false when the
// iteration did not converge (the pair then goes to the FP64 solver).
// guess: 0 = t/r0, 2 = second order.  out[0..2] = delta_r/m,
// out[3..5] = delta_v/m.
__device__ __forceinline__ bool pair32_solve(const Pair32 &p, float tau, float post, int guess,
                                             float out[6], int &iters)
{
    const float ir0 = rsqrtf(p.r2);
    const float r0 = p.r2 * ir0;
    const float beta = fmaf(2.0f * p.m, ir0, -p.v2);
    const float zeta0 = fmaf(-beta, r0, p.m);
    float t = tau;
    if (beta > 0.0f) {
        const float b3 = beta * beta * beta;
        const float tm = 6.2831853f * p.m;
        if (tau * tau * b3 > tm * tm) t = fmodf(tau, tm * rsqrtf(b3));
    }
    float s = t * ir0;
    if (guess == 2) {
        const float c = 0.5f * s * (p.eta * ir0);
        if (fabsf(c) < 0.5f) s = fmaf(-c, s, s);
    }
    float G1 = 0.0f, G2 = 0.0f, G3 = 0.0f, ir = ir0;
    bool done = (t == 0.0f);
    iters = 0;
    for (int it = 0; it < kFp32MaxIter && !done; ++it) {
        const Stumpff32 c = stumpff_fp32(beta * s * s);
        const float s2 = s * s;
        G1 = s * c.c1;
        G2 = s2 * c.c2;
        G3 = s2 * s * c.c3;
        const float F = fmaf(r0, s, fmaf(p.eta, G2, fmaf(zeta0, G3, -t)));
        const float Fp = fmaf(p.eta, G1, fmaf(zeta0, G2, r0));
        const float Fpp = fmaf(p.eta, c.c0, zeta0 * G1);
        ir = rcp_approx(Fp);
        const float q = F * ir;
        ++iters;
        const float u = 1.25f * q * Fpp * ir;
        const float den = 1.0f + 4.0f * fsqrt_approx(fabsf(1.0f - u));
        const float step = 5.0f * q * rcp_approx(den);
        s = s - step;
        // a Laguerre step below 2^-11 of the scale: the root is reached to
        // single-precision round-off, so carry G1..G3 and F' = r to it by
        // their Taylor series (dG_k/ds = G_{k-1}, G_0 = c0, dG_0/ds = -beta
        // G1) instead of evaluating again; lanes near their root then finish
        // together
        if (fabsf(step) <= 0x1p-11f * fmaxf(fabsf(s), fabsf(t * ir))) {
            const float h2 = 0.5f * step * step;
            const float F3 = fmaf(-p.eta * beta, G1, zeta0 * c.c0);  // dF''/ds
            const float nG3 = fmaf(h2, G1, fmaf(-step, G2, G3));
            const float nG2 = fmaf(h2, c.c0, fmaf(-step, G1, G2));
            const float nG1 = fmaf(h2, -beta * G1, fmaf(-step, c.c0, G1));
            ir = rcp_approx(fmaf(h2, F3, fmaf(-step, Fpp, Fp)));
            G1 = nG1;
            G2 = nG2;
            G3 = nG3;
            done = true;
            break;
        }
    }
    if (!done) return false;
    const float fm1 = -G2 * ir0;
    float gmt = -G3;
    if (t != tau) gmt += (t - tau) / p.m;
    const float fd = -G1 * ir0 * ir;
    const float gdm1 = -G2 * ir;
    const float qtau = post * tau;
    const float A = fmaf(-qtau, fd, fm1);
    const float B = fmaf(-qtau, gdm1, gmt);
    out[3] = fmaf(fd, p.x0, gdm1 * p.vx);
    out[4] = fmaf(fd, p.y0, gdm1 * p.vy);
    out[5] = fmaf(fd, p.z0, gdm1 * p.vz);
    out[0] = fmaf(A, p.x0, B * p.vx);
    out[1] = fmaf(A, p.y0, B * p.vy);
    out[2] = fmaf(A, p.z0, B * p.vz);
    return isfinite(out[0] + out[1] + out[2] + out[3] + out[4] + out[5]);
}

}  // namespace sakura
