// kepler_fp64.cuh -- FP64 device math of the Sakura pair map.
//
// One ordered pair (i, j) of the W step (Eq. 14, increments by Eq. 23):
//   rr0 = r_i - r_j, vv0 = v_i - v_j                        (after the drift)
//   r0  = rr0 - pre*tau*vv0, v0 = vv0                       (Eq. 17, backward drift)
//   (r1, v1) = kepler_solver(tau, m_i + m_j, r0, v0)        (Eq. 18)
//   rr1 = r1 - post*tau*v1                                  (Eq. 17)
//   delta_r = rr1 - rr0, delta_v = v1 - vv0
// with (pre, post) = (1/2, 1/2) for Eq. 26, (0, 1) for Eq. 19a and (1, 0)
// for Eq. 19b.  Because pre + post = 1 the increments are formed directly
// from the small Lagrange coefficients f-1, g-tau, fdot, gdot-1,
//   delta_v = fdot r0 + (gdot-1) v0
//   delta_r = ((f-1) - post*tau*fdot) r0 + ((g-tau) - post*tau*(gdot-1)) v0,
// which never subtracts two nearly equal positions.
//
// Kepler flow in the universal variable s (ds/dt = 1/r):
//   t(s) = r0 s + eta0 G2(s) + zeta0 G3(s),  r(s) = r0 + eta0 G1 + zeta0 G2,
//   G_k(s) = s^k c_k(beta s^2), beta = 2m/r0 - v0^2, eta0 = r0.v0,
//   zeta0 = m - beta r0,
//   f - 1 = -m G2 / r0, g - t = -m G3, fdot = -m G1 / (r0 r), gdot - 1 = -m G2 / r.
// The root of F(s) = t(s) - t is found by Laguerre's method of order 5
// (Conway 1986), with a bracket safeguard and a bisection fallback.  F is
// strictly increasing (F' = r > 0) so the root is unique.
//
// Stumpff functions c_k(x) = sum_n (-x)^n / (k+2n)!: the argument is
// quartered until |x| <= 0.1, the series for c2 and c3 is summed to 7 terms
// (truncation < 1e-17 relative), c0 = 1 - x c2 and c1 = 1 - x c3, and the
// quarterings are undone with the doubling identities
//   c0(4x) = 1 - 4x c2(4x), c1(4x) = c0 c1, c2(4x) = c1^2 / 2,
//   c3(4x) = (c2 + c0 c3) / 4.
// No trigonometric or hyperbolic function is called, and the common case
// (|x| <= 0.1) takes no branch.
#pragma once

#include <cstdint>

namespace sakura {

constexpr double kPi = 3.14159265358979323846;

// status bits written to the device status word
constexpr unsigned kStatusCoincident = 1u;
constexpr unsigned kStatusNonfinite = 2u;
constexpr unsigned kStatusKepler = 4u;
constexpr unsigned kStatusMass = 8u;
constexpr unsigned kStatusTimeout = 16u;

struct Stumpff {
    double c0, c1, c2, c3;
};

__device__ __forceinline__ Stumpff stumpff_fp64(double x)
{
    int k = 0;
    while (fabs(x) > 0.1 && k < 80) {
        x *= 0.25;
        ++k;
    }
    const double y = -x;
    // 1/(2n+2)! and 1/(2n+3)!, n = 0..6
    double c2 = 1.0 / 87178291200.0;
    c2 = fma(c2, y, 1.0 / 479001600.0);
    c2 = fma(c2, y, 1.0 / 3628800.0);
    c2 = fma(c2, y, 1.0 / 40320.0);
    c2 = fma(c2, y, 1.0 / 720.0);
    c2 = fma(c2, y, 1.0 / 24.0);
    c2 = fma(c2, y, 1.0 / 2.0);
    double c3 = 1.0 / 1307674368000.0;
    c3 = fma(c3, y, 1.0 / 6227020800.0);
    c3 = fma(c3, y, 1.0 / 39916800.0);
    c3 = fma(c3, y, 1.0 / 362880.0);
    c3 = fma(c3, y, 1.0 / 5040.0);
    c3 = fma(c3, y, 1.0 / 120.0);
    c3 = fma(c3, y, 1.0 / 6.0);
    double c0 = fma(y, c2, 1.0);
    double c1 = fma(y, c3, 1.0);
    for (; k > 0; --k) {
        const double n3 = 0.25 * fma(c0, c3, c2);
        const double n2 = 0.5 * c1 * c1;
        const double n1 = c0 * c1;
        x *= 4.0;
        c0 = fma(-x, n2, 1.0);
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    return {c0, c1, c2, c3};
}

struct KeplerParams {
    double tol;       // kepler_tol * DBL_EPSILON
    int max_iter;     // Laguerre steps before bisection
    int bisection;    // 1: bisection fallback
};

struct PairResult {
    double dr[3];
    double dv[3];
    int iters;
    int fallback;
    unsigned status;
};

// Universal functions G0..G3 at s, and F, F', F''.
struct KepEval {
    double G0, G1, G2, G3, F, Fp, Fpp;
};

__device__ __forceinline__ KepEval kep_eval_fp64(double s, double beta, double r0, double eta0,
                                                 double zeta0, double t)
{
    const Stumpff c = stumpff_fp64(beta * s * s);
    KepEval e;
    const double s2 = s * s;
    e.G0 = c.c0;
    e.G1 = s * c.c1;
    e.G2 = s2 * c.c2;
    e.G3 = s2 * s * c.c3;
    e.F = fma(r0, s, fma(eta0, e.G2, fma(zeta0, e.G3, -t)));
    e.Fp = fma(eta0, e.G1, fma(zeta0, e.G2, r0));
    e.Fpp = fma(eta0, e.G0, zeta0 * e.G1);
    return e;
}

// Pair increments (delta_r, delta_v) of one ordered pair, see the file header.
// rr0, vv0: relative state after the one-subscript drift; m: m_i + m_j.
__device__ __forceinline__ PairResult pair_increment_fp64(double tau, double m, double rx,
                                                          double ry, double rz, double vx,
                                                          double vy, double vz, double pre,
                                                          double post, const KeplerParams &kp)
{
    PairResult out;
    out.iters = 0;
    out.fallback = 0;
    out.status = 0;
    // Eq. 17: backward drift before the Kepler flow
    const double ptau = pre * tau;
    const double x0 = fma(-ptau, vx, rx);
    const double y0 = fma(-ptau, vy, ry);
    const double z0 = fma(-ptau, vz, rz);
    const double r0sq = fma(x0, x0, fma(y0, y0, z0 * z0));
    if (!(r0sq > 0.0)) {
        out.status = (r0sq == 0.0) ? kStatusCoincident : kStatusNonfinite;
        for (int q = 0; q < 3; ++q) out.dr[q] = out.dv[q] = 0.0;
        return out;
    }
    const double r0 = sqrt(r0sq);
    const double ir0 = 1.0 / r0;
    const double eta0 = fma(x0, vx, fma(y0, vy, z0 * vz));
    const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
    const double beta = fma(2.0 * m, ir0, -v2);
    const double zeta0 = fma(-beta, r0, m);
    double t = tau;
    if (beta > 0.0) {
        const double P = 2.0 * kPi * m / (beta * sqrt(beta));
        if (fabs(t) > P) t = fmod(t, P);
    }

    KepEval e{0.0, 0.0, 0.0, 0.0, 0.0, r0, 0.0};
    if (t != 0.0) {
        double s = t * ir0;  // standard initial guess
        double lo, hi;
        if (t > 0.0) {
            lo = 0.0;
            hi = __longlong_as_double(0x7ff0000000000000LL);
        } else {
            lo = -__longlong_as_double(0x7ff0000000000000LL);
            hi = 0.0;
        }
        bool done = false;
        int it = 0;
        for (; it < kp.max_iter; ++it) {
            e = kep_eval_fp64(s, beta, r0, eta0, zeta0, t);
            const double scale = fmax(fabs(t), r0 * fabs(s));
            if (fabs(e.F) <= kp.tol * scale) {
                done = true;
                ++it;
                break;
            }
            if (e.F < 0.0)
                lo = s;
            else
                hi = s;
            const double disc = fma(16.0 * e.Fp, e.Fp, -20.0 * e.F * e.Fpp);
            const double den = e.Fp + copysign(sqrt(fabs(disc)), e.Fp);
            const double ds = 5.0 * e.F / den;
            double sn = s - ds;
            if (fabs(ds) <= kp.tol * fabs(sn)) {
                done = true;
                ++it;
                break;
            }
            if (!(sn > lo && sn < hi)) {
                if (isinf(hi))
                    sn = 2.0 * fmax(lo, s);
                else if (isinf(lo))
                    sn = 2.0 * fmin(hi, s);
                else
                    sn = 0.5 * (lo + hi);
            }
            s = sn;
        }
        out.iters = it;
        if (!done) {
            if (!kp.bisection) {
                out.status |= kStatusKepler;
            } else {
                // expand an open bracket, then bisect to about two ulp
                out.fallback = 1;
                for (int q = 0; q < 2100 && isinf(hi); ++q) {
                    const double c = 2.0 * fmax(lo, fabs(t) * ir0);
                    e = kep_eval_fp64(c, beta, r0, eta0, zeta0, t);
                    if (e.F < 0.0) lo = c; else hi = c;
                }
                for (int q = 0; q < 2100 && isinf(lo); ++q) {
                    const double c = 2.0 * fmin(hi, -fabs(t) * ir0);
                    e = kep_eval_fp64(c, beta, r0, eta0, zeta0, t);
                    if (e.F > 0.0) hi = c; else lo = c;
                }
                double mid = 0.5 * (lo + hi);
                for (int q = 0; q < 2200; ++q) {
                    mid = 0.5 * (lo + hi);
                    if (!(mid > lo && mid < hi)) break;
                    if (hi - lo <= 2.2204460492503131e-16 * 2.0 * fmax(fabs(lo), fabs(hi))) break;
                    e = kep_eval_fp64(mid, beta, r0, eta0, zeta0, t);
                    if (e.F < 0.0) lo = mid;
                    else if (e.F > 0.0) hi = mid;
                    else break;
                    ++out.iters;
                }
                e = kep_eval_fp64(mid, beta, r0, eta0, zeta0, t);
                if (isinf(lo) || isinf(hi)) out.status |= kStatusKepler;
            }
        }
    }
    // Lagrange coefficients in increment form
    const double r = e.Fp;
    const double ir = 1.0 / r;
    const double mG2 = m * e.G2;
    const double fm1 = -mG2 * ir0;
    const double gmt = (t - tau) - m * e.G3;
    const double fd = -m * e.G1 * ir0 * ir;
    const double gdm1 = -mG2 * ir;
    const double qtau = post * tau;
    const double A = fma(-qtau, fd, fm1);
    const double B = fma(-qtau, gdm1, gmt);
    out.dv[0] = fma(fd, x0, gdm1 * vx);
    out.dv[1] = fma(fd, y0, gdm1 * vy);
    out.dv[2] = fma(fd, z0, gdm1 * vz);
    out.dr[0] = fma(A, x0, B * vx);
    out.dr[1] = fma(A, y0, B * vy);
    out.dr[2] = fma(A, z0, B * vz);
    return out;
}

}  // namespace sakura
