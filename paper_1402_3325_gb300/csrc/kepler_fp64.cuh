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
// which never subtracts two nearly equal positions.  Every coefficient is
// proportional to m = m_i + m_j except the period-reduction term (t - tau),
// so the kernel forms delta / m and weights it by m_j: mu_ij delta / m_i =
// m_j (delta / m), which is the Eq. 23 increment without a division.
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
// Laguerre step (n = 5, F' > 0):
//   ds = 5F / (F' + 4 F' sqrt|1 - u|),  u = (5/4) F F'' / F'^2,
// rewritten with q = F / F' (the Newton step) as ds = q (1 + k),
// k = c / (1 - c), c = (4/5) u / (1 + sqrt(1 - u)) for |u| < 1/2 (and
// k = 5 / (1 + 4 sqrt|1 - u|) - 1 otherwise, far from the root).  q is FP64;
// k is a correction of size O(u) = O(F) and is formed in FP32, so its
// rounding vanishes as F -> 0 and the iteration keeps its cubic convergence
// to the FP64 root.
//
// Convergence: the Newton step q = F / F' is the first-order estimate of the
// remaining |s - root|; a lane stops when |q| <= tol max(|s|, |t| / r), i.e.
// |ds| <= 4 eps |s| or |F| <= 4 eps max(r |s|, |t|).
//
// Stumpff functions c_k(x) = sum_n (-x)^n / (k+2n)!: the argument is
// quartered until |x| <= 0.1, the series for c2 and c3 is summed with a
// warp-uniform number of terms chosen from the largest |x| in the warp
// (3 terms up to 1e-4, 4 up to 3e-3, 5 up to 2.5e-2, 6 up to 0.1; the first
// omitted term is below 2^-55 relative), c0 = 1 - x c2, c1 = 1 - x c3, and
// the quarterings are undone with the doubling identities
//   c0(4x) = 1 - 4x c2(4x), c1(4x) = c0 c1, c2(4x) = c1^2 / 2,
//   c3(4x) = (c2 + c0 c3) / 4.
// No trigonometric or hyperbolic function is called.
//
// Reciprocals and reciprocal square roots start from the single-precision
// hardware approximation of the operand truncated to float (relative error
// about 2^-22; the FP64 approximations, rcp/rsqrt.approx.ftz.f64 with error
// below 2^-19, only for operands outside float's range: they measured about
// 5 % of the pair kernel's time as seeds) and take one third-order step of
// the Newton-Raphson family (Householder order 2),
//   y <- y (1 + e + e^2),          e = 1 - x y,
//   y <- y (1 + e/2 + 3 e^2 / 8),  e = 1 - x y^2,
// which takes the error from d to O(d^3).
//
// Part of a solve's multiplies can be formed on the integer pipes instead of
// the FP64 pipe (fp64_emu.cuh), chosen per kernel by the template argument
// EMU; the IEEE results are the same.  (Adds and FMAs formed there measured
// slower than on the FP64 pipe, so none of the kernels moves them.)
#pragma once

#include <cstdint>

#include "fp64_emu.cuh"
#include "fp_bits.cuh"

namespace sakura {

// Which FP64 operations of a solve are formed on the integer pipes
// (fp64_emu.cuh) instead of the FP64 pipe: a kernel passes the OR of these
// bits as the template argument EMU of the solver functions.  The results are
// the same IEEE values either way; only the pipes that compute them differ.
constexpr int kEmuIncMul = 1;    // the increments' multiplies
constexpr int kEmuSetupMul = 2;  // the setup's multiplies
constexpr int kEmuIterMul = 4;   // the multiplies of a Laguerre iteration
constexpr int kEmuCarryMul = 8;  // the Taylor carry's multiplies

template <int EMU, int BIT>
__device__ __forceinline__ double xmul(double a, double b)
{
    if constexpr ((EMU & BIT) != 0) return emu::mul(a, b);
    else return a * b;
}

// -a b, the sign an operand in either form
template <int EMU, int BIT>
__device__ __forceinline__ double xmul_neg(double a, double b)
{
    if constexpr ((EMU & BIT) != 0) return emu::mul_neg(a, b);
    else return -a * b;
}

constexpr double kPi = 3.14159265358979323846;

// status bits written to the device status word
constexpr unsigned kStatusCoincident = 1u;
constexpr unsigned kStatusNonfinite = 2u;
constexpr unsigned kStatusKepler = 4u;
constexpr unsigned kStatusMass = 8u;
constexpr unsigned kStatusTimeout = 16u;

// The bit pattern of a double, read through an opaque move.  Tests of a
// pattern read with a plain bit cast are turned back into FP64 instructions
// by the compiler: a zero test or an exponent-field test into an FP64
// comparison, a sign flip into an FP64 negation, each a slot of the narrow
// FP64 pipe.
__device__ __forceinline__ long long dbits(double a)
{
    long long b;
    asm("mov.b64 %0, %1;" : "=l"(b) : "d"(a));
    return b;
}

// The seeds of 1/x and 1/sqrt(x) come from the FP32 approximations of x
// truncated to float, formed and widened on the integer pipe (the FP64 pipe
// bounds the solver): relative error about 2^-22 (the truncation 2^-23 plus
// the approximation's).  Operands with |x| outside [2^-126, 2^126), where the
// float or its reciprocal would not be a normal float, take the FP64
// approximations (error <= 2^-19).
__device__ __forceinline__ bool f32_range(long long b)
{
    const int e = (int)((b >> 52) & 0x7ff);
    return e >= 1023 - 126 && e < 1023 + 126;
}

__device__ __forceinline__ float trunc_to_f32(long long b)
{
    const unsigned e = (unsigned)((b >> 52) & 0x7ff) - 1023u + 127u;
    const unsigned m = (unsigned)(b >> 29) & 0x7fffffu;
    const unsigned sign = (unsigned)((unsigned long long)b >> 32) & 0x80000000u;
    return __uint_as_float(sign | (e << 23) | m);
}

__device__ __forceinline__ double widen_f32(float f)
{
    const unsigned u = __float_as_uint(f);
    return __longlong_as_double((long long)((((unsigned long long)(u & 0x80000000u)) << 32) |
                                            ((unsigned long long)(((u >> 23) & 0xffu) + 896u)
                                             << 52) |
                                            ((unsigned long long)(u & 0x7fffffu) << 29)));
}

__device__ __forceinline__ double rcp_seed(double x)
{
    const long long b = dbits(x);
    if (f32_range(b)) {
        float y;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(trunc_to_f32(b)));
        return widen_f32(y);
    }
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

__device__ __forceinline__ double rsqrt_seed(double x)
{
    const long long b = dbits(x);
    if (f32_range(b)) {
        float y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(trunc_to_f32(b)));
        return widen_f32(y);
    }
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

// 1/x to about one ulp (x normal and finite): seed error d <= 2^-19, one
// cubic step y (1 + e + e^2), e = 1 - x y, leaves O(d^3).
__device__ __forceinline__ double rcp_nr(double x)
{
    const double y = rcp_seed(x);
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// 1/x to a relative error of about 2^-38: one quadratic step y (1 + e).
__device__ __forceinline__ double rcp_nr2(double x)
{
    const double y = rcp_seed(x);
    return fma(y, fma(-x, y, 1.0), y);
}

// 1/sqrt(x) to about one ulp (x > 0 normal and finite): one cubic step
// y (1 + e/2 + 3 e^2 / 8), e = 1 - x y^2, from a seed with error <= 2^-19.
template <int EMU = 0>
__device__ __forceinline__ double rsqrt_nr(double x)
{
    const double y = rsqrt_seed(x);
    const double e = fma(-x, xmul<EMU, kEmuSetupMul>(y, y), 1.0);
    return fma(xmul<EMU, kEmuSetupMul>(y, e), fma(0.375, e, 0.5), y);
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Comparisons on IEEE bit patterns run on the integer pipe instead of the
// narrow FP64 pipe.  For doubles that are not NaN, okey() is monotone:
// a < b  <=>  okey(a) < okey(b).  magbits() is the pattern of |a|, monotone
// in |a| (NaN compares above +inf).
__device__ __forceinline__ long long okey(double a)
{
    const long long b = dbits(a);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

__device__ __forceinline__ long long magbits(double a) { return dbits(a) & 0x7fffffffffffffffLL; }

__device__ __forceinline__ bool is_neg(double a) { return dbits(a) < 0; }

constexpr long long kInfBits = 0x7ff0000000000000LL;
constexpr long long kBits0p1 = 0x3fb999999999999aLL;  // 0.1
constexpr long long kBits2p1000 = 0x7e70000000000000LL;  // 2^1000

struct Stumpff {
    double c0, c1, c2, c3;
};

// Number of series terms for c2 and c3 when every |x| in the warp has a
// high word (sign, exponent, top mantissa bits) of at most hx: strictly
// below the high word of 2^-14, 2^-9 and 2^-6 means |x| < 6.1e-5, 1.95e-3
// and 1.56e-2, inside the 3-, 4- and 5-term limits above.
__device__ __forceinline__ int stumpff_terms(unsigned hx)
{
    return hx < 0x3f100000u ? 3 : (hx < 0x3f600000u ? 4 : (hx < 0x3f900000u ? 5 : 6));
}

__device__ __forceinline__ unsigned abs_hiword(double x)
{
    return (unsigned)(magbits(x) >> 32);
}

// c0..c3 at x; nt: warp-uniform number of series terms (3..6) valid for the
// reduced argument (see stumpff_terms).  Arguments with |x| > 0.1 are quartered first (per lane).
__device__ __forceinline__ Stumpff stumpff_fp64(double x, int nt)
{
    int k = 0;
    while (magbits(x) > kBits0p1 && k < 80) {
        x *= 0.25;
        ++k;
    }
    if (k > 0) nt = 6;
    // Horner in y = -x from the highest kept term; 1/(2n+2)! and 1/(2n+3)!.
    // Each step c y + a is written fma(-c, x, a): the same value, with the
    // sign an operand of the FMA rather than a separate FP64 negation of x.
    double c2, c3;
    if (nt >= 6) {
        c2 = fma(-1.0 / 479001600.0, x, 1.0 / 3628800.0);
        c3 = fma(-1.0 / 6227020800.0, x, 1.0 / 39916800.0);
        c2 = fma(-c2, x, 1.0 / 40320.0);
        c3 = fma(-c3, x, 1.0 / 362880.0);
        c2 = fma(-c2, x, 1.0 / 720.0);
        c3 = fma(-c3, x, 1.0 / 5040.0);
    } else if (nt == 5) {
        c2 = fma(-1.0 / 3628800.0, x, 1.0 / 40320.0);
        c3 = fma(-1.0 / 39916800.0, x, 1.0 / 362880.0);
        c2 = fma(-c2, x, 1.0 / 720.0);
        c3 = fma(-c3, x, 1.0 / 5040.0);
    } else if (nt == 4) {
        c2 = fma(-1.0 / 40320.0, x, 1.0 / 720.0);
        c3 = fma(-1.0 / 362880.0, x, 1.0 / 5040.0);
    } else {
        c2 = 1.0 / 720.0;
        c3 = 1.0 / 5040.0;
    }
    c2 = fma(-c2, x, 1.0 / 24.0);
    c3 = fma(-c3, x, 1.0 / 120.0);
    c2 = fma(-c2, x, 0.5);
    c3 = fma(-c3, x, 1.0 / 6.0);
    double c0 = fma(-x, c2, 1.0);
    double c1 = fma(-x, c3, 1.0);
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

// Per-lane state of one pair's Kepler solve.
struct PairSolve {
    double x0, y0, z0, vx, vy, vz;  // Kepler input r0 (back-drifted) and v0
    double r0, ir0, eta0, beta, zeta0, m, t;
    double s, lo, hi;
    double G1, G2, G3, Fp, ir;      // at the accepted s (ir = 1 / Fp)
    int iters;
    bool done;
    bool carried;                   // finished by a Taylor carry to the root
    unsigned status;
};

// Setup of one pair: backward drift, invariants, period reduction, guess.
// rr0, vv0: relative state after the one-subscript drift; m: m_i + m_j.
// guess: -1 = none (the caller sets s; s = 0 here); 0 = standard s0 = t/r0;
// 2 = second order in t, s0 = (t/r0)(1 -
// eta0 t / (2 r0^2)), from ds/dt = 1/r and d2s/dt2 = -eta0/r0^3 at t = 0;
// when the correction exceeds 1/2 in size (fast radial motion over the
// step) the expansion is not trusted and the standard guess is used.
template <int EMU = 0>
__device__ __forceinline__ void pair_setup(PairSolve &p, double tau, double m, double rx,
                                           double ry, double rz, double vx, double vy,
                                           double vz, double pre, int guess)
{
    const double ptau = pre * tau;
    p.status = 0;
    p.iters = 0;
    p.carried = false;
    p.m = m;
    p.vx = vx;
    p.vy = vy;
    p.vz = vz;
    p.x0 = fma(-ptau, vx, rx);
    p.y0 = fma(-ptau, vy, ry);
    p.z0 = fma(-ptau, vz, rz);
    const double r0sq = fma(p.x0, p.x0, fma(p.y0, p.y0, xmul<EMU, kEmuSetupMul>(p.z0, p.z0)));
    p.G1 = p.G2 = p.G3 = 0.0;
    const long long rb = dbits(r0sq);
    if (!(rb > 0 && rb < 0x7e37e43c8800759cLL)) {  // 0 < r0^2 < 1e300, not NaN
        p.status = magbits(r0sq) == 0 ? kStatusCoincident : kStatusNonfinite;
        p.done = true;
        p.r0 = p.ir0 = 1.0;
        p.Fp = p.ir = 1.0;
        p.beta = p.eta0 = p.zeta0 = p.s = 0.0;
        p.t = tau;
        p.lo = p.hi = 0.0;
        return;
    }
    p.ir0 = rsqrt_nr<EMU>(r0sq);
    p.r0 = xmul<EMU, kEmuSetupMul>(r0sq, p.ir0);
    p.Fp = p.r0;
    p.ir = p.ir0;
    p.eta0 = fma(p.x0, vx, fma(p.y0, vy, xmul<EMU, kEmuSetupMul>(p.z0, vz)));
    const double v2 = fma(vx, vx, fma(vy, vy, xmul<EMU, kEmuSetupMul>(vz, vz)));
    p.beta = fma(scale2(m, 1), p.ir0, -v2);
    p.zeta0 = fma(-p.beta, p.r0, m);
    p.t = tau;
    // bound orbit with |t| > P = 2 pi m / beta^1.5  <=>  t^2 beta^3 > (2 pi m)^2
    if (dbits(p.beta) > 0) {
        const double b3 =
            xmul<EMU, kEmuSetupMul>(xmul<EMU, kEmuSetupMul>(p.beta, p.beta), p.beta);
        const double tm = xmul<EMU, kEmuSetupMul>(2.0 * kPi, m);
        const double tt = xmul<EMU, kEmuSetupMul>(tau, tau);
        if (okey(xmul<EMU, kEmuSetupMul>(tt, b3)) > okey(xmul<EMU, kEmuSetupMul>(tm, tm))) {
            const double P = xmul<EMU, kEmuSetupMul>(tm, rsqrt_nr<EMU>(b3));
            p.t = fmod(tau, P);
        }
    }
    p.s = guess < 0 ? 0.0 : xmul<EMU, kEmuSetupMul>(p.t, p.ir0);  // standard initial guess
    if (guess == 2) {
        const double c = 0.5 * p.s * (p.eta0 * p.ir0);  // eta0 t / (2 r0^2)
        if (magbits(c) < 0x3fe0000000000000LL) p.s = fma(-c, p.s, p.s);  // |c| < 1/2
    }
    if (!is_neg(p.t)) {
        p.lo = 0.0;
        p.hi = __longlong_as_double(kInfBits);
    } else {
        p.lo = -__longlong_as_double(kInfBits);
        p.hi = 0.0;
    }
    p.done = (magbits(p.t) == 0);
}

// One Laguerre iteration of a lane that is not done, at s2 = s^2 and x =
// beta s^2; nt is warp-uniform.  Returns true when the new iterate would
// leave the bracket (the caller then applies pair_safeguard in a warp-uniform
// branch).  CARRY: finish with a Taylor carry when the step is small (used
// where the initial guess is already close for every lane, so that whole
// warps finish after one evaluation).  With the carry, 1/F' at the iterate
// only forms the step (to 2^-38, a relative error that vanishes with the
// step) and is recomputed in full at the accepted root.
template <bool CARRY, int EMU = 0>
__device__ __forceinline__ bool pair_iterate(PairSolve &p, double x, double s2, int nt,
                                             const KeplerParams &kp)
{
    const double s = p.s;
    const Stumpff c = stumpff_fp64(x, nt);
    const double G1 = xmul<EMU, kEmuIterMul>(s, c.c1);
    const double G2 = xmul<EMU, kEmuIterMul>(s2, c.c2);
    const double G3 = xmul<EMU, kEmuIterMul>(xmul<EMU, kEmuIterMul>(s2, s), c.c3);
    const double F = fma(p.r0, s, fma(p.eta0, G2, fma(p.zeta0, G3, -p.t)));
    const double Fp = fma(p.eta0, G1, fma(p.zeta0, G2, p.r0));
    const double Fpp = fma(p.eta0, c.c0, xmul<EMU, kEmuIterMul>(p.zeta0, G1));
    const double ip = CARRY ? rcp_nr2(Fp) : rcp_nr(Fp);
    const double q = xmul<EMU, kEmuIterMul>(F, ip);
    p.G1 = G1;
    p.G2 = G2;
    p.G3 = G3;
    p.Fp = Fp;
    p.ir = ip;
    ++p.iters;
    // an iterate so far out that the G functions overflowed, or that r(s) =
    // F' passed 2^1000 (its reciprocal would flush to zero and fake
    // convergence): r at the root is the pair's separation, so the root lies
    // between the iterate and the origin and the iterate bounds the bracket
    if ((dbits(F) & kInfBits) == kInfBits || magbits(Fp) >= kBits2p1000) {
        if (is_neg(s))
            p.lo = s;
        else
            p.hi = s;
        return true;
    }
    // |q| <= tol * max(|s|, |t| / r) (with the carry, a small step is taken
    // and carried instead, on the scale |s|)
    const long long sc = CARRY ? magbits(s) : max(magbits(s), magbits(p.t * ip));
    if (!CARRY && magbits(q) <= magbits(kp.tol * __longlong_as_double(sc))) {
        p.done = true;
        return false;
    }
    if (is_neg(F))
        p.lo = s;
    else
        p.hi = s;
    const double qh = xmul<EMU, kEmuIterMul>(q, xmul<EMU, kEmuIterMul>(Fpp, ip));  // = u / 1.25
    double step;
    if (CARRY && magbits(qh) < 0x3f50000000000000LL) {
        // |u| < 2^-10 (a root next to the seed): the Laguerre step
        // q (1 + k) with k = u / 2.5 + O(u^2), Halley's correction, whose
        // cubic error is far below round-off here
        step = fma(scale2(q, -1), qh, q);
    } else {
        const float u = (float)(1.25 * qh);
        const float r = sqrt_approx(fabsf(1.0f - u));
        const float cf = __fdividef(0.8f * u, 1.0f + r);
        const float k = fabsf(u) < 0.5f ? __fdividef(cf, 1.0f - cf)
                                        : __fdividef(5.0f, fmaf(4.0f, r, 1.0f)) - 1.0f;
        step = fma(q, (double)k, q);
    }
    const double sn = s - step;
    // a step below 2^-20 of the scale: the cubically convergent Laguerre step
    // has reached the root to about 2^-60, so take it and carry G1..G3 and
    // F' = r there by their Taylor series (dG_k/ds = G_{k-1}, G_0 = c0,
    // dG_0/ds = -beta G1; third-order terms below 2^-60) instead of
    // evaluating at the new point
    const long long sc20 = sc > (20LL << 52) ? sc - (20LL << 52) : 0;
    if (CARRY && magbits(step) <= sc20) {
        const double h2 = scale2(xmul<EMU, kEmuCarryMul>(step, step), -1);
        const double F3 = fma(xmul_neg<EMU, kEmuCarryMul>(p.eta0, p.beta), G1,
                              xmul<EMU, kEmuCarryMul>(p.zeta0, c.c0));  // dF''/ds
        p.G3 = fma(h2, G1, fma(-step, G2, G3));
        p.G2 = fma(h2, c.c0, fma(-step, G1, G2));
        p.G1 = fma(h2, xmul_neg<EMU, kEmuCarryMul>(p.beta, G1), fma(-step, c.c0, G1));
        p.Fp = fma(h2, F3, fma(-step, Fpp, Fp));
        p.ir = rcp_nr(p.Fp);
        p.s = sn;
        p.done = true;
        p.carried = true;
        return false;
    }
    const long long ks = okey(sn);
    if (ks > okey(p.lo) && ks < okey(p.hi)) {
        p.s = sn;
        return false;
    }
    return true;
}

// Replacement iterate when a Laguerre step left the bracket [lo, hi]:
// double an open bracket's finite end, or bisect a closed one.
__device__ __forceinline__ void pair_safeguard(PairSolve &p)
{
    if (magbits(p.hi) == kInfBits)
        p.s = 2.0 * fmax(p.lo, p.s);
    else if (magbits(p.lo) == kInfBits)
        p.s = 2.0 * fmin(p.hi, p.s);
    else
        p.s = 0.5 * (p.lo + p.hi);
}

// F and its slope at s, with the G functions (bisection path; nt = 6).
__device__ __forceinline__ double pair_eval(PairSolve &p, double s)
{
    const Stumpff c = stumpff_fp64(p.beta * s * s, 6);
    const double s2 = s * s;
    p.G1 = s * c.c1;
    p.G2 = s2 * c.c2;
    p.G3 = s2 * s * c.c3;
    p.Fp = fma(p.eta0, p.G1, fma(p.zeta0, p.G2, p.r0));
    p.ir = rcp_nr(p.Fp);
    return fma(p.r0, s, fma(p.eta0, p.G2, fma(p.zeta0, p.G3, -p.t)));
}

// Bounded bisection on the bracket for a lane whose iteration did not
// converge (rare); sets kStatusKepler if the bracket cannot be closed.
__device__ __forceinline__ void pair_bisect(PairSolve &p)
{
    const double at = fabs(p.t) * p.ir0;
    for (int q = 0; q < 2100 && isinf(p.hi); ++q) {
        const double c = 2.0 * fmax(p.lo, at);
        if (pair_eval(p, c) < 0.0) p.lo = c; else p.hi = c;
    }
    for (int q = 0; q < 2100 && isinf(p.lo); ++q) {
        const double c = 2.0 * fmin(p.hi, -at);
        if (pair_eval(p, c) > 0.0) p.hi = c; else p.lo = c;
    }
    double mid = 0.5 * (p.lo + p.hi);
    for (int q = 0; q < 2200; ++q) {
        mid = 0.5 * (p.lo + p.hi);
        if (!(mid > p.lo && mid < p.hi)) break;
        if (p.hi - p.lo <= 4.4408920985006262e-16 * fmax(fabs(p.lo), fabs(p.hi))) break;
        const double F = pair_eval(p, mid);
        if (F < 0.0) p.lo = mid;
        else if (F > 0.0) p.hi = mid;
        else if (F == 0.0) break;
        else if (is_neg(mid)) p.lo = mid;  // overflow: mid lies past the root
        else p.hi = mid;
        ++p.iters;
    }
    pair_eval(p, mid);
    if (isinf(p.lo) || isinf(p.hi)) p.status |= kStatusKepler;
    p.done = true;
}

// Increments divided by m = m_i + m_j: out[0..2] = delta_r / m,
// out[3..5] = delta_v / m; qtau = post * tau.
template <int EMU = 0>
__device__ __forceinline__ void pair_increment_over_m(const PairSolve &p, double tau, double qtau,
                                                      double out[6])
{
    const double ir = p.ir;
    const double fm1 = xmul_neg<EMU, kEmuIncMul>(p.G2, p.ir0);
    // g - tau = -m G3 / m ... with t reduced modulo the period, + (t - tau) / m;
    // kept as its negation g3 so that B's addend takes the sign as an operand
    double g3 = p.G3;
    if (dbits(p.t) != dbits(tau)) g3 -= (p.t - tau) * rcp_nr(p.m);
    const double fd = xmul<EMU, kEmuIncMul>(xmul_neg<EMU, kEmuIncMul>(p.G1, p.ir0), ir);
    const double gdm1 = xmul_neg<EMU, kEmuIncMul>(p.G2, ir);
    const double A = fma(-qtau, fd, fm1);
    const double B = fma(-qtau, gdm1, -g3);
    out[3] = fma(fd, p.x0, xmul<EMU, kEmuIncMul>(gdm1, p.vx));
    out[4] = fma(fd, p.y0, xmul<EMU, kEmuIncMul>(gdm1, p.vy));
    out[5] = fma(fd, p.z0, xmul<EMU, kEmuIncMul>(gdm1, p.vz));
    out[0] = fma(A, p.x0, xmul<EMU, kEmuIncMul>(B, p.vx));
    out[1] = fma(A, p.y0, xmul<EMU, kEmuIncMul>(B, p.vy));
    out[2] = fma(A, p.z0, xmul<EMU, kEmuIncMul>(B, p.vz));
}

}  // namespace sakura
