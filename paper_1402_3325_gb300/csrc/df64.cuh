// df64.cuh -- double-word ("double-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum h + l of two floats with |l| <= ulp(h) / 2,
// about 48 significant bits.  On GB300 the FP32 pipe issues 64 times as many
// operations per clock as the FP64 pipe, so a computation that needs FP64
// accuracy but little FP64 range can run faster in double-word form.
//
// The algorithms are the published error-free transformations and their
// double-word compositions:
//   two_sum       Knuth, TAOCP vol. 2 (1969): s + e = a + b exactly;
//   fast_two_sum  Dekker (1971): the same when |a| >= |b| (or a = 0);
//   two_prod      with a fused multiply-add: p + e = a * b exactly;
//   dw_add        Joldes, Muller & Popescu, "Tight and rigorous error bounds
//                 for basic building blocks of double-word arithmetic", ACM
//                 TOMS 44 (2017), Alg. 6 (relative error <= 3u^2, u = 2^-24);
//   dw_add_f      ibid. Alg. 4 (double-word plus float, <= 2u^2);
//   dw_add_nc     ibid. Alg. 5 (no cancellation: like signs or a much
//                 smaller term, <= 3u^2);
//   dw_mul        ibid. Alg. 12 (<= 4u^2 with FMA; here the l*l term kept);
//   dw_mul_f      ibid. Alg. 9 (double-word times float, <= 2u^2);
// and Newton corrections for 1/y and 1/sqrt(x) from a float approximation
// refined to about u, whose residual is formed exactly with an FMA.
//
// Every plain operation goes through fadd/fsub/fmul (round to nearest, never
// contracted into an FMA) or ffma, so the error-free transformations stay
// exact.  The functions also compile as host C++ (built with
// -ffp-contract=off) so that a CPU test can check their error bounds.
#pragma once

#include <cmath>

#if defined(__CUDACC__)
#define DW_HD __host__ __device__ __forceinline__
#else
#define DW_HD inline
#endif

namespace sakura {

struct dw {
    float h, l;
};

#if !defined(__CUDA_ARCH__) && defined(SAKURA_DW_COUNT)
// host build only: tally of floating-point operations (FMA = 2) and of
// special-function approximations, for counting the work of one solve
extern long long sakura_dw_flops, sakura_dw_mufu;
#define SAKURA_DW_TALLY(k) (sakura_dw_flops += (k))
#define SAKURA_DW_MUFU() (++sakura_dw_mufu)
#else
#define SAKURA_DW_TALLY(k) ((void)0)
#define SAKURA_DW_MUFU() ((void)0)
#endif

#if defined(__CUDA_ARCH__)
DW_HD float fadd(float a, float b) { return __fadd_rn(a, b); }
DW_HD float fsub(float a, float b) { return __fsub_rn(a, b); }
DW_HD float fmul(float a, float b) { return __fmul_rn(a, b); }
DW_HD float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// hardware approximations (relative error about 2^-22), refined below
DW_HD float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
DW_HD float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
DW_HD float fsqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
#else
DW_HD float fadd(float a, float b)
{
    SAKURA_DW_TALLY(1);
    return a + b;
}
DW_HD float fsub(float a, float b)
{
    SAKURA_DW_TALLY(1);
    return a - b;
}
DW_HD float fmul(float a, float b)
{
    SAKURA_DW_TALLY(1);
    return a * b;
}
DW_HD float ffma(float a, float b, float c)
{
    SAKURA_DW_TALLY(2);
    return std::fmaf(a, b, c);
}
DW_HD float rcp_approx(float x)
{
    SAKURA_DW_MUFU();
    return 1.0f / x;
}
DW_HD float rsqrt_approx(float x)
{
    SAKURA_DW_MUFU();
    return 1.0f / std::sqrt(x);
}
DW_HD float fsqrt_approx(float x)
{
    SAKURA_DW_MUFU();
    return std::sqrt(x);
}
#endif

DW_HD dw two_sum(float a, float b)
{
    const float s = fadd(a, b);
    const float bb = fsub(s, a);
    const float e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
    return {s, e};
}

DW_HD dw fast_two_sum(float a, float b)
{
    const float s = fadd(a, b);
    return {s, fsub(b, fsub(s, a))};
}

DW_HD dw two_prod(float a, float b)
{
    const float p = fmul(a, b);
    return {p, ffma(a, b, -p)};
}

DW_HD dw dw_from(float a) { return {a, 0.0f}; }
DW_HD dw dw_neg(dw x) { return {-x.h, -x.l}; }
// multiplication by a power of two is exact
DW_HD dw dw_scale(dw x, float p2) { return {fmul(x.h, p2), fmul(x.l, p2)}; }

DW_HD dw dw_add(dw x, dw y)
{
    const dw s = two_sum(x.h, y.h);
    const dw t = two_sum(x.l, y.l);
    const float c = fadd(s.l, t.h);
    const dw v = fast_two_sum(s.h, c);
    const float w = fadd(t.l, v.l);
    return fast_two_sum(v.h, w);
}

DW_HD dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }

// ibid. Alg. 5 (sloppy sum): relative error <= 3u^2 when x and y have the
// same sign; used only for sums of like-signed terms and for a term much
// smaller than the other (no cancellation)
DW_HD dw dw_add_nc(dw x, dw y)
{
    const dw s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, fadd(s.l, fadd(x.l, y.l)));
}

DW_HD dw dw_add_f(dw x, float y)
{
    const dw s = two_sum(x.h, y);
    const float v = fadd(x.l, s.l);
    return fast_two_sum(s.h, v);
}

DW_HD dw dw_mul(dw x, dw y)
{
    const dw c = two_prod(x.h, y.h);
    const float t0 = fmul(x.l, y.l);
    const float t1 = ffma(x.h, y.l, t0);
    const float t2 = ffma(x.l, y.h, t1);
    return fast_two_sum(c.h, fadd(c.l, t2));
}

DW_HD dw dw_mul_f(dw x, float y)
{
    const dw c = two_prod(x.h, y);
    return fast_two_sum(c.h, ffma(x.l, y, c.l));
}

DW_HD dw dw_sqr(dw x)
{
    const dw c = two_prod(x.h, x.h);
    const float t = ffma(fadd(x.h, x.h), x.l, fmul(x.l, x.l));
    return fast_two_sum(c.h, fadd(c.l, t));
}

// x * y + z
DW_HD dw dw_fma(dw x, dw y, dw z) { return dw_add(dw_mul(x, y), z); }

// 1 / y: a float reciprocal refined to about u, then the Newton correction
// r (1 + e + e^2) with e = 1 - y r (the leading part of e is exact by FMA
// because r is within a few ulp of 1 / y.h)
DW_HD dw dw_rcp(dw y)
{
    float r = rcp_approx(y.h);
    r = ffma(r, ffma(-y.h, r, 1.0f), r);
    const float e = ffma(-y.l, r, ffma(-y.h, r, 1.0f));
    return fast_two_sum(r, fmul(r, ffma(e, e, e)));
}

// 1 / sqrt(x), x > 0: a float value y refined to about u, then the Newton
// correction y (1 + e/2 + 3e^2/8) with e = 1 - x y^2; x.h y^2 is split
// exactly (y^2 = p.h + p.l by two_prod, x.h p.h = q.h + q.l), so 1 - q.h is
// exact and only the small remainder is rounded
DW_HD dw dw_rsqrt(dw x)
{
    float y = rsqrt_approx(x.h);
    const float hy = fmul(0.5f, y);
    y = ffma(hy, ffma(-x.h, fmul(y, y), 1.0f), y);
    const dw p = two_prod(y, y);
    const dw q = two_prod(x.h, p.h);
    const float t = ffma(x.h, p.l, ffma(x.l, p.h, q.l));
    const float e = fsub(fsub(1.0f, q.h), t);
    return fast_two_sum(y, fmul(y, fmul(e, ffma(0.375f, e, 0.5f))));
}

// A double held exactly as three floats, d = d0 + d1 + d2 (d0 = fl(d),
// d1 = fl(d - d0), d2 = d - d0 - d1; 72 bits cover the 53 of a double).
DW_HD void tf_split(double d, float &d0, float &d1, float &d2)
{
    d0 = (float)d;
    const double r = d - (double)d0;
    d1 = (float)r;
    d2 = (float)(r - (double)d1);
}

// a - b for a, b in tf_split form, rounded to double-word form: the leading
// and middle differences are formed exactly by two_sum and only terms of
// order u |a - b| are rounded, so the relative error is about u^2 of
// |a - b| however close a and b are (a double-word copy of each coordinate
// would leave an error of u^2 |a| instead).
DW_HD dw tf_diff(float a0, float a1, float a2, float b0, float b1, float b2)
{
    const dw s = two_sum(a0, -b0);
    const dw t = two_sum(a1, -b1);
    const float r = fsub(a2, b2);
    const dw u = two_sum(s.h, t.h);
    const float w = fadd(fadd(fadd(u.l, s.l), t.l), r);
    return two_sum(u.h, w);
}

DW_HD float dw_to_float(dw x) { return fadd(x.h, x.l); }

// magnitude comparisons used for branch decisions (exact to within u^2)
DW_HD bool dw_lt0(dw x) { return x.h < 0.0f || (x.h == 0.0f && x.l < 0.0f); }

}  // namespace sakura
