// fp64_emu.cuh -- IEEE binary64 multiply, add and fused multiply-add,
// correctly rounded to nearest-even, formed on the 32-bit integer pipes.
//
// GB300 issues one FP64 warp instruction per ~19 cycles per SM, while its
// integer and FP32 pipes issue several warp instructions per cycle; the FP64
// pair kernels keep the FP64 pipe ~89 % busy and leave ~90 % of the issue
// slots idle.  Moving part of a solve's FP64 operations to these routines
// trades one FP64 slot for a few dozen integer instructions and leaves
// every result bit unchanged: each routine returns exactly the IEEE 754
// result of the operation it replaces (round to nearest, ties to even).
//
// Each routine takes a fast path for normal finite operands whose result is
// normal (zeros included) and calls the hardware instruction for everything
// else (subnormal operands or results, overflow, infinities, NaN), in a
// function that is not inlined so that the common path never issues it.
// The arithmetic is the schoolbook one of IEEE 754 (Section 4 of the
// standard: the exact result, then one rounding):
//   product: the two 53-bit significands multiplied exactly (106 bits) from
//     32 x 32 -> 64-bit partial products;
//   sum: the smaller operand's significand shifted right by the exponent
//     difference, the bits shifted out kept as a sticky bit (ten extra bits
//     below the significand: more than the guard, round and sticky bits that
//     exact rounding needs), the sum or difference normalised by a
//     count of leading zeros;
//   rounding: up when the bits below the 53rd exceed half an ulp, or equal
//     it and the 53rd bit is odd.
// Built for the device and the host (the host tests compare every result
// with the host's own IEEE arithmetic bit for bit).
#pragma once

#include <cstdint>
#include <cstring>
#include <cmath>

#if defined(__CUDACC__)
#define EMU_HD __host__ __device__ __forceinline__
#else
#define EMU_HD inline
#endif

namespace sakura {
namespace emu {

// On the device the pattern is read through an opaque move, so that the
// compiler cannot turn integer work on it back into FP64 instructions (a
// sign flip into an FP64 negation, a zero test into an FP64 comparison).
EMU_HD uint64_t bits_of(double x)
{
#if defined(__CUDA_ARCH__)
    unsigned long long u;
    asm("mov.b64 %0, %1;" : "=l"(u) : "d"(x));
    return u;
#else
    uint64_t u;
    std::memcpy(&u, &x, 8);
    return u;
#endif
}

EMU_HD double from_bits(uint64_t u)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double x;
    std::memcpy(&x, &u, 8);
    return x;
#endif
}

EMU_HD int clz64(uint64_t x)
{
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return __builtin_clzll(x);
#endif
}

// The hardware operations, for the operands the fast paths leave out.  On
// the device they are calls (never predicated into the common path).
#if defined(__CUDA_ARCH__)
__device__ __noinline__ double hw_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __noinline__ double hw_mul_neg(double a, double b) { return __dmul_rn(-a, b); }
__device__ __noinline__ double hw_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __noinline__ double hw_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
#else
inline double hw_mul(double a, double b) { return a * b; }
inline double hw_mul_neg(double a, double b) { return -a * b; }
inline double hw_add(double a, double b) { return a + b; }
inline double hw_fma(double a, double b, double c) { return std::fma(a, b, c); }
#endif

// Fast path of a * b, or of (-a) * b with NEG (the sign flipped in the
// integer sign word, not by a separate negation of a).  Returns false (and
// leaves r undefined) unless both operands are normal or zero and, for
// nonzero operands, the biased exponent of the product before normalisation,
// ea + eb - 1023, lies in [1, 2045]: then the result is normal, or overflows
// to infinity by rounding, which the packing below produces too.
template <bool NEG = false>
EMU_HD bool mul_fast(double a, double b, double &r)
{
    const uint64_t A = bits_of(a), B = bits_of(b);
    const uint32_t ah = (uint32_t)(A >> 32), al = (uint32_t)A;
    const uint32_t bh = (uint32_t)(B >> 32), bl = (uint32_t)B;
    const uint32_t ea = (ah >> 20) & 0x7ffu, eb = (bh >> 20) & 0x7ffu;
    const uint32_t sign = ((ah ^ bh) & 0x80000000u) ^ (NEG ? 0x80000000u : 0u);
    const bool za = ((ah & 0x7fffffffu) | al) == 0, zb = ((bh & 0x7fffffffu) | bl) == 0;
    if (za || zb) {
        // 0 times a finite number: a zero with the product's sign
        r = from_bits((uint64_t)sign << 32);
        return ea != 0x7ffu && eb != 0x7ffu && (za || ea != 0) && (zb || eb != 0);
    }
    const int e0 = (int)ea + (int)eb - 1023;
    if (ea - 1u >= 2046u || eb - 1u >= 2046u || (unsigned)(e0 - 1) >= 2045u) return false;
    // significands m = mh 2^32 + l, mh = the hidden bit and 20 fraction bits
    const uint32_t mh = (ah & 0xfffffu) | 0x100000u, nh = (bh & 0xfffffu) | 0x100000u;
    // exact product P = ma mb in [2^104, 2^106) as Qh 2^64 + wl 2^32 + zl
    const uint64_t Z = (uint64_t)al * bl;
    const uint64_t Y = (uint64_t)mh * bl + (Z >> 32);
    const uint64_t W = (uint64_t)al * nh + Y;
    const uint64_t Qh = (uint64_t)mh * nh + (W >> 32);
    const uint32_t wl = (uint32_t)W, zl = (uint32_t)Z;
    const uint32_t nrm = (uint32_t)(Qh >> 41);  // 1 when P >= 2^105
    const uint32_t sh = 20u + nrm;              // P >> (52 + nrm) = Qh << (32 - sh) | wl >> sh
    const uint64_t mant = (Qh << (32u - sh)) | (wl >> sh);
    // the bits below the significand: the first of them at bit 31 of t, the
    // rest of wl below it, then a sticky 1 for a nonzero zl
    const uint32_t t = (wl << (32u - sh)) | (zl != 0u ? 1u : 0u);
    const uint32_t up = t > 0x80000000u - (uint32_t)(mant & 1u) ? 1u : 0u;
    const int e = e0 + (int)nrm;
    // (e - 1) 2^52 + mant: mant carries the hidden bit into the exponent, and
    // a rounding carry out of the fraction raises the exponent
    const uint64_t m = ((uint64_t)(uint32_t)(e - 1) << 52) + mant + up;
    r = from_bits(m | ((uint64_t)sign << 32));
    return true;
}

EMU_HD double mul(double a, double b)
{
    double r;
    if (mul_fast(a, b, r)) return r;
    return hw_mul(a, b);
}

// (-a) * b
EMU_HD double mul_neg(double a, double b)
{
    double r;
    if (mul_fast<true>(a, b, r)) return r;
    return hw_mul_neg(a, b);
}

// Fast path of a + b.  Returns false unless the operand of larger magnitude
// is normal with a biased exponent of at most 2045 (so the sum cannot
// overflow), the other is normal or zero, and the sum is normal or an exact
// zero (+0, as round to nearest gives for x + (-x)).
EMU_HD bool add_fast(double a, double b, double &r)
{
    uint64_t A = bits_of(a), B = bits_of(b);
    const uint64_t kMag = 0x7fffffffffffffffull;
    if ((B & kMag) > (A & kMag)) {
        const uint64_t T = A;
        A = B;
        B = T;
    }
    const uint32_t ea = (uint32_t)(A >> 52) & 0x7ffu, eb = (uint32_t)(B >> 52) & 0x7ffu;
    if (ea - 1u >= 2045u) return false;
    if ((B & kMag) == 0) {  // x + (+-0) = x for x != 0
        r = from_bits(A);
        return true;
    }
    if (eb == 0) return false;
    const uint64_t kFrac = 0x000fffffffffffffull, kHidden = 0x0010000000000000ull;
    // significands with ten bits below them, the larger one's top bit at 62
    const uint64_t sa = ((A & kFrac) | kHidden) << 10, sb = ((B & kFrac) | kHidden) << 10;
    // the smaller one shifted right by the exponent difference (at most 63:
    // beyond that it is all sticky), a nonzero remainder jammed into bit 0
    const uint32_t d = ea - eb < 63u ? ea - eb : 63u;
    const uint64_t sbs = sb >> d;
    const uint64_t sbj = sbs | ((sbs << d) != sb ? 1ull : 0ull);
    const uint64_t S = ((A ^ B) >> 63) ? sa - sbj : sa + sbj;
    if (S == 0) {
        r = 0.0;
        return true;
    }
    const int lz = clz64(S);
    const int e = (int)ea + 1 - lz;
    if (e < 1) return false;
    const uint64_t Sn = S << lz;  // top bit at 63
    const uint64_t mant = Sn >> 11;
    const uint32_t rb = (uint32_t)Sn & 0x7ffu;
    const uint64_t up = rb > 0x400u - (uint32_t)(mant & 1u) ? 1ull : 0ull;
    const uint64_t m = ((uint64_t)(uint32_t)(e - 1) << 52) + mant + up;
    r = from_bits(m | (A & ~kMag));
    return true;
}

EMU_HD double add(double a, double b)
{
    double r;
    if (add_fast(a, b, r)) return r;
    return hw_add(a, b);
}

// (h, l) >>= k for a 128-bit value, a nonzero remainder jammed into bit 0.
EMU_HD void shr128_jam(uint64_t &h, uint64_t &l, uint32_t k)
{
    if (k == 0) return;
    uint64_t sticky;
    if (k < 64) {
        sticky = (l << (64u - k)) != 0 ? 1ull : 0ull;
        l = (l >> k) | (h << (64u - k));
        h >>= k;
    } else if (k < 128) {
        const uint32_t j = k - 64u;
        sticky = (l != 0 || (j != 0 && (h << (64u - j)) != 0)) ? 1ull : 0ull;
        l = j != 0 ? h >> j : h;
        h = 0;
    } else {
        sticky = (h | l) != 0 ? 1ull : 0ull;
        l = h = 0;
    }
    l |= sticky;
}

// (h, l) <<= k for a 128-bit value, k < 128.
EMU_HD void shl128(uint64_t &h, uint64_t &l, uint32_t k)
{
    if (k == 0) return;
    if (k < 64) {
        h = (h << k) | (l >> (64u - k));
        l <<= k;
    } else {
        h = l << (k - 64u);
        l = 0;
    }
}

// Fast path of fma(a, b, c) = a b + c with one rounding.  Returns false
// unless every operand is normal or zero and the result is normal (or an
// exact zero, or overflows to infinity by rounding).  The exact product
// P = ma mb, 106 bits, and the addend's significand are placed in 128 bits
// with their top bits at bit 125 (the product's at 125 or 126); the one of
// smaller exponent is shifted right by the exponent difference with a
// sticky bit (when the difference is 0 or 1 nothing is shifted out, so a
// difference that changes sign is exact).
EMU_HD bool fma_fast(double a, double b, double c, double &r)
{
    const uint64_t A = bits_of(a), B = bits_of(b), C = bits_of(c);
    const uint64_t kMag = 0x7fffffffffffffffull;
    const uint64_t kFrac = 0x000fffffffffffffull, kHidden = 0x0010000000000000ull;
    const uint32_t ah = (uint32_t)(A >> 32), al = (uint32_t)A;
    const uint32_t bh = (uint32_t)(B >> 32), bl = (uint32_t)B;
    const uint32_t ea = (ah >> 20) & 0x7ffu, eb = (bh >> 20) & 0x7ffu;
    const uint32_t ec = (uint32_t)(C >> 52) & 0x7ffu;
    const bool za = (A & kMag) == 0, zb = (B & kMag) == 0, zc = (C & kMag) == 0;
    if (!((ea - 1u < 2046u || za) && (eb - 1u < 2046u || zb) && (ec - 1u < 2046u || zc)))
        return false;
    const uint32_t sp = (ah ^ bh) & 0x80000000u, sc = (uint32_t)(C >> 32) & 0x80000000u;
    if (za || zb) {
        // an exact zero product: c, or for c = 0 the sum of two zeros
        // (-0 only when both are -0)
        r = zc ? from_bits((uint64_t)(sp & sc) << 32) : c;
        return true;
    }
    if (zc) return mul_fast(a, b, r);
    const uint32_t mh = (ah & 0xfffffu) | 0x100000u, nh = (bh & 0xfffffu) | 0x100000u;
    const uint64_t Z = (uint64_t)al * bl;
    const uint64_t Y = (uint64_t)mh * bl + (Z >> 32);
    const uint64_t W = (uint64_t)al * nh + Y;
    const uint64_t Qh = (uint64_t)mh * nh + (W >> 32);
    const uint32_t wl = (uint32_t)W, zl = (uint32_t)Z;
    // X = P << 21 and the addend's mc << 73, as (high, low) 64-bit words
    const uint64_t xh = (Qh << 21) | (wl >> 11);
    const uint64_t xl = ((uint64_t)wl << 53) | ((uint64_t)zl << 21);
    const uint64_t yh = ((C & kFrac) | kHidden) << 9, yl = 0;
    const int pe = (int)ea + (int)eb - 1023;  // biased exponent of X's bit 125
    const int dexp = pe - (int)ec;
    uint64_t gh, gl, sh, sl;  // the operand of larger exponent, the other
    uint32_t sg;
    int base;
    if (dexp >= 0) {
        gh = xh; gl = xl; sh = yh; sl = yl; sg = sp; base = pe;
    } else {
        gh = yh; gl = yl; sh = xh; sl = xl; sg = sc; base = (int)ec;
    }
    const uint32_t k = dexp >= 0 ? (uint32_t)dexp : (uint32_t)(-dexp);
    shr128_jam(sh, sl, k < 128u ? k : 128u);
    uint64_t Sh, Sl;
    if (sp == sc) {
        Sl = gl + sl;
        Sh = gh + sh + (Sl < gl ? 1ull : 0ull);
    } else {
        Sl = gl - sl;
        Sh = gh - sh - (gl < sl ? 1ull : 0ull);
        if ((int64_t)Sh < 0) {  // the other operand was larger: negate
            Sl = ~Sl + 1ull;
            Sh = ~Sh + (Sl == 0 ? 1ull : 0ull);
            sg ^= 0x80000000u;
        }
    }
    if ((Sh | Sl) == 0) {
        r = 0.0;
        return true;
    }
    const int lz = Sh != 0 ? clz64(Sh) : 64 + clz64(Sl);
    shl128(Sh, Sl, (uint32_t)lz);  // top bit at 127
    const int e = base + 2 - lz;
    if (e < 1 || e > 2046) return false;
    const uint64_t mant = Sh >> 11;
    const uint32_t rb = (((uint32_t)Sh & 0x7ffu) << 1) | (Sl != 0 ? 1u : 0u);
    const uint64_t up = rb > 0x800u - (uint32_t)(mant & 1u) ? 1ull : 0ull;
    const uint64_t m = ((uint64_t)(uint32_t)(e - 1) << 52) + mant + up;
    r = from_bits(m | ((uint64_t)sg << 32));
    return true;
}

EMU_HD double fma(double a, double b, double c)
{
    double r;
    if (fma_fast(a, b, c, r)) return r;
    return hw_fma(a, b, c);
}

}  // namespace emu
}  // namespace sakura
