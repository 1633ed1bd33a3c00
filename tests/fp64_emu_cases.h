// Operand generator for the checks of csrc/fp64_emu.cuh, shared by the host
// check (tests/fp64_emu_host.cpp) and the device check
// (tests/fp64_emu_probe.cu): the same cases, compared against the host's
// IEEE arithmetic on one side and the GPU's FP64 instructions on the other.
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define CASES_HD __host__ __device__ inline
#else
#define CASES_HD inline
#endif

namespace emucases {

CASES_HD uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

CASES_HD uint64_t bits(double x) { return sakura::emu::bits_of(x); }
CASES_HD double dbl(uint64_t u) { return sakura::emu::from_bits(u); }

// A double of the given kind:
//   0: any 64-bit pattern (every class: zeros, subnormals, infinities, NaN);
//   1: biased exponent 1023 +- 60, random fraction;
//   2: as 1, with the fraction's low k bits cleared, k random in [0, 52]
//      (exact products and sums, and exact halfway cases);
//   3: a special or boundary value.
CASES_HD double draw(uint64_t &s, int kind)
{
    const uint64_t r = splitmix(s);
    const uint64_t sign = r & 0x8000000000000000ull;
    if (kind == 0) return dbl(r);
    if (kind == 3) {
        const uint64_t edge[14] = {
            0x0000000000000000ull,  // 0
            0x0010000000000000ull,  // least normal
            0x000fffffffffffffull,  // largest subnormal
            0x0000000000000001ull,  // least subnormal
            0x7fefffffffffffffull,  // largest finite
            0x7fe0000000000000ull,  // 2^1023
            0x7ff0000000000000ull,  // infinity
            0x7ff8000000000000ull,  // NaN
            0x3ff0000000000000ull,  // 1
            0x3fffffffffffffffull,  // just below 2
            0x0020000000000000ull,  // 2^-1021
            0x3ff0000000000001ull,  // 1 + ulp
            0x5ff0000000000000ull,  // 2^512
            0x2000000000000000ull,  // 2^-511
        };
        return dbl(edge[(r >> 8) % 14] | sign);
    }
    const uint64_t ex = 1023 - 60 + (r >> 1) % 121;
    uint64_t frac = splitmix(s) & 0x000fffffffffffffull;
    if (kind == 2) {
        const int k = (int)((r >> 20) % 53);
        frac = frac >> k << k;
    }
    return dbl(sign | ex << 52 | frac);
}

// The operands of one case of op (0: a * b, 1: a + b, 2: fma(a, b, c)) of
// the given kind: 0..3 as draw(), every operand of that kind; 4: each
// operand of its own random kind; 5: as 4, then (sums) the second addend a
// near-negation of the first or a power-of-two multiple of it, for
// cancellation; 6: near-ties, a significand whose low word is half a word
// plus or minus a little, times 1 + k 2^-52 (products whose bits below the
// 53rd sit next to one half, with or without bits further down), and for
// the sums an addend of about half an ulp.
CASES_HD void make_case(uint64_t &s, int op, int kind, double &a, double &b, double &c)
{
    const bool mix = kind == 4 || kind == 5;
    const int ka = mix ? (int)(splitmix(s) % 4) : (kind == 6 ? 1 : kind);
    const int kb = mix ? (int)(splitmix(s) % 4) : (kind == 6 ? 1 : kind);
    const int kc = mix ? (int)(splitmix(s) % 4) : (kind == 6 ? 1 : kind);
    a = draw(s, ka);
    b = draw(s, kb);
    c = draw(s, kc);
    if (kind == 5) {
        const uint64_t r = splitmix(s);
        const double ref = op == 1 ? a : a * b;
        const double near = dbl(bits(-ref) + (r % 9) - 4);
        if (op == 1) b = (r >> 8) & 1 ? near : ldexp(-a, (int)((r >> 9) % 5) - 2);
        else c = (r >> 8) & 1 ? near : ldexp(-ref, (int)((r >> 9) % 5) - 2);
    } else if (kind == 6) {
        const uint64_t r = splitmix(s);
        const uint64_t lo = (r & 1 ? 0x80000000ull : 0ull) + ((r >> 1) % 9) - 4;
        a = dbl((bits(a) & ~0xffffffffull) | (lo & 0xffffffffull));
        const double one_k = dbl(0x3ff0000000000000ull | ((r >> 8) % 5 + 1));
        const int ex = ilogb(a);
        if (op == 1) {
            b = ldexp((r >> 12) & 1 ? -one_k : one_k, ex - 53 + (int)((r >> 13) % 5) - 2);
        } else {
            b = ldexp(one_k, (int)((r >> 16) % 41) - 20);
            c = ldexp((r >> 12) & 1 ? -one_k : one_k,
                      ex + ilogb(b) - 53 + (int)((r >> 13) % 7) - 3);
        }
    }
}

CASES_HD bool same(double x, double y)
{
    if (x != x || y != y) return x != x && y != y;
    return bits(x) == bits(y);
}

}  // namespace emucases
