// fp_bits.cuh -- exact FP64 operations done on the integer pipe.
//
// On GB300 the FP64 pipe issues one warp instruction per ~20 cycles per SM,
// and the FP64 pair kernels are bound by it; conversions between float and
// double run on that pipe too.  Where an operation is exact and its operand
// is normal, the same bits can be formed with integer operations instead:
//   scale2(x, k) = x * 2^k  (x and the result normal: only the exponent
//                            field changes, so the product is exact)
//   f2d(f)       = (double)f (f normal: sign, rebiased exponent, mantissa
//                             shifted into place)
// Any other operand (zero, subnormal, infinity, NaN, or a result outside the
// normal range) takes the FP64 instruction, so the result is always the one
// the FP64 operation gives.  Host C++ builds (tests) use memcpy bit casts.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define FPB_HD __host__ __device__ __forceinline__
#else
#define FPB_HD inline
#endif

namespace sakura {

FPB_HD int64_t fpb_bits(double x)
{
#if defined(__CUDA_ARCH__)
    return __double_as_longlong(x);
#else
    int64_t b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}

FPB_HD double fpb_double(int64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double(b);
#else
    double x;
    std::memcpy(&x, &b, sizeof x);
    return x;
#endif
}

FPB_HD uint32_t fpb_fbits(float f)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(f);
#else
    uint32_t u;
    std::memcpy(&u, &f, sizeof u);
    return u;
#endif
}

// x * 2^k for k = -1 or +1 (the scales the solver uses)
FPB_HD double scale2(double x, int k)
{
    const int64_t b = fpb_bits(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e >= 1 && e <= 2046 && e + k >= 1 && e + k <= 2046)
        return fpb_double(b + ((int64_t)k << 52));
    return x * (k > 0 ? 2.0 : 0.5);
}

// (double)f
FPB_HD double f2d(float f)
{
    const uint32_t u = fpb_fbits(f);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e >= 1u && e <= 254u)
        return fpb_double((int64_t)((((uint64_t)(u & 0x80000000u)) << 32) |
                                    ((uint64_t)(e + 896u) << 52) |
                                    ((uint64_t)(u & 0x7fffffu) << 29)));
    return (double)f;
}

}  // namespace sakura
