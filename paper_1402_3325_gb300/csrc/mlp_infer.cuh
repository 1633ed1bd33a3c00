// mlp_infer.cuh -- the learned initial guess: features and warp-level BF16
// inference of the 6-64-64-1 tanh perceptron.
//
// Guess model.  After the pair setup, with the standard guess s_std = t/r0
// and the second-order guess s_T2 (kepler_fp64.cuh), the learned guess is
//     s0 = s_T2 * exp(w * g(x)),   w = q / (1 + q),
//     q  = tau'^2 (1 + eta'^2 + |beta'|),
// in the dimensionless variables tau' = |t| sqrt(m / r0^3),
// eta' = sign(t) eta0 / sqrt(m r0), beta' = beta r0 / m (the Kepler problem
// in units r0 and sqrt(r0^3/m) depends on these three only, and reversing t
// is the same as reversing eta0).  q measures how far the pair is from the
// regime where the expansion is exact; the gate w keeps the network's
// rounding error from spoiling weak pairs, where s_T2 is already accurate, and
// a warp whose pairs all have w <= 1e-4 does not evaluate the network at all.
// Features x = (log tau', asinh eta', asinh beta', tanh(eta' tau'),
// tanh(beta' tau'^2), w), normalised by the mean and scale stored with the
// weights.  The network output is g = y * oscale + oshift, clamped to [-4, 4].
//
// Inference: one warp evaluates the network for its 32 pairs with
// mma.sync.m16n8k16 (BF16 inputs and weights, FP32 accumulation): the 32 x 16
// input tile (features padded with zeros) is staged in shared memory; the
// FP32 accumulator fragments of a layer, after tanh and BF16 rounding, are
// exactly the A fragments of the next layer's 16-wide k tiles, so the hidden
// activations never leave registers.  88 mma per 32 pairs.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace sakura {

constexpr int kMlpIn = 6;
constexpr int kMlpHidden = 64;
constexpr int kMlpParams = 6 * 64 + 64 + 64 * 64 + 64 + 64 + 1;  // 4673
constexpr int kMlpBlob = kMlpParams + 6 + 6 + 2;                   // 4687

// Device copy of the network in the layouts the MMA fragments read.
struct MlpWeights {
    __nv_bfloat16 W1[64 * 16];  // [n][k], k = input feature padded to 16
    __nv_bfloat16 W2[64 * 64];  // [n][k]
    __nv_bfloat16 W3[8 * 64];   // [n][k], row 0 = output weights, rows 1..7 zero
    float b1[64], b2[64];
    float b3;
    float mean[6], inv_scale[6];
    float oscale, oshift;
};

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// double -> float by truncating the mantissa, on the integer pipe (the
// FP64 pipe is the kernel's bottleneck; features need no rounding).  Values
// below the float range become 0, above it infinity.
__device__ __forceinline__ float d2f_trunc(double x)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned sign = (unsigned)hi & 0x80000000u;
    const int e = ((hi >> 20) & 0x7ff) - 896;  // float biased exponent
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    const unsigned mant = (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
    return __uint_as_float(sign | ((unsigned)e << 23) | mant);
}

// Dimensionless pair variables and the gate w (cheap part of the features).
struct GuessVars {
    float tp, ep, bp, w;
};

__device__ __forceinline__ bool guess_gate(double t, double m, double r0, double ir0,
                                           double eta0, double beta, GuessVars &gv)
{
    const float tf = d2f_trunc(t);
    const float mf = d2f_trunc(m), r0f = d2f_trunc(r0), ir0f = d2f_trunc(ir0);
    const float sgn = tf < 0.0f ? -1.0f : 1.0f;
    gv.tp = fabsf(tf) * sqrtf(mf * ir0f) * ir0f;
    gv.ep = sgn * d2f_trunc(eta0) * rsqrtf(mf * r0f);
    gv.bp = d2f_trunc(beta) * r0f / mf;
    const float q = gv.tp * gv.tp * (1.0f + gv.ep * gv.ep + fabsf(gv.bp));
    gv.w = q / (1.0f + q);
    if (!(gv.tp > 0.0f) || !isfinite(q)) {
        gv.w = 0.0f;
        return false;
    }
    return true;
}

__device__ __forceinline__ void guess_features_from(const GuessVars &gv, float f[6])
{
    f[0] = __logf(gv.tp);
    f[1] = asinhf(gv.ep);
    f[2] = asinhf(gv.bp);
    f[3] = tanhf(gv.ep * gv.tp);
    f[4] = tanhf(gv.bp * gv.tp * gv.tp);
    f[5] = gv.w;
}

// Features of a pair (FP32).  Returns false if the pair has no usable
// features (t = 0 or degenerate); w is the gate.
__device__ __forceinline__ bool guess_features(double t, double m, double r0, double ir0,
                                               double eta0, double beta, float f[6], float &w)
{
    GuessVars gv;
    const bool ok = guess_gate(t, m, r0, ir0, eta0, beta, gv);
    w = gv.w;
    if (!ok) {
        for (int k = 0; k < 6; ++k) f[k] = 0.0f;
        return false;
    }
    guess_features_from(gv, f);
    return true;
}

// Network output g for the 32 lanes' feature vectors (every lane calls; lanes
// without a pair pass zeros).  W: weights in shared memory; stage: 32 x 16
// bf16 scratch of this warp in shared memory.
__device__ __forceinline__ float mlp_eval_warp(const MlpWeights &W, __nv_bfloat16 *stage,
                                               const float f[6])
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, tg = lane & 3;
    // stage normalised inputs, row = lane, columns 6..15 zero
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float v = k < 6 ? (f[k] - W.mean[k]) * W.inv_scale[k] : 0.0f;
        stage[lane * 16 + k] = __float2bfloat16_rn(v);
    }
    __syncwarp();
    const uint32_t *st = reinterpret_cast<const uint32_t *>(stage);
    uint32_t a1[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = mt * 16 + g;
        a1[mt][0] = st[(r0 * 16 + 2 * tg) >> 1];
        a1[mt][1] = st[((r0 + 8) * 16 + 2 * tg) >> 1];
        a1[mt][2] = st[(r0 * 16 + 8 + 2 * tg) >> 1];
        a1[mt][3] = st[((r0 + 8) * 16 + 8 + 2 * tg) >> 1];
    }
    __syncwarp();
    const uint32_t *w1 = reinterpret_cast<const uint32_t *>(W.W1);
    const uint32_t *w2 = reinterpret_cast<const uint32_t *>(W.W2);
    const uint32_t *w3 = reinterpret_cast<const uint32_t *>(W.W3);
    // layer 1: 32 x 64 = X (32 x 16) W1^T, tanh, repacked as layer-2 A tiles
    uint32_t a2[2][4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int n = nt * 8 + g;
        const uint32_t b0 = w1[(n * 16 + 2 * tg) >> 1];
        const uint32_t b1 = w1[(n * 16 + 8 + 2 * tg) >> 1];
        const float bb0 = W.b1[nt * 8 + 2 * tg], bb1 = W.b1[nt * 8 + 2 * tg + 1];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            float d[4] = {bb0, bb1, bb0, bb1};
            mma_bf16(d, a1[mt], b0, b1);
            const uint32_t lo = pack_bf16(tanh_approx(d[0]), tanh_approx(d[1]));
            const uint32_t hi = pack_bf16(tanh_approx(d[2]), tanh_approx(d[3]));
            const int kt = nt >> 1;
            if ((nt & 1) == 0) {
                a2[mt][kt][0] = lo;
                a2[mt][kt][1] = hi;
            } else {
                a2[mt][kt][2] = lo;
                a2[mt][kt][3] = hi;
            }
        }
    }
    // layer 2: 32 x 64 = H1 W2^T, tanh, repacked as layer-3 A tiles
    uint32_t a3[2][4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int n = nt * 8 + g;
        const float bb0 = W.b2[nt * 8 + 2 * tg], bb1 = W.b2[nt * 8 + 2 * tg + 1];
        float d[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            d[mt][0] = bb0;
            d[mt][1] = bb1;
            d[mt][2] = bb0;
            d[mt][3] = bb1;
        }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const uint32_t b0 = w2[(n * 64 + kt * 16 + 2 * tg) >> 1];
            const uint32_t b1 = w2[(n * 64 + kt * 16 + 8 + 2 * tg) >> 1];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma_bf16(d[mt], a2[mt][kt], b0, b1);
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const uint32_t lo = pack_bf16(tanh_approx(d[mt][0]), tanh_approx(d[mt][1]));
            const uint32_t hi = pack_bf16(tanh_approx(d[mt][2]), tanh_approx(d[mt][3]));
            const int kt = nt >> 1;
            if ((nt & 1) == 0) {
                a3[mt][kt][0] = lo;
                a3[mt][kt][1] = hi;
            } else {
                a3[mt][kt][2] = lo;
                a3[mt][kt][3] = hi;
            }
        }
    }
    // layer 3: column 0 of H2 W3^T (rows 1..7 of W3 are zero)
    float out[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        out[mt][0] = out[mt][1] = out[mt][2] = out[mt][3] = 0.0f;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const uint32_t b0 = w3[(g * 64 + kt * 16 + 2 * tg) >> 1];
            const uint32_t b1 = w3[(g * 64 + kt * 16 + 8 + 2 * tg) >> 1];
            mma_bf16(out[mt], a3[mt][kt], b0, b1);
        }
    }
    // sample r = 16 mt + 8 h + gg sits in lane 4 gg, register 2 h (column 0)
    const int r = lane;
    const int mt = r >> 4, h = (r >> 3) & 1, gg = r & 7;
    const float v00 = __shfl_sync(0xffffffffu, out[0][0], 4 * gg);
    const float v02 = __shfl_sync(0xffffffffu, out[0][2], 4 * gg);
    const float v10 = __shfl_sync(0xffffffffu, out[1][0], 4 * gg);
    const float v12 = __shfl_sync(0xffffffffu, out[1][2], 4 * gg);
    const float y = (mt == 0 ? (h == 0 ? v00 : v02) : (h == 0 ? v10 : v12)) + W.b3;
    const float gout = y * W.oscale + W.oshift;
    return fminf(4.0f, fmaxf(-4.0f, gout));
}

// Copy the network into shared memory (all threads of the block call).
__device__ __forceinline__ void mlp_load_shared(MlpWeights &dst, const MlpWeights *src)
{
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(MlpWeights) / 4); k += blockDim.x) d[k] = s[k];
    __syncthreads();
}

}  // namespace sakura
