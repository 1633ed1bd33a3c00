// mlp.cu -- data, training and evaluation kernels of the learned initial guess.
//
// Training data: for given ordered pairs of a system, the pair's Kepler solve
// is run with the FP64 solver (standard guess) and the features of
// mlp_infer.cuh and the target g = log(s / s_T2) / w are written.
//
// Training (FP32, the project's own kernels):
//   forward/backward kernel: one thread per sample computes the forward pass,
//     the residual and the back-propagated dz2, dz1 (stored per sample);
//   gradient kernels: each weight gradient is a sum over the batch, computed
//     by one thread per weight in sample order (deterministic, no atomics);
//   Adam kernel: bias-corrected Adam update of the FP32 master parameters.
// Parameter layout (FP32): W1[64][6], b1[64], W2[64][64], b2[64], W3[64], b3.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>

#include "kepler_fp64.cuh"
#include "mlp_infer.cuh"
#include "pair_batch_fp64.cuh"
#include "step_common.cuh"

namespace sakura {

constexpr int kOffW1 = 0, kOffB1 = 384, kOffW2 = 448, kOffB2 = 4544, kOffW3 = 4608,
              kOffB3 = 4672;

// ---------------------------------------------------------------- data
__global__ void __launch_bounds__(128)
    sample_pairs_kernel(const double *X, int64_t n, double tau, double pre, const int64_t *ids,
                        int64_t count, float *feat, float *target, int *iters_out,
                        double tol, unsigned *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) - lane;
    const int64_t k = base + lane;
    const bool valid_id = k < count;
    int64_t i = 0, j = 0;
    if (valid_id) {
        i = ids[k] / n;
        j = ids[k] - i * n;
    }
    const bool valid = valid_id && i != j && i >= 0 && i < n;
    PairSolve p;
    double s_t2 = 0.0;
    if (valid) {
        pair_setup(p, tau, X[6 * n + i] + X[6 * n + j], X[i] - X[j], X[n + i] - X[n + j],
                   X[2 * n + i] - X[2 * n + j], X[3 * n + i] - X[3 * n + j],
                   X[4 * n + i] - X[4 * n + j], X[5 * n + i] - X[5 * n + j], pre, 2);
        s_t2 = p.s;
        p.s = p.t * p.ir0;  // solve from the standard guess
    } else {
        p.done = true;
        p.beta = p.s = 0.0;
        p.iters = 0;
        p.status = 0;
    }
    const KeplerParams kp{tol, 50, 1};
    double d[6];
    int it = 0, fb = 0;
    fp64_solve_warp(p, valid, tau, (1.0 - pre) * tau, kp, d, it, fb);
    if (!valid_id) return;
    float f[6] = {0, 0, 0, 0, 0, 0}, w = 0.0f, tg = 0.0f;
    if (valid && guess_features(p.t, p.m, p.r0, p.ir0, p.eta0, p.beta, f, w) && w > 0.0f) {
        const double ratio = p.s / s_t2;
        tg = ratio > 0.0 ? (float)(log(ratio) / (double)w) : 0.0f;
    }
    for (int q = 0; q < 6; ++q) feat[k * 6 + q] = f[q];
    target[k] = tg;
    if (iters_out) iters_out[k] = it;
    if (valid && p.status) atomicOr(status, p.status);
}

// ------------------------------------------------------------- training
// dy, dz2 [B][64], dz1 [B][64], h1, h2 [B][64], xn [B][6], r2 (squared
// residuals) are per-sample scratch.
__global__ void __launch_bounds__(64)
    mlp_fwd_bwd_kernel(const float *P, const float *norm, const float *feat, const float *target,
                       int64_t B, float *xn, float *h1, float *h2, float *dy, float *dz2,
                       float *dz1, float *r2)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float x[6];
    for (int k = 0; k < 6; ++k) {
        x[k] = (feat[b * 6 + k] - norm[k]) / norm[6 + k];
        xn[b * 6 + k] = x[k];
    }
    float a1[64];
    for (int o = 0; o < 64; ++o) {
        float z = P[kOffB1 + o];
        for (int k = 0; k < 6; ++k) z = fmaf(P[kOffW1 + o * 6 + k], x[k], z);
        a1[o] = tanhf(z);
        h1[b * 64 + o] = a1[o];
    }
    float y = P[kOffB3];
    for (int o = 0; o < 64; ++o) {
        float z = P[kOffB2 + o];
        for (int k = 0; k < 64; ++k) z = fmaf(P[kOffW2 + o * 64 + k], a1[k], z);
        const float a2 = tanhf(z);
        h2[b * 64 + o] = a2;
        y = fmaf(P[kOffW3 + o], a2, y);
    }
    const float r = y - target[b];
    r2[b] = r * r;
    const float g = 2.0f * r / (float)B;
    dy[b] = g;
    float dh1[64];
    for (int k = 0; k < 64; ++k) dh1[k] = 0.0f;
    for (int o = 0; o < 64; ++o) {
        const float a2 = h2[b * 64 + o];
        const float d2 = g * P[kOffW3 + o] * (1.0f - a2 * a2);
        dz2[b * 64 + o] = d2;
        for (int k = 0; k < 64; ++k) dh1[k] = fmaf(P[kOffW2 + o * 64 + k], d2, dh1[k]);
    }
    for (int k = 0; k < 64; ++k) dz1[b * 64 + k] = dh1[k] * (1.0f - a1[k] * a1[k]);
}

// grad[p] = sum_b left[b][row(p)] * right[b][col(p)] for each weight, plus
// bias gradients and the loss.  One thread per gradient entry.
__global__ void mlp_grad_kernel(const float *xn, const float *h1, const float *h2,
                                const float *dy, const float *dz2, const float *dz1,
                                const float *r2, int64_t B, float *grad, float *loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kMlpParams) return;
    float acc = 0.0f;
    if (p < kOffB1) {  // W1[o][k]
        const int o = p / 6, k = p % 6;
        for (int64_t b = 0; b < B; ++b) acc = fmaf(dz1[b * 64 + o], xn[b * 6 + k], acc);
    } else if (p < kOffW2) {
        const int o = p - kOffB1;
        for (int64_t b = 0; b < B; ++b) acc += dz1[b * 64 + o];
    } else if (p < kOffB2) {  // W2[o][k]
        const int q = p - kOffW2, o = q / 64, k = q % 64;
        for (int64_t b = 0; b < B; ++b) acc = fmaf(dz2[b * 64 + o], h1[b * 64 + k], acc);
    } else if (p < kOffW3) {
        const int o = p - kOffB2;
        for (int64_t b = 0; b < B; ++b) acc += dz2[b * 64 + o];
    } else if (p < kOffB3) {
        const int o = p - kOffW3;
        for (int64_t b = 0; b < B; ++b) acc = fmaf(dy[b], h2[b * 64 + o], acc);
    } else if (p == kOffB3) {
        for (int64_t b = 0; b < B; ++b) acc += dy[b];
    } else {  // p == kMlpParams: the loss
        for (int64_t b = 0; b < B; ++b) acc += r2[b];
        acc /= (float)B;
        *loss = acc;
        return;
    }
    grad[p] = acc;
}

__global__ void adam_kernel(float *P, float *m, float *v, const float *g, int n, float lr,
                            float b1t, float b2t)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float b1 = 0.9f, b2 = 0.999f;
    const float gi = g[p];
    const float mi = b1 * m[p] + (1.0f - b1) * gi;
    const float vi = b2 * v[p] + (1.0f - b2) * gi * gi;
    m[p] = mi;
    v[p] = vi;
    const float mh = mi / (1.0f - b1t), vh = vi / (1.0f - b2t);
    P[p] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// ------------------------------------------------------------ inference
__global__ void mlp_eval_kernel(const MlpWeights *Wg, const float *feat, int64_t count,
                                float *out)
{
    __shared__ MlpWeights W;
    __shared__ __nv_bfloat16 stage[4][32 * 16];
    mlp_load_shared(W, Wg);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float f[6] = {0, 0, 0, 0, 0, 0};
    if (k < count)
        for (int q = 0; q < 6; ++q) f[q] = feat[k * 6 + q];
    const float g = mlp_eval_warp(W, stage[wib], f);
    (void)lane;
    if (k < count) out[k] = g;
}

// blob (host FP32, kMlpBlob floats) -> device MlpWeights (BF16 weights)
__global__ void mlp_pack_kernel(const float *blob, MlpWeights *W)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const float *P = blob;
    if (t < 64 * 16) {
        const int n = t / 16, k = t % 16;
        W->W1[t] = __float2bfloat16_rn(k < 6 ? P[kOffW1 + n * 6 + k] : 0.0f);
    }
    if (t < 64 * 64) W->W2[t] = __float2bfloat16_rn(P[kOffW2 + t]);
    if (t < 8 * 64) {
        const int n = t / 64, k = t % 64;
        W->W3[t] = __float2bfloat16_rn(n == 0 ? P[kOffW3 + k] : 0.0f);
    }
    if (t < 64) {
        W->b1[t] = P[kOffB1 + t];
        W->b2[t] = P[kOffB2 + t];
    }
    if (t < 6) {
        W->mean[t] = P[kMlpParams + t];
        W->inv_scale[t] = 1.0f / P[kMlpParams + 6 + t];
    }
    if (t == 0) {
        W->b3 = P[kOffB3];
        W->oscale = P[kMlpParams + 12];
        W->oshift = P[kMlpParams + 13];
    }
}

// --------------------------------------------------------------- launchers
void launch_sample_pairs(const double *X, int64_t n, double tau, double pre, const int64_t *ids,
                         int64_t count, float *feat, float *target, int *iters, double tol,
                         unsigned *status, cudaStream_t s)
{
    const int64_t blocks = (count + 127) / 128;
    sample_pairs_kernel<<<(unsigned)blocks, 128, 0, s>>>(X, n, tau, pre, ids, count, feat, target,
                                                         iters, tol, status);
}

void launch_mlp_grad(const float *P, const float *norm, const float *feat, const float *target,
                     int64_t B, float *scratch, float *grad, float *loss, cudaStream_t s)
{
    float *xn = scratch;
    float *h1 = xn + B * 6;
    float *h2 = h1 + B * 64;
    float *dz2 = h2 + B * 64;
    float *dz1 = dz2 + B * 64;
    float *dy = dz1 + B * 64;
    float *r2 = dy + B;
    mlp_fwd_bwd_kernel<<<(unsigned)((B + 63) / 64), 64, 0, s>>>(P, norm, feat, target, B, xn, h1,
                                                                h2, dy, dz2, dz1, r2);
    mlp_grad_kernel<<<(kMlpParams + 1 + 127) / 128, 128, 0, s>>>(xn, h1, h2, dy, dz2, dz1, r2, B,
                                                                 grad, loss);
}

size_t mlp_grad_scratch_floats(int64_t B) { return (size_t)B * (6 + 64 * 4 + 2); }

void launch_adam(float *P, float *m, float *v, const float *g, float lr, float b1t, float b2t,
                 cudaStream_t s)
{
    adam_kernel<<<(kMlpParams + 127) / 128, 128, 0, s>>>(P, m, v, g, kMlpParams, lr, b1t, b2t);
}

void launch_mlp_pack(const float *blob, MlpWeights *W, cudaStream_t s)
{
    mlp_pack_kernel<<<(64 * 64 + 127) / 128, 128, 0, s>>>(blob, W);
}

void launch_mlp_eval(const MlpWeights *W, const float *feat, int64_t count, float *out,
                     cudaStream_t s)
{
    mlp_eval_kernel<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(W, feat, count, out);
}

}  // namespace sakura
