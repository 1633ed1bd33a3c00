// energy.cu -- total energy E = T + U of a device state (Eqs. 1-3).
//
// Stage 1: each warp takes row pairs (i, n-1-i) so that every warp sees the
// same number of pair terms, lanes stride over j > i, and every lane keeps a
// double-double (two-sum) accumulator of -m_i m_j / r_ij.  Warps reduce their
// lanes in double-double and write one (hi, lo) pair each.
// Stage 2: one block adds the kinetic terms m_i v_i^2 / 2 and the warp
// partials in a fixed order, in double-double.  No atomics on FP64 data; the
// result does not depend on timing.
#include <cuda_runtime.h>

#include "kepler_fp64.cuh"
#include "step_common.cuh"

namespace sakura {
namespace {

constexpr int kEnergyThreads = 256;
constexpr int kEnergyBlocks = 152 * 4;

__device__ __forceinline__ void dd_add(double &s, double &c, double x)
{
    const double t = s + x;
    const double bp = t - s;
    const double e = (s - (t - bp)) + (x - bp);
    s = t;
    c += e;
}

__device__ __forceinline__ void dd_merge(double &s, double &c, double s2, double c2)
{
    dd_add(s, c, s2);
    c += c2;
}

__device__ __forceinline__ void row_potential(const double *state, const double *mass, int64_t n,
                                              int64_t i, int lane, double &s, double &c,
                                              unsigned &st)
{
    const double xi = state[i], yi = state[n + i], zi = state[2 * n + i], mi = mass[i];
    for (int64_t j = i + 1 + lane; j < n; j += 32) {
        const double dx = xi - state[j], dy = yi - state[n + j], dz = zi - state[2 * n + j];
        const double d = sqrt(fma(dx, dx, fma(dy, dy, dz * dz)));
        if (!(d > 0.0)) st |= kStatusCoincident;
        dd_add(s, c, -(mi * mass[j]) / d);
    }
}

__global__ void __launch_bounds__(kEnergyThreads)
    energy_pairs_kernel(const double *state, const double *mass, int64_t n, double *work,
                        unsigned *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double s = 0.0, c = 0.0;
    unsigned st = 0;
    const int64_t half = (n + 1) / 2;
    for (int64_t r = w; r < half; r += W) {
        row_potential(state, mass, n, r, lane, s, c, st);
        const int64_t r2 = n - 1 - r;
        if (r2 != r) row_potential(state, mass, n, r2, lane, s, c, st);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const double c2 = __shfl_xor_sync(0xffffffffu, c, o);
        // combine in a lane-order-independent way: the lower lane id keeps its
        // own value first, so both partners compute the same bits
        if ((lane & o) == 0) {
            dd_merge(s, c, s2, c2);
        } else {
            double a = s2, b = c2;
            dd_merge(a, b, s, c);
            s = a;
            c = b;
        }
    }
    st = __reduce_or_sync(0xffffffffu, st);
    if (lane == 0) {
        work[w] = s;
        work[W + w] = c;
        if (st) atomicOr(status, st);
    }
}

__global__ void __launch_bounds__(1024)
    energy_final_kernel(const double *state, const double *mass, int64_t n, const double *work,
                        int64_t W, double *out)
{
    __shared__ double sh_s[1024], sh_c[1024], sh_t[1024], sh_tc[1024];
    const int t = threadIdx.x;
    double ks = 0.0, kc = 0.0, us = 0.0, uc = 0.0;
    for (int64_t i = t; i < n; i += blockDim.x) {
        const double vx = state[3 * n + i], vy = state[4 * n + i], vz = state[5 * n + i];
        dd_add(ks, kc, 0.5 * mass[i] * fma(vx, vx, fma(vy, vy, vz * vz)));
    }
    for (int64_t w = t; w < W; w += blockDim.x) dd_merge(us, uc, work[w], work[W + w]);
    sh_s[t] = us;
    sh_c[t] = uc;
    sh_t[t] = ks;
    sh_tc[t] = kc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (t < h) {
            double a = sh_s[t], b = sh_c[t];
            dd_merge(a, b, sh_s[t + h], sh_c[t + h]);
            sh_s[t] = a;
            sh_c[t] = b;
            double p = sh_t[t], q = sh_tc[t];
            dd_merge(p, q, sh_t[t + h], sh_tc[t + h]);
            sh_t[t] = p;
            sh_tc[t] = q;
        }
        __syncthreads();
    }
    if (t == 0) {
        double es = 0.0, ec = 0.0;
        dd_merge(es, ec, sh_t[0], sh_tc[0]);
        dd_merge(es, ec, sh_s[0], sh_c[0]);
        out[0] = es + ec;
        out[1] = sh_t[0] + sh_tc[0];
        out[2] = sh_s[0] + sh_c[0];
    }
}

}  // namespace

int energy_work_size(int64_t n)
{
    (void)n;
    return 2 * kEnergyBlocks * (kEnergyThreads / 32);
}

void launch_energy(const double *state, const double *mass, int64_t n, double *work, int nwork,
                   double *out, unsigned *status, cudaStream_t s)
{
    (void)nwork;
    energy_pairs_kernel<<<kEnergyBlocks, kEnergyThreads, 0, s>>>(state, mass, n, work, status);
    const int64_t W = (int64_t)kEnergyBlocks * (kEnergyThreads / 32);
    energy_final_kernel<<<1, 1024, 0, s>>>(state, mass, n, work, W, out);
}

}  // namespace sakura
