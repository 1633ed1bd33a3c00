// step_fp64.cu -- FP64 W-step kernels of the Sakura integrator.
//
// One step = pair kernel + apply kernel, both on the library stream.
//
// pair kernel: block = WARPS warps; warp w of block b owns row
//   i = b * WARPS + w and block column y owns the j segment
//   [y * jchunk, (y+1) * jchunk).  The block stages j-tiles of 256 particles
//   (positions drifted on load, velocities, masses; 14 KB) in shared memory;
//   lane l of a warp solves the pairs (i, j) with j = tile + l + 32k.  Each lane
//   keeps six FP64 accumulators of mu_ij * (delta_r, delta_v) (Eq. 23); the
//   warp reduces them with xor shuffles and lane 0 stores the row's partial
//   sum for its segment in partial[y][6][n].  No atomics touch FP64 data.
// apply kernel: sums the segments in a fixed order (deterministic) and
//   applies Eqs. 27b-d (or the order-1 forms) to the state in place.
#include <cuda_runtime.h>

#include "kepler_fp64.cuh"
#include "step_common.cuh"

namespace sakura {

template <int WARPS, bool STATS>
__global__ void __launch_bounds__(WARPS * 32)
    pair_step_fp64_kernel(StepArgs a)
{
    constexpr int kTile = 256;
    __shared__ double sx[kTile], sy[kTile], sz[kTile], svx[kTile], svy[kTile], svz[kTile],
        sm[kTile];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t n = a.n;
    const int64_t i = (int64_t)blockIdx.x * WARPS + warp;
    const bool row = i < n;
    const int64_t j0 = (int64_t)blockIdx.y * a.jchunk;
    const int64_t j1 = min(n, j0 + a.jchunk);

    double xi = 0, yi = 0, zi = 0, vxi = 0, vyi = 0, vzi = 0, mi = 1;
    if (row) {
        vxi = a.state[3 * n + i];
        vyi = a.state[4 * n + i];
        vzi = a.state[5 * n + i];
        xi = fma(vxi, a.drift, a.state[i]);
        yi = fma(vyi, a.drift, a.state[n + i]);
        zi = fma(vzi, a.drift, a.state[2 * n + i]);
        mi = a.mass[i];
    }
    double acc[6] = {0, 0, 0, 0, 0, 0};
    unsigned status = 0;
    long long it_sum = 0, slots = 0, fallbacks = 0;
    int it_max = 0;
    const KeplerParams kp{a.tol, a.max_iter, a.bisection};

    for (int64_t jt = j0; jt < j1; jt += kTile) {
        __syncthreads();
        for (int q = threadIdx.x; q < kTile; q += WARPS * 32) {
            const int64_t j = jt + q;
            if (j < j1) {
                const double vx = a.state[3 * n + j], vy = a.state[4 * n + j],
                             vz = a.state[5 * n + j];
                svx[q] = vx;
                svy[q] = vy;
                svz[q] = vz;
                sx[q] = fma(vx, a.drift, a.state[j]);
                sy[q] = fma(vy, a.drift, a.state[n + j]);
                sz[q] = fma(vz, a.drift, a.state[2 * n + j]);
                sm[q] = a.mass[j];
            }
        }
        __syncthreads();
        if (!row) continue;
        const int cnt = (int)min((int64_t)kTile, j1 - jt);
        // every lane runs the same trip count; invalid slots are predicated
        for (int kb = 0; kb < cnt; kb += 32) {
            const int k = kb + lane;
            const int64_t j = jt + k;
            const bool valid = (k < cnt) && (j != i);
            int iters = 0;
            if (valid) {
                const double mj = sm[k];
                const double mij = mi + mj;
                const double mu = mi * mj / mij;
                PairResult p = pair_increment_fp64(a.tau, mij, xi - sx[k], yi - sy[k],
                                                   zi - sz[k], vxi - svx[k], vyi - svy[k],
                                                   vzi - svz[k], a.pre, a.post, kp);
                status |= p.status;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    acc[q] = fma(mu, p.dr[q], acc[q]);
                    acc[3 + q] = fma(mu, p.dv[q], acc[3 + q]);
                }
                iters = p.iters;
                fallbacks += p.fallback;
            }
            if (STATS) {
                it_sum += iters;
                it_max = max(it_max, iters);
                const int wmax = __reduce_max_sync(0xffffffffu, iters);
                if (lane == 0) slots += 32LL * wmax;
            }
        }
    }
    // warp reduction of the six row sums
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        double v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[q] = v;
    }
    if (row && lane == 0) {
        double *dst = a.partial + (int64_t)blockIdx.y * 6 * n;
#pragma unroll
        for (int q = 0; q < 6; ++q) dst[q * n + i] = acc[q];
    }
    status = __reduce_or_sync(0xffffffffu, status);
    if (lane == 0 && status) atomicOr(a.status, status);
    if (STATS) {
        long long s1 = it_sum, s2 = slots, s3 = fallbacks;
        int mx = it_max;
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            s3 += __shfl_xor_sync(0xffffffffu, s3, o);
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            atomicAdd(&a.stats[kStatIters], (unsigned long long)s1);
            atomicAdd(&a.stats[kStatSlots], (unsigned long long)s2);
            atomicAdd(&a.stats[kStatFallbacks], (unsigned long long)s3);
            atomicMax(&a.stats[kStatMaxIters], (unsigned long long)mx);
        }
    }
}

// Eqs. 27b-d (order 2) and the first-order forms; sums segment partials in
// segment order.
__global__ void apply_step_kernel(double *state, const double *mass, const double *partial,
                                  int64_t n, int nsplit, double tau, int order,
                                  unsigned *status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d[6] = {0, 0, 0, 0, 0, 0};
    for (int s = 0; s < nsplit; ++s) {
        const double *src = partial + (int64_t)s * 6 * n;
#pragma unroll
        for (int q = 0; q < 6; ++q) d[q] += src[q * n + i];
    }
    const double m = mass[i];
    unsigned st = 0;
    if (!(m > 0.0)) st |= kStatusMass;
    double x[3], v[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        x[q] = state[q * n + i];
        v[q] = state[(3 + q) * n + i];
    }
    if (order == 2) {
        const double h = 0.5 * tau;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double xh = fma(v[q], h, x[q]);        // 27a
            const double xt = xh + d[q] / m;             // 27b
            const double v1 = v[q] + d[3 + q] / m;       // 27c
            x[q] = fma(v1, h, xt);                       // 27d
            v[q] = v1;
        }
    } else if (order == 1) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double xw = x[q] + d[q] / m;
            const double vw = v[q] + d[3 + q] / m;
            x[q] = fma(vw, tau, xw);
            v[q] = vw;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double xd = fma(v[q], tau, x[q]);
            x[q] = xd + d[q] / m;
            v[q] = v[q] + d[3 + q] / m;
        }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (!isfinite(x[q]) || !isfinite(v[q])) st |= kStatusNonfinite;
        state[q * n + i] = x[q];
        state[(3 + q) * n + i] = v[q];
    }
    if (st) atomicOr(status, st);
}

void launch_pair_step_fp64(const StepArgs &a, int warps, int nsplit, bool stats,
                           cudaStream_t s)
{
    const dim3 grid((unsigned)((a.n + warps - 1) / warps), (unsigned)nsplit);
#define SAKURA_LAUNCH(W)                                                               \
    if (stats)                                                                         \
        pair_step_fp64_kernel<W, true><<<grid, W * 32, 0, s>>>(a);                     \
    else                                                                               \
        pair_step_fp64_kernel<W, false><<<grid, W * 32, 0, s>>>(a);
    switch (warps) {
    case 4: SAKURA_LAUNCH(4) break;
    case 16: SAKURA_LAUNCH(16) break;
    default: SAKURA_LAUNCH(8) break;
    }
#undef SAKURA_LAUNCH
}

void launch_apply_step(double *state, const double *mass, const double *partial, int64_t n,
                       int nsplit, double tau, int order, unsigned *status, cudaStream_t s)
{
    const int threads = 256;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    apply_step_kernel<<<blocks, threads, 0, s>>>(state, mass, partial, n, nsplit, tau, order,
                                                 status);
}

}  // namespace sakura
