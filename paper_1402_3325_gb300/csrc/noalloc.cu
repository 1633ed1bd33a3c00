// noalloc.cu -- sakura_step_noalloc: an FP64 step without any device
// allocation.
//
// Some callers cannot call cudaMalloc.  A host program whose device memory is
// entirely held by another allocator (for example a framework's caching
// allocator that has reserved the GPU) gets out-of-memory from it, and a
// latency-critical loop cannot afford cudaMalloc/cudaFree, which may
// synchronise the device.  For them this entry point runs the ordered-pair
// FP64 kernels of sakura_step (every ordered pair solved, standard initial
// guess t/r0, tolerance 4 eps, 50 Laguerre steps, bisection fallback; it
// reads no sakura_config), but keeps the pair kernel's row-sum scratch and
// the fault status word in file-scope device arrays that exist for as long
// as the library is loaded.
//
// Limits and sharing rules:
//   - n <= SAKURA_NOALLOC_MAX_N (65536); larger n returns SAKURA_E_ARG.
//   - The scratch (20 x 65536 doubles = 10 MiB) and the status word are shared
//     by every call on a device and keep the last call's contents.  Every
//     scratch entry a call reads is written earlier in the same call; the
//     status word is cleared at the start of each call.  Calls whose work
//     overlaps on the GPU (other streams, other host threads) race on both.
//   - The first call on a device looks up the arrays' device addresses with
//     cudaGetSymbolAddress while that device is current; make that first call
//     before any stream capture.  Host threads may make their first calls
//     concurrently: each device's look-up runs once (std::call_once) and
//     later calls see its result.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>

#include "kepler_fp64.cuh"
#include "sakura.h"
#include "step_common.cuh"

namespace {

constexpr int64_t kMaxN = SAKURA_NOALLOC_MAX_N;
// drifted state X[7][n] plus the pair kernel's row partials, ceil(W/n) + 1
// slots of 6 n doubles for W warps.  While W <= n that is 2 slots, 19 n
// doubles, within 20 kMaxN for every n <= kMaxN; the launch below halves
// the grid until the layout fits (smaller n may use W > n).
constexpr int64_t kScratchDoubles = 20 * kMaxN;
constexpr int kMaxDevices = 64;

// The host-side names below are stand-ins for device memory: host code never
// dereferences them and only passes the addresses returned by
// cudaGetSymbolAddress to kernels.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];
static __device__ __align__(256) unsigned g_noalloc_status[64];

struct DeviceSymbols {
    int rc = SAKURA_E_CUDA;  // result of the look-up
    double *scratch = nullptr;
    unsigned *status = nullptr;
    int sm_count = 152;
};

DeviceSymbols g_dev[kMaxDevices];
std::once_flag g_dev_once[kMaxDevices];

// Device addresses of the arrays on device dev (the calling thread's current
// device), looked up once per device; the once_flag orders the look-up
// before every later read of its result.
int setup_device(int dev, DeviceSymbols **out)
{
    if (dev < 0 || dev >= kMaxDevices) return SAKURA_E_ARG;
    DeviceSymbols &d = g_dev[dev];
    std::call_once(g_dev_once[dev], [&d, dev]() {
        void *p = nullptr, *q = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p ||
            cudaGetSymbolAddress(&q, g_noalloc_status) != cudaSuccess || !q) {
            cudaGetLastError();
            d.rc = SAKURA_E_CUDA;
            return;
        }
        d.scratch = (double *)p;
        d.status = (unsigned *)q;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            sms > 0)
            d.sm_count = sms;
        d.rc = SAKURA_OK;
    });
    if (d.rc != SAKURA_OK) return d.rc;
    *out = &d;
    return SAKURA_OK;
}

int code_from_status(unsigned st)
{
    if (st & sakura::kStatusMass) return SAKURA_E_MASS;
    if (st & sakura::kStatusNonfinite) return SAKURA_E_NONFINITE;
    if (st & sakura::kStatusCoincident) return SAKURA_E_COINCIDENT;
    if (st & sakura::kStatusKepler) return SAKURA_E_KEPLER;
    if (st & sakura::kStatusTimeout) return SAKURA_E_TIMEOUT;
    return SAKURA_OK;
}

}  // namespace

extern "C" int sakura_step_noalloc(double *state, const double *masses, int64_t n, double dt,
                                   int order, void *stream)
{
    if (!state || !masses || n < 1 || !std::isfinite(dt)) return SAKURA_E_ARG;
    if (!(order == 2 || order == 1 || order == -1)) return SAKURA_E_ARG;
    if (n > kMaxN) return SAKURA_E_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SAKURA_E_CUDA;
    }
    DeviceSymbols *d = nullptr;
    int rc = setup_device(dev, &d);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;

    // persistent grid: one wave of resident blocks, within the fixed scratch
    const int warps = 4;
    const int64_t nb = (n + 31) / 32;
    const int64_t B = n * nb;
    int64_t blocks = (int64_t)d->sm_count * sakura::pair_step_fp64_blocks_per_sm(warps, false);
    // at most one warp per 32-pair batch, so every slot of a row is written
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, B / warps));
    while (blocks > 1 &&
           7 * n + sakura::pair_step_slots(n, blocks * warps) * 6 * n > kScratchDoubles)
        blocks /= 2;
    if (7 * n + sakura::pair_step_slots(n, blocks * warps) * 6 * n > kScratchDoubles)
        return SAKURA_E_ARG;  // unreachable for n <= kMaxN (19 n <= 20 kMaxN at W <= n)
    const int64_t W = blocks * warps;
    double *X = d->scratch;
    double *partial = X + 7 * n;

    if (cudaMemsetAsync(d->status, 0, sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return SAKURA_E_CUDA;
    }
    const double drift = order == 2 ? 0.5 * dt : (order == 1 ? 0.0 : dt);
    const double post_drift = order == 2 ? 0.5 * dt : (order == 1 ? dt : 0.0);
    sakura::launch_prep_step(state, masses, X, nullptr, n, drift, d->status, s);
    sakura::StepArgs a{};
    a.X = X;
    a.partial = partial;
    a.n = n;
    a.tau = dt;
    a.pre = order == 2 ? 0.5 : (order == 1 ? 0.0 : 1.0);
    a.post = 1.0 - a.pre;
    a.tol = 4.0 * DBL_EPSILON;
    a.max_iter = 50;
    a.bisection = 1;
    a.guess = 0;
    a.mlp = nullptr;
    a.status = d->status;
    a.stats = nullptr;
    if (n > 1) sakura::launch_pair_step_fp64(a, warps, (int)blocks, false, s);
    sakura::launch_apply_step(state, X, partial, n, n > 1 ? W : 0, post_drift, d->status, s);
    if (cudaGetLastError() != cudaSuccess) return SAKURA_E_CUDA;
    unsigned st = 0;
    if (cudaMemcpyAsync(&st, d->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return SAKURA_E_CUDA;
    }
    return code_from_status(st);
}
