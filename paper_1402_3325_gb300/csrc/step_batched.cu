// step_batched.cu -- many independent small systems in one persistent launch.
//
// The systems of an ensemble never interact, so a warp can take a system (or
// several small ones) and run all requested steps on it without any
// synchronisation beyond its own lanes: the state lives in shared memory for
// the whole launch.
//
// Each unordered pair is solved once (Newton's third law, as in the symmetric
// single-system kernel): the increments of (i, j) and (j, i) are exact
// negatives, so the solving lane adds m_j delta / m_ij to i and
// -m_i delta / m_ij to j (Eq. 23).  A system of N >= 2 particles takes
// h = floor(N / 2) lanes and walks its pairs in the round-robin ("circle")
// order, so that its lanes x rounds equal its N (N - 1) / 2 pairs:
//   N even, M = N - 1: round r = 0 .. M-1 pairs particle M with particle r
//     (lane 0 of the system) and (r + k) mod M with (r - k) mod M (lane k =
//     1 .. h-1);
//   N odd: round r = 0 .. N-1 pairs (r + k) mod N with (r - k) mod N (lane
//     k - 1 for k = 1 .. h); particle r sits the round out.
// No particle is in two pairs of a round, so the lanes add to disjoint
// accumulators (shared memory, in round order: deterministic); over the
// rounds every unordered pair comes up exactly once.  A single particle
// takes one lane and no rounds.
//
// Schedule (built on the host when the offsets change): systems are packed
// best-fit-decreasing into tasks of at most 32 lanes and kBatchMaxN = 64
// particles (build_batch_schedule); a task's lockstep length is the largest
// round count among its systems.  Tasks are sorted by that length and
// handed out through an atomic counter (dynamic longest-first), one task to
// a block at a time.
//
// Per step, per block: lane k of a system drifts its particles 2k and 2k + 1
// (and the last particle of an odd system, on its last lane) (Eq. 27a),
// the rounds run as warp-synchronous FP64 Kepler solves (same solver as the
// single-system kernel) split over the block's warps, and after a block
// barrier each lane applies Eqs. 27b-d to its particles.  Each system keeps
// its own dt.
//
// The counter reset and the launch form a CUDA graph that is built once per
// (buffers, schedule, nsteps, order, launch shape) and replayed.  A small
// autotuner times the candidate block shapes on a scratch copy of the state
// the first time a schedule is used.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstring>
#include <numeric>
#include <vector>

#include "kepler_df64.cuh"
#include "kepler_fp64.cuh"
#include "mlp_infer.cuh"
#include "pair_batch_fp64.cuh"
#include "step_common.cuh"
#include "step_batched.cuh"

namespace sakura {

constexpr int kBatchMaxN = 64;

// lanes and rounds of a system of N particles (see above)
__host__ __device__ __forceinline__ int batch_lanes(int N) { return N < 2 ? 1 : N / 2; }
__host__ __device__ __forceinline__ int batch_rounds(int N)
{
    return N < 2 ? 0 : ((N & 1) ? N : N - 1);
}

// One task per block: its WARPS warps share the task's state in shared
// memory and split the rounds of every step, warp w taking rounds r = w,
// w + WARPS, ... into its own accumulators; the apply adds the WARPS
// accumulators in warp order (deterministic).  A warp's solve round is
// latency-bound, so the largest systems (63 rounds per step for N = 64) set
// the length of the launch; splitting their rounds shortens it.
// SEED: the single-precision seed and the Taylor carry of the symmetric
// FP64 kernel (float copies of the drifted state in shared memory, hi + lo
// positions, refreshed after every drift).
// Dynamic shared memory: the accumulators [WARPS][6][kBatchMaxN] doubles,
// then (LEARNED) the network and its per-warp staging.
template <int WARPS, bool STATS, bool LEARNED, bool SEED>
__global__ void __launch_bounds__(WARPS * 32)
    batched_kernel(BatchArgs a)
{
    __shared__ double S[7][kBatchMaxN];
    __shared__ float S32[SEED ? 10 : 1][kBatchMaxN];
    __shared__ int s_task;
    extern __shared__ __align__(16) unsigned char dsm[];
    double(*shacc)[6][kBatchMaxN] = reinterpret_cast<double(*)[6][kBatchMaxN]>(dsm);
    unsigned char *dnet = dsm + (size_t)WARPS * 6 * kBatchMaxN * sizeof(double);
    MlpWeights *mlpW = reinterpret_cast<MlpWeights *>(dnet);
    __nv_bfloat16 *mlpStage = reinterpret_cast<__nv_bfloat16 *>(dnet + sizeof(MlpWeights));
    if (LEARNED) mlp_load_shared(*mlpW, a.mlp);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    double(*A)[kBatchMaxN] = shacc[wib];
    const int64_t tot = a.total;
    const KeplerParams kp{a.tol, a.max_iter, a.bisection};
    unsigned status = 0;
    long long it_sum = 0, slots = 0, fallbacks = 0, carries = 0;
    int it_max = 0;

    while (true) {
        if (threadIdx.x == 0) s_task = atomicAdd(a.counter, 1);
        __syncthreads();
        const int t = s_task;
        if (t >= a.ntasks) break;
        const int sb = a.task_begin[t], se = a.task_begin[t + 1];
        // the lane's system: its particles at my_base .. my_base + my_N - 1,
        // the lane's index my_k in the system (-1: no system); the same in
        // every warp of the block
        int my_k = -1, my_base = 0, my_N = 0;
        double dt = 0.0;
        int base = 0, lbase = 0;
        for (int q = sb; q < se; ++q) {
            const int k = a.task_sys[q];
            const int64_t o0 = a.offsets[k];
            const int Nk = (int)(a.offsets[k + 1] - o0);
            for (int pi = threadIdx.x; pi < Nk; pi += WARPS * 32) {
#pragma unroll
                for (int c = 0; c < 6; ++c) S[c][base + pi] = a.state[c * tot + o0 + pi];
                const double m = a.mass[o0 + pi];
                if (!(m > 0.0)) status |= kStatusMass;
                S[6][base + pi] = m;
            }
            const int hk = batch_lanes(Nk);
            if (lane >= lbase && lane < lbase + hk) {
                my_k = lane - lbase;
                my_base = base;
                my_N = Nk;
                dt = a.dt[k];
            }
            base += Nk;
            lbase += hk;
        }
        __syncthreads();
        const bool odd = (my_N & 1) != 0;
        const int rounds = my_k >= 0 ? batch_rounds(my_N) : 0;
        const int M = odd ? my_N : my_N - 1;  // circle length
        const int maxr = __reduce_max_sync(0xffffffffu, rounds);
        // the lane's particles 2k, 2k + 1 (and, on the last lane of an odd
        // system, 2k + 2 = N - 1): drift, accumulators, apply
        const int np = my_k < 0 ? 0
                                : (my_N < 2 ? 1
                                            : 2 + ((odd && my_k == batch_lanes(my_N) - 1) ? 1 : 0));

        for (int64_t sub = 0; sub < (int64_t)a.nsteps * a.nsub; ++sub) {
            // sub-step sub % nsub of the composition (one sub-step for orders 2, 1, -1)
            const double tau = dt * a.sub[(int)(sub % a.nsub)];
            const double drift = a.drift_frac * tau;
            const double post_drift = a.post_drift_frac * tau;
            const double qtau = a.post * tau;
            for (int e = 0; e < np; ++e) {
                const int i = my_base + 2 * my_k + e;
                if (wib == 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) S[c][i] = fma(S[3 + c][i], drift, S[c][i]);
                    if (SEED) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float hi = __double2float_rn(S[c][i]);
                            S32[c][i] = hi;
                            S32[3 + c][i] = __double2float_rn(S[c][i] - (double)hi);
                            S32[6 + c][i] = __double2float_rn(S[3 + c][i]);
                        }
                        S32[9][i] = __double2float_rn(S[6][i]);
                    }
                }
#pragma unroll
                for (int c = 0; c < 6; ++c) A[c][i] = 0.0;
            }
            __syncthreads();
            const float ptau32 = (float)(a.pre * tau), t32 = (float)tau;
            for (int r = wib; r < maxr; r += WARPS) {
                // the lane's pair of round r (local indices)
                int il = my_N, jl = 0;
                if (r < rounds) {
                    if (!odd && my_k == 0) {
                        il = M;
                        jl = r;
                    } else {
                        const int k = odd ? my_k + 1 : my_k;
                        il = r + k;
                        if (il >= M) il -= M;
                        jl = r - k;
                        if (jl < 0) jl += M;
                    }
                }
                const bool valid = il < my_N;
                const int i = my_base + il, j = my_base + jl;
                PairSolve p;
                double mi = 0.0, mj = 0.0;
                if (valid) {
                    mi = S[6][i];
                    mj = S[6][j];
                    K32 o;
                    if (SEED) {
                        // single-precision seed: the root of the FP32 solve of
                        // the same pair (unless t is reduced modulo the period)
                        float dr[3], dv[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            dr[c] = __fadd_rn(__fsub_rn(S32[c][i], S32[c][j]),
                                              __fsub_rn(S32[3 + c][i], S32[3 + c][j]));
                            dv[c] = __fsub_rn(S32[6 + c][i], S32[6 + c][j]);
                        }
                        o = k32_phase1(dr, dv, S32[9][i] + S32[9][j], ptau32, t32, 2);
                    }
                    pair_setup(p, tau, mi + mj, S[0][i] - S[0][j], S[1][i] - S[1][j],
                               S[2][i] - S[2][j], S[3][i] - S[3][j], S[4][i] - S[4][j],
                               S[5][i] - S[5][j], a.pre, LEARNED ? 2 : (SEED ? -1 : a.guess));
                    if (SEED) {
                        if (o.ok && __double_as_longlong(p.t) == __double_as_longlong(tau) &&
                            !p.done) {
                            p.s = f2d(o.s);
                        } else if (!p.done) {
                            // no usable seed: the second-order guess, as
                            // pair_setup computes it
                            p.s = p.t * p.ir0;
                            const double cq = 0.5 * p.s * (p.eta0 * p.ir0);
                            if (magbits(cq) < 0x3fe0000000000000LL) p.s = fma(-cq, p.s, p.s);
                        }
                    }
                } else {
                    p.done = true;
                    p.beta = p.s = 0.0;
                    p.iters = 0;
                    p.status = 0;
                }
                if (LEARNED) learned_guess_warp(p, valid, *mlpW, mlpStage + wib * 32 * 16);
                double d[6];
                int iters = 0, fb = 0;
                fp64_solve_warp<SEED>(p, valid, tau, qtau, kp, d, iters, fb);
                if (STATS) carries += (valid && p.carried) ? 1 : 0;
                if (valid) {
                    // i and j are in no other lane's pair of this round; the
                    // warp's own accumulators
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        A[q][i] = fma(mj, d[q], A[q][i]);
                        A[q][j] = fma(-mi, d[q], A[q][j]);
                    }
                    status |= p.status;
                }
                if (STATS) {
                    it_sum += iters;
                    fallbacks += fb;
                    it_max = max(it_max, iters);
                    const int wmax = __reduce_max_sync(0xffffffffu, iters);
                    if (lane == 0) slots += 32LL * wmax;
                }
                __syncwarp();  // the warp's next round reads these sums
            }
            __syncthreads();
            if (wib == 0) {
                for (int e = 0; e < np; ++e) {
                    const int i = my_base + 2 * my_k + e;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        double sr = shacc[0][c][i], sv = shacc[0][3 + c][i];
#pragma unroll
                        for (int w = 1; w < WARPS; ++w) {
                            sr += shacc[w][c][i];
                            sv += shacc[w][3 + c][i];
                        }
                        const double v1 = S[3 + c][i] + sv;
                        S[c][i] = fma(v1, post_drift, S[c][i] + sr);
                        S[3 + c][i] = v1;
                    }
                }
            }
            __syncthreads();
        }
        // write the task's systems back
        base = 0;
        for (int q = sb; q < se; ++q) {
            const int k = a.task_sys[q];
            const int64_t o0 = a.offsets[k];
            const int Nk = (int)(a.offsets[k + 1] - o0);
            for (int pi = threadIdx.x; pi < Nk; pi += WARPS * 32) {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    const double x = S[c][base + pi];
                    if (!isfinite(x)) status |= kStatusNonfinite;
                    a.state[c * tot + o0 + pi] = x;
                }
            }
            base += Nk;
        }
        __syncthreads();
    }
    status = __reduce_or_sync(0xffffffffu, status);
    if (lane == 0 && status) atomicOr(a.status, status);
    if (STATS) {
        long long s1 = it_sum, s2 = slots, s3 = fallbacks, s4 = carries;
        int mx = it_max;
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            s3 += __shfl_xor_sync(0xffffffffu, s3, o);
            s4 += __shfl_xor_sync(0xffffffffu, s4, o);
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            atomicAdd(&a.stats[kStatIters], (unsigned long long)s1);
            atomicAdd(&a.stats[kStatSlots], (unsigned long long)s2);
            atomicAdd(&a.stats[kStatFallbacks], (unsigned long long)s3);
            atomicAdd(&a.stats[kStatCarries], (unsigned long long)s4);
            atomicMax(&a.stats[kStatMaxIters], (unsigned long long)mx);
        }
    }
}

namespace {

template <int W>
const void *kernel_ptr(bool stats, bool learned, bool seed)
{
    if (learned)
        return stats ? (const void *)batched_kernel<W, true, true, false>
                     : (const void *)batched_kernel<W, false, true, false>;
    if (seed)
        return stats ? (const void *)batched_kernel<W, true, false, true>
                     : (const void *)batched_kernel<W, false, false, true>;
    return stats ? (const void *)batched_kernel<W, true, false, false>
                 : (const void *)batched_kernel<W, false, false, false>;
}

const void *batched_kernel_ptr(int warps, bool stats, bool learned, bool seed)
{
    switch (warps) {
    case 1: return kernel_ptr<1>(stats, learned, seed);
    case 2: return kernel_ptr<2>(stats, learned, seed);
    case 8: return kernel_ptr<8>(stats, learned, seed);
    default: return kernel_ptr<4>(stats, learned, seed);
    }
}

size_t batched_dyn_smem(int warps, bool learned)
{
    return (size_t)warps * 6 * kBatchMaxN * sizeof(double) +
           (learned ? sizeof(MlpWeights) + (size_t)warps * 32 * 16 * 2 : 0);
}

// kernel pointer, with its dynamic shared memory allowed (above 48 KB per
// block with the static arrays for 8 warps)
const void *batched_kernel_ready(int warps, bool stats, bool learned, bool seed)
{
    const void *fn = batched_kernel_ptr(warps, stats, learned, seed);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)batched_dyn_smem(warps, learned));
    return fn;
}

}  // namespace

int batched_blocks_per_sm(int warps, bool stats, bool learned, bool seed)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b,
                                                      batched_kernel_ready(warps, stats, learned,
                                                                           seed),
                                                      warps * 32,
                                                      batched_dyn_smem(warps, learned)) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return b > 0 ? b : 1;
}

// Schedule: systems packed best-fit-decreasing into warps of at most 32
// lanes (batch_lanes) and kBatchMaxN particles (the shared-memory state):
// each system, largest first, goes to the open warp with the fewest free
// lanes that still takes it (warps kept in buckets by free lanes, so every
// placement looks at 33 buckets, not at every warp).  On the 4096-system
// ensemble (N uniform in [3, 64]) this fills 88 % of the lane-rounds, where
// first fit over only the most recent warps filled 79 %.  Tasks are sorted
// by cost (the lockstep length, the task's largest round count) so the
// atomic counter hands out the longest first.
void build_batch_schedule(const int64_t *offsets, int nsys, std::vector<int> &task_begin,
                          std::vector<int> &task_sys)
{
    std::vector<int> order(nsys);
    std::iota(order.begin(), order.end(), 0);
    auto size = [&](int k) { return (int)(offsets[k + 1] - offsets[k]); };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return size(a) > size(b); });
    struct Bin {
        int lanes;  // free lanes
        int room;   // free particle slots
        int cost;
        std::vector<int> sys;
    };
    std::vector<Bin> bins;
    std::vector<std::vector<int>> by_free(33);  // open bins by free lanes
    for (int k : order) {
        const int N = size(k);
        const int h = batch_lanes(N), rounds = batch_rounds(N);
        int chosen = -1;
        for (int f = h; f <= 32 && chosen < 0; ++f) {
            std::vector<int> &bl = by_free[f];
            // the 8 most recent bins of the bucket (a bin can lack particle
            // room for a system whose lanes it has; the bound keeps every
            // placement O(33 x 8) however many such bins collect)
            for (int q = (int)bl.size() - 1; q >= 0 && q >= (int)bl.size() - 8; --q) {
                if (bins[bl[q]].room >= N) {
                    chosen = bl[q];
                    bl.erase(bl.begin() + q);
                    break;
                }
            }
        }
        if (chosen < 0) {
            chosen = (int)bins.size();
            bins.push_back({32, kBatchMaxN, 0, {}});
        }
        Bin &b = bins[chosen];
        b.lanes -= h;
        b.room -= N;
        b.sys.push_back(k);
        b.cost = std::max(b.cost, rounds);
        by_free[b.lanes].push_back(chosen);
    }
    std::stable_sort(bins.begin(), bins.end(),
                     [](const Bin &a, const Bin &b) { return a.cost > b.cost; });
    task_begin.assign(1, 0);
    task_sys.clear();
    for (const Bin &b : bins) {
        for (int k : b.sys) task_sys.push_back(k);
        task_begin.push_back((int)task_sys.size());
    }
}

void launch_batched(const BatchArgs &a, int warps, int blocks, bool stats, cudaStream_t s)
{
    const bool learned = a.mlp != nullptr;
    void *args[] = {(void *)&a};
    cudaLaunchKernel(batched_kernel_ready(warps, stats, learned, a.seed != 0), dim3(blocks),
                     dim3(warps * 32), args, batched_dyn_smem(warps, learned), s);
}

cudaError_t build_batched_graph(const BatchArgs &a, int warps, int blocks, bool stats,
                                cudaGraphExec_t *exec)
{
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    cudaMemsetParams mp;
    std::memset(&mp, 0, sizeof(mp));
    mp.dst = (void *)a.counter;
    mp.value = 0;
    mp.elementSize = sizeof(int);
    mp.width = 1;
    mp.height = 1;
    mp.pitch = sizeof(int);
    cudaGraphNode_t mset = nullptr, kern = nullptr;
    e = cudaGraphAddMemsetNode(&mset, graph, nullptr, 0, &mp);
    if (e == cudaSuccess) {
        BatchArgs copy = a;
        void *args[] = {(void *)&copy};
        cudaKernelNodeParams kpar;
        std::memset(&kpar, 0, sizeof(kpar));
        kpar.func = (void *)batched_kernel_ready(warps, stats, a.mlp != nullptr, a.seed != 0);
        kpar.gridDim = dim3(blocks);
        kpar.blockDim = dim3(warps * 32);
        kpar.sharedMemBytes = (unsigned)batched_dyn_smem(warps, a.mlp != nullptr);
        kpar.kernelParams = args;
        e = cudaGraphAddKernelNode(&kern, graph, &mset, 1, &kpar);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

}  // namespace sakura
