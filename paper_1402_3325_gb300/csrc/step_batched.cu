// step_batched.cu -- many independent small systems in one persistent launch.
//
// The systems of an ensemble never interact, so a block can take a few of
// them and run all requested steps on them with their state in shared memory
// for the whole launch.
//
// Each unordered pair is solved once (Newton's third law, as in the
// symmetric single-system kernel): the increments of (i, j) and (j, i) are
// exact negatives.  A task is a set of systems of at most kBatchMaxN = 64
// particles in all.  Its pairs are numbered system by system, row by row
// within a system (pair (a, b), a < b, of a system of N particles at
// a N - a (a + 1) / 2 + b - a - 1 after the pairs of the systems before it),
// and packed densely over the lanes: lane l of chunk c solves pair 32 c + l,
// chunks dealt out over the block's warps.  (A warp instruction costs the
// FP64 pipe the same however many lanes are active, so dense packing matters:
// a round-robin order, n / 2 lanes for n - 1 rounds per system, filled 88 %
// of the lanes on the 4096-system ensemble; this fills 99 %.)  A task has at
// most 64 * 63 / 2 = 2016 pairs, whose increments divided by m_ab go to
// shared memory; after a block barrier element (i, c) adds particle i's
// increments of component c over its own system in ascending j (+m_j d for
// the pair (i, j), -m_j d for (j, i); Eq. 23 with 1/m_i folded in), a fixed
// order independent of the packing and of the block shape, and applies
// Eqs. 27b-d.  The per-particle work (drift and sums) runs on consecutive
// threads (element e on thread e), so that a warp's lanes mostly hold one
// system (one loop length) and as few warps as possible issue it: the kernel
// is bound by the FP64 pipe's throughput, and a warp instruction costs the
// same however many of its lanes work.  The step's time values of each
// particle's system (tau, post tau and their single-precision copies) are
// formed once per particle and sub-step, not once per pair.
//
// Schedule (built on the host when the offsets change): systems packed
// best-fit-decreasing by particles into tasks of at most 64; tasks sorted by
// pair count and handed out through an atomic counter (dynamic
// longest-first), one task to a block at a time.  Each system keeps its own
// dt.
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

// The FP64 operations formed on the integer pipes (kepler_fp64.cuh), per
// initial guess, as measured on 4096 planetary systems: the increments', the
// setup's and the iterations' multiplies with the seed (9.47e9 -> 1.15e10
// N^2 steps/s; 1.08e10 with the increments' only), none with the learned
// guess (no change measured), the increments' and the iterations'
// multiplies with the standard guess (6.36e9 -> 8.53e9; 7.94e9 with the
// setup's too).
constexpr int kBatEmuSeed = kEmuIncMul | kEmuSetupMul | kEmuIterMul;
constexpr int kBatEmuLearned = 0;
constexpr int kBatEmuStandard = kEmuIncMul | kEmuIterMul;

// the sign bit of a double, flipped by an integer XOR
constexpr long long kSignBit = (long long)0x8000000000000000ULL;

constexpr int kBatchMaxN = 64;                                      // particles of a task
constexpr int kBatchMaxPairs = kBatchMaxN * (kBatchMaxN - 1) / 2;  // 2016

// pair index of (a, b), a < b, within a system of N particles
__host__ __device__ __forceinline__ int local_pair(int a, int b, int N)
{
    return a * N - a * (a + 1) / 2 + b - a - 1;
}

// One task per block; WARPS warps share its state in shared memory.
// SEED: the single-precision seed and the Taylor carry of the symmetric FP64
// kernel (float copies of the drifted state, hi + lo positions, refreshed
// after every drift).  LEARNED: the network guess.
// Dynamic shared memory: the increments D[6][kBatchMaxPairs] doubles, then
// (LEARNED) the network and its per-warp staging.
template <int WARPS, bool STATS, bool LEARNED, bool SEED>
__global__ void __launch_bounds__(WARPS * 32)
    batched_kernel(BatchArgs a)
{
    constexpr int kBatEmu = SEED ? kBatEmuSeed : (LEARNED ? kBatEmuLearned : kBatEmuStandard);
    __shared__ double S[7][kBatchMaxN];
    __shared__ float S32[SEED ? 10 : 1][kBatchMaxN];
    __shared__ double Pdt[kBatchMaxN];           // the particle's system's dt
    __shared__ double Ptau[kBatchMaxN], Pqtau[kBatchMaxN];  // tau, post tau of the sub-step
    __shared__ float Pptau32[kBatchMaxN], Pt32[kBatchMaxN];  // (float)(pre tau), (float)tau
    __shared__ unsigned char Pbase[kBatchMaxN];  // its system's first slot
    __shared__ unsigned char PN[kBatchMaxN];     // its system's size
    __shared__ unsigned short Ppb[kBatchMaxN];   // its system's first pair
    __shared__ unsigned char PA[kBatchMaxPairs], PB[kBatchMaxPairs];
    __shared__ int s_task;
    extern __shared__ __align__(16) unsigned char dsm[];
    double(*D)[kBatchMaxPairs] = reinterpret_cast<double(*)[kBatchMaxPairs]>(dsm);
    unsigned char *dnet = dsm + (size_t)6 * kBatchMaxPairs * sizeof(double);
    MlpWeights *mlpW = reinterpret_cast<MlpWeights *>(dnet);
    __nv_bfloat16 *mlpStage = reinterpret_cast<__nv_bfloat16 *>(dnet + sizeof(MlpWeights));
    if (LEARNED) mlp_load_shared(*mlpW, a.mlp);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
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
        // load the task's systems, their per-particle data and pair table
        int npart = 0, npairs = 0;
        for (int q = sb; q < se; ++q) {
            const int k = a.task_sys[q];
            const int64_t o0 = a.offsets[k];
            const int Nk = (int)(a.offsets[k + 1] - o0);
            const double dtk = a.dt[k];
            for (int pi = threadIdx.x; pi < Nk; pi += WARPS * 32) {
                const int i = npart + pi;
#pragma unroll
                for (int c = 0; c < 6; ++c) S[c][i] = a.state[c * tot + o0 + pi];
                const double m = a.mass[o0 + pi];
                if (!(m > 0.0)) status |= kStatusMass;
                S[6][i] = m;
                Pdt[i] = dtk;
                Pbase[i] = (unsigned char)npart;
                PN[i] = (unsigned char)Nk;
                Ppb[i] = (unsigned short)npairs;
                int p = npairs + local_pair(pi, pi + 1, Nk);  // the pairs (pi, b), b > pi
                for (int b = pi + 1; b < Nk; ++b, ++p) {
                    PA[p] = (unsigned char)i;
                    PB[p] = (unsigned char)(npart + b);
                }
            }
            npart += Nk;
            npairs += Nk * (Nk - 1) / 2;
        }
        __syncthreads();
        const int chunks = (npairs + 31) >> 5;

        for (int64_t sub = 0; sub < (int64_t)a.nsteps * a.nsub; ++sub) {
            // sub-step sub % nsub of the composition (one sub-step for orders 2, 1, -1)
            const double w = a.sub[(int)(sub % a.nsub)];
            for (int e = threadIdx.x; e < 3 * npart; e += WARPS * 32) {  // Eq. 27a, (i, c)
                const int c = e / npart, i = e - c * npart;
                const double tau = Pdt[i] * w;
                if (c == 0) {
                    Ptau[i] = tau;
                    Pqtau[i] = a.post * tau;
                    Pptau32[i] = (float)(a.pre * tau);
                    Pt32[i] = (float)tau;
                }
                const double x = fma(S[3 + c][i], a.drift_frac * tau, S[c][i]);
                S[c][i] = x;
                if (SEED) {
                    const float hi = __double2float_rn(x);
                    S32[c][i] = hi;
                    S32[3 + c][i] = __double2float_rn(x - (double)hi);
                    S32[6 + c][i] = __double2float_rn(S[3 + c][i]);
                    if (c == 0) S32[9][i] = __double2float_rn(S[6][i]);
                }
            }
            __syncthreads();
            for (int ch = wib; ch < chunks; ch += WARPS) {
                const int p = 32 * ch + lane;
                const bool valid = p < npairs;
                const int i = valid ? PA[p] : 0, j = valid ? PB[p] : 0;
                const double tau = Ptau[i];
                PairSolve ps;
                if (valid) {
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
                        o = k32_phase1(dr, dv, S32[9][i] + S32[9][j], Pptau32[i], Pt32[i], 2);
                    }
                    pair_setup<kBatEmu>(ps, tau, S[6][i] + S[6][j], S[0][i] - S[0][j],
                                        S[1][i] - S[1][j], S[2][i] - S[2][j], S[3][i] - S[3][j],
                                        S[4][i] - S[4][j], S[5][i] - S[5][j], a.pre,
                                        LEARNED ? 2 : (SEED ? -1 : a.guess));
                    if (SEED) {
                        if (o.ok && dbits(ps.t) == dbits(tau) &&
                            !ps.done) {
                            ps.s = f2d(o.s);
                        } else if (!ps.done) {
                            // no usable seed: the second-order guess, as
                            // pair_setup computes it
                            ps.s = ps.t * ps.ir0;
                            const double cq = 0.5 * ps.s * (ps.eta0 * ps.ir0);
                            if (magbits(cq) < 0x3fe0000000000000LL) ps.s = fma(-cq, ps.s, ps.s);
                        }
                    }
                } else {
                    ps.done = true;
                    ps.beta = ps.s = 0.0;
                    ps.iters = 0;
                    ps.status = 0;
                }
                if (LEARNED) learned_guess_warp(ps, valid, *mlpW, mlpStage + wib * 32 * 16);
                double d[6];
                int iters = 0, fb = 0;
                fp64_solve_warp<SEED, kBatEmu>(ps, valid, tau, Pqtau[i], kp, d, iters, fb);
                if (valid) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) D[q][p] = d[q];
                    status |= ps.status;
                }
                if (STATS) {
                    carries += (valid && ps.carried) ? 1 : 0;
                    it_sum += iters;
                    fallbacks += fb;
                    it_max = max(it_max, iters);
                    const int wmax = __reduce_max_sync(0xffffffffu, iters);
                    if (lane == 0) slots += 32LL * wmax;
                }
            }
            __syncthreads();
            // Eqs. 23 and 27b-d: element (i, c) sums particle i's increments
            // of component c over its system in ascending j and updates v_c, x_c
            for (int e = threadIdx.x; e < 3 * npart; e += WARPS * 32) {
                const int c = e / npart, i = e - c * npart;
                const int b0 = Pbase[i], N = PN[i], pb = Ppb[i], ai = i - b0;
                double sr = 0.0, sv = 0.0;
                for (int aj = 0; aj < N; ++aj) {
                    if (aj == ai) continue;
                    // the pair (j, i) for j < i gives -m_j d, the pair (i, j)
                    // +m_j d; the sign set by an integer XOR of the sign bit
                    // (the same bits as -m_j, without an FP64 instruction;
                    // one loop, so the lanes of a warp do not diverge)
                    const int p = pb + local_pair(min(ai, aj), max(ai, aj), N);
                    const double wj = __longlong_as_double(
                        dbits(S[6][b0 + aj]) ^ (aj < ai ? kSignBit : 0LL));
                    sr = fma(wj, D[c][p], sr);
                    sv = fma(wj, D[3 + c][p], sv);
                }
                const double v1 = S[3 + c][i] + sv;
                S[c][i] = fma(v1, a.post_drift_frac * Ptau[i], S[c][i] + sr);
                S[3 + c][i] = v1;
            }
            __syncthreads();
        }
        // write the task's systems back
        int base = 0;
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
    return (size_t)6 * kBatchMaxPairs * sizeof(double) +
           (learned ? sizeof(MlpWeights) + (size_t)warps * 32 * 16 * 2 : 0);
}

// kernel pointer, with its dynamic shared memory allowed (the increments
// take 94.5 KB)
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

// Schedule: systems packed best-fit-decreasing by particles into tasks of at
// most kBatchMaxN particles: each system, largest first, goes to the open
// task with the least room that still takes it (tasks kept in buckets by
// free room, so a placement looks at 65 buckets).  A task's work is its
// pair count, which fills ceil(pairs / 32) warp-wide chunks: on the
// 4096-system ensemble (N uniform in [3, 64]) 99 % of the lanes are busy.
// Tasks are sorted by pair count so the atomic counter hands out the
// longest first.
void build_batch_schedule(const int64_t *offsets, int nsys, std::vector<int> &task_begin,
                          std::vector<int> &task_sys)
{
    std::vector<int> order(nsys);
    std::iota(order.begin(), order.end(), 0);
    auto size = [&](int k) { return (int)(offsets[k + 1] - offsets[k]); };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return size(a) > size(b); });
    struct Bin {
        int room;   // free particle slots
        int pairs;  // unordered pairs of its systems
        std::vector<int> sys;
    };
    std::vector<Bin> bins;
    std::vector<std::vector<int>> by_room(kBatchMaxN + 1);  // open bins by free room
    for (int k : order) {
        const int N = size(k);
        int chosen = -1;
        for (int f = N; f <= kBatchMaxN && chosen < 0; ++f) {
            if (!by_room[f].empty()) {
                chosen = by_room[f].back();
                by_room[f].pop_back();
            }
        }
        if (chosen < 0) {
            chosen = (int)bins.size();
            bins.push_back({kBatchMaxN, 0, {}});
        }
        Bin &b = bins[chosen];
        b.room -= N;
        b.pairs += N * (N - 1) / 2;
        b.sys.push_back(k);
        by_room[b.room].push_back(chosen);
    }
    std::stable_sort(bins.begin(), bins.end(),
                     [](const Bin &a, const Bin &b) { return a.pairs > b.pairs; });
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
