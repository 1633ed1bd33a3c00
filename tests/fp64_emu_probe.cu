// Device check of csrc/fp64_emu.cuh (tests/test_gpu_fp64_emu.py): the
// integer-pipe multiply (also with the first operand negated), add and fused
// multiply-add of the FP64 pair kernels against the GPU's own FP64
// instructions (__dmul_rn, __dadd_rn, __fma_rn), bit for bit, on the operand
// kinds of tests/fp64_emu_cases.h.
//
// Each thread runs kPerThread cases from its own generator state; a grid of
// 4 waves of 256-thread blocks per SM.  Prints one line per operation and
// kind: "op kind cases mismatches fast a b c" (the bits of the first
// mismatch's operands in hex, or zeros).  Buffers: out[5] per launch, in
// bounds (every thread adds to out[0..1], one thread writes out[2..4]).
#include "../paper_1402_3325_gb300/csrc/fp64_emu.cuh"
#include "fp64_emu_cases.h"

#include <cstdio>
#include <cuda_runtime.h>

using namespace sakura;
using namespace emucases;

constexpr int kPerThread = 64;

__global__ void emu_check_kernel(int op, int kind, uint64_t seed, unsigned long long *out,
                                 unsigned *first)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t s = seed ^ (t * 0xd1342543de82ef95ull);
    (void)splitmix(s);
    unsigned long long mism = 0, fast_n = 0;
    for (int i = 0; i < kPerThread; ++i) {
        double a, b, c;
        make_case(s, op, kind, a, b, c);
        double want, got, fast;
        bool took;
        if (op == 0) {
            want = __dmul_rn(a, b);
            got = emu::mul(a, b);
            took = emu::mul_fast(a, b, fast);
        } else if (op == 3) {
            want = __dmul_rn(-a, b);
            got = emu::mul_neg(a, b);
            took = emu::mul_fast<true>(a, b, fast);
        } else if (op == 1) {
            want = __dadd_rn(a, b);
            got = emu::add(a, b);
            took = emu::add_fast(a, b, fast);
        } else {
            want = __fma_rn(a, b, c);
            got = emu::fma(a, b, c);
            took = emu::fma_fast(a, b, c, fast);
        }
        fast_n += took ? 1 : 0;
        if (!same(want, got) || (took && !same(want, fast))) {
            ++mism;
            if (atomicCAS(first, 0u, 1u) == 0u) {
                out[2] = bits(a);
                out[3] = bits(b);
                out[4] = bits(c);
            }
        }
    }
    atomicAdd(&out[0], mism);
    atomicAdd(&out[1], fast_n);
}

int main()
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return 1;
    const int threads = 256, blocks = sms * 4 * 8;
    unsigned long long *out = nullptr;
    unsigned *first = nullptr;
    if (cudaMalloc(&out, 5 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&first, sizeof(unsigned)) != cudaSuccess)
        return 1;
    for (int op = 0; op < 4; ++op) {
        for (int kind = 0; kind <= 6; ++kind) {
            if ((op == 0 || op == 3) && kind == 5) continue;
            cudaMemset(out, 0, 5 * sizeof(unsigned long long));
            cudaMemset(first, 0, sizeof(unsigned));
            emu_check_kernel<<<blocks, threads>>>(op, kind, 0x5EEDull + 131 * kind + op, out,
                                                  first);
            unsigned long long h[5];
            if (cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 2;
            printf("op %d kind %d cases %lld mism %llu fast %llu %016llx %016llx %016llx\n", op,
                   kind, (long long)blocks * threads * kPerThread, h[0], h[1], h[2], h[3], h[4]);
        }
    }
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 3;
}
