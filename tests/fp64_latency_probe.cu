// FP64 issue of a single warp on GB300, for the design of latency-bound
// kernels (the single-block kernel of small systems).
//
// One block of one warp on one SM: the clock64() cycles per operation of
// (a) a dependent chain of FP64 fused multiply-adds, (b) a dependent chain of
// FP64 adds, (c) a dependent chain of FP32 fused multiply-adds and (d) eight
// independent FP64 FMA chains interleaved.  (d) shows how often one warp can
// issue an FP64 instruction at all: the sub-partition's share of the SM's
// FP64 rate.  Each loop runs 256 times; the figures include its counter and
// branch.  The kernel writes one double per thread and four counters.
#include <cstdio>
#include <cuda_runtime.h>

__global__ void latency_chains(double *out, double a, double b, float fa, float fb,
                               long long *cyc)
{
    double x = a, y0 = a, y1 = a + 1, y2 = a + 2, y3 = a + 3, y4 = a + 4, y5 = a + 5,
           y6 = a + 6, y7 = a + 7;
    float f = fa;
    const long long t0 = clock64();
#pragma unroll 1
    for (int k = 0; k < 256; ++k) x = fma(x, b, a);
    const long long t1 = clock64();
#pragma unroll 1
    for (int k = 0; k < 256; ++k) x = x + b;
    const long long t2 = clock64();
#pragma unroll 1
    for (int k = 0; k < 256; ++k) f = fmaf(f, fb, fa);
    const long long t3 = clock64();
#pragma unroll 1
    for (int k = 0; k < 256; ++k) {
        y0 = fma(y0, b, a);
        y1 = fma(y1, b, a);
        y2 = fma(y2, b, a);
        y3 = fma(y3, b, a);
        y4 = fma(y4, b, a);
        y5 = fma(y5, b, a);
        y6 = fma(y6, b, a);
        y7 = fma(y7, b, a);
    }
    const long long t4 = clock64();
    out[threadIdx.x] = x + (double)f + y0 + y1 + y2 + y3 + y4 + y5 + y6 + y7;
    if (threadIdx.x == 0) {
        cyc[0] = t1 - t0;
        cyc[1] = t2 - t1;
        cyc[2] = t3 - t2;
        cyc[3] = t4 - t3;
    }
}

int main()
{
    double *out = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&out, 32 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&cyc, 4 * sizeof(long long)) != cudaSuccess)
        return 1;
    long long h[4] = {0, 0, 0, 0};
    for (int rep = 0; rep < 3; ++rep) {  // the first launch warms up
        latency_chains<<<1, 32>>>(out, 1e-3, 0.999, 1e-3f, 0.999f, cyc);
        if (cudaDeviceSynchronize() != cudaSuccess) return 1;
        cudaMemcpy(h, cyc, sizeof(h), cudaMemcpyDeviceToHost);
    }
    printf("dfma_dep %.1f dadd_dep %.1f ffma_dep %.1f dfma_8chains %.1f\n", h[0] / 256.0,
           h[1] / 256.0, h[2] / 256.0, h[3] / 2048.0);
    const cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? 0 : 1;
}
