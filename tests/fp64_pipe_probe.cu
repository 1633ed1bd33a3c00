// FP64 pipe throughput on this GPU, for the roofline of the FP64 kernels.
//
// Every warp of a one-wave grid (152 x 16 warps of 32 threads on GB300) runs
// 8 independent chains of kSteps fused multiply-adds on its first k lanes
// (the other lanes return at once).  The printed rate of warp instructions
// per second shows whether a partly active warp costs the pipe less than a
// full one; the rate at k = 32 is the pipe's sustained FMA throughput.
// Each active thread reads one double and writes one (in bounds: the arrays
// hold one double per thread of the grid).
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

constexpr int kSteps = 4096;

__global__ void fma_chains(const double *in, double *out, int k)
{
    const int lane = threadIdx.x & 31;
    if (lane >= k) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double a0 = in[i], a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    double a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    for (int c = 0; c < kSteps; ++c) {
        a0 = fma(a0, 0.9999999, 1e-9);
        a1 = fma(a1, 0.9999999, 1e-9);
        a2 = fma(a2, 0.9999999, 1e-9);
        a3 = fma(a3, 0.9999999, 1e-9);
        a4 = fma(a4, 0.9999999, 1e-9);
        a5 = fma(a5, 0.9999999, 1e-9);
        a6 = fma(a6, 0.9999999, 1e-9);
        a7 = fma(a7, 0.9999999, 1e-9);
    }
    out[i] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

int main()
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int blocks = sms * 16, threads = 32, n = blocks * threads;
    double *in = nullptr, *out = nullptr;
    if (cudaMalloc(&in, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&out, n * sizeof(double)) != cudaSuccess)
        return 1;
    cudaMemset(in, 0, n * sizeof(double));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int ks[] = {32, 16, 8, 1};
    for (int k : ks) {
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0);
            fma_chains<<<blocks, threads>>>(in, out, k);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;  // the first launch warms up
        }
        const double winst = (double)blocks * 8.0 * kSteps;
        printf("k %d ms %.4f warp_inst_per_s %.6e lane_fma_per_s %.6e\n", k, best, winst / (best * 1e-3),
               winst * k / (best * 1e-3));
    }
    const cudaError_t err = cudaGetLastError();
    printf("sms %d status %s\n", sms, cudaGetErrorString(err));
    return err == cudaSuccess ? 0 : 1;
}
