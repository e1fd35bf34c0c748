// Roofline denominators measured on the device itself.
//
// FP64 issue rate: every thread runs 8 independent chains of fused
// multiply-adds (enough independent work to cover the FP64 pipe latency),
// with a grid of 8 CTAs x 256 threads per SM.  The chain values stay
// bounded (x <- x * b + c with |b| < 1) so no operand becomes denormal.
#include "common.cuh"
#include "kernels.cuh"

namespace mpdd {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fp64_fma_chains(double *out, int iters, double b,
                                                       double c) {
    double x[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = 1e-3 * (threadIdx.x + q + 1);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) x[q] = __fma_rn(x[q], b, c);
    }
    double sum = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) sum += x[q];
    if (sum == 12345.678) out[blockIdx.x] = sum;  // keeps the chains live
}

}  // namespace

int run_peak_fp64(cudaStream_t stream, double *rate) {
    const int sms = sm_count();
    const int blocks = sms * 8, threads = 256, iters = 1 << 13;
    double *out = nullptr;
    cudaError_t e = cudaMallocAsync(&out, sizeof(double) * blocks, stream);
    if (e != cudaSuccess) return cuda_fail(e, "peak_fp64 alloc");
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(t0, stream);
        fp64_fma_chains<<<blocks, threads, 0, stream>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(t1, stream);
        cudaEventSynchronize(t1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (rep > 0 && ms < best) best = ms;  // first launch is warm-up
    }
    int rc = check_launch("fp64_fma_chains");
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFreeAsync(out, stream);
    cudaStreamSynchronize(stream);
    if (rc) return rc;
    *rate = (double)blocks * threads * (double)iters * kChains / (best * 1e-3);
    return 0;
}

}  // namespace mpdd
