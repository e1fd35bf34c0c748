// Roofline denominators measured on the device itself.
//
// FP64 issue rate: every thread runs 8 independent chains of fused
// multiply-adds (enough independent work to cover the FP64 pipe latency),
// with a grid of 8 CTAs x 256 threads per SM.  The chain values stay
// bounded (x <- x * b + c with |b| < 1) so no operand becomes denormal.
//
// INT8 tensor rate of the warp-level path: sm_103a has no tcgen05 kind::i8,
// so the only INT8 x INT8 -> INT32 tensor instruction is the legacy
// mma.sync.m16n8k32 (s8 inputs, exact s32 accumulation).  Every warp runs
// kImmaChains independent accumulator chains on register operands (no memory
// traffic), 8 warps per CTA and 4 CTAs per SM, so the measured rate is the
// issue ceiling of that instruction.
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

constexpr int kImmaChains = 6;

// D (16 x 8 s32) += A (16 x 32 s8, row) B (32 x 8 s8, col), one warp.
__device__ __forceinline__ void imma_m16n8k32(int (&d)[4], const uint32_t (&a)[4],
                                              const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(256) imma_chains(int *out, int iters) {
    // small non-zero bytes that differ between lanes; the sums wrap harmlessly
    const uint32_t s = 0x01010101u * (1u + (threadIdx.x & 7u));
    uint32_t a[4] = {s, s ^ 0x02020202u, s ^ 0x03030303u, s ^ 0x04040404u};
    uint32_t b[2] = {s ^ 0x05050505u, s ^ 0x06060606u};
    int d[kImmaChains][4];
#pragma unroll
    for (int q = 0; q < kImmaChains; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) d[q][r] = q + r;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kImmaChains; ++q) imma_m16n8k32(d[q], a, b);
    }
    int sum = 0;
#pragma unroll
    for (int q = 0; q < kImmaChains; ++q) sum += d[q][0] + d[q][1] + d[q][2] + d[q][3];
    if (sum == 0x7fffabcd) out[blockIdx.x] = sum;  // keeps the chains live
}

}  // namespace

int run_peak_imma(cudaStream_t stream, double *rate) {
    const int sms = sm_count();
    const int blocks = sms * 4, threads = 256, iters = 1 << 14;
    int *out = nullptr;
    cudaError_t e = cudaMallocAsync(&out, sizeof(int) * blocks, stream);
    if (e != cudaSuccess) return cuda_fail(e, "peak_imma alloc");
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(t0, stream);
        imma_chains<<<blocks, threads, 0, stream>>>(out, iters);
        cudaEventRecord(t1, stream);
        cudaEventSynchronize(t1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (rep > 0 && ms < best) best = ms;  // first launch is warm-up
    }
    int rc = check_launch("imma_chains");
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFreeAsync(out, stream);
    cudaStreamSynchronize(stream);
    if (rc) return rc;
    // one m16n8k32 = 16 * 8 * 32 multiply-adds = 8192 integer operations
    const double warps = (double)blocks * threads / 32.0;
    *rate = warps * (double)iters * kImmaChains * 8192.0 / (best * 1e-3);
    return 0;
}

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
