// Roofline denominators measured on the device itself.
//
// FP64 issue rate: every thread runs 8 independent chains of fused
// multiply-adds (enough independent work to cover the FP64 pipe latency),
// with a grid of 8 CTAs x 256 threads per SM.  The chain values stay
// bounded (x <- x * b + c with |b| < 1) so no operand becomes denormal.
//
// dd multiply-add rate: the plain kernel's own multiply-add (mac_deferred,
// renorm every kRenormEvery steps) on a 4 x 4 block of accumulators per
// thread, with operands that change every step through integer operations
// on their bit patterns (no FP64 instruction and no memory access besides
// the multiply-adds, and nothing the compiler can hoist): the ceiling of the
// plain kernel's instruction mix on this GPU's FP64 pipe.
//
// INT8 tensor rate of the warp-level path: sm_103a has no tcgen05 kind::i8,
// so the only INT8 x INT8 -> INT32 tensor instruction is the legacy
// mma.sync.m16n8k32 (s8 inputs, exact s32 accumulation).  Every warp runs
// kImmaChains independent accumulator chains on register operands (no memory
// traffic), 8 warps per CTA and 4 CTAs per SM, so the measured rate is the
// issue ceiling of that instruction.
#include "common.cuh"
#include "dd_arith.cuh"
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

__global__ void __launch_bounds__(256) ddmac_mix(double *out, int iters) {
    dd acc[16];
    long long ab[4], bb[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        ab[r] = __double_as_longlong(0.5 + 1e-3 * r + 1e-6 * threadIdx.x);
        bb[r] = __double_as_longlong(0.75 - 1e-3 * r);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = dd{1e-3 * (threadIdx.x + q), 0.0};
    for (int it = 0; it < iters; ++it) {
#pragma unroll 1
        for (int l4 = 0; l4 < 16; l4 += kRenormEvery) {
#pragma unroll
            for (int l = l4; l < l4 + kRenormEvery; ++l) {
                const long long v = (long long)((it * 16 + l) & 255);
                dd a[4], b[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    // low parts 60 binades below: normalised dd operands
                    a[r] = dd{__longlong_as_double(ab[r] ^ v),
                              __longlong_as_double((ab[r] ^ v) - (60ll << 52))};
                    b[r] = dd{__longlong_as_double(bb[r] ^ (v << 3)),
                              __longlong_as_double((bb[r] ^ v) - (61ll << 52))};
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) mac_deferred(acc[4 * r + c], a[r], b[c]);
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) renorm(acc[q]);
        }
    }
    double sum = 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q) sum += acc[q].hi + acc[q].lo;
    if (sum == 12345.678) out[blockIdx.x] = sum;  // keeps the accumulators live
}

}  // namespace

int run_peak_ddmac(cudaStream_t stream, double *rate) {
    const int sms = sm_count();
    const int blocks = sms, threads = 256, iters = 1 << 7;
    double *out = nullptr;
    cudaError_t e = cudaMallocAsync(&out, sizeof(double) * blocks, stream);
    if (e != cudaSuccess) return cuda_fail(e, "peak_ddmac alloc");
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(t0, stream);
        ddmac_mix<<<blocks, threads, 0, stream>>>(out, iters);
        cudaEventRecord(t1, stream);
        cudaEventSynchronize(t1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (rep > 0 && ms < best) best = ms;  // first launch is warm-up
    }
    int rc = check_launch("ddmac_mix");
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFreeAsync(out, stream);
    cudaStreamSynchronize(stream);
    if (rc) return rc;
    // 16 steps x 16 multiply-adds per thread and iteration
    *rate = (double)blocks * threads * (double)iters * 256.0 / (best * 1e-3);
    return 0;
}

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
