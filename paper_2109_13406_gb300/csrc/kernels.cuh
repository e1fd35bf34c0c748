// Internal launch interfaces between the C ABI (abi.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "mpdd.h"

namespace mpdd {

// One dd Rgemm / Rsyrk problem, already validated by the ABI layer.
struct GemmArgs {
    int64_t m, n, k;
    mp_dd alpha, beta;
    const double *ah, *al;
    int64_t lda;
    const double *bh, *bl;
    int64_t ldb;
    double *ch, *cl;
    int64_t ldc;
    int ta, tb;      // op(A), op(B): 0 = as stored, 1 = transposed
    int tri;         // 0 = full C (Rgemm); 1 = upper, 2 = lower triangle (Rsyrk)
    int alpha_zero;  // alpha == 0: A and B are not read
    int alpha_one;   // alpha == 1: the product is stored without scaling
    int beta_zero;   // beta == 0: C is write-only
    const int64_t *info = nullptr;  // optional device word: non-zero -> leave C as is
    // Rsyr2k: a second product op(A2) op(B2) (same transposes and k) summed
    // into the same accumulators after the first; a2h == nullptr: none.
    const double *a2h = nullptr, *a2l = nullptr, *b2h = nullptr, *b2l = nullptr;
    int64_t lda2 = 0, ldb2 = 0;
    // Rsymm: op(A) (sym_a) or op(B) (sym_b) is symmetric with one triangle
    // stored: 0 = no, 1 = upper stored, 2 = lower stored (transpose flag 0).
    int sym_a = 0, sym_b = 0;
    // Fallback of a split-precision call: when gate != nullptr the kernel
    // computes C only if *gate (the call's certificate margin, as bits) is
    // below gate_below, i.e. when no operand width certified the bound.
    const unsigned int *gate = nullptr;
    unsigned int gate_below = 0;
};

// Plain FP64 dd kernel (64 x 64 output tiles, 4 x 4 dd accumulators per thread).
int launch_gemm_plain(const GemmArgs &p, cudaStream_t stream);
// The TMA-staged form of the plain kernel (dd_gemm_tma.cu): 1 when it took the
// problem (*rc its launch status), 0 when the register-staged kernels must.
int try_launch_gemm_tma(const GemmArgs &p, cudaStream_t stream, int *rc);
// Busiest-SM time of the plain kernel on 16r x 16r tiles, in units of a 16 x
// 16 tile (ceil(tiles / SMs) r^2), and the r the register path takes.
int64_t plain_tile_cost(const GemmArgs &p, int r);
int plain_tile_r(const GemmArgs &p);
// Operand staging of the plain kernel: 0 automatic, 1 registers, 2 TMA.
void set_plain_staging(int mode);
int plain_staging();
// CTA pairs for the 256-wide split-precision band products (dd_sliced.cu):
// 0 for triangle products (the default), 1 wherever they apply, 2 never.
void set_band_pairs(int mode);

// FP64 issue-rate microbenchmark; *rate in FP64 instructions per second.
int run_peak_fp64(cudaStream_t stream, double *rate);
// INT8 warp-level tensor rate (mma.sync m16n8k32 s8); *rate in integer ops/s.
int run_peak_imma(cudaStream_t stream, double *rate);
// dd multiply-add rate of the plain kernel's instruction mix (registers only).
int run_peak_ddmac(cudaStream_t stream, double *rate);

// Split-precision (sliced) Rgemm on the fp16 tensor cores.
constexpr int kDefaultSlices = 14;  // base-256 digits per operand entry
constexpr int kMaxSlices = 15;      // the slicing integer must fit 128 bits
size_t sliced_workspace_bytes(int64_t m, int64_t n, int64_t k, int slices);
int sliced_layout(int64_t m, int64_t n, int64_t k, int slices, size_t *offsets);
int run_sliced(const GemmArgs &p, int slices, void *ws, size_t ws_bytes, cudaStream_t stream);
int read_status(const void *ws, int *status);
// The certificate and width of the last split-precision call on `ws`.
int split_report(const void *ws, mp_dd_split_info *info);
// Byte offsets of the certificate's magnitude planes (op(A), op(B)^T).
int sliced_magnitude_offsets(int64_t m, int64_t n, int64_t k, int slices, size_t *offsets);
int crt_magnitude_offsets(int64_t m, int64_t n, int64_t k, bool sym, size_t *offsets);
void sliced_timing_enable(int on);
void sliced_timing_mark(int phase, cudaStream_t stream);  // phases 0..3 of a timed call
int sliced_timing_read(float *ms);
int sliced_timing_log(float *ms, int max_calls, int *calls);

// Grouped dd Rgemm (one persistent launch over many problems).
size_t grouped_workspace_bytes(int64_t count, const mp_dd_gemm_desc *descs);
int grouped_prepare(int64_t count, const mp_dd_gemm_desc *descs, void *ws, size_t bytes,
                    cudaStream_t stream);
int grouped_run(void *ws, cudaStream_t stream);

// dd Cholesky (blocked, LAPACK order) and its building blocks.
int run_potrf(int lower, int64_t n, double *ah, double *al, int64_t lda, int64_t *info,
              cudaStream_t stream, void *ws = nullptr, size_t ws_bytes = 0);
size_t potrf_crt_workspace_bytes(int64_t n);
int run_dd_elementwise(int op, int64_t n, const double *xh, const double *xl, const double *yh,
                       const double *yl, double *zh, double *zl, cudaStream_t stream);
int run_potrs(int lower, int64_t n, int64_t nrhs, const double *ah, const double *al,
              int64_t lda, double *bh, double *bl, int64_t ldb, const int64_t *info,
              cudaStream_t stream);
// dd Rtrsm (every side / uplo / trans / diag variant), alpha != 0, m, n > 0.
int run_trsm(int right, int lower, int trans, int unit, int64_t m, int64_t n, mp_dd alpha,
             const double *ah, const double *al, int64_t lda, double *bh, double *bl,
             int64_t ldb, cudaStream_t stream);
// dd Rgetrf / Rgetrs (recursive LU with partial pivoting); ipiv one-based,
// device memory; info device int64 (LAPACK convention).
int run_getrf(int64_t m, int64_t n, double *ah, double *al, int64_t lda, int64_t *ipiv,
              int64_t *info, cudaStream_t stream);
int run_getrs(int trans, int64_t n, int64_t nrhs, const double *ah, const double *al,
              int64_t lda, const int64_t *ipiv, double *bh, double *bl, int64_t ldb,
              cudaStream_t stream);
int launch_potrf_diag_batch(int64_t count, const mp_dd_potrf_diag_desc *ds, cudaStream_t st);
int launch_trsm_batch(int64_t count, const mp_dd_trsm_desc *ds, int64_t max_rhs,
                      cudaStream_t st);

// Residue (CRT) form of the split-precision Rgemm.
size_t crt_workspace_bytes(int64_t m, int64_t n, int64_t k, bool sym = false);
int crt_layout_query(int64_t m, int64_t n, int64_t k, size_t *offsets, int *count);
// p.tri != 0: the Rsyrk form (op(B) = op(A)^T, one triangle of C).
int run_crt(const GemmArgs &p, void *ws, size_t ws_bytes, cudaStream_t stream);

// Quad-double Rgemm (four planes per matrix, four components per scalar).
int run_qd_gemm(int ta, int tb, int64_t m, int64_t n, int64_t k, const double *alpha,
                const double *const *a, int64_t lda, const double *const *b, int64_t ldb,
                const double *beta, double *const *c, int64_t ldc, cudaStream_t stream);

// Sliced Rgemm on the library's built-in scratch array (no allocation).
size_t noalloc_scratch_bytes();
int run_sliced_noalloc(const GemmArgs &p, int slices, cudaStream_t stream);
int noalloc_report(mp_dd_split_info *info);

}  // namespace mpdd
