/*
 * mpdd -- double-double (dd) Rgemm / Rsyrk for one GB300 GPU (sm_103a).
 *
 * C ABI of libmpdd.so.  Semantics follow MPBLAS as described in the
 * MPLAPACK 2.0.1 user manual (arXiv 2109.13406):
 *
 *  - A dd number is the unevaluated sum hi + lo of two binary64 numbers with
 *    |lo| <= ulp(hi)/2 (Sec. 5, "Supported Floating point formats"; the dd
 *    arithmetic is built from Knuth's TwoSum and Dekker's exact product).
 *  - Matrices are one-dimensional column-major arrays with a leading
 *    dimension, element (i, j) at index i + j*ld (Sec. 7.3, "How to use
 *    MPBLAS").  A dd matrix is two such arrays, the hi plane and the lo
 *    plane, which share the leading dimension.
 *  - Argument lists are those of the BLAS/LAPACK routine each call mirrors
 *    (Sec. 7.3 gives the Rgemm prototype and its one-to-one correspondence
 *    with DGEMM: CHARACTER -> const char*, INTEGER -> 64-bit integer, arrays
 *    -> pointers).  Flags are case-insensitive first characters, as with the
 *    BLAS lsame ('N', 'T', 'C'; 'U', 'L'); 'C' means 'T' for real data.
 *
 * Ownership and execution: unless a call says otherwise, every matrix
 * pointer is DEVICE memory owned by the caller, and every call is
 * asynchronous on the calling thread's current stream (mp_dd_set_stream).
 * The library keeps nothing allocated beyond a call except what a call
 * documents (the host forms' memory pool, the no-allocation form's fixed
 * array).
 *
 * Return codes (all int-returning calls):
 *    0            success
 *   -i            argument i (1-based, numbered as in the mirrored BLAS or
 *                 LAPACK routine) is illegal -- the xerbla convention the
 *                 manual's MPBLAS tests compare (Sec. 8.1)
 *   1000 + e      CUDA runtime error e while launching or copying
 *   2001          a device-side wait ran out of time (the kernel stopped
 *                 early; the output is undefined)
 *   2002          requested size beyond a documented limit
 *   2003          workspace too small
 *   2004          the CUDA extension cannot run (no device / wrong arch)
 * mp_dd_last_error() describes the last non-zero return on this thread.
 */
#ifndef MPDD_H
#define MPDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* dd scalar: value = hi + lo (passed by value). */
typedef struct {
    double hi, lo;
} mp_dd;

/* Read-only dd matrix: device hi and lo planes sharing one leading dimension. */
typedef struct {
    const double *hi, *lo;
} mp_dd_cmat;

/* Writable dd matrix planes. */
typedef struct {
    double *hi, *lo;
} mp_dd_mat;

/* Quad-double (qd) scalar: value = x[0] + x[1] + x[2] + x[3], components
 * non-overlapping, largest first (the manual's quad-double format, Sec. 5). */
typedef struct {
    double x[4];
} mp_qd;

/* Read-only qd matrix: four device planes (component t of every entry in
 * plane t) sharing one column-major leading dimension. */
typedef struct {
    const double *x[4];
} mp_qd_cmat;

/* Writable qd matrix planes. */
typedef struct {
    double *x[4];
} mp_qd_mat;

#define MP_DD_OK 0
#define MP_DD_ERR_CUDA_BASE 1000
#define MP_DD_ERR_TIMEOUT 2001
#define MP_DD_ERR_TOO_LARGE 2002
#define MP_DD_ERR_WORKSPACE 2003
#define MP_DD_ERR_NO_DEVICE 2004

/* ------------------------------------------------------------------------ */
/* Streams and errors                                                        */
/* ------------------------------------------------------------------------ */

/* Set the CUDA stream (a cudaStream_t, or NULL for the legacy default
 * stream) used by later calls made from the calling thread.  Returns 0. */
int mp_dd_set_stream(void *stream);

/* The calling thread's current stream. */
void *mp_dd_get_stream(void);

/* Human-readable description of the calling thread's last error ("" if none).
 * The string is owned by the library and valid until the next call. */
const char *mp_dd_last_error(void);

/* Library ABI version (increments when a declaration here changes). */
int mp_dd_version(void);

/* ------------------------------------------------------------------------ */
/* Level-3 MPBLAS: plain double-double path (FP64 DFMA arithmetic)           */
/* ------------------------------------------------------------------------ */

/* Rgemm (manual Sec. 7.3 prototype; Sec. 6 table of MPBLAS routines;
 * CUDA dd Rgemm in Sec. 7.3 "CUDA accelerated MPBLAS"):
 *
 *     C := alpha * op(A) * op(B) + beta * C,   op(X) = X or X^T,
 *
 * op(A) is m x k, op(B) is k x n, C is m x n.  A is stored m x k (transa N)
 * or k x m (T/C) with leading dimension lda >= max(1, rows stored); same
 * for B (k x n or n x k, ldb) and C (m x n, ldc >= max(1, m)).
 * Arithmetic: every multiply-add is dd arithmetic -- the exact product of
 * the hi parts by FMA plus the two cross products, accumulated with TwoSum
 * (exact) with a FastTwoSum renormalisation every 4 steps of k (at the same
 * k positions in every kernel); the summation order over k is fixed
 * (l = 0, 1, ..., k-1), so results are bitwise reproducible run to run and
 * independent of the launch configuration.  Accuracy: componentwise
 * |C - C_exact| <= 4 k 2^-104 (|alpha| |op(A)| |op(B)| + |beta| |C|).
 * BLAS semantics: m == 0, n == 0, or ((alpha == 0 or k == 0) and
 * beta == 1) returns at once; beta == 0 means C is write-only (NaNs in C
 * are not propagated); alpha == 0 means A and B are not read.
 * Errors: -1 transa, -2 transb, -3 m < 0, -4 n < 0, -5 k < 0,
 * -7 A.hi/A.lo NULL, -8 lda, -9 B planes NULL, -10 ldb, -12 C planes NULL,
 * -13 ldc (DGEMM's numbering). */
int mp_dd_Rgemm(const char *transa, const char *transb, int64_t m, int64_t n, int64_t k,
                mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_cmat B, int64_t ldb, mp_dd beta,
                mp_dd_mat C, int64_t ldc);

/* Operand staging of the plain Rgemm / Rsyrk kernel (no counterpart in the
 * manual; process-wide, for tuning and testing).  mode 0 (the default):
 * Rgemm products large enough for 64 x 64 output tiles whose A and B planes
 * start on 16-byte boundaries with even leading dimensions are computed by
 * a kernel whose op(A) / op(B) panels arrive by TMA tile copies into a ring
 * of shared-memory stages (mbarrier-synchronised, one producer warp, eight
 * computing warps); the others (thin products, the Rsyrk triangle) by the
 * register-staged kernels on the tile size that fills the SMs best.  mode 1: register staging only.  mode 2: TMA
 * staging wherever its alignment rules allow, whatever the size.  Every
 * mode gives bitwise the same results (the per-entry operation sequence is
 * the same).  Returns 0, or -1 for another mode. */
int mp_dd_set_plain_staging(int mode);

/* Scheduling of the split-precision band / residue products on 128 x 256
 * tiles (no counterpart in the manual; process-wide, for tuning and
 * testing).  A CTA pair is a cluster of two CTAs computing a 256 x 256 tile
 * with the 2-SM tensor-core MMA: each CTA holds its 128 rows of op(A) and
 * half of the op(B) panel, a third fewer operand bytes per SM; it needs an
 * even number of 128-row tiles.  mode 0 (the default): pairs for the Rsyrk
 * triangle (4 % faster at 8192), one CTA per tile for full products (where
 * pairs measured 2.5 % slower); mode 1: pairs wherever they apply; mode 2:
 * never.  The products are exact integers, so every mode gives bitwise the
 * same results.  Returns 0, or -1 for another mode. */
int mp_dd_set_band_pairs(int mode);

/* Rsyrk (Sec. 6 table; CUDA dd Rsyrk in Sec. 7.3):
 *
 *     C := alpha * A * A^T + beta * C   (trans N, A is n x k), or
 *     C := alpha * A^T * A + beta * C   (trans T/C, A is k x n),
 *
 * updating only the uplo ('U' upper, 'L' lower) triangle of the n x n C;
 * the other triangle is neither read nor written.  Arithmetic and accuracy
 * as mp_dd_Rgemm; every entry of the triangle is bitwise equal to the same
 * entry of mp_dd_Rgemm(N, T) (trans N) or (T, N) (trans T) on A, A.
 * Errors: -1 uplo, -2 trans, -3 n < 0, -4 k < 0, -6 A planes NULL,
 * -7 lda < max(1, n (N) or k (T)), -9 C planes NULL, -10 ldc < max(1, n)
 * (DSYRK's numbering). */
int mp_dd_Rsyrk(const char *uplo, const char *trans, int64_t n, int64_t k, mp_dd alpha,
                mp_dd_cmat A, int64_t lda, mp_dd beta, mp_dd_mat C, int64_t ldc);

/* Rsyr2k (MPBLAS routine table, Sec. 6; DSYR2K semantics):
 *
 *     C := alpha (A B^T + B A^T) + beta C   (trans N, A and B n x k), or
 *     C := alpha (A^T B + B^T A) + beta C   (trans T/C, A and B k x n),
 *
 * updating only the uplo triangle of the n x n C.  Each entry accumulates
 * the k products of the first term and then the k of the second in one dd
 * accumulator (the plain kernel's multiply-add), then applies alpha and
 * beta once.  Accuracy: |C - C_exact| <= 4 (2k) 2^-104 (|alpha| (|A||B^T| +
 * |B||A^T|) + |beta||C|) componentwise (trans N; transposed for T).
 * Quick return and beta = 0 as mp_dd_Rsyrk.  Errors: -1 uplo, -2 trans,
 * -3 n < 0, -4 k < 0, -6 A NULL, -7 lda < max(1, n (N) or k (T)), -8 B NULL,
 * -9 ldb < max(1, n (N) or k (T)), -11 C NULL, -12 ldc < max(1, n)
 * (DSYR2K's numbering). */
int mp_dd_Rsyr2k(const char *uplo, const char *trans, int64_t n, int64_t k, mp_dd alpha,
                 mp_dd_cmat A, int64_t lda, mp_dd_cmat B, int64_t ldb, mp_dd beta,
                 mp_dd_mat C, int64_t ldc);

/* Rsymm (MPBLAS routine table, Sec. 6; DSYMM semantics):
 *
 *     C := alpha A B + beta C   (side L, A m x m), or
 *     C := alpha B A + beta C   (side R, A n x n),
 *
 * A symmetric with only its uplo triangle read (A(i, l) outside it is read
 * as A(l, i)), B and C m x n.  Arithmetic, accuracy (k = order of A) and
 * beta / alpha semantics as mp_dd_Rgemm.  Errors: -1 side, -2 uplo,
 * -3 m < 0, -4 n < 0, -6 A NULL, -7 lda < max(1, order of A), -8 B NULL,
 * -9 ldb < max(1, m), -11 C NULL, -12 ldc < max(1, m) (DSYMM's numbering). */
int mp_dd_Rsymm(const char *side, const char *uplo, int64_t m, int64_t n, mp_dd alpha,
                mp_dd_cmat A, int64_t lda, mp_dd_cmat B, int64_t ldb, mp_dd beta, mp_dd_mat C,
                int64_t ldc);

/* Host-buffer forms of mp_dd_Rgemm and mp_dd_Rsyrk, as the manual's CUDA MPBLAS is
 * used (Sec. 7.3: the caller passes host arrays; the library moves them to
 * the GPU and back -- the "with host-GPU transfer" figures of Sec. 10).
 * All matrix pointers are HOST memory (pinned memory gives the fastest
 * copies).  The call takes device buffers for the operands from a
 * stream-ordered memory pool the library owns (one per device, created at
 * the first such call), copies in, computes, copies C back, returns the
 * buffers to the pool and synchronises the stream before returning.  The
 * pool keeps freed memory mapped for later calls (its release threshold is
 * unlimited): device memory once used by a host-form call stays reserved
 * by the library until the process exits.  Same arguments, accuracy and
 * error codes as the device forms. */
int mp_dd_Rgemm_host(const char *transa, const char *transb, int64_t m, int64_t n, int64_t k,
                     mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_cmat B, int64_t ldb,
                     mp_dd beta, mp_dd_mat C, int64_t ldc);
int mp_dd_Rsyrk_host(const char *uplo, const char *trans, int64_t n, int64_t k, mp_dd alpha,
                     mp_dd_cmat A, int64_t lda, mp_dd beta, mp_dd_mat C, int64_t ldc);

/* Rtrsm (MPBLAS routine table, Sec. 6; DTRSM semantics): solve
 *
 *     op(A) X = alpha B   (side 'L', A m x m), or
 *     X op(A) = alpha B   (side 'R', A n x n),
 *
 * for X, which overwrites the m x n B (column-major dd planes, ldb).  A is
 * upper (uplo 'U') or lower ('L') triangular and only that triangle is
 * read; diag 'U' takes its diagonal as one without reading it, 'N' divides
 * by it.  op(A) = A ('N') or A^T ('T'; 'C' is 'T' for real data).  Flags are
 * case-insensitive.  alpha = 0 sets B to zero without reading A or B; m = 0
 * or n = 0 returns at once.  Arithmetic: substitution on 64 x 64 diagonal
 * blocks (dd division by the diagonal) and dd Rgemm updates of the
 * off-diagonal blocks, split recursively in halves so that the updates are
 * large products.  Accuracy: the componentwise backward error of
 * substitution, |op(A) X - alpha B| <= 4 (n_A + 2) 2^-104 (|op(A)||X| +
 * |alpha B|), n_A the order of A; a zero diagonal entry gives Inf/NaN as
 * DTRSM does (no check).  Asynchronous on the current stream.
 * Errors: -1 side, -2 uplo, -3 transa, -4 diag, -5 m < 0, -6 n < 0,
 * -8 A planes NULL, -9 lda < max(1, order of A), -10 B planes NULL,
 * -11 ldb < max(1, m) (DTRSM's numbering). */
int mp_dd_Rtrsm(const char *side, const char *uplo, const char *transa, const char *diag,
                int64_t m, int64_t n, mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_mat B,
                int64_t ldb);

/* ------------------------------------------------------------------------ */
/* MPLAPACK: dd LU factorisation and solve                                   */
/* ------------------------------------------------------------------------ */

/* Rgetrf (MPLAPACK routine table, Sec. 6; DGETRF semantics): P A = L U with
 * partial pivoting of the m x n A; L (unit lower, not stored diagonal) and
 * U overwrite A.  ipiv (DEVICE int64[min(m, n)]) receives the one-based row
 * interchanged with row j at step j.  The pivot of a column is the first row
 * of largest dd magnitude.  *info (DEVICE int64, required) receives 0 or
 * j > 0 when U(j, j) is exactly zero (the factorisation completes, as in
 * LAPACK).  Recursive column splitting (LAPACK's dgetrf2): the updates are
 * dd Rtrsm and dd Rgemm products, the leaves panels of at most 32 columns,
 * each one cooperative launch with its rows spread over the SMs.  A
 * panel's grid-barrier waits are bounded (~2 s, which co-resident CTAs
 * never reach); a wait that gives up stops the panel and sets *info = -1.
 * Accuracy: the backward error of Gaussian elimination in dd arithmetic
 * (LAPACK test ratio ||P A - L U|| / (n ||A|| 2^-104) < 30).  Asynchronous
 * (a small stream-ordered allocation holds the panels' exchange buffers).
 * Errors: -1 m < 0, -2 n < 0, -3 A NULL, -4 lda < max(1, m), -5 ipiv NULL,
 * -6 info NULL. */
int mp_dd_Rgetrf(int64_t m, int64_t n, mp_dd_mat A, int64_t lda, int64_t *ipiv,
                 int64_t *info);

/* Rgetrs (DGETRS semantics): solve A X = B (trans 'N') or A^T X = B ('T';
 * 'C' is 'T') with the factors and ipiv (device) of mp_dd_Rgetrf on the
 * n x n A; B (n x nrhs) is overwritten by X.  Row interchanges, then unit
 * lower and upper dd Rtrsm (reverse order for 'T').  Asynchronous.
 * Errors: -1 trans, -2 n < 0, -3 nrhs < 0, -4 A NULL, -5 lda < max(1, n),
 * -6 ipiv NULL, -7 B NULL, -8 ldb < max(1, n). */
int mp_dd_Rgetrs(const char *trans, int64_t n, int64_t nrhs, mp_dd_cmat A, int64_t lda,
                 const int64_t *ipiv, mp_dd_mat B, int64_t ldb);

/* ------------------------------------------------------------------------ */
/* MPLAPACK: dd Cholesky factorisation and solve                             */
/* ------------------------------------------------------------------------ */

/* Rpotrf (MPLAPACK routine table, Sec. 6; Rpotrf benchmark, Sec. 10.5;
 * DPOTRF semantics): A = U^T U (uplo 'U', U in the upper triangle) or
 * A = L L^T ('L'), A n x n symmetric positive definite, the other triangle
 * not referenced.  Blocked right-looking in blocks of 64: unblocked dd
 * Cholesky of each diagonal block, dd triangular solve for the panel, dd
 * Rsyrk trailing update.  *info (DEVICE int64, required) receives 0 or
 * j > 0 when the leading minor of order j is not positive definite; the
 * factorisation stops there (later blocks are left as they were).
 * Asynchronous.  Errors: -1 uplo, -2 n < 0, -3 A NULL, -4 lda < max(1,n),
 * -5 info NULL. */
int mp_dd_Rpotrf(const char *uplo, int64_t n, mp_dd_mat A, int64_t lda, int64_t *info);

/* Rpotrf with the updates on the tensor cores.  Outer steps of 256 columns
 * factor the diagonal block as mp_dd_Rpotrf does, solve the panel U(J, J+1:)
 * by 64-row blocks (each first subtracting the blocks above it, a
 * residue-form Rgemm, see mp_dd_Rgemm_crt) and update the trailing matrix
 * with one residue-form Rsyrk of depth 256 (see mp_dd_Rsyrk_crt); updates
 * of fewer than 512 columns run on the FP64 pipe.  Same arguments,
 * semantics and info as mp_dd_Rpotrf; after a failing pivot the later
 * updates leave A as it is.  workspace: device memory of at least
 * mp_dd_Rpotrf_crt_workspace(n) bytes (0 for n < 768: then the call
 * factors like mp_dd_Rpotrf).  Errors: as mp_dd_Rpotrf, 2003 workspace NULL
 * or too small. */
size_t mp_dd_Rpotrf_crt_workspace(int64_t n);
int mp_dd_Rpotrf_crt(const char *uplo, int64_t n, mp_dd_mat A, int64_t lda, int64_t *info,
                     void *workspace, size_t workspace_bytes);

/* Rpotrs (DPOTRS semantics): solve A X = B with the factor from
 * mp_dd_Rpotrf (same uplo); B (n x nrhs, ldb) is overwritten by X.  Blocked
 * forward (U^T) and backward (U) substitution with dd Rgemm updates.
 * factor_info (device, may be NULL): when it holds a non-zero value the
 * solve leaves B unchanged.  Asynchronous.  Errors: -1 uplo, -2 n < 0,
 * -3 nrhs < 0, -4 A NULL, -5 lda, -6 B NULL, -7 ldb < max(1, n). */
int mp_dd_Rpotrs(const char *uplo, int64_t n, int64_t nrhs, mp_dd_cmat A, int64_t lda,
                 mp_dd_mat B, int64_t ldb, const int64_t *factor_info);

/* Batched building blocks of the two routines (no counterpart in the
 * manual), used to advance many independent factorisations in one launch.
 * Descriptor arrays are DEVICE memory. */

/* Unblocked dd Cholesky of one diagonal block (n <= 64; a larger n is
 * taken as 64) whose top-left element is a_hi/a_lo; lower selects the 'L'
 * storage.  offset is the block's first column in the whole matrix (for
 * info = offset + j + 1).  A launch runs each block on a cluster of up to 8
 * CTAs (fewer as count grows); the result does not depend on it. */
typedef struct {
    double *a_hi, *a_lo;
    int64_t lda, n, offset;
    int64_t *info;
    int32_t lower, reserved;
} mp_dd_potrf_diag_desc;

/* Solve U^T X = B (trans 1) or U X = B (trans 0) in place, U the n x n
 * (n <= 64; a larger n is taken as 64) upper factor block at u_hi/u_lo (lower_u: read it from 'L'
 * storage), B n x nrhs at b_hi/b_lo (lower_b: B is stored transposed, as
 * the panel of an 'L' factor is).  unit_diag != 0 takes U's diagonal as
 * one without reading it. */
typedef struct {
    const double *u_hi, *u_lo;
    int64_t ldu;
    double *b_hi, *b_lo;
    int64_t ldb;
    int64_t n, nrhs;
    const int64_t *info;
    int32_t trans, lower_u, lower_b, unit_diag;
} mp_dd_trsm_desc;

/* One launch: one CTA per diagonal block.  Errors: -1 count, -2 descs. */
int mp_dd_potrf_diag_batch(int64_t count, const mp_dd_potrf_diag_desc *descs);

/* One launch over count descriptors, 4 to 32 right-hand-side columns per
 * CTA (chosen from count and max_nrhs; the result does not depend on it);
 * max_nrhs is the largest nrhs in the batch.  Errors: -1, -2, -3. */
int mp_dd_trsm_batch(int64_t count, const mp_dd_trsm_desc *descs, int64_t max_nrhs);

/* ------------------------------------------------------------------------ */
/* Grouped Rgemm: many independent problems in one launch (no counterpart    */
/* in the manual, which batches nothing)                                     */
/* ------------------------------------------------------------------------ */

/* One problem C := alpha op(A) op(B) + beta C of a group; fields as the
 * mp_dd_Rgemm arguments (device pointers), transa/transb 0 = N, 1 = T, and
 * tile the output tile shape: -1 = the library's choice (least zero-padded
 * work weighted by per-shape speed), 0 = 32x32, 1 = 64x32, 2 = 32x64,
 * 3 = 16x16 (m x n).  The shape changes speed only: every entry is bitwise
 * equal to mp_dd_Rgemm's for the same problem. */
typedef struct {
    int64_t m, n, k;
    mp_dd alpha, beta;
    const double *a_hi, *a_lo;
    int64_t lda;
    const double *b_hi, *b_lo;
    int64_t ldb;
    double *c_hi, *c_lo;
    int64_t ldc;
    int32_t transa, transb;
    int32_t tile;
    int32_t uplo;             /* 0 = all of C; 1 / 2 = only the upper / lower
                                 triangle of a square C (Rsyrk-style update) */
    const int64_t *info;      /* optional device word: if non-zero when the
                                 kernel reaches this problem, C is left as is */
} mp_dd_gemm_desc;

/* Device workspace bytes a group of `count` host descriptors needs. */
size_t mp_dd_Rgemm_grouped_workspace(int64_t count, const mp_dd_gemm_desc *descs);

/* Check the host descriptors (DGEMM rules per problem; a bad one returns -2
 * and mp_dd_last_error names it), cut every problem into tiles of its shape,
 * order all tiles longest first (k x tile area), and copy descriptors and
 * tile list into `workspace` (device memory owned by the caller).  The
 * upload is asynchronous on the current stream (staged through pinned memory
 * the library owns), so the host descriptors may be reused at once and the
 * call does not wait for earlier work; a run must follow on the same stream.
 * The problems' matrices are not touched.  Errors: -1 count, -2 descriptor,
 * -3 workspace NULL, 2003 workspace too small. */
int mp_dd_Rgemm_grouped_prepare(int64_t count, const mp_dd_gemm_desc *descs, void *workspace,
                                size_t workspace_bytes);

/* Run a prepared group: resets the work counter and launches one persistent
 * kernel whose CTAs take tiles from the list until it is empty.  Only
 * enqueues work on the current stream (a memset and one kernel), so it can
 * be captured in a CUDA graph and replayed; the group's matrices may change
 * between runs, its descriptors may not.  Runs that share a workspace must
 * not overlap on the device. */
int mp_dd_Rgemm_grouped_run(void *workspace);

/* ------------------------------------------------------------------------ */
/* MPBLAS: quad-double Rgemm                                                 */
/* ------------------------------------------------------------------------ */

/* Rgemm in quad-double (the manual's qd_real MPBLAS, Sec. 5 and 7.3; DGEMM
 * semantics): C := alpha op(A) op(B) + beta C on four-plane qd matrices.
 * Each multiply-add forms the products of order 1, 2^-53 and 2^-106 of the
 * components exactly and adds them error-free into a four-level
 * accumulator; only the lowest level rounds.  Accuracy:
 * |C - C_exact| <= 4 k 2^-209 (|alpha||A||B| + |beta||C|) componentwise
 * (2^-209 is MPLAPACK's Rlamch epsilon for qd_real, Sec. 7.6).  beta = 0:
 * C is write-only; alpha = 0 or k = 0: A and B are not read; the BLAS
 * quick return applies.  Output entries are non-overlapping qd values.
 * Errors and their numbering as mp_dd_Rgemm (-7 / -9 / -12 when any plane
 * of A / B / C is NULL). */
int mp_qd_Rgemm(const char *transa, const char *transb, int64_t m, int64_t n, int64_t k,
                mp_qd alpha, mp_qd_cmat A, int64_t lda, mp_qd_cmat B, int64_t ldb, mp_qd beta,
                mp_qd_mat C, int64_t ldc);

/* ------------------------------------------------------------------------ */
/* Split-precision Rgemm on the tensor cores (no counterpart in the manual)  */
/* ------------------------------------------------------------------------ */

/* What the last split-precision call on a workspace did (no counterpart in
 * the manual): the certificate's outcome and a guaranteed error estimate. */
typedef struct mp_dd_split_info_s {
    int status;          /* 0, or 2001 when a device wait timed out (C undefined) */
    int form;            /* 1 digit slices, 2 residues; 0: no product was formed
                            (alpha = 0 or k = 0: C := beta C) */
    int width_bits;      /* bits W each operand entry was rounded to (8 S, or
                            112 / 120 / 128); 0: the plain FP64 kernel computed C */
    int count;           /* slices S (form 1) or moduli N (form 2); 0 with W = 0 */
    double max_err_est;  /* upper bound of max_ij |C - C_exact|_ij / bound_ij, the
                            bound of mp_dd_Rgemm; <= 1 whenever status is 0 */
    double dmin;         /* the certificate's smallest margin
                            min_ij (L_ij + |beta/alpha||c_ij|) 2^-(e_i+f_j), L_ij a
                            lower bound of (|A||B|)_ij (+inf: nothing constrains) */
} mp_dd_split_info;

/* Workspace bytes mp_dd_Rgemm_sliced needs for an m x n x k product with
 * `slices` digits per operand entry (0 = chosen per call, 14 or 15: sized
 * for 15 when k allows it). */
size_t mp_dd_Rgemm_sliced_workspace(int64_t m, int64_t n, int64_t k, int slices);

/* Rgemm with the same arguments and result contract as mp_dd_Rgemm
 * (arguments 1-13 numbered as there), computed by the Ozaki scheme on the
 * fp16 tensor cores instead of FP64 DFMA:
 *  - each row of op(A) and column of op(B) is scaled by a power of two so
 *    its entries are below 1/2 in magnitude; every dd entry is then rounded
 *    to a multiple of 2^-8S of that scale (error at most one unit) and cut
 *    into S signed base-256 digits in [-128, 128];
 *  - the digit products are exact integer GEMMs (fp16 inputs, fp32
 *    accumulation kept exact by draining every 1024 products, int32 sums),
 *    grouped by digit significance t + u = b for b < S;
 *  - the band sums are combined exactly in integer arithmetic, rounded once
 *    to dd, scaled back, and alpha/beta are applied in dd arithmetic.
 * Accuracy (unconditional): |C - C_exact| <= 4 k 2^-104 (|alpha||A||B| +
 * |beta||C|) componentwise, as mp_dd_Rgemm.  Per product the error of the
 * digits is at most C_S 2^(e_i + f_j - 8S) (C_S = 1 + (S-1)/(4 (1 - 2^-8)),
 * 2^(e_i - 1) > max_l |A_il|, 2^(f_j - 1) > max_l |B_lj|).  Before slicing,
 * the call certifies this on the device, entry by entry, against a
 * guaranteed lower bound of |A||B| (one bf16 tensor-core product of the
 * operands' magnitudes, rounded toward zero); `slices` = 0 lets it take
 * S = 14 or, if needed, 15 (the narrowest that certifies); a non-zero
 * `slices` is the only S tried.  When no S certifies the bound, the plain
 * FP64 kernel of mp_dd_Rgemm computes C instead, within the same call (no
 * host synchronisation); mp_dd_split_report tells which happened.
 * Limits: 2 <= slices <= 15; k * S <= 131071 (int32 band sums).
 * `workspace` is device memory of at least
 * mp_dd_Rgemm_sliced_workspace(m, n, k, slices) bytes owned by the caller;
 * it begins with a header (status word, certificate) that
 * mp_dd_workspace_status and mp_dd_split_report read after the call.
 * Calls sharing a workspace must not overlap on the device.  Asynchronous.
 * Errors: as mp_dd_Rgemm, plus -14 slices out of range, -15 workspace NULL,
 * 2003 workspace too small, 2002 k * slices too large. */
int mp_dd_Rgemm_sliced(const char *transa, const char *transb, int64_t m, int64_t n,
                       int64_t k, mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_cmat B,
                       int64_t ldb, mp_dd beta, mp_dd_mat C, int64_t ldc, int slices,
                       void *workspace, size_t workspace_bytes);

/* Allocation-free form of mp_dd_Rgemm_sliced (the manual has no
 * counterpart).  For callers that keep the MPBLAS Rgemm argument list (no
 * workspace argument) in a program where the library may not allocate
 * device memory: an application that hands all device memory to its own
 * pool at start-up, or a latency-critical loop that must never reach a
 * cudaMalloc.  The scratch memory is a fixed array of
 * MP_DD_NOALLOC_SCRATCH_BYTES compiled into the library; every device on
 * which the library's device code is loaded holds it until the process
 * exits.  Neither this call nor anything it calls allocates or frees memory.
 * Same arguments 1-14, result and errors as mp_dd_Rgemm_sliced; a problem
 * whose workspace (mp_dd_Rgemm_sliced_workspace) exceeds the array --
 * e.g. anything above m = n = k = 512 at the default 14 slices -- is
 * rejected with 2002 before any device work.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress, with that
 * device current) and caches it; make that first call before any stream
 * capture starts.  All calls share the one array, which keeps the last
 * call's contents: each call clears what must start at zero itself, and
 * calls that overlap on the GPU (different streams or unordered threads)
 * race on it and give wrong results.  The array begins with the same header
 * as a workspace: mp_dd_noalloc_report reads it.  The cached address is
 * looked up again on every call made outside stream capture, so a device
 * reset (which reloads the library's device code) is picked up. */
#define MP_DD_NOALLOC_SCRATCH_BYTES (32u << 20)
int mp_dd_Rgemm_sliced_noalloc(const char *transa, const char *transb, int64_t m, int64_t n,
                               int64_t k, mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_cmat B,
                               int64_t ldb, mp_dd beta, mp_dd_mat C, int64_t ldc, int slices);

/* mp_dd_split_report for the built-in scratch array of the current device:
 * the status word (0, or 2001 when a device wait of the last
 * mp_dd_Rgemm_sliced_noalloc call timed out) and its certificate.  Waits for
 * the calling thread's current stream.  Errors: -1 info NULL, 1000 + e. */
int mp_dd_noalloc_report(mp_dd_split_info *info);

/* Residue (CRT) form of the split-precision Rgemm (no counterpart in the
 * manual).  Same arguments 1-13, result contract and errors as
 * mp_dd_Rgemm_sliced.  Every entry of a row of op(A) / column of op(B) is
 * rounded to a multiple of 2^(e - W) of its power-of-two scale (|error| <=
 * one unit), and the exact integer product of the rounded operands is formed
 * through the Chinese remainder theorem: residues modulo N pairwise coprime
 * moduli <= 256 (the product of the moduli at least k 2^(2W)), one fp16
 * tensor-core GEMM per modulus with exact int32 accumulation, and an exact
 * multiword reconstruction rounded once to dd.  The only error is the
 * operand rounding, at most (1 + 2^-W) 2^(e_i + f_j - W) per product.  The
 * call certifies it on the device as mp_dd_Rgemm_sliced does and takes the
 * narrowest of W = 112, 120, 128 bits that meets the bound (N = 32, 36, 38
 * moduli at k = 8192), else computes C with the plain FP64 kernel; so the
 * mp_dd_Rgemm bound holds unconditionally.  Limits: k <= 131071.
 * workspace: device memory of at least mp_dd_Rgemm_crt_workspace(m, n, k)
 * bytes (sized for the widest W), header first (mp_dd_workspace_status,
 * mp_dd_split_report).  Asynchronous.  Errors: as mp_dd_Rgemm, -14
 * workspace NULL, 2003 workspace too small, 2002 k too large. */
size_t mp_dd_Rgemm_crt_workspace(int64_t m, int64_t n, int64_t k);
int mp_dd_Rgemm_crt(const char *transa, const char *transb, int64_t m, int64_t n, int64_t k,
                    mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_cmat B, int64_t ldb,
                    mp_dd beta, mp_dd_mat C, int64_t ldc, void *workspace,
                    size_t workspace_bytes);

/* Rsyrk in the residue (CRT) form (the manual's Rsyrk, Sec. 7.3, on the
 * tensor cores; DSYRK argument list and error numbering, -12 workspace NULL):
 *
 *     C := alpha A A^T + beta C   (trans N, A n x k), or
 *     C := alpha A^T A + beta C   (trans T, A k x n),
 *
 * on the uplo triangle of C only (the other is neither read nor written).
 * op(A) is rounded and reduced once and serves as both operands, and only
 * the tiles and entries of the triangle are formed: about half the work of
 * mp_dd_Rgemm_crt on (A, A^T).  Every entry of the triangle is bitwise equal
 * to mp_dd_Rgemm_crt(N, T) (trans N) or (T, N) (trans T) on A, A.  Accuracy
 * (certified per call, over the triangle only) and limits as
 * mp_dd_Rgemm_crt.  workspace: at least
 * mp_dd_Rsyrk_crt_workspace(n, k) bytes.  Asynchronous. */
size_t mp_dd_Rsyrk_crt_workspace(int64_t n, int64_t k);
int mp_dd_Rsyrk_crt(const char *uplo, const char *trans, int64_t n, int64_t k, mp_dd alpha,
                    mp_dd_cmat A, int64_t lda, mp_dd beta, mp_dd_mat C, int64_t ldc,
                    void *workspace, size_t workspace_bytes);

/* Workspace layout of mp_dd_Rgemm_crt (for inspection and testing):
 * offsets[0..4] byte offsets of the row maxima (uint64), column maxima,
 * residue planes of op(A) (fp16 [N][m_pad][k_pad]), of op(B)^T (fp16
 * [N][n_pad][k_pad]) and the products reduced mod p_i (uint8
 * [N][n_pad][m_pad]); offsets[5..7] m_pad, n_pad, k_pad; offsets[8..8+N)
 * the moduli; *moduli = N, the planes the workspace holds (the widest
 * width's count; a call fills the first mp_dd_split_info.count of them).
 * Returns 0. */
int mp_dd_crt_layout(int64_t m, int64_t n, int64_t k, size_t offsets[48], int *moduli);

/* Byte offsets of the intermediate arrays inside a sliced-Rgemm workspace
 * (for inspection and testing): offsets[0] row maxima of op(A) (uint64 bit
 * patterns of max |hi|, m_pad entries), [1] column maxima of op(B) (n_pad),
 * [2] digit planes of op(A) (fp16 [slices][m_pad][k_pad]), [3] digit planes
 * of op(B)^T (fp16 [slices][n_pad][k_pad]), [4] band sums (int32
 * [slices][n_pad][m_pad], column-major per band); offsets[5..7] hold m_pad,
 * n_pad, k_pad.  Returns 0. */
int mp_dd_sliced_layout(int64_t m, int64_t n, int64_t k, int slices, size_t offsets[8]);

/* Read the device status word of a workspace (waits for the calling
 * thread's current stream, then copies). */
int mp_dd_workspace_status(const void *workspace, int *status);

/* Fill *info from the header of `workspace` after a mp_dd_Rgemm_sliced,
 * mp_dd_Rgemm_crt or mp_dd_Rsyrk_crt call (waits for the calling thread's
 * current stream, then copies the header).  A call that returned before any
 * device work (argument error, BLAS quick return) leaves the header as it
 * was.  Errors: -1 workspace NULL, -2 info NULL, 1000 + e copy failure. */
int mp_dd_split_report(const void *workspace, mp_dd_split_info *info);

/* Byte offsets of the certificate's magnitude planes in a workspace (for
 * inspection and testing): offsets[0] op(A) (bf16 [m_pad][k_pad]: the
 * largest bf16 not above |hi| 2^-e_i), offsets[1] op(B)^T (bf16
 * [n_pad][k_pad]; equal to offsets[0] for the Rsyrk form).  form: 1 sliced
 * (slices as for mp_dd_Rgemm_sliced_workspace), 2 CRT Rgemm, 3 CRT Rsyrk
 * (m = n).  Returns 0, or -1 form, -2 .. -4 a negative size, -5 slices out
 * of range, -6 offsets NULL. */
int mp_dd_magnitude_layout(int form, int64_t m, int64_t n, int64_t k, int slices,
                           size_t offsets[2]);

/* Per-phase timing of split-precision calls (no counterpart in the manual).
 * With enable != 0, later mp_dd_Rgemm_sliced, mp_dd_Rgemm_crt and
 * mp_dd_Rsyrk_crt calls from this thread record CUDA events around their
 * three phases on the current stream: (0) scaling, certificate and slicing
 * (or residues), (1) the tensor-core products, (2) recombination (or CRT
 * reconstruction), epilogue and the plain fallback launch.  Enabling (again)
 * starts a new log of up to 4096 calls.  mp_dd_sliced_phase_ms waits for the
 * last timed call and writes its three milliseconds (2002 if no call was
 * timed); mp_dd_sliced_phase_log waits for the first max_calls logged calls,
 * writes their times to ms[3 c + phase] and the number of logged calls to
 * *calls (errors: -1 ms NULL with max_calls > 0, -2 max_calls < 0, -3 calls
 * NULL). */
int mp_dd_sliced_timing(int enable);
int mp_dd_sliced_phase_ms(float ms[3]);
int mp_dd_sliced_phase_log(float *ms, int max_calls, int *calls);

/* ------------------------------------------------------------------------ */
/* Elementwise dd arithmetic (the dd format's scalar operations, Sec. 5)      */
/* ------------------------------------------------------------------------ */

/* z_i := x_i op y_i for i < n on device arrays (hi, lo planes, contiguous),
 * with the scalar dd operations the kernels use:
 *   "add"  accurate dd addition (two TwoSums, relative error <= 3u^2+13u^3);
 *   "mul"  dd product (exact hi*hi by FMA plus the cross products);
 *   "div"  two-digit long division (first digit RN(x.hi / y.hi), second
 *          from the exact remainder), relative error below ~11 u^2;
 *   "divr" the same with the second digit taken by RN(1 / y.hi) (as the
 *          Cholesky and triangular-solve kernels divide), below ~20 u^2;
 *   "sqrt" sqrt(x) (y not read): RN(sqrt(x.hi)) plus one Newton step by
 *          rsqrt; 0 for x <= 0;
 *   "rcp"  1 / x (y not read), as the LU panels form their multipliers.
 * u = 2^-53.  div, divr and sqrt are exact when the exact result is a
 * binary64 number and the operands' lo parts are 0.  Asynchronous on the
 * current stream.  Errors: -1 unknown op, -2 n < 0, -3/-4/-5 x/y/z NULL
 * (y only for the binary ops). */
int mp_dd_elementwise(const char *op, int64_t n, mp_dd_cmat x, mp_dd_cmat y, mp_dd_mat z);

/* ------------------------------------------------------------------------ */
/* Measured roofline denominators (no counterpart in the manual)             */
/* ------------------------------------------------------------------------ */

/* Time a kernel of independent FP64 fused multiply-add chains filling every
 * SM and report the issue rate in FP64 instructions per second in *rate.
 * Synchronous (synchronises the current stream).  Returns 0 or an error. */
int mp_dd_peak_fp64(double *rate);

/* Time a kernel of independent INT8 warp-level tensor instructions
 * (mma.sync m16n8k32, s8 inputs, s32 accumulation; sm_103a offers no
 * tcgen05 INT8 form) filling every SM, and report the rate in integer
 * operations per second (2 per multiply-add) in *rate.  This is the ceiling
 * of an INT8-slice split-precision product on this GPU, against which the
 * fp16 tcgen05 path is compared.  Synchronous.  Returns 0 or an error. */
int mp_dd_peak_imma(double *rate);

/* Time the plain kernel's dd multiply-add (the same operation sequence, 4 x 4
 * accumulators per thread, renormalised every 4 steps) on operands that stay
 * in registers and change every step by integer operations only, filling
 * every SM, and report the rate in dd multiply-adds per second in *rate: the
 * ceiling of the plain kernel's instruction mix on this GPU's FP64 pipe
 * (twice it in dd-flop/s).  Synchronous.  Returns 0 or an error. */
int mp_dd_peak_ddmac(double *rate);

#ifdef __cplusplus
}
#endif

#endif /* MPDD_H */
