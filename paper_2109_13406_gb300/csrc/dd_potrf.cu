// dd Cholesky factorisation and solve (Rpotrf / Rpotrs, MPLAPACK routine
// table of the manual's Sec. 6; the Rpotrf benchmark of Sec. 10.5), built as
// the LAPACK blocked right-looking algorithm on three kernels, and the
// triangular solve Rtrsm (MPBLAS, Sec. 6) on the same two of them:
//
//  * diag:  unblocked Cholesky of one nb x nb diagonal block (nb <= 64), in
//           shared memory, one CTA per block;
//  * trsm:  triangular solve with one nb x nb factor block for up to 32
//           right-hand-side columns per CTA (forward with U^T, backward
//           with U), optionally scaling the right-hand sides by alpha and
//           taking the diagonal as unit;
//  * the trailing updates are the dd Rsyrk / Rgemm kernels.
//
// Storage follows LAPACK: uplo 'U' factors A = U^T U in the upper triangle,
// 'L' factors A = L L^T in the lower one.  Both are handled by one code path
// through an accessor: U(i, j) = A[i + j lda] for 'U' and A[j + i lda] (= L(j,
// i)) for 'L'; right-hand-side panels are accessed the same way.
//
// info (device int64, LAPACK convention): 0, or j > 0 when the leading minor
// of order j is not positive definite.  The first failing pivot is
// recorded; the launches that follow see info != 0 and leave their matrices
// untouched.
#include "common.cuh"
#include "dd_arith.cuh"
#include "kernels.cuh"

namespace mpdd {
namespace {

constexpr int NB = 64;        // largest diagonal block
constexpr int NT = 256;

__host__ __device__ __forceinline__ int64_t uidx(int lower, int64_t i, int64_t j, int64_t ld) {
    return lower ? (j + i * ld) : (i + j * ld);
}

struct DiagSmem {
    double h[NB][NB + 1], l[NB][NB + 1];   // U block, [row][col], upper part used
    int fail;
};

__device__ void potrf_diag_one(const mp_dd_potrf_diag_desc &d, DiagSmem &s) {
    const int nbe = (int)d.n;
    const int tid = threadIdx.x;
    if (d.info != nullptr && *d.info != 0) return;   // an earlier block failed
    for (int e = tid; e < nbe * nbe; e += NT) {
        int r = e % nbe, c = e / nbe;
        if (r <= c) {
            int64_t o = uidx(d.lower, r, c, d.lda);
            s.h[r][c] = d.a_hi[o];
            s.l[r][c] = d.a_lo[o];
        }
    }
    if (tid == 0) s.fail = 0;
    __syncthreads();
    for (int j = 0; j < nbe; ++j) {
        if (tid == 0) {
            dd p{s.h[j][j], s.l[j][j]};
            if (!(p.hi > 0.0)) {
                s.fail = 1;
                if (d.info != nullptr)
                    atomicCAS(reinterpret_cast<unsigned long long *>(d.info), 0ull,
                              (unsigned long long)(d.offset + j + 1));
            } else {
                dd u = sqrt_dd(p);
                s.h[j][j] = u.hi;
                s.l[j][j] = u.lo;
            }
        }
        __syncthreads();
        if (s.fail) break;
        const dd ujj{s.h[j][j], s.l[j][j]};
        for (int c = j + 1 + tid; c < nbe; c += NT) {
            dd v = div(dd{s.h[j][c], s.l[j][c]}, ujj);
            s.h[j][c] = v.hi;
            s.l[j][c] = v.lo;
        }
        __syncthreads();
        // trailing update of the block: U(r, c) -= U(j, r) U(j, c), j < r <= c
        const int w = nbe - j - 1;
        for (int e = tid; e < w * w; e += NT) {
            int r = j + 1 + e % w, c = j + 1 + e / w;
            if (r <= c) {
                dd a{s.h[r][c], s.l[r][c]};
                mac(a, dd{-s.h[j][r], -s.l[j][r]}, dd{s.h[j][c], s.l[j][c]});
                s.h[r][c] = a.hi;
                s.l[r][c] = a.lo;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < nbe * nbe; e += NT) {
        int r = e % nbe, c = e / nbe;
        if (r <= c) {
            int64_t o = uidx(d.lower, r, c, d.lda);
            d.a_hi[o] = s.h[r][c];
            d.a_lo[o] = s.l[r][c];
        }
    }
}

__global__ void __launch_bounds__(NT) potrf_diag_batch_kernel(const mp_dd_potrf_diag_desc *ds) {
    extern __shared__ double smem_d[];
    potrf_diag_one(ds[blockIdx.x], *reinterpret_cast<DiagSmem *>(smem_d));
}

__global__ void __launch_bounds__(NT) potrf_diag_single_kernel(const mp_dd_potrf_diag_desc d) {
    extern __shared__ double smem_d[];
    potrf_diag_one(d, *reinterpret_cast<DiagSmem *>(smem_d));
}

// ------------------------------------------------------------------ trsm

constexpr int TC = 32;   // right-hand-side columns per CTA

struct TrsmSmem {
    double uh[NB][NB + 1], ul[NB][NB + 1];
    double bh[NB][TC + 1], bl[NB][TC + 1];
};

// B := alpha B before the solve when scale != 0.
struct TrsmScale {
    dd alpha;
    int scale;
};

// Solve U^T X = B (trans = 1) or U X = B (trans = 0) for the columns
// [c0, c0 + TC) of B, in place.  U is the n x n upper factor block; with
// d.unit_diag its diagonal is taken as one and never read.
__device__ void trsm_one(const mp_dd_trsm_desc &d, int64_t c0, TrsmSmem &s, TrsmScale sc) {
    const int n = (int)d.n;
    const int tid = threadIdx.x;
    if (d.info != nullptr && *d.info != 0) return;
    const int64_t ncol = d.nrhs - c0 < TC ? d.nrhs - c0 : TC;
    if (ncol <= 0) return;
    const int unit = d.unit_diag != 0;
    for (int e = tid; e < n * n; e += NT) {
        int r = e % n, c = e / n;
        if (r < c || (r == c && !unit)) {
            int64_t o = uidx(d.lower_u, r, c, d.ldu);
            s.uh[r][c] = d.u_hi[o];
            s.ul[r][c] = d.u_lo[o];
        }
    }
    for (int e = tid; e < n * TC; e += NT) {
        int r = e % n, c = e / n;
        if (c < ncol) {
            int64_t o = uidx(d.lower_b, r, c0 + c, d.ldb);
            dd b{d.b_hi[o], d.b_lo[o]};
            if (sc.scale) b = mul(sc.alpha, b);
            s.bh[r][c] = b.hi;
            s.bl[r][c] = b.lo;
        }
    }
    __syncthreads();
    for (int step = 0; step < n; ++step) {
        const int i = d.trans ? step : n - 1 - step;
        if (tid < ncol && !unit) {
            dd x = div(dd{s.bh[i][tid], s.bl[i][tid]}, dd{s.uh[i][i], s.ul[i][i]});
            s.bh[i][tid] = x.hi;
            s.bl[i][tid] = x.lo;
        }
        __syncthreads();
        // eliminate x_i from the remaining rows: U^T: rows r > i use U(i, r);
        // U: rows r < i use U(r, i)
        const int lo_r = d.trans ? i + 1 : 0, hi_r = d.trans ? n : i;
        const int rows = hi_r - lo_r;
        for (int e = tid; e < rows * (int)ncol; e += NT) {
            int r = lo_r + e % rows, c = e / rows;
            dd u = d.trans ? dd{s.uh[i][r], s.ul[i][r]} : dd{s.uh[r][i], s.ul[r][i]};
            dd b{s.bh[r][c], s.bl[r][c]};
            mac(b, dd{-u.hi, -u.lo}, dd{s.bh[i][c], s.bl[i][c]});
            s.bh[r][c] = b.hi;
            s.bl[r][c] = b.lo;
        }
        __syncthreads();
    }
    for (int e = tid; e < n * TC; e += NT) {
        int r = e % n, c = e / n;
        if (c < ncol) {
            int64_t o = uidx(d.lower_b, r, c0 + c, d.ldb);
            d.b_hi[o] = s.bh[r][c];
            d.b_lo[o] = s.bl[r][c];
        }
    }
}

__global__ void __launch_bounds__(NT) trsm_batch_kernel(const mp_dd_trsm_desc *ds) {
    extern __shared__ double smem_t[];
    trsm_one(ds[blockIdx.x], (int64_t)blockIdx.y * TC, *reinterpret_cast<TrsmSmem *>(smem_t),
             TrsmScale{dd{1.0, 0.0}, 0});
}

__global__ void __launch_bounds__(NT) trsm_single_kernel(const mp_dd_trsm_desc d,
                                                         TrsmScale sc) {
    extern __shared__ double smem_t[];
    trsm_one(d, (int64_t)blockIdx.y * TC, *reinterpret_cast<TrsmSmem *>(smem_t), sc);
}

constexpr TrsmScale kNoScale{dd{1.0, 0.0}, 0};

bool g_attr_done = false;

int set_attrs() {
    if (g_attr_done) return 0;
    cudaError_t e = cudaFuncSetAttribute(potrf_diag_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(DiagSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(potrf_diag_single_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(DiagSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(trsm_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(TrsmSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(trsm_single_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(TrsmSmem));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(potrf kernels)");
    g_attr_done = true;
    return 0;
}

}  // namespace

int launch_potrf_diag_batch(int64_t count, const mp_dd_potrf_diag_desc *ds, cudaStream_t st) {
    if (count == 0) return 0;
    int rc = set_attrs();
    if (rc) return rc;
    if (count > 0x7fffffffLL) return fail(MP_DD_ERR_TOO_LARGE, "too many blocks");
    potrf_diag_batch_kernel<<<(unsigned)count, NT, sizeof(DiagSmem), st>>>(ds);
    return check_launch("potrf_diag_batch_kernel");
}

int launch_trsm_batch(int64_t count, const mp_dd_trsm_desc *ds, int64_t max_rhs,
                      cudaStream_t st) {
    if (count == 0 || max_rhs == 0) return 0;
    int rc = set_attrs();
    if (rc) return rc;
    dim3 grid((unsigned)count, (unsigned)ceil_div(max_rhs, TC));
    if (grid.y > 65535) return fail(MP_DD_ERR_TOO_LARGE, "too many right-hand sides");
    trsm_batch_kernel<<<grid, NT, sizeof(TrsmSmem), st>>>(ds);
    return check_launch("trsm_batch_kernel");
}

// Blocked right-looking Cholesky of one matrix (LAPACK dpotrf order).
int run_potrf(int lower, int64_t n, double *ah, double *al, int64_t lda, int64_t *info,
              cudaStream_t st) {
    int rc = set_attrs();
    if (rc) return rc;
    if (info != nullptr) {
        cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int64_t), st);
        if (e != cudaSuccess) return cuda_fail(e, "info reset");
    }
    for (int64_t j = 0; j < n; j += NB) {
        const int64_t nb = n - j < NB ? n - j : NB;
        mp_dd_potrf_diag_desc dg{};
        int64_t o = uidx(lower, j, j, lda);
        dg.a_hi = ah + o; dg.a_lo = al + o; dg.lda = lda; dg.n = nb; dg.offset = j;
        dg.info = info; dg.lower = lower;
        potrf_diag_single_kernel<<<1, NT, sizeof(DiagSmem), st>>>(dg);
        if ((rc = check_launch("potrf_diag_single_kernel"))) return rc;
        const int64_t rest = n - j - nb;
        if (rest <= 0) break;
        // panel: U(J, J+1:) := U_JJ^-T A(J, J+1:)
        mp_dd_trsm_desc tr{};
        tr.u_hi = ah + o; tr.u_lo = al + o; tr.ldu = lda;
        int64_t ob = uidx(lower, j, j + nb, lda);
        tr.b_hi = ah + ob; tr.b_lo = al + ob; tr.ldb = lda;
        tr.n = nb; tr.nrhs = rest; tr.trans = 1; tr.lower_u = lower; tr.lower_b = lower;
        tr.info = info;
        dim3 grid(1, (unsigned)ceil_div(rest, TC));
        trsm_single_kernel<<<grid, NT, sizeof(TrsmSmem), st>>>(tr, kNoScale);
        if ((rc = check_launch("trsm_single_kernel"))) return rc;
        // trailing: A(J+1:, J+1:) -= U(J, J+1:)^T U(J, J+1:) on the stored triangle
        GemmArgs p{};
        p.m = rest; p.n = rest; p.k = nb;
        p.alpha = mp_dd{-1.0, 0.0}; p.beta = mp_dd{1.0, 0.0};
        p.ah = ah + ob; p.al = al + ob; p.lda = lda;
        p.bh = ah + ob; p.bl = al + ob; p.ldb = lda;
        int64_t oc = uidx(lower, j + nb, j + nb, lda);
        p.ch = ah + oc; p.cl = al + oc; p.ldc = lda;
        // upper: C -= P^T P with P = U(J, J+1:) (nb x rest, column-major): (T, N)
        // lower: C -= P P^T with P = L(J+1:, J) (rest x nb): (N, T)
        p.ta = lower ? 0 : 1; p.tb = lower ? 1 : 0; p.tri = lower ? 2 : 1;
        p.alpha_zero = 0; p.alpha_one = 0; p.beta_zero = 0;
        p.info = info;
        if ((rc = launch_gemm_plain(p, st))) return rc;
    }
    return 0;
}

// Solve A X = B with the factor of run_potrf (blocked forward and backward
// substitution; updates through the plain dd Rgemm kernel).
int run_potrs(int lower, int64_t n, int64_t nrhs, const double *ah, const double *al,
              int64_t lda, double *bh, double *bl, int64_t ldb, const int64_t *info,
              cudaStream_t st) {
    int rc = set_attrs();
    if (rc) return rc;
    const int64_t nblk = ceil_div(n, NB);
    auto solve_block = [&](int64_t j, int trans) -> int {
        const int64_t nb = n - j < NB ? n - j : NB;
        mp_dd_trsm_desc tr{};
        int64_t o = uidx(lower, j, j, lda);
        tr.u_hi = ah + o; tr.u_lo = al + o; tr.ldu = lda;
        tr.b_hi = bh + j; tr.b_lo = bl + j; tr.ldb = ldb;
        // B is a plain n x nrhs matrix (column-major whatever uplo is); U is
        // read through the factor accessor
        tr.n = nb; tr.nrhs = nrhs; tr.trans = trans; tr.lower_u = lower; tr.lower_b = 0;
        tr.info = info;
        dim3 grid(1, (unsigned)ceil_div(nrhs, TC));
        trsm_single_kernel<<<grid, NT, sizeof(TrsmSmem), st>>>(tr, kNoScale);
        return check_launch("trsm_single_kernel");
    };
    auto update = [&](int64_t j, int forward) -> int {
        const int64_t nb = n - j < NB ? n - j : NB;
        GemmArgs p{};
        p.alpha = mp_dd{-1.0, 0.0}; p.beta = mp_dd{1.0, 0.0};
        p.alpha_zero = 0; p.alpha_one = 0; p.beta_zero = 0; p.tri = 0; p.info = info;
        if (forward) {
            // B(J+1:) -= U(J, J+1:)^T B(J)
            const int64_t rest = n - j - nb;
            if (rest <= 0) return 0;
            int64_t ou = uidx(lower, j, j + nb, lda);
            p.m = rest; p.n = nrhs; p.k = nb;
            p.ah = ah + ou; p.al = al + ou; p.lda = lda;
            p.ta = lower ? 0 : 1;   // upper: U(J, J+1:) is nb x rest -> transpose
            p.bh = bh + j; p.bl = bl + j; p.ldb = ldb; p.tb = 0;
            p.ch = bh + j + nb; p.cl = bl + j + nb; p.ldc = ldb;
        } else {
            // B(0:J) -= U(0:J, J) B(J)
            if (j == 0) return 0;
            int64_t ou = uidx(lower, 0, j, lda);
            p.m = j; p.n = nrhs; p.k = nb;
            p.ah = ah + ou; p.al = al + ou; p.lda = lda;
            p.ta = lower ? 1 : 0;   // upper: U(0:J, J) is j x nb as stored
            p.bh = bh + j; p.bl = bl + j; p.ldb = ldb; p.tb = 0;
            p.ch = bh; p.cl = bl; p.ldc = ldb;
        }
        return launch_gemm_plain(p, st);
    };
    for (int64_t b = 0; b < nblk; ++b) {
        if ((rc = solve_block(b * NB, 1))) return rc;
        if ((rc = update(b * NB, 1))) return rc;
    }
    for (int64_t b = nblk - 1; b >= 0; --b) {
        if ((rc = solve_block(b * NB, 0))) return rc;
        if ((rc = update(b * NB, 0))) return rc;
    }
    return 0;
}

// ------------------------------------------------------------------ Rtrsm
//
// Every DTRSM variant is one triangular system T Y = B' with several
// right-hand sides: for side 'L' T = op(A) and B' = B; for side 'R'
// X op(A) = B is op(A)^T X^T = B^T, so T = op(A)^T and B' = B^T (read
// through the transposed accessor).  T is then either U^T (lower: forward
// substitution) or U (upper: backward substitution) for the upper-stored
// view U(r, c) = A[uidx(lower_a, r, c)] of A's triangle.  The solve splits
// T recursively into halves (at multiples of 64): solve the first half,
// update the second half's right-hand sides with one dd Rgemm of the whole
// off-diagonal block, solve the second half.  The leaves are 64 x 64
// diagonal blocks in shared memory.  alpha is applied where each row block
// of B' is first touched: by the leaf kernel (the first block) or as the
// beta of its first Rgemm update.

namespace {

struct TrsmPlan {
    int lower_a;   // A's triangle is 'L' (read through the transposed accessor)
    int forward;   // T is lower: forward substitution
    int right;     // B' = B^T
    int unit;
    const double *ah, *al;
    int64_t lda;
    double *bh, *bl;
    int64_t ldb;
    int64_t nrhs;  // columns of B'
    mp_dd alpha;
    int alpha_one;
    cudaStream_t st;
};

int trsm_leaf(const TrsmPlan &P, int64_t j0, int64_t nt, bool first) {
    mp_dd_trsm_desc tr{};
    const int64_t o = uidx(P.lower_a, j0, j0, P.lda);
    tr.u_hi = P.ah + o; tr.u_lo = P.al + o; tr.ldu = P.lda;
    const int64_t ob = uidx(P.right, j0, 0, P.ldb);
    tr.b_hi = P.bh + ob; tr.b_lo = P.bl + ob; tr.ldb = P.ldb;
    tr.n = nt; tr.nrhs = P.nrhs; tr.trans = P.forward; tr.lower_u = P.lower_a;
    tr.lower_b = P.right; tr.unit_diag = P.unit; tr.info = nullptr;
    const TrsmScale sc{dd{P.alpha.hi, P.alpha.lo}, first && !P.alpha_one};
    const int64_t gy = ceil_div(P.nrhs, TC);
    if (gy > 65535) return fail(MP_DD_ERR_TOO_LARGE, "Rtrsm: too many right-hand sides");
    trsm_single_kernel<<<dim3(1, (unsigned)gy), NT, sizeof(TrsmSmem), P.st>>>(tr, sc);
    return check_launch("trsm_single_kernel");
}

// B'(rows r0 .. r0+mr) -= T(rows, cols c0 .. c0+kc) B'(cols), with beta = alpha
// when these rows are touched for the first time.
int trsm_update(const TrsmPlan &P, int64_t r0, int64_t mr, int64_t c0, int64_t kc,
                bool first) {
    // T(r, c) off the diagonal is A[uidx(tl, r, c)]: as stored (tl = 0) or
    // transposed (tl = 1); the block starts at uidx(tl, r0, c0)
    const int tl = P.lower_a ^ P.forward;
    const int64_t ot = uidx(tl, r0, c0, P.lda);
    GemmArgs p{};
    p.alpha = mp_dd{-1.0, 0.0};
    p.beta = first ? P.alpha : mp_dd{1.0, 0.0};
    p.alpha_zero = 0; p.alpha_one = 0; p.beta_zero = 0; p.tri = 0; p.info = nullptr;
    if (!P.right) {
        // B(r0:, :) -= T_sub B(c0:, :)
        p.m = mr; p.n = P.nrhs; p.k = kc;
        p.ah = P.ah + ot; p.al = P.al + ot; p.lda = P.lda; p.ta = tl;
        p.bh = P.bh + c0; p.bl = P.bl + c0; p.ldb = P.ldb; p.tb = 0;
        p.ch = P.bh + r0; p.cl = P.bl + r0; p.ldc = P.ldb;
    } else {
        // B(:, r0:) -= B(:, c0:) T_sub^T
        p.m = P.nrhs; p.n = mr; p.k = kc;
        p.ah = P.bh + c0 * P.ldb; p.al = P.bl + c0 * P.ldb; p.lda = P.ldb; p.ta = 0;
        p.bh = P.ah + ot; p.bl = P.al + ot; p.ldb = P.lda; p.tb = !tl;
        p.ch = P.bh + r0 * P.ldb; p.cl = P.bl + r0 * P.ldb; p.ldc = P.ldb;
    }
    return launch_gemm_plain(p, P.st);
}

int trsm_rec(const TrsmPlan &P, int64_t j0, int64_t nt, bool first) {
    if (nt <= NB) return trsm_leaf(P, j0, nt, first);
    const int64_t h = ceil_div(nt / 2, (int64_t)NB) * NB;   // 64 <= h < nt
    int rc;
    if (P.forward) {
        if ((rc = trsm_rec(P, j0, h, first))) return rc;
        if ((rc = trsm_update(P, j0 + h, nt - h, j0, h, first))) return rc;
        return trsm_rec(P, j0 + h, nt - h, false);
    }
    if ((rc = trsm_rec(P, j0 + h, nt - h, first))) return rc;
    if ((rc = trsm_update(P, j0, h, j0 + h, nt - h, first))) return rc;
    return trsm_rec(P, j0, h, false);
}

}  // namespace

int run_trsm(int right, int lower, int trans, int unit, int64_t m, int64_t n, mp_dd alpha,
             const double *ah, const double *al, int64_t lda, double *bh, double *bl,
             int64_t ldb, cudaStream_t st) {
    int rc = set_attrs();
    if (rc) return rc;
    TrsmPlan P{};
    P.lower_a = lower;
    P.forward = lower ^ trans ^ right;
    P.right = right;
    P.unit = unit;
    P.ah = ah; P.al = al; P.lda = lda;
    P.bh = bh; P.bl = bl; P.ldb = ldb;
    P.nrhs = right ? m : n;
    P.alpha = alpha;
    P.alpha_one = alpha.hi == 1.0 && alpha.lo == 0.0;
    P.st = st;
    return trsm_rec(P, 0, right ? n : m, true);
}

}  // namespace mpdd
