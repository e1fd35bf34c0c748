/*
 * Oracle for the double-double (dd) BLAS/LAPACK hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it, and this file
 * shares no code, header or constant with the CUDA sources.
 *
 * Three tiers, each written from the manual's description of the method
 * (MPLAPACK 2.0.1 user manual, arXiv 2109.13406; sections by number and title):
 *
 *   1. Scalar dd arithmetic (Sec. 5, "Supported Floating point formats"):
 *      a dd number is the unevaluated sum hi + lo of two binary64 numbers;
 *      addition and multiplication are built from Knuth's TwoSum and
 *      Dekker's exact product (here the product error is obtained with one
 *      fused multiply-add).  The manual warns that dd code must be compiled
 *      without value-changing floating-point optimisation (Sec. 3, the
 *      Intel compiler note): this file is compiled with -ffp-contract=off and
 *      without -ffast-math, and every fused multiply-add is an explicit fma().
 *
 *   2. Scalar dd Rgemm / Rsyrk / Rpotrf / Rpotrs (Sec. 6 routine tables and the
 *      Rgemm prototype/argument list of Sec. 7.3, which mirrors DGEMM):
 *      a plain triple loop in a fixed summation order with the accurate dd
 *      add and the full dd product (including the lo*lo term).
 *
 *   3. Exact tier: the mathematical definition C = alpha*op(A)*op(B) + beta*C,
 *      with every dd input taken as the exact rational hi + lo, evaluated in
 *      an exact fixed-point superaccumulator and rounded once to the nearest
 *      dd (hi = RN(x), lo = RN(x - hi)).  Exact as long as no partial product
 *      of three binary64 numbers underflows (|product| >= 2^-960 or zero).
 *
 * Column-major storage with a leading dimension, element (i, j) of a matrix
 * at index i + j*ld (Sec. 7.3: MPBLAS always uses one-dimensional column-major
 * arrays).  A dd matrix is two such arrays (hi plane, lo plane) sharing ld.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Tier 1: scalar dd arithmetic                                               */
/* ------------------------------------------------------------------------- */

typedef struct {
    double hi, lo;
} odd;

/* Knuth TwoSum: s + e == a + b exactly, s = fl(a + b). */
static void two_sum(double a, double b, double *s, double *e) {
    double sum = a + b;
    double bv = sum - a;
    double av = sum - bv;
    *s = sum;
    *e = (a - av) + (b - bv);
}

/* Dekker FastTwoSum, valid when |a| >= |b| (or a == 0). */
static void fast_two_sum(double a, double b, double *s, double *e) {
    double sum = a + b;
    *s = sum;
    *e = b - (sum - a);
}

/* Exact product: p + e == a * b, p = fl(a * b); the error by one FMA. */
static void two_prod(double a, double b, double *p, double *e) {
    double prod = a * b;
    *p = prod;
    *e = fma(a, b, -prod);
}

/* Accurate dd addition: both component pairs are added error-free, then the
 * result is renormalised twice. */
static odd dd_add(odd a, odd b) {
    double s1, s2, t1, t2;
    two_sum(a.hi, b.hi, &s1, &s2);
    two_sum(a.lo, b.lo, &t1, &t2);
    s2 += t1;
    fast_two_sum(s1, s2, &s1, &s2);
    s2 += t2;
    fast_two_sum(s1, s2, &s1, &s2);
    odd r = {s1, s2};
    return r;
}

static odd dd_neg(odd a) {
    odd r = {-a.hi, -a.lo};
    return r;
}

static odd dd_sub(odd a, odd b) { return dd_add(a, dd_neg(b)); }

/* Full dd product: exact hi*hi product plus all three cross terms. */
static odd dd_mul(odd a, odd b) {
    double p, e;
    two_prod(a.hi, b.hi, &p, &e);
    e += a.hi * b.lo + a.lo * b.hi + a.lo * b.lo;
    fast_two_sum(p, e, &p, &e);
    odd r = {p, e};
    return r;
}

/* dd division by long division with three binary64 quotient digits. */
static odd dd_div(odd a, odd b) {
    double q1 = a.hi / b.hi;
    odd r = dd_sub(a, dd_mul((odd){q1, 0.0}, b));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul((odd){q2, 0.0}, b));
    double q3 = r.hi / b.hi;
    double s, e;
    fast_two_sum(q1, q2, &s, &e);
    odd q = {s, e};
    return dd_add(q, (odd){q3, 0.0});
}

/* dd square root: one Newton correction of the binary64 root,
 * x + (a - x^2) / (2x), with the residual evaluated in dd. */
static odd dd_sqrt(odd a) {
    if (a.hi <= 0.0) {
        odd z = {0.0, 0.0};
        return z;
    }
    double x = sqrt(a.hi);
    odd xx = dd_mul((odd){x, 0.0}, (odd){x, 0.0});
    odd res = dd_sub(a, xx);
    double corr = res.hi / (2.0 * x);
    double s, e;
    fast_two_sum(x, corr, &s, &e);
    odd r = {s, e};
    return r;
}

/* Vectorised wrappers so the pins can exercise the scalar layer directly. */
void oracle_two_sum(int64_t n, const double *a, const double *b, double *s, double *e) {
    for (int64_t i = 0; i < n; ++i) two_sum(a[i], b[i], &s[i], &e[i]);
}
void oracle_two_prod(int64_t n, const double *a, const double *b, double *p, double *e) {
    for (int64_t i = 0; i < n; ++i) two_prod(a[i], b[i], &p[i], &e[i]);
}
void oracle_dd_add(int64_t n, const double *ah, const double *al, const double *bh,
                   const double *bl, double *rh, double *rl) {
    for (int64_t i = 0; i < n; ++i) {
        odd r = dd_add((odd){ah[i], al[i]}, (odd){bh[i], bl[i]});
        rh[i] = r.hi;
        rl[i] = r.lo;
    }
}
void oracle_dd_mul(int64_t n, const double *ah, const double *al, const double *bh,
                   const double *bl, double *rh, double *rl) {
    for (int64_t i = 0; i < n; ++i) {
        odd r = dd_mul((odd){ah[i], al[i]}, (odd){bh[i], bl[i]});
        rh[i] = r.hi;
        rl[i] = r.lo;
    }
}
void oracle_dd_div(int64_t n, const double *ah, const double *al, const double *bh,
                   const double *bl, double *rh, double *rl) {
    for (int64_t i = 0; i < n; ++i) {
        odd r = dd_div((odd){ah[i], al[i]}, (odd){bh[i], bl[i]});
        rh[i] = r.hi;
        rl[i] = r.lo;
    }
}
void oracle_dd_sqrt(int64_t n, const double *ah, const double *al, double *rh, double *rl) {
    for (int64_t i = 0; i < n; ++i) {
        odd r = dd_sqrt((odd){ah[i], al[i]});
        rh[i] = r.hi;
        rl[i] = r.lo;
    }
}

/* ------------------------------------------------------------------------- */
/* Tier 2: scalar dd Rgemm / Rsyrk / Rpotrf / Rpotrs                          */
/* ------------------------------------------------------------------------- */

static int is_trans(char c) { return c == 'T' || c == 't' || c == 'C' || c == 'c'; }

/* Element (r, c) of op(X) where X is column-major with leading dimension ld. */
static odd op_elem(const double *xh, const double *xl, int64_t ld, int trans, int64_t r,
                   int64_t c) {
    int64_t idx = trans ? (c + r * ld) : (r + c * ld);
    odd v = {xh[idx], xl[idx]};
    return v;
}

/* One output entry of alpha*op(A)*op(B) + beta*C_in with BLAS semantics:
 * beta == 0 means C_in is not read; alpha == 0 means no products are formed. */
static odd gemm_entry(int ta, int tb, int64_t i, int64_t j, int64_t k, odd alpha,
                      const double *ah, const double *al, int64_t lda, const double *bh,
                      const double *bl, int64_t ldb, odd beta, odd cin) {
    odd acc = {0.0, 0.0};
    int alpha_zero = (alpha.hi == 0.0 && alpha.lo == 0.0);
    if (!alpha_zero) {
        for (int64_t l = 0; l < k; ++l) {
            odd a = op_elem(ah, al, lda, ta, i, l);
            odd b = op_elem(bh, bl, ldb, tb, l, j);
            acc = dd_add(acc, dd_mul(a, b));
        }
        acc = dd_mul(alpha, acc);
    }
    if (beta.hi == 0.0 && beta.lo == 0.0) return acc;
    return dd_add(acc, dd_mul(beta, cin));
}

/* Rgemm: C := alpha*op(A)*op(B) + beta*C (argument list of DGEMM). */
void oracle_dd_gemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha_hi,
                    double alpha_lo, const double *ah, const double *al, int64_t lda,
                    const double *bh, const double *bl, int64_t ldb, double beta_hi,
                    double beta_lo, double *ch, double *cl, int64_t ldc) {
    odd alpha = {alpha_hi, alpha_lo}, beta = {beta_hi, beta_lo};
    int ta = is_trans(transa), tb = is_trans(transb);
    int alpha_zero = (alpha.hi == 0.0 && alpha.lo == 0.0);
    if (m == 0 || n == 0) return;
    if ((alpha_zero || k == 0) && beta.hi == 1.0 && beta.lo == 0.0) return;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) {
            odd cin = {ch[i + j * ldc], cl[i + j * ldc]};
            odd r = gemm_entry(ta, tb, i, j, k, alpha, ah, al, lda, bh, bl, ldb, beta, cin);
            ch[i + j * ldc] = r.hi;
            cl[i + j * ldc] = r.lo;
        }
    }
}

/* Selected entries only: out[q] = entry (rows[q], cols[q]) of the Rgemm result.
 * Used for sampled blocks of large problems; C is read-only here. */
void oracle_dd_gemm_entries(char transa, char transb, int64_t k, double alpha_hi,
                            double alpha_lo, const double *ah, const double *al, int64_t lda,
                            const double *bh, const double *bl, int64_t ldb, double beta_hi,
                            double beta_lo, const double *ch, const double *cl, int64_t ldc,
                            int64_t count, const int64_t *rows, const int64_t *cols,
                            double *out_hi, double *out_lo) {
    odd alpha = {alpha_hi, alpha_lo}, beta = {beta_hi, beta_lo};
    int ta = is_trans(transa), tb = is_trans(transb);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < count; ++q) {
        int64_t i = rows[q], j = cols[q];
        odd cin = {0.0, 0.0};
        if (!(beta.hi == 0.0 && beta.lo == 0.0)) {
            cin.hi = ch[i + j * ldc];
            cin.lo = cl[i + j * ldc];
        }
        odd r = gemm_entry(ta, tb, i, j, k, alpha, ah, al, lda, bh, bl, ldb, beta, cin);
        out_hi[q] = r.hi;
        out_lo[q] = r.lo;
    }
}

/* Rsyrk: C := alpha*A*A^T + beta*C (trans = 'N', A is n x k) or
 * C := alpha*A^T*A + beta*C (trans = 'T', A is k x n); only the uplo triangle
 * of C is referenced. */
void oracle_dd_syrk(char uplo, char trans, int64_t n, int64_t k, double alpha_hi,
                    double alpha_lo, const double *ah, const double *al, int64_t lda,
                    double beta_hi, double beta_lo, double *ch, double *cl, int64_t ldc) {
    odd alpha = {alpha_hi, alpha_lo}, beta = {beta_hi, beta_lo};
    int upper = (uplo == 'U' || uplo == 'u');
    int t = is_trans(trans);
    int alpha_zero = (alpha.hi == 0.0 && alpha.lo == 0.0);
    if (n == 0) return;
    if ((alpha_zero || k == 0) && beta.hi == 1.0 && beta.lo == 0.0) return;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j) {
        int64_t i0 = upper ? 0 : j, i1 = upper ? j + 1 : n;
        for (int64_t i = i0; i < i1; ++i) {
            odd cin = {ch[i + j * ldc], cl[i + j * ldc]};
            /* op(A) = A (n x k) for trans = N, so the entry is row i of op(A)
             * times row j of op(A); the second operand is op(A)^T. */
            odd r = gemm_entry(t, !t, i, j, k, alpha, ah, al, lda, ah, al, lda, beta, cin);
            ch[i + j * ldc] = r.hi;
            cl[i + j * ldc] = r.lo;
        }
    }
}

/* Rsyr2k: C := alpha*(A*B^T + B*A^T) + beta*C (trans = 'N', A and B n x k) or
 * C := alpha*(A^T*B + B^T*A) + beta*C (trans = 'T', A and B k x n); only the
 * uplo triangle of C is referenced (DSYR2K semantics).  Each entry sums the
 * 2k products a_il b_jl (l = 0..k-1) and then b_il a_jl in that order. */
void oracle_dd_syr2k(char uplo, char trans, int64_t n, int64_t k, double alpha_hi,
                     double alpha_lo, const double *ah, const double *al, int64_t lda,
                     const double *bh, const double *bl, int64_t ldb, double beta_hi,
                     double beta_lo, double *ch, double *cl, int64_t ldc) {
    odd alpha = {alpha_hi, alpha_lo}, beta = {beta_hi, beta_lo};
    int upper = (uplo == 'U' || uplo == 'u');
    int t = is_trans(trans);
    int alpha_zero = (alpha.hi == 0.0 && alpha.lo == 0.0);
    int beta_zero = (beta.hi == 0.0 && beta.lo == 0.0);
    if (n == 0) return;
    if ((alpha_zero || k == 0) && beta.hi == 1.0 && beta.lo == 0.0) return;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j) {
        int64_t i0 = upper ? 0 : j, i1 = upper ? j + 1 : n;
        for (int64_t i = i0; i < i1; ++i) {
            odd acc = {0.0, 0.0};
            if (!alpha_zero) {
                /* row i of op(A) is A(i, :) (N) or A(:, i) (T) */
                for (int64_t l = 0; l < k; ++l)
                    acc = dd_add(acc, dd_mul(op_elem(ah, al, lda, t, i, l),
                                             op_elem(bh, bl, ldb, t, j, l)));
                for (int64_t l = 0; l < k; ++l)
                    acc = dd_add(acc, dd_mul(op_elem(bh, bl, ldb, t, i, l),
                                             op_elem(ah, al, lda, t, j, l)));
                acc = dd_mul(alpha, acc);
            }
            if (!beta_zero)
                acc = dd_add(acc, dd_mul(beta, (odd){ch[i + j * ldc], cl[i + j * ldc]}));
            ch[i + j * ldc] = acc.hi;
            cl[i + j * ldc] = acc.lo;
        }
    }
}

/* Rsymm: C := alpha*A*B + beta*C (side = 'L', A m x m) or alpha*B*A + beta*C
 * (side = 'R', A n x n), A symmetric with only its uplo triangle read, B and
 * C m x n (DSYMM semantics).  A(r, c) outside the stored triangle is read
 * as A(c, r).  Products in the natural order of the inner index. */
void oracle_dd_symm(char side, char uplo, int64_t m, int64_t n, double alpha_hi,
                    double alpha_lo, const double *ah, const double *al, int64_t lda,
                    const double *bh, const double *bl, int64_t ldb, double beta_hi,
                    double beta_lo, double *ch, double *cl, int64_t ldc) {
    odd alpha = {alpha_hi, alpha_lo}, beta = {beta_hi, beta_lo};
    int left = !(side == 'R' || side == 'r');
    int upper = (uplo == 'U' || uplo == 'u');
    int alpha_zero = (alpha.hi == 0.0 && alpha.lo == 0.0);
    int beta_zero = (beta.hi == 0.0 && beta.lo == 0.0);
    if (m == 0 || n == 0) return;
    if (alpha_zero && beta.hi == 1.0 && beta.lo == 0.0) return;
    const int64_t k = left ? m : n;
#define SYM(r, c) ((upper ? (r) <= (c) : (r) >= (c)) ? ((r) + (c) * lda) : ((c) + (r) * lda))
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) {
            odd acc = {0.0, 0.0};
            if (!alpha_zero) {
                for (int64_t l = 0; l < k; ++l) {
                    odd a, b;
                    if (left) {
                        a = (odd){ah[SYM(i, l)], al[SYM(i, l)]};
                        b = (odd){bh[l + j * ldb], bl[l + j * ldb]};
                    } else {
                        a = (odd){bh[i + l * ldb], bl[i + l * ldb]};
                        b = (odd){ah[SYM(l, j)], al[SYM(l, j)]};
                    }
                    acc = dd_add(acc, dd_mul(a, b));
                }
                acc = dd_mul(alpha, acc);
            }
            if (!beta_zero)
                acc = dd_add(acc, dd_mul(beta, (odd){ch[i + j * ldc], cl[i + j * ldc]}));
            ch[i + j * ldc] = acc.hi;
            cl[i + j * ldc] = acc.lo;
        }
    }
#undef SYM
}

/* Rpotrf: Cholesky factorisation A = U^T U (uplo = 'U') or A = L L^T
 * (uplo = 'L'), unblocked, column by column (the LAPACK dpotf2 order).
 * Returns info: 0 on success, j > 0 if the leading minor of order j is not
 * positive definite (the factorisation stops there). */
int64_t oracle_dd_potrf(char uplo, int64_t n, double *ah, double *al, int64_t lda) {
    int upper = (uplo == 'U' || uplo == 'u');
    for (int64_t j = 0; j < n; ++j) {
        /* Element (r, c) of the stored triangle: U(r, c) with r <= c, or
         * L(c, r) = U(r, c)^T for the lower case. */
#define TRI(r, c) (upper ? ((r) + (c) * lda) : ((c) + (r) * lda))
        odd d = {ah[TRI(j, j)], al[TRI(j, j)]};
        for (int64_t i = 0; i < j; ++i) {
            odd u = {ah[TRI(i, j)], al[TRI(i, j)]};
            d = dd_sub(d, dd_mul(u, u));
        }
        if (!(d.hi > 0.0) || isnan(d.hi)) {
            ah[TRI(j, j)] = d.hi;
            al[TRI(j, j)] = d.lo;
            return j + 1;
        }
        odd ujj = dd_sqrt(d);
        ah[TRI(j, j)] = ujj.hi;
        al[TRI(j, j)] = ujj.lo;
        for (int64_t c = j + 1; c < n; ++c) {
            odd s = {ah[TRI(j, c)], al[TRI(j, c)]};
            for (int64_t i = 0; i < j; ++i) {
                odd uij = {ah[TRI(i, j)], al[TRI(i, j)]};
                odd uic = {ah[TRI(i, c)], al[TRI(i, c)]};
                s = dd_sub(s, dd_mul(uij, uic));
            }
            odd v = dd_div(s, ujj);
            ah[TRI(j, c)] = v.hi;
            al[TRI(j, c)] = v.lo;
        }
#undef TRI
    }
    return 0;
}

/* Rpotrs: solve A X = B with the factor from oracle_dd_potrf:
 * U^T U X = B (forward substitution with U^T, then back substitution with U),
 * or L L^T X = B.  B (n x nrhs) is overwritten by X. */
void oracle_dd_potrs(char uplo, int64_t n, int64_t nrhs, const double *ah, const double *al,
                     int64_t lda, double *bh, double *bl, int64_t ldb) {
    int upper = (uplo == 'U' || uplo == 'u');
#define UF(r, c) (upper ? ((r) + (c) * lda) : ((c) + (r) * lda))
    for (int64_t q = 0; q < nrhs; ++q) {
        double *xh = bh + q * ldb, *xl = bl + q * ldb;
        /* U^T y = b: y_i = (b_i - sum_{r<i} U(r,i) y_r) / U(i,i) */
        for (int64_t i = 0; i < n; ++i) {
            odd s = {xh[i], xl[i]};
            for (int64_t r = 0; r < i; ++r) {
                odd u = {ah[UF(r, i)], al[UF(r, i)]};
                s = dd_sub(s, dd_mul(u, (odd){xh[r], xl[r]}));
            }
            odd v = dd_div(s, (odd){ah[UF(i, i)], al[UF(i, i)]});
            xh[i] = v.hi;
            xl[i] = v.lo;
        }
        /* U x = y: x_i = (y_i - sum_{c>i} U(i,c) x_c) / U(i,i) */
        for (int64_t i = n - 1; i >= 0; --i) {
            odd s = {xh[i], xl[i]};
            for (int64_t c = i + 1; c < n; ++c) {
                odd u = {ah[UF(i, c)], al[UF(i, c)]};
                s = dd_sub(s, dd_mul(u, (odd){xh[c], xl[c]}));
            }
            odd v = dd_div(s, (odd){ah[UF(i, i)], al[UF(i, i)]});
            xh[i] = v.hi;
            xl[i] = v.lo;
        }
    }
#undef UF
}

/* Rtrsm: solve op(A) X = alpha B (side 'L') or X op(A) = alpha B (side 'R')
 * for X, which overwrites the m x n matrix B; A is triangular (uplo), unit
 * or not (diag), and only its uplo triangle is read.  DTRSM's semantics, the
 * routine MPBLAS lists among its real routines (manual Sec. 6).  Plain
 * substitution on one right-hand side at a time: for side 'L' the right-hand
 * sides are the columns of B and the triangular matrix is T = op(A); for
 * side 'R' they are the rows of B and T = op(A)^T, because x op(A) = b is
 * op(A)^T x^T = b^T.  Each b is first scaled by alpha (a dd product), then
 * x_i = (b_i - sum_c T(i, c) x_c) / T(i, i), the sum over the solved
 * components in their natural order, and the division skipped for a unit
 * diagonal.  alpha = 0 sets B to zero without reading A or B. */
void oracle_dd_trsm(char side, char uplo, char transa, char diag, int64_t m, int64_t n,
                    double alpha_hi, double alpha_lo, const double *ah, const double *al,
                    int64_t lda, double *bh, double *bl, int64_t ldb) {
    int right = (side == 'R' || side == 'r');
    int upper = (uplo == 'U' || uplo == 'u');
    int ta = is_trans(transa);
    int unit = (diag == 'U' || diag == 'u');
    odd alpha = {alpha_hi, alpha_lo};
    if (m == 0 || n == 0) return;
    if (alpha.hi == 0.0 && alpha.lo == 0.0) {
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < m; ++i) bh[i + j * ldb] = bl[i + j * ldb] = 0.0;
        return;
    }
    const int64_t order = right ? n : m;    /* order of T */
    const int64_t count = right ? m : n;    /* right-hand sides */
    /* T lower for (upper op(A) and side R) or (lower op(A) and side L) */
    const int op_upper = upper ^ ta;
    const int t_lower = right ? op_upper : !op_upper;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < count; ++q) {
        /* element i of right-hand side q */
#define BI(i) (right ? (q + (i) * ldb) : ((i) + q * ldb))
        /* T(r, c) = op(A)(r, c) (side L) or op(A)(c, r) (side R);
         * op(A)(r, c) = A(r, c), or A(c, r) when transposed */
#define TIDX(r, c) ((right ^ ta) ? ((c) + (r) * lda) : ((r) + (c) * lda))
        for (int64_t i = 0; i < order; ++i) {
            odd b = {bh[BI(i)], bl[BI(i)]};
            b = dd_mul(alpha, b);
            bh[BI(i)] = b.hi;
            bl[BI(i)] = b.lo;
        }
        for (int64_t s = 0; s < order; ++s) {
            const int64_t i = t_lower ? s : order - 1 - s;
            odd x = {bh[BI(i)], bl[BI(i)]};
            const int64_t c0 = t_lower ? 0 : i + 1, c1 = t_lower ? i : order;
            for (int64_t c = c0; c < c1; ++c) {
                odd t = {ah[TIDX(i, c)], al[TIDX(i, c)]};
                x = dd_sub(x, dd_mul(t, (odd){bh[BI(c)], bl[BI(c)]}));
            }
            if (!unit) x = dd_div(x, (odd){ah[TIDX(i, i)], al[TIDX(i, i)]});
            bh[BI(i)] = x.hi;
            bl[BI(i)] = x.lo;
        }
#undef TIDX
#undef BI
    }
}

/* |a| > |b| for normalised dd values (compares hi, then lo, of the absolute
 * values). */
static int dd_abs_greater(odd a, odd b) {
    if (a.hi < 0.0 || (a.hi == 0.0 && a.lo < 0.0)) a = dd_neg(a);
    if (b.hi < 0.0 || (b.hi == 0.0 && b.lo < 0.0)) b = dd_neg(b);
    return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}

/* Rgetrf: LU factorisation with partial pivoting, P A = L U, of the m x n A
 * (DGETRF semantics; MPLAPACK routine table, Sec. 6).  Unblocked, column by
 * column (the LAPACK dgetf2 order): the pivot of column j is the first row
 * p >= j of largest |A(p, j)|; rows j and p are interchanged across all n
 * columns (ipiv[j] = p + 1, one-based); the entries below the diagonal are
 * divided by the pivot (the multipliers, L's strict lower part); the
 * trailing (m-j-1) x (n-j-1) block receives the rank-one update
 * A(i, c) -= L(i, j) U(j, c).  A zero pivot sets info = j + 1 (the first
 * one), skips the division and the factorisation continues.  Returns info. */
int64_t oracle_dd_getrf(int64_t m, int64_t n, double *ah, double *al, int64_t lda,
                        int64_t *ipiv) {
    int64_t info = 0;
    const int64_t mn = m < n ? m : n;
    for (int64_t j = 0; j < mn; ++j) {
        int64_t p = j;
        for (int64_t i = j + 1; i < m; ++i)
            if (dd_abs_greater((odd){ah[i + j * lda], al[i + j * lda]},
                               (odd){ah[p + j * lda], al[p + j * lda]}))
                p = i;
        ipiv[j] = p + 1;
        const odd piv = {ah[p + j * lda], al[p + j * lda]};
        if (piv.hi == 0.0 && piv.lo == 0.0) {
            if (info == 0) info = j + 1;
            continue;
        }
        if (p != j)
            for (int64_t c = 0; c < n; ++c) {
                double th = ah[j + c * lda], tl = al[j + c * lda];
                ah[j + c * lda] = ah[p + c * lda];
                al[j + c * lda] = al[p + c * lda];
                ah[p + c * lda] = th;
                al[p + c * lda] = tl;
            }
        for (int64_t i = j + 1; i < m; ++i) {
            odd v = dd_div((odd){ah[i + j * lda], al[i + j * lda]}, piv);
            ah[i + j * lda] = v.hi;
            al[i + j * lda] = v.lo;
        }
#pragma omp parallel for schedule(static)
        for (int64_t c = j + 1; c < n; ++c) {
            const odd u = {ah[j + c * lda], al[j + c * lda]};
            for (int64_t i = j + 1; i < m; ++i) {
                odd x = {ah[i + c * lda], al[i + c * lda]};
                x = dd_sub(x, dd_mul((odd){ah[i + j * lda], al[i + j * lda]}, u));
                ah[i + c * lda] = x.hi;
                al[i + c * lda] = x.lo;
            }
        }
    }
    return info;
}

/* Rgetrs: solve A X = B (trans 'N') or A^T X = B ('T') with the factors and
 * pivots of oracle_dd_getrf (n x n), B n x nrhs overwritten by X (DGETRS
 * semantics).  'N': interchange B's rows as ipiv says (in order), solve
 * L Y = B (unit diagonal) forward, then U X = Y backward.  'T': solve
 * U^T Y = B forward, L^T Z = Y (unit) backward, then undo the interchanges
 * in reverse order. */
void oracle_dd_getrs(char trans, int64_t n, int64_t nrhs, const double *ah, const double *al,
                     int64_t lda, const int64_t *ipiv, double *bh, double *bl, int64_t ldb) {
    const int t = is_trans(trans);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nrhs; ++q) {
        double *xh = bh + q * ldb, *xl = bl + q * ldb;
#define SWAPROW(a, b)                                                   \
        do {                                                            \
            double th = xh[a], tl = xl[a];                              \
            xh[a] = xh[b]; xl[a] = xl[b]; xh[b] = th; xl[b] = tl;       \
        } while (0)
        if (!t) {
            for (int64_t j = 0; j < n; ++j)
                if (ipiv[j] - 1 != j) SWAPROW(j, ipiv[j] - 1);
            for (int64_t i = 0; i < n; ++i) {          /* L y = b */
                odd s = {xh[i], xl[i]};
                for (int64_t c = 0; c < i; ++c)
                    s = dd_sub(s, dd_mul((odd){ah[i + c * lda], al[i + c * lda]},
                                         (odd){xh[c], xl[c]}));
                xh[i] = s.hi; xl[i] = s.lo;
            }
            for (int64_t i = n - 1; i >= 0; --i) {     /* U x = y */
                odd s = {xh[i], xl[i]};
                for (int64_t c = i + 1; c < n; ++c)
                    s = dd_sub(s, dd_mul((odd){ah[i + c * lda], al[i + c * lda]},
                                         (odd){xh[c], xl[c]}));
                s = dd_div(s, (odd){ah[i + i * lda], al[i + i * lda]});
                xh[i] = s.hi; xl[i] = s.lo;
            }
        } else {
            for (int64_t i = 0; i < n; ++i) {          /* U^T y = b */
                odd s = {xh[i], xl[i]};
                for (int64_t c = 0; c < i; ++c)
                    s = dd_sub(s, dd_mul((odd){ah[c + i * lda], al[c + i * lda]},
                                         (odd){xh[c], xl[c]}));
                s = dd_div(s, (odd){ah[i + i * lda], al[i + i * lda]});
                xh[i] = s.hi; xl[i] = s.lo;
            }
            for (int64_t i = n - 1; i >= 0; --i) {     /* L^T z = y */
                odd s = {xh[i], xl[i]};
                for (int64_t c = i + 1; c < n; ++c)
                    s = dd_sub(s, dd_mul((odd){ah[c + i * lda], al[c + i * lda]},
                                         (odd){xh[c], xl[c]}));
                xh[i] = s.hi; xl[i] = s.lo;
            }
            for (int64_t j = n - 1; j >= 0; --j)
                if (ipiv[j] - 1 != j) SWAPROW(j, ipiv[j] - 1);
        }
#undef SWAPROW
    }
}

/* ------------------------------------------------------------------------- */
/* Tier 3: exact evaluation in a fixed-point superaccumulator                 */
/* ------------------------------------------------------------------------- */

/* The accumulator holds sum_d digit[d] * 2^(32*d + SA_LOW) with digits kept in
 * int64 so that up to 2^30 additions need no carry propagation.  Bits from
 * 2^SA_LOW to 2^(SA_LOW + 32*SA_DIGITS) are covered: every binary64 value and
 * every exact product of two or three binary64 values above 2^-2200. */
#define SA_DIGITS 144
#define SA_LOW (-2304)

typedef struct {
    int64_t d[SA_DIGITS];
    int64_t adds;
} superacc;

static void sa_clear(superacc *s) { memset(s, 0, sizeof(*s)); }

static void sa_normalise(superacc *s) {
    int64_t carry = 0;
    for (int i = 0; i < SA_DIGITS; ++i) {
        int64_t v = s->d[i] + carry;
        /* floor division by 2^32 keeps every digit in [0, 2^32) */
        int64_t q = v >> 32;
        s->d[i] = v - (q << 32);
        carry = q;
    }
    /* a non-zero carry out means the value is negative (two's complement in
     * base 2^32); keep it in the top digit so the sign can be read back */
    s->d[SA_DIGITS - 1] += carry << 32;
    s->adds = 0;
}

/* Add a binary64 value exactly. */
static void sa_add(superacc *s, double x) {
    if (x == 0.0) return;
    int e;
    double f = frexp(x, &e);                 /* x = f * 2^e, 0.5 <= |f| < 1 */
    int64_t mant = (int64_t)ldexp(f, 53);    /* exact, |mant| < 2^53 */
    int64_t pos = (int64_t)e - 53 - SA_LOW;  /* bit position of the mantissa LSB */
    if (pos < 0) abort();                    /* outside the covered range */
    int64_t di = pos / 32, sh = pos % 32;
    int neg = mant < 0;
    uint64_t um = (uint64_t)(neg ? -mant : mant);
    /* um << sh has at most 53 + 31 = 84 bits: three base-2^32 digits */
    unsigned __int128 v = (unsigned __int128)um << sh;
    int64_t sg = neg ? -1 : 1;
    if (di + 2 >= SA_DIGITS) abort();
    s->d[di] += sg * (int64_t)(uint64_t)(v & 0xffffffffULL);
    s->d[di + 1] += sg * (int64_t)(uint64_t)((v >> 32) & 0xffffffffULL);
    s->d[di + 2] += sg * (int64_t)(uint64_t)(v >> 64);
    if (++s->adds >= (1LL << 30)) sa_normalise(s);
}

/* Add the exact product x*y (two binary64 values). */
static void sa_add_prod2(superacc *s, double x, double y) {
    double p, e;
    two_prod(x, y, &p, &e);
    sa_add(s, p);
    sa_add(s, e);
}

/* Add the exact product x*y*z. */
static void sa_add_prod3(superacc *s, double x, double y, double z) {
    double p, e, p2, e2, p3, e3;
    two_prod(x, y, &p, &e);
    two_prod(p, z, &p2, &e2);
    two_prod(e, z, &p3, &e3);
    sa_add(s, p2);
    sa_add(s, e2);
    sa_add(s, p3);
    sa_add(s, e3);
}

/* Round the (normalised) accumulator to the nearest binary64, ties to even. */
static double sa_round(const superacc *src) {
    superacc s = *src;
    int neg = s.d[SA_DIGITS - 1] < 0;
    if (neg) {
        /* negate: value -> -value, digits back into [0, 2^32) */
        for (int i = 0; i < SA_DIGITS; ++i) s.d[i] = -s.d[i];
        sa_normalise(&s);
    }
    int top = -1;
    for (int i = SA_DIGITS - 1; i >= 0; --i)
        if (s.d[i] != 0) {
            top = i;
            break;
        }
    if (top < 0) return 0.0;
    /* absolute bit index of the most significant set bit */
    int b = 31;
    while (!((s.d[top] >> b) & 1)) --b;
    int64_t msb = (int64_t)top * 32 + b;
#define BIT(p) ((p) < 0 ? 0 : (int)((s.d[(p) / 32] >> ((p) % 32)) & 1))
    uint64_t mant = 0;
    for (int64_t p = msb; p > msb - 53; --p) mant = (mant << 1) | (uint64_t)BIT(p);
    int64_t rpos = msb - 53;
    int round_bit = BIT(rpos);
    int sticky = 0;
    for (int64_t p = rpos - 1; p >= 0 && !sticky; --p) sticky = BIT(p);
#undef BIT
    if (round_bit && (sticky || (mant & 1))) mant += 1;
    double r = ldexp((double)mant, (int)(msb - 52 + SA_LOW));
    return neg ? -r : r;
}

/* Round the exact value to the nearest dd: hi = RN(x), lo = RN(x - hi). */
static odd sa_round_dd(superacc *s) {
    sa_normalise(s);
    double hi = sa_round(s);
    sa_add(s, -hi);
    sa_normalise(s);
    double lo = sa_round(s);
    odd r = {hi, lo};
    return r;
}

/* Exact Rgemm entries: out[q] = RN_dd(alpha*sum_l op(A)(i,l)*op(B)(l,j) + beta*C(i,j))
 * for (i, j) = (rows[q], cols[q]); C is read only if beta != 0. */
void oracle_exact_gemm_entries(char transa, char transb, int64_t k, double alpha_hi,
                               double alpha_lo, const double *ah, const double *al,
                               int64_t lda, const double *bh, const double *bl, int64_t ldb,
                               double beta_hi, double beta_lo, const double *ch,
                               const double *cl, int64_t ldc, int64_t count,
                               const int64_t *rows, const int64_t *cols, double *out_hi,
                               double *out_lo) {
    int ta = is_trans(transa), tb = is_trans(transb);
    double alpha[2] = {alpha_hi, alpha_lo};
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < count; ++q) {
        superacc *s = (superacc *)malloc(sizeof(superacc));
        sa_clear(s);
        int64_t i = rows[q], j = cols[q];
        for (int64_t l = 0; l < k; ++l) {
            odd a = op_elem(ah, al, lda, ta, i, l);
            odd b = op_elem(bh, bl, ldb, tb, l, j);
            double av[2] = {a.hi, a.lo}, bv[2] = {b.hi, b.lo};
            for (int x = 0; x < 2; ++x)
                for (int y = 0; y < 2; ++y)
                    for (int z = 0; z < 2; ++z)
                        if (alpha[x] != 0.0 && av[y] != 0.0 && bv[z] != 0.0)
                            sa_add_prod3(s, alpha[x], av[y], bv[z]);
        }
        if (!(beta_hi == 0.0 && beta_lo == 0.0)) {
            double bt[2] = {beta_hi, beta_lo};
            double cv[2] = {ch[i + j * ldc], cl[i + j * ldc]};
            for (int x = 0; x < 2; ++x)
                for (int y = 0; y < 2; ++y)
                    if (bt[x] != 0.0 && cv[y] != 0.0) sa_add_prod2(s, bt[x], cv[y]);
        }
        odd r = sa_round_dd(s);
        out_hi[q] = r.hi;
        out_lo[q] = r.lo;
        free(s);
    }
}

/* ------------------------------------------------------------------------- */
/* Quad-double (qd): a value is x0 + x1 + x2 + x3 of four binary64 numbers    */
/* (the manual's quad-double format, Sec. 5, from the QD library)             */
/* ------------------------------------------------------------------------- */

/* Round the accumulator to qd: x0 = RN(S), x1 = RN(S - x0), x2 = RN(S - x0 -
 * x1), x3 = RN(S - x0 - x1 - x2); every subtraction is exact in the
 * accumulator, so |S - (x0 + x1 + x2 + x3)| <= ulp(x3) / 2. */
static void sa_round_qd(superacc *s, double out[4]) {
    for (int t = 0; t < 4; ++t) {
        sa_normalise(s);
        out[t] = sa_round(s);
        sa_add(s, -out[t]);
    }
}

/* Exact qd Rgemm entries: out[t][q] = component t of RN_qd(alpha*sum_l
 * op(A)(i,l)*op(B)(l,j) + beta*C(i,j)) for (i, j) = (rows[q], cols[q]).
 * alpha, beta: 4 components each; A, B, C, out: 4 column-major planes each
 * (A and B with leading dimensions lda, ldb; C with ldc, read only if beta
 * != 0).  Every one of the 64 triple products alpha_t a_u b_v per l is
 * accumulated exactly. */
void oracle_exact_qd_gemm_entries(char transa, char transb, int64_t k, const double *alpha,
                                  const double *const *A, int64_t lda, const double *const *B,
                                  int64_t ldb, const double *beta, const double *const *C,
                                  int64_t ldc, int64_t count, const int64_t *rows,
                                  const int64_t *cols, double *const *out) {
    int ta = is_trans(transa), tb = is_trans(transb);
    int beta_zero = beta[0] == 0.0 && beta[1] == 0.0 && beta[2] == 0.0 && beta[3] == 0.0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < count; ++q) {
        superacc *s = (superacc *)malloc(sizeof(superacc));
        sa_clear(s);
        int64_t i = rows[q], j = cols[q];
        for (int64_t l = 0; l < k; ++l) {
            int64_t ia = ta ? (l + i * lda) : (i + l * lda);
            int64_t ib = tb ? (j + l * ldb) : (l + j * ldb);
            for (int x = 0; x < 4; ++x)
                for (int y = 0; y < 4; ++y)
                    for (int z = 0; z < 4; ++z)
                        if (alpha[x] != 0.0 && A[y][ia] != 0.0 && B[z][ib] != 0.0)
                            sa_add_prod3(s, alpha[x], A[y][ia], B[z][ib]);
        }
        if (!beta_zero)
            for (int x = 0; x < 4; ++x)
                for (int y = 0; y < 4; ++y)
                    if (beta[x] != 0.0 && C[y][i + j * ldc] != 0.0)
                        sa_add_prod2(s, beta[x], C[y][i + j * ldc]);
        double r[4];
        sa_round_qd(s, r);
        for (int t = 0; t < 4; ++t) out[t][q] = r[t];
        free(s);
    }
}

/* Exact sum of an array of binary64 values, rounded to dd (pins the
 * superaccumulator itself against known sums). */
void oracle_exact_sum(int64_t n, const double *x, double *out_hi, double *out_lo) {
    superacc *s = (superacc *)malloc(sizeof(superacc));
    sa_clear(s);
    for (int64_t i = 0; i < n; ++i) sa_add(s, x[i]);
    odd r = sa_round_dd(s);
    *out_hi = r.hi;
    *out_lo = r.lo;
    free(s);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
