// Quad-double (qd) Rgemm on the FP64 pipe: C := alpha op(A) op(B) + beta C
// with every operand a qd value x0 + x1 + x2 + x3 of four binary64 numbers
// (the manual's quad-double format, Sec. 5: the QD library's qd_real; Rgemm
// argument list of Sec. 7.3).
//
// Multiply-add, built on the error-free transformations the manual names
// (Knuth's TwoSum; the product split exactly by one FMA): the accumulator
// is four levels L0..L3 of decreasing order of magnitude (L_t ~ u^t |acc|,
// u = 2^-53).  For a step a * b the products of order 1, u and u^2 (a0 b0;
// a0 b1, a1 b0; a0 b2, a1 b1, a2 b0) are split exactly into value and error
// (two_prod); each value enters the level of its order and each error the
// level below, all through TwoSum, whose error in turn moves one level
// down; level 3 receives those errors and the u^3 products (a0 b3 + a1 b2 +
// a2 b1 + a3 b0, one FMA chain) in plain binary64.  The only roundings are
// level 3's additions (each within u^4 (|acc| + c |a b|)) and the dropped
// products of order u^4 and below (within 7 u^4 |a b|), so the result
// stays within the qd bound 4 k 2^-209 (|alpha||A||B| + |beta||C|).  Every
// 4 steps one bottom-up TwoSum pass (L2+L3, L1+L2, L0+L1) brings level t
// back to order u^t |acc|; the pass is exact.  113 FP64 operations per
// step plus 4.5 for the pass.
//
// Tiles: 16R x 16R of C per CTA (R = 2 or 1, the larger one when the tiles
// still fill the SMs), R x R qd accumulators per thread, the four planes of
// the op(A) and op(B) panels staged through shared memory 16 columns of k
// at a time.  The per-entry operation sequence does not depend on R.
#include "common.cuh"
#include "dd_arith.cuh"
#include "kernels.cuh"

namespace mpdd {
namespace {

constexpr int QBK = 16, QNT = 256, kQdRenormEvery = 4;

struct qd4 {
    double x0, x1, x2, x3;
};

__device__ __forceinline__ void qd_mac(double (&L)[4], const qd4 &a, const qd4 &b) {
    double e, f0, f1, f2, f3;
    const double p0 = __dmul_rn(a.x0, b.x0), q0 = __fma_rn(a.x0, b.x0, -p0);
    two_sum(L[0], p0, L[0], e);
    const double p1 = __dmul_rn(a.x0, b.x1), q1 = __fma_rn(a.x0, b.x1, -p1);
    const double p2 = __dmul_rn(a.x1, b.x0), q2 = __fma_rn(a.x1, b.x0, -p2);
    two_sum(L[1], e, L[1], f0);
    two_sum(L[1], q0, L[1], f1);
    two_sum(L[1], p1, L[1], f2);
    two_sum(L[1], p2, L[1], f3);
    const double p3 = __dmul_rn(a.x0, b.x2), q3 = __fma_rn(a.x0, b.x2, -p3);
    const double p4 = __dmul_rn(a.x1, b.x1), q4 = __fma_rn(a.x1, b.x1, -p4);
    const double p5 = __dmul_rn(a.x2, b.x0), q5 = __fma_rn(a.x2, b.x0, -p5);
    double g0, g1, g2, g3, g4, g5, g6, g7, g8;
    two_sum(L[2], f0, L[2], g0);
    two_sum(L[2], f1, L[2], g1);
    two_sum(L[2], f2, L[2], g2);
    two_sum(L[2], f3, L[2], g3);
    two_sum(L[2], q1, L[2], g4);
    two_sum(L[2], q2, L[2], g5);
    two_sum(L[2], p3, L[2], g6);
    two_sum(L[2], p4, L[2], g7);
    two_sum(L[2], p5, L[2], g8);
    const double t3 =
        __fma_rn(a.x0, b.x3, __fma_rn(a.x1, b.x2, __fma_rn(a.x2, b.x1, __dmul_rn(a.x3, b.x0))));
    const double s = __dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn(g0, g1), __dadd_rn(g2, g3)),
                                         __dadd_rn(__dadd_rn(g4, g5), __dadd_rn(g6, g7))),
                               __dadd_rn(g8, __dadd_rn(__dadd_rn(q3, q4), __dadd_rn(q5, t3))));
    L[3] = __dadd_rn(L[3], s);
}

__device__ __forceinline__ void qd_pass(double (&L)[4]) {
    two_sum(L[2], L[3], L[2], L[3]);
    two_sum(L[1], L[2], L[1], L[2]);
    two_sum(L[0], L[1], L[0], L[1]);
}

// Four non-overlapping components (|x_{t+1}| <= ulp(x_t) / 2) of the value of
// the levels: three exact bottom-up passes concentrate the value in the
// leading terms, then a top-down FastTwoSum pass separates them.
__device__ __forceinline__ qd4 qd_finish(double (&L)[4]) {
    qd_pass(L);
    qd_pass(L);
    qd_pass(L);
    fast_two_sum(L[0], L[1], L[0], L[1]);
    fast_two_sum(L[1], L[2], L[1], L[2]);
    fast_two_sum(L[2], L[3], L[2], L[3]);
    return qd4{L[0], L[1], L[2], L[3]};
}

struct QdArgs {
    int64_t m, n, k;
    qd4 alpha, beta;
    const double *a[4];
    int64_t lda;
    const double *b[4];
    int64_t ldb;
    double *c[4];
    int64_t ldc;
    int alpha_zero, alpha_one, beta_zero;
};

template <int R>
struct QdSmem {
    static constexpr int B = 16 * R;
    double a[4][QBK][B + 1];   // op(A) panel planes, [l][i]
    double b[4][QBK][B + 1];   // op(B) panel planes, [l][j]
};

template <int TA, int TB, int R>
__global__ void __launch_bounds__(QNT, 1) qd_gemm_kernel(const QdArgs p) {
    constexpr int BM = 16 * R;
    __shared__ QdSmem<R> s;
    const int64_t tm = (p.m + BM - 1) / BM;
    const int64_t bi = blockIdx.x % tm, bj = blockIdx.x / tm;
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    const int64_t i0 = bi * BM, j0 = bj * BM;
    const int64_t kk = p.alpha_zero ? 0 : p.k;

    double L[R][R][4];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c)
#pragma unroll
            for (int v = 0; v < 4; ++v) L[r][c][v] = 0.0;

    double ra[4][R], rb[4][R];
    auto a_pos = [&](int q, int &ii, int &ll) {
        const int idx = t + QNT * q;
        if (!TA) { ii = idx % BM; ll = idx / BM; }
        else     { ll = idx % QBK; ii = idx / QBK; }
    };
    auto b_pos = [&](int q, int &jj, int &ll) {
        const int idx = t + QNT * q;
        if (!TB) { ll = idx % QBK; jj = idx / QBK; }
        else     { jj = idx % BM; ll = idx / BM; }
    };
    auto load = [&](int64_t l0) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            int ii, jj, ll;
            a_pos(q, ii, ll);
            int64_t gi = i0 + ii, gl = l0 + ll;
            bool ok = gi < p.m && gl < kk;
            int64_t off = TA ? (gl + gi * p.lda) : (gi + gl * p.lda);
#pragma unroll
            for (int v = 0; v < 4; ++v) ra[v][q] = ok ? p.a[v][off] : 0.0;
            b_pos(q, jj, ll);
            const int64_t gj = j0 + jj;
            gl = l0 + ll;
            ok = gj < p.n && gl < kk;
            off = TB ? (gj + gl * p.ldb) : (gl + gj * p.ldb);
#pragma unroll
            for (int v = 0; v < 4; ++v) rb[v][q] = ok ? p.b[v][off] : 0.0;
        }
    };
    auto stage = [&]() {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            int ii, jj, ll;
            a_pos(q, ii, ll);
#pragma unroll
            for (int v = 0; v < 4; ++v) s.a[v][ll][ii] = ra[v][q];
            b_pos(q, jj, ll);
#pragma unroll
            for (int v = 0; v < 4; ++v) s.b[v][ll][jj] = rb[v][q];
        }
    };

    if (kk > 0) {
        load(0);
        for (int64_t l0 = 0; l0 < kk; l0 += QBK) {
            __syncthreads();
            stage();
            __syncthreads();
            if (l0 + QBK < kk) load(l0 + QBK);
#pragma unroll 1
            for (int l4 = 0; l4 < QBK; l4 += kQdRenormEvery) {
#pragma unroll 1
                for (int l = l4; l < l4 + kQdRenormEvery; ++l) {
                    qd4 a[R], b[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int i = tx + 16 * r;
                        a[r] = qd4{s.a[0][l][i], s.a[1][l][i], s.a[2][l][i], s.a[3][l][i]};
                    }
#pragma unroll
                    for (int c = 0; c < R; ++c) {
                        const int j = ty + 16 * c;
                        b[c] = qd4{s.b[0][l][j], s.b[1][l][j], s.b[2][l][j], s.b[3][l][j]};
                    }
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int c = 0; c < R; ++c) qd_mac(L[r][c], a[r], b[c]);
                }
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int c = 0; c < R; ++c) qd_pass(L[r][c]);
            }
        }
    }

    // epilogue: C := alpha acc + beta C, the two products accumulated in
    // fresh levels the same way as the k loop
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) {
            const int64_t i = i0 + tx + 16 * r, j = j0 + ty + 16 * c;
            if (i >= p.m || j >= p.n) continue;
            const int64_t off = i + j * p.ldc;
            double E[4] = {0.0, 0.0, 0.0, 0.0};
            if (p.alpha_one) {
#pragma unroll
                for (int v = 0; v < 4; ++v) E[v] = L[r][c][v];
            } else if (!p.alpha_zero) {
                const qd4 acc = qd_finish(L[r][c]);
                qd_mac(E, p.alpha, acc);
                qd_pass(E);
            }
            if (!p.beta_zero) {
                const qd4 cin{p.c[0][off], p.c[1][off], p.c[2][off], p.c[3][off]};
                qd_mac(E, p.beta, cin);
            }
            const qd4 out = qd_finish(E);
            p.c[0][off] = out.x0;
            p.c[1][off] = out.x1;
            p.c[2][off] = out.x2;
            p.c[3][off] = out.x3;
        }
}

template <int TA, int TB, int R>
void qd_launch(const QdArgs &p, cudaStream_t st) {
    const int64_t b = 16 * R;
    const dim3 grid((unsigned)(ceil_div(p.m, b) * ceil_div(p.n, b)));
    qd_gemm_kernel<TA, TB, R><<<grid, QNT, 0, st>>>(p);
}

template <int R>
int qd_launch_r(const QdArgs &p, int ta, int tb, cudaStream_t st) {
    const int64_t b = 16 * R;
    if (ceil_div(p.m, b) * ceil_div(p.n, b) > 0x7fffffffLL)
        return fail(MP_DD_ERR_TOO_LARGE, "qd Rgemm: m x n too large");
    if (!ta && !tb) qd_launch<0, 0, R>(p, st);
    else if (ta && !tb) qd_launch<1, 0, R>(p, st);
    else if (!ta && tb) qd_launch<0, 1, R>(p, st);
    else qd_launch<1, 1, R>(p, st);
    return check_launch("qd_gemm_kernel");
}

}  // namespace

int run_qd_gemm(int ta, int tb, int64_t m, int64_t n, int64_t k, const double *alpha,
                const double *const *a, int64_t lda, const double *const *b, int64_t ldb,
                const double *beta, double *const *c, int64_t ldc, cudaStream_t st) {
    QdArgs p{};
    p.m = m; p.n = n; p.k = k;
    p.alpha = qd4{alpha[0], alpha[1], alpha[2], alpha[3]};
    p.beta = qd4{beta[0], beta[1], beta[2], beta[3]};
    for (int v = 0; v < 4; ++v) {
        p.a[v] = a[v];
        p.b[v] = b[v];
        p.c[v] = c[v];
    }
    p.lda = lda; p.ldb = ldb; p.ldc = ldc;
    p.alpha_zero = (alpha[0] == 0.0 && alpha[1] == 0.0 && alpha[2] == 0.0 && alpha[3] == 0.0) ||
                   k == 0;
    p.alpha_one = alpha[0] == 1.0 && alpha[1] == 0.0 && alpha[2] == 0.0 && alpha[3] == 0.0;
    p.beta_zero = beta[0] == 0.0 && beta[1] == 0.0 && beta[2] == 0.0 && beta[3] == 0.0;
    // R = 2 when its tiles fill the SMs at least as well as R = 1's (time
    // ~ ceil(tiles / SMs) R^2), else R = 1
    const int64_t sms = sm_count() > 0 ? sm_count() : 152;
    const int64_t t2 = ceil_div(ceil_div(m, 32) * ceil_div(n, 32), sms) * 4;
    const int64_t t1 = ceil_div(ceil_div(m, 16) * ceil_div(n, 16), sms);
    return t2 <= t1 ? qd_launch_r<2>(p, ta, tb, st) : qd_launch_r<1>(p, ta, tb, st);
}

}  // namespace mpdd
