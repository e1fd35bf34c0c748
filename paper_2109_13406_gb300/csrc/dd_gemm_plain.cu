// Plain double-double Rgemm / Rsyrk kernel for sm_103a (FP64 DFMA path).
//
// Computes C := alpha op(A) op(B) + beta C (Rgemm), one triangle of
// alpha A A^T + beta C (Rsyrk) or of alpha (A B^T + B A^T) + beta C (Rsyr2k:
// the second product continues the same k loop), and alpha S B + beta C or
// alpha B S + beta C with S symmetric and one triangle stored (Rsymm: the
// operand is read through the stored triangle); MPBLAS semantics (manual
// Sec. 7.3 and the routine table of Sec. 6).  Every multiply-add is dd
// arithmetic: the exact product of the hi parts by FMA, the two cross
// products, TwoSum into the accumulator, and a FastTwoSum renormalisation
// every 4 steps of k (dd_arith.cuh).
//
// On GB300 the FP64 pipe is the bottleneck by a wide margin (12.75 FP64
// instructions per dd multiply-add), so the kernel is organised to keep that
// pipe busy and nothing else (large plain products go to the TMA-staged form
// of this kernel, dd_gemm_tma.cu, whose per-entry arithmetic is identical): each CTA owns a 16R x 16R tile of C (R = 4, 2
// or 1), each thread an R x R block of dd accumulators, and the hi/lo planes
// of the op(A) and op(B) panels are staged through shared memory 16 columns
// of k at a time with a register prefetch of the next panel.  One SM's FP64
// pipe issues only 2 lanes per clock, so a few warps keep it busy whatever R
// is; the launch picks R so that the tiles fill all SMs (large products:
// 64 x 64, the fewest operand loads per multiply-add; thin ones: smaller
// tiles, more CTAs).  Loads are zero-filled outside the matrices; a zero product leaves
// a normalised accumulator bitwise unchanged, so the per-entry operation
// sequence (l = 0, 1, ..., k-1) and hence the result are independent of the
// tiling.  Rsyrk uses the same instantiation as Rgemm(N, T) / (T, N) over
// the tiles of one triangle, so its entries equal Rgemm's bit for bit.
#include "common.cuh"
#include "dd_arith.cuh"
#include "kernels.cuh"
#include "ozaki_common.cuh"

namespace mpdd {
namespace {

constexpr int BK = 16, NT = 256;

template <int R>
struct PlainSmem {
    static constexpr int B = 16 * R;
    double ah[BK][B + 1], al[BK][B + 1];  // op(A) panel, [l][i]
    double bh[BK][B + 1], bl[BK][B + 1];  // op(B) panel, [l][j]
};

constexpr int GROUP_N = 8;  // tile columns per rasterisation group

// Tile (bi, bj) of this CTA.  Rgemm: a 1-D grid walked in groups of GROUP_N
// tile columns with the tile row fastest inside a group, so the CTAs
// resident at one time share a few A row panels and B column panels in L2
// (a plain column-by-column order re-reads all of A for every tile column).
// Rsyrk: a 1-D grid over the tiles of one triangle, t -> (row, col) with
// row <= col (upper) or row >= col (lower).
template <int BM, int BN>
__device__ __forceinline__ void tile_coords(const GemmArgs &p, int64_t &bi, int64_t &bj) {
    if (p.tri == 0) {
        const int64_t tm = (p.m + BM - 1) / BM, tn = (p.n + BN - 1) / BN;
        const int64_t t = blockIdx.x;
        const int64_t group = t / (tm * GROUP_N);
        const int64_t first = group * GROUP_N;
        const int64_t gn = tn - first < GROUP_N ? tn - first : GROUP_N;
        const int64_t local = t - group * tm * GROUP_N;
        bj = first + local % gn;
        bi = local / gn;
        return;
    }
    int64_t t = blockIdx.x;
    int64_t r = (int64_t)((__dsqrt_rn(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    int64_t c = t - r * (r + 1) / 2;  // 0 <= c <= r
    if (p.tri == 1) {
        bi = c;
        bj = r;
    } else {
        bi = r;
        bj = c;
    }
}

template <int TA, int TB, int R>
__device__ __forceinline__ void plain_body(const GemmArgs &p, PlainSmem<R> &s) {
    constexpr int BM = 16 * R, BN = 16 * R;
    if (p.info != nullptr && *p.info != 0) return;  // an earlier step failed
    // behind a split-precision call: compute only when its certificate failed
    if (p.gate != nullptr &&
        *reinterpret_cast<const volatile unsigned int *>(p.gate) >= p.gate_below)
        return;
    int64_t bi, bj;
    tile_coords<BM, BN>(p, bi, bj);
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    const int64_t i0 = bi * BM, j0 = bj * BN;
    // the k loop: [0, k) over (A, B), then for Rsyr2k [k1, k1 + k) over
    // (A2, B2), k1 = k rounded up to whole panels (zero products between)
    const int64_t k1 = (p.k + BK - 1) / BK * BK;
    const int64_t kk = p.alpha_zero ? 0 : (p.a2h != nullptr ? k1 + p.k : p.k);

    dd acc[R][R];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) acc[r][c] = dd{0.0, 0.0};

    // a panel holds 16R x 16 entries of op(A) and of op(B): R per thread
    double rah[R], ral[R], rbh[R], rbl[R];
    // Element q of this thread's share of a panel: (row-in-panel, l).
    auto a_pos = [&](int q, int &ii, int &ll) {
        int idx = t + NT * q;
        if (!TA) { ii = idx % BM; ll = idx / BM; }   // contiguous in i
        else     { ll = idx % BK; ii = idx / BK; }   // contiguous in l
    };
    auto b_pos = [&](int q, int &jj, int &ll) {
        int idx = t + NT * q;
        if (!TB) { ll = idx % BK; jj = idx / BK; }   // contiguous in l
        else     { jj = idx % BN; ll = idx / BN; }   // contiguous in j
    };
    auto load = [&](int64_t l0) {
        const bool second = p.a2h != nullptr && l0 >= k1;
        const double *Ah = second ? p.a2h : p.ah, *Al = second ? p.a2l : p.al;
        const double *Bh = second ? p.b2h : p.bh, *Bl = second ? p.b2l : p.bl;
        const int64_t lda = second ? p.lda2 : p.lda, ldb = second ? p.ldb2 : p.ldb;
        const int64_t lb = second ? l0 - k1 : l0;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            int ii, ll;
            a_pos(q, ii, ll);
            int64_t gi = i0 + ii, gl = lb + ll;
            bool ok = gi < p.m && gl < p.k;
            int64_t off = TA ? (gl + gi * lda) : (gi + gl * lda);
            if (p.sym_a) {
                const bool direct = p.sym_a == 1 ? gi <= gl : gi >= gl;
                off = direct ? gi + gl * lda : gl + gi * lda;
            }
            rah[q] = ok ? Ah[off] : 0.0;
            ral[q] = ok ? Al[off] : 0.0;
            int jj;
            b_pos(q, jj, ll);
            int64_t gj = j0 + jj;
            gl = lb + ll;
            ok = gj < p.n && gl < p.k;
            off = TB ? (gj + gl * ldb) : (gl + gj * ldb);
            if (p.sym_b) {
                const bool direct = p.sym_b == 1 ? gl <= gj : gl >= gj;
                off = direct ? gl + gj * ldb : gj + gl * ldb;
            }
            rbh[q] = ok ? Bh[off] : 0.0;
            rbl[q] = ok ? Bl[off] : 0.0;
        }
    };
    auto stage = [&]() {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            int ii, jj, ll;
            a_pos(q, ii, ll);
            s.ah[ll][ii] = rah[q];
            s.al[ll][ii] = ral[q];
            b_pos(q, jj, ll);
            s.bh[ll][jj] = rbh[q];
            s.bl[ll][jj] = rbl[q];
        }
    };

    if (kk > 0) {
        load(0);
        for (int64_t l0 = 0; l0 < kk; l0 += BK) {
            __syncthreads();
            stage();
            __syncthreads();
            if (l0 + BK < kk) load(l0 + BK);
#pragma unroll 1
            for (int l4 = 0; l4 < BK; l4 += kRenormEvery) {
#pragma unroll
                for (int l = l4; l < l4 + kRenormEvery; ++l) {
                    dd a[R], b[R];
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        a[r] = dd{s.ah[l][tx + 16 * r], s.al[l][tx + 16 * r]};
#pragma unroll
                    for (int c = 0; c < R; ++c)
                        b[c] = dd{s.bh[l][ty + 16 * c], s.bl[l][ty + 16 * c]};
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int c = 0; c < R; ++c) mac_deferred(acc[r][c], a[r], b[c]);
                }
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int c = 0; c < R; ++c) renorm(acc[r][c]);
            }
        }
    }

    const dd alpha{p.alpha.hi, p.alpha.lo}, beta{p.beta.hi, p.beta.lo};
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) {
            int64_t i = i0 + tx + 16 * r, j = j0 + ty + 16 * c;
            if (i >= p.m || j >= p.n) continue;
            if ((p.tri == 1 && i > j) || (p.tri == 2 && i < j)) continue;
            dd v = p.alpha_one ? acc[r][c] : mul(alpha, acc[r][c]);
            int64_t off = i + j * p.ldc;
            if (!p.beta_zero) v = add(v, mul(beta, dd{p.ch[off], p.cl[off]}));
            p.ch[off] = v.hi;
            p.cl[off] = v.lo;
        }
}

// 64 x 64 tiles (one CTA per SM by registers) and the smaller tiles (two or
// more CTAs per SM, registers capped accordingly).
template <int TA, int TB>
__global__ void __launch_bounds__(NT) dd_gemm_plain_kernel(const GemmArgs p) {
    __shared__ PlainSmem<4> s;
    plain_body<TA, TB, 4>(p, s);
}

template <int TA, int TB, int R>
__global__ void __launch_bounds__(NT, 2) dd_gemm_plain_small_kernel(const GemmArgs p) {
    __shared__ PlainSmem<R> s;
    plain_body<TA, TB, R>(p, s);
}

}  // namespace

namespace {

int64_t tile_count(const GemmArgs &p, int b) {
    const int64_t tm = ceil_div(p.m, b), tn = ceil_div(p.n, b);
    return p.tri == 0 ? tm * tn : tm * (tm + 1) / 2;
}

template <int TA, int TB, int R>
void launch_one(dim3 grid, const GemmArgs &p, cudaStream_t stream) {
    if constexpr (R == 4)
        dd_gemm_plain_kernel<TA, TB><<<grid, NT, 0, stream>>>(p);
    else
        dd_gemm_plain_small_kernel<TA, TB, R><<<grid, NT, 0, stream>>>(p);
}

template <int R>
int launch_r(const GemmArgs &p, cudaStream_t stream) {
    const int64_t tiles = tile_count(p, 16 * R);
    if (tiles > 0x7fffffffLL) return fail(MP_DD_ERR_TOO_LARGE, "m x n too large");
    const dim3 grid((unsigned)tiles);
    if (p.ta == 0 && p.tb == 0) launch_one<0, 0, R>(grid, p, stream);
    else if (p.ta == 1 && p.tb == 0) launch_one<1, 0, R>(grid, p, stream);
    else if (p.ta == 0 && p.tb == 1) launch_one<0, 1, R>(grid, p, stream);
    else launch_one<1, 1, R>(grid, p, stream);
    return check_launch("dd_gemm_plain_kernel");
}

}  // namespace

// Tile size: the time of a launch is about (tiles per SM, rounded up) x
// (work per tile), i.e. ceil(tiles_R / SMs) R^2 in units of a 16 x 16 tile;
// the largest R with the least such time wins (the per-entry operation
// sequence, and hence the result, does not depend on R).
int64_t plain_tile_cost(const GemmArgs &p, int r) {
    const int64_t sms = sm_count() > 0 ? sm_count() : 152;
    return ceil_div(tile_count(p, 16 * r), sms) * r * r;
}

int plain_tile_r(const GemmArgs &p) {
    int best = 4;
    int64_t best_t = -1;
    for (int r = 4; r >= 1; r /= 2) {
        const int64_t t = plain_tile_cost(p, r);
        if (best_t < 0 || t < best_t) { best_t = t; best = r; }
    }
    return best;
}

// The plain kernel behind a split-precision call: the same launch, gated on
// the call's certificate (every CTA returns at once when a width certified
// the bound).
int launch_plain_fallback(const GemmArgs &p, const SplitPlan &plan, cudaStream_t stream) {
    GemmArgs q = p;
    q.gate = plan.dmin;
    q.gate_below = plan.thr[plan.ncand - 1];
    // with the gate closed every CTA returns at once, so the launch costs
    // about its CTA count: the persistent TMA-staged kernel where it applies,
    // else the 64 x 64 tiles whenever they fill the SMs twice (the result
    // does not depend on the staging or the tile size)
    int rc = 0;
    if (try_launch_gemm_tma(q, stream, &rc)) return rc;
    const int64_t sms = sm_count() > 0 ? sm_count() : 152;
    if (tile_count(q, 64) >= 2 * sms) return launch_r<4>(q, stream);
    return launch_gemm_plain(q, stream);
}

int launch_gemm_plain(const GemmArgs &p, cudaStream_t stream) {
    int rc = 0;
    if (try_launch_gemm_tma(p, stream, &rc)) return rc;
    switch (plain_tile_r(p)) {
        case 1: return launch_r<1>(p, stream);
        case 2: return launch_r<2>(p, stream);
        default: return launch_r<4>(p, stream);
    }
}

}  // namespace mpdd
