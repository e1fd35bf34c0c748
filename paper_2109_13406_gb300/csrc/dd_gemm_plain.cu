// Plain double-double Rgemm / Rsyrk kernel for sm_103a (FP64 DFMA path).
//
// Computes C := alpha op(A) op(B) + beta C (Rgemm) or one triangle of
// alpha A A^T + beta C (Rsyrk), MPBLAS semantics (manual Sec. 7.3 and the
// routine table of Sec. 6).  Every multiply-add is dd arithmetic: the exact
// product of the hi parts by FMA, the two cross products, TwoSum into the
// accumulator, and a FastTwoSum renormalisation every 4 steps of k
// (dd_arith.cuh).
//
// On GB300 the FP64 pipe is the bottleneck by a wide margin (12.75 FP64
// instructions per dd multiply-add), so the kernel is organised to keep that
// pipe busy and nothing else: each CTA owns a 64 x 64 tile of C, each thread
// a 4 x 4 block of dd accumulators (16 independent dependency chains), and
// the hi/lo planes of the op(A) and op(B) panels are staged through shared
// memory 16 columns of k at a time with a register prefetch of the next
// panel.  Loads are zero-filled outside the matrices; a zero product leaves
// a normalised accumulator bitwise unchanged, so the per-entry operation
// sequence (l = 0, 1, ..., k-1) and hence the result are independent of the
// tiling.  Rsyrk uses the same instantiation as Rgemm(N, T) / (T, N) over
// the tiles of one triangle, so its entries equal Rgemm's bit for bit.
#include "common.cuh"
#include "dd_arith.cuh"
#include "kernels.cuh"

namespace mpdd {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

struct PlainSmem {
    double ah[BK][BM + 1], al[BK][BM + 1];  // op(A) panel, [l][i]
    double bh[BK][BN + 1], bl[BK][BN + 1];  // op(B) panel, [l][j]
};

constexpr int GROUP_N = 8;  // tile columns per rasterisation group

// Tile (bi, bj) of this CTA.  Rgemm: a 1-D grid walked in groups of GROUP_N
// tile columns with the tile row fastest inside a group, so the CTAs
// resident at one time share a few A row panels and B column panels in L2
// (a plain column-by-column order re-reads all of A for every tile column).
// Rsyrk: a 1-D grid over the tiles of one triangle, t -> (row, col) with
// row <= col (upper) or row >= col (lower).
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

template <int TA, int TB>
__global__ void __launch_bounds__(NT) dd_gemm_plain_kernel(const GemmArgs p) {
    __shared__ PlainSmem s;
    if (p.info != nullptr && *p.info != 0) return;  // an earlier step failed
    int64_t bi, bj;
    tile_coords(p, bi, bj);
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    const int64_t i0 = bi * BM, j0 = bj * BN;
    const int64_t kk = p.alpha_zero ? 0 : p.k;

    dd acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = dd{0.0, 0.0};

    double rah[4], ral[4], rbh[4], rbl[4];
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
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int ii, ll;
            a_pos(q, ii, ll);
            int64_t gi = i0 + ii, gl = l0 + ll;
            bool ok = gi < p.m && gl < kk;
            int64_t off = TA ? (gl + gi * p.lda) : (gi + gl * p.lda);
            rah[q] = ok ? p.ah[off] : 0.0;
            ral[q] = ok ? p.al[off] : 0.0;
            int jj;
            b_pos(q, jj, ll);
            int64_t gj = j0 + jj;
            gl = l0 + ll;
            ok = gj < p.n && gl < kk;
            off = TB ? (gj + gl * p.ldb) : (gl + gj * p.ldb);
            rbh[q] = ok ? p.bh[off] : 0.0;
            rbl[q] = ok ? p.bl[off] : 0.0;
        }
    };
    auto stage = [&]() {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
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
                    dd a[4], b[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        a[r] = dd{s.ah[l][tx + 16 * r], s.al[l][tx + 16 * r]};
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        b[c] = dd{s.bh[l][ty + 16 * c], s.bl[l][ty + 16 * c]};
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) mac_deferred(acc[r][c], a[r], b[c]);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) renorm(acc[r][c]);
            }
        }
    }

    const dd alpha{p.alpha.hi, p.alpha.lo}, beta{p.beta.hi, p.beta.lo};
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
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

}  // namespace

int launch_gemm_plain(const GemmArgs &p, cudaStream_t stream) {
    dim3 block(NT);
    dim3 grid;
    int64_t tm = ceil_div(p.m, BM), tn = ceil_div(p.n, BN);
    if (p.tri == 0) {
        if (tm * tn > 0x7fffffffLL) return fail(MP_DD_ERR_TOO_LARGE, "m x n too large");
        grid = dim3((unsigned)(tm * tn));
    } else {
        int64_t tiles = tm * (tm + 1) / 2;
        if (tiles > 0x7fffffffLL) return fail(MP_DD_ERR_TOO_LARGE, "n too large");
        grid = dim3((unsigned)tiles);
    }
    if (p.ta == 0 && p.tb == 0) dd_gemm_plain_kernel<0, 0><<<grid, block, 0, stream>>>(p);
    else if (p.ta == 1 && p.tb == 0) dd_gemm_plain_kernel<1, 0><<<grid, block, 0, stream>>>(p);
    else if (p.ta == 0 && p.tb == 1) dd_gemm_plain_kernel<0, 1><<<grid, block, 0, stream>>>(p);
    else dd_gemm_plain_kernel<1, 1><<<grid, block, 0, stream>>>(p);
    return check_launch("dd_gemm_plain_kernel");
}

}  // namespace mpdd
