// Grouped dd Rgemm: thousands of independent, uneven problems in one
// persistent kernel launch.
//
// Host side (mp_dd_Rgemm_grouped_prepare): every descriptor is checked with
// the DGEMM rules, split into output tiles of its tile shape, and the tiles
// of all problems are put in one list ordered by decreasing cost (k times
// the tile area: longest-processing-time first).  The descriptors and the
// tile list go to the caller's device workspace.
//
// Device side (mp_dd_Rgemm_grouped_run): one launch of a persistent kernel,
// one CTA per SM slot; CTAs take tiles from the list through an atomic
// counter and run the same dd multiply-add as the plain kernel (TwoProd by
// FMA, TwoSum, renormalisation every 4 steps; l = 0 .. k-1 in order), so every entry is
// bitwise equal to what mp_dd_Rgemm produces for that problem alone,
// whatever tile shape it was computed with.  run only enqueues a memset of
// the counter and the kernel, so it can be captured in a CUDA graph.
//
// Tile shapes: 16*RM x 16*RN with (RM, RN) in {(2,2), (4,2), (2,4), (1,1)};
// the 256 threads form a 16 x 16 grid and each holds an RM x RN block of dd
// accumulators.  Small shapes waste fewer zero-padded multiply-adds on
// ragged problems (each costs the full 12.75 FP64 instructions); larger ones
// give each thread more independent chains.  All shapes fit 128 registers,
// so two CTAs share an SM.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "dd_arith.cuh"
#include "kernels.cuh"

namespace mpdd {
namespace {

constexpr int NT = 256, BK = 16, MAXB = 64;

struct TileRef {
    int32_t problem, bi, bj, shape;
};

// Workspace layout: [header, 256 B] [descriptors] [tile list].  The kernel
// reads everything it needs from the workspace, so a run needs only its
// address.
struct GroupedHeader {
    unsigned long long counter;  // next tile to hand out (reset by every run)
    long long num_tiles;
    long long count;
    long long tiles_offset;      // byte offset of the tile list
};

struct GroupedSmem {
    double ah[BK][MAXB + 1], al[BK][MAXB + 1];
    double bh[BK][MAXB + 1], bl[BK][MAXB + 1];
};

// Shape id -> (RM, RN): 0 = 2x2 (32x32), 1 = 4x2 (64x32), 2 = 2x4 (32x64),
// 3 = 1x1 (16x16).
__host__ __device__ inline void shape_dims(int s, int &rm, int &rn) {
    rm = s == 1 ? 4 : s == 3 ? 1 : 2;
    rn = s == 2 ? 4 : s == 3 ? 1 : 2;
}

template <int RM, int RN>
__device__ __forceinline__ void dd_tile(const mp_dd_gemm_desc &d, int64_t bi, int64_t bj,
                                        GroupedSmem &s) {
    constexpr int BM = 16 * RM, BN = 16 * RN;
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    const int64_t i0 = bi * BM, j0 = bj * BN;
    if (d.info != nullptr && *d.info != 0) return;   // the problem's owner failed earlier
    const bool alpha_zero = (d.alpha.hi == 0.0 && d.alpha.lo == 0.0) || d.k == 0;
    const int64_t kk = alpha_zero ? 0 : d.k;
    const int ta = d.transa, tb = d.transb;

    dd acc[RM][RN];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < RN; ++c) acc[r][c] = dd{0.0, 0.0};

    double rah[RM], ral[RM], rbh[RN], rbl[RN];
    // A panel: BM x BK = 256 * RM elements, RM per thread; B panel: RN per thread.
    auto a_pos = [&](int q, int &ii, int &ll) {
        int idx = t + NT * q;
        if (!ta) { ii = idx % BM; ll = idx / BM; }
        else     { ll = idx % BK; ii = idx / BK; }
    };
    auto b_pos = [&](int q, int &jj, int &ll) {
        int idx = t + NT * q;
        if (!tb) { ll = idx % BK; jj = idx / BK; }
        else     { jj = idx % BN; ll = idx / BN; }
    };
    auto load = [&](int64_t l0) {
#pragma unroll
        for (int q = 0; q < RM; ++q) {
            int ii, ll;
            a_pos(q, ii, ll);
            int64_t gi = i0 + ii, gl = l0 + ll;
            bool ok = gi < d.m && gl < kk;
            int64_t off = ta ? (gl + gi * d.lda) : (gi + gl * d.lda);
            rah[q] = ok ? d.a_hi[off] : 0.0;
            ral[q] = ok ? d.a_lo[off] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < RN; ++q) {
            int jj, ll;
            b_pos(q, jj, ll);
            int64_t gj = j0 + jj, gl = l0 + ll;
            bool ok = gj < d.n && gl < kk;
            int64_t off = tb ? (gj + gl * d.ldb) : (gl + gj * d.ldb);
            rbh[q] = ok ? d.b_hi[off] : 0.0;
            rbl[q] = ok ? d.b_lo[off] : 0.0;
        }
    };
    auto stage = [&]() {
#pragma unroll
        for (int q = 0; q < RM; ++q) {
            int ii, ll;
            a_pos(q, ii, ll);
            s.ah[ll][ii] = rah[q];
            s.al[ll][ii] = ral[q];
        }
#pragma unroll
        for (int q = 0; q < RN; ++q) {
            int jj, ll;
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
            // the groups of 4 steps wholly past k only add zero products and
            // renormalise an already normalised sum: skipping them changes
            // no bit
            const int64_t left = kk - l0;
            const int lend = left >= BK ? BK
                                        : (int)((left + kRenormEvery - 1) / kRenormEvery) *
                                              kRenormEvery;
#pragma unroll 1
            for (int l4 = 0; l4 < lend; l4 += kRenormEvery) {
#pragma unroll
                for (int l = l4; l < l4 + kRenormEvery; ++l) {
                    dd a[RM], b[RN];
#pragma unroll
                    for (int r = 0; r < RM; ++r)
                        a[r] = dd{s.ah[l][tx + 16 * r], s.al[l][tx + 16 * r]};
#pragma unroll
                    for (int c = 0; c < RN; ++c)
                        b[c] = dd{s.bh[l][ty + 16 * c], s.bl[l][ty + 16 * c]};
#pragma unroll
                    for (int r = 0; r < RM; ++r)
#pragma unroll
                        for (int c = 0; c < RN; ++c) mac_deferred(acc[r][c], a[r], b[c]);
                }
#pragma unroll
                for (int r = 0; r < RM; ++r)
#pragma unroll
                    for (int c = 0; c < RN; ++c) renorm(acc[r][c]);
            }
        }
    }

    const dd alpha{d.alpha.hi, d.alpha.lo}, beta{d.beta.hi, d.beta.lo};
    const bool alpha_one = d.alpha.hi == 1.0 && d.alpha.lo == 0.0;
    const bool beta_zero = d.beta.hi == 0.0 && d.beta.lo == 0.0;
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < RN; ++c) {
            int64_t i = i0 + tx + 16 * r, j = j0 + ty + 16 * c;
            if (i >= d.m || j >= d.n) continue;
            if ((d.uplo == 1 && i > j) || (d.uplo == 2 && i < j)) continue;
            dd v = alpha_one ? acc[r][c] : mul(alpha, acc[r][c]);
            int64_t off = i + j * d.ldc;
            if (!beta_zero) v = add(v, mul(beta, dd{d.c_hi[off], d.c_lo[off]}));
            d.c_hi[off] = v.hi;
            d.c_lo[off] = v.lo;
        }
    __syncthreads();  // the shared panels are reused by the next tile
}

__global__ void __launch_bounds__(NT, 2) grouped_gemm_kernel(uint8_t *ws) {
    __shared__ GroupedSmem s;
    __shared__ long long next;
    GroupedHeader *h = reinterpret_cast<GroupedHeader *>(ws);
    const long long num_tiles = h->num_tiles;
    const mp_dd_gemm_desc *descs = reinterpret_cast<const mp_dd_gemm_desc *>(ws + 256);
    const TileRef *tiles = reinterpret_cast<const TileRef *>(ws + h->tiles_offset);
    while (true) {
        if (threadIdx.x == 0) next = (long long)atomicAdd(&h->counter, 1ull);
        __syncthreads();
        const long long t = next;
        __syncthreads();
        if (t >= num_tiles) break;
        const TileRef tr = tiles[t];
        const mp_dd_gemm_desc &d = descs[tr.problem];
        switch (tr.shape) {
            case 0: dd_tile<2, 2>(d, tr.bi, tr.bj, s); break;
            case 1: dd_tile<4, 2>(d, tr.bi, tr.bj, s); break;
            case 2: dd_tile<2, 4>(d, tr.bi, tr.bj, s); break;
            default: dd_tile<1, 1>(d, tr.bi, tr.bj, s); break;
        }
    }
}

size_t desc_offset() { return 256; }
size_t tiles_offset(int64_t count) {
    return (desc_offset() + sizeof(mp_dd_gemm_desc) * (size_t)count + 255) / 256 * 256;
}

// Whether tile (bi, bj) of shape (bm x bn) holds any entry of the stored
// triangle of a triangular (uplo != 0) problem.
bool tile_in_triangle(int uplo, int64_t bi, int64_t bj, int bm, int bn) {
    if (uplo == 1) return bi * bm <= (bj + 1) * bn - 1;   // some i <= j
    if (uplo == 2) return (bi + 1) * bm - 1 >= bj * bn;   // some i >= j
    return true;
}

int64_t tiles_of(const mp_dd_gemm_desc &d, int shape) {
    int rm, rn;
    shape_dims(shape, rm, rn);
    if (d.m == 0 || d.n == 0) return 0;
    const int64_t tm = ceil_div(d.m, 16 * rm), tn = ceil_div(d.n, 16 * rn);
    if (d.uplo == 0) return tm * tn;
    int64_t c = 0;
    for (int64_t bj = 0; bj < tn; ++bj)
        for (int64_t bi = 0; bi < tm; ++bi) c += tile_in_triangle(d.uplo, bi, bj, 16 * rm, 16 * rn);
    return c;
}

// Default shape when a descriptor leaves it to the library (tile < 0): the
// least padded work divided by a per-shape efficiency (independent
// accumulator chains per thread: 1 for 16x16 runs the FP64 pipe at roughly
// half rate).  An autotuned table replaces this per size class.
int default_shape(const mp_dd_gemm_desc &d) {
    static const double eff[4] = {0.92, 1.0, 1.0, 0.5};
    int best = 0;
    double best_cost = -1.0;
    for (int s = 0; s < 4; ++s) {
        int rm, rn;
        shape_dims(s, rm, rn);
        double area = (double)(ceil_div(d.m, 16 * rm) * 16 * rm) *
                      (double)(ceil_div(d.n, 16 * rn) * 16 * rn);
        double cost = area / eff[s];
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = s;
        }
    }
    return best;
}

int check_desc(const mp_dd_gemm_desc &d, int64_t idx) {
    if (d.transa < 0 || d.transa > 1 || d.transb < 0 || d.transb > 1)
        return fail(-2, "grouped: descriptor %lld: trans flags must be 0 or 1", (long long)idx);
    if (d.m < 0 || d.n < 0 || d.k < 0)
        return fail(-2, "grouped: descriptor %lld: negative size", (long long)idx);
    int64_t nrowa = d.transa ? d.k : d.m, nrowb = d.transb ? d.n : d.k;
    if (d.lda < imax(1, nrowa) || d.ldb < imax(1, nrowb) || d.ldc < imax(1, d.m))
        return fail(-2, "grouped: descriptor %lld: leading dimension too small", (long long)idx);
    if (d.tile > 3) return fail(-2, "grouped: descriptor %lld: tile shape %d", (long long)idx,
                                d.tile);
    if (d.uplo < 0 || d.uplo > 2 || (d.uplo != 0 && d.m != d.n))
        return fail(-2, "grouped: descriptor %lld: uplo needs 0..2 and m == n", (long long)idx);
    bool need_ab = d.m > 0 && d.n > 0 && d.k > 0 && !(d.alpha.hi == 0.0 && d.alpha.lo == 0.0);
    if (need_ab && (!d.a_hi || !d.a_lo || !d.b_hi || !d.b_lo))
        return fail(-2, "grouped: descriptor %lld: NULL operand", (long long)idx);
    if (d.m > 0 && d.n > 0 && (!d.c_hi || !d.c_lo))
        return fail(-2, "grouped: descriptor %lld: NULL C", (long long)idx);
    return 0;
}

// BLAS quick return for one problem: no tiles.
bool desc_is_noop(const mp_dd_gemm_desc &d) {
    if (d.m == 0 || d.n == 0) return true;
    bool az = (d.alpha.hi == 0.0 && d.alpha.lo == 0.0) || d.k == 0;
    return az && d.beta.hi == 1.0 && d.beta.lo == 0.0;
}

}  // namespace

size_t grouped_workspace_bytes(int64_t count, const mp_dd_gemm_desc *descs) {
    int64_t tiles = 0;
    for (int64_t i = 0; i < count; ++i) {
        if (desc_is_noop(descs[i])) continue;
        int s = descs[i].tile < 0 ? default_shape(descs[i]) : descs[i].tile;
        if (s > 3) s = 3;
        tiles += tiles_of(descs[i], s);
    }
    return tiles_offset(count) + sizeof(TileRef) * (size_t)(tiles > 0 ? tiles : 1);
}

namespace {

// Pinned staging blocks for the uploads of grouped_prepare: the image of the
// workspace head (header, descriptors, tile list) is written into a block
// and copied with one asynchronous cudaMemcpyAsync; an event recorded after
// the copy marks when the block may be written again.  Blocks are kept for
// reuse, so steady-state calls neither allocate nor wait for the GPU.
struct StageBlock {
    void *ptr = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
};

std::mutex g_stage_mu;
std::vector<StageBlock> g_stage;

int stage_upload(void *dst, const void *src, size_t bytes, cudaStream_t st) {
    std::lock_guard<std::mutex> lock(g_stage_mu);
    StageBlock *blk = nullptr;
    for (auto &b : g_stage)
        if (b.cap >= bytes && cudaEventQuery(b.done) == cudaSuccess) {
            blk = &b;
            break;
        }
    cudaGetLastError();   // a not-ready query leaves an error state to clear
    if (blk == nullptr) {
        StageBlock nb;
        nb.cap = 64 * 1024;
        while (nb.cap < bytes) nb.cap *= 2;
        cudaError_t e = cudaHostAlloc(&nb.ptr, nb.cap, cudaHostAllocDefault);
        if (e != cudaSuccess) return cuda_fail(e, "grouped: pinned staging");
        e = cudaEventCreateWithFlags(&nb.done, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "grouped: staging event");
        g_stage.push_back(nb);
        blk = &g_stage.back();
    }
    std::memcpy(blk->ptr, src, bytes);
    cudaError_t e = cudaMemcpyAsync(dst, blk->ptr, bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(blk->done, st);
    return e == cudaSuccess ? 0 : cuda_fail(e, "grouped: upload");
}

}  // namespace

int grouped_prepare(int64_t count, const mp_dd_gemm_desc *descs, void *ws, size_t bytes,
                    cudaStream_t st) {
    std::vector<mp_dd_gemm_desc> dv(descs, descs + count);
    std::vector<TileRef> tiles;
    std::vector<double> cost;
    for (int64_t i = 0; i < count; ++i) {
        int rc = check_desc(dv[i], i);
        if (rc) return rc;
        if (desc_is_noop(dv[i])) continue;
        int s = dv[i].tile < 0 ? default_shape(dv[i]) : dv[i].tile;
        dv[i].tile = s;
        int rm, rn;
        shape_dims(s, rm, rn);
        int64_t tm = ceil_div(dv[i].m, 16 * rm), tn = ceil_div(dv[i].n, 16 * rn);
        if (tm > 0x7fffffffLL || tn > 0x7fffffffLL || i > 0x7fffffffLL)
            return fail(MP_DD_ERR_TOO_LARGE, "grouped: problem %lld too large", (long long)i);
        for (int64_t bj = 0; bj < tn; ++bj)
            for (int64_t bi = 0; bi < tm; ++bi)
                if (tile_in_triangle(dv[i].uplo, bi, bj, 16 * rm, 16 * rn))
                    tiles.push_back(TileRef{(int32_t)i, (int32_t)bi, (int32_t)bj, s});
    }
    const size_t need = tiles_offset(count) + sizeof(TileRef) * (tiles.empty() ? 1 : tiles.size());
    if (ws == nullptr) return fail(-3, "grouped: workspace is NULL");
    if (bytes < need)
        return fail(MP_DD_ERR_WORKSPACE, "grouped: workspace needs %zu bytes, got %zu", need,
                    bytes);
    // longest tiles first (k * tile area), stable so the order is reproducible
    std::vector<int64_t> order(tiles.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = (int64_t)q;
    auto tile_cost = [&](const TileRef &t) {
        int rm, rn;
        shape_dims(t.shape, rm, rn);
        return (double)dv[t.problem].k * rm * rn;
    };
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        return tile_cost(tiles[a]) > tile_cost(tiles[b]);
    });
    std::vector<TileRef> sorted(tiles.size());
    for (size_t q = 0; q < order.size(); ++q) sorted[q] = tiles[order[q]];
    GroupedHeader h{0ull, (long long)sorted.size(), (long long)count,
                    (long long)tiles_offset(count)};
    // one image of header, descriptors and tile list, uploaded asynchronously
    const size_t img = tiles_offset(count) + sizeof(TileRef) * sorted.size();
    std::vector<uint8_t> image(img, 0);
    std::memcpy(image.data(), &h, sizeof(h));
    if (count > 0)
        std::memcpy(image.data() + desc_offset(), dv.data(), sizeof(mp_dd_gemm_desc) * count);
    if (!sorted.empty())
        std::memcpy(image.data() + tiles_offset(count), sorted.data(),
                    sizeof(TileRef) * sorted.size());
    return stage_upload(ws, image.data(), img, st);
}

int grouped_run(void *ws, cudaStream_t st) {
    uint8_t *w = static_cast<uint8_t *>(ws);
    cudaError_t e = cudaMemsetAsync(w, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "grouped: counter reset");
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grouped_gemm_kernel, NT, 0);
        if (per_sm < 1) per_sm = 1;
    }
    grouped_gemm_kernel<<<(unsigned)(sm_count() * per_sm), NT, 0, st>>>(w);
    return check_launch("grouped_gemm_kernel");
}

}  // namespace mpdd
