// Plain double-double Rgemm / Rsyrk with TMA-staged operand panels (sm_103a).
//
// The same computation as dd_gemm_plain.cu -- C := alpha op(A) op(B) + beta C,
// or one triangle of it for Rsyrk, every multiply-add the dd multiply-add of
// dd_arith.cuh with the renormalisation every 4 steps of k, l = 0 .. k-1 in
// order -- with the operand panels moved by the tensor memory accelerator:
//
//  * one CTA per 64 x 64 output tile (the plain kernel's tile order: groups
//    of 8 tile columns, or the triangle), one CTA per SM at a time, so the
//    hardware hands the next tile to whichever SM finishes first;
//  * one producer warp issues, for every 16-wide panel of k, four 2-D tile
//    copies (cp.async.bulk.tensor: the hi and lo planes of op(A) and op(B),
//    64 x 16 binary64 each) into a ring of kStages stages, completing the
//    stage's mbarrier, up to kStages panels ahead of the consumers;
//  * eight consumer warps (the plain kernel's 16 x 16 thread layout, a 4 x 4
//    block of dd accumulators per thread) wait on a stage's full barrier,
//    run its 16 steps of k, and release it through its empty barrier; no
//    block-wide barrier is left in the loop;
//  * elements outside the matrices are filled with zeros by the copy, and a
//    zero product leaves a normalised accumulator unchanged, so every entry's
//    operation sequence, and hence its bits, equal the register-staged
//    kernel's.
//
// Shared-memory layouts: a panel that is contiguous along the tile's row
// (or column) index lands as [l][i] without swizzle; a panel contiguous
// along k lands as [i][l], 128 bytes per row, with the 128-byte swizzle
// (16-byte chunk c of row i stored at chunk c ^ (i mod 8)), so the 16
// consumer rows of a warp read 8 distinct bank groups.
//
// Every wait is bounded (sm100.cuh): a wait that runs out sets the CTA's
// abort flag, every role leaves its loop, and the producer lets its copies
// in flight land before the CTA exits (C is then incomplete).
#include <cuda.h>

#include <atomic>
#include <mutex>

#include "common.cuh"
#include "dd_arith.cuh"
#include "kernels.cuh"
#include "ozaki_common.cuh"
#include "sm100.cuh"

namespace mpdd {
namespace {

using namespace sm100;

constexpr int kTile = 64, kBK = 16, kStages = 4;
constexpr int kConsumerWarps = 8, kThreads = 32 * (kConsumerWarps + 1);
constexpr uint32_t kPanelBytes = kTile * kBK * 8;          // 8 KB: one plane of one operand
constexpr uint32_t kStageBytes = 4 * kPanelBytes;          // A hi, A lo, B hi, B lo
constexpr size_t kSmem = (size_t)kStages * kStageBytes + 1024 + 256;
constexpr int kGroupN = 8;                                 // tile columns per group

struct TmaGemmArgs {
    GemmArgs p;
    int64_t tiles_m, tiles_n, tiles;
    int64_t tile_stride;   // tiles a CTA steps over (the grid size)
    int kb_count;
};

// Byte offset of element (row, l) of a panel: [l][row] (row-contiguous
// panels) or the swizzled [row][l] (k-contiguous panels).
template <bool KCONTIG>
__device__ __forceinline__ uint32_t panel_off(int row, int l) {
    if (KCONTIG)
        return (uint32_t)(row * 128 + ((((l >> 1) ^ (row & 7))) << 4) + ((l & 1) << 3));
    return (uint32_t)((l * kTile + row) << 3);
}

__device__ __forceinline__ void tile_of(const TmaGemmArgs &a, int64_t t, int64_t &bi,
                                        int64_t &bj) {
    if (a.p.tri == 0) {
        const int64_t group = t / (a.tiles_m * kGroupN);
        const int64_t first = group * kGroupN;
        const int64_t gn = a.tiles_n - first < kGroupN ? a.tiles_n - first : kGroupN;
        const int64_t local = t - group * a.tiles_m * kGroupN;
        bj = first + local % gn;
        bi = local / gn;
        return;
    }
    int64_t r = (int64_t)((__dsqrt_rn(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    const int64_t c = t - r * (r + 1) / 2;
    if (a.p.tri == 1) {
        bi = c;
        bj = r;
    } else {
        bi = r;
        bj = c;
    }
}

// TA / TB: op(A) = A^T / op(B) = B^T.  op(A) panels are k-contiguous when
// TA, op(B) panels when !TB.
template <int TA, int TB>
__global__ void __launch_bounds__(kThreads, 1)
    dd_gemm_tma_kernel(const __grid_constant__ CUtensorMap tAh,
                       const __grid_constant__ CUtensorMap tAl,
                       const __grid_constant__ CUtensorMap tBh,
                       const __grid_constant__ CUtensorMap tBl, const TmaGemmArgs a) {
    const GemmArgs &p = a.p;
    if (p.info != nullptr && *p.info != 0) return;   // an earlier step failed
    if (p.gate != nullptr &&
        *reinterpret_cast<const volatile unsigned int *>(p.gate) >= p.gate_below)
        return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    uint64_t *empty = full + kStages;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + kStages);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();

    if (warp == kConsumerWarps) {
        // ---------------- producer: one elected lane issues the tile copies
        if (lane == 0) {
            prefetch_tmap(&tAh);
            prefetch_tmap(&tAl);
            prefetch_tmap(&tBh);
            prefetch_tmap(&tBl);
            uint32_t it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < a.tiles && ok; t += a.tile_stride) {
                int64_t bi, bj;
                tile_of(a, t, bi, bj);
                const int i0 = (int)(bi * kTile), j0 = (int)(bj * kTile);
                for (int kb = 0; kb < a.kb_count; ++kb, ++it) {
                    const int s = (int)(it % kStages);
                    const uint32_t f = it / kStages;
                    // a stage is consumed in ~200 us (16 steps of k on the FP64
                    // pipe) and the ring runs kStages ahead: poll its release
                    // every 8 us, keeping the shared-memory pipe (which the
                    // consumers' FP64 instructions queue behind) nearly idle
                    if (it >= (uint32_t)kStages &&
                        !mbar_wait_sleep(&empty[s], (f & 1) ^ 1, abort_flag, 8000)) {
                        ok = false;
                        break;
                    }
                    uint8_t *st = smem + (size_t)s * kStageBytes;
                    mbar_arrive_expect_tx(&full[s], kStageBytes);
                    const int l0 = kb * kBK;
                    // coordinates are (innermost, outer): (row, l) or (l, row)
                    if (TA) {
                        tma_load_2d(st, &tAh, &full[s], l0, i0);
                        tma_load_2d(st + kPanelBytes, &tAl, &full[s], l0, i0);
                    } else {
                        tma_load_2d(st, &tAh, &full[s], i0, l0);
                        tma_load_2d(st + kPanelBytes, &tAl, &full[s], i0, l0);
                    }
                    if (!TB) {
                        tma_load_2d(st + 2 * kPanelBytes, &tBh, &full[s], l0, j0);
                        tma_load_2d(st + 3 * kPanelBytes, &tBl, &full[s], l0, j0);
                    } else {
                        tma_load_2d(st + 2 * kPanelBytes, &tBh, &full[s], j0, l0);
                        tma_load_2d(st + 3 * kPanelBytes, &tBl, &full[s], j0, l0);
                    }
                }
            }
            if (!ok) {
                // let the copies already issued land before the CTA exits
                const uint32_t first = it > (uint32_t)kStages ? it - kStages : 0;
                for (uint32_t j = first; j < it; ++j) {
                    const long long t0 = clock64();
                    while (!mbar_try_wait(&full[j % kStages], (j / kStages) & 1) &&
                           clock64() - t0 < kWaitCycles / 4) {
                    }
                }
            }
        }
        __syncwarp();
        return;
    }

    // ---------------- consumers
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    const dd alpha{p.alpha.hi, p.alpha.lo}, beta{p.beta.hi, p.beta.lo};
    uint32_t it = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < a.tiles && ok; tile += a.tile_stride) {
        int64_t bi, bj;
        tile_of(a, tile, bi, bj);
        dd acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = dd{0.0, 0.0};
        for (int kb = 0; kb < a.kb_count; ++kb, ++it) {
            const int s = (int)(it % kStages);
            if (!mbar_wait(&full[s], (it / kStages) & 1, abort_flag)) {
                ok = false;
                break;
            }
            const uint8_t *st = smem + (size_t)s * kStageBytes;
            const uint8_t *sah = st, *sal = st + kPanelBytes;
            const uint8_t *sbh = st + 2 * kPanelBytes, *sbl = st + 3 * kPanelBytes;
#pragma unroll 1
            for (int l4 = 0; l4 < kBK; l4 += kRenormEvery) {
#pragma unroll
                for (int l = l4; l < l4 + kRenormEvery; ++l) {
                    dd av[4], bv[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const uint32_t o = panel_off<TA != 0>(tx + 16 * r, l);
                        av[r] = dd{*reinterpret_cast<const double *>(sah + o),
                                   *reinterpret_cast<const double *>(sal + o)};
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint32_t o = panel_off<TB == 0>(ty + 16 * c, l);
                        bv[c] = dd{*reinterpret_cast<const double *>(sbh + o),
                                   *reinterpret_cast<const double *>(sbl + o)};
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) mac_deferred(acc[r][c], av[r], bv[c]);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) renorm(acc[r][c]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        if (!ok) break;
        // epilogue: the plain kernel's, entry by entry
        const int64_t i0 = bi * kTile, j0 = bj * kTile;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t i = i0 + tx + 16 * r, j = j0 + ty + 16 * c;
                if (i >= p.m || j >= p.n) continue;
                if ((p.tri == 1 && i > j) || (p.tri == 2 && i < j)) continue;
                dd v = p.alpha_one ? acc[r][c] : mul(alpha, acc[r][c]);
                const int64_t off = i + j * p.ldc;
                if (!p.beta_zero) v = add(v, mul(beta, dd{p.ch[off], p.cl[off]}));
                p.ch[off] = v.hi;
                p.cl[off] = v.lo;
            }
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *q = nullptr;
        cudaDriverEntryPointQueryResult r;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000,
                                             cudaEnableDefault, &r) == cudaSuccess &&
            r == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(q);
    });
    return fn;
}

// Tensor map of a column-major binary64 plane (rows x cols, leading dimension
// ld) whose box is 64 rows x 16 columns (inner = rows: the rows are the
// tile's row or column index) or 16 rows x 64 columns (inner = rows = k,
// with the 128-byte swizzle).
int plane_map(CUtensorMap *m, const double *base, int64_t rows, int64_t cols, int64_t ld,
              bool inner_is_k) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return fail(MP_DD_ERR_NO_DEVICE, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
    cuuint32_t box[2] = {inner_is_k ? (cuuint32_t)kBK : (cuuint32_t)kTile,
                         inner_is_k ? (cuuint32_t)kTile : (cuuint32_t)kBK};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(base), dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    inner_is_k ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(MP_DD_ERR_NO_DEVICE, "cuTensorMapEncodeTiled (plain panels): CUresult %d",
                    (int)r);
    return 0;
}

template <int TA, int TB>
int launch_t(const CUtensorMap (&m)[4], const TmaGemmArgs &a, int grid, cudaStream_t st) {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(dd_gemm_tma_kernel<TA, TB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    });
    dd_gemm_tma_kernel<TA, TB><<<grid, kThreads, kSmem, st>>>(m[0], m[1], m[2], m[3], a);
    return check_launch("dd_gemm_tma_kernel");
}

std::atomic<int> g_staging{0};   // 0 automatic, 1 registers only, 2 TMA where it applies

bool aligned16(const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

}  // namespace

void set_plain_staging(int mode) { g_staging.store(mode); }
int plain_staging() { return g_staging.load(); }

// The TMA-staged kernel applies to plain Rgemm / Rsyrk products (no second
// product, no symmetric operand, alpha != 0) whose planes start on 16-byte
// boundaries with even leading dimensions (the copy engine's stride rule).
// Automatically it takes the Rgemm products large enough for 64 x 64 tiles
// (measured on GB300: 85.8 dd-GFlop/s at 4096, as the register-staged
// kernel; at 2048 and for the Rsyrk triangle the smaller register-staged
// tiles are faster).  Returns 1 when it launched (or failed to: *rc), 0 when
// the caller should use the register-staged kernels.
int try_launch_gemm_tma(const GemmArgs &p, cudaStream_t st, int *rc) {
    if (g_staging.load() == 1) return 0;
    if (p.a2h != nullptr || p.sym_a || p.sym_b || p.alpha_zero || p.k <= 0) return 0;
    if (p.m <= 0 || p.n <= 0) return 0;
    if (!aligned16(p.ah) || !aligned16(p.al) || !aligned16(p.bh) || !aligned16(p.bl))
        return 0;
    if ((p.lda & 1) || (p.ldb & 1)) return 0;
    const int64_t tm = ceil_div(p.m, kTile), tn = ceil_div(p.n, kTile);
    const int64_t tiles = p.tri == 0 ? tm * tn : tm * (tm + 1) / 2;
    const int sms = sm_count() > 0 ? sm_count() : 152;
    if (g_staging.load() == 0) {
        // automatic: Rgemm products whose 64 x 64 tiling is within 1 % of the
        // best tile size's busiest-SM time (thinner products and the Rsyrk
        // triangle run faster on the smaller register-staged tiles)
        if (p.tri != 0 || tiles < sms) return 0;
        int64_t best = plain_tile_cost(p, 4);
        for (int r = 2; r >= 1; r /= 2) {
            const int64_t c = plain_tile_cost(p, r);
            best = c < best ? c : best;
        }
        if (100 * plain_tile_cost(p, 4) > 101 * best) return 0;
    }
    if (p.k > ((int64_t)1 << 31) - 1 || p.m > ((int64_t)1 << 31) - 1 ||
        p.n > ((int64_t)1 << 31) - 1)
        return 0;
    // op(A) is m x k: stored m x k (rows = m, contiguous) or k x m (rows = k)
    CUtensorMap maps[4];
    const bool ta = p.ta != 0, tb = p.tb != 0;
    int r;
    if ((r = plane_map(&maps[0], p.ah, ta ? p.k : p.m, ta ? p.m : p.k, p.lda, ta)) ||
        (r = plane_map(&maps[1], p.al, ta ? p.k : p.m, ta ? p.m : p.k, p.lda, ta)) ||
        (r = plane_map(&maps[2], p.bh, tb ? p.n : p.k, tb ? p.k : p.n, p.ldb, !tb)) ||
        (r = plane_map(&maps[3], p.bl, tb ? p.n : p.k, tb ? p.k : p.n, p.ldb, !tb))) {
        *rc = r;
        return 1;
    }
    TmaGemmArgs a{};
    a.p = p;
    a.tiles_m = tm;
    a.tiles_n = tn;
    a.tiles = tiles;
    a.kb_count = (int)ceil_div(p.k, kBK);
    // one CTA per tile while the grid fits a launch, else a grid-stride walk
    const int64_t max_grid = 0x7fffffffLL;
    const int grid = (int)(tiles < max_grid ? tiles : max_grid);
    a.tile_stride = grid;
    if (!ta && !tb) *rc = launch_t<0, 0>(maps, a, grid, st);
    else if (ta && !tb) *rc = launch_t<1, 0>(maps, a, grid, st);
    else if (!ta && tb) *rc = launch_t<0, 1>(maps, a, grid, st);
    else *rc = launch_t<1, 1>(maps, a, grid, st);
    return 1;
}

}  // namespace mpdd
