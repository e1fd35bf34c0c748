// Split-precision dd Rgemm on the fp16 tensor cores (tcgen05, sm_103a).
//
// C := alpha op(A) op(B) + beta C with the products of op(A) op(B) formed
// from error-free integer slices (the Ozaki scheme):
//
//  1. Scaling.  Row i of op(A) gets e_i with max_l |A_il| < 2^(e_i - 1); column
//     j of op(B) gets f_j likewise.  Then |a 2^-e_i| < 1/2 for every entry.
//  2. Slicing.  Each dd entry x = hi + lo of row i becomes the integer
//     X = RNE(hi 2^(8S - e_i)) + RNE(lo 2^(8S - e_i))  (|x 2^(8S-e_i) - X| <= 1)
//     written in balanced base 256: X = sum_{t<S} d_t 256^(S-1-t), with
//     d_t in [-128, 128].  Each digit plane is stored as fp16 (exact) in a
//     K-major [row][k] layout padded to the tile sizes with zeros.
//  3. Band products.  For b = 0 .. S-1 the exact integer matrix
//     P_b = sum_{t+u=b} D_A[t] D_B[u]^T is computed on the tensor cores with
//     fp32 accumulation in tensor memory, drained every 1024 products: a
//     run of 1024 products of |d| <= 128 stays within 2^24 in magnitude, so
//     every partial sum is an integer the fp32 accumulator holds exactly
//     (an fp32 addition whose exact sum is representable does not round).  The drained values
//     are summed in int32 registers (|P_b| < 2^31 for k (b+1) 2^14 < 2^31).
//     Pairs with t + u >= S are dropped (triangular truncation).
//  4. Recombination.  V = sum_b P_b 256^(S-1-b) is formed exactly in 192-bit
//     integer arithmetic, rounded once to the nearest dd and scaled by
//     2^(e_i + f_j - 8S - 8); the alpha/beta epilogue is dd arithmetic.
//
// Error: per product |a b - sum_{t+u<S} d_t d'_u 256^-(t+u+2) 2^(e_i+f_j)|
// <= C_S 2^(e_i + f_j - 8S) with C_S = 1 + (S - 1) / (4 (1 - 2^-8)) (one unit
// of operand rounding per factor, and the dropped pairs t + u >= S).  Before
// slicing, every call certifies this against the bound
// 4 k 2^-104 (|alpha||A||B| + |beta||C|) entry by entry (ozaki_common.cuh):
// a bf16 tensor-core product of the magnitude planes gives a lower bound of
// |A||B|, the smallest margin picks S (14 or 15 when the caller passes 0,
// else the caller's S), and when no S certifies the bound the plain FP64
// kernel computes C instead.
//
// Only the scaling epilogue uses the FP64 pipe (about 30 instructions per
// output entry); slicing and recombination are integer arithmetic, and the
// O(mnk) work runs on the tensor cores.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <limits>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "dd_arith.cuh"
#include "kernels.cuh"
#include "ozaki_common.cuh"
#include "sm100.cuh"

namespace mpdd {
namespace {

using namespace sm100;

constexpr int TM = 128, TK = 64;            // tile rows and k-block
constexpr int CHUNK_KB = 16;                // k-blocks per exact fp32 run (1024 products)
// The magnitude product needs no exact runs (its fp32 sums only have to stay
// within the certificate's safety factor): one run over the whole k.
template <bool MAG>
__host__ __device__ constexpr int chunk_kb() { return MAG ? (1 << 30) : CHUNK_KB; }
// Tile columns per rasterisation group: 8 for full products; 4 for the
// Rsyrk triangle, where the balance of the skipped tiles over the CTAs
// matters more than operand reuse (13 % faster at 8192; 4 and 16 are 1.4 %
// slower than 8 on full products).
constexpr int kGroupFull = 8, kGroupTri = 4;
// Accumulator columns per epilogue thread: 64 on the 128 x 128 tile, 128 on
// the 128 x 256 tile; 8 epilogue warps either way (10 in all, up to 168
// registers), for the residue and magnitude products alike.  On the
// wide tile 8 warps of 128 columns drain faster alongside the MMAs than 16 of
// 64: 1.4 % off the 8192 Rgemm band phase, 3.3 % off the Rsyrk triangle's.
// (Loads of 32 columns at a time spill and measured slower; so did sums
// reduced mod p per run and packed two columns to a word, in 4 or 8 warps:
// the extra arithmetic per drained value slows the MMAs.)
constexpr int kEpiCols = 64;
constexpr int kEpiColsWide = 128;

// Two tile widths: 128 x 128 (6-stage ring of 32 KB, 8 epilogue warps) and
// 128 x 256 (4 stages of 48 KB, 8 epilogue warps, all 512 TMEM columns);
// the wider tile reads 25 % fewer operand bytes per flop.  PAIR: a CTA pair
// on a 256 x 256 tile with the 2-SM MMA, each CTA holding its 128 rows of A
// and 128 of the 256 rows of B: 32 KB per stage and SM, 6 stages.
template <int TN, bool PAIR = false>
struct BandCfg {
    static constexpr int STAGES = PAIR ? 6 : (TN == 256 ? 4 : 6);
    static constexpr int EPI_COLS = TN == 256 ? kEpiColsWide : kEpiCols;
    static constexpr int EPI_WARPS = TN / EPI_COLS * 4;   // 4 lane quadrants
    static constexpr int THREADS = 32 * (2 + EPI_WARPS);  // producer, MMA, epilogue
    static constexpr int TMEM_COLS = 2 * TN;              // two fp32 accumulators
    static constexpr uint32_t A_BYTES = TM * TK * 2, B_BYTES = (PAIR ? TN / 2 : TN) * TK * 2;
    static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
    // stages, 1 KB alignment slack, barriers; SMEM_TRI adds the triangle
    // table (only launches that use it reserve it: the rest keep the L1)
    static constexpr size_t SMEM = STAGES * (size_t)STAGE_BYTES + 1024 + 256;
    static constexpr size_t SMEM_TRI = SMEM + 4 * kTriMax;
};

}  // namespace

// Tile width used for an m x n product: the wide tile once there are enough
// tiles to fill the GPU twice over.
int band_tn(int64_t m, int64_t n) {
    return (ceil_div(m, TM) * ceil_div(n, 256) >= 304) ? 256 : 128;
}

namespace {

// ------------------------------------------------------------------ layout

struct Layout {
    int64_t m, n, k, S, m_pad, n_pad, k_pad;
    size_t off_rowmax, off_colmax, off_da, off_db, off_p, off_ma, off_mb, total;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

Layout make_layout(int64_t m, int64_t n, int64_t k, int S) {
    Layout L{};
    L.m = m; L.n = n; L.k = k; L.S = S;
    const int TN = band_tn(m, n);
    L.m_pad = ceil_div(imax(m, 1), TM) * TM;
    L.n_pad = ceil_div(imax(n, 1), TN) * TN;
    L.k_pad = ceil_div(imax(k, 1), TK) * TK;
    size_t o = 1024;  // header: status word and call parameters
    L.off_rowmax = o; o = align_up(o + 8 * (size_t)L.m_pad, 1024);
    L.off_colmax = o; o = align_up(o + 8 * (size_t)L.n_pad, 1024);
    L.off_da = o; o = align_up(o + 2 * (size_t)S * L.m_pad * L.k_pad, 1024);
    L.off_db = o; o = align_up(o + 2 * (size_t)S * L.n_pad * L.k_pad, 1024);
    L.off_p = o; o = align_up(o + 4 * (size_t)S * L.n_pad * L.m_pad, 1024);
    L.off_ma = o; o = align_up(o + 2 * (size_t)L.m_pad * L.k_pad, 1024);
    L.off_mb = o; o = align_up(o + 2 * (size_t)L.n_pad * L.k_pad, 1024);
    L.total = o;
    return L;
}

// Candidate slice counts of a call: the caller's S, or (slices = 0) 14 and,
// when k 15 stays within the int32 band sums, 15.
int slice_candidates(int slices, int64_t k, int *cand) {
    if (slices != 0) {
        cand[0] = slices;
        return 1;
    }
    cand[0] = kDefaultSlices;
    if ((int64_t)(kDefaultSlices + 1) * k <= ((int64_t)1 << 17) - 1 &&
        kDefaultSlices + 1 <= kMaxSlices) {
        cand[1] = kDefaultSlices + 1;
        return 2;
    }
    return 1;
}

// Per-product error constant of S digit slices: one unit of operand
// rounding plus the dropped pairs, sum_{h >= 0} (S - 1 - h) 2^-2 2^-8h.
double slice_constant(int S) { return 1.0 + 0x1p-50 + (S - 1) / (4.0 * (1.0 - 0x1p-8)); }

// ------------------------------------------------------------------ step 1

// Running maximum of |hi| (as the bit pattern of a non-negative double, which
// orders like the value) over row r of a column-major plane viewed as
// rows x k: element (r, l) at X[r + l*ld] (row_contig) or X[l + r*ld].
__global__ void absmax_kernel(const double *__restrict__ X, int64_t ld, int row_contig,
                              int64_t rows, int64_t k, int64_t lchunk,
                              unsigned long long *__restrict__ out) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int64_t l0 = (int64_t)blockIdx.y * lchunk, l1 = l0 + lchunk < k ? l0 + lchunk : k;
    unsigned long long mx = 0;
    for (int64_t l = l0; l < l1; ++l) {
        double v = row_contig ? X[r + l * ld] : X[l + r * ld];
        unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
        mx = b > mx ? b : mx;
    }
    if (mx) atomicMax(out + r, mx);
}

// Digits of 8 consecutive entries (l0 .. l0+7) of one row, written as S
// planes of 8 fp16 values (16 bytes each).
template <int S>
__device__ __forceinline__ void slice8(const double *__restrict__ Xh,
                                       const double *__restrict__ Xl, int64_t ld, int row_contig,
                                       int64_t r, int64_t rows, int64_t l0, int64_t k, int shift,
                                       __half *__restrict__ D, int64_t rows_pad, int64_t k_pad) {
    __half2 out[S][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        int dg[2][S];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int64_t l = l0 + e + h;
            double hi = 0.0, lo = 0.0;
            if (r < rows && l < k) {
                int64_t off = row_contig ? (r + l * ld) : (l + r * ld);
                hi = Xh[off];
                lo = Xl[off];
            }
            dd_digits<S>(hi, lo, shift, dg[h]);
        }
        // fp16 of a digit d in [-128, 128] without a conversion instruction:
        // the fp16 with bits 0x6600 + d is exactly 1536 + d (binade
        // [1024, 2048), unit spacing), so subtracting 1536 leaves d exactly.
#pragma unroll
        for (int t = 0; t < S; ++t) {
            const uint32_t bits = (uint32_t)(0x6600 + dg[0][t]) |
                                  ((uint32_t)(0x6600 + dg[1][t]) << 16);
            __half2 x;
            memcpy(&x, &bits, 4);
            out[t][e / 2] = __hsub2(x, __floats2half2_rn(1536.0f, 1536.0f));
        }
    }
#pragma unroll
    for (int t = 0; t < S; ++t) {
        uint4 v;
        memcpy(&v, &out[t][0], 16);
        *reinterpret_cast<uint4 *>(D + ((int64_t)t * rows_pad + r) * k_pad + l0) = v;
    }
}

// Two threads per (row, 16 consecutive k): the lane pair (2i, 2i+1) takes row
// i of the block and k halves l0 .. l0+7 and l0+8 .. l0+15, so every 32-byte
// sector of a digit plane is written whole by one store instruction, and the
// row_contig reads of 16 consecutive rows per k column coalesce.
// The slice count comes from the call's certificate (plan): SA or SB digits
// (SA == SB for a caller-chosen S); no certified S: nothing to slice.
template <int SA, int SB>
__global__ void __launch_bounds__(128) slice_kernel(const double *__restrict__ Xh,
                                                    const double *__restrict__ Xl, int64_t ld,
                                                    int row_contig, int64_t rows, int64_t k,
                                                    int64_t rows_pad, int64_t k_pad,
                                                    const unsigned long long *__restrict__ rmax,
                                                    __half *__restrict__ D, const SplitPlan plan) {
    const PlanPick pk = plan_choice(plan);
    if (pk.c < 0) return;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 2) + threadIdx.x / 2;
    if (r >= rows_pad) return;
    const int64_t l0 = (int64_t)blockIdx.y * 16 + 8 * (threadIdx.x & 1);
    const int e = r < rows ? scale_exponent(rmax[r]) : 0;
    if (SA == SB || pk.count == SA)
        slice8<SA>(Xh, Xl, ld, row_contig, r, rows, l0, k, 8 * SA - e, D, rows_pad, k_pad);
    else
        slice8<SB>(Xh, Xl, ld, row_contig, r, rows, l0, k, 8 * SB - e, D, rows_pad, k_pad);
}

// The largest bf16 not above |v| 2^-e, as its bit pattern, for finite v
// with |v| 2^-e < 1/2, from the binary64 fields with integer operations
// only (the FP64 pipe is the slow one): truncate the significand to 8 bits
// (bf16 normal range, exponents >= -126) or to a multiple of 2^-133 (bf16
// subnormals; 0 below).
__device__ __forceinline__ uint16_t bf16_floor_scaled(double v, int e) {
    const unsigned long long u =
        (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    if (u == 0) return 0;
    int E = (int)(u >> 52);
    unsigned long long m = u & ((1ull << 52) - 1);
    if (E == 0) {                               // binary64 subnormal: normalise
        const int sh = __clzll((long long)m) - 11;
        m <<= sh;
        E = 1 - sh;
    } else {
        m |= 1ull << 52;
    }
    const int x = E - 1023 - e;                 // |v| 2^-e = m 2^(x - 52), m in [2^52, 2^53)
    if (x >= -126) return (uint16_t)(((x + 127) << 7) | (int)((m >> 45) & 0x7F));
    const int s = -81 - x;                      // 52 - (x + 133): multiples of 2^-133
    return s >= 53 ? (uint16_t)0 : (uint16_t)(m >> s);
}

// Magnitude planes of the certificate: M[r][l] = the largest bf16 not above
// |hi_rl| 2^-e_r (zero in the padding), K-major like the digit planes.  Two
// threads per (row, 16 consecutive k), eight entries and one 16-byte store
// each.  Block (0, 0) of the launch given `hdr` first writes the call's
// header image (plan, dmin = +inf); the magnitude product runs after it.
__global__ void __launch_bounds__(128) magnitude_kernel(
    const double *__restrict__ Xh, int64_t ld, int row_contig, int64_t rows, int64_t k,
    int64_t rows_pad, int64_t k_pad, const unsigned long long *__restrict__ rmax,
    __nv_bfloat16 *__restrict__ M, SplitHeader *hdr, const SplitHeader init) {
    if (hdr != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *hdr = init;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 2) + threadIdx.x / 2;
    if (r >= rows_pad) return;
    const int64_t l0 = (int64_t)blockIdx.y * 16 + 8 * (threadIdx.x & 1);
    const int e = r < rows ? scale_exponent(rmax[r]) : 0;
    uint16_t out[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int64_t l = l0 + q;
        double v = 0.0;
        if (r < rows && l < k) v = Xh[row_contig ? (r + l * ld) : (l + r * ld)];
        out[q] = bf16_floor_scaled(v, e);
    }
    uint4 w;
    memcpy(&w, out, 16);
    *reinterpret_cast<uint4 *>(M + r * k_pad + l0) = w;
}

// ------------------------------------------------------------------ step 3

__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int group_n,
                                            int &tm, int &tn) {
    int group = tile / (tiles_m * group_n);
    int first = group * group_n;
    int gn = tiles_n - first < group_n ? tiles_n - first : group_n;
    int local = tile - group * tiles_m * group_n;
    tn = first + local % gn;
    tm = local / gn;
}

// Work item -> output tile and the bands [b0, b1) it accumulates.  Digit
// pairs (sliced form): one item per tile, all S bands, so each tile's int32
// sums are finished in one visit.  Residues (diagonal mode): one item per
// (modulus, tile) with the modulus slowest, so the CTAs resident at one time
// share one modulus's operand panels in L2.
// Tiles entirely outside the requested triangle (Rsyrk form) get an empty
// band range, so every role skips them alike.
template <int TN, bool PAIR>
__device__ __forceinline__ void item_coords(const BandArgs &p, int S, int item, int num_tiles,
                                            int rank, const int *tri_s, int &tm, int &tn,
                                            int &b0, int &b1) {
    int tile = item;
    b0 = 0;
    b1 = S;
    if (p.diag) {
        b0 = item / num_tiles;
        b1 = b0 + 1;
        tile = item % num_tiles;
    }
    if (tri_s != nullptr) {
        // tile-th tile inside the triangle: the last (group, row unit) whose
        // cumulative count is at most tile, then the column within it
        int lo = 0, hi = p.tri_rows;   // tri_s[lo] <= tile < tri_s[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tri_s[mid] <= tile) lo = mid;
            else hi = mid;
        }
        const int grp = lo / p.tri_units, u = lo - grp * p.tri_units;
        const TriGeom g{p.tri, PAIR ? 2 * TM : TM, TN, p.tiles_n, kGroupTri};
        int c_lo, c_hi;
        tri_range(g, grp, u, c_lo, c_hi);
        tn = c_lo + (tile - tri_s[lo]);
        tm = PAIR ? 2 * u + rank : u;
        return;
    }
    // a CTA pair takes two vertically adjacent tiles (one per CTA) and skips
    // a triangle item only when both tiles lie outside
    int64_t r0, rows;
    if (PAIR) {
        int tp;
        tile_coords(tile, p.tiles_m / 2, p.tiles_n, p.tri ? kGroupTri : kGroupFull, tp, tn);
        tm = 2 * tp + rank;
        r0 = (int64_t)tp * 2 * TM;
        rows = 2 * TM;
    } else {
        tile_coords(tile, p.tiles_m, p.tiles_n, p.tri ? kGroupTri : kGroupFull, tm, tn);
        r0 = (int64_t)tm * TM;
        rows = TM;
    }
    const int64_t c0 = (int64_t)tn * TN;
    if ((p.tri == 1 && r0 > c0 + TN - 1) || (p.tri == 2 && r0 + rows - 1 < c0)) b1 = b0;
}

constexpr unsigned int kInfBits32 = 0x7F800000u;   // +inf as fp32 bits

// A lower bound of |c| 2^-s (c a finite binary64, s an integer) as an fp32:
// the significand truncated to 24 bits and the exponent shifted; 0 below
// the fp32 normal range, the largest finite fp32 above it; +inf for an
// infinite or NaN c (such an entry does not constrain the certificate).
__device__ __forceinline__ float scaled_floor_f32(double c, int s) {
    const unsigned long long u =
        (unsigned long long)__double_as_longlong(c) & 0x7FFFFFFFFFFFFFFFull;
    const int E = (int)(u >> 52);
    if (E == 0x7FF) return __int_as_float(0x7F800000);
    if (E == 0) return 0.0f;                    // subnormal c: its part is dropped
    const int x = E - 1023 - s;                 // exponent of |c| 2^-s
    if (x < -126) return 0.0f;
    if (x > 127) return __int_as_float(0x7F7FFFFF);
    return __int_as_float(((x + 127) << 23) | (int)((u >> 29) & 0x7FFFFF));
}

// Certificate margin of the entries (i, j0 .. j0 + EC - 1) from their
// fp32 magnitude sums s_ij (read from tensor memory 16 columns at a time):
//   d_ij = s_ij c1 + r |c_ij| 2^-(e_i + f_j),  r <= |beta / alpha|,
// in fp32 with every step rounded toward zero, so d_ij is at most the exact
// margin of a lower bound of (|A||B|)_ij.  Rows or columns that are all zero
// (exact in every form), entries outside C or the requested triangle, and
// entries whose C is infinite or NaN (then so is the result) do not
// constrain.  Used by all 32 lanes of an epilogue warp (rows i of the lanes,
// the same EC columns): each lane loads EC / 32 column maxima and the warp
// shares them by shuffles.  C is read 16 columns at a time, the first 16
// before the tile's accumulator is complete (under the tile's MMAs).  The
// minimum over the warp goes to *dmin_out with one atomic.
template <int EC>
struct Margin {
    static_assert(EC == 64 || EC == 128, "64 or 128 columns");
    static constexpr int NC = EC / 32;   // column maxima per lane
    unsigned mask;
    int fcol[NC];
    bool zcol[NC];
    bool row_ok, use_c;
    int ei;
    unsigned int dm;
    int64_t i, j0;

    __device__ __forceinline__ Margin(const BandArgs &p, int64_t i_, int64_t j0_)
        : i(i_), j0(j0_) {
        mask = __activemask();
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int h = 0; h < NC; ++h) {
            const int64_t j = j0 + 32 * h + lane;
            const unsigned long long cm = j < p.n ? p.cmax[j] : 0ull;
            zcol[h] = cm == 0;
            fcol[h] = scale_exponent(cm);
        }
        const unsigned long long rm = i < p.m ? p.rmax[i] : 0ull;
        row_ok = rm != 0;
        ei = scale_exponent(rm);
        use_c = p.ba_ratio32 > 0.0f;
        dm = kInfBits32;
    }
    // C of columns j0 + 16 g .. + 15 (zero where it does not count)
    __device__ __forceinline__ void load(const BandArgs &p, int g, double (&cv)[16]) const {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int64_t j = j0 + 16 * g + u;
            cv[u] = (use_c && row_ok && j < p.n) ? p.ch[i + j * p.ldc] : 0.0;
        }
    }
    // the margins of those columns from their sums (fp32 bits in r)
    __device__ __forceinline__ void eval(const BandArgs &p, int g, const uint32_t (&r)[16],
                                         const double (&cv)[16]) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int jj = 16 * g + u;
            const int64_t j = j0 + jj;
            const int fj = __shfl_sync(mask, fcol[jj / 32], jj % 32);
            const bool zj = __shfl_sync(mask, (int)zcol[jj / 32], jj % 32) != 0;
            float d = __fmul_rz(__uint_as_float(r[u]), p.c1);
            if (use_c) d = __fadd_rz(d, __fmul_rz(scaled_floor_f32(cv[u], ei + fj), p.ba_ratio32));
            const bool inside = row_ok && !zj && j < p.n && !(p.tri == 1 && i > j) &&
                                !(p.tri == 2 && i < j);
            const unsigned int db = __float_as_uint(d);
            dm = (inside && db < dm) ? db : dm;
        }
    }
    __device__ __forceinline__ void finish(const BandArgs &p) {
        dm = __reduce_min_sync(mask, dm);
        if ((threadIdx.x & 31) == 0 && dm != kInfBits32) atomicMin(p.dmin_out, dm);
    }
};

// MAG: the certificate's magnitude product (bf16 operands, fp32 sums, the
// margin d_ij of every entry reduced to its minimum); otherwise the integer
// band products with the band count taken from the call's plan.
// PAIR: a cluster of two CTAs on a 256 x 256 tile (vertically adjacent
// 128-row halves, the same 256 columns) multiplied by the 2-SM MMA.  Each
// CTA copies its own op(A) panel and one half of the op(B) panel (tmB's box
// is TN / 2 rows) into its shared memory, with completion on the leader's
// (rank 0) "full" barrier, which expects both CTAs' bytes.  The leader's MMA
// thread issues the pair MMAs; its commits arrive on the "empty" and
// "accumulator full" barriers of both CTAs.  Each CTA's epilogue drains its
// own tensor memory and releases a buffer with one arrival per warp on the
// leader's "accumulator empty" barrier.  Every tcgen05 operation of this
// instantiation is of the pair form.
// TRI: the work items are the tiles inside the triangle (p.tri_cum); the
// other instantiations carry no code for it.
template <int TN, bool MAG, bool PAIR = false, bool TRI = false>
__global__ void __launch_bounds__(BandCfg<TN, PAIR>::THREADS, 1)
    band_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB, const BandArgs p) {
    int S = p.S;
    if (!MAG && p.plan.dmin != nullptr) {
        // the same decision in every thread of every CTA: a word written by
        // an earlier launch of this call
        const PlanPick pk = plan_choice(p.plan);
        if (pk.c < 0) return;
        S = pk.count;
    }
    using Cfg = BandCfg<TN, PAIR>;
    constexpr int STAGES = Cfg::STAGES;
    constexpr uint32_t kStageBytes = Cfg::STAGE_BYTES;
    constexpr int kTmemCols = Cfg::TMEM_COLS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * Cfg::A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * kStageBytes);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;
    uint64_t *acce = accf + 2;
    uint64_t *fin = acce + 2;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(fin + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    int *tri_s = TRI ? reinterpret_cast<int *>(smem + STAGES * kStageBytes + 256) : nullptr;
    if (TRI)   // the triangle table, read by every role per item
        for (int x = threadIdx.x; x <= p.tri_rows; x += blockDim.x) tri_s[x] = p.tri_cum[x];

    static_assert(!PAIR || (TN == 256 && !MAG), "CTA pairs: residue / digit products, 256 wide");
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int rank = PAIR ? (int)cluster_ctarank() : 0;
    const int item0 = PAIR ? (int)cluster_id_x() : (int)blockIdx.x;
    const int item_step = PAIR ? (int)cluster_count_x() : (int)gridDim.x;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            // PAIR: one arrival per epilogue warp of either CTA
            mbar_init(&acce[b], PAIR ? 2 * Cfg::EPI_WARPS : 32 * Cfg::EPI_WARPS);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        if (PAIR) {
            tmem_alloc_pair(tmem_holder, kTmemCols);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(tmem_holder, kTmemCols);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (PAIR) cluster_sync();   // the peer's barriers exist before anything lands there
    const uint32_t tmem = *tmem_holder;

    const int num_tiles = TRI ? p.tri_tiles : (PAIR ? p.tiles_m / 2 : p.tiles_m) * p.tiles_n;
    const int KB = p.kb_count;
    const int num_items = p.diag ? num_tiles * S : num_tiles;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            prefetch_tmap(&tmA);
            prefetch_tmap(&tmB);
            uint32_t it = 0;
            bool ok = true;
            for (int item = item0; item < num_items && ok; item += item_step) {
                int tm, tn, b0, b1;
                item_coords<TN, PAIR>(p, S, item, num_tiles, rank, tri_s, tm, tn, b0, b1);
                for (int b = b0; b < b1 && ok; ++b)
                    for (int t = p.diag ? b : 0; t <= b && ok; ++t) {
                        const int ya = (int)(t * p.m_pad) + tm * TM;
                        const int yb = (int)((p.diag ? b : b - t) * p.n_pad) + tn * TN;
                        for (int kb = 0; kb < KB; ++kb, ++it) {
                            const int s = it % STAGES;
                            const uint32_t f = it / STAGES;
                            if (!mbar_wait(&empty[s], (f & 1) ^ 1, abort_flag)) {
                                ok = false;
                                break;
                            }
                            if (PAIR) {
                                // both CTAs' copies complete on the leader's barrier,
                                // which the leader arms for both
                                const uint32_t fl = cluster_map(&full[s], 0);
                                if (rank == 0) mbar_arrive_expect_tx(&full[s], 2 * kStageBytes);
                                tma_load_2d_pair(sA + s * Cfg::A_BYTES, &tmA, fl, kb * TK, ya);
                                tma_load_2d_pair(sB + s * Cfg::B_BYTES, &tmB, fl, kb * TK,
                                                 yb + rank * (TN / 2));
                            } else {
                                mbar_arrive_expect_tx(&full[s], kStageBytes);
                                tma_load_2d(sA + s * Cfg::A_BYTES, &tmA, &full[s], kb * TK, ya);
                                tma_load_2d(sB + s * Cfg::B_BYTES, &tmB, &full[s], kb * TK, yb);
                            }
                        }
                    }
            }
            if (PAIR && ok) {
                // the leader's last commits on this CTA's barriers have
                // landed before it may exit
                const uint32_t first = it > STAGES ? it - STAGES : 0;
                for (uint32_t j = first; j < it && ok; ++j)
                    ok = mbar_wait(&empty[j % STAGES], (j / STAGES) & 1, abort_flag);
            }
            if (!ok) {
                // let the copies already issued land before the CTA exits
                const uint32_t first = it > STAGES ? it - STAGES : 0;
                for (uint32_t j = first; j < it; ++j) {
                    const long long t0 = clock64();
                    while (!mbar_try_wait(&full[j % STAGES], (j / STAGES) & 1) &&
                           clock64() - t0 < kWaitCycles / 4) {
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer (PAIR: the leader's, for both CTAs)
        if (lane == 0 && (!PAIR || rank == 0)) {
            const uint32_t idesc = MAG ? idesc_bf16_f32(TM, TN)
                                       : idesc_f16_f32(PAIR ? 2 * TM : TM, TN);
            uint32_t it = 0, chunk = 0;
            bool ok = true;
            for (int item = item0; item < num_items && ok; item += item_step) {
                int tm, tn, b0, b1;
                item_coords<TN, PAIR>(p, S, item, num_tiles, rank, tri_s, tm, tn, b0, b1);
                for (int b = b0; b < b1 && ok; ++b) {
                    const int steps = (p.diag ? 1 : b + 1) * KB;
                    int sidx = 0;
                    for (int t = p.diag ? b : 0; t <= b && ok; ++t)
                        for (int kb = 0; kb < KB; ++kb, ++it, ++sidx) {
                            const int s = it % STAGES;
                            const uint32_t f = it / STAGES;
                            const bool first = (sidx % chunk_kb<MAG>()) == 0;
                            const bool last =
                                ((sidx + 1) % chunk_kb<MAG>()) == 0 || sidx + 1 == steps;
                            const uint32_t buf = chunk & 1, use = chunk >> 1;
                            if (first) {
                                if (!mbar_wait(&acce[buf], (use & 1) ^ 1, abort_flag)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                            }
                            if (!mbar_wait(&full[s], f & 1, abort_flag)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t d = tmem + buf * TN;
                            const uint32_t a0 = smem_u32(sA + s * Cfg::A_BYTES);
                            const uint32_t b0 = smem_u32(sB + s * Cfg::B_BYTES);
#pragma unroll
                            for (int kk = 0; kk < TK / 16; ++kk) {
                                if (PAIR)
                                    mma_f16_pair(d, desc_sw128_kmajor(a0 + kk * 32),
                                                 desc_sw128_kmajor(b0 + kk * 32), idesc,
                                                 (first && kk == 0) ? 0u : 1u);
                                else
                                    mma_f16(d, desc_sw128_kmajor(a0 + kk * 32),
                                            desc_sw128_kmajor(b0 + kk * 32), idesc,
                                            (first && kk == 0) ? 0u : 1u);
                            }
                            if (PAIR) {
                                mma_commit_pair(&empty[s], (uint16_t)3);
                                if (last) {
                                    mma_commit_pair(&accf[buf], (uint16_t)3);
                                    ++chunk;
                                }
                            } else {
                                mma_commit(&empty[s]);
                                if (last) {
                                    mma_commit(&accf[buf]);
                                    ++chunk;
                                }
                            }
                        }
                }
            }
            // every issued MMA has completed before the tensor memory is freed
            if (PAIR)
                mma_commit_pair(fin, (uint16_t)1);
            else
                mma_commit(fin);
            long long t0 = clock64();
            while (!mbar_try_wait(fin, 0) && clock64() - t0 < kWaitCycles) {
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: drain chunks into int32 band sums
        const int q = warp % 4;                 // tensor-memory lane quadrant
        constexpr int EC = Cfg::EPI_COLS;             // accumulator columns of this thread
        const int col0 = ((warp - 2) / 4) * EC;       // first accumulator column
        const int row = q * 32 + lane;          // row of the tile this thread owns
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        uint32_t chunk = 0;
        bool ok = true;
        for (int item = item0; item < num_items && ok; item += item_step) {
            int tm, tn, b0, b1;
            item_coords<TN, PAIR>(p, S, item, num_tiles, rank, tri_s, tm, tn, b0, b1);
            for (int b = b0; b < b1 && ok; ++b) {
                if constexpr (MAG) {   // one fp32 run per tile
                    const uint32_t buf = chunk & 1, use = chunk >> 1;
                    ++chunk;
                    Margin<EC> mg(p, (int64_t)tm * TM + row, (int64_t)tn * TN + col0);
                    double cv[16];
                    mg.load(p, 0, cv);
                    if (!mbar_wait(&accf[buf], use & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int cc = 0; cc < EC / 16; ++cc) {
                        uint32_t r[16];
                        tmem_ld_32x32b_x16(tmem + lane_base + buf * TN + col0 + cc * 16, r);
                        tmem_ld_wait();
                        mg.eval(p, cc, r, cv);
                        if (cc + 1 < EC / 16) mg.load(p, cc + 1, cv);
                    }
                    tc_fence_before();
                    mbar_arrive(&acce[buf]);
                    mg.finish(p);
                    continue;
                }
                int32_t acc[EC];
#pragma unroll
                for (int j = 0; j < EC; ++j) acc[j] = 0;
                const int steps = (p.diag ? 1 : b + 1) * KB;
                const int nchunks = (steps + chunk_kb<MAG>() - 1) / chunk_kb<MAG>();
                for (int c = 0; c < nchunks; ++c, ++chunk) {
                    const uint32_t buf = chunk & 1, use = chunk >> 1;
                    if (!mbar_wait(&accf[buf], use & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int cc = 0; cc < EC / 16; ++cc) {
                        uint32_t r[16];
                        tmem_ld_32x32b_x16(tmem + lane_base + buf * TN + col0 + cc * 16, r);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            acc[cc * 16 + j] += __float2int_rn(__uint_as_float(r[j]));
                    }
                    tc_fence_before();
                    if (PAIR) {   // one arrival per warp on the leader's barrier
                        __syncwarp();
                        if (lane == 0) mbar_arrive_cluster(cluster_map(&acce[buf], 0));
                    } else {
                        mbar_arrive(&acce[buf]);
                    }
                }
                if (!ok) break;
                const int64_t off = ((int64_t)b * p.n_pad + (int64_t)tn * TN + col0) * p.m_pad +
                                    (int64_t)tm * TM + row;
                if (p.diag) {
                    const int pm = p.moduli[b];
                    uint8_t *dst = p.R + off;
#pragma unroll
                    for (int j = 0; j < EC; ++j) {
                        int r = acc[j] % pm;
                        dst[(int64_t)j * p.m_pad] = (uint8_t)(r < 0 ? r + pm : r);
                    }
                } else {
                    int32_t *dst = p.P + off;
#pragma unroll
                    for (int j = 0; j < EC; ++j) dst[(int64_t)j * p.m_pad] = acc[j];
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (PAIR) {
        cluster_sync();   // both CTAs done with the pair's tensor memory
        if (warp == 1) tmem_dealloc_pair(tmem, kTmemCols);
    } else if (warp == 1) {
        tmem_dealloc(tmem, kTmemCols);
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(p.status, MP_DD_ERR_TIMEOUT);
    if (PAIR) cluster_sync();   // no CTA leaves while its peer may still signal it
}

// ------------------------------------------------------------------ step 4

struct RecArgs {
    SplitPlan plan;   // the slice count (no certified count: nothing to do)
    int64_t m, n, m_pad, n_pad;
    const int32_t *P;
    const unsigned long long *rmax, *cmax;
    mp_dd alpha, beta;
    int alpha_one, beta_zero;
    double *ch, *cl;
    int64_t ldc;
};

// x * 2^e, exact for results in the normal range.
__device__ __forceinline__ double mul_pow2(double x, int e) {
    while (e > 1000) {
        x = __dmul_rn(x, __longlong_as_double((long long)(1000 + 1023) << 52));
        e -= 1000;
    }
    while (e < -1000) {
        x = __dmul_rn(x, __longlong_as_double((long long)(-1000 + 1023) << 52));
        e += 1000;
    }
    return __dmul_rn(x, __longlong_as_double((long long)(e + 1023) << 52));
}

__device__ __forceinline__ int msb64(unsigned long long x) { return 63 - __clzll(x); }

// Signed 128-bit integer to the nearest binary64.
__device__ __forceinline__ double i128_to_double(__int128 v) {
    bool neg = v < 0;
    unsigned __int128 a = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
    double r;
    if (hi == 0) {
        r = __ull2double_rn(lo);
    } else {
        int p = 64 + msb64(hi);               // >= 64
        int sh = p - 63;                      // keep the top 64 bits
        unsigned __int128 top = a >> sh;
        unsigned long long w = (unsigned long long)top;
        unsigned __int128 dropped = a & (((unsigned __int128)1 << sh) - 1);
        if (dropped != 0) w |= 1ull;          // sticky bit below the rounding point
        r = mul_pow2(__ull2double_rn(w), sh);
    }
    return neg ? -r : r;
}

__global__ void __launch_bounds__(256) recombine_kernel(const RecArgs p) {
    const PlanPick pk = plan_choice(p.plan);
    if (pk.c < 0) return;
    const int S = pk.count;
    const int64_t total = p.m * p.n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx % p.m, j = idx / p.m;
        // V = sum_b P_b 256^(S-1-b) in 192-bit two's complement (hi:lo)
        unsigned __int128 lo = 0;
        long long hi = 0;
        for (int b = 0; b < S; ++b) {
            const int32_t v = p.P[((int64_t)b * p.n_pad + j) * p.m_pad + i];
            hi = (long long)(((unsigned long long)hi << 8) | (unsigned long long)(lo >> 120));
            lo <<= 8;
            const unsigned __int128 ext = (unsigned __int128)(__int128)(long long)v;
            const unsigned __int128 sum = lo + ext;
            hi += (sum < lo ? 1 : 0) + (v < 0 ? -1 : 0);
            lo = sum;
        }
        const bool neg = hi < 0;
        if (neg) {
            lo = ~lo + 1;
            hi = (long long)(~(unsigned long long)hi + (lo == 0 ? 1ull : 0ull));
        }
        double vh = 0.0, vl = 0.0;
        const unsigned long long w2 = (unsigned long long)hi;
        const unsigned long long w1 = (unsigned long long)(lo >> 64), w0 = (unsigned long long)lo;
        int pbit = -1;
        if (w2) pbit = 128 + msb64(w2);
        else if (w1) pbit = 64 + msb64(w1);
        else if (w0) pbit = msb64(w0);
        const int sc = scale_exponent(p.rmax[i]) + scale_exponent(p.cmax[j]) - 8 * S - 8;
        if (pbit >= 0 && pbit <= 52) {
            vh = mul_pow2(__ull2double_rn(w0), sc);
        } else if (pbit > 52) {
            const int q = pbit - 52;          // <= 88 for |V| < 2^141
            const unsigned __int128 shifted =
                (lo >> q) | (q < 128 ? ((unsigned __int128)w2 << (128 - q)) : 0);
            unsigned long long H = (unsigned long long)shifted;
            const unsigned __int128 mask = ((unsigned __int128)1 << q) - 1;
            const unsigned __int128 R = lo & mask;
            const unsigned __int128 half = (unsigned __int128)1 << (q - 1);
            __int128 Rs = (__int128)R;
            if (R > half || (R == half && (H & 1))) {
                ++H;
                Rs = (__int128)R - ((__int128)1 << q);
            }
            vh = mul_pow2(__ull2double_rn(H), q + sc);
            vl = mul_pow2(i128_to_double(Rs), sc);
        }
        if (neg) {
            vh = -vh;
            vl = -vl;
        }
        dd v{vh, vl};
        if (!p.alpha_one) v = mul(dd{p.alpha.hi, p.alpha.lo}, v);
        const int64_t off = i + j * p.ldc;
        if (!p.beta_zero)
            v = add_sloppy(v, mul(dd{p.beta.hi, p.beta.lo}, dd{p.ch[off], p.cl[off]}));
        p.ch[off] = v.hi;
        p.cl[off] = v.lo;
    }
}

// ------------------------------------------------------------------ host

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

}  // namespace

// Tensor map of a [rows][k_pad] fp16 (elem 0) or bf16 (elem 1) array, box
// 64 (k) x box_rows.
int make_tmap(CUtensorMap *m, void *base, int64_t rows, int64_t k_pad, int box_rows, int elem) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return fail(MP_DD_ERR_NO_DEVICE, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)k_pad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)k_pad * 2};
    cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, elem ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                    2, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(MP_DD_ERR_NO_DEVICE, "cuTensorMapEncodeTiled failed: CUresult %d", (int)r);
    return 0;
}

int launch_absmax(const double *X, int64_t ld, int row_contig, int64_t rows, int64_t k,
                  unsigned long long *out, cudaStream_t st) {
    if (rows == 0 || k == 0) return 0;
    const int64_t lchunk = 256;
    dim3 grid((unsigned)ceil_div(rows, 128), (unsigned)ceil_div(k, lchunk));
    if (grid.y > 65535) return fail(MP_DD_ERR_TOO_LARGE, "k too large for the scaling pass");
    absmax_kernel<<<grid, 128, 0, st>>>(X, ld, row_contig, rows, k, lchunk, out);
    return check_launch("absmax_kernel");
}

namespace {

template <int SA, int SB>
void launch_slice_s(const double *Xh, const double *Xl, int64_t ld, int row_contig,
                    int64_t rows, int64_t k, int64_t rows_pad, int64_t k_pad,
                    const unsigned long long *rmax, __half *D, const SplitPlan &plan,
                    cudaStream_t st) {
    dim3 grid((unsigned)ceil_div(rows_pad, 64), (unsigned)(k_pad / 16));
    slice_kernel<SA, SB><<<grid, 128, 0, st>>>(Xh, Xl, ld, row_contig, rows, k, rows_pad, k_pad,
                                               rmax, D, plan);
}

// Slice with the certified count among the plan's candidates (one fixed S,
// or 14 / 15).
int launch_slice(const SplitPlan &plan, const double *Xh, const double *Xl, int64_t ld,
                 int row_contig, int64_t rows, int64_t k, int64_t rows_pad, int64_t k_pad,
                 const unsigned long long *rmax, __half *D, cudaStream_t st) {
    if (k_pad / 16 > 65535) return fail(MP_DD_ERR_TOO_LARGE, "k too large for slicing");
    if (plan.ncand == 2) {
        if (plan.count[0] != 14 || plan.count[1] != 15)
            return fail(MP_DD_ERR_TOO_LARGE, "unexpected slice candidates");
        launch_slice_s<14, 15>(Xh, Xl, ld, row_contig, rows, k, rows_pad, k_pad, rmax, D, plan,
                               st);
        return check_launch("slice_kernel");
    }
#define MPDD_SLICE_CASE(SS)                                                                  \
    case SS:                                                                                 \
        launch_slice_s<SS, SS>(Xh, Xl, ld, row_contig, rows, k, rows_pad, k_pad, rmax, D, plan, \
                               st);                                                          \
        break;
    switch (plan.count[0]) {
        MPDD_SLICE_CASE(2) MPDD_SLICE_CASE(3) MPDD_SLICE_CASE(4) MPDD_SLICE_CASE(5)
        MPDD_SLICE_CASE(6) MPDD_SLICE_CASE(7) MPDD_SLICE_CASE(8) MPDD_SLICE_CASE(9)
        MPDD_SLICE_CASE(10) MPDD_SLICE_CASE(11) MPDD_SLICE_CASE(12) MPDD_SLICE_CASE(13)
        MPDD_SLICE_CASE(14) MPDD_SLICE_CASE(15)
        default:
            return fail(MP_DD_ERR_TOO_LARGE, "slices = %d outside [2, 15]", plan.count[0]);
    }
#undef MPDD_SLICE_CASE
    return check_launch("slice_kernel");
}

// Optional per-phase CUDA-event timing of split-precision calls made by this
// thread (scaling, certificate and splitting; tensor-core products;
// recombination or reconstruction): four events per call, kept for every
// call since timing was enabled (up to kMaxTimedCalls).
constexpr int kMaxTimedCalls = 4096;

struct PhaseTimer {
    bool on = false;
    int calls = 0;              // completed timed calls since enabling
    std::vector<cudaEvent_t> ev;  // 4 per call slot
    void mark(int i, cudaStream_t st) {
        if (!on || calls >= kMaxTimedCalls) return;
        const size_t slot = (size_t)calls * 4 + (size_t)i;
        while (ev.size() <= slot) {
            cudaEvent_t e = nullptr;
            cudaEventCreate(&e);
            ev.push_back(e);
        }
        cudaEventRecord(ev[slot], st);
        if (i == 3) ++calls;
    }
};

PhaseTimer &timer() {
    static thread_local PhaseTimer t;
    return t;
}

}  // namespace

void sliced_timing_mark(int phase, cudaStream_t st) { timer().mark(phase, st); }

void sliced_timing_enable(int on) {
    timer().on = on != 0;
    timer().calls = 0;
}

int sliced_timing_read(float *ms) {
    PhaseTimer &t = timer();
    if (t.calls == 0) return fail(MP_DD_ERR_TOO_LARGE, "no timed sliced call on this thread");
    const size_t b = (size_t)(t.calls - 1) * 4;
    cudaError_t e = cudaEventSynchronize(t.ev[b + 3]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    for (int i = 0; i < 3; ++i) cudaEventElapsedTime(&ms[i], t.ev[b + i], t.ev[b + i + 1]);
    return 0;
}

int sliced_timing_log(float *ms, int max_calls, int *calls) {
    PhaseTimer &t = timer();
    const int n = t.calls < max_calls ? t.calls : max_calls;
    for (int c = 0; c < n; ++c) {
        const size_t b = (size_t)c * 4;
        cudaError_t e = cudaEventSynchronize(t.ev[b + 3]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        for (int i = 0; i < 3; ++i)
            cudaEventElapsedTime(&ms[3 * c + i], t.ev[b + i], t.ev[b + i + 1]);
    }
    *calls = t.calls;
    return 0;
}

namespace {

// Slices the workspace holds: the caller's S, or the widest auto candidate.
int slices_allocated(int slices, int64_t k) {
    int cand[kMaxCand];
    const int nc = slice_candidates(slices, k, cand);
    return cand[nc - 1];
}

}  // namespace

size_t sliced_workspace_bytes(int64_t m, int64_t n, int64_t k, int S) {
    return make_layout(m, n, k, slices_allocated(S, k)).total;
}

int sliced_layout(int64_t m, int64_t n, int64_t k, int S, size_t *offsets) {
    Layout L = make_layout(m, n, k, slices_allocated(S, k));
    offsets[0] = L.off_rowmax;
    offsets[1] = L.off_colmax;
    offsets[2] = L.off_da;
    offsets[3] = L.off_db;
    offsets[4] = L.off_p;
    offsets[5] = (size_t)L.m_pad;
    offsets[6] = (size_t)L.n_pad;
    offsets[7] = (size_t)L.k_pad;
    return 0;
}

int sliced_magnitude_offsets(int64_t m, int64_t n, int64_t k, int S, size_t *offsets) {
    Layout L = make_layout(m, n, k, slices_allocated(S, k));
    offsets[0] = L.off_ma;
    offsets[1] = L.off_mb;
    return 0;
}

// ------------------------------------------------------------------ certificate (host)

SplitPlan make_plan(SplitHeader *h, unsigned int *dmin_dev, int form, int64_t k, int ncand,
                    const int *widths, const int *counts, const double *cst) {
    SplitPlan pl{};
    pl.dmin = dmin_dev;
    pl.ncand = ncand;
    *h = SplitHeader{};
    h->form = form;
    h->ncand = ncand;
    h->k = k;
    h->dmin = 0x7F800000u;   // +inf until the magnitude product lowers it
    for (int c = 0; c < ncand; ++c) {
        // cst 2^(106 - W) / 12 rounded up to fp32: the power of two is exact,
        // the binary64 quotient is within 2^-53 of itself, (1 + 2^-50) covers
        // that, and the conversion to fp32 rounds up (to +inf if too large)
        const double t = std::ldexp(cst[c], 106 - widths[c]) / 12.0 * (1.0 + 0x1p-50);
        float f = (float)t;
        if ((double)f < t) f = std::nextafter(f, std::numeric_limits<float>::infinity());
        unsigned int bits;
        memcpy(&bits, &f, 4);
        pl.thr[c] = h->thr[c] = bits;
        pl.count[c] = h->count[c] = counts[c];
        pl.width[c] = h->width[c] = widths[c];
    }
    return pl;
}

int launch_magnitude(const double *X, int64_t ld, int row_contig, int64_t rows, int64_t k,
                     int64_t rows_pad, int64_t k_pad, const unsigned long long *rmax, void *M,
                     SplitHeader *hdr, const SplitHeader *init, cudaStream_t st) {
    if (k_pad / 16 > 65535) return fail(MP_DD_ERR_TOO_LARGE, "k too large for the certificate");
    dim3 grid((unsigned)ceil_div(rows_pad, 64), (unsigned)(k_pad / 16));
    magnitude_kernel<<<grid, 128, 0, st>>>(X, ld, row_contig, rows, k, rows_pad, k_pad, rmax,
                                          static_cast<__nv_bfloat16 *>(M),
                                          init ? hdr : nullptr, init ? *init : SplitHeader{});
    return check_launch("magnitude_kernel");
}

namespace {

// A lower bound of |beta| / |alpha| for dd scalars: |x| >= |x.hi| (1 - 2^-53)
// for a normalised dd, the binary64 quotient is within 2^-53 of the exact
// one, and the factor (1 - 2^-49) absorbs both.
double ratio_lower(mp_dd beta, mp_dd alpha) {
    return std::fabs(beta.hi) / std::fabs(alpha.hi) * (1.0 - 0x1p-49);
}

}  // namespace

int launch_certificate(const GemmArgs &p, void *MA, void *MB, int64_t m_pad, int64_t n_pad,
                       int64_t k_pad, int TN, const unsigned long long *rmax,
                       const unsigned long long *cmax, SplitHeader *hdr, cudaStream_t st,
                       int *tri_table) {
    // the product's own tile width (n_pad is a multiple of it) when that
    // leaves at least 1024 tiles (~7 per SM): at 8192 the 128 x 256 tiles
    // take the magnitude product from 1.23 to 1.09 ms, at 4096 their 512
    // tiles (3.4 per SM) took 254 us against 189 us on 128 x 128 tiles
    if (TN != 256 || (m_pad / TM) * (n_pad / 256) < 1024) TN = 128;
    int rc;
    CUtensorMap tmA, tmB;
    if ((rc = make_tmap(&tmA, MA, m_pad, k_pad, TM, 1))) return rc;
    if ((rc = make_tmap(&tmB, MB, n_pad, k_pad, TN, 1))) return rc;
    BandArgs ba{};
    ba.S = 1;
    ba.kb_count = (int)(k_pad / TK);
    ba.tiles_m = (int)(m_pad / TM);
    ba.tiles_n = (int)(n_pad / TN);
    ba.m_pad = m_pad;
    ba.n_pad = n_pad;
    ba.status = &hdr->status;
    ba.diag = 1;
    ba.tri = p.tri;
    ba.mag = 1;
    ba.m = p.m;
    ba.n = p.n;
    ba.ldc = p.ldc;
    ba.rmax = rmax;
    ba.cmax = cmax;
    ba.ch = p.ch;
    ba.ba_ratio = p.beta_zero ? 0.0 : ratio_lower(p.beta, p.alpha);
    {   // rounded toward zero to fp32
        float f = (float)ba.ba_ratio;
        if ((double)f > ba.ba_ratio) f = std::nextafter(f, 0.0f);
        ba.ba_ratio32 = f;
    }
    // Safety factor of the fp32 sums.  Each bf16 x bf16 product is exact
    // (16 significant bits) or, flushed, smaller; the k products are
    // non-negative, so each fp32 addition raises the running sum by at most
    // 2^-23 of the final sum (round to nearest: 2^-24; truncation lowers it),
    // and the computed sum is at most (1 + k 2^-23) times the exact one.
    // With |hi| >= (1 - 2^-53) |hi + lo| as well, multiplying by
    // 1 - (k+1) 2^-20 (exact in fp32 for k < 2^17) leaves a lower bound of
    // (|A||B|)_ij 2^-(e_i+f_j) with an eightfold margin on the additions.
    ba.c1 = (float)(1.0 - (double)(p.k + 1) * 0x1p-20);
    ba.dmin_out = &hdr->dmin;
    ba.tri_cum = p.tri ? tri_table : nullptr;
    return launch_band(tmA, tmB, ba, TN, st);
}

int run_sliced(const GemmArgs &p, int slices, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (slices != 0 && (slices < 2 || slices > kMaxSlices))
        return fail(MP_DD_ERR_TOO_LARGE, "slices = %d outside [2, %d]", slices, kMaxSlices);
    int cand[kMaxCand];
    const int ncand = slice_candidates(slices, p.k, cand);
    // |P_b| <= (b + 1) k 2^14 must stay below 2^31 for the int32 band sums
    if ((int64_t)cand[0] * p.k > ((int64_t)1 << 17) - 1)
        return fail(MP_DD_ERR_TOO_LARGE, "k * slices = %lld exceeds 131071",
                    (long long)(cand[0] * p.k));
    const int S = cand[ncand - 1];   // planes the workspace holds
    Layout L = make_layout(p.m, p.n, p.k, S);
    if (ws == nullptr || ws_bytes < L.total)
        return fail(MP_DD_ERR_WORKSPACE, "sliced Rgemm needs %zu workspace bytes, got %zu",
                    L.total, ws_bytes);
    if (L.n_pad * (int64_t)S > 0x7fffffffLL || L.m_pad * (int64_t)S > 0x7fffffffLL)
        return fail(MP_DD_ERR_TOO_LARGE, "matrix too large for the sliced path");
    const int TN = band_tn(p.m, p.n);

    uint8_t *w = static_cast<uint8_t *>(ws);
    cudaError_t e = cudaMemsetAsync(w, 0, L.off_da, st);  // header (form 0) and maxima
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (p.alpha_zero) return launch_gemm_plain(p, st);  // C := beta C only
    auto *rmax = reinterpret_cast<unsigned long long *>(w + L.off_rowmax);
    auto *cmax = reinterpret_cast<unsigned long long *>(w + L.off_colmax);
    auto *DA = reinterpret_cast<__half *>(w + L.off_da);
    auto *DB = reinterpret_cast<__half *>(w + L.off_db);
    auto *P = reinterpret_cast<int32_t *>(w + L.off_p);
    auto *hdr = reinterpret_cast<SplitHeader *>(w);

    int widths[kMaxCand];
    double cst[kMaxCand];
    for (int c = 0; c < ncand; ++c) {
        widths[c] = 8 * cand[c];
        cst[c] = slice_constant(cand[c]);
    }
    SplitHeader init;
    const SplitPlan plan = make_plan(&init, &hdr->dmin, 1, p.k, ncand, widths, cand, cst);

    // op(A) rows: A[i + l lda] when transa = N; op(B) columns as rows: B[l + j ldb]
    // when transb = N (contiguous in l), B[j + l ldb] when transb = T.
    const int a_rc = p.ta ? 0 : 1, b_rc = p.tb ? 1 : 0;
    int rc;
    timer().mark(0, st);
    if ((rc = launch_absmax(p.ah, p.lda, a_rc, p.m, p.k, rmax, st))) return rc;
    if ((rc = launch_absmax(p.bh, p.ldb, b_rc, p.n, p.k, cmax, st))) return rc;
    if ((rc = launch_magnitude(p.ah, p.lda, a_rc, p.m, p.k, L.m_pad, L.k_pad, rmax,
                               w + L.off_ma, hdr, &init, st)))
        return rc;
    if ((rc = launch_magnitude(p.bh, p.ldb, b_rc, p.n, p.k, L.n_pad, L.k_pad, cmax,
                               w + L.off_mb, hdr, nullptr, st)))
        return rc;
    if ((rc = launch_certificate(p, w + L.off_ma, w + L.off_mb, L.m_pad, L.n_pad, L.k_pad, TN,
                                 rmax, cmax, hdr, st)))
        return rc;
    if ((rc = launch_slice(plan, p.ah, p.al, p.lda, a_rc, p.m, p.k, L.m_pad, L.k_pad, rmax, DA,
                           st)))
        return rc;
    if ((rc = launch_slice(plan, p.bh, p.bl, p.ldb, b_rc, p.n, p.k, L.n_pad, L.k_pad, cmax, DB,
                           st)))
        return rc;

    timer().mark(1, st);
    CUtensorMap tmA, tmB;
    if ((rc = make_tmap(&tmA, DA, (int64_t)S * L.m_pad, L.k_pad, TM))) return rc;
    if ((rc = make_tmap(&tmB, DB, (int64_t)S * L.n_pad, L.k_pad, TN))) return rc;
    CUtensorMap tmB_half;   // half-height boxes for CTA pairs on 256-wide tiles
    if ((rc = make_tmap(&tmB_half, DB, (int64_t)S * L.n_pad, L.k_pad, TN / 2))) return rc;
    BandArgs ba{};
    ba.S = S;
    ba.kb_count = (int)(L.k_pad / TK);
    ba.tiles_m = (int)(L.m_pad / TM);
    ba.tiles_n = (int)(L.n_pad / TN);  // n_pad is a multiple of this call's tile width
    ba.m_pad = L.m_pad;
    ba.n_pad = L.n_pad;
    ba.P = P;
    ba.R = nullptr;
    ba.diag = 0;
    ba.status = &hdr->status;
    ba.plan = plan;
    if ((rc = launch_band(tmA, tmB, ba, TN, st, &tmB_half))) return rc;
    timer().mark(2, st);

    RecArgs ra{};
    ra.plan = plan;
    ra.m = p.m; ra.n = p.n; ra.m_pad = L.m_pad; ra.n_pad = L.n_pad;
    ra.P = P; ra.rmax = rmax; ra.cmax = cmax;
    ra.alpha = p.alpha; ra.beta = p.beta;
    ra.alpha_one = p.alpha_one; ra.beta_zero = p.beta_zero;
    ra.ch = p.ch; ra.cl = p.cl; ra.ldc = p.ldc;
    const int64_t total = p.m * p.n;
    int64_t blocks = ceil_div(total, 256);
    if (blocks > (int64_t)sm_count() * 32) blocks = (int64_t)sm_count() * 32;
    recombine_kernel<<<(unsigned)blocks, 256, 0, st>>>(ra);
    if ((rc = check_launch("recombine_kernel"))) return rc;
    rc = launch_plain_fallback(p, plan, st);
    timer().mark(3, st);
    return rc;
}

namespace {

}  // namespace

namespace {

// The triangle table of launch_band: cum[x] = tiles inside the triangle
// before (group, row unit) x in raster order, x = 0 .. rows (one block).
__global__ void __launch_bounds__(256) tri_table_kernel(TriGeom g, int units, int rows,
                                                        int *cum) {
    __shared__ int part[256];
    const int per = (rows + 255) / 256, x0 = threadIdx.x * per;
    int s = 0;
    for (int x = x0; x < x0 + per && x < rows; ++x) {
        int lo, hi;
        tri_range(g, x / units, x % units, lo, hi);
        s += hi >= lo ? hi - lo + 1 : 0;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < 256; ++t) {
            const int v = part[t];
            part[t] = run;
            run += v;
        }
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int x = x0; x < x0 + per && x < rows; ++x) {
        cum[x] = run;
        int lo, hi;
        tri_range(g, x / units, x % units, lo, hi);
        run += hi >= lo ? hi - lo + 1 : 0;
    }
    if (threadIdx.x == 255) cum[rows] = run;
}

// Geometry of the triangle table for a launch; 0 when the table does not
// apply (no triangle, no table memory, or too many rows for shared memory).
int tri_prepare(BandArgs &ba, int TN, bool pair, cudaStream_t st) {
    if (!ba.tri || ba.tri_cum == nullptr) {
        ba.tri_cum = nullptr;
        return 0;
    }
    const TriGeom g{ba.tri, pair ? 2 * TM : TM, TN, ba.tiles_n, kGroupTri};
    const int units = pair ? ba.tiles_m / 2 : ba.tiles_m;
    const int groups = (ba.tiles_n + kGroupTri - 1) / kGroupTri;
    const int rows = groups * units;
    if (rows + 1 > kTriMax) {
        ba.tri_cum = nullptr;
        return 0;
    }
    int tiles = 0;
    for (int x = 0; x < rows; ++x) {
        int lo, hi;
        tri_range(g, x / units, x % units, lo, hi);
        tiles += hi >= lo ? hi - lo + 1 : 0;
    }
    ba.tri_rows = rows;
    ba.tri_units = units;
    ba.tri_tiles = tiles;
    tri_table_kernel<<<1, 256, 0, st>>>(g, units, rows, ba.tri_cum);
    return check_launch("tri_table_kernel");
}

// 0: CTA pairs (the 2-SM MMA) for the Rsyrk triangle, single CTAs for full
// products; 1: pairs wherever they apply; 2: never.  At 8192 pairs take the
// triangle's band phase from 13.0 to 12.5 ms and the full product's from
// 20.5 to 21.0 ms.
std::atomic<int> g_band_pairs{0};

// Clusters of two band CTAs that fit on the GPU at once (0: none).
int pair_clusters() {
    static int count = -1;
    static std::once_flag once;
    std::call_once(once, [] {
        using Cfg = BandCfg<256, true>;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(2 * sm_count());
        cfg.blockDim = dim3(Cfg::THREADS);
        cfg.dynamicSmemBytes = Cfg::SMEM;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, band_gemm_kernel<256, false, true>, &cfg) !=
            cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        count = n;
    });
    return count;
}

}  // namespace

void set_band_pairs(int mode) { g_band_pairs.store(mode); }

int launch_band(const CUtensorMap &tmA, const CUtensorMap &tmB, const BandArgs &ba, int TN,
                cudaStream_t st, const CUtensorMap *tmB_half) {
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        auto big = [](const void *f, size_t bytes) {
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        };
        big((const void *)band_gemm_kernel<128, false>, BandCfg<128>::SMEM);
        big((const void *)band_gemm_kernel<256, false>, BandCfg<256>::SMEM);
        big((const void *)band_gemm_kernel<128, true>, BandCfg<128>::SMEM);
        big((const void *)band_gemm_kernel<256, false, true>, BandCfg<256, true>::SMEM);
        big((const void *)band_gemm_kernel<128, false, false, true>, BandCfg<128>::SMEM_TRI);
        big((const void *)band_gemm_kernel<256, false, false, true>, BandCfg<256>::SMEM_TRI);
        big((const void *)band_gemm_kernel<128, true, false, true>, BandCfg<128>::SMEM_TRI);
        big((const void *)band_gemm_kernel<256, false, true, true>, BandCfg<256, true>::SMEM_TRI);
        big((const void *)band_gemm_kernel<256, true>, BandCfg<256>::SMEM);
        big((const void *)band_gemm_kernel<256, true, false, true>, BandCfg<256>::SMEM_TRI);
    });
    const bool pair = !ba.mag && TN == 256 && tmB_half != nullptr && ba.tiles_m % 2 == 0 &&
                      (g_band_pairs.load() == 1 || (g_band_pairs.load() == 0 && ba.tri != 0)) &&
                      pair_clusters() > 0;
    BandArgs b = ba;
    int rc;
    if ((rc = tri_prepare(b, TN, pair, st))) return rc;
    // work items (see item_coords; S: the most bands the plan may choose)
    const int units = pair ? b.tiles_m / 2 : b.tiles_m;
    const int tiles = b.tri_cum != nullptr ? b.tri_tiles : units * b.tiles_n;
    const int items = b.diag ? tiles * b.S : tiles;
    const bool tt = b.tri_cum != nullptr;
    if (pair) {
        const int clusters = items < pair_clusters() ? items : pair_clusters();
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(2 * (clusters > 0 ? clusters : 1));
        cfg.blockDim = dim3(BandCfg<256, true>::THREADS);
        cfg.dynamicSmemBytes = tt ? BandCfg<256, true>::SMEM_TRI : BandCfg<256, true>::SMEM;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const cudaError_t e =
            tt ? cudaLaunchKernelEx(&cfg, band_gemm_kernel<256, false, true, true>, tmA,
                                    *tmB_half, b)
               : cudaLaunchKernelEx(&cfg, band_gemm_kernel<256, false, true>, tmA, *tmB_half, b);
        if (e != cudaSuccess) return cuda_fail(e, "band_gemm_kernel (CTA pairs)");
        return check_launch("band_gemm_kernel");
    }
    const int grid = items < sm_count() ? (items > 0 ? items : 1) : sm_count();
#define MPDD_BAND(TN_, MAG_, TRI_)                                                          \
    band_gemm_kernel<TN_, MAG_, false, TRI_>                                                \
        <<<grid, BandCfg<TN_>::THREADS, TRI_ ? BandCfg<TN_>::SMEM_TRI : BandCfg<TN_>::SMEM, \
           st>>>(tmA, tmB, b)
    if (b.mag && TN == 256) {
        if (tt) MPDD_BAND(256, true, true);
        else MPDD_BAND(256, true, false);
    } else if (b.mag) {
        if (tt) MPDD_BAND(128, true, true);
        else MPDD_BAND(128, true, false);
    } else if (TN == 256) {
        if (tt) MPDD_BAND(256, false, true);
        else MPDD_BAND(256, false, false);
    } else {
        if (tt) MPDD_BAND(128, false, true);
        else MPDD_BAND(128, false, false);
    }
#undef MPDD_BAND
    return check_launch("band_gemm_kernel");
}

int read_status(const void *ws, int *status) {
    cudaError_t e = cudaStreamSynchronize(tls().stream);
    if (e == cudaSuccess) e = cudaMemcpy(status, ws, sizeof(int), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? 0 : cuda_fail(e, "status read");
}

// The header of the last split-precision call on a workspace, interpreted:
// the certified width (or the plain kernel), and the guaranteed bound of
// max |C - C_exact| / bound.
int split_report(const void *ws, mp_dd_split_info *info) {
    SplitHeader h;
    cudaError_t e = cudaStreamSynchronize(tls().stream);
    if (e == cudaSuccess) e = cudaMemcpy(&h, ws, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "split report read");
    *info = mp_dd_split_info{};
    info->status = h.status;
    info->form = h.form;
    float dmin32;
    memcpy(&dmin32, &h.dmin, 4);
    const double dmin = dmin32;
    info->dmin = dmin;
    if (h.form == 0 || h.ncand < 1 || h.ncand > kMaxCand) {
        info->max_err_est = 0.0;   // no product formed: C := beta C, as the plain path
        return 0;
    }
    const double fin = 0.25 / (double)(h.k > 0 ? h.k : 1);   // final roundings
    int c = -1;
    for (int q = 0; q < h.ncand && c < 0; ++q)
        if (h.dmin >= h.thr[q]) c = q;
    if (c < 0) {
        // the plain kernel: within half the bound (its per-step error, read
        // from its dd multiply-add), plus the final roundings
        info->width_bits = 0;
        info->count = 0;
        info->max_err_est = 0.5 + fin;
        return 0;
    }
    float thr32;
    memcpy(&thr32, &h.thr[c], 4);
    const double thr = thr32;
    info->width_bits = h.width[c];
    info->count = h.count[c];
    // operand rounding: cst 2^(106 - W) / (16 dmin) = (3/4) thr / dmin
    info->max_err_est = (dmin > 0.0 ? 0.75 * thr / dmin : 0.0) + fin;
    return 0;
}

}  // namespace mpdd
