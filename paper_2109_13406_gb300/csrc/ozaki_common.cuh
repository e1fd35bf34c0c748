// Device helpers shared by the split-precision Rgemm forms (slices and
// residues): the power-of-two row/column scale, the exact rounding of a dd
// entry to a 128-bit integer, its balanced base-256 digits, and the per-call
// accuracy certificate (magnitude planes, the header it is kept in, and the
// rule that turns it into a width).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace mpdd {

// ------------------------------------------------------------------ certificate
//
// Every split-precision call first bounds, per output entry, the error its
// rounded operands can cause against the accuracy target
// 4 k 2^-104 (|alpha||A||B| + |beta||C|)_ij, and only then picks the operand
// width (or hands the product to the plain FP64 kernel).  With e_i, f_j the
// row / column scales and W the width in bits, every product of rounded
// operands is off by at most cst 2^(e_i + f_j - W) (cst per form), so the
// call meets the target with a quarter of it left for the final roundings
// when
//
//   cst 2^(106 - W) / 12  <=  d_ij := L_ij 2^-(e_i+f_j) + |beta/alpha||c_ij| 2^-(e_i+f_j)
//
// for every entry, L_ij a lower bound of (|A||B|)_ij.  L comes from one
// tensor-core product of magnitude planes |hi| 2^-e rounded toward zero to
// bf16, accumulated in fp32 and scaled by (1 - (k+1) 2^-20) (see the
// magnitude kernel and the band kernel's magnitude mode); d_ij is formed in
// fp32 with every step rounded toward zero, and the smallest d_ij of the
// call is kept in the workspace header as its fp32 bit pattern
// (non-negative floats order like their bits).  Every later kernel of the
// call derives the same decision from it with plan_choice().
constexpr int kMaxCand = 3;

// Workspace header (the first bytes of every split-precision workspace).
struct SplitHeader {
    int status;                        // 0, or 2001 when a device wait timed out
    int form;                          // 1 digit slices, 2 residues; 0: no product formed
    int ncand;                         // candidate widths, ascending
    int reserved;
    unsigned int dmin;                 // fp32 bits of min_ij d_ij (+inf: no entry constrains)
    unsigned int reserved2;
    long long k;
    unsigned int thr[kMaxCand];        // fp32 bits of cst_c 2^(106 - W_c) / 12, rounded up
    int count[kMaxCand];               // slices or moduli of candidate c
    int width[kMaxCand];               // W_c in bits
};

// The decision rule as kernel arguments: candidate c is taken when dmin is at
// least thr[c] (the first such c, i.e. the narrowest width); -1: none, the
// plain kernel computes the product.
struct SplitPlan {
    const unsigned int *dmin;          // header word; nullptr: no certificate (count[0])
    unsigned int thr[kMaxCand];
    int count[kMaxCand];
    int width[kMaxCand];
    int ncand;
};

struct PlanPick {
    int c, count, width;   // c = -1: no candidate certifies the bound
};

// (Every index below is a constant after unrolling, so the plan stays in the
// kernel's parameter space instead of being copied to local memory.)
__device__ __forceinline__ PlanPick plan_choice(const SplitPlan &pl) {
    if (pl.dmin == nullptr) return PlanPick{0, pl.count[0], pl.width[0]};
    const unsigned int d = *reinterpret_cast<const volatile unsigned int *>(pl.dmin);
    PlanPick r{-1, 0, 0};
#pragma unroll
    for (int c = kMaxCand - 1; c >= 0; --c)
        if (c < pl.ncand && d >= pl.thr[c]) r = PlanPick{c, pl.count[c], pl.width[c]};
    return r;
}

// One band-product launch.  Triangle mode (diag = 0): band b sums the pairs
// (t, b - t) of digit planes and is stored as int32 in P.  Diagonal mode
// (diag = 1): band b is the single product of planes (b, b) -- the residue
// form -- and is stored reduced modulo moduli[b] as uint8 in R.  Magnitude
// mode (mag = 1, diagonal, one band): the bf16 product of the magnitude
// planes, summed in fp32, turned into the certificate margin d_ij of every
// entry and reduced to its minimum in *dmin_out.  With plan.dmin set, the
// band count is plan.count[plan_choice(plan)] and a failed choice makes the
// launch return at once.
constexpr int kMaxBands = 48;
struct BandArgs {
    int S, kb_count, tiles_m, tiles_n;
    int64_t m_pad, n_pad;
    int32_t *P;   // [S][n_pad][m_pad] (triangle mode)
    uint8_t *R;   // [S][n_pad][m_pad] (diagonal mode)
    int *status;
    int diag;
    int tri;      // diagonal / magnitude mode: 1 / 2 = only the upper / lower triangle
    int moduli[kMaxBands];
    SplitPlan plan;
    // magnitude mode
    int mag;
    int64_t m, n, ldc;
    const unsigned long long *rmax, *cmax;
    const double *ch;          // hi plane of C (read when ba_ratio > 0)
    double ba_ratio;           // lower bound of |beta| / |alpha|, 0 when beta = 0
    float c1;                  // 1 - (k + 1) 2^-20 (exact in fp32): the sums' safety factor
    float ba_ratio32;          // ba_ratio rounded toward zero to fp32
    unsigned int *dmin_out;
    // triangle mode: the work items are the tiles inside the triangle only,
    // in raster order, through a table of cumulative tile counts per
    // (raster group, row unit) (tri_rows + 1 entries in device memory,
    // filled by launch_band); NULL: all tiles, the outside ones skipped
    int *tri_cum;
    int tri_rows, tri_units, tri_tiles;
};

// Tiles inside the triangle, enumerated as the band kernel's raster does: by
// group of `group` tile columns, then by row unit (a tile, or a CTA pair's
// two tiles: R rows), then by column.  For row unit u of group grp the
// inside columns are [lo, hi] (empty when lo > hi), the tiles whose rows and
// columns meet the triangle of C (tri = 1 upper, 2 lower).
constexpr int kTriMax = 4096;   // largest table (entries) the kernel holds in shared memory
struct TriGeom {
    int tri, R, TN, tiles_n, group;
};
__host__ __device__ inline void tri_range(const TriGeom &g, int grp, int u, int &lo, int &hi) {
    const int first = grp * g.group;
    const int last = (first + g.group < g.tiles_n ? first + g.group : g.tiles_n) - 1;
    const long long r0 = (long long)u * g.R;
    if (g.tri == 1) {   // r0 <= c0 + TN - 1: columns from ceil((r0 - TN + 1) / TN)
        const long long t0 = r0 - g.TN + 1;
        const int tmin = t0 <= 0 ? 0 : (int)((t0 + g.TN - 1) / g.TN);
        lo = tmin > first ? tmin : first;
        hi = last;
    } else {            // r0 + R - 1 >= c0: columns up to floor((r0 + R - 1) / TN)
        const int tmax = (int)((r0 + g.R - 1) / g.TN);
        lo = first;
        hi = tmax < last ? tmax : last;
    }
}

// Host launchers shared by the two forms (defined in dd_sliced.cu).
// elem: 0 = fp16, 1 = bf16 elements.
int make_tmap(CUtensorMap *m, void *base, int64_t rows, int64_t k_pad, int box_rows,
              int elem = 0);
int launch_absmax(const double *X, int64_t ld, int row_contig, int64_t rows, int64_t k,
                  unsigned long long *out, cudaStream_t st);
// tmB_half: the op(B) map with TN / 2-row boxes; given for a product that may
// run on CTA pairs (NULL: single CTAs).
int launch_band(const CUtensorMap &tmA, const CUtensorMap &tmB, const BandArgs &ba, int TN,
                cudaStream_t st, const CUtensorMap *tmB_half = nullptr);
constexpr int kBandTM = 128, kBandTK = 64;
int band_tn(int64_t m, int64_t n);

// Magnitude planes and the certificate (dd_sliced.cu).  form: 1 slices, 2
// residues; widths[c] / counts[c] / cst[c] the candidates (ascending width)
// and their per-product error constants.  make_plan also fills the header
// image that the first magnitude launch writes (init != nullptr).
SplitPlan make_plan(SplitHeader *hdr_image, unsigned int *dmin_dev, int form, int64_t k,
                    int ncand, const int *widths, const int *counts, const double *cst);
int launch_magnitude(const double *X, int64_t ld, int row_contig, int64_t rows, int64_t k,
                     int64_t rows_pad, int64_t k_pad, const unsigned long long *rmax, void *M,
                     SplitHeader *hdr, const SplitHeader *init, cudaStream_t st);
// The magnitude product and its reduction into the header (MA [m_pad][k_pad],
// MB [n_pad][k_pad] bf16).
struct GemmArgs;
int launch_certificate(const GemmArgs &p, void *MA, void *MB, int64_t m_pad, int64_t n_pad,
                       int64_t k_pad, int TN, const unsigned long long *rmax,
                       const unsigned long long *cmax, SplitHeader *hdr, cudaStream_t st,
                       int *tri_table = nullptr);
// The plain kernel behind the split-precision call: runs only when the
// certificate fails (plan_choice < 0).
int launch_plain_fallback(const GemmArgs &p, const SplitPlan &plan, cudaStream_t st);

// e with max |x| < 2^(e-1): from the biased exponent E of the maximum,
// max in [2^(E-1023), 2^(E-1022)) -> e = E - 1021 (E = 0, subnormal: same).
__device__ __forceinline__ int scale_exponent(unsigned long long maxbits) {
    if (maxbits == 0) return 0;
    return (int)(maxbits >> 52) - 1021;
}

// ------------------------------------------------------------------ step 2

// RNE(v * 2^s) as a signed 128-bit integer, by integer operations on the
// binary64 fields (|v 2^s| < 2^127 by construction).
__device__ __forceinline__ __int128 scaled_round(double v, int s) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    int E = (int)((bits >> 52) & 0x7FF);
    unsigned long long mant = bits & ((1ull << 52) - 1);
    int ex;
    if (E == 0) {
        ex = 1 - 1075;
    } else {
        mant |= 1ull << 52;
        ex = E - 1075;
    }
    if (mant == 0) return 0;
    int sh = ex + s;
    __int128 r;
    if (sh >= 0) {
        r = (__int128)((unsigned __int128)mant << sh);
    } else {
        int rs = -sh;
        if (rs > 54) {
            r = 0;
        } else {
            unsigned long long q = mant >> rs;
            unsigned long long rem = mant & ((1ull << rs) - 1);
            unsigned long long half = 1ull << (rs - 1);
            if (rem > half || (rem == half && (q & 1))) ++q;
            r = (__int128)q;
        }
    }
    return (bits >> 63) ? -r : r;
}

// Balanced base-256 digits of X = RNE(hi 2^shift) + RNE(lo 2^shift):
// X = sum_t d[t] 256^(S-1-t), d[t] in [-128, 127] for t >= 1, d[0] in
// [-128, 128] (the residue of X mod 256 taken in [-128, 127], carried up).
template <int S>
__device__ __forceinline__ void dd_digits(double hi, double lo, int shift, int (&d)[S]) {
    const __int128 X = scaled_round(hi, shift) + scaled_round(lo, shift);
    const unsigned __int128 u = (unsigned __int128)X;
    int carry = 0;
#pragma unroll
    for (int t = S - 1; t >= 1; --t) {
        int byte = (int)((unsigned)(u >> (8 * (S - 1 - t))) & 0xFFu) + carry;
        carry = byte >= 128;
        d[t] = byte - (carry << 8);
    }
    d[0] = (int)(X >> (8 * (S - 1))) + carry;
}

}  // namespace mpdd
