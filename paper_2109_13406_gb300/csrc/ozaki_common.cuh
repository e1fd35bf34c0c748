// Device helpers shared by the split-precision Rgemm forms (slices and
// residues): the power-of-two row/column scale, the exact rounding of a dd
// entry to a 128-bit integer, and its balanced base-256 digits.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace mpdd {

// One band-product launch.  Triangle mode (diag = 0): band b sums the pairs
// (t, b - t) of digit planes and is stored as int32 in P.  Diagonal mode
// (diag = 1): band b is the single product of planes (b, b) -- the residue
// form -- and is stored reduced modulo moduli[b] as uint8 in R.
constexpr int kMaxBands = 48;
struct BandArgs {
    int S, kb_count, tiles_m, tiles_n;
    int64_t m_pad, n_pad;
    int32_t *P;   // [S][n_pad][m_pad] (triangle mode)
    uint8_t *R;   // [S][n_pad][m_pad] (diagonal mode)
    int *status;
    int diag;
    int tri;      // diagonal mode: 1 / 2 = only tiles meeting the upper / lower triangle
    int moduli[kMaxBands];
};

// Host launchers shared by the two forms (defined in dd_sliced.cu).
int make_tmap(CUtensorMap *m, void *base, int64_t rows, int64_t k_pad, int box_rows);
int launch_absmax(const double *X, int64_t ld, int row_contig, int64_t rows, int64_t k,
                  unsigned long long *out, cudaStream_t st);
int launch_band(const CUtensorMap &tmA, const CUtensorMap &tmB, const BandArgs &ba, int TN,
                cudaStream_t st);
constexpr int kBandTM = 128, kBandTK = 64;
int band_tn(int64_t m, int64_t n);

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
