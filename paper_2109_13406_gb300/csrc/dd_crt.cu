// Residue (CRT) form of the split-precision dd Rgemm on the fp16 tensor cores.
//
// The exact integers of the sliced form at a width of W = 8D bits --
// X = RNE(hi 2^(W - e)) + RNE(lo 2^(W - e)) for an entry x = hi + lo of a row
// of op(A) with scale e (and likewise for the columns of op(B)),
// |X| < 2^(W-1) -- are multiplied exactly through the Chinese remainder
// theorem instead of through digit pairs:
//
//  1. residues: r_i = X mod p_i in the symmetric range (|r_i| <= 128) for
//     N pairwise coprime moduli p_i <= 256, stored as exact fp16 planes;
//  2. products: C_i = R^A_i (R^B_i)^T on the tensor cores with the exact
//     fp32-run / int32 accumulation of the band kernel (diagonal mode), each
//     stored reduced mod p_i (one byte);
//  3. reconstruction: C' = sum_i c_i w_i mod P with P = prod p_i and the CRT
//     weights w_i = (P/p_i) ((P/p_i)^-1 mod p_i), in multiword integer
//     arithmetic, mapped to the symmetric range; since P >= k 2^(2W) >
//     4 |A' B'|, C' is exactly the integer product A'B'; it is rounded once
//     to dd, scaled by 2^(e_i + f_j - 2W), and alpha/beta are applied in dd.
//
// The only error is the rounding of A and B to W bits: at most
// (1 + 2^-W) 2^(e_i + f_j - W) per product.  Each call certifies it against
// the accuracy bound before choosing W (ozaki_common.cuh): 112 bits (D = 14
// digits, 32 moduli at k = 8192) when that suffices, else 120 or 128 bits
// (more moduli), else the plain FP64 kernel computes the product.  N is the
// smallest even count with P >= k 2^(2W), against S(S+1)/2 = 105 pair
// products of the 14-digit sliced form at W = 112.
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "bigfloat.cuh"
#include "common.cuh"
#include "dd_arith.cuh"
#include "kernels.cuh"
#include "ozaki_common.cuh"

namespace mpdd {
namespace {

constexpr int kMinDigits = 14;        // X has D base-256 digits, W = 8 D bits
constexpr int kMaxDigits = 16;        // |X| < 2^127: a signed 128-bit integer
constexpr int kMaxMod = 40;
constexpr int kWords = 11;           // 32-bit words for sums below 2^352
// pairwise coprime moduli <= 256, largest first: 2^8, 3*5*17, 11*23, 13*19
// and primes not dividing those
__host__ __device__ constexpr int modulus(int i) {
    constexpr int m[kMaxMod] = {256, 255, 253, 251, 247, 241, 239, 233, 229, 227,
                                223, 211, 199, 197, 193, 191, 181, 179, 173, 167,
                                163, 157, 151, 149, 139, 137, 131, 127, 113, 109,
                                107, 103, 101, 97,  89,  83,  79,  73,  71,  67};
    return m[i];
}

// 256^(kMaxDigits-1-u) mod p_i as exact floats (< 256), and 1/p_i.  Digit t
// of a D-digit expansion has the weight w[i][kMaxDigits - D + t].
struct ModWeights {
    float w[kMaxMod][kMaxDigits];
    float inv[kMaxMod];
};

constexpr ModWeights make_mod_weights() {
    ModWeights mw{};
    for (int i = 0; i < kMaxMod; ++i) {
        const int p = modulus(i);
        int v = 1;
        for (int t = kMaxDigits - 1; t >= 0; --t) {
            mw.w[i][t] = (float)v;
            v = (v * 256) % p;
        }
        mw.inv[i] = 1.0f / (float)p;
    }
    return mw;
}

__constant__ ModWeights c_mod_weights = make_mod_weights();

// The same weights, each duplicated into both halves of a float2, with the
// packed constants of the quotient step: the residue kernel works on two
// entries at once with the packed fp32 instructions (f32x2), whose lanes are
// the same IEEE operations as the scalar ones.
struct ModWeights2 {
    float2 w[kMaxMod][kMaxDigits];
    float2 inv[kMaxMod];
    float2 negp[kMaxMod];
};

constexpr ModWeights2 make_mod_weights2() {
    ModWeights2 m{};
    const ModWeights s = make_mod_weights();
    for (int i = 0; i < kMaxMod; ++i) {
        for (int t = 0; t < kMaxDigits; ++t) m.w[i][t] = float2{s.w[i][t], s.w[i][t]};
        m.inv[i] = float2{s.inv[i], s.inv[i]};
        m.negp[i] = float2{-(float)modulus(i), -(float)modulus(i)};
    }
    return m;
}

__constant__ ModWeights2 c_mod_weights2 = make_mod_weights2();

// Residues of an op(X) whose rows are contiguous in memory, on the FP32
// pipe: 4 threads per (row, 16 consecutive k), 4 entries each, one 8-byte store
// per residue plane and thread (a quad of lanes writes one 32-byte sector).
// Residues from the balanced digits d_t of X on the FP32 pipe:
// s = sum_t d_t (256^(D-1-t) mod p) is an integer below 16 * 128 * 255 < 2^24,
// so every partial sum is exact in fp32, and r = s - p rint(s / p) is the
// residue in [-(p-1)/2, (p-1)/2] for odd p: the fp32 quotient is within
// |s / p| 2^-23 < 1e-3 of s / p, while s / p, an integer over an odd p, is
// never within 1 / (2 p) > 0.0019 of a half-integer.  For p = 256 the
// lowest digit, in [-128, 127], is the residue.  The first N planes are
// written (N and D from the call's certificate).
template <int NP, int DG>
__device__ __forceinline__ void residue_rows_body(
    const double *__restrict__ Xh, const double *__restrict__ Xl, int64_t ld, int row_contig,
    int64_t rows, int64_t k, int64_t rows_pad, int64_t k_pad,
    const unsigned long long *__restrict__ rmax, __half *__restrict__ R, int N) {
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 4) + threadIdx.x / 4;
    if (r >= rows_pad) return;
    const int64_t l0 = (int64_t)blockIdx.y * 16 + 4 * (threadIdx.x & 3);
    const int e = r < rows ? scale_exponent(rmax[r]) : 0;
    const int shift = 8 * DG - e;
    // digits of the entry pairs (l0, l0 + 1) and (l0 + 2, l0 + 3), packed
    float2 d2[2][DG];
    int lowest[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int dg[2][DG];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t l = l0 + 2 * h + u;
            double hi = 0.0, lo = 0.0;
            if (r < rows && l < k) {
                const int64_t off = row_contig ? (r + l * ld) : (l + r * ld);
                hi = Xh[off];
                lo = Xl[off];
            }
            dd_digits<DG>(hi, lo, shift, dg[u]);
            lowest[2 * h + u] = dg[u][DG - 1];
        }
        // d as a float without a conversion instruction: the bits of
        // 2^23 + 128 + d (exact, d in [-128, 128]) minus 2^23 + 128
#pragma unroll
        for (int t = 0; t < DG; ++t)
            d2[h][t] = __fadd2_rn(float2{__int_as_float(0x4B000000 + 128 + dg[0][t]),
                                         __int_as_float(0x4B000000 + 128 + dg[1][t])},
                                  float2{-8388736.0f, -8388736.0f});
    }
    // plane 0 (p = 256): the lowest digits, exact in fp16
    {
        const __half2 h01 = __floats2half2_rn((float)lowest[0], (float)lowest[1]);
        const __half2 h23 = __floats2half2_rn((float)lowest[2], (float)lowest[3]);
        *reinterpret_cast<uint2 *>(R + r * k_pad + l0) =
            make_uint2(*reinterpret_cast<const uint32_t *>(&h01),
                       *reinterpret_cast<const uint32_t *>(&h23));
    }
    const float2 magic{12582912.0f, 12582912.0f}, nmagic{-12582912.0f, -12582912.0f};
#pragma unroll
    for (int i = 1; i < 2 * NP; ++i) {
        if (i >= N) break;
        uint32_t packed[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 s2{0.0f, 0.0f};
#pragma unroll
            for (int t = 0; t < DG; ++t)
                s2 = __ffma2_rn(d2[h][t], c_mod_weights2.w[i][kMaxDigits - DG + t], s2);
            // rint(s / p) by the 1.5 2^23 shift (|s / p| < 2^22), then the residue
            const float2 qn = __fadd2_rn(__ffma2_rn(s2, c_mod_weights2.inv[i], magic), nmagic);
            const float2 res = __ffma2_rn(c_mod_weights2.negp[i], qn, s2);
            const __half2 hv = __float22half2_rn(res);
            packed[h] = *reinterpret_cast<const uint32_t *>(&hv);
        }
        *reinterpret_cast<uint2 *>(R + ((int64_t)i * rows_pad + r) * k_pad + l0) =
            make_uint2(packed[0], packed[1]);
    }
}

template <int NP>
__global__ void __launch_bounds__(128) residue_rows_kernel(
    const double *__restrict__ Xh, const double *__restrict__ Xl, int64_t ld, int row_contig,
    int64_t rows, int64_t k, int64_t rows_pad, int64_t k_pad,
    const unsigned long long *__restrict__ rmax, __half *__restrict__ R, const SplitPlan plan) {
    const PlanPick pk = plan_choice(plan);
    if (pk.c < 0) return;
    const int N = pk.count;
    switch (pk.width) {
        case 8 * 14:
            residue_rows_body<NP, 14>(Xh, Xl, ld, row_contig, rows, k, rows_pad, k_pad, rmax, R, N);
            break;
        case 8 * 15:
            residue_rows_body<NP, 15>(Xh, Xl, ld, row_contig, rows, k, rows_pad, k_pad, rmax, R, N);
            break;
        default:
            residue_rows_body<NP, 16>(Xh, Xl, ld, row_contig, rows, k, rows_pad, k_pad, rmax, R, N);
            break;
    }
}

// Residues on the tensor cores.  For an entry X (the scaled integer of
// RNE(hi 2^s) + RNE(lo 2^s), |X| < 2^(8D-1) for D digit bytes) the biased
// X' = X + 2^(8D-1) has D unsigned bytes x_t, and
//     s_b = sum_t x_t (256^t mod p_b) - (2^(8D-1) mod p_b)
// is congruent to X mod p_b with -255 <= s_b < 16 255^2 < 2^22.  Over 16
// entries the sums are the product [16 entries x 16 bytes] x [16 bytes x 8
// moduli], done by mma.sync m16n8k16: a byte is the fp16 1024 + x_t (exact)
// and the fp32 accumulator of modulus b starts at -1024 sum_t (256^t mod
// p_b) - (2^(8D-1) mod p_b), so it ends at exactly s_b (every partial sum an
// integer below 2^23 in magnitude).  r = s - p rint(s / p) is then the
// residue in [-(p-1)/2, (p-1)/2] for odd p: the fp32 quotient is within
// |s / p| 2^-23 of s / p, below 1 / (2 p), while s / p, an integer over an
// odd p, is never within 1 / (2 p) of a half-integer.  For p = 256 the
// lowest byte of X, taken in [-128, 127], is the residue.  Moduli 1 .. N-1
// sit in n-tiles of 8; the first N planes are written (N and D from the
// call's certificate).
//
// A warp computes 32 entries: each lane forms X' of one entry, and the quad
// exchanges words so that lane (g, q) holds bytes 2q, 2q+1, 2q+8, 2q+9 of
// its four entries (the A fragments of two m16 tiles); its accumulators
// then hold two moduli of four consecutive k, stored as one 8-byte write
// per modulus.  Entries: rows r, columns l of op(X); with l contiguous in
// memory (row_contig = 0) a warp takes 32 consecutive l of one row, else 4
// consecutive l of 8 consecutive rows.
constexpr int kResNT = (kMaxMod - 1 + 7) / 8;   // n-tiles of moduli 1 .. 39

// D = A B + C for one m16n8k16 tile: fp16 A (row) and B (col), fp32 C / D.
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint2 b,
                                          const float (&c)[4]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%10,%11,%12,%13};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y), "f"(c[0]), "f"(c[1]),
          "f"(c[2]), "f"(c[3]));
}

struct ResLane {     // per n-tile and lane: B fragment, accumulator starts,
    uint32_t b0, b1; // and the reduction constants of the lane's 2 moduli
    float init0, init1;
    float4 inv, negp;   // {1/p0, 1/p0, 1/p1, 1/p1}, {-p0, -p0, -p1, -p1}
};

__device__ __forceinline__ uint32_t res_weight(int b, int t, int N, int DG) {
    // 256^t mod p_b (0 past N or past the digit count); plane 0 is not here
    return (b < N && t < DG) ? (uint32_t)c_mod_weights.w[b][kMaxDigits - 1 - t] : 0u;
}

__device__ void res_setup(int N, int DG, ResLane *tab) {
    for (int x = threadIdx.x; x < kResNT * 32; x += blockDim.x) {
        const int lane = x % 32, nt = x / 32, g = lane >> 2, q = lane & 3;
        const int bm = 1 + 8 * nt + g;   // B column g
        auto h = [&](int t) {
            return (uint32_t)__half_as_ushort(__uint2half_rn(res_weight(bm, t, N, DG)));
        };
        ResLane L;
        L.b0 = h(2 * q) | (h(2 * q + 1) << 16);
        L.b1 = h(2 * q + 8) | (h(2 * q + 9) << 16);
        float init[2], inv[2], negp[2];
        for (int e = 0; e < 2; ++e) {
            const int m = 1 + 8 * nt + 2 * q + e;   // C column 2q + e
            init[e] = inv[e] = negp[e] = 0.0f;
            if (m < N) {
                const int pm = modulus(m);
                uint32_t ws = 0;
                for (int t = 0; t < DG; ++t) ws += res_weight(m, t, N, DG);
                const uint32_t bias = (128u * res_weight(m, DG - 1, N, DG)) % (uint32_t)pm;
                init[e] = -1024.0f * (float)ws - (float)bias;   // exact: below 2^23
                inv[e] = c_mod_weights.inv[m];
                negp[e] = -(float)pm;
            }
        }
        L.init0 = init[0];
        L.init1 = init[1];
        L.inv = make_float4(inv[0], inv[0], inv[1], inv[1]);
        L.negp = make_float4(negp[0], negp[0], negp[1], negp[1]);
        tab[x] = L;
    }
}

template <int DG>
__device__ __forceinline__ void residue_warp(
    const double *__restrict__ Xh, const double *__restrict__ Xl, int64_t ld, int row_contig,
    int64_t rows, int64_t k, int64_t rows_pad, int64_t k_pad,
    const unsigned long long *__restrict__ rmax, __half *__restrict__ R, int N,
    const ResLane *tab) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int64_t lchunks = row_contig ? k_pad / 4 : k_pad / 32;
    const int64_t items = row_contig ? (rows_pad / 8) * lchunks : rows_pad * lchunks;
    const int ntiles = (N - 1 + 7) / 8;
    const uint32_t sel = (q & 1) ? 0x4342u : 0x4140u;   // halfword q&1 as two fp16 1024 + x
    const float2 magic{12582912.0f, 12582912.0f}, nmagic{-12582912.0f, -12582912.0f};
    for (int64_t item = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; item < items;
         item += (int64_t)gridDim.x * (blockDim.x / 32)) {
        // this lane's entry and the four entries (same row, consecutive l) it stores
        const int64_t a = item / lchunks, c = item - a * lchunks;
        const int64_t row = row_contig ? 8 * a + g : a;
        const int64_t lbase = row_contig ? 4 * c : 32 * c + 4 * g;
        const int64_t l = lbase + q;
        double hi = 0.0, lo = 0.0;
        int e = 0;
        if (row < rows) {
            e = scale_exponent(rmax[row]);
            if (l < k) {
                const int64_t off = row_contig ? (row + l * ld) : (l + row * ld);
                hi = Xh[off];
                lo = Xl[off];
            }
        }
        const int shift = 8 * DG - e;
        const unsigned __int128 Xb = (unsigned __int128)(scaled_round(hi, shift) +
                                                         scaled_round(lo, shift)) +
                                     ((unsigned __int128)1 << (8 * DG - 1));
        const uint32_t w0 = (uint32_t)Xb, w1 = (uint32_t)(Xb >> 32), w2 = (uint32_t)(Xb >> 64),
                       w3 = (uint32_t)(Xb >> 96);
        // words q/2 and 2 + q/2 of the quad's four entries
        uint32_t lw[4], hw[4];
#pragma unroll
        for (int E = 0; E < 4; ++E) {
            const int src = (lane & ~3) | E;
            const uint32_t x0 = __shfl_sync(0xFFFFFFFFu, w0, src);
            const uint32_t x1 = __shfl_sync(0xFFFFFFFFu, w1, src);
            const uint32_t x2 = __shfl_sync(0xFFFFFFFFu, w2, src);
            const uint32_t x3 = __shfl_sync(0xFFFFFFFFu, w3, src);
            lw[E] = (q >> 1) ? x1 : x0;
            hw[E] = (q >> 1) ? x3 : x2;
        }
        // plane 0 (p = 256): the lowest byte of X, signed; lane q = 0 holds it for all four
        if (q == 0) {
            const __half2 h01 = __floats2half2_rn((float)(int8_t)(lw[0] & 0xFFu),
                                                  (float)(int8_t)(lw[1] & 0xFFu));
            const __half2 h23 = __floats2half2_rn((float)(int8_t)(lw[2] & 0xFFu),
                                                  (float)(int8_t)(lw[3] & 0xFFu));
            *reinterpret_cast<uint2 *>(R + row * k_pad + lbase) =
                make_uint2(*reinterpret_cast<const uint32_t *>(&h01),
                           *reinterpret_cast<const uint32_t *>(&h23));
        }
        // A fragments of tile t: row g = entry 2t, row g + 8 = entry 2t + 1
        uint32_t A[2][4];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            A[t][0] = __byte_perm(lw[2 * t], 0x64646464u, sel);
            A[t][1] = __byte_perm(lw[2 * t + 1], 0x64646464u, sel);
            A[t][2] = __byte_perm(hw[2 * t], 0x64646464u, sel);
            A[t][3] = __byte_perm(hw[2 * t + 1], 0x64646464u, sel);
        }
#pragma unroll
        for (int nt = 0; nt < kResNT; ++nt) {
            if (nt >= ntiles) break;
            const ResLane L = tab[nt * 32 + lane];
            const float c0[4] = {L.init0, L.init1, L.init0, L.init1};
            float acc[2][4];
            const uint2 bf = make_uint2(L.b0, L.b1);
#pragma unroll
            for (int t = 0; t < 2; ++t) mma_16816(acc[t], A[t], bf, c0);
            const float2 inv0{L.inv.x, L.inv.y}, inv1{L.inv.z, L.inv.w};
            const float2 np0{L.negp.x, L.negp.y}, np1{L.negp.z, L.negp.w};
#pragma unroll
            for (int e2 = 0; e2 < 2; ++e2) {   // the lane's moduli 1 + 8nt + 2q + e2
                const int m = 1 + 8 * nt + 2 * q + e2;
                uint32_t packed[2];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const float2 s2{acc[t][e2], acc[t][2 + e2]};   // entries 2t, 2t + 1
                    const float2 qn =
                        __fadd2_rn(__ffma2_rn(s2, e2 ? inv1 : inv0, magic), nmagic);
                    const float2 rr = __ffma2_rn(e2 ? np1 : np0, qn, s2);
                    const __half2 hv = __float22half2_rn(rr);
                    packed[t] = *reinterpret_cast<const uint32_t *>(&hv);
                }
                if (m < N)
                    *reinterpret_cast<uint2 *>(R + ((int64_t)m * rows_pad + row) * k_pad + lbase) =
                        make_uint2(packed[0], packed[1]);
            }
        }
    }
}

__global__ void __launch_bounds__(256) residue_kernel(
    const double *__restrict__ Xh, const double *__restrict__ Xl, int64_t ld, int row_contig,
    int64_t rows, int64_t k, int64_t rows_pad, int64_t k_pad,
    const unsigned long long *__restrict__ rmax, __half *__restrict__ R, const SplitPlan plan) {
    __shared__ ResLane tab[kResNT * 32];
    const PlanPick pk = plan_choice(plan);
    if (pk.c < 0) return;
    const int N = pk.count, DG = pk.width / 8;
    res_setup(N, DG, tab);
    __syncthreads();
    switch (DG) {
        case 14:
            residue_warp<14>(Xh, Xl, ld, row_contig, rows, k, rows_pad, k_pad, rmax, R, N, tab);
            break;
        case 15:
            residue_warp<15>(Xh, Xl, ld, row_contig, rows, k, rows_pad, k_pad, rmax, R, N, tab);
            break;
        default:
            residue_warp<16>(Xh, Xl, ld, row_contig, rows, k, rows_pad, k_pad, rmax, R, N, tab);
            break;
    }
}

// ------------------------------------------------------------------ CRT

// Reconstruction constants of one moduli count N.
struct CrtTables {
    uint32_t P[kWords];                   // product of the moduli
    // Byte t of the CRT weights w_b = (P / p_b) ((P / p_b)^-1 mod p_b) of the
    // four moduli b = 4g .. 4g+3, packed in one word (zero past N): the dp4a
    // operand of digit t of the sums.
    uint32_t wp[kMaxMod / 4][4 * kWords];
    // The same for qfix_b = RN(2^24 ((P / p_b)^-1 mod p_b) / p_b), w_b / P in
    // fixed point (three bytes).
    uint32_t qp[kMaxMod / 4][3];
};

struct CrtArgs {
    SplitPlan plan;                       // N and W of the call (tab[c] for candidate c)
    CrtTables tab[kMaxCand];
    int64_t m, n, m_pad, n_pad;
    const uint8_t *res;                   // [N][n_pad][m_pad] products mod p_i
    const unsigned long long *rmax, *cmax;
    mp_dd alpha, beta;
    int alpha_one, beta_zero;
    int ab_mode;                          // 0 general; alpha = +-1 and beta = 0 (1) or 1 (2)
    int alpha_neg;                        // alpha = -1 (modes 1, 2)
    double *ch, *cl;
    int64_t ldc;
    int tri;                              // 0: all of C; 1 / 2: upper / lower triangle
    const int64_t *info;                  // optional: non-zero -> leave C as is
};

// alpha v + beta c in dd with one rounding chain: the two leading products
// split exactly (product and FMA error), their sum by TwoSum, every
// lower-order term added into the error word, one FastTwoSum.  Absolute error
// within about 3u^2 (|alpha v| + |beta c|), u = 2^-53; 20 FP64 operations
// against 25 for two dd products and a dd sum.
__device__ __forceinline__ dd axpby_dd(dd alpha, dd v, dd beta, dd c) {
    const double p1 = __dmul_rn(alpha.hi, v.hi), e1 = __fma_rn(alpha.hi, v.hi, -p1);
    const double p2 = __dmul_rn(beta.hi, c.hi), e2 = __fma_rn(beta.hi, c.hi, -p2);
    double s, t;
    two_sum(p1, p2, s, t);
    const double low = __fma_rn(alpha.hi, v.lo,
                                __fma_rn(alpha.lo, v.hi, __fma_rn(beta.hi, c.lo,
                                                                  __dmul_rn(beta.lo, c.hi))));
    t = __dadd_rn(t, __dadd_rn(__dadd_rn(e1, e2), low));
    dd r;
    fast_two_sum(s, t, r.hi, r.lo);
    return r;
}

// The CRT sums of two adjacent entries (i, j), (i + 1, j) from the N
// products reduced mod p_b: S = sum_b c_b w_b over NW 32-bit words and the
// fixed-point quotient column Q = sum_b c_b qfix_b.  The residues of both
// entries come in one 2-byte load per modulus and are packed four moduli to
// a register, so each byte digit t of the sums is one dp4a per four moduli
// (the digit sums stay below 40 255^2 < 2^22, exact in 32 bits) before the
// digits are carried into words.  T is a reference into the kernel's
// parameter block: the packed weights are constant-bank operands.
constexpr int kCrtGroups = kMaxMod / 4;

// The residues of entries (i, i + 1), i even (2-byte aligned): word h holds
// moduli 2h and 2h + 1 as bytes e0b e1b e0b' e1b' (zero past N).
__device__ __forceinline__ void crt_load_pair(const CrtArgs &p, int N, int64_t i, int64_t j,
                                              uint32_t (&v)[kMaxMod / 2]) {
    const uint8_t *res = p.res + j * p.m_pad + i;
    const int64_t plane = p.n_pad * p.m_pad;
#pragma unroll
    for (int h = 0; h < kMaxMod / 2; ++h) {
        const uint32_t lo = 2 * h < N
            ? (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(res + 2 * h * plane)) : 0u;
        const uint32_t hi = 2 * h + 1 < N
            ? (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(res + (2 * h + 1) * plane))
            : 0u;
        v[h] = lo | (hi << 16);
    }
}

template <int NW>
__device__ __forceinline__ void crt_sums(const CrtTables &T, int N,
                                         const uint32_t (&v)[kMaxMod / 2],
                                         uint32_t (&S0)[NW], uint32_t (&S1)[NW], uint64_t &Q0,
                                         uint64_t &Q1) {
    constexpr int G = kCrtGroups;
    uint32_t R0[G], R1[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        // v[2g] = e0b0 e1b0 e0b1 e1b1, v[2g + 1] = e0b2 e1b2 e0b3 e1b3
        R0[g] = __byte_perm(v[2 * g], v[2 * g + 1], 0x6420);   // entry i: moduli 4g .. 4g+3
        R1[g] = __byte_perm(v[2 * g], v[2 * g + 1], 0x7531);   // entry i + 1
    }
    const int groups = (N + 3) / 4;
    uint64_t c0 = 0, c1 = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        uint32_t d0[4] = {0u, 0u, 0u, 0u}, d1[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g >= groups) break;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                d0[u] = __dp4a(R0[g], T.wp[g][4 * k + u], d0[u]);
                d1[u] = __dp4a(R1[g], T.wp[g][4 * k + u], d1[u]);
            }
        }
        // word k: d[0] + d[1] 2^8 + d[2] 2^16 + d[3] 2^24 + the carry
        const uint64_t v0 = c0 + (d0[0] + (d0[1] << 8)) + ((uint64_t)(d0[2] + (d0[3] << 8)) << 16);
        const uint64_t v1 = c1 + (d1[0] + (d1[1] << 8)) + ((uint64_t)(d1[2] + (d1[3] << 8)) << 16);
        S0[k] = (uint32_t)v0;
        S1[k] = (uint32_t)v1;
        c0 = v0 >> 32;
        c1 = v1 >> 32;
    }
    uint32_t q0[3] = {0u, 0u, 0u}, q1[3] = {0u, 0u, 0u};
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (g >= groups) break;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            q0[u] = __dp4a(R0[g], T.qp[g][u], q0[u]);
            q1[u] = __dp4a(R1[g], T.qp[g][u], q1[u]);
        }
    }
    Q0 = q0[0] + ((uint64_t)q0[1] << 8) + ((uint64_t)q0[2] << 16);
    Q1 = q1[0] + ((uint64_t)q1[1] << 8) + ((uint64_t)q1[2] << 16);
}

// One output entry from its sums: the symmetric representative of S mod P,
// then the alpha/beta epilogue rounded once to dd.
// NW: 32-bit words of the sums (P < 2^(32 (NW - 1)), and the sum of N
// residues < 256 times the weights < P stays below 2^(32 NW)).
// ch, cl: C(i, j) when the epilogue reads it; rbits, cbits: the row and
// column maxima of op(A) and op(B) (loaded ahead by the caller).
template <int NW>
__device__ __forceinline__ void crt_entry(const CrtArgs &p, const CrtTables &T, int W,
                                          uint32_t (&S)[NW], uint64_t Q, int64_t i, int64_t j,
                                          double ch, double cl, unsigned long long rbits,
                                          unsigned long long cbits) {
    // The symmetric representative is Z = S - q P with q the integer
    // nearest to S / P = sum_b c_b (inv_b / p_b): |Z| < k 2^(2W-2) <= P / 4,
    // and Q 2^-24 is within N 255 2^-25 < 0.0004 of S / P (each qfix_b
    // within 2^-25 of inv_b / p_b), so rounding it gives q.
    const uint64_t q = (Q + (1ull << 23)) >> 24;
    // Z = S - q P in two's complement over NW words (exact: |Z| < 2^(32 NW - 1))
    {
        uint64_t mc = 0, borrow = 0;
#pragma unroll
        for (int t = 0; t < NW; ++t) {
            const uint64_t prod = q * T.P[t] + mc;
            mc = prod >> 32;
            const uint64_t d = (uint64_t)S[t] - (uint32_t)prod - borrow;
            S[t] = (uint32_t)d;
            borrow = (d >> 63) & 1;
        }
    }
    // magnitude and sign
    const bool negative = (S[NW - 1] & 0x80000000u) != 0;
    if (negative) {
        uint64_t c2 = 1;
#pragma unroll
        for (int t = 0; t < NW; ++t) {
            const uint64_t v = (uint64_t)(uint32_t)~S[t] + c2;
            S[t] = (uint32_t)v;
            c2 = v >> 32;
        }
    }
    const int sc = scale_exponent(rbits) + scale_exponent(cbits) - 2 * W;
    // v = Z 2^sc rounded once to dd by integer operations (no FP64), then
    // the alpha / beta epilogue in dd arithmetic
    dd v;
    bigf::to_dd(bigf::from_words<NW>(S, negative ? 1u : 0u, sc), v.hi, v.lo);
    const int64_t off = i + j * p.ldc;
    dd r;
    switch (p.ab_mode) {
        case 1:   // alpha = +-1, beta = 0: the product itself
            r = p.alpha_neg ? dd{-v.hi, -v.lo} : v;
            break;
        case 2:   // alpha = +-1, beta = 1 (every Cholesky update): one dd addition
            r = add_sloppy(dd{ch, cl}, p.alpha_neg ? dd{-v.hi, -v.lo} : v);
            break;
        default:
            if (!p.beta_zero)
                r = axpby_dd(dd{p.alpha.hi, p.alpha.lo}, v, dd{p.beta.hi, p.beta.lo}, dd{ch, cl});
            else
                r = p.alpha_one ? v : mul(dd{p.alpha.hi, p.alpha.lo}, v);
    }
    p.ch[off] = r.hi;
    p.cl[off] = r.lo;
}

// Entry pairs (i, i + 1) of column j, i even (m_pad is even, so the pair's
// residues exist even when i + 1 = m).  (Requesting the next pair's loads
// ahead measured slower: the extra registers cost more occupancy than the
// overlap gains.)
template <int NW>
__device__ __forceinline__ void crt_pair(const CrtArgs &p, const CrtTables &T, int N, int W,
                                         int64_t i, int64_t j) {
    const bool in0 = !((p.tri == 1 && i > j) || (p.tri == 2 && i < j));
    const bool in1 = i + 1 < p.m && !((p.tri == 1 && i + 1 > j) || (p.tri == 2 && i + 1 < j));
    if (!in0 && !in1) return;
    uint32_t v[kMaxMod / 2];
    crt_load_pair(p, N, i, j, v);
    uint32_t S0[NW], S1[NW];
    uint64_t Q0, Q1;
    crt_sums<NW>(T, N, v, S0, S1, Q0, Q1);
    const bool use_c = p.ab_mode == 2 || (p.ab_mode == 0 && !p.beta_zero);
    const unsigned long long cb = __ldg(p.cmax + j);
    if (in0) {
        const int64_t off = i + j * p.ldc;
        crt_entry<NW>(p, T, W, S0, Q0, i, j, use_c ? p.ch[off] : 0.0, use_c ? p.cl[off] : 0.0,
                      __ldg(p.rmax + i), cb);
    }
    if (in1) {
        const int64_t off = i + 1 + j * p.ldc;
        crt_entry<NW>(p, T, W, S1, Q1, i + 1, j, use_c ? p.ch[off] : 0.0,
                      use_c ? p.cl[off] : 0.0, __ldg(p.rmax + i + 1), cb);
    }
}

template <int NW>
__device__ __forceinline__ void crt_loop(const CrtArgs &p, const CrtTables &T, int N, int W) {
    const int64_t mh = (p.m + 1) / 2;
    const int64_t total = mh * p.n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (total <= 0xFFFFFFFFll) {   // 32-bit index arithmetic
        const uint32_t m32 = (uint32_t)mh;
        for (; idx < total; idx += stride) {
            const uint32_t u = (uint32_t)idx, jj = u / m32, ih = u - jj * m32;
            crt_pair<NW>(p, T, N, W, 2 * (int64_t)ih, jj);
        }
        return;
    }
    for (; idx < total; idx += stride) crt_pair<NW>(p, T, N, W, 2 * (idx % mh), idx / mh);
}

// NW0..NW2: words of the sums for the three candidate widths.
template <int NW0, int NW1, int NW2>
__global__ void __launch_bounds__(256) crt_kernel(const __grid_constant__ CrtArgs p) {
    if (p.info != nullptr && *p.info != 0) return;   // an earlier step failed
    const PlanPick pk = plan_choice(p.plan);
    if (pk.c < 0) return;                            // the plain kernel computes C
    if (pk.c == 0) crt_loop<NW0>(p, p.tab[0], pk.count, pk.width);
    else if (pk.c == 1) crt_loop<NW1>(p, p.tab[1], pk.count, pk.width);
    else crt_loop<NW2>(p, p.tab[2], pk.count, pk.width);
}

// ------------------------------------------------------------------ host

// 256-thread blocks of the three crt_kernel instantiations resident per SM
// (occupancy query, once per instantiation; 1 if the query fails).
int crt_resident_blocks(int which) {
    static int cached[3] = {0, 0, 0};
    static std::once_flag once[3];
    std::call_once(once[which], [which] {
        int b = 0;
        const void *f = which == 0 ? (const void *)crt_kernel<8, 9, 10>
                        : which == 1 ? (const void *)crt_kernel<9, 9, 10>
                                     : (const void *)crt_kernel<9, 10, 10>;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, 256, 0) != cudaSuccess) {
            cudaGetLastError();
            b = 0;
        }
        cached[which] = b > 0 ? b : 1;
    });
    return cached[which];
}

// Little-endian multiword helpers (host).
using Big = std::vector<uint32_t>;

Big big_mul_small(const Big &a, uint32_t s) {
    Big r(a.size() + 1, 0);
    uint64_t c = 0;
    for (size_t i = 0; i < a.size(); ++i) {
        uint64_t v = (uint64_t)a[i] * s + c;
        r[i] = (uint32_t)v;
        c = v >> 32;
    }
    r[a.size()] = (uint32_t)c;
    while (r.size() > 1 && r.back() == 0) r.pop_back();
    return r;
}

Big big_div_small(const Big &a, uint32_t s, uint32_t *rem) {
    Big r(a.size(), 0);
    uint64_t c = 0;
    for (size_t i = a.size(); i-- > 0;) {
        uint64_t v = (c << 32) | a[i];
        r[i] = (uint32_t)(v / s);
        c = v % s;
    }
    if (rem) *rem = (uint32_t)c;
    while (r.size() > 1 && r.back() == 0) r.pop_back();
    return r;
}

int big_bits(const Big &a) {
    for (size_t i = a.size(); i-- > 0;)
        if (a[i]) return (int)(32 * i + 32 - __builtin_clz(a[i]));
    return 0;
}

uint32_t inv_mod(uint32_t a, uint32_t p) {   // a^-1 mod p (gcd(a, p) = 1)
    int64_t t = 0, nt = 1, r = p, nr = a % p;
    while (nr) {
        int64_t q = r / nr, tmp = t - q * nt;
        t = nt;
        nt = tmp;
        tmp = r - q * nr;
        r = nr;
        nr = tmp;
    }
    if (t < 0) t += p;
    return (uint32_t)t;
}

// Smallest even moduli count with P >= k 2^(2W) > 4 max |A' B'| (|A'|,
// |B'| < 2^(W-1)); -1 when the 40 moduli do not reach it.
int moduli_count(int64_t k, int W) {
    const int need = 2 * W + (int)std::ceil(std::log2((double)(k > 1 ? k : 1)));
    Big P{1};
    for (int N = 1; N <= kMaxMod; ++N) {
        P = big_mul_small(P, modulus(N - 1));
        if (big_bits(P) > need) {                        // P >= 2^need
            const int even = N % 2 ? N + 1 : N;          // residues come in pairs
            return even <= kMaxMod ? even : -1;
        }
    }
    return -1;
}

// Candidate widths of a call: 112, 120 and 128 bits, with their moduli counts.
int crt_candidates(int64_t k, int *widths, int *counts) {
    int nc = 0;
    for (int D = kMinDigits; D <= kMaxDigits; ++D) {
        const int N = moduli_count(k, 8 * D);
        if (N < 0) break;
        widths[nc] = 8 * D;
        counts[nc] = N;
        ++nc;
    }
    return nc;
}

struct CrtLayout {
    int N;                                 // moduli the workspace holds (the widest candidate)
    int64_t m_pad, n_pad, k_pad;
    size_t off_rowmax, off_colmax, off_ra, off_rb, off_res, off_ma, off_mb, off_tri, total;
};

size_t align1k(size_t x) { return (x + 1023) / 1024 * 1024; }

// Tile width of the residue products: 256 (a quarter fewer operand bytes per
// flop than 128) once the (modulus, tile) work items fill the SMs twice over
// and the wider padding of n adds at most n / 8.
int crt_band_tn(int64_t m, int64_t n, int N) {
    const int64_t items = ceil_div(imax(m, 1), kBandTM) * ceil_div(imax(n, 1), 256) * N;
    const int64_t pad256 = ceil_div(imax(n, 1), 256) * 256;
    const int64_t pad128 = ceil_div(imax(n, 1), 128) * 128;
    return (items >= 2 * 152 && (pad256 - pad128) * 8 <= imax(n, 1)) ? 256 : 128;
}

// sym: the Rsyrk form, op(B) = op(A)^T (m = n): one set of maxima and
// residue planes serves both operands, padded alike (m_pad = n_pad).
CrtLayout crt_layout(int64_t m, int64_t n, int64_t k, bool sym = false) {
    CrtLayout L{};
    int widths[kMaxCand], counts[kMaxCand];
    const int nc = crt_candidates(k, widths, counts);
    L.N = nc > 0 ? counts[nc - 1] : -1;
    const int TN = crt_band_tn(m, n, L.N);
    L.n_pad = ceil_div(imax(n, 1), TN) * TN;
    L.m_pad = sym ? L.n_pad : ceil_div(imax(m, 1), kBandTM) * kBandTM;
    L.k_pad = ceil_div(imax(k, 1), kBandTK) * kBandTK;
    const size_t N = L.N > 0 ? (size_t)L.N : 0;
    size_t o = 1024;
    L.off_rowmax = o; o = align1k(o + 8 * (size_t)L.m_pad);
    L.off_colmax = sym ? L.off_rowmax : o;
    if (!sym) o = align1k(o + 8 * (size_t)L.n_pad);
    L.off_ra = o; o = align1k(o + 2 * N * L.m_pad * L.k_pad);
    L.off_rb = sym ? L.off_ra : o;
    if (!sym) o = align1k(o + 2 * N * L.n_pad * L.k_pad);
    L.off_res = o; o = align1k(o + N * L.n_pad * L.m_pad);
    L.off_ma = o; o = align1k(o + 2 * (size_t)L.m_pad * L.k_pad);
    L.off_mb = sym ? L.off_ma : o;
    if (!sym) o = align1k(o + 2 * (size_t)L.n_pad * L.k_pad);
    L.off_tri = o;   // the band launches' triangle table (Rsyrk form)
    if (sym) o = align1k(o + 4 * (size_t)kTriMax);
    L.total = o;
    return L;
}

template <int NP>
void launch_residues_rows(const double *Xh, const double *Xl, int64_t ld, int rc, int64_t rows,
                        int64_t k, int64_t rows_pad, int64_t k_pad,
                        const unsigned long long *rmax, __half *R, const SplitPlan &plan,
                        cudaStream_t st) {
    dim3 grid((unsigned)ceil_div(rows_pad, 32), (unsigned)(k_pad / 16));
    residue_rows_kernel<NP><<<grid, 128, 0, st>>>(Xh, Xl, ld, rc, rows, k, rows_pad, k_pad, rmax, R,
                                             plan);
}

// Residues for up to Nmax moduli (the plan's widest candidate): one warp
// per 32 entries, blocks resident at once, looping.
int launch_residues(int Nmax, const double *Xh, const double *Xl, int64_t ld, int rc,
                    int64_t rows, int64_t k, int64_t rows_pad, int64_t k_pad,
                    const unsigned long long *rmax, __half *R, const SplitPlan &plan,
                    cudaStream_t st) {
    if (rc) {   // rows contiguous: the FP32 kernel (full-sector stores along k)
        if (k_pad / 16 > 65535) return fail(MP_DD_ERR_TOO_LARGE, "k too large for residues");
        switch (Nmax / 2) {
#define MPDD_RES_CASE(NP)                                                                      \
    case NP:                                                                                   \
        launch_residues_rows<NP>(Xh, Xl, ld, rc, rows, k, rows_pad, k_pad, rmax, R, plan, st); \
        break;
            MPDD_RES_CASE(14) MPDD_RES_CASE(15) MPDD_RES_CASE(16) MPDD_RES_CASE(17)
            MPDD_RES_CASE(18) MPDD_RES_CASE(19) MPDD_RES_CASE(20)
#undef MPDD_RES_CASE
            default:
                return fail(MP_DD_ERR_TOO_LARGE, "residue count %d outside [28, 40]", Nmax);
        }
        return check_launch("residue_rows_kernel");
    }
    if (Nmax < 2 || Nmax > kMaxMod)
        return fail(MP_DD_ERR_TOO_LARGE, "residue count %d outside [2, %d]", Nmax, kMaxMod);
    const int64_t warps = rows_pad * k_pad / 32;
    int64_t blocks = ceil_div(warps, 8);
    if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
    if (blocks < 1) blocks = 1;
    residue_kernel<<<(unsigned)blocks, 256, 0, st>>>(Xh, Xl, ld, rc, rows, k, rows_pad, k_pad,
                                                     rmax, R, plan);
    return check_launch("residue_kernel");
}

// Reconstruction constants for the first N moduli.
int crt_tables(int N, CrtTables &T, int *nwords) {
    memset(&T, 0, sizeof T);
    Big P{1};
    for (int i = 0; i < N; ++i) P = big_mul_small(P, modulus(i));
    if ((int)P.size() > kWords - 1) return fail(MP_DD_ERR_TOO_LARGE, "moduli product too wide");
    for (int t = 0; t < kWords; ++t) T.P[t] = t < (int)P.size() ? P[t] : 0;
    for (int i = 0; i < N; ++i) {
        uint32_t mi_mod = 0;
        Big Mi = big_div_small(P, modulus(i), nullptr);
        big_div_small(Mi, modulus(i), &mi_mod);
        const uint32_t inv = inv_mod(mi_mod, modulus(i));
        Big wi = big_mul_small(Mi, inv);
        const int g = i / 4, sh = 8 * (i % 4);
        for (int t = 0; t < 4 * kWords; ++t) {
            const uint32_t word = t / 4 < (int)wi.size() ? wi[t / 4] : 0u;
            T.wp[g][t] |= ((word >> (8 * (t % 4))) & 0xFFu) << sh;
        }
        const uint32_t qfix = (uint32_t)((((uint64_t)inv << 24) + modulus(i) / 2) / modulus(i));
        for (int t = 0; t < 3; ++t) T.qp[g][t] |= ((qfix >> (8 * t)) & 0xFFu) << sh;
    }
    // words of the sums: S = sum_b c_b w_b < N 255 P, and Z = S - q P takes
    // a sign bit: bits(P) + ceil(log2(255 N)) + 1
    int need = big_bits(P) + 1;
    for (int64_t x = 255LL * N - 1; x > 0; x >>= 1) ++need;
    *nwords = (need + 31) / 32;
    return 0;
}

}  // namespace

size_t crt_workspace_bytes(int64_t m, int64_t n, int64_t k, bool sym) {
    return crt_layout(m, n, k, sym).total;
}

int crt_layout_query(int64_t m, int64_t n, int64_t k, size_t *off, int *count) {
    CrtLayout L = crt_layout(m, n, k);
    off[0] = L.off_rowmax;
    off[1] = L.off_colmax;
    off[2] = L.off_ra;
    off[3] = L.off_rb;
    off[4] = L.off_res;
    off[5] = (size_t)L.m_pad;
    off[6] = (size_t)L.n_pad;
    off[7] = (size_t)L.k_pad;
    *count = L.N;
    for (int i = 0; i < L.N && i < kMaxMod; ++i) off[8 + i] = (size_t)modulus(i);
    return 0;
}

int crt_magnitude_offsets(int64_t m, int64_t n, int64_t k, bool sym, size_t *off) {
    CrtLayout L = crt_layout(m, n, k, sym);
    off[0] = L.off_ma;
    off[1] = L.off_mb;
    return 0;
}

int run_crt(const GemmArgs &p, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (p.k > ((int64_t)1 << 17) - 1)
        return fail(MP_DD_ERR_TOO_LARGE, "k = %lld exceeds 131071 (int32 products)",
                    (long long)p.k);
    // the Rsyrk form: one triangle of op(A) op(A)^T
    const bool sym = p.tri != 0;
    if (sym && (p.m != p.n || p.ah != p.bh || p.al != p.bl || p.lda != p.ldb || p.ta == p.tb))
        return fail(MP_DD_ERR_TOO_LARGE, "CRT Rsyrk: operands are not A and A^T");
    CrtLayout L = crt_layout(p.m, p.n, p.k, sym);
    int widths[kMaxCand], counts[kMaxCand];
    const int ncand = crt_candidates(p.k, widths, counts);
    if (ncand < 1 || L.N < 0 || L.N > kMaxMod)
        return fail(MP_DD_ERR_TOO_LARGE, "k too large for the moduli");
    if (ws == nullptr || ws_bytes < L.total)
        return fail(MP_DD_ERR_WORKSPACE, "CRT Rgemm needs %zu workspace bytes, got %zu",
                    L.total, ws_bytes);
    if ((int64_t)L.N * L.m_pad > 0x7fffffffLL || (int64_t)L.N * L.n_pad > 0x7fffffffLL)
        return fail(MP_DD_ERR_TOO_LARGE, "matrix too large for the CRT path");
    const int TN = crt_band_tn(p.m, p.n, L.N);

    uint8_t *w = static_cast<uint8_t *>(ws);
    cudaError_t e = cudaMemsetAsync(w, 0, L.off_ra, st);   // header (form 0) and maxima
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (p.alpha_zero) return launch_gemm_plain(p, st);
    auto *rmax = reinterpret_cast<unsigned long long *>(w + L.off_rowmax);
    auto *cmax = reinterpret_cast<unsigned long long *>(w + L.off_colmax);
    auto *RA = reinterpret_cast<__half *>(w + L.off_ra);
    auto *RB = reinterpret_cast<__half *>(w + L.off_rb);
    auto *RES = reinterpret_cast<uint8_t *>(w + L.off_res);
    auto *hdr = reinterpret_cast<SplitHeader *>(w);

    double cst[kMaxCand];
    for (int c = 0; c < ncand; ++c) cst[c] = 1.0 + 0x1p-50;   // (1 + 2^-W), rounded up
    SplitHeader init;
    const SplitPlan plan = make_plan(&init, &hdr->dmin, 2, p.k, ncand, widths, counts, cst);

    const int a_rc = p.ta ? 0 : 1, b_rc = p.tb ? 1 : 0;
    int rc;
    sliced_timing_mark(0, st);
    if ((rc = launch_absmax(p.ah, p.lda, a_rc, p.m, p.k, rmax, st))) return rc;
    if (!sym && (rc = launch_absmax(p.bh, p.ldb, b_rc, p.n, p.k, cmax, st))) return rc;
    if ((rc = launch_magnitude(p.ah, p.lda, a_rc, p.m, p.k, L.m_pad, L.k_pad, rmax,
                               w + L.off_ma, hdr, &init, st)))
        return rc;
    if (!sym && (rc = launch_magnitude(p.bh, p.ldb, b_rc, p.n, p.k, L.n_pad, L.k_pad, cmax,
                                       w + L.off_mb, hdr, nullptr, st)))
        return rc;
    int *tri_table = (p.tri && sym) ? reinterpret_cast<int *>(w + L.off_tri) : nullptr;
    if ((rc = launch_certificate(p, w + L.off_ma, w + L.off_mb, L.m_pad, L.n_pad, L.k_pad, TN,
                                 rmax, cmax, hdr, st, tri_table)))
        return rc;
    if ((rc = launch_residues(L.N, p.ah, p.al, p.lda, a_rc, p.m, p.k, L.m_pad, L.k_pad, rmax,
                              RA, plan, st)))
        return rc;
    if (!sym) {   // (the Rsyrk form reuses the maxima and planes of op(A))
        if ((rc = launch_residues(L.N, p.bh, p.bl, p.ldb, b_rc, p.n, p.k, L.n_pad, L.k_pad,
                                  cmax, RB, plan, st)))
            return rc;
    }

    sliced_timing_mark(1, st);
    CUtensorMap tmA, tmB;
    if ((rc = make_tmap(&tmA, RA, (int64_t)L.N * L.m_pad, L.k_pad, kBandTM))) return rc;
    if ((rc = make_tmap(&tmB, RB, (int64_t)L.N * L.n_pad, L.k_pad, TN))) return rc;
    CUtensorMap tmB_half;   // half-height boxes for CTA pairs on 256-wide tiles
    if ((rc = make_tmap(&tmB_half, RB, (int64_t)L.N * L.n_pad, L.k_pad, TN / 2))) return rc;
    BandArgs ba{};
    ba.S = L.N;
    ba.kb_count = (int)(L.k_pad / kBandTK);
    ba.tiles_m = (int)(L.m_pad / kBandTM);
    ba.tiles_n = (int)(L.n_pad / TN);
    ba.m_pad = L.m_pad;
    ba.n_pad = L.n_pad;
    ba.P = nullptr;
    ba.R = RES;
    ba.status = &hdr->status;
    ba.diag = 1;
    ba.tri = p.tri;
    ba.tri_cum = tri_table;
    ba.plan = plan;
    for (int i = 0; i < L.N; ++i) ba.moduli[i] = modulus(i);
    if ((rc = launch_band(tmA, tmB, ba, TN, st, &tmB_half))) return rc;
    sliced_timing_mark(2, st);

    // CRT constants of every candidate
    CrtArgs ca{};
    ca.plan = plan;
    ca.m = p.m; ca.n = p.n; ca.m_pad = L.m_pad; ca.n_pad = L.n_pad;
    ca.res = RES; ca.rmax = rmax; ca.cmax = sym ? rmax : cmax;
    ca.alpha = p.alpha; ca.beta = p.beta;
    ca.alpha_one = p.alpha_one; ca.beta_zero = p.beta_zero;
    ca.ch = p.ch; ca.cl = p.cl; ca.ldc = p.ldc;
    ca.tri = p.tri;
    ca.info = p.info;
    {
        const bool a_pm1 = p.alpha.lo == 0.0 && (p.alpha.hi == 1.0 || p.alpha.hi == -1.0);
        const bool b_one = p.beta.hi == 1.0 && p.beta.lo == 0.0;
        ca.ab_mode = a_pm1 && p.beta_zero ? 1 : (a_pm1 && b_one ? 2 : 0);
        ca.alpha_neg = p.alpha.hi < 0.0;
    }
    int nw[kMaxCand] = {0, 0, 0};
    for (int c = 0; c < ncand; ++c)
        if ((rc = crt_tables(counts[c], ca.tab[c], &nw[c]))) return rc;
    for (int c = ncand; c < kMaxCand; ++c) nw[c] = nw[ncand - 1];   // (never chosen)
    // the word counts that occur for k < 2^17: 8 at 112 bits (9 for the
    // largest k), 9 at 120 bits, 9 or 10 at 128 bits; a kernel with more
    // words than needed gives the same result (the weights are zero-padded)
    if (nw[0] > 9 || nw[1] > 10 || nw[2] > 10)
        return fail(MP_DD_ERR_TOO_LARGE, "CRT word counts %d/%d/%d beyond the kernel's", nw[0],
                    nw[1], nw[2]);
    // one thread per entry pair, looping.  Full products: as many blocks as
    // are resident at once (three per SM at 80 registers; eight per SM left
    // the last two-thirds wave with a third of the slots idle: 3.65-3.68
    // against 3.70-3.73 ms at 8192).  Triangles: eight per SM, which the
    // block scheduler balances over the uneven work of the skipped entries
    // (resident blocks only: 2.61 against 2.41-2.45 ms).
    const int64_t pairs = ceil_div(p.m, 2) * p.n;
    const int which = nw[0] <= 8 && nw[1] <= 9 ? 0 : (nw[1] <= 9 ? 1 : 2);
    int64_t blocks = ceil_div(pairs, 256);
    const int64_t cap = (int64_t)sm_count() * (p.tri ? 8 : crt_resident_blocks(which));
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    const unsigned nb = (unsigned)blocks;
    if (which == 0) crt_kernel<8, 9, 10><<<nb, 256, 0, st>>>(ca);
    else if (which == 1) crt_kernel<9, 9, 10><<<nb, 256, 0, st>>>(ca);
    else crt_kernel<9, 10, 10><<<nb, 256, 0, st>>>(ca);
    if ((rc = check_launch("crt_kernel"))) return rc;
    rc = launch_plain_fallback(p, plan, st);
    sliced_timing_mark(3, st);
    return rc;
}

}  // namespace mpdd
