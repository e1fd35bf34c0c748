// Binary floating point with a 128-bit significand held in four 32-bit
// integer registers: the exact rounding of the residue (CRT) form's
// reconstructed integer to dd.
//
// The reconstructed product Z 2^s is an exact multiword integer; its leading
// 128 bits are taken with integer instructions and rounded to the nearest dd
// (hi = RN(x), lo = RN(x - hi)).  On this GPU an FP64 operation issues at
// about 2 per clock per SM against 64 for integer ALU work, so the rounding
// stays off the FP64 pipe, which the alpha/beta epilogue uses.
//
// Accuracy: the bits below the leading 128 are dropped (relative error below
// 2^-127), so |x - (hi + lo)| <= (2^-106 + 2^-126) |x|.
#pragma once

#include <cstdint>
#include <cstring>

namespace mpdd {
namespace bigf {

#define BF_HD __host__ __device__ __forceinline__

// value = (-1)^neg * M * 2^(e - 127), M = m[3]:m[2]:m[1]:m[0] with bit 127
// set; M = 0 (m[3] == 0) is zero.
struct BF {
    uint32_t m[4];
    int e;
    uint32_t neg;
};

BF_HD int clz32(uint32_t x) {
#if defined(__CUDA_ARCH__)
    return __clz((int)x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

BF_HD int clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

// (hi:lo << s) >> 32 for 0 <= s <= 31.
BF_HD uint32_t fshl(uint32_t lo, uint32_t hi, int s) {
#if defined(__CUDA_ARCH__)
    return __funnelshift_l(lo, hi, s);
#else
    return (uint32_t)(((((uint64_t)hi << 32) | lo) << s) >> 32);
#endif
}
BF_HD double bitsd(uint64_t u) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, 8);
    return x;
#endif
}

BF_HD BF bf_zero() {
    BF r;
    r.m[0] = r.m[1] = r.m[2] = r.m[3] = 0;
    r.e = 0;
    r.neg = 0;
    return r;
}

BF_HD bool is_zero(const BF &a) { return a.m[3] == 0; }

// M << s for 0 <= s < 128.
BF_HD void shl128(uint32_t (&m)[4], int s) {
    if (s <= 0) return;
    const int w = s >> 5, b = s & 31;
    const uint32_t t3 = w == 0 ? m[3] : w == 1 ? m[2] : w == 2 ? m[1] : m[0];
    const uint32_t t2 = w == 0 ? m[2] : w == 1 ? m[1] : w == 2 ? m[0] : 0u;
    const uint32_t t1 = w == 0 ? m[1] : w == 1 ? m[0] : 0u;
    const uint32_t t0 = w == 0 ? m[0] : 0u;
    m[3] = fshl(t2, t3, b);
    m[2] = fshl(t1, t2, b);
    m[1] = fshl(t0, t1, b);
    m[0] = t0 << b;
}

// Leading zeros of the 128-bit M (128 for zero).
BF_HD int clz128(const uint32_t (&m)[4]) {
    return m[3] ? clz32(m[3])
                : m[2] ? 32 + clz32(m[2]) : m[1] ? 64 + clz32(m[1]) : m[0] ? 96 + clz32(m[0]) : 128;
}

// |Z| 2^s for the magnitude words z (little endian), with sign neg.  The top
// 128 bits are kept (the bits below them truncated: relative error < 2^-127).
template <int NW>
BF_HD BF from_words(const uint32_t (&z)[NW], uint32_t neg, int s) {
    int p = -1;
#pragma unroll
    for (int t = 0; t < NW; ++t)
        if (z[t] != 0) p = t;
    BF r = bf_zero();
    if (p < 0) return r;
    uint32_t w4 = 0, w3 = 0, w2 = 0, w1 = 0, w0 = 0;
#pragma unroll
    for (int t = 0; t < NW; ++t) {
        if (p == t) {
            w4 = z[t];
            w3 = t >= 1 ? z[t - 1] : 0u;
            w2 = t >= 2 ? z[t - 2] : 0u;
            w1 = t >= 3 ? z[t - 3] : 0u;
            w0 = t >= 4 ? z[t - 4] : 0u;
        }
    }
    const int lz = clz32(w4);
    r.m[3] = fshl(w3, w4, lz);
    r.m[2] = fshl(w2, w3, lz);
    r.m[1] = fshl(w1, w2, lz);
    r.m[0] = fshl(w0, w1, lz);
    r.e = 32 * p + 31 - lz + s;
    r.neg = neg;
    return r;
}

// m 2^e (m < 2^53) as a binary64 with the sign bit sg; the exponent field
// is assembled directly when the result is normal, else (overflow or a
// subnormal result) the FP64 unit scales it.
BF_HD double make_double(uint64_t m, int e, uint32_t sg) {
    if (m == 0) return sg ? -0.0 : 0.0;
    const int top = 63 - clz64(m);
    const int E = top + e + 1023;
    if (top == 52 && E >= 1 && E <= 2046)
        return bitsd(((uint64_t)sg << 63) | ((uint64_t)E << 52) | (m & ((1ull << 52) - 1)));
    // rare: subnormal or overflowing result (m < 2^53 is exact in binary64)
    double x = (double)m;
    int k = e;
    while (k > 1000) {
        x *= 0x1p1000;
        k -= 1000;
    }
    while (k < -1000) {
        x *= 0x1p-1000;
        k += 1000;
    }
    x *= bitsd((uint64_t)(k + 1023) << 52);
    return sg ? -x : x;
}

// The nearest dd: hi = RN(x), lo = RN(x - hi) (ties to even), for the
// 128-bit significand (bits below it are treated as zero).
BF_HD void to_dd(const BF &x, double &hi, double &lo) {
    if (is_zero(x)) {
        hi = 0.0;
        lo = 0.0;
        return;
    }
    // hi: significand bits 127..75; round bit 74; the remainder R = bits 0..74
    uint64_t mh = ((uint64_t)x.m[3] << 21) | (x.m[2] >> 11);
    const uint32_t r2 = x.m[2] & 0x7FFu, r1 = x.m[1], r0 = x.m[0];
    const bool rbit = (r2 >> 10) & 1u;
    const bool sticky = (r2 & 0x3FFu) | r1 | r0;
    const bool up = rbit && (sticky || (mh & 1u));
    // |x - hi| in units of 2^(e - 127): R, or 2^75 - R when rounded up
    uint32_t l2 = r2, l1 = r1, l0 = r0;
    if (up) {
        uint64_t d = (uint64_t)0 - r0;
        l0 = (uint32_t)d;
        d = (uint64_t)0 - r1 - (d >> 63);
        l1 = (uint32_t)d;
        d = (uint64_t)0x800u - r2 - (d >> 63);
        l2 = (uint32_t)d;
        mh += 1;
    }
    hi = make_double(mh, x.e - 52, x.neg);   // mh <= 2^53: exact
    // lo = RN(L 2^(e - 127)), L < 2^75 in l2:l1:l0
    const uint32_t lsg = x.neg ^ (up ? 1u : 0u);
    uint32_t m[4] = {l0, l1, l2, 0u};
    const int lz = clz128(m);
    if (lz == 128) {
        lo = 0.0;
        return;
    }
    shl128(m, lz);                               // L's leading bit at 127
    uint64_t ml = ((uint64_t)m[3] << 21) | (m[2] >> 11);
    const bool lr = (m[2] >> 10) & 1u;
    const bool ls = (m[2] & 0x3FFu) | m[1] | m[0];
    if (lr && (ls || (ml & 1u))) ml += 1;
    // L's leading bit is bit (127 - lz) of the frame 2^(e - 127)
    lo = make_double(ml, x.e - 127 + (127 - lz) - 52, lsg);
}

#undef BF_HD

}  // namespace bigf
}  // namespace mpdd
