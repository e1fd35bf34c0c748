// Device double-double arithmetic.
//
// A dd value is hi + lo with |lo| <= ulp(hi)/2 (the manual's dd format,
// Sec. 5: Knuth's TwoSum and Dekker's exact product on binary64).  Every
// operation here is written with the explicitly rounded intrinsics
// __dadd_rn / __dsub_rn / __dmul_rn / __fma_rn: the compiler never fuses or
// reassociates them, which the error-free transformations rely on (the
// manual's compiler note asks for the same: no value-changing FP
// optimisation for dd code).
#pragma once

namespace mpdd {

struct dd {
    double hi, lo;
};

// Knuth TwoSum: s + e == a + b exactly, s = fl(a + b).  6 FP64 operations.
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

// Dekker FastTwoSum (|a| >= |b| or a == 0): s + e == a + b.  3 operations.
__device__ __forceinline__ void fast_two_sum(double a, double b, double &s, double &e) {
    s = __dadd_rn(a, b);
    e = __dsub_rn(b, __dsub_rn(s, a));
}

// Product terms of a*b: p = fl(ah*bh), e = its exact error plus the two
// cross products ah*bl + al*bh (al*bl, below 2^-106 relative, is dropped).
// 1 DMUL + 3 DFMA.
__device__ __forceinline__ void prod_terms(dd a, dd b, double &p, double &e) {
    p = __dmul_rn(a.hi, b.hi);
    e = __fma_rn(a.hi, b.hi, -p);
    e = __fma_rn(a.hi, b.lo, e);
    e = __fma_rn(a.lo, b.hi, e);
}

// acc += (p + e), renormalised: TwoSum on the leading parts, the low parts
// added, FastTwoSum.  11 FP64 operations; absolute error at most ~2u^2
// (|acc| + |p|) per step (u = 2^-53).
__device__ __forceinline__ void acc_add(dd &acc, double p, double e) {
    double s, t;
    two_sum(acc.hi, p, s, t);
    t = __dadd_rn(t, __dadd_rn(acc.lo, e));
    fast_two_sum(s, t, acc.hi, acc.lo);
}

// One dd multiply-add: acc += a * b (15 FP64 operations).
__device__ __forceinline__ void mac(dd &acc, dd a, dd b) {
    double p, e;
    prod_terms(a, b, p, e);
    acc_add(acc, p, e);
}

// GEMM-loop multiply-add with deferred renormalisation: the leading parts
// are summed with TwoSum (exact), the TwoSum error and the product's low
// part are added into acc.lo, and the FastTwoSum is left to renorm(), which
// the GEMM kernels call after every kRenormEvery steps of k (at l = 3, 7, 11,
// ... counted from the start of k, so every kernel renormalises at the same
// places).  4 + 6 + 2 = 12 FP64 operations per step, 12.75 with the
// renormalisation.  Between renormalisations |acc.lo| stays within a few
// ulps of acc.hi, so each step's rounding error is at most ~(G+4) u^2
// (|acc| + |a b|) with G = 4: within the Rgemm bound 4 k 2^-104 (...).  A
// zero product leaves the state unchanged, so zero padding of k does not
// alter the result.
constexpr int kRenormEvery = 4;

__device__ __forceinline__ void mac_deferred(dd &acc, dd a, dd b) {
    double p, e, s, e1;
    prod_terms(a, b, p, e);
    two_sum(acc.hi, p, s, e1);
    acc.hi = s;
    acc.lo = __dadd_rn(acc.lo, __dadd_rn(e1, e));
}

__device__ __forceinline__ void renorm(dd &acc) { fast_two_sum(acc.hi, acc.lo, acc.hi, acc.lo); }

// dd product, renormalised.
__device__ __forceinline__ dd mul(dd a, dd b) {
    double p, e;
    prod_terms(a, b, p, e);
    dd r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// Accurate dd addition (two TwoSums, two renormalisations): relative error
// at most 3u^2 + 13u^3.
__device__ __forceinline__ dd add(dd a, dd b) {
    double s1, s2, t1, t2;
    two_sum(a.hi, b.hi, s1, s2);
    two_sum(a.lo, b.lo, t1, t2);
    s2 = __dadd_rn(s2, t1);
    fast_two_sum(s1, s2, s1, s2);
    s2 = __dadd_rn(s2, t2);
    dd r;
    fast_two_sum(s1, s2, r.hi, r.lo);
    return r;
}

// Sloppy dd addition (TwoSum on the leading parts, low parts added,
// FastTwoSum): 11 FP64 operations, absolute error at most ~2u^2 (|a| + |b|)
// (the relative error can be large under cancellation).  Used where the
// accuracy target is the absolute bound 4 k 2^-104 (|alpha||A||B| +
// |beta||C|), e.g. the final alpha/beta combination.
__device__ __forceinline__ dd add_sloppy(dd a, dd b) {
    double s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __dadd_rn(e, __dadd_rn(a.lo, b.lo));
    dd r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ dd neg(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd sub(dd a, dd b) { return add(a, neg(b)); }

// dd division by two steps of long division.  q1 = RN(a.hi / b.hi); the
// remainder of a correctly rounded quotient, a.hi - q1 b.hi, is a binary64
// number, so one FMA gives it exactly; the rest of a - q1 b (a.lo - q1 b.lo)
// is added with two roundings, and q2 = RN(remainder / b.hi).  Relative
// error at most ~11 u^2 (u = 2^-53).  When a and b are binary64 numbers
// (a.lo = b.lo = 0) whose quotient is one too, q1 is that quotient, the
// remainder is 0 and the result exact.  The dependent chain is two
// divisions and five FP64 operations: this is what the row-serial
// triangular solves and the Cholesky pivots wait on.
__device__ __forceinline__ dd div(dd a, dd b) {
    const double q1 = __ddiv_rn(a.hi, b.hi);
    double r = __fma_rn(-q1, b.hi, a.hi);
    r = __dadd_rn(r, __fma_rn(-q1, b.lo, a.lo));
    const double q2 = __ddiv_rn(r, b.hi);
    dd q;
    fast_two_sum(q1, q2, q.hi, q.lo);
    return q;
}

// dd division with a given approximate reciprocal y of b.hi (within a few
// ulps): div's long division with the second quotient digit taken as
// remainder * y instead of a second binary64 division, so the dependent
// chain holds one division.  The second digit's extra relative error (a few
// u) is scaled by |q2| <= ~3u |a / b|: the result's relative error stays
// at most ~20 u^2, and an exactly representable quotient of binary64
// operands is still exact (its remainder is 0).  a need not be
// renormalised: |a.lo| may be a few ulps of a.hi.
__device__ __forceinline__ dd div_rcp(dd a, dd b, double y) {
    const double q1 = __ddiv_rn(a.hi, b.hi);
    double r = __fma_rn(-q1, b.hi, a.hi);
    r = __dadd_rn(r, __fma_rn(-q1, b.lo, a.lo));
    const double q2 = __dmul_rn(r, y);
    dd q;
    fast_two_sum(q1, q2, q.hi, q.lo);
    return q;
}

// dd reciprocal 1 / b: div(1, b) with the first digit RN(1 / b.hi) from
// the correctly rounded reciprocal (the same number as the division gives)
// and the second taken by it as well: one reciprocal, five FP64 operations.
__device__ __forceinline__ dd rcp_dd(dd b) {
    const double y = __drcp_rn(b.hi);
    double r = __fma_rn(-y, b.hi, 1.0);
    r = __fma_rn(-y, b.lo, r);
    dd q;
    fast_two_sum(y, __dmul_rn(r, y), q.hi, q.lo);
    return q;
}

// dd square root: x = RN(sqrt(a.hi)), whose remainder a.hi - x^2 is a
// binary64 number (one FMA gives it exactly), plus one Newton correction
// (a - x^2) / (2x) with a.lo added, the division taken as a product with
// z = rsqrt(a.hi) (1 ulp); the neglected second-order term is below u^2 / 8
// relative.  Exact when a.hi is the square of a binary64 number and a.lo =
// 0.  z, an approximate reciprocal of the result's leading part within a
// few ulps, is returned for div_rcp.  a need not be renormalised.  Returns
// 0 (and z = 0) for a <= 0.
__device__ __forceinline__ dd sqrt_dd(dd a, double &z) {
    z = 0.0;
    if (!(a.hi > 0.0)) return dd{0.0, 0.0};
    const double x = __dsqrt_rn(a.hi);
    z = rsqrt(a.hi);
    const double r = __dadd_rn(__fma_rn(-x, x, a.hi), a.lo);
    const double corr = __dmul_rn(__dmul_rn(r, z), 0.5);
    dd s;
    fast_two_sum(x, corr, s.hi, s.lo);
    return s;
}

}  // namespace mpdd
