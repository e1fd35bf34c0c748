"""Oracle for the split-precision (Ozaki-scheme) dd Rgemm.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``); shares nothing with
the CUDA code.  The manual has no split-precision Rgemm: this follows the
method's definition as the library documents it, in exact integer
arithmetic (Python ints and ``fractions``), one function per step:

1. ``scale_exponent``: e with max |hi| < 2^(e-1) for a row of op(A) (a column
   of op(B)); 0 for an all-zero row.
2. ``split_row``: for x = hi + lo, X = RNE(hi 2^(8S-e)) + RNE(lo 2^(8S-e));
   its digits d_0..d_{S-1} with X = sum_t d_t 256^(S-1-t), d_t in
   [-128, 127] for t >= 1 (the residue of X mod 256 taken in that range) and
   d_0 the remaining top part.
3. ``band_products``: P_b = sum_{t+u=b} D_A[t] D_B[u]^T, b < S, exact
   integer matrix products (numpy int64; the values stay far below 2^63).
4. ``recombine_exact``: sum_b P_b 2^(e_i+f_j-8(b+2)) as exact rationals.

5. the residue (CRT) form: ``crt_moduli``, ``residue_planes`` (symmetric
   residues of the same integers X), ``crt_products`` (R^A_i R^B_i^T mod p_i)
   and ``crt_reconstruct`` (the textbook CRT sum mapped to (-P/2, P/2]).
6. the per-call certificate: ``bf16_floor`` / ``magnitude_row`` (the
   magnitude planes), ``product_error_constant`` (the error of one product
   of rounded operands, per form), ``exact_margins`` (the margin of every
   output entry from the exact |A||B|) and ``certified_width`` (the rule
   that turns the smallest margin into an operand width, 0 = none).

Parity status: pinned by ``tests/test_ozaki_oracle.py`` -- digit expansions
reproduce X exactly and stay in range, X approximates x within one unit of
2^(e-8S), the recombined value approximates the exact product within the
documented truncation bound, and it equals the exact product when every
digit beyond the first band is zero (integer and power-of-two inputs); the
CRT reconstruction equals the integer product of the rounded operands, and
the moduli are pairwise coprime; bf16_floor is the largest bf16 below its
argument (brute force over the neighbouring bf16 values); every product of
rounded operands stays within its form's constant times 2^(e_i+f_j-W); and a
certified width keeps the exact error of a call within the bound while the
default width (112 bits) does not on the stress inputs.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def scale_exponent(row_hi) -> int:
    m = max((abs(float(v)) for v in row_hi), default=0.0)
    if m == 0.0:
        return 0
    _, E = math.frexp(m)          # m = f 2^E with 1/2 <= f < 1, so m < 2^E
    return E + 1                  # 2^(e-1) = 2^E > m


def rne_scaled(v: float, s: int) -> int:
    """Round-half-even of v * 2^s to an integer (exact rational arithmetic)."""
    return round(Fraction(v) * (Fraction(2) ** s))


def digits_of(X: int, S: int) -> list[int]:
    d = [0] * S
    for t in range(S - 1, 0, -1):
        r = ((X + 128) % 256) - 128
        d[t] = r
        X = (X - r) // 256
    d[0] = X
    return d


def split_row(hi_row, lo_row, S: int):
    """Digits (S x len) and the exponent of one row of op(A) (column of op(B))."""
    e = scale_exponent(hi_row)
    out = np.zeros((S, len(hi_row)), dtype=np.int64)
    for l, (h, lo) in enumerate(zip(hi_row, lo_row)):
        X = rne_scaled(float(h), 8 * S - e) + rne_scaled(float(lo), 8 * S - e)
        out[:, l] = digits_of(X, S)
    return out, e


def split_matrix(rows_hi: np.ndarray, rows_lo: np.ndarray, S: int):
    """rows x k planes (row r = one row of op(A) or one column of op(B)) ->
    digits [S][rows][k] and exponents [rows]."""
    R, K = rows_hi.shape
    D = np.zeros((S, R, K), dtype=np.int64)
    E = np.zeros(R, dtype=np.int64)
    for r in range(R):
        D[:, r, :], E[r] = split_row(rows_hi[r], rows_lo[r], S)
    return D, E


def band_products(DA: np.ndarray, DB: np.ndarray) -> np.ndarray:
    """P[b] = sum_{t+u=b} DA[t] @ DB[u]^T for b < S (int64)."""
    S = DA.shape[0]
    P = np.zeros((S, DA.shape[1], DB.shape[1]), dtype=np.int64)
    for b in range(S):
        for t in range(b + 1):
            P[b] += DA[t] @ DB[b - t].T
    return P


def recombine_exact(P: np.ndarray, ea, fb):
    """Exact value of sum_b P_b 2^(e_i + f_j - 8(b+2)) per entry (Fractions)."""
    S, m, n = P.shape
    out = [[Fraction(0)] * n for _ in range(m)]
    for i in range(m):
        for j in range(n):
            v = sum(int(P[b, i, j]) * 256 ** (S - 1 - b) for b in range(S))
            out[i][j] = Fraction(v) * Fraction(2) ** (int(ea[i]) + int(fb[j]) - 8 * S - 8)
    return out


def op_rows(X, trans: bool, rows: int, k: int):
    """Rows of op(X) (rows x k) from a column-major stored (hi, lo) pair."""
    h, l = X
    if trans:
        return np.ascontiguousarray(h[:k, :rows].T), np.ascontiguousarray(l[:k, :rows].T)
    return np.ascontiguousarray(h[:rows, :k]), np.ascontiguousarray(l[:rows, :k])


def op_cols(X, trans: bool, k: int, cols: int):
    """Columns of op(X) (k x cols) as rows (cols x k)."""
    h, l = X
    if trans:
        return np.ascontiguousarray(h[:cols, :k]), np.ascontiguousarray(l[:cols, :k])
    return np.ascontiguousarray(h[:k, :cols].T), np.ascontiguousarray(l[:k, :cols].T)


# ----------------------------------------------------------------------------
# Residue (CRT) form: the same rounded integers multiplied through the
# Chinese remainder theorem
# ----------------------------------------------------------------------------

def _is_prime(p: int) -> bool:
    return p > 1 and all(p % d for d in range(2, int(p ** 0.5) + 1))


def crt_moduli(count: int = 40) -> list[int]:
    """Pairwise coprime moduli <= 256, largest first: 2^8, 3*5*17, 11*23,
    13*19, then the primes below 256, in decreasing order, that divide none
    of those four."""
    composites = [256, 255, 253, 247]
    primes = [p for p in range(2, 256) if _is_prime(p) and all(c % p for c in composites)]
    return sorted(composites + primes, reverse=True)[:count]


def scaled_integers(hi_row, lo_row, S: int = 14):
    """The exact integers X = RNE(hi 2^(8S-e)) + RNE(lo 2^(8S-e)) of one row
    (Python ints) and its exponent e."""
    e = scale_exponent(hi_row)
    return [rne_scaled(float(h), 8 * S - e) + rne_scaled(float(l), 8 * S - e)
            for h, l in zip(hi_row, lo_row)], e


def sym_residue(x: int, p: int) -> int:
    """x mod p in [-floor(p/2), ceil(p/2) - 1]."""
    r = x % p
    return r - p if r > (p - 1) // 2 else r


def residue_planes(rows_hi, rows_lo, moduli, S: int = 14):
    """[N][rows][k] symmetric residues of the scaled integers, and exponents."""
    R, K = rows_hi.shape
    out = np.zeros((len(moduli), R, K), dtype=np.int64)
    ex = np.zeros(R, dtype=np.int64)
    for r in range(R):
        X, ex[r] = scaled_integers(rows_hi[r], rows_lo[r], S)
        for i, p in enumerate(moduli):
            out[i, r, :] = [sym_residue(x, p) for x in X]
    return out, ex


def crt_products(RA, RB, moduli):
    """(R^A_i R^B_i^T) mod p_i in [0, p_i) (exact int64 products)."""
    return np.stack([np.mod(RA[i] @ RB[i].T, p) for i, p in enumerate(moduli)])


def crt_reconstruct(res, moduli):
    """The unique x in (-P/2, P/2] with x = res_i mod p_i (P = prod p_i), by
    the textbook CRT sum (Python ints), for every entry of res[i]."""
    P = 1
    for p in moduli:
        P *= p
    weights = []
    for p in moduli:
        M = P // p
        weights.append(M * pow(M % p, -1, p))
    shape = res.shape[1:]
    out = np.empty(shape, dtype=object)
    for idx in np.ndindex(*shape):
        s = sum(int(res[(i,) + idx]) * w for i, w in enumerate(weights)) % P
        out[idx] = s - P if 2 * s > P else s
    return out


# ----------------------------------------------------------------------------
# Per-call certificate: the operand width that meets the accuracy bound
# ----------------------------------------------------------------------------

def bf16_floor(x: Fraction) -> Fraction:
    """The largest bf16 value not above x >= 0: 8 significant bits for
    x >= 2^-126, multiples of 2^-133 below (bf16 subnormals)."""
    x = Fraction(x)
    if x <= 0:
        return Fraction(0)
    E = math.floor(math.log2(x.numerator) - math.log2(x.denominator))
    while Fraction(2) ** E > x:          # 2^E <= x < 2^(E+1), exactly
        E -= 1
    while Fraction(2) ** (E + 1) <= x:
        E += 1
    unit = Fraction(2) ** (E - 7) if E >= -126 else Fraction(2) ** -133
    return math.floor(x / unit) * unit


def magnitude_row(hi_row, e: int):
    """Magnitude plane entries of one row: bf16_floor(|hi| 2^-e)."""
    return [bf16_floor(abs(Fraction(float(h))) * Fraction(2) ** -e) for h in hi_row]


def product_error_constant(form: str, W: int) -> Fraction:
    """cst with |a b - (the form's product of rounded a, b)| <= cst 2^(e+f-W):
    "crt": one unit of rounding per factor, (1 + 2^-W); "sliced" (W = 8S):
    that plus the digit pairs t + u >= S the band sums drop,
    sum_{h >= 0} (S - 1 - h) 2^-2 256^-h <= (S - 1) / (4 (1 - 2^-8))."""
    if form == "crt":
        return 1 + Fraction(2) ** -W
    S = W // 8
    return 1 + Fraction(2) ** -W + Fraction(S - 1, 4) / (1 - Fraction(1, 256))


def exact_margins(a_rows, b_cols, alpha, beta, C=None, tri: int = 0):
    """{(i, j): d_ij} with d_ij = ((|A||B|)_ij + |beta/alpha| |c_ij|) 2^-(e_i+f_j)
    for the rows of op(A) and columns of op(B) given as (hi, lo) row arrays,
    from the exact dd values; rows or columns that are all zero, and entries
    outside the requested triangle (tri 1 upper, 2 lower), are left out."""
    ah, al = a_rows
    bh, bl = b_cols
    m, k = ah.shape
    n = bh.shape[0]
    ea = [scale_exponent(ah[i]) for i in range(m)]
    fb = [scale_exponent(bh[j]) for j in range(n)]
    A = [[abs(Fraction(float(ah[i, l])) + Fraction(float(al[i, l]))) for l in range(k)]
         for i in range(m)]
    B = [[abs(Fraction(float(bh[j, l])) + Fraction(float(bl[j, l]))) for l in range(k)]
         for j in range(n)]
    ratio = abs(Fraction(beta[0]) + Fraction(beta[1])) / abs(Fraction(alpha[0]) +
                                                             Fraction(alpha[1]))
    out = {}
    for i in range(m):
        if not any(ah[i]):
            continue
        for j in range(n):
            if not any(bh[j]) or (tri == 1 and i > j) or (tri == 2 and i < j):
                continue
            ab = sum(x * y for x, y in zip(A[i], B[j]))
            cc = 0 if C is None or ratio == 0 else abs(Fraction(float(C[0][i, j])) +
                                                      Fraction(float(C[1][i, j])))
            out[(i, j)] = (ab + ratio * cc) * Fraction(2) ** -(ea[i] + fb[j])
    return out


def certified_width(dmin: Fraction, form: str, widths) -> int:
    """The narrowest W in ``widths`` (ascending) with
    cst 2^(106 - W) / 12 <= dmin: then every product error, summed over k,
    is at most 12 k 2^-106 (|A||B| + |beta/alpha||C|)_ij, three quarters of
    the bound 4 k 2^-104 (...) per unit of |alpha|, the rest left for the
    final roundings.  0: no width qualifies."""
    for W in widths:
        if product_error_constant(form, W) * Fraction(2) ** (106 - W) / 12 <= dmin:
            return W
    return 0

