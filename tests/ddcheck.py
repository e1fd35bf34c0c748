"""Comparison helpers shared by the tests: the componentwise accuracy bound.

The bound (the accuracy target of the dd Rgemm / Rsyrk path):

    |C - C_exact|_ij <= 4 * k * eps_dd * (|alpha| |op(A)| |op(B)| + |beta| |C_in|)_ij,

with eps_dd = 2^-104, the dd machine epsilon of the manual's Rlamch table.
It is evaluated from the hi planes in binary64 and inflated so that it is an
over-estimate: |x| <= |x.hi| (1 + 2^-52) for a normalised dd, and a binary64
sum of k non-negative terms is at least (1 - (k+1) u) times the exact sum.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

EPS_DD = 2.0 ** -104
U = 2.0 ** -53


def _inflate(k: int) -> float:
    return (1.0 + 2.0 ** -50) * (1.0 + 2.0 * (k + 3) * U)


def gemm_bound_entries(transa, transb, m, n, k, alpha, A, B, beta, C, rows, cols):
    """Bound at entries (rows[q], cols[q])."""
    ta, tb = transa.upper() in "TC", transb.upper() in "TC"
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    ur, ir = np.unique(rows, return_inverse=True)
    uc, ic = np.unique(cols, return_inverse=True)
    Ah = np.abs(A[0][:k, ur].T if ta else A[0][ur, :k])   # rows ur of |op(A)|
    Bh = np.abs(B[0][uc, :k].T if tb else B[0][:k, uc])   # columns uc of |op(B)|
    prod = Ah @ Bh
    ab = prod[ir, ic]
    a = abs(alpha[0]) * (1 + 2.0 ** -52)
    b = abs(beta[0]) * (1 + 2.0 ** -52)
    cin = np.zeros_like(ab) if b == 0 else np.abs(C[0][rows, cols])
    return 4.0 * max(k, 1) * EPS_DD * (a * ab + b * cin) * _inflate(k)


def gemm_bound(transa, transb, m, n, k, alpha, A, B, beta, C):
    rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    return gemm_bound_entries(transa, transb, m, n, k, alpha, A, B, beta, C, rr.ravel(),
                              cc.ravel()).reshape(m, n)


def dd_diff(h1, l1, h2, l2):
    """(h1 + l1) - (h2 + l2) in binary64; h1 - h2 is exact when the two values
    are within a factor 2 of each other (Sterbenz), which is the case of interest."""
    return (np.asarray(h1) - np.asarray(h2)) + (np.asarray(l1) - np.asarray(l2))


def err_over_bound(got, ref, bound):
    """max |got - ref| / bound (0/0 counted as 0)."""
    d = np.abs(dd_diff(got[0], got[1], ref[0], ref[1]))
    bound = np.asarray(bound, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(d == 0, 0.0, d / bound)
    return float(np.max(r)) if r.size else 0.0


def is_normalised(hi, lo) -> bool:
    """hi == fl(hi + lo) for every entry (the dd representation invariant)."""
    hi = np.asarray(hi)
    lo = np.asarray(lo)
    return bool(np.all((hi + lo) == hi))


def frac_diff(a, b):
    return abs(Fraction(a[0]) + Fraction(a[1]) - Fraction(b[0]) - Fraction(b[1]))


EPS_QD = 2.0 ** -209   # Rlamch epsilon of qd_real


def qd_bound_entries(transa, transb, m, n, k, alpha, A, B, beta, C, rows, cols):
    """4 k 2^-209 (|alpha||A||B| + |beta||C|) at the given entries, from the
    leading components (the dd bound helper scaled to the qd epsilon)."""
    return gemm_bound_entries(transa, transb, m, n, k, alpha[:2], (A[0], A[1]), (B[0], B[1]),
                              beta[:2], None if C is None else (C[0], C[1]), rows,
                              cols) * (EPS_QD / EPS_DD)


def qd_is_normalised(comps) -> bool:
    """|x_{t+1}| <= ulp(x_t) / 2 for every entry (zero tails after a zero)."""
    x = [np.asarray(c, dtype=np.float64) for c in comps]
    for t in range(3):
        half_ulp = np.where(x[t] == 0, 0.0, np.spacing(np.abs(x[t])) / 2)
        if (np.abs(x[t + 1]) > half_ulp).any():
            return False
    return True
