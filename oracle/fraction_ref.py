"""Exact rational reference for tiny problems (pure Python ``fractions``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Independent of the C
oracle: it shares no code with it, so a disagreement between the two points
at one of them.

A dd value is the exact rational hi + lo (manual Sec. 5).  ``round_dd`` gives
the nearest dd: hi = RN(x), lo = RN(x - hi); CPython's ``float(Fraction)``
divides two integers with correct rounding (ties to even).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def frac(hi: float, lo: float = 0.0) -> Fraction:
    return Fraction(float(hi)) + Fraction(float(lo))


def round_dd(x: Fraction) -> tuple[float, float]:
    hi = float(x)
    lo = float(x - Fraction(hi))
    return hi, lo


def _op(X, trans: bool, r: int, c: int) -> Fraction:
    xh, xl = X
    if trans:
        return frac(xh[c, r], xl[c, r])
    return frac(xh[r, c], xl[r, c])


def gemm_exact(transa: str, transb: str, m: int, n: int, k: int, alpha, A, B, beta, C):
    """Exact alpha*op(A)*op(B) + beta*C as a list of lists of Fractions.

    BLAS semantics: beta == 0 means C is not read."""
    ta, tb = transa.upper() in "TC", transb.upper() in "TC"
    al, be = frac(*alpha), frac(*beta)
    out = []
    for i in range(m):
        row = []
        for j in range(n):
            s = Fraction(0)
            for l in range(k):
                s += _op(A, ta, i, l) * _op(B, tb, l, j)
            v = al * s
            if be != 0:
                v += be * frac(C[0][i, j], C[1][i, j])
            row.append(v)
        out.append(row)
    return out


def gemm_exact_dd(*args, **kw):
    """``gemm_exact`` rounded entrywise to the nearest dd: (hi, lo) arrays."""
    ex = gemm_exact(*args, **kw)
    m, n = len(ex), len(ex[0]) if ex else 0
    hi, lo = np.zeros((m, n), order="F"), np.zeros((m, n), order="F")
    for i in range(m):
        for j in range(n):
            hi[i, j], lo[i, j] = round_dd(ex[i][j])
    return hi, lo


def syrk_exact(uplo: str, trans: str, n: int, k: int, alpha, A, beta, C):
    """Exact Rsyrk result on the uplo triangle (Fractions); other entries None."""
    t = trans.upper() in "TC"
    al, be = frac(*alpha), frac(*beta)
    upper = uplo.upper() == "U"
    out = [[None] * n for _ in range(n)]
    for j in range(n):
        for i in (range(j + 1) if upper else range(j, n)):
            s = Fraction(0)
            for l in range(k):
                s += _op(A, t, i, l) * _op(A, t, j, l)
            v = al * s
            if be != 0:
                v += be * frac(C[0][i, j], C[1][i, j])
            out[i][j] = v
    return out
