"""Checks of triangular solves shared by the oracle pins and the GPU parity
tests: op(A) as a dense array, and the componentwise backward error of a
computed X with the residual op(A) X - alpha B evaluated exactly by the
oracle's superaccumulator tier."""
from __future__ import annotations

import numpy as np

import oracle
from ddcheck import EPS_DD

TRSM_VARIANTS = [(s, u, t, d) for s in "LR" for u in "UL" for t in "NT" for d in "NU"]


def op_triangle(A, uplo, transa, diag, order):
    """op(A) as a dense float array: the uplo triangle of A (ones on a unit
    diagonal, zeros elsewhere), transposed for transa = 'T'."""
    T = np.triu(A[:order, :order]) if uplo == "U" else np.tril(A[:order, :order])
    T = np.nan_to_num(T, nan=0.0)
    if diag == "U":
        np.fill_diagonal(T, 1.0)
    return T.T if transa == "T" else T


def trsm_residual_over_bound(c, X, rows=None, cols=None):
    """max_ij |op(A) X - alpha B|_ij / (4 (order + 2) 2^-104 (|op(A)||X| + |alpha B|)_ij),
    the residual evaluated exactly by the superaccumulator tier (the
    componentwise backward-error bound of substitution in dd arithmetic)."""
    order = c.m if c.side == "L" else c.n
    T = op_triangle(c.A[0], c.uplo, c.transa, c.diag, order)
    Tl = op_triangle(c.A[1], c.uplo, c.transa, "N", order)
    if c.diag == "U":
        np.fill_diagonal(Tl, 0.0)
    Td = (np.asfortranarray(T), np.asfortranarray(Tl))
    Bd = (c.B[0][:c.m, :c.n], c.B[1][:c.m, :c.n])
    if rows is None:
        rr, cc = np.meshgrid(np.arange(c.m), np.arange(c.n), indexing="ij")
        rows, cols = rr.ravel(), cc.ravel()
    rows, cols = np.asarray(rows), np.asarray(cols)
    neg = (-c.alpha[0], -c.alpha[1])
    if c.side == "L":
        R = oracle.exact_gemm_entries("N", "N", order, (1.0, 0.0), Td, X, neg, Bd, rows, cols)
        scale = (np.abs(T[rows, :]) * np.abs(X[0][:, cols]).T).sum(axis=1)
    else:
        R = oracle.exact_gemm_entries("N", "N", order, (1.0, 0.0), X, Td, neg, Bd, rows, cols)
        scale = (np.abs(X[0][rows, :]) * np.abs(T[:, cols]).T).sum(axis=1)
    scale = scale + abs(c.alpha[0]) * np.abs(Bd[0][rows, cols])
    bound = 4 * (order + 2) * EPS_DD * scale * (1 + 2.0 ** -40)
    return (np.abs(R[0]) / bound).max()
