"""Rsyr2k and Rsymm as the Rgemm they equal, for the oracle pins and the GPU
parity tests: the exact result and the accuracy bound at chosen entries come
from the oracle's exact tier and the Rgemm bound applied to concatenated
(Rsyr2k) or symmetrised (Rsymm) operands.

Rsyr2k:  alpha (A B^T + B A^T) = alpha [A B] [B A]^T          (trans N)
         alpha (A^T B + B^T A) = alpha [A; B]^T [B; A]        (trans T)
Rsymm:   alpha S B (side L) or alpha B S (side R), S the symmetric matrix
         whose uplo triangle is stored in A.
"""
from __future__ import annotations

import numpy as np

import oracle
from ddcheck import gemm_bound_entries


def _part(X, rows, cols):
    return tuple(np.asfortranarray(P[:rows, :cols]) for P in X)


def syr2k_as_gemm(trans, n, k, A, B):
    """(transa, transb, kk, A', B') of the equivalent Rgemm."""
    if trans.upper() == "N":
        a, b = _part(A, n, k), _part(B, n, k)
        Ap = tuple(np.asfortranarray(np.hstack([x, y])) for x, y in zip(a, b))
        Bp = tuple(np.asfortranarray(np.hstack([y, x])) for x, y in zip(a, b))
        return "N", "T", 2 * k, Ap, Bp
    a, b = _part(A, k, n), _part(B, k, n)
    Ap = tuple(np.asfortranarray(np.vstack([x, y])) for x, y in zip(a, b))
    Bp = tuple(np.asfortranarray(np.vstack([y, x])) for x, y in zip(a, b))
    return "T", "N", 2 * k, Ap, Bp


def symmetrise(A, uplo, order):
    """The full symmetric matrix whose uplo triangle is stored in A."""
    out = []
    for P in A:
        T = np.triu(np.nan_to_num(P[:order, :order])) if uplo.upper() == "U" else \
            np.tril(np.nan_to_num(P[:order, :order]))
        d = np.diag(np.diag(T))
        out.append(np.asfortranarray(T + T.T - d))
    return tuple(out)


def symm_as_gemm(side, uplo, m, n, A, B):
    if side.upper() == "L":
        return "N", "N", m, symmetrise(A, uplo, m), _part(B, m, n)
    return "N", "N", n, _part(B, m, n), symmetrise(A, uplo, n)


def exact_and_bound(equiv, m, n, alpha, beta, C, rows, cols):
    ta, tb, kk, Ap, Bp = equiv
    Cp = _part(C, m, n)
    ex = oracle.exact_gemm_entries(ta, tb, kk, alpha, Ap, Bp, beta, Cp, rows, cols)
    bound = gemm_bound_entries(ta, tb, m, n, kk, alpha, Ap, Bp, beta, Cp, rows, cols)
    return ex, bound


def triangle_entries(n, uplo):
    r, c = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    keep = (r <= c) if uplo.upper() == "U" else (r >= c)
    return r[keep], c[keep]
