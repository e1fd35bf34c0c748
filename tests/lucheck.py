"""LU checks shared by the oracle pins and the GPU parity tests: a dyadic
factorisation with known pivots (exact in dd arithmetic), the row
interchanges of an ipiv vector, and the LAPACK residual ratio and the
componentwise backward error of computed factors with P A - L U evaluated
exactly by the oracle's superaccumulator tier."""
from __future__ import annotations

import numpy as np

import datagen
import oracle
from ddcheck import EPS_DD


def dyadic_lu_case(seed, m, n):
    """A = (rows of L U placed at rows sigma) with L unit lower, |L| <= 1/2
    below the diagonal in quarters, U integer with a power-of-two diagonal:
    partial pivoting must find sigma, L and U exactly.  Returns A, L, U and
    the expected one-based ipiv."""
    g = datagen.rng(seed)
    mn = min(m, n)
    L = np.tril(g.choice([-0.5, -0.25, 0.0, 0.25, 0.5], (m, mn)), -1)
    L[np.arange(mn), np.arange(mn)] = 1.0
    U = np.triu(g.integers(-5, 6, (mn, n)).astype(np.float64))
    U[np.arange(mn), np.arange(mn)] = g.choice([-4.0, -2.0, -1.0, 1.0, 2.0, 4.0], mn)
    sigma = g.permutation(m)
    A = np.zeros((m, n))
    A[sigma, :] = L @ U
    cur = list(range(m))
    ipiv = []
    for j in range(mn):
        p = cur.index(sigma[j])
        ipiv.append(p + 1)
        cur[j], cur[p] = cur[p], cur[j]
    # P A = L' U with L' the rows of L in the final order of A's rows
    inv = np.argsort(sigma)
    return np.asfortranarray(A), L[inv[cur]], U, np.array(ipiv)


def apply_ipiv(X, ipiv):
    """Rows of X interchanged as ipiv says (in order): P X."""
    X = X.copy()
    for j, p in enumerate(ipiv):
        X[[j, p - 1]] = X[[p - 1, j]]
    return X


def lu_residual_ratio(A, LU, ipiv, m, n):
    """||P A - L U||_1 / (n ||A||_1 eps_dd), the product evaluated exactly."""
    A = tuple(P[:m, :n] for P in A)
    LU = tuple(P[:m, :n] for P in LU)
    mn = min(m, n)
    L = [np.tril(P[:, :mn], -1) for P in LU]
    L[0][np.arange(mn), np.arange(mn)] = 1.0
    U = [np.triu(P[:mn, :]) for P in LU]
    PA = tuple(np.asfortranarray(apply_ipiv(P, ipiv)) for P in A)
    rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    R = oracle.exact_gemm_entries("N", "N", mn, (1.0, 0.0), tuple(np.asfortranarray(x) for x in L),
                                  tuple(np.asfortranarray(x) for x in U), (-1.0, 0.0), PA,
                                  rr.ravel(), cc.ravel())
    Rn = np.abs(R[0].reshape(m, n)).sum(axis=0).max()
    return Rn / (n * np.abs(A[0]).sum(axis=0).max() * EPS_DD)


def unpack_lu(LU, m, n):
    """(L, U) pairs of planes from a packed factorisation (unit diagonal)."""
    mn = min(m, n)
    L = [np.asfortranarray(np.tril(P[:m, :mn], -1)) for P in LU]
    L[0][np.arange(mn), np.arange(mn)] = 1.0
    U = [np.asfortranarray(np.triu(P[:mn, :n])) for P in LU]
    return tuple(L), tuple(U)


def lu_backward_over_bound(A, LU, ipiv, m, n, rows, cols):
    """max |P A - L U|_ij / (4 (min(m, n) + 2) 2^-104 (|L||U|)_ij) at the given
    entries (the componentwise backward error of Gaussian elimination)."""
    mn = min(m, n)
    L, U = unpack_lu(LU, m, n)
    PA = tuple(np.asfortranarray(apply_ipiv(P[:m, :n], ipiv)) for P in A)
    R = oracle.exact_gemm_entries("N", "N", mn, (1.0, 0.0), L, U, (-1.0, 0.0), PA, rows, cols)
    scale = (np.abs(L[0][rows, :]) * np.abs(U[0][:, cols]).T).sum(axis=1)
    bound = 4 * (mn + 2) * EPS_DD * scale * (1 + 2.0 ** -40)
    return (np.abs(R[0]) / bound).max()
