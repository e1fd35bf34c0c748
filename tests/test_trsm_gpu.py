"""dd Rtrsm through the C ABI (GPU).

Pins: every side/uplo/trans/diag variant recovers an exact integer solution
bit for bit (the unused triangle, padding rows and a unit diagonal hold NaN,
so a stray read shows); ragged sizes that span several 64-row blocks and
both recursion orders meet the componentwise backward-error bound with the
residual evaluated by the oracle's exact tier, and agree with the oracle's
substitution within the forward error that the bound allows on these
diagonally dominant matrices; the ill-conditioned Cholesky factor of a
served request meets the same backward bound; alpha = 0, empty sizes and
illegal arguments behave as DTRSM; repeated calls are bitwise identical.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import datagen
import oracle
from gpucase import dev, host
from trsmcheck import TRSM_VARIANTS, op_triangle, trsm_residual_over_bound

pytestmark = pytest.mark.gpu


def gpu_trsm(mp, c):
    A, B = dev(c.A), dev(c.B)
    mp.mp_dd_Rtrsm(c.side, c.uplo, c.transa, c.diag, c.m, c.n, c.alpha, A, c.A[0].shape[0], B,
                   c.B[0].shape[0])
    return host(B, c.m, c.n)


def integer_case(side, uplo, transa, diag, m, n, seed):
    """A TrsmCase whose solution is the integer matrix X: A has small integer
    entries and a power-of-two diagonal, alpha = 2 and B = op(A) X / 2 (or
    X op(A) / 2), exact in binary64."""
    g = datagen.rng(seed)
    order = m if side == "L" else n
    A = g.integers(-3, 4, (order, order)).astype(np.float64)
    np.fill_diagonal(A, g.choice([-2.0, -1.0, 1.0, 2.0], order))
    X = g.integers(-9, 10, (m, n)).astype(np.float64)
    T = op_triangle(A, uplo, transa, diag, order)
    Bx = (T @ X if side == "L" else X @ T) / 2.0
    assert np.abs(Bx).max() < 2.0 ** 50
    pad = 5
    Ah = np.full((order + pad, order), np.nan, order="F")
    r, cidx = np.meshgrid(np.arange(order), np.arange(order), indexing="ij")
    used = (r <= cidx) if uplo == "U" else (r >= cidx)
    if diag == "U":
        used &= r != cidx
    Ah[:order][used] = A[used]
    Al = np.where(np.isnan(Ah), np.nan, 0.0)
    Bh = np.full((m + pad, n), np.nan, order="F")
    Bh[:m] = Bx
    Bl = np.where(np.isnan(Bh), np.nan, 0.0)
    c = datagen.TrsmCase(side, uplo, transa, diag, m, n, (2.0, 0.0),
                         (np.asfortranarray(Ah), np.asfortranarray(Al)),
                         (np.asfortranarray(Bh), np.asfortranarray(Bl)))
    return c, X


@pytest.mark.parametrize("side,uplo,transa,diag", TRSM_VARIANTS)
def test_integer_solution_exact(cuda_lib, side, uplo, transa, diag):
    m, n = (150, 70) if side == "L" else (70, 150)
    c, X = integer_case(side, uplo, transa, diag, m, n, 800)
    xh, xl = gpu_trsm(cuda_lib, c)
    assert np.array_equal(xh, X) and not xl.any()


@pytest.mark.parametrize("side,uplo,transa,diag", TRSM_VARIANTS)
def test_ragged_against_exact_residual_and_oracle(cuda_lib, side, uplo, transa, diag):
    m, n = (150, 70) if side == "L" else (70, 150)
    c = datagen.trsm_case(810, side, uplo, transa, diag, m, n, pad=3)
    got = gpu_trsm(cuda_lib, c)
    assert np.isfinite(got[0]).all()
    assert trsm_residual_over_bound(c, got) <= 1.0
    ref = oracle.dd_trsm(side, uplo, transa, diag, c.alpha, c.A, c.B, m, n)
    ref = (ref[0][:m, :n], ref[1][:m, :n])
    # both solutions have backward error <= 4 (order + 2) 2^-104 on a matrix
    # of condition < 4, so they differ by far less than 2^-90 of the largest
    # solution entry of their column
    diff = np.abs((got[0] - ref[0]) + (got[1] - ref[1]))
    col = np.abs(ref[0]).max(axis=0, keepdims=True)
    assert (diff <= 2.0 ** -90 * col).all()


@pytest.mark.parametrize("side,uplo,transa,diag",
                         [("L", "U", "N", "N"), ("L", "L", "T", "U"), ("R", "U", "T", "N"),
                          ("R", "L", "N", "N")])
def test_larger_sampled(cuda_lib, side, uplo, transa, diag):
    """Orders 700 / 1000 (several recursion levels) on sampled entries."""
    m, n = (1000, 300) if side == "L" else (300, 700)
    c = datagen.trsm_case(820, side, uplo, transa, diag, m, n)
    got = gpu_trsm(cuda_lib, c)
    g = datagen.rng(821)
    rows = g.integers(0, m, 1500)
    cols = g.integers(0, n, 1500)
    # include the last rows/columns (the end of each sweep)
    rows[:50], cols[50:100] = m - 1, n - 1
    assert trsm_residual_over_bound(c, got, rows, cols) <= 1.0


def test_cholesky_factor_of_served_request(cuda_lib):
    """F = G G^T of a served request (condition ~1e20); its dd Cholesky factor
    U (condition ~1e10) solves U^T Y = B then U X = Y within the backward
    bound each time."""
    n = 200
    G, B = datagen.spd_request(830, n)
    Fd = oracle.dd_syrk("U", "N", (1.0, 0.0), G, (0.0, 0.0),
                        (np.zeros((n, n), order="F"), np.zeros((n, n), order="F")))
    fh, fl, info = oracle.dd_potrf("U", Fd)
    assert info == 0
    U = (np.where(np.triu(np.ones((n, n))) > 0, fh, np.nan),
         np.where(np.triu(np.ones((n, n))) > 0, fl, np.nan))
    U = tuple(np.asfortranarray(x) for x in U)
    for transa in "TN":
        c = datagen.TrsmCase("L", "U", transa, "N", n, B[0].shape[1], (1.0, 0.0), U, B)
        got = gpu_trsm(cuda_lib, c)
        assert trsm_residual_over_bound(c, got) <= 1.0
        B = tuple(np.asfortranarray(x) for x in got)


def test_alpha_zero_empty_and_errors(cuda_lib):
    mp = cuda_lib
    c = datagen.trsm_case(840, "L", "U", "N", "N", 40, 30)
    A, B = dev(c.A), dev(c.B)
    nanA = tuple(torch.full_like(x, float("nan")) for x in A)
    mp.mp_dd_Rtrsm("L", "U", "N", "N", 40, 30, (0.0, 0.0), nanA, 40, B, 40)
    xh, xl = host(B)
    assert not xh.any() and not xl.any()
    B = dev(c.B)
    mp.mp_dd_Rtrsm("L", "U", "N", "N", 0, 30, c.alpha, A, 40, B, 40)
    mp.mp_dd_Rtrsm("R", "U", "N", "N", 40, 0, c.alpha, A, 1, B, 40)
    xh, xl = host(B)
    assert np.array_equal(xh, c.B[0]) and np.array_equal(xl, c.B[1])
    bad = [(("X", "U", "N", "N", 40, 30, 40, 40), -1), (("L", "X", "N", "N", 40, 30, 40, 40), -2),
           (("L", "U", "X", "N", 40, 30, 40, 40), -3), (("L", "U", "N", "X", 40, 30, 40, 40), -4),
           (("L", "U", "N", "N", -1, 30, 40, 40), -5), (("L", "U", "N", "N", 40, -1, 40, 40), -6),
           (("L", "U", "N", "N", 40, 30, 39, 40), -9), (("R", "U", "N", "N", 40, 30, 29, 40), -9),
           (("L", "U", "N", "N", 40, 30, 40, 39), -11)]
    for (s, u, t, d, m, n, lda, ldb), code in bad:
        rc = mp.mp_dd_Rtrsm(s, u, t, d, m, n, c.alpha, A, lda, B, ldb, check=False)
        assert rc == code, (s, u, t, d, m, n, lda, ldb, rc)
    # lower-case and 'C' flags are accepted
    B = dev(c.B)
    mp.mp_dd_Rtrsm("l", "u", "c", "n", 40, 30, c.alpha, A, 40, B, 40)


def test_deterministic(cuda_lib):
    c = datagen.trsm_case(850, "R", "L", "T", "N", 90, 260)
    a = gpu_trsm(cuda_lib, c)
    b = gpu_trsm(cuda_lib, c)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("transa", ["N", "T"])
def test_result_independent_of_columns_per_cta(cuda_lib, transa):
    """The solve kernel runs 32, 16, 8 or 4 right-hand-side columns per CTA
    depending on how many columns there are; each column's result is the
    same bits in every configuration."""
    m, wide = 150, 10000
    c = datagen.trsm_case(851, "L", "U", transa, "N", m, wide)
    outs = []
    for n in (6, 2500, 5000, wide):
        B = tuple(np.asfortranarray(P[:, :n]) for P in c.B)
        sub = datagen.TrsmCase(c.side, c.uplo, c.transa, c.diag, m, n, c.alpha, c.A, B)
        outs.append(gpu_trsm(cuda_lib, sub))
    for h, l in outs[1:]:
        assert np.array_equal(h[:, :6], outs[0][0]) and np.array_equal(l[:, :6], outs[0][1])
