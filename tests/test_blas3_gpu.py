"""dd Rsyr2k and Rsymm through the C ABI (GPU).

Pins: every uplo/trans (Rsyr2k) and side/uplo (Rsymm) variant at ragged
sizes that span several 64 x 64 tiles meets the Rgemm accuracy bound of the
equivalent concatenated / symmetrised product against the oracle's exact
tier; Rsyr2k leaves the other triangle untouched and, when k is a multiple
of the 16-wide k panel, equals mp_dd_Rgemm on the concatenated operands bit
for bit; Rsymm never reads the unstored triangle (NaN there) and equals
mp_dd_Rgemm on the symmetrised matrix bit for bit; larger problems are
checked on sampled blocks; alpha = 0 and argument errors follow DSYR2K /
DSYMM.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import blas3check as b3
import datagen
from ddcheck import err_over_bound, is_normalised
from gpucase import dev, host, sample_blocks

pytestmark = pytest.mark.gpu


def syr2k_case(seed, trans, n, k, pad=3):
    g = datagen.rng(seed)
    ar, ac = (n, k) if trans == "N" else (k, n)
    A = datagen.dd_matrix(g, ar, ac, ar + pad)
    B = datagen.dd_matrix(g, ar, ac, ar + pad)
    C = datagen.dd_matrix(g, n, n, n + pad)
    return A, B, C, datagen.dd_scalar(g), datagen.dd_scalar(g)


def gpu_syr2k(mp, uplo, trans, n, k, A, B, C, al, be):
    dA, dB, dC = dev(A), dev(B), dev(C)
    mp.mp_dd_Rsyr2k(uplo, trans, n, k, al, dA, A[0].shape[0], dB, B[0].shape[0], be, dC,
                    C[0].shape[0])
    return host(dC)


@pytest.mark.parametrize("uplo", ["U", "L"])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_syr2k_ragged_against_exact(cuda_lib, uplo, trans):
    n, k = 150, 70
    A, B, C, al, be = syr2k_case(900, trans, n, k)
    got = gpu_syr2k(cuda_lib, uplo, trans, n, k, A, B, C, al, be)
    rows, cols = b3.triangle_entries(n, uplo)
    ex, bound = b3.exact_and_bound(b3.syr2k_as_gemm(trans, n, k, A, B), n, n, al, be, C,
                                   rows, cols)
    g = (got[0][rows, cols], got[1][rows, cols])
    assert is_normalised(*g)
    assert err_over_bound(g, ex, bound) <= 1.0
    other = np.ones(C[0].shape, bool)
    other[rows, cols] = False
    assert np.array_equal(got[0][other], C[0][other], equal_nan=True)
    assert np.array_equal(got[1][other], C[1][other], equal_nan=True)


@pytest.mark.parametrize("trans", ["N", "T"])
def test_syr2k_equals_rgemm_on_concatenated_operands(cuda_lib, trans):
    n, k = 130, 64
    A, B, C, al, be = syr2k_case(901, trans, n, k, pad=0)
    got = gpu_syr2k(cuda_lib, "U", trans, n, k, A, B, C, al, be)
    ta, tb, kk, Ap, Bp = b3.syr2k_as_gemm(trans, n, k, A, B)
    dA, dB, dC = dev(Ap), dev(Bp), dev(C)
    cuda_lib.mp_dd_Rgemm(ta, tb, n, n, kk, al, dA, Ap[0].shape[0], dB, Bp[0].shape[0], be, dC, n)
    ref = host(dC)
    rows, cols = b3.triangle_entries(n, "U")
    assert np.array_equal(got[0][rows, cols], ref[0][rows, cols])
    assert np.array_equal(got[1][rows, cols], ref[1][rows, cols])


def symm_case(seed, side, uplo, m, n):
    g = datagen.rng(seed)
    order = m if side == "L" else n
    A = datagen.dd_matrix(g, order, order, order + 2)
    r, c = np.meshgrid(np.arange(order), np.arange(order), indexing="ij")
    unused = (r > c) if uplo == "U" else (r < c)
    for P in A:
        P[:order][unused] = np.nan
    B = datagen.dd_matrix(g, m, n, m + 1)
    C = datagen.dd_matrix(g, m, n, m + 3)
    return A, B, C, datagen.dd_scalar(g), datagen.dd_scalar(g)


def gpu_symm(mp, side, uplo, m, n, A, B, C, al, be):
    dA, dB, dC = dev(A), dev(B), dev(C)
    mp.mp_dd_Rsymm(side, uplo, m, n, al, dA, A[0].shape[0], dB, B[0].shape[0], be, dC,
                   C[0].shape[0])
    return host(dC, m, n)


@pytest.mark.parametrize("side", ["L", "R"])
@pytest.mark.parametrize("uplo", ["U", "L"])
def test_symm_ragged_against_exact_and_rgemm(cuda_lib, side, uplo):
    m, n = 150, 90
    A, B, C, al, be = symm_case(910, side, uplo, m, n)
    got = gpu_symm(cuda_lib, side, uplo, m, n, A, B, C, al, be)
    assert np.isfinite(got[0]).all() and is_normalised(*got)
    rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    rows, cols = rr.ravel(), cc.ravel()
    equiv = b3.symm_as_gemm(side, uplo, m, n, A, B)
    ex, bound = b3.exact_and_bound(equiv, m, n, al, be, C, rows, cols)
    assert err_over_bound((got[0][rows, cols], got[1][rows, cols]), ex, bound) <= 1.0
    ta, tb, kk, Ap, Bp = equiv
    dA, dB, dC = dev(Ap), dev(Bp), dev(C)
    cuda_lib.mp_dd_Rgemm(ta, tb, m, n, kk, al, dA, Ap[0].shape[0], dB, Bp[0].shape[0], be, dC,
                         C[0].shape[0])
    ref = host(dC, m, n)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_larger_sampled(cuda_lib):
    n, k = 1000, 500
    A, B, C, al, be = syr2k_case(920, "N", n, k, pad=0)
    got = gpu_syr2k(cuda_lib, "L", "N", n, k, A, B, C, al, be)
    rows, cols = sample_blocks(n, n, seed=921)
    keep = rows >= cols
    rows, cols = rows[keep], cols[keep]
    ex, bound = b3.exact_and_bound(b3.syr2k_as_gemm("N", n, k, A, B), n, n, al, be, C, rows,
                                   cols)
    assert err_over_bound((got[0][rows, cols], got[1][rows, cols]), ex, bound) <= 1.0
    m, n = 700, 900
    A, B, C, al, be = symm_case(922, "R", "U", m, n)
    got = gpu_symm(cuda_lib, "R", "U", m, n, A, B, C, al, be)
    rows, cols = sample_blocks(m, n, seed=923)
    ex, bound = b3.exact_and_bound(b3.symm_as_gemm("R", "U", m, n, A, B), m, n, al, be, C,
                                   rows, cols)
    assert err_over_bound((got[0][rows, cols], got[1][rows, cols]), ex, bound) <= 1.0


def test_alpha_zero_and_errors(cuda_lib):
    mp = cuda_lib
    n, k = 40, 20
    A, B, C, al, be = syr2k_case(930, "N", n, k, pad=0)
    nan = tuple(torch.full((n, k), float("nan"), dtype=torch.float64, device="cuda")
                for _ in range(2))
    dC = dev(C)
    mp.mp_dd_Rsyr2k("U", "N", n, k, (0.0, 0.0), nan, n, nan, n, (0.0, 0.0), dC, n)
    got = host(dC)
    rows, cols = b3.triangle_entries(n, "U")
    assert not got[0][rows, cols].any() and not got[1][rows, cols].any()
    dA, dB = dev(A), dev(B)
    bad = [(("X", "N", n, k, n, n, n), -1), (("U", "X", n, k, n, n, n), -2),
           (("U", "N", -1, k, n, n, n), -3), (("U", "N", n, -1, n, n, n), -4),
           (("U", "N", n, k, n - 1, n, n), -7), (("U", "N", n, k, n, n - 1, n), -9),
           (("U", "N", n, k, n, n, n - 1), -12), (("U", "T", n, k, k - 1, k, n), -7)]
    for (u, t, nn, kk, lda, ldb, ldc), code in bad:
        rc = mp.mp_dd_Rsyr2k(u, t, nn, kk, al, dA, lda, dB, ldb, be, dC, ldc, check=False)
        assert rc == code, (u, t, rc)
    m, n = 30, 20
    A, B, C, al, be = symm_case(931, "L", "U", m, n)
    dA, dB, dC = dev(A), dev(B), dev(C)
    bad = [(("X", "U", m, n, m + 2, m + 1, m + 3), -1), (("L", "X", m, n, m + 2, m + 1, m + 3), -2),
           (("L", "U", -1, n, m + 2, m + 1, m + 3), -3), (("L", "U", m, -1, m + 2, m + 1, m + 3), -4),
           (("L", "U", m, n, m - 1, m + 1, m + 3), -7), (("R", "U", m, 40, 39, m + 1, m + 3), -7),
           (("L", "U", m, n, m + 2, m - 1, m + 3), -9), (("L", "U", m, n, m + 2, m + 1, m - 1), -12)]
    for (s, u, mm, nn, lda, ldb, ldc), code in bad:
        rc = mp.mp_dd_Rsymm(s, u, mm, nn, al, dA, lda, dB, ldb, be, dC, ldc, check=False)
        assert rc == code, (s, u, rc)
