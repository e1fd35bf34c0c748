"""The input recipes (datagen.py), checked against their stated definitions.

Every comparison of the GPU path with the oracle, and every benchmark, takes
its inputs from these generators; this pins that they produce what the
recipes say: normalised dd entries with lo drawn as hi 2^-53 U(-1, 1), NaN
in padding rows, dd scalars in [0.5, 2], outer ill-scaling by exact powers of
two with exponents in [-30, 30], diagonally dominant triangles with NaN where
a solve may not read, grouped sizes and served orders log-uniform in their
ranges, SPD requests with singular values geometric from 1 to 1e-10 (so
G G^T has condition ~1e20) and Poisson arrivals; and that a seed fixes the
bits.
"""
from __future__ import annotations

import numpy as np

import datagen


def normalised(hi, lo):
    return bool(np.all(np.abs(lo) <= np.abs(np.spacing(hi)) / 2) and np.all(hi + lo == hi))


def test_dd_matrix_entries_padding_and_seed():
    g = datagen.rng(1)
    H, L = datagen.dd_matrix(g, 50, 30, 53)
    assert H.shape == (53, 30) and H.flags.f_contiguous
    assert np.isnan(H[50:]).all() and np.isnan(L[50:]).all()
    h, l = H[:50], L[:50]
    assert normalised(h, l)
    assert (np.abs(h) < 1.0 + 2.0 ** -52).all()
    # lo is a tiny multiple of hi: |lo| <= |hi| 2^-53 (up to the renormalisation)
    assert (np.abs(l) <= np.abs(h) * 2.0 ** -52).all()
    assert (l != 0).mean() > 0.9
    H2, L2 = datagen.dd_matrix(datagen.rng(1), 50, 30, 53)
    assert np.array_equal(H, H2, equal_nan=True) and np.array_equal(L, L2, equal_nan=True)


def test_dd_scalars_in_range():
    g = datagen.rng(2)
    for _ in range(100):
        hi, lo = datagen.dd_scalar(g)
        assert 0.5 <= hi <= 2.0 and normalised(np.array([hi]), np.array([lo]))


def test_outer_ill_scaling_is_exact_powers_of_two():
    m, n, k = 40, 30, 20
    base = datagen.gemm_case(7, "N", "N", m, n, k)
    ill = datagen.gemm_case(7, "N", "N", m, n, k, ill="outer")
    ra = ill.A[0] / base.A[0]                      # row i of A scaled by 2^e_i
    for i in range(m):
        e = np.log2(ra[i])
        assert np.all(e == e[0]) and e[0] == np.round(e[0]) and -30 <= e[0] <= 30
    assert np.array_equal(ill.A[1] / base.A[1], ra)
    cb = ill.B[0] / base.B[0]                      # column j of B scaled by 2^f_j
    for j in range(n):
        f = np.log2(cb[:, j])
        assert np.all(f == f[0]) and f[0] == np.round(f[0]) and -30 <= f[0] <= 30
    assert np.array_equal(ill.C[0], base.C[0])
    spread = np.log2(ra[:, 0])
    assert spread.max() - spread.min() >= 30       # the exponents really spread


def test_triangular_cases_nan_where_unread():
    g = datagen.rng(3)
    H, L = datagen.triangular_dd(g, 20, "L", "U", 22)
    r, c = np.meshgrid(np.arange(20), np.arange(20), indexing="ij")
    assert np.isnan(H[:20][r <= c]).all()           # upper triangle and unit diagonal
    assert np.isfinite(H[:20][r > c]).all()
    H, L = datagen.triangular_dd(g, 20, "U", "N", 20)
    d = np.abs(np.diag(H))
    off = np.nansum(np.abs(np.triu(np.nan_to_num(H), 1)), axis=1)
    assert (d >= 20).all() and (d > off).all()        # strictly diagonally dominant


def test_grouped_and_served_sizes_log_uniform():
    s = datagen.grouped_problems(4, count=4096)
    assert s.shape == (4096, 3) and s.min() >= 16 and s.max() <= 512
    # log-uniform: about half of the draws below the geometric midpoint sqrt(16 512)
    assert 0.45 < (s < np.sqrt(16 * 512)).mean() < 0.55
    n = datagen.request_sizes(0, 2000)
    assert n.min() >= 64 and n.max() <= 2048
    assert 0.45 < (n < np.sqrt(64 * 2048)).mean() < 0.55


def test_spd_request_spectrum():
    n = 60
    (gh, gl), (bh, bl) = datagen.spd_request(5, n)
    assert gh.shape == (n, 2 * n) and bh.shape == (n, 4)
    assert normalised(gh, gl) and normalised(bh, bl)
    s = np.linalg.svd(gh, compute_uv=False)
    expect = np.geomspace(1.0, 1e-10, n)
    assert np.allclose(s, expect, rtol=1e-6)
    assert 0.9e20 < (s[0] / s[-1]) ** 2 < 1.1e20     # cond(G G^T)


def test_poisson_arrivals():
    a = datagen.poisson_arrivals(0, 20000, 100.0)
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 0.01) < 0.0005
    assert abs(gaps.std() - 0.01) < 0.0007          # exponential: std = mean
