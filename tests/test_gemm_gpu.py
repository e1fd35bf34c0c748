"""Parity of the plain dd Rgemm / Rsyrk CUDA path with the oracle (GPU).

Bar: componentwise |C_gpu - C_exact| <= 4 k 2^-104 (|alpha||A||B| + |beta||C|)
against the oracle's exact tier (or twice that against its scalar dd tier at
sizes where the exact tier is too slow), outputs normalised dd, and the
bitwise invariants the kernel guarantees (determinism, Rsyrk == Rgemm
triangle, power-of-two scaling, host == device forms).
"""
from __future__ import annotations

import numpy as np
import pytest

import datagen
import oracle
from ddcheck import err_over_bound, gemm_bound_entries
from gpucase import (check_against_exact, check_against_scalar, dev, host, run_gemm,
                     sample_blocks)
from test_oracle import (cgemm_case, check_cgemm_result, complex_gemm_via_real, read_golden,
                         rows_real)

pytestmark = pytest.mark.gpu


def test_config0_nn_256_alpha1_beta0(cuda_lib):
    """256^3 NN, alpha = 1, beta = 0, seed 0; C is write-only (NaN-filled)."""
    c = datagen.gemm_case(0, "N", "N", 256, 256, 256, alpha=(1.0, 0.0), beta=(0.0, 0.0))
    c.C = (np.full_like(c.C[0], np.nan), np.full_like(c.C[1], np.nan))
    got = run_gemm(c)
    assert check_against_exact(c, got) <= 1.0
    rr, cc = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    assert check_against_scalar(c, got, rr.ravel(), cc.ravel()) <= 1.0


SHAPES = [(1, 1, 1), (2, 3, 5), (17, 63, 64), (65, 64, 127), (63, 65, 257), (130, 70, 33),
          (5, 129, 1), (64, 64, 16)]


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("shape", SHAPES)
def test_ragged_shapes_all_transposes(cuda_lib, ta, tb, shape):
    m, n, k = shape
    seed = 100 + 4 * SHAPES.index(shape) + ["NN", "TN", "NT", "TT"].index(ta + tb)
    c = datagen.gemm_case(seed, ta, tb, m, n, k, pad=3)
    got = run_gemm(c)
    assert check_against_exact(c, got) <= 1.0


def test_rgemm_worked_example_bitwise(cuda_lib):
    gd = read_golden("rgemm_worked_example.txt")
    mats = [np.array([[float(x) for x in r] for r in rows_real(gd[k])], order="F")
            for k in ("A", "B", "C")]
    A, B, C = (dev((M, np.zeros_like(M))) for M in mats)
    cuda_lib.mp_dd_Rgemm("N", "N", 3, 3, 3, (3.0, 0.0), A, 3, B, 3, (-2.0, 0.0), C, 3)
    got = host(C)
    ans = np.array([[float(x) for x in r] for r in rows_real(gd["ANSWER"])])
    assert np.array_equal(got[0], ans) and not got[1].any()


@pytest.mark.parametrize("variant", ["binary64", "decimal"])
def test_cgemm_worked_example_through_gpu_rgemm(cuda_lib, variant):
    alpha, A, B, beta, C, ans = cgemm_case(variant)

    def gemm(al, X, Y, be, Z):
        m, k = X[0].shape
        n = Y[0].shape[1]
        Xd, Yd, Zd = dev(X), dev(Y), dev(Z)
        cuda_lib.mp_dd_Rgemm("N", "N", m, n, k, al, Xd, m, Yd, k, be, Zd, m)
        return host(Zd)

    re, im = complex_gemm_via_real(gemm, alpha, A, B, beta, C)
    check_cgemm_result(re, im, alpha, A, B, beta, C, ans)


def test_beta_zero_ignores_nan_and_alpha_zero_scales(cuda_lib):
    c = datagen.gemm_case(5, "N", "N", 70, 50, 40)
    c.beta = (0.0, 0.0)
    c.C = (np.full_like(c.C[0], np.nan), np.full_like(c.C[1], np.nan))
    got = run_gemm(c)
    assert np.isfinite(got[0]).all() and check_against_exact(c, got) <= 1.0
    # alpha == 0: A and B are not read (NaN), C := beta*C
    c = datagen.gemm_case(6, "N", "N", 70, 50, 40)
    c.alpha = (0.0, 0.0)
    c.A = (np.full_like(c.A[0], np.nan), np.full_like(c.A[1], np.nan))
    got = run_gemm(c)
    assert np.isfinite(got[0]).all()
    c.A = (np.zeros_like(c.A[0]), np.zeros_like(c.A[1]))
    assert check_against_exact(c, got) <= 1.0
    # alpha == 0, beta == 1: quick return, C untouched even if NaN
    c.beta = (1.0, 0.0)
    c.C = (np.full_like(c.C[0], np.nan), c.C[1])
    got = run_gemm(c)
    assert np.isnan(got[0]).all()


def test_deterministic_and_scaling_invariant(cuda_lib):
    c = datagen.gemm_case(7, "N", "T", 150, 90, 200)
    g1 = run_gemm(c)
    g2 = run_gemm(c)
    assert np.array_equal(g1[0], g2[0]) and np.array_equal(g1[1], g2[1])
    # scale row i of op(A) by 2^er[i], column j of op(B) by 2^ec[j], C by both:
    # the output scales exactly (every operation commutes with powers of two)
    g = datagen.rng(70)
    er = g.integers(-20, 20, c.m)
    ec = g.integers(-20, 20, c.n)
    s = datagen.GemmCase(**vars(c))
    s.A = datagen._scale_rows_padded(c.A, er)
    s.B = datagen._scale_rows_padded(c.B, ec)
    s.C = datagen.scale_cols(datagen._scale_rows_padded(c.C, er), ec)
    gs = run_gemm(s)
    f = np.ldexp(1.0, er)[:, None] * np.ldexp(1.0, ec)[None, :]
    assert np.array_equal(gs[0], g1[0] * f) and np.array_equal(gs[1], g1[1] * f)


@pytest.mark.parametrize("uplo,trans", [("U", "N"), ("L", "N"), ("U", "T"), ("L", "T")])
@pytest.mark.parametrize("n,k", [(1, 1), (70, 33), (129, 200)])
def test_rsyrk_parity_and_bitwise_gemm_triangle(cuda_lib, uplo, trans, n, k):
    t = trans == "T"
    g = datagen.rng(80 + n)
    A = datagen.dd_matrix(g, k if t else n, n if t else k, (k if t else n) + 2)
    C = datagen.dd_matrix(g, n, n, n + 1)
    al, be = datagen.dd_scalar(g), datagen.dd_scalar(g)
    Ad, Cd = dev(A), dev(C)
    cuda_lib.mp_dd_Rsyrk(uplo, trans, n, k, al, Ad, A[0].shape[0], be, Cd, C[0].shape[0])
    got = host(Cd, n, n)
    tri = np.triu(np.ones((n, n), bool)) if uplo == "U" else np.tril(np.ones((n, n), bool))
    # the other triangle is untouched
    assert np.array_equal(got[0][~tri], C[0][:n, :n][~tri])
    # bitwise equal to Rgemm (N,T) / (T,N) on the triangle
    Cg = dev(C)
    ta, tb = ("T", "N") if t else ("N", "T")
    cuda_lib.mp_dd_Rgemm(ta, tb, n, n, k, al, Ad, A[0].shape[0], Ad, A[0].shape[0], be, Cg,
                         C[0].shape[0])
    gg = host(Cg, n, n)
    assert np.array_equal(got[0][tri], gg[0][tri]) and np.array_equal(got[1][tri], gg[1][tri])
    # within the bound of the exact result
    rows, cols = np.nonzero(tri)
    ex = oracle.exact_gemm_entries(ta, tb, k, al, A, A, be, C, rows, cols)
    bound = gemm_bound_entries(ta, tb, n, n, k, al, A, A, be, C, rows, cols)
    assert err_over_bound((got[0][rows, cols], got[1][rows, cols]), ex, bound) <= 1.0


def test_host_forms_equal_device_forms(cuda_lib):
    c = datagen.gemm_case(9, "T", "N", 100, 77, 130, pad=2)
    dgot = run_gemm(c)
    Ch = (np.array(c.C[0], order="F"), np.array(c.C[1], order="F"))
    cuda_lib.mp_dd_Rgemm_host(c.transa, c.transb, c.m, c.n, c.k, c.alpha, c.A, c.A[0].shape[0],
                              c.B, c.B[0].shape[0], c.beta, Ch, Ch[0].shape[0])
    assert np.array_equal(Ch[0][:c.m, :c.n], dgot[0]) and np.array_equal(Ch[1][:c.m, :c.n],
                                                                          dgot[1])
    assert np.isnan(Ch[0][c.m:, :]).all()  # padding rows of C untouched
    n, k = 90, 60
    g = datagen.rng(91)
    A = datagen.dd_matrix(g, n, k, n + 1)
    C = datagen.dd_matrix(g, n, n)
    Cd = dev(C)
    cuda_lib.mp_dd_Rsyrk("U", "N", n, k, (1.0, 0.0), dev(A), n + 1, (0.5, 0.0), Cd, n)
    Chost = (np.array(C[0], order="F"), np.array(C[1], order="F"))
    cuda_lib.mp_dd_Rsyrk_host("U", "N", n, k, (1.0, 0.0), A, n + 1, (0.5, 0.0), Chost, n)
    dd_ = host(Cd)
    assert np.array_equal(Chost[0], dd_[0]) and np.array_equal(Chost[1], dd_[1])


@pytest.mark.parametrize("ta", ["N", "T"])
def test_config1_large_sampled_blocks(cuda_lib, ta):
    """Plain path at the benchmarked size: 64 x 64 blocks (corners, diagonal,
    random) against the scalar dd oracle, and a subset against the exact tier."""
    n = 2048
    c = datagen.gemm_case(1, ta, "N", n, n, n)
    got = run_gemm(c)
    rows, cols = sample_blocks(n, n)
    assert check_against_scalar(c, got, rows, cols) <= 1.0
    sub = np.arange(0, rows.size, 37)
    assert check_against_exact(c, got, rows[sub], cols[sub]) <= 1.0


def test_fp64_peak_is_positive(cuda_lib):
    r = cuda_lib.mp_dd_peak_fp64()
    assert r > 1e10


def test_imma_peak_is_positive(cuda_lib):
    """The warp-level INT8 tensor rate (mma.sync m16n8k32) is measurable."""
    r = cuda_lib.mp_dd_peak_imma()
    assert r > 1e12


def test_ddmac_peak_is_positive(cuda_lib):
    """The plain kernel's multiply-add mix rate is measurable and below the
    FP64 issue rate divided by the 12 FP64 instructions it needs at least."""
    r = cuda_lib.mp_dd_peak_ddmac()
    assert 1e9 < r < cuda_lib.mp_dd_peak_fp64() / 10
