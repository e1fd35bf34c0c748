"""Quad-double Rgemm through the C ABI (GPU).

Pins: ragged shapes under all four transpose pairs and non-tight leading
dimensions meet the qd bound 4 k 2^-209 (|alpha||A||B| + |beta||C|) against
the oracle's exact qd tier on every entry, and every output is a
normalised qd value; a larger product on sampled blocks; integer inputs
give the exact integer product; beta = 0 never reads C (NaN there), alpha
= 0 never reads A and B; quick returns, argument errors and determinism.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest
import torch

import datagen
import oracle
from ddcheck import qd_bound_entries, qd_is_normalised
from gpucase import sample_blocks

pytestmark = pytest.mark.gpu


def dev4(planes):
    import paper_2109_13406_gb300 as mp

    return tuple(mp.to_device(P) for P in planes)


def host4(planes, rows=None, cols=None):
    torch.cuda.synchronize()
    out = tuple(P.t().contiguous().cpu().numpy().T for P in planes)
    if rows is not None:
        out = tuple(P[:rows, :cols] for P in out)
    return out


def qd_case(seed, ta, tb, m, n, k, pad=0, alpha=None, beta=None):
    g = datagen.rng(seed)
    ar, ac = (k, m) if ta == "T" else (m, k)
    br, bc = (n, k) if tb == "T" else (k, n)
    A = datagen.qd_matrix(g, ar, ac, ar + pad)
    B = datagen.qd_matrix(g, br, bc, br + pad)
    C = datagen.qd_matrix(g, m, n, m + pad)
    al = datagen.qd_scalar(g) if alpha is None else alpha
    be = datagen.qd_scalar(g) if beta is None else beta
    return A, B, C, al, be


def run_qd(mp, ta, tb, m, n, k, A, B, C, al, be):
    dA, dB, dC = dev4(A), dev4(B), dev4(C)
    mp.mp_qd_Rgemm(ta, tb, m, n, k, al, dA, A[0].shape[0], dB, B[0].shape[0], be, dC,
                   C[0].shape[0])
    return host4(dC, m, n)


def max_err_over_bound(got, ta, tb, m, n, k, A, B, C, al, be, rows, cols):
    ex = oracle.exact_qd_gemm_entries(ta, tb, k, al, A, B, be, C, rows, cols)
    bound = qd_bound_entries(ta, tb, m, n, k, al, A, B, be, C, rows, cols)
    worst = 0.0
    for q, (i, j) in enumerate(zip(rows, cols)):
        d = sum(Fraction(float(got[t][i, j])) - Fraction(float(ex[t][q])) for t in range(4))
        worst = max(worst, float(abs(d)) / bound[q])
    return worst


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_ragged_against_exact_qd(cuda_lib, ta, tb):
    m, n, k = 70, 50, 90
    A, B, C, al, be = qd_case(1000, ta, tb, m, n, k, pad=3)
    got = run_qd(cuda_lib, ta, tb, m, n, k, A, B, C, al, be)
    assert qd_is_normalised(got)
    rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    assert max_err_over_bound(got, ta, tb, m, n, k, A, B, C, al, be, rr.ravel(),
                              cc.ravel()) <= 1.0


def test_larger_sampled(cuda_lib):
    m = n = k = 300
    A, B, C, al, be = qd_case(1001, "N", "N", m, n, k)
    got = run_qd(cuda_lib, "N", "N", m, n, k, A, B, C, al, be)
    assert qd_is_normalised(got)
    rows, cols = sample_blocks(m, n, bs=16, count=8, seed=1002)
    assert max_err_over_bound(got, "N", "N", m, n, k, A, B, C, al, be, rows, cols) <= 1.0


def test_integer_inputs_exact(cuda_lib):
    g = datagen.rng(1003)
    m, n, k = 40, 33, 65
    A = g.integers(-99, 100, (m, k)).astype(np.float64)
    B = g.integers(-99, 100, (k, n)).astype(np.float64)
    z = lambda P: np.zeros_like(P, order="F")
    Aq = (np.asfortranarray(A), z(A), z(A), z(A))
    Bq = (np.asfortranarray(B), z(B), z(B), z(B))
    Cq = tuple(np.full((m, n), np.nan, order="F") for _ in range(4))
    got = run_qd(cuda_lib, "N", "N", m, n, k, Aq, Bq, Cq, (1.0, 0, 0, 0), (0.0, 0, 0, 0))
    assert np.array_equal(got[0], A @ B)
    assert not got[1].any() and not got[2].any() and not got[3].any()


def test_alpha_zero_beta_zero_quick_returns_and_errors(cuda_lib):
    mp = cuda_lib
    m, n, k = 20, 30, 10
    A, B, C, al, be = qd_case(1004, "N", "N", m, n, k)
    nanA = tuple(np.full_like(P, np.nan) for P in A)
    got = run_qd(mp, "N", "N", m, n, k, nanA, nanA, C, (0.0, 0, 0, 0), be)
    rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    ex = oracle.exact_qd_gemm_entries("N", "N", k, (0.0, 0, 0, 0), A, B, be, C, rr.ravel(),
                                      cc.ravel())
    bound = qd_bound_entries("N", "N", m, n, 1, (0.0, 0.0), A, B, be, C, rr.ravel(), cc.ravel())
    diff = np.abs(sum(got[t].ravel() - ex[t] for t in range(4)))
    assert (diff <= bound).all()
    # alpha = 1, beta = 0 with NaN C: equals the exact product within the bound
    nanC = tuple(np.full_like(P, np.nan) for P in C)
    got = run_qd(mp, "N", "N", m, n, k, A, B, nanC, (1.0, 0, 0, 0), (0.0, 0, 0, 0))
    assert np.isfinite(got[0]).all() and qd_is_normalised(got)
    # quick returns leave C untouched
    dA, dB, dC = dev4(A), dev4(B), dev4(C)
    mp.mp_qd_Rgemm("N", "N", 0, n, k, al, dA, m, dB, k, be, dC, m)
    mp.mp_qd_Rgemm("N", "N", m, n, k, (0.0, 0, 0, 0), dA, m, dB, k, (1.0, 0, 0, 0), dC, m)
    back = host4(dC)
    assert all(np.array_equal(back[t], C[t]) for t in range(4))
    bad = [(("X", "N", m, n, k, m, k, m), -1), (("N", "X", m, n, k, m, k, m), -2),
           (("N", "N", -1, n, k, m, k, m), -3), (("N", "N", m, -1, k, m, k, m), -4),
           (("N", "N", m, n, -1, m, k, m), -5), (("N", "N", m, n, k, m - 1, k, m), -8),
           (("N", "N", m, n, k, m, k - 1, m), -10), (("N", "N", m, n, k, m, k, m - 1), -13)]
    for (ta, tb, mm, nn, kk, lda, ldb, ldc), code in bad:
        rc = mp.mp_qd_Rgemm(ta, tb, mm, nn, kk, al, dA, lda, dB, ldb, be, dC, ldc, check=False)
        assert rc == code, (ta, tb, rc)


def test_deterministic(cuda_lib):
    m, n, k = 64, 96, 120
    A, B, C, al, be = qd_case(1005, "T", "N", m, n, k)
    a = run_qd(cuda_lib, "T", "N", m, n, k, A, B, C, al, be)
    b = run_qd(cuda_lib, "T", "N", m, n, k, A, B, C, al, be)
    assert all(np.array_equal(a[t], b[t]) for t in range(4))
