"""dd Rgetrf / Rgetrs through the C ABI (GPU).

Pins: a dyadic matrix with a known permutation and L U factorisation is
factored exactly (L, U and ipiv bit for bit) at square, tall and wide
shapes spanning several recursion levels; random dd matrices give the
oracle's pivots, factors within the forward error that the backward bound
allows, the LAPACK residual ratio (< 30) and the componentwise backward
bound with P A - L U evaluated exactly; an exactly singular column gives
LAPACK's info and the factorisation completes; Rgetrs solves A X = B and
A^T X = B within the LAPACK ratio; argument errors follow DGETRF / DGETRS.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import datagen
import oracle
from ddcheck import EPS_DD
from gpucase import dev, host
from lucheck import dyadic_lu_case, lu_backward_over_bound, lu_residual_ratio

pytestmark = pytest.mark.gpu


def gpu_getrf(mp, A, m, n):
    dA = dev(A)
    ipiv = torch.zeros(max(1, min(m, n)), dtype=torch.int64, device="cuda")
    info = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    mp.mp_dd_Rgetrf(m, n, dA, A[0].shape[0], ipiv, info)
    torch.cuda.synchronize()
    return host(dA), ipiv[:min(m, n)].cpu().numpy(), int(info.item())


@pytest.mark.parametrize("m,n", [(150, 150), (170, 110), (90, 160), (1, 5), (6, 1)])
def test_dyadic_factorisation_exact(cuda_lib, m, n):
    A, L, U, ipiv = dyadic_lu_case(700 + m + n, m, n)
    (lh, ll), piv, info = gpu_getrf(cuda_lib, (A, np.zeros_like(A)), m, n)
    assert info == 0
    assert np.array_equal(piv, ipiv)
    assert not ll.any()
    mn = min(m, n)
    assert np.array_equal(np.tril(lh[:, :mn], -1), np.tril(L, -1))
    assert np.array_equal(np.triu(lh[:mn, :]), U)


@pytest.mark.parametrize("m,n", [(200, 200), (260, 170), (170, 260)])
def test_random_against_oracle(cuda_lib, m, n):
    g = datagen.rng(710 + m)
    A = datagen.dd_matrix(g, m, n, m + 3)
    (lh, ll), piv, info = gpu_getrf(cuda_lib, A, m, n)
    oh, ol, opiv, oinfo = oracle.dd_getrf(A, m, n)
    assert info == 0 == oinfo
    assert np.array_equal(piv, opiv)
    got = (lh[:m, :n], ll[:m, :n])
    assert lu_residual_ratio(A, got, piv, m, n) < 30
    rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    assert lu_backward_over_bound(A, got, piv, m, n, rr.ravel(), cc.ravel()) <= 1.0
    # both factorisations are backward stable with the same pivots; on these
    # matrices (growth ~ 10, condition ~ 1e3) they agree far below 2^-80
    diff = np.abs((lh[:m, :n] - oh[:m, :n]) + (ll[:m, :n] - ol[:m, :n]))
    assert diff.max() <= 2.0 ** -80 * np.abs(oh[:m, :n]).max()


def test_larger_sampled(cuda_lib):
    n = 1024
    g = datagen.rng(720)
    A = datagen.dd_matrix(g, n, n)
    (lh, ll), piv, info = gpu_getrf(cuda_lib, A, n, n)
    _, _, opiv, oinfo = oracle.dd_getrf(A)
    assert info == 0 == oinfo and np.array_equal(piv, opiv)
    rows = g.integers(0, n, 3000)
    cols = g.integers(0, n, 3000)
    rows[:64], cols[64:128] = n - 1, n - 1
    assert lu_backward_over_bound(A, (lh, ll), piv, n, n, rows, cols) <= 1.0


def test_singular_column_info(cuda_lib):
    n = 100
    g = datagen.rng(730)
    A = datagen.dd_matrix(g, n, n)
    for P in A:
        P[:, 70] = 0.0
    (lh, ll), piv, info = gpu_getrf(cuda_lib, A, n, n)
    _, _, opiv, oinfo = oracle.dd_getrf(A)
    assert info == oinfo == 71
    assert np.array_equal(piv, opiv)
    assert np.isfinite(lh).all()


@pytest.mark.parametrize("trans", ["N", "T"])
def test_getrs_lapack_ratio(cuda_lib, trans):
    n, nrhs = 230, 6
    g = datagen.rng(740)
    A = datagen.dd_matrix(g, n, n)
    B = datagen.dd_matrix(g, n, nrhs, n + 2)
    dA = dev(A)
    ipiv = torch.zeros(n, dtype=torch.int64, device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    cuda_lib.mp_dd_Rgetrf(n, n, dA, n, ipiv, info)
    dB = dev(B)
    cuda_lib.mp_dd_Rgetrs(trans, n, nrhs, dA, n, ipiv, dB, n + 2)
    X = host(dB, n, nrhs)
    assert int(info.item()) == 0
    rr, cc = np.meshgrid(np.arange(n), np.arange(nrhs), indexing="ij")
    R = oracle.exact_gemm_entries(trans, "N", n, (-1.0, 0.0), A, X, (1.0, 0.0),
                                  (B[0][:n], B[1][:n]), rr.ravel(), cc.ravel())
    An = np.abs(A[0]).sum(axis=0).max()
    Xn = np.abs(X[0]).sum(axis=0).max()
    assert np.abs(R[0]).reshape(n, nrhs).sum(axis=0).max() / (An * Xn * EPS_DD) < 30
    ref = oracle.dd_getrs(trans, oracle.dd_getrf(A)[:2], oracle.dd_getrf(A)[2],
                          (B[0][:n], B[1][:n]))
    assert np.abs((X[0] - ref[0]) + (X[1] - ref[1])).max() <= 2.0 ** -80 * np.abs(ref[0]).max()


def test_errors_and_empty(cuda_lib):
    mp = cuda_lib
    A = dev(datagen.dd_matrix(datagen.rng(750), 8, 8))
    ipiv = torch.zeros(8, dtype=torch.int64, device="cuda")
    info = torch.full((1,), 5, dtype=torch.int64, device="cuda")
    assert mp.mp_dd_Rgetrf(-1, 8, A, 8, ipiv, info, check=False) == -1
    assert mp.mp_dd_Rgetrf(8, -1, A, 8, ipiv, info, check=False) == -2
    assert mp.mp_dd_Rgetrf(8, 8, A, 7, ipiv, info, check=False) == -4
    assert mp.mp_dd_Rgetrf(8, 8, A, 8, None, info, check=False) == -5
    assert mp.mp_dd_Rgetrf(8, 8, A, 8, ipiv, None, check=False) == -6
    mp.mp_dd_Rgetrf(0, 8, A, 1, ipiv, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert mp.mp_dd_Rgetrs("X", 8, 1, A, 8, ipiv, A, 8, check=False) == -1
    assert mp.mp_dd_Rgetrs("N", -1, 1, A, 8, ipiv, A, 8, check=False) == -2
    assert mp.mp_dd_Rgetrs("N", 8, -1, A, 8, ipiv, A, 8, check=False) == -3
    assert mp.mp_dd_Rgetrs("N", 8, 1, A, 7, ipiv, A, 8, check=False) == -5
    assert mp.mp_dd_Rgetrs("N", 8, 1, A, 8, None, A, 8, check=False) == -6
    assert mp.mp_dd_Rgetrs("N", 8, 1, A, 8, ipiv, A, 7, check=False) == -8


@pytest.mark.parametrize("m,n", [(3000, 40), (2500, 33)])
def test_tall_panels_over_many_ctas(cuda_lib, m, n):
    """Panels of up to 32 columns run as one cooperative launch with their
    rows spread over up to one CTA per SM (here ~150 CTAs of ~20 rows): the
    oracle's pivots, the LAPACK ratio and the backward bound on sampled
    entries."""
    g = datagen.rng(730 + n)
    A = datagen.dd_matrix(g, m, n)
    (lh, ll), piv, info = gpu_getrf(cuda_lib, A, m, n)
    _, _, opiv, oinfo = oracle.dd_getrf(A, m, n)
    assert info == 0 == oinfo and np.array_equal(piv, opiv)
    assert lu_residual_ratio(A, (lh, ll), piv, m, n) < 30
    rows = g.integers(0, m, 2000)
    cols = g.integers(0, n, 2000)
    rows[:40], cols[40:80] = m - 1, n - 1
    assert lu_backward_over_bound(A, (lh, ll), piv, m, n, rows, cols) <= 1.0


def test_deterministic(cuda_lib):
    g = datagen.rng(740)
    A = datagen.dd_matrix(g, 300, 300)
    a = gpu_getrf(cuda_lib, A, 300, 300)
    b = gpu_getrf(cuda_lib, A, 300, 300)
    assert np.array_equal(a[0][0], b[0][0]) and np.array_equal(a[0][1], b[0][1])
    assert np.array_equal(a[1], b[1])
