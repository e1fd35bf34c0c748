"""The TMA-staged plain kernel (dd_gemm_tma.cu) against the register-staged
one (GPU).

Both compute every entry with the same dd multiply-add sequence (l = 0 .. k-1,
renormalisation every 4 steps, the same epilogue), so results must be bitwise
equal: all four transposes, ragged shapes (partial tiles in m, n and k, k
below one panel), non-tight even leading dimensions, Rsyrk both triangles and
both transposes, alpha / beta special cases, and one product large enough
for the automatic choice; plus the exact tier on one case.  Odd leading
dimensions and planes not on 16-byte boundaries must fall back to the
register-staged kernel (equal results as well).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import datagen
from gpucase import check_against_exact, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture()
def staging(cuda_lib):
    yield cuda_lib.mp_dd_set_plain_staging
    cuda_lib.mp_dd_set_plain_staging(0)


def gemm_both(mp, staging, c, offset=0):
    outs = []
    for mode in (1, 2):
        staging(mode)
        A, B = dev(c.A), dev(c.B)
        if offset:   # the same planes one element further on: 8-byte aligned only
            A = tuple(x.t().reshape(-1)[offset:] for x in A)
            B = tuple(x.t().reshape(-1)[offset:] for x in B)
        C = dev(c.C)
        mp.mp_dd_Rgemm(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, c.A[0].shape[0], B,
                       c.B[0].shape[0], c.beta, C, c.C[0].shape[0])
        outs.append(host(C, c.m, c.n))
    return outs


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("shape", [(64, 64, 16), (130, 70, 45), (5, 200, 3), (257, 129, 260),
                                   (64, 64, 1)])
def test_tma_equals_register_staging(cuda_lib, staging, ta, tb, shape):
    m, n, k = shape
    c = datagen.gemm_case(900 + m + n + k, ta, tb, m, n, k, pad=2)
    regs, tma = gemm_both(cuda_lib, staging, c)
    assert np.array_equal(regs[0], tma[0]) and np.array_equal(regs[1], tma[1])


@pytest.mark.parametrize("alpha,beta", [((1.0, 0.0), (0.0, 0.0)), ((-1.0, 0.0), (1.0, 0.0)),
                                        (None, None)])
def test_tma_alpha_beta_cases_and_exact_tier(cuda_lib, staging, alpha, beta):
    c = datagen.gemm_case(950, "T", "N", 150, 140, 100, alpha=alpha, beta=beta, pad=2)
    regs, tma = gemm_both(cuda_lib, staging, c)
    assert np.array_equal(regs[0], tma[0]) and np.array_equal(regs[1], tma[1])
    assert check_against_exact(c, tma) <= 1.0


def test_tma_large_automatic_choice(cuda_lib, staging):
    """4096 x 4096 x 64 fills the SMs with 64 x 64 tiles as well as with any
    smaller tile: mode 0 takes the TMA kernel; all three agree bit for bit."""
    m = n = 4096
    k = 64
    c = datagen.gemm_case(960, "N", "N", m, n, k)
    regs, tma = gemm_both(cuda_lib, staging, c)
    staging(0)
    A, B, C = dev(c.A), dev(c.B), dev(c.C)
    cuda_lib.mp_dd_Rgemm("N", "N", m, n, k, c.alpha, A, m, B, k, c.beta, C, m)
    auto = host(C)
    assert np.array_equal(regs[0], tma[0]) and np.array_equal(regs[1], tma[1])
    assert np.array_equal(auto[0], tma[0]) and np.array_equal(auto[1], tma[1])


@pytest.mark.parametrize("uplo", ["U", "L"])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_tma_rsyrk_triangle(cuda_lib, staging, uplo, trans):
    mp = cuda_lib
    n, k = 200, 90
    g = datagen.rng(970 + "UL".index(uplo) * 2 + "NT".index(trans))
    ar, ac = (n, k) if trans == "N" else (k, n)
    A = datagen.dd_matrix(g, ar, ac, ar + 2)
    C0 = datagen.dd_matrix(g, n, n, n + 2)
    al, be = datagen.dd_scalar(g), datagen.dd_scalar(g)
    outs = []
    for mode in (1, 2):
        staging(mode)
        dA, dC = dev(A), dev(C0)
        mp.mp_dd_Rsyrk(uplo, trans, n, k, al, dA, ar + 2, be, dC, n + 2)
        outs.append(host(dC))
    assert np.array_equal(outs[0][0], outs[1][0], equal_nan=True)
    assert np.array_equal(outs[0][1], outs[1][1], equal_nan=True)


def test_fallback_on_odd_ld_and_unaligned_planes(cuda_lib, staging):
    c = datagen.gemm_case(980, "N", "N", 100, 90, 80, pad=1)      # ld = 101, 81: odd
    regs, tma = gemm_both(cuda_lib, staging, c)
    assert np.array_equal(regs[0], tma[0]) and np.array_equal(regs[1], tma[1])
    c2 = datagen.gemm_case(981, "N", "N", 100, 90, 80, pad=2)
    # 8-byte offset planes (the shift brings the NaN padding row in: NaNs
    # must come out in the same places)
    a = gemm_both(cuda_lib, staging, c2, offset=1)
    assert np.array_equal(a[0][0], a[1][0], equal_nan=True)
    assert np.array_equal(a[0][1], a[1][1], equal_nan=True)


def test_staging_mode_errors(cuda_lib):
    assert cuda_lib._LIB.mp_dd_set_plain_staging(3) == -1
    assert cuda_lib._LIB.mp_dd_set_plain_staging(0) == 0
