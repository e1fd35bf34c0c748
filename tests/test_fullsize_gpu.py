"""Parity at the benchmarked sizes, in the benchmarked launch configurations (GPU).

The default benchmark's plain step (Rgemm NN and TN, Rsyrk U/N at
m = n = k = 4096, the same seeded inputs) and the split-precision workload
(the residue-form and the sliced Rgemm NN at 8192, well-scaled and outer
ill-scaled, the same seeded inputs) are run through the C ABI as the
benchmark runs them, and sampled 16 x 16 blocks (the four corners, the
diagonal, random interior blocks) are compared with the oracle's exact tier
within the accuracy bound 4 k 2^-104 (|alpha||A||B| + |beta||C|).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import datagen
from gpucase import check_against_exact, dev, host, run_gemm, sample_blocks

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,ta", [(1, "N"), (2, "T")])
def test_plain_rgemm_4096(cuda_lib, seed, ta):
    n = 4096
    c = datagen.gemm_case(seed, ta, "N", n, n, n)
    got = run_gemm(c)
    rr, cc = sample_blocks(n, n, bs=16, count=8, seed=seed)
    assert check_against_exact(c, got, rr, cc) <= 1.0


def test_plain_rsyrk_4096(cuda_lib):
    mp = cuda_lib
    n = 4096
    g = datagen.rng(3)
    A = datagen.dd_matrix(g, n, n)
    C = datagen.dd_matrix(g, n, n)
    al, be = datagen.dd_scalar(g), datagen.dd_scalar(g)
    dC = dev(C)
    mp.mp_dd_Rsyrk("U", "N", n, n, al, dev(A), n, be, dC, n)
    got = host(dC)
    rr, cc = sample_blocks(n, n, bs=16, count=8, seed=3)
    keep = rr <= cc
    c = datagen.GemmCase("N", "T", n, n, n, al, A, A, be, C)
    assert check_against_exact(c, got, rr[keep], cc[keep]) <= 1.0
    # the lower triangle is C's own
    low = rr > cc
    assert np.array_equal(got[0][rr[low], cc[low]], C[0][rr[low], cc[low]])


@pytest.fixture(scope="module", params=[None, "outer"])
def case_8192(request):
    return datagen.gemm_case(2, "N", "N", 8192, 8192, 8192, ill=request.param)


@pytest.mark.parametrize("form", ["crt", "sliced"])
def test_split_precision_8192(cuda_lib, case_8192, form):
    mp = cuda_lib
    c = case_8192
    n = c.m
    A, B, C = dev(c.A), dev(c.B), dev(c.C)
    if form == "crt":
        ws = mp.workspace(mp.mp_dd_Rgemm_crt_workspace(n, n, n))
        mp.mp_dd_Rgemm_crt("N", "N", n, n, n, c.alpha, A, n, B, n, c.beta, C, n, ws, ws.numel())
    else:
        ws = mp.workspace(mp.mp_dd_Rgemm_sliced_workspace(n, n, n, 14))
        mp.mp_dd_Rgemm_sliced("N", "N", n, n, n, c.alpha, A, n, B, n, c.beta, C, n, 14, ws,
                              ws.numel())
    torch.cuda.synchronize()
    assert mp.mp_dd_workspace_status(ws) == 0
    got = host(C)
    del A, B, C, ws
    torch.cuda.empty_cache()
    rr, cc = sample_blocks(n, n, bs=16, count=8, seed=5)
    assert check_against_exact(c, got, rr, cc) <= 1.0
