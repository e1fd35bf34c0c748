"""CTA pairs for the 256-wide band / residue products (GPU).

The products are exact integers, so a CTA pair computing a 256 x 256 tile
with the 2-SM MMA must give bitwise the same residue products and results
as one CTA per 128 x 256 tile: checked on the residue form (Rgemm, ragged edges, the
Rsyrk triangles) and the sliced form, plus one odd tile count that keeps
single CTAs.  Results are also held against the oracle's exact tier.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import datagen
from gpucase import check_against_exact, dev, host, sample_blocks

pytestmark = pytest.mark.gpu


def crt_once(mp, c, pairs):
    mp.mp_dd_set_band_pairs(pairs)
    try:
        A, B, C = dev(c.A), dev(c.B), dev(c.C)
        ws = mp.workspace(mp.mp_dd_Rgemm_crt_workspace(c.m, c.n, c.k))
        mp.mp_dd_Rgemm_crt(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, c.A[0].shape[0], B,
                           c.B[0].shape[0], c.beta, C, c.C[0].shape[0], ws, ws.numel())
        torch.cuda.synchronize()
        assert mp.mp_dd_workspace_status(ws) == 0
        L = mp.mp_dd_crt_layout(c.m, c.n, c.k)
        N = mp.mp_dd_split_report(ws)["count"]
        nb = N * L["n_pad"] * L["m_pad"]
        prods = ws[L["products"]: L["products"] + nb].cpu().numpy().copy()
        return host(C, c.m, c.n), prods
    finally:
        mp.mp_dd_set_band_pairs(0)


@pytest.mark.parametrize("shape", [(4096, 2560, 192), (4000, 2600, 130), (3900, 2600, 64)])
def test_crt_pairs_bitwise_equal_single(cuda_lib, shape):
    """(4096, 2560) and (4000, 2600): 32 tile rows, pairs; (3900, 2600): 31
    tile rows, single CTAs in both modes."""
    m, n, k = shape
    c = datagen.gemm_case(780 + k, "N", "T", m, n, k, pad=1)
    got1, p1 = crt_once(cuda_lib, c, 1)
    got0, p0 = crt_once(cuda_lib, c, 2)
    assert np.array_equal(p1, p0)
    assert np.array_equal(got1[0], got0[0]) and np.array_equal(got1[1], got0[1])
    rr, cc = sample_blocks(m, n, bs=16, count=6)
    assert check_against_exact(c, got1, rr, cc) <= 1.0


@pytest.mark.parametrize("uplo", ["U", "L"])
def test_rsyrk_crt_pairs_bitwise_equal_single(cuda_lib, uplo):
    """The triangle skips whole pairs only when both tiles lie outside."""
    mp = cuda_lib
    n, k = 4096, 96
    g = datagen.rng(790 + "UL".index(uplo))
    A = datagen.dd_matrix(g, n, k, n)
    C = datagen.dd_matrix(g, n, n, n)
    al, be = datagen.dd_scalar(g), datagen.dd_scalar(g)
    outs = []
    for pairs in (1, 2):
        mp.mp_dd_set_band_pairs(pairs)
        try:
            dA, dC = dev(A), dev(C)
            ws = mp.workspace(mp.mp_dd_Rsyrk_crt_workspace(n, k))
            mp.mp_dd_Rsyrk_crt(uplo, "N", n, k, al, dA, n, be, dC, n, ws, ws.numel())
            torch.cuda.synchronize()
            assert mp.mp_dd_workspace_status(ws) == 0
            outs.append(host(dC))
        finally:
            mp.mp_dd_set_band_pairs(0)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    r, cc = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    keep = (r <= cc) if uplo == "U" else (r >= cc)
    untouched = ~keep
    assert np.array_equal(outs[0][0][untouched], C[0][untouched])
    c = datagen.GemmCase("N", "T", n, n, k, al, A, A, be, C)
    rows, cols = np.nonzero(keep)
    pick = np.linspace(0, rows.size - 1, 3000).astype(int)
    assert check_against_exact(c, outs[0], rows[pick], cols[pick]) <= 1.0


def test_sliced_pairs_bitwise_equal_single(cuda_lib):
    mp = cuda_lib
    m, n, k = 4096, 2560, 128
    c = datagen.gemm_case(795, "N", "N", m, n, k)
    outs = []
    for pairs in (1, 2):
        mp.mp_dd_set_band_pairs(pairs)
        try:
            A, B, C = dev(c.A), dev(c.B), dev(c.C)
            ws = mp.workspace(mp.mp_dd_Rgemm_sliced_workspace(m, n, k, 0))
            mp.mp_dd_Rgemm_sliced("N", "N", m, n, k, c.alpha, A, m, B, k, c.beta, C, m, 0, ws,
                                  ws.numel())
            torch.cuda.synchronize()
            assert mp.mp_dd_workspace_status(ws) == 0
            outs.append(host(C, m, n))
        finally:
            mp.mp_dd_set_band_pairs(0)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    rr, cc = sample_blocks(m, n, bs=16, count=6)
    assert check_against_exact(c, outs[0], rr, cc) <= 1.0


def test_set_band_pairs_rejects_other_modes(cuda_lib):
    assert cuda_lib.lib().mp_dd_set_band_pairs(3) == -1
    assert cuda_lib.lib().mp_dd_set_band_pairs(-1) == -1
    assert cuda_lib.lib().mp_dd_set_band_pairs(0) == 0
