"""Parity of the split-precision (sliced) Rgemm CUDA path (GPU).

Each step is checked on its own against the oracle:
  scaling maxima and digit planes -- bit-exact (integer work),
  band products P_b -- bit-exact against integer products of the oracle's
  digits (so the tensor-core accumulation is checked for exactness),
  the final C -- within the accuracy bound of the exact result.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import datagen
import oracle
from oracle import ozaki_ref as oz
from gpucase import check_against_exact, dev, host, sample_blocks

pytestmark = pytest.mark.gpu


def run_sliced(mp, c, slices=0, ws=None):
    A, B, C = dev(c.A), dev(c.B), dev(c.C)
    need = mp.mp_dd_Rgemm_sliced_workspace(c.m, c.n, c.k, slices)
    if ws is None or ws.numel() < need:
        ws = mp.workspace(need)
    mp.mp_dd_Rgemm_sliced(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, c.A[0].shape[0], B,
                          c.B[0].shape[0], c.beta, C, c.C[0].shape[0], slices, ws, ws.numel())
    torch.cuda.synchronize()
    assert mp.mp_dd_workspace_status(ws) == 0
    return host(C, c.m, c.n), ws


def ws_view(ws, off, count, dtype):
    return ws[off: off + count * np.dtype(dtype).itemsize].cpu().numpy().view(dtype)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_intermediates_bit_exact(cuda_lib, ta, tb):
    m, n, k, S = 150, 70, 200, 14
    c = datagen.gemm_case(200 + "NT".index(ta) * 2 + "NT".index(tb), ta, tb, m, n, k, pad=2)
    got, ws = run_sliced(cuda_lib, c, S)
    L = cuda_lib.mp_dd_sliced_layout(m, n, k, S)
    mp_, np_, kp = L["m_pad"], L["n_pad"], L["k_pad"]
    DA, ea = oz.split_matrix(*oz.op_rows(c.A, ta == "T", m, k), S)
    DB, fb = oz.split_matrix(*oz.op_cols(c.B, tb == "T", k, n), S)
    # scaling maxima: bit patterns of max |hi|
    rmax = ws_view(ws, L["rowmax"], mp_, np.uint64)[:m]
    Ah = oz.op_rows(c.A, ta == "T", m, k)[0]
    assert np.array_equal(rmax, np.abs(Ah).max(axis=1).view(np.uint64))
    # digit planes, including the zero padding
    da = ws_view(ws, L["digits_a"], S * mp_ * kp, np.float16).reshape(S, mp_, kp)
    db = ws_view(ws, L["digits_b"], S * np_ * kp, np.float16).reshape(S, np_, kp)
    assert np.array_equal(da[:, :m, :k].astype(np.int64), DA)
    assert np.array_equal(db[:, :n, :k].astype(np.int64), DB)
    assert not da[:, m:, :].any() and not da[:, :, k:].any() and not db[:, n:, :].any()
    # band products from the oracle's digits
    P = oz.band_products(DA, DB)
    bands = ws_view(ws, L["bands"], S * np_ * mp_, np.int32).reshape(S, np_, mp_)
    assert np.array_equal(bands[:, :n, :m].transpose(0, 2, 1).astype(np.int64), P)
    # final result within the bound of the exact result
    assert check_against_exact(c, got) <= 1.0


def test_accumulation_exact_at_the_chunk_limit(cuda_lib):
    """Every product is 128 * 128 = 2^14 and all have one sign, so each
    512-product run of the fp32 accumulator reaches exactly 2^23."""
    m = n = 128
    k = 2048
    x = 0.5 - 2.0 ** -40
    A = (np.full((m, k), x, order="F"), np.zeros((m, k), order="F"))
    B = (np.full((k, n), x, order="F"), np.zeros((k, n), order="F"))
    C = (np.zeros((m, n), order="F"), np.zeros((m, n), order="F"))
    c = datagen.GemmCase("N", "N", m, n, k, (1.0, 0.0), A, B, (0.0, 0.0), C)
    got, ws = run_sliced(cuda_lib, c, 14)
    L = cuda_lib.mp_dd_sliced_layout(m, n, k, 14)
    da = ws_view(ws, L["digits_a"], L["m_pad"] * L["k_pad"], np.float16)
    assert (da == 128).all()                      # the top digit is maximal everywhere
    bands = ws_view(ws, L["bands"], L["n_pad"] * L["m_pad"], np.int32)
    assert (bands == k * 128 * 128).all()         # band 0 exact: 2^25 from 4 runs of 2^23
    assert check_against_exact(c, got) <= 1.0


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 7), (129, 130, 65), (200, 64, 300)])
def test_ragged_shapes(cuda_lib, shape):
    m, n, k = shape
    c = datagen.gemm_case(300 + sum(shape), "N", "T", m, n, k, pad=1)
    got, _ = run_sliced(cuda_lib, c)
    assert check_against_exact(c, got) <= 1.0


def test_beta_zero_alpha_zero_and_errors(cuda_lib):
    c = datagen.gemm_case(7, "N", "N", 90, 60, 70)
    c.beta = (0.0, 0.0)
    c.C = (np.full_like(c.C[0], np.nan), np.full_like(c.C[1], np.nan))
    got, ws = run_sliced(cuda_lib, c)
    assert np.isfinite(got[0]).all()
    c2 = datagen.gemm_case(7, "N", "N", 90, 60, 70)
    c2.beta = (0.0, 0.0)
    assert check_against_exact(c2, got) <= 1.0
    # argument errors
    z = dev(c.C)
    rc = cuda_lib.mp_dd_Rgemm_sliced("N", "N", 90, 60, 70, (1.0, 0.0), z, 90, z, 70, (0.0, 0.0),
                                     z, 90, 16, ws, ws.numel(), check=False)
    assert rc == -14
    rc = cuda_lib.mp_dd_Rgemm_sliced("N", "N", 90, 60, 70, (1.0, 0.0), z, 90, z, 70, (0.0, 0.0),
                                     z, 90, 14, ws, 100, check=False)
    assert rc == 2003


@pytest.mark.parametrize("ill", [None, "outer"])
def test_config2_sampled_blocks_2048(cuda_lib, ill):
    """2048^3, well- and ill-scaled inputs: sampled 64 x 64 blocks against
    the exact tier, and the plain path on the same inputs for comparison."""
    n = 2048
    c = datagen.gemm_case(2, "N", "N", n, n, n, ill=ill)
    got, ws = run_sliced(cuda_lib, c)
    rep = cuda_lib.mp_dd_split_report(ws)
    assert rep["width_bits"] == 112 and rep["count"] == 14 and rep["max_err_est"] < 0.05
    rows, cols = sample_blocks(n, n, bs=16, count=8)
    ratio = check_against_exact(c, got, rows, cols)
    assert ratio <= 1.0


def test_wide_tiles_4096x4096_k256_bands_and_result(cuda_lib):
    """m = n = 4096 selects the 128 x 256 tile kernel: band sums at sampled
    entries bit-exact against the integer oracle, the result within the bound."""
    m = n = 4096
    k, S = 256, 14
    c = datagen.gemm_case(400, "N", "N", m, n, k)
    got, ws = run_sliced(cuda_lib, c, S)
    L = cuda_lib.mp_dd_sliced_layout(m, n, k, S)
    assert L["n_pad"] % 256 == 0
    g = datagen.rng(401)
    rows = np.concatenate([[0, 127, 128, m - 1], g.integers(0, m, 12)])
    cols = np.concatenate([[0, 255, 256, n - 1], g.integers(0, n, 12)])
    Ah, Al = oz.op_rows(c.A, False, m, k)
    Bh, Bl = oz.op_cols(c.B, False, k, n)
    DA, _ = oz.split_matrix(Ah[rows], Al[rows], S)
    DB, _ = oz.split_matrix(Bh[cols], Bl[cols], S)
    P = oz.band_products(DA, DB)
    mp_, np_ = L["m_pad"], L["n_pad"]
    bands = ws_view(ws, L["bands"], S * np_ * mp_, np.int32).reshape(S, np_, mp_)
    got_bands = bands[:, cols][:, :, rows].transpose(0, 2, 1).astype(np.int64)
    assert np.array_equal(got_bands, P)
    rr, cc = sample_blocks(m, n, bs=16, count=8)
    assert check_against_exact(c, got, rr, cc) <= 1.0
