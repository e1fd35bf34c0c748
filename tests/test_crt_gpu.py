"""Parity of the residue (CRT) form of the split-precision Rgemm (GPU).

Residue planes and the products reduced mod each modulus are integer work:
bit-exact against the oracle (oracle/ozaki_ref.py).  The result is checked
against the oracle's exact tier within the accuracy bound.
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


def run_crt(mp, c):
    A, B, C = dev(c.A), dev(c.B), dev(c.C)
    ws = mp.workspace(mp.mp_dd_Rgemm_crt_workspace(c.m, c.n, c.k))
    mp.mp_dd_Rgemm_crt(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, c.A[0].shape[0], B,
                       c.B[0].shape[0], c.beta, C, c.C[0].shape[0], ws, ws.numel())
    torch.cuda.synchronize()
    assert mp.mp_dd_workspace_status(ws) == 0
    return host(C, c.m, c.n), ws


def view(ws, off, count, dtype):
    return ws[off: off + count * np.dtype(dtype).itemsize].cpu().numpy().view(dtype)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_crt_intermediates_bit_exact(cuda_lib, ta, tb):
    m, n, k = 70, 50, 150
    c = datagen.gemm_case(700 + "NT".index(ta) * 2 + "NT".index(tb), ta, tb, m, n, k, pad=1)
    got, ws = run_crt(cuda_lib, c)
    L = cuda_lib.mp_dd_crt_layout(m, n, k)
    assert L["moduli"] == oz.crt_moduli(len(L["moduli"]))
    rep = cuda_lib.mp_dd_split_report(ws)
    N, W = rep["count"], rep["width_bits"]
    assert W == 112 and N <= len(L["moduli"])   # well-scaled inputs: the narrowest width
    mods = L["moduli"][:N]
    P = 1
    for p in mods:
        P *= p
    assert P >= k * 2 ** (2 * W)       # the reconstruction is exact
    mp_, np_, kp = L["m_pad"], L["n_pad"], L["k_pad"]
    RA, _ = oz.residue_planes(*oz.op_rows(c.A, ta == "T", m, k), mods, W // 8)
    RB, _ = oz.residue_planes(*oz.op_cols(c.B, tb == "T", k, n), mods, W // 8)
    ra = view(ws, L["residues_a"], N * mp_ * kp, np.float16).reshape(N, mp_, kp)
    rb = view(ws, L["residues_b"], N * np_ * kp, np.float16).reshape(N, np_, kp)
    assert np.array_equal(ra[:, :m, :k].astype(np.int64), RA)
    assert np.array_equal(rb[:, :n, :k].astype(np.int64), RB)
    assert not ra[:, m:, :].any() and not ra[:, :, k:].any()
    prods = view(ws, L["products"], N * np_ * mp_, np.uint8).reshape(N, np_, mp_)
    want = oz.crt_products(RA, RB, mods)
    assert np.array_equal(prods[:, :n, :m].transpose(0, 2, 1).astype(np.int64), want)
    assert check_against_exact(c, got) <= 1.0


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 7), (129, 130, 65), (200, 64, 300)])
def test_crt_ragged_shapes(cuda_lib, shape):
    m, n, k = shape
    c = datagen.gemm_case(710 + sum(shape), "N", "T", m, n, k, pad=1)
    got, _ = run_crt(cuda_lib, c)
    assert check_against_exact(c, got) <= 1.0


def test_crt_beta_zero_and_limits(cuda_lib):
    c = datagen.gemm_case(720, "N", "N", 90, 60, 70)
    c.beta = (0.0, 0.0)
    clean = datagen.gemm_case(720, "N", "N", 90, 60, 70)
    clean.beta = (0.0, 0.0)
    c.C = (np.full_like(c.C[0], np.nan), np.full_like(c.C[1], np.nan))
    got, ws = run_crt(cuda_lib, c)
    assert np.isfinite(got[0]).all() and check_against_exact(clean, got) <= 1.0
    z = dev(c.C)
    assert cuda_lib.mp_dd_Rgemm_crt("N", "N", 90, 60, 70, (1.0, 0.0), z, 90, z, 70, (0.0, 0.0),
                                    z, 90, ws, 100, check=False) == 2003


def test_crt_wide_tiles_and_ill_scaled(cuda_lib):
    """4096 x 4096 (k = 256) uses the 128 x 256 tile kernel; sampled product
    residues bit-exact, sampled results within the bound, with ill-scaled
    (outer) inputs."""
    m = n = 4096
    k = 256
    c = datagen.gemm_case(730, "N", "N", m, n, k, ill="outer")
    got, ws = run_crt(cuda_lib, c)
    L = cuda_lib.mp_dd_crt_layout(m, n, k)
    rep = cuda_lib.mp_dd_split_report(ws)
    assert rep["width_bits"] == 112
    mods = L["moduli"][:rep["count"]]
    g = datagen.rng(731)
    rows = np.concatenate([[0, m - 1], g.integers(0, m, 10)])
    cols = np.concatenate([[0, 255, 256, n - 1], g.integers(0, n, 8)])
    Ah, Al = oz.op_rows(c.A, False, m, k)
    Bh, Bl = oz.op_cols(c.B, False, k, n)
    RA, _ = oz.residue_planes(Ah[rows], Al[rows], mods)
    RB, _ = oz.residue_planes(Bh[cols], Bl[cols], mods)
    N, mp_, np_ = len(mods), L["m_pad"], L["n_pad"]
    prods = view(ws, L["products"], N * np_ * mp_, np.uint8).reshape(N, np_, mp_)
    sel = prods[:, cols][:, :, rows].transpose(0, 2, 1).astype(np.int64)
    assert np.array_equal(sel, oz.crt_products(RA, RB, mods))
    rr, cc = sample_blocks(m, n, bs=16, count=8)
    assert check_against_exact(c, got, rr, cc) <= 1.0


@pytest.mark.parametrize("ill", [None, "outer"])
def test_crt_config2_2048(cuda_lib, ill):
    n = 2048
    c = datagen.gemm_case(2, "N", "N", n, n, n, ill=ill)
    got, ws = run_crt(cuda_lib, c)
    rep = cuda_lib.mp_dd_split_report(ws)
    assert rep["width_bits"] == 112 and rep["count"] == 32 and rep["max_err_est"] < 0.01
    rr, cc = sample_blocks(n, n, bs=16, count=8)
    assert check_against_exact(c, got, rr, cc) <= 1.0


@pytest.mark.parametrize("uplo", ["U", "L"])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_rsyrk_crt_triangle_equals_rgemm_crt(cuda_lib, uplo, trans):
    """The Rsyrk form: only the uplo triangle is read and written (NaN in the
    other one stays NaN), and it equals mp_dd_Rgemm_crt on (A, A^T) bit for
    bit; the triangle meets the bound against the exact tier."""
    mp = cuda_lib
    n, k = 300, 200
    g = datagen.rng(760 + "UL".index(uplo) * 2 + "NT".index(trans))
    ar, ac = (n, k) if trans == "N" else (k, n)
    A = datagen.dd_matrix(g, ar, ac, ar + 2)
    C = datagen.dd_matrix(g, n, n, n + 1)
    al, be = datagen.dd_scalar(g), datagen.dd_scalar(g)
    r, cc = np.meshgrid(np.arange(n + 1), np.arange(n), indexing="ij")
    other = (r > cc) if uplo == "U" else (r < cc)
    other |= r >= n
    Cn = tuple(np.where(other, np.nan, P) for P in C)
    dA, dC = dev(A), dev(tuple(np.asfortranarray(P) for P in Cn))
    ws = mp.workspace(mp.mp_dd_Rsyrk_crt_workspace(n, k))
    mp.mp_dd_Rsyrk_crt(uplo, trans, n, k, al, dA, ar + 2, be, dC, n + 1, ws, ws.numel())
    got = host(dC)
    assert mp.mp_dd_workspace_status(ws) == 0
    assert np.isnan(got[0][other]).all() and np.isnan(got[1][other]).all()
    # the same triangle through the Rgemm form
    ta, tb = ("N", "T") if trans == "N" else ("T", "N")
    dC2 = dev(C)
    ws2 = mp.workspace(mp.mp_dd_Rgemm_crt_workspace(n, n, k))
    mp.mp_dd_Rgemm_crt(ta, tb, n, n, k, al, dA, ar + 2, dA, ar + 2, be, dC2, n + 1, ws2,
                       ws2.numel())
    ref = host(dC2)
    keep = ~other
    assert np.array_equal(got[0][keep], ref[0][keep])
    assert np.array_equal(got[1][keep], ref[1][keep])
    c = datagen.GemmCase(ta, tb, n, n, k, al, A, A, be, C)
    rows, cols = np.nonzero(keep[:n])
    pick = np.linspace(0, rows.size - 1, 4000).astype(int)
    assert check_against_exact(c, (got[0][:n], got[1][:n]), rows[pick], cols[pick]) <= 1.0


def test_rsyrk_crt_errors(cuda_lib):
    mp = cuda_lib
    A = dev(datagen.dd_matrix(datagen.rng(770), 8, 4))
    C = dev(datagen.dd_matrix(datagen.rng(771), 8, 8))
    ws = mp.workspace(mp.mp_dd_Rsyrk_crt_workspace(8, 4))
    assert mp.mp_dd_Rsyrk_crt("X", "N", 8, 4, (1.0, 0.0), A, 8, (0.0, 0.0), C, 8, ws, ws.numel(),
                              check=False) == -1
    assert mp.mp_dd_Rsyrk_crt("U", "X", 8, 4, (1.0, 0.0), A, 8, (0.0, 0.0), C, 8, ws, ws.numel(),
                              check=False) == -2
    assert mp.mp_dd_Rsyrk_crt("U", "N", 8, 4, (1.0, 0.0), A, 7, (0.0, 0.0), C, 8, ws, ws.numel(),
                              check=False) == -7
    assert mp.mp_dd_Rsyrk_crt("U", "N", 8, 4, (1.0, 0.0), A, 8, (0.0, 0.0), C, 7, ws, ws.numel(),
                              check=False) == -10
    assert mp.mp_dd_Rsyrk_crt("U", "N", 8, 4, (1.0, 0.0), A, 8, (0.0, 0.0), C, 8, None, 0,
                              check=False) == -12
    assert mp.mp_dd_Rsyrk_crt("U", "N", 8, 4, (1.0, 0.0), A, 8, (0.0, 0.0), C, 8, ws, 16,
                              check=False) == 2003


def test_crt_exact_runs_at_their_bound(cuda_lib):
    """Entries +-(1/2 + 2^-104) scale to X = +-(2^110 + 2^7), whose residue
    mod 256 is -128 whatever the sign: every product of the 256 plane is
    2^14, so each run of 1024 products sums to exactly 2^24, the largest
    partial sum an exact fp32 run may reach.  Product planes bit-exact
    against the oracle; the result within the bound."""
    mp = cuda_lib
    m, n, k = 16, 24, 2048
    g = datagen.rng(740)
    sa = np.where(g.random((m, k)) < 0.5, -1.0, 1.0)
    sb = np.where(g.random((k, n)) < 0.5, -1.0, 1.0)
    A = (np.asfortranarray(0.5 * sa), np.asfortranarray(2.0 ** -104 * sa))
    B = (np.asfortranarray(0.5 * sb), np.asfortranarray(2.0 ** -104 * sb))
    C = datagen.dd_matrix(g, m, n, m)
    c = datagen.GemmCase("N", "N", m, n, k, (1.0, 0.0), A, B, (1.0, 0.0), C)
    got, ws = run_crt(mp, c)
    rep = mp.mp_dd_split_report(ws)
    assert rep["width_bits"] == 112
    L = mp.mp_dd_crt_layout(m, n, k)
    mods = L["moduli"][:rep["count"]]
    assert mods[0] == 256
    RA, _ = oz.residue_planes(*oz.op_rows(c.A, False, m, k), mods, 14)
    RB, _ = oz.residue_planes(*oz.op_cols(c.B, False, k, n), mods, 14)
    assert (RA[0] == -128).all() and (RB[0] == -128).all()
    N, mp_, np_ = len(mods), L["m_pad"], L["n_pad"]
    prods = view(ws, L["products"], N * np_ * mp_, np.uint8).reshape(N, np_, mp_)
    want = oz.crt_products(RA, RB, mods)
    assert np.array_equal(prods[:, :n, :m].transpose(0, 2, 1).astype(np.int64), want)
    assert check_against_exact(c, got) <= 1.0


@pytest.mark.parametrize("alpha,beta", [((1.0, 0.0), (0.0, 0.0)), ((-1.0, 0.0), (0.0, 0.0)),
                                        ((1.0, 0.0), (1.0, 0.0)), ((-1.0, 0.0), (1.0, 0.0)),
                                        ((1.0, 0.0), None), (None, (0.0, 0.0))])
def test_crt_alpha_beta_forms(cuda_lib, alpha, beta):
    """alpha = +-1 with beta in {0, 1} (the specialised epilogues), alpha = 1
    with a general beta and a general alpha with beta = 0."""
    c = datagen.gemm_case(745, "N", "T", 150, 90, 200, pad=1)
    if alpha is not None:
        c.alpha = alpha
    if beta is not None:
        c.beta = beta
    got, _ = run_crt(cuda_lib, c)
    assert check_against_exact(c, got) <= 1.0


@pytest.mark.parametrize("c_exp", [60, -60, 600])
def test_crt_c_far_from_the_product(cuda_lib, c_exp):
    """|C| about 2^c_exp times |alpha A B|: the aligned sum of the epilogue
    over its whole exponent range."""
    c = datagen.gemm_case(746 + c_exp, "N", "N", 96, 80, 120)
    c.C = (c.C[0] * 2.0 ** c_exp, c.C[1] * 2.0 ** c_exp)
    got, _ = run_crt(cuda_lib, c)
    assert check_against_exact(c, got) <= 1.0


def test_crt_cancellation(cuda_lib):
    """C = -(alpha A B rounded to dd), beta = 1: the result is the tiny
    rounding residual, within the bound of the exact value."""
    m, n, k = 64, 48, 100
    c = datagen.gemm_case(747, "N", "N", m, n, k)
    c.beta = (1.0, 0.0)
    rows, cols = np.repeat(np.arange(m), n), np.tile(np.arange(n), m)
    oh, ol = oracle.exact_gemm_entries(c.transa, c.transb, c.k, c.alpha, c.A, c.B, (0.0, 0.0),
                                       None, rows, cols)
    c.C = (np.asfortranarray(-oh.reshape(m, n)), np.asfortranarray(-ol.reshape(m, n)))
    got, _ = run_crt(cuda_lib, c)
    assert check_against_exact(c, got) <= 1.0
    assert np.abs(got[0]).max() < 1e-25


def test_crt_non_finite_c_entries(cuda_lib):
    """Inf and NaN in C with beta != 0 give non-finite results at those
    entries (dd arithmetic turns an infinite C into NaN: the error term of
    beta c is inf - inf); the other entries meet the bound."""
    m, n, k = 40, 30, 64
    c = datagen.gemm_case(748, "N", "N", m, n, k)
    C0 = (c.C[0].copy(order="F"), c.C[1].copy(order="F"))
    C0[0][3, 4] = np.inf
    C0[0][5, 6] = -np.inf
    C0[0][7, 8] = np.nan
    c.C = C0
    got, _ = run_crt(cuda_lib, c)
    assert not np.isfinite(got[0][3, 4]) and not np.isfinite(got[0][5, 6])
    assert np.isnan(got[0][7, 8])
    keep = np.ones((m, n), bool)
    keep[3, 4] = keep[5, 6] = keep[7, 8] = False
    rows, cols = np.nonzero(keep)
    clean = datagen.gemm_case(748, "N", "N", m, n, k)
    assert check_against_exact(clean, got, rows, cols) <= 1.0
