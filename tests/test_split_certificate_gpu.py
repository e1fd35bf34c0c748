"""The per-call accuracy certificate of the split-precision calls (GPU).

Each mp_dd_Rgemm_sliced / mp_dd_Rgemm_crt / mp_dd_Rsyrk_crt call bounds, on
the device, the error its rounded operands can cause at every output entry
(a bf16 tensor-core product of the operands' magnitudes gives a lower bound
of |A||B|), picks the narrowest operand width that keeps the result within
4 k 2^-104 (|alpha||A||B| + |beta||C|), or computes C with the plain FP64
kernel.  Checked here through the C ABI:

* the reported margin is a safe lower bound of the exact margin
  (oracle/ozaki_ref.exact_margins) and within a few percent of it;
* the width follows the documented rule (ozaki_ref.certified_width) and is
  never narrower than the exact margin allows;
* on stress inputs (exponents spread along k; entries 2^40 below their row
  maximum) the result meets the bound against the exact tier, by a wider
  width or by the plain kernel, and the reported estimate is at most 1;
* the magnitude planes are bit-exact against the oracle's definition.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest
import torch

import datagen
from oracle import ozaki_ref as oz
from gpucase import check_against_exact, dev, host

pytestmark = pytest.mark.gpu

CRT_WIDTHS = [112, 120, 128]


def run_form(mp, form, c, slices=0):
    """Run GemmCase ``c`` through "crt" or "sliced"; (result, workspace, report)."""
    A, B, C = dev(c.A), dev(c.B), dev(c.C)
    lda, ldb, ldc = c.A[0].shape[0], c.B[0].shape[0], c.C[0].shape[0]
    if form == "crt":
        ws = mp.workspace(mp.mp_dd_Rgemm_crt_workspace(c.m, c.n, c.k))
        mp.mp_dd_Rgemm_crt(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, lda, B, ldb, c.beta,
                           C, ldc, ws, ws.numel())
    else:
        ws = mp.workspace(mp.mp_dd_Rgemm_sliced_workspace(c.m, c.n, c.k, slices))
        mp.mp_dd_Rgemm_sliced(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, lda, B, ldb,
                              c.beta, C, ldc, slices, ws, ws.numel())
    torch.cuda.synchronize()
    rep = mp.mp_dd_split_report(ws)
    assert rep["status"] == 0
    return host(C, c.m, c.n), ws, rep


def run_syrk_crt(mp, uplo, trans, n, k, alpha, A, beta, C):
    dA, dC = dev(A), dev(C)
    ws = mp.workspace(mp.mp_dd_Rsyrk_crt_workspace(n, k))
    mp.mp_dd_Rsyrk_crt(uplo, trans, n, k, alpha, dA, A[0].shape[0], beta, dC, C[0].shape[0],
                       ws, ws.numel())
    torch.cuda.synchronize()
    rep = mp.mp_dd_split_report(ws)
    assert rep["status"] == 0
    return host(dC), rep


def exact_dmin(c, tri=0):
    d = oz.exact_margins(oz.op_rows(c.A, c.transa == "T", c.m, c.k),
                         oz.op_cols(c.B, c.transb == "T", c.k, c.n), c.alpha, c.beta, c.C,
                         tri=tri)
    return min(d.values())


def adversarial_case(seed, m, n, k, tiny=2.0 ** -40):
    """Rows of A: 0.9 in column 0, dd entries of size `tiny` elsewhere; row 0
    of B zero, the rest U(-1, 1) dd."""
    g = datagen.rng(seed)
    ah = g.uniform(0.5, 1.0, (m, k)) * tiny
    ah[:, 0] = 0.9
    bh = g.uniform(-1, 1, (k, n))
    bh[0, :] = 0.0
    ah, al = datagen.dd_lo_for(ah, g)
    bh, bl = datagen.dd_lo_for(bh, g)
    A = (np.asfortranarray(ah), np.asfortranarray(al))
    B = (np.asfortranarray(bh), np.asfortranarray(bl))
    C = datagen.dd_matrix(g, m, n)
    return datagen.GemmCase("N", "N", m, n, k, (1.0, 0.0), A, B, (0.0, 0.0), C)


def beta_heavy_case(seed):
    """Ill-scaled (inner) operands with a large beta C: the beta term of the
    bound carries the margin."""
    c = datagen.gemm_case(seed, "N", "T", 24, 20, 256, ill="inner")
    c.C = (c.C[0] * 2.0 ** 40, c.C[1] * 2.0 ** 40)
    return c


CASES = {
    "well": lambda: datagen.gemm_case(800, "N", "N", 24, 20, 256),
    "outer": lambda: datagen.gemm_case(801, "T", "N", 24, 20, 256, ill="outer"),
    "inner": lambda: datagen.gemm_case(802, "N", "N", 24, 20, 256, ill="inner"),
    "adversarial": lambda: adversarial_case(803, 24, 20, 256),
    "beta": lambda: beta_heavy_case(804),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("form", ["crt", "sliced"])
def test_margin_is_a_safe_lower_bound(cuda_lib, name, form):
    c = CASES[name]()
    got, _, rep = run_form(cuda_lib, form, c)
    ex = exact_dmin(c)
    d = Fraction(rep["dmin"])
    assert d <= ex, "the certificate over-estimated the margin"
    assert d >= Fraction(97, 100) * ex
    # the width follows the rule on the reported margin, and is never
    # narrower than the exact margin allows
    widths = CRT_WIDTHS if form == "crt" else [112, 120]
    assert rep["width_bits"] == oz.certified_width(d, form, widths)
    w_exact = oz.certified_width(ex, form, widths)
    assert rep["width_bits"] == 0 or rep["width_bits"] >= w_exact
    assert rep["max_err_est"] <= 1.0
    assert check_against_exact(c, got) <= 1.0


def test_inner_scaling_takes_128_bits_in_residue_form(cuda_lib):
    """Exponents spread along k: 112 bits would miss the bound by far (see the
    oracle pin); the residue form certifies 128 bits and meets it, the digit
    form (at most 15 slices) hands the product to the plain kernel."""
    c = datagen.gemm_case(810, "N", "N", 160, 130, 512, ill="inner", pad=1)
    got, _, rep = run_form(cuda_lib, "crt", c)
    assert rep["width_bits"] == 128 and rep["count"] >= 36
    assert rep["max_err_est"] <= 1.0
    assert check_against_exact(c, got) <= 1.0
    got2, _, rep2 = run_form(cuda_lib, "sliced", c)
    assert rep2["width_bits"] == 0 and rep2["count"] == 0
    assert check_against_exact(c, got2) <= 1.0


@pytest.mark.parametrize("form", ["crt", "sliced"])
def test_adversarial_operands_fall_back_to_the_plain_kernel(cuda_lib, form):
    c = adversarial_case(820, 2, 2, 64)
    got, _, rep = run_form(cuda_lib, form, c)
    assert rep["width_bits"] == 0
    assert rep["max_err_est"] == pytest.approx(0.5 + 0.25 / 64)
    assert check_against_exact(c, got) <= 1.0


def test_explicit_slice_count_that_cannot_certify_falls_back(cuda_lib):
    c = datagen.gemm_case(830, "N", "N", 100, 90, 100)
    got, _, rep = run_form(cuda_lib, "sliced", c, slices=10)
    assert rep["width_bits"] == 0
    assert check_against_exact(c, got) <= 1.0
    got, _, rep = run_form(cuda_lib, "sliced", c, slices=14)
    assert rep["width_bits"] == 112 and rep["count"] == 14
    assert check_against_exact(c, got) <= 1.0


def _syrk_stress(seed, n, k, tiny):
    """A (n x k): row i holds 0.9 in column i mod k and dd entries of size
    `tiny` elsewhere, so off-diagonal entries of A A^T are ~tiny while the
    row maxima are ~1."""
    g = datagen.rng(seed)
    ah = g.uniform(0.5, 1.0, (n, k)) * tiny
    ah[np.arange(n), np.arange(n) % k] = 0.9
    ah, al = datagen.dd_lo_for(ah, g)
    return (np.asfortranarray(ah), np.asfortranarray(al))


@pytest.mark.parametrize("tiny,want", [(2.0 ** -20, 128), (2.0 ** -45, 0)])
def test_rsyrk_crt_certificate_on_its_triangle(cuda_lib, tiny, want):
    n, k = 96, 80
    A = _syrk_stress(840, n, k, tiny)
    g = datagen.rng(841)
    C = datagen.dd_matrix(g, n, n)
    got, rep = run_syrk_crt(cuda_lib, "U", "N", n, k, (1.0, 0.0), A, (0.0, 0.0), C)
    assert rep["width_bits"] == want
    c = datagen.GemmCase("N", "T", n, n, k, (1.0, 0.0), A, A, (0.0, 0.0), C)
    d = Fraction(rep["dmin"])
    assert d <= exact_dmin(c, tri=1)
    rows, cols = np.triu_indices(n)
    assert check_against_exact(c, got, rows, cols) <= 1.0
    # the lower triangle is untouched
    low = np.tril_indices(n, -1)
    assert np.array_equal(got[0][low], C[0][low])


@pytest.mark.parametrize("form,sym", [(1, False), (2, False), (3, True)])
def test_magnitude_planes_bit_exact(cuda_lib, form, sym):
    mp = cuda_lib
    m, n, k = 70, 50, 150
    if sym:
        n = m
        g = datagen.rng(850)
        A = datagen.dd_matrix(g, m, k, m + 1)
        C = datagen.dd_matrix(g, m, m)
        dA, dC = dev(A), dev(C)
        ws = mp.workspace(mp.mp_dd_Rsyrk_crt_workspace(m, k))
        mp.mp_dd_Rsyrk_crt("U", "N", m, k, (1.0, 0.0), dA, m + 1, (0.0, 0.0), dC, m, ws,
                           ws.numel())
        rows_a = oz.op_rows(A, False, m, k)
        rows_b = rows_a
        L = mp.mp_dd_crt_layout(m, m, k)
    else:
        c = datagen.gemm_case(851 + form, "T", "N", m, n, k, pad=2, ill="outer")
        if form == 1:
            _, ws, _ = run_form(mp, "sliced", c)
            L = mp.mp_dd_sliced_layout(m, n, k, 0)
        else:
            _, ws, _ = run_form(mp, "crt", c)
            L = mp.mp_dd_crt_layout(m, n, k)
        rows_a = oz.op_rows(c.A, True, m, k)
        rows_b = oz.op_cols(c.B, False, k, n)
    torch.cuda.synchronize()
    off = mp.mp_dd_magnitude_layout(form, m, n, k, 0)
    kp = L["k_pad"]
    mpad = L["m_pad"]
    npad = L["n_pad"] if not sym else L["m_pad"]
    raw = ws.cpu().numpy()

    def plane(offset, rows):
        u16 = raw[offset: offset + rows * kp * 2].view(np.uint16).astype(np.uint32) << 16
        return u16.view(np.float32).reshape(rows, kp)

    for key, (rh, _), pad in (("magnitude_a", rows_a, mpad), ("magnitude_b", rows_b, npad)):
        P = plane(off[key], pad)
        R = rh.shape[0]
        for r in range(R):
            want = oz.magnitude_row(rh[r], oz.scale_exponent(rh[r]))
            assert [Fraction(float(v)) for v in P[r, :k]] == want
        assert not P[R:, :].any() and not P[:, k:].any()
    if sym:
        assert off["magnitude_a"] == off["magnitude_b"]


def test_alpha_zero_reports_no_product(cuda_lib):
    c = datagen.gemm_case(860, "N", "N", 30, 20, 40, alpha=(0.0, 0.0))
    _, _, rep = run_form(cuda_lib, "crt", c)
    assert rep["form"] == 0 and rep["width_bits"] == 0
