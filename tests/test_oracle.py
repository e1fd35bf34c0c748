"""Pins for the oracle (CPU only).

The oracle is checked against things other than itself: exact rational
arithmetic (``fractions``), values the manual prints for its worked examples
(``tests/golden/``), closed forms, special cases that reduce to binary64
library routines, and LAPACK-style test ratios.  ``test_planted_mistakes``
re-runs this file against deliberately broken copies of the oracle and
requires every copy to fail.
"""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import datagen
import oracle
from oracle import fraction_ref as fr
from ddcheck import EPS_DD, U, err_over_bound, gemm_bound, is_normalised
from trsmcheck import TRSM_VARIANTS, op_triangle, trsm_residual_over_bound
import blas3check as b3
from lucheck import dyadic_lu_case, lu_residual_ratio

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")
U2 = U * U


# ---------------------------------------------------------------------------
# golden fixtures
# ---------------------------------------------------------------------------

def read_golden(name):
    """Parse a fixture: 'key value...' lines and named blocks of matrix rows."""
    out, block = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if len(parts) == 1 and parts[0].isupper() or parts[0].startswith("ANSWER"):
                block = parts[0]
                out[block] = []
            elif block is None or parts[0] in ("alpha", "beta", "epsilon", "precision",
                                               "digits"):
                out[parts[0]] = parts[1:]
            else:
                out[block].append(line)
    return out


def rows_real(lines):
    return [[Fraction(x) for x in l.split()] for l in lines]


def rows_complex(lines):
    res = []
    for l in lines:
        row = []
        for cell in l.split("|"):
            re, im = cell.split()
            row.append((re, im))
        res.append(row)
    return res


def dd_plane_from_fracs(F, conv):
    """Column-major (hi, lo) planes from a list of rows of Fractions."""
    m, n = len(F), len(F[0])
    hi, lo = np.zeros((m, n), order="F"), np.zeros((m, n), order="F")
    for i in range(m):
        for j in range(n):
            hi[i, j], lo[i, j] = conv(F[i][j])
    return hi, lo


# ---------------------------------------------------------------------------
# scalar dd layer
# ---------------------------------------------------------------------------

def random_dd(g, n, emin=-40, emax=40):
    hi = g.uniform(-1, 1, n) * np.ldexp(1.0, g.integers(emin, emax, n))
    return datagen.dd_lo_for(hi, g)


def adversarial_pairs(g, n):
    a = random_dd(g, n)
    b = random_dd(g, n)
    # a third of the pairs nearly cancel: b = -a + small perturbation
    k = n // 3
    bh = -a[0][:k] * (1 + g.uniform(-1, 1, k) * 2.0 ** -40)
    bl = -a[1][:k] * g.uniform(0, 2, k)
    bh, bl = datagen._renormalise(bh, bl)
    b = (np.concatenate([bh, b[0][k:]]), np.concatenate([bl, b[1][k:]]))
    return a, b


def F(h, l=0.0):
    return Fraction(float(h)) + Fraction(float(l))


def test_two_sum_and_two_prod_are_exact():
    g = datagen.rng(1)
    a = g.uniform(-1, 1, 2000) * np.ldexp(1.0, g.integers(-60, 60, 2000))
    b = g.uniform(-1, 1, 2000) * np.ldexp(1.0, g.integers(-60, 60, 2000))
    s, e = oracle.two_sum(a, b)
    p, q = oracle.two_prod(a, b)
    assert np.array_equal(s, a + b)
    assert np.array_equal(p, a * b)
    for i in range(a.size):
        assert F(s[i]) + F(e[i]) == F(a[i]) + F(b[i])
        assert F(p[i]) + F(q[i]) == F(a[i]) * F(b[i])


def rel_errs(got_h, got_l, exact):
    out = []
    for h, l, x in zip(got_h, got_l, exact):
        if x == 0:
            out.append(0.0 if h == 0 and l == 0 else float("inf"))
        else:
            out.append(float(abs(F(h, l) - x) / abs(x)))
    return np.array(out)


def test_dd_add_relative_error():
    g = datagen.rng(2)
    a, b = adversarial_pairs(g, 1500)
    rh, rl = oracle.dd_add(a, b)
    exact = [F(a[0][i], a[1][i]) + F(b[0][i], b[1][i]) for i in range(rh.size)]
    # accurate dd addition: relative error <= 3u^2 + 13u^3
    assert rel_errs(rh, rl, exact).max() <= 3.0001 * U2
    assert is_normalised(rh, rl)


def test_dd_mul_div_sqrt_relative_error():
    g = datagen.rng(3)
    a, b = random_dd(g, 1500), random_dd(g, 1500)
    mh, ml = oracle.dd_mul(a, b)
    ex = [F(a[0][i], a[1][i]) * F(b[0][i], b[1][i]) for i in range(mh.size)]
    assert rel_errs(mh, ml, ex).max() <= 6 * U2
    dh, dl = oracle.dd_div(a, b)
    ex = [F(a[0][i], a[1][i]) / F(b[0][i], b[1][i]) for i in range(dh.size)]
    assert rel_errs(dh, dl, ex).max() <= 8 * U2
    pos = (np.abs(a[0]), np.where(a[0] < 0, -a[1], a[1]))
    sh, sl = oracle.dd_sqrt(pos)
    for i in range(sh.size):
        x = F(pos[0][i], pos[1][i])
        r = F(sh[i], sl[i])
        # |r - sqrt(x)| = |r^2 - x| / (r + sqrt(x)) ~ |r^2 - x| / (2r)
        assert abs(r * r - x) / (2 * r) <= 8 * U2 * r
    assert is_normalised(mh, ml) and is_normalised(dh, dl) and is_normalised(sh, sl)


# ---------------------------------------------------------------------------
# exact tier
# ---------------------------------------------------------------------------

def test_exact_sum_known_values():
    assert oracle.exact_sum([1.0, 2.0 ** -100, -1.0]) == (2.0 ** -100, 0.0)
    assert oracle.exact_sum([1e308, 1e308, -1e308]) == (1e308, 0.0)
    assert oracle.exact_sum([1.0, 2.0 ** -60]) == (1.0, 2.0 ** -60)
    assert oracle.exact_sum([-3.0, 2.0 ** -200, 2.0 ** -201]) == (-3.0, 3 * 2.0 ** -201)
    # 1 + 2^-53 is a rounding tie for hi; the 2^-160 below it breaks the tie
    # upward (sticky bit), so hi = 1 + 2^-52 and lo = RN(-2^-53 + 2^-160) = -2^-53
    assert oracle.exact_sum([1.0, 2.0 ** -53, 2.0 ** -160]) == (1.0 + 2.0 ** -52, -2.0 ** -53)
    assert oracle.exact_sum([1.0, 2.0 ** -53]) == (1.0, 2.0 ** -53)
    g = datagen.rng(4)
    for _ in range(50):
        v = g.uniform(-1, 1, 40) * np.ldexp(1.0, g.integers(-300, 300, 40))
        assert oracle.exact_sum(v) == fr.round_dd(sum(F(t) for t in v))


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_exact_tier_equals_fraction_rounding(ta, tb):
    for seed, (m, n, k) in enumerate([(3, 4, 5), (5, 2, 7), (1, 1, 1), (4, 4, 0), (2, 6, 3)]):
        c = datagen.gemm_case(10 + seed, ta, tb, m, n, k, pad=1)
        if seed == 3:
            c.beta = (0.0, 0.0)
        rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
        got = oracle.exact_gemm_entries(ta, tb, k, c.alpha, c.A, c.B, c.beta, c.C, rr.ravel(),
                                        cc.ravel())
        want = fr.gemm_exact_dd(ta, tb, m, n, k, c.alpha, c.A, c.B, c.beta, c.C)
        assert np.array_equal(got[0].reshape(m, n), want[0])
        assert np.array_equal(got[1].reshape(m, n), want[1])


# ---------------------------------------------------------------------------
# scalar dd Rgemm
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("t", "c")])
def test_scalar_gemm_within_bound(ta, tb):
    m, n, k = 7, 5, 33
    c = datagen.gemm_case(20, ta, tb, m, n, k, pad=2)
    got = oracle.dd_gemm(ta, tb, c.alpha, c.A, c.B, c.beta, c.C, m, n, k)
    got = (got[0][:m, :n], got[1][:m, :n])
    want = fr.gemm_exact_dd(ta, tb, m, n, k, c.alpha, c.A, c.B, c.beta, c.C)
    bound = gemm_bound(ta, tb, m, n, k, c.alpha, c.A, c.B, c.beta, c.C)
    assert err_over_bound(got, want, bound) <= 1.0
    assert is_normalised(*got)


def test_rgemm_worked_example_exact():
    gd = read_golden("rgemm_worked_example.txt")
    A = rows_real(gd["A"])
    B = rows_real(gd["B"])
    C = rows_real(gd["C"])
    to = lambda x: (float(x), 0.0)
    Ad, Bd, Cd = (dd_plane_from_fracs(M, to) for M in (A, B, C))
    al = (float(gd["alpha"][0]), 0.0)
    be = (float(gd["beta"][0]), 0.0)
    got = oracle.dd_gemm("N", "N", al, Ad, Bd, be, Cd)
    ans = np.array([[float(x) for x in r] for r in rows_real(gd["ANSWER"])])
    assert np.array_equal(got[0], ans) and not got[1].any()


def complex_gemm_via_real(gemm, alpha, A, B, beta, C):
    """alpha*A*B + beta*C for complex dd data through six real Rgemm calls.

    ``gemm(alpha, A, B, beta, C)`` is a real 'N','N' dd Rgemm on (hi, lo)
    planes returning the new C.  Re/Im parts: A = (Ar, Ai) etc."""
    (Ar, Ai), (Br, Bi), (Cr, Ci) = A, B, C
    neg = lambda X: (-X[0], -X[1])
    hcat = lambda X, Y: (np.hstack([X[0], Y[0]]), np.hstack([X[1], Y[1]]))
    vcat = lambda X, Y: (np.vstack([X[0], Y[0]]), np.vstack([X[1], Y[1]]))
    n = Cr[0].shape[1]
    eye = (np.eye(n), np.zeros((n, n)))
    (ar, ai), (br, bi) = alpha, beta
    one = (1.0, 0.0)
    A1, B1 = hcat(Ar, neg(Ai)), vcat(Br, Bi)   # A1 @ B1 = Re(AB)
    A2, B2 = hcat(Ar, Ai), vcat(Bi, Br)        # A2 @ B2 = Im(AB)
    re = gemm(ar, A1, B1, br, Cr)
    re = gemm((-ai[0], -ai[1]), A2, B2, one, re)
    re = gemm((-bi[0], -bi[1]), Ci, eye, one, re)
    im = gemm(ar, A2, B2, br, Ci)
    im = gemm(ai, A1, B1, one, im)
    im = gemm(bi, Cr, eye, one, im)
    return re, im


def cgemm_case(variant):
    gd = read_golden("cgemm_worked_example.txt")
    if variant == "binary64":
        conv = lambda s: (float(s), 0.0)
        ans_lines = gd["ANSWER_BINARY64"]
    else:
        conv = lambda s: fr.round_dd(Fraction(s))
        ans_lines = gd["ANSWER_DECIMAL"]

    def planes(lines):
        cells = rows_complex(lines)
        re = [[Fraction(c[0]) if variant == "decimal" else Fraction(float(c[0])) for c in r]
              for r in cells]
        im = [[Fraction(c[1]) if variant == "decimal" else Fraction(float(c[1])) for c in r]
              for r in cells]
        tod = (lambda x: fr.round_dd(x))
        return dd_plane_from_fracs(re, tod), dd_plane_from_fracs(im, tod)

    A, B, C = planes(gd["A"]), planes(gd["B"]), planes(gd["C"])
    alpha = tuple(conv(s) for s in gd["alpha"])
    beta = tuple(conv(s) for s in gd["beta"])
    ans = rows_complex(ans_lines)
    return alpha, A, B, beta, C, ans


def check_cgemm_result(re, im, alpha, A, B, beta, C, ans):
    """Compare with the printed 64-digit answer; tolerance derived from the
    accuracy bound of the six real calls (k <= 6 each, three per part)."""
    mag = lambda X: np.abs(X[0])
    a = abs(alpha[0][0]) + abs(alpha[1][0])
    b = abs(beta[0][0]) + abs(beta[1][0])
    M = a * (mag(A[0]) + mag(A[1])) @ (mag(B[0]) + mag(B[1])) + b * (mag(C[0]) + mag(C[1]))
    tol = 3 * 4 * 6 * EPS_DD * M * 1.01 + 8 * U2 * M
    for i in range(3):
        for j in range(3):
            er = abs(F(re[0][i, j], re[1][i, j]) - Fraction(ans[i][j][0]))
            ei = abs(F(im[0][i, j], im[1][i, j]) - Fraction(ans[i][j][1]))
            assert er <= Fraction(tol[i, j]) and ei <= Fraction(tol[i, j]), (i, j, float(er),
                                                                              float(ei))


@pytest.mark.parametrize("variant", ["binary64", "decimal"])
def test_cgemm_worked_example_through_real_rgemm(variant):
    alpha, A, B, beta, C, ans = cgemm_case(variant)

    def gemm(al, X, Y, be, Z):
        return oracle.dd_gemm("N", "N", al, X, Y, be, Z)

    re, im = complex_gemm_via_real(gemm, alpha, A, B, beta, C)
    check_cgemm_result(re, im, alpha, A, B, beta, C, ans)


def test_rlamch_dd_epsilon_is_the_bound_constant():
    gd = read_golden("rlamch_dd.txt")
    eps = Fraction(gd["epsilon"][0])
    # the printed epsilon is a 15-significant-digit decimal of 2^-104 carried
    # as a binary64 constant, so it agrees with 2^-104 to ~1e-15 relative
    assert abs(eps - Fraction(EPS_DD)) / Fraction(EPS_DD) < Fraction(1, 10 ** 14)
    assert int(float(gd["digits"][0])) == 106          # 2 x 53 significand bits
    assert Fraction(gd["precision"][0]) == 2 * eps     # eps * base


def test_closed_forms():
    g = datagen.rng(5)
    m, n = 6, 4
    # k = 1: C = alpha*a*b + beta*c, one product per entry
    c = datagen.gemm_case(30, "N", "N", m, n, 1)
    got = oracle.dd_gemm("N", "N", c.alpha, c.A, c.B, c.beta, c.C)
    for i in range(m):
        for j in range(n):
            x = (F(*c.alpha) * F(c.A[0][i, 0], c.A[1][i, 0]) * F(c.B[0][0, j], c.B[1][0, j])
                 + F(*c.beta) * F(c.C[0][i, j], c.C[1][i, j]))
            assert abs(F(got[0][i, j], got[1][i, j]) - x) <= 16 * U2 * (
                abs(F(*c.alpha) * F(c.A[0][i, 0]) * F(c.B[0][0, j]))
                + abs(F(*c.beta) * F(c.C[0][i, j])))
    # A = I: C = alpha*B + beta*C
    c = datagen.gemm_case(31, "N", "N", m, n, m)
    I = (np.eye(m), np.zeros((m, m)))
    got = oracle.dd_gemm("N", "N", c.alpha, I, c.B[:1] + c.B[1:], c.beta, c.C)
    B = (c.B[0][:m, :n], c.B[1][:m, :n])
    want = oracle.dd_add(oracle.dd_mul((np.full(m * n, c.alpha[0]), np.full(m * n, c.alpha[1])),
                                       (B[0].ravel("F"), B[1].ravel("F"))),
                         oracle.dd_mul((np.full(m * n, c.beta[0]), np.full(m * n, c.beta[1])),
                                       (c.C[0].ravel("F"), c.C[1].ravel("F"))))
    assert np.array_equal(got[0].ravel("F"), want[0]) and np.array_equal(got[1].ravel("F"),
                                                                         want[1])
    # alpha = 0: C = beta*C exactly as one dd product per entry, A and B unread
    nanA = (np.full((m, 3), np.nan), np.full((m, 3), np.nan))
    nanB = (np.full((3, n), np.nan), np.full((3, n), np.nan))
    got = oracle.dd_gemm("N", "N", (0.0, 0.0), nanA, nanB, c.beta, c.C)
    want = oracle.dd_mul((np.full(m * n, c.beta[0]), np.full(m * n, c.beta[1])),
                         (c.C[0].ravel("F"), c.C[1].ravel("F")))
    assert np.array_equal(got[0].ravel("F"), want[0])


def test_integer_inputs_match_binary64_matmul():
    g = datagen.rng(6)
    for ta, tb in [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")]:
        m, n, k = 9, 7, 11
        A = g.integers(-50, 50, (k, m) if ta == "T" else (m, k)).astype(np.float64)
        B = g.integers(-50, 50, (n, k) if tb == "T" else (k, n)).astype(np.float64)
        C = g.integers(-50, 50, (m, n)).astype(np.float64)
        z = np.zeros_like
        got = oracle.dd_gemm(ta, tb, (3.0, 0.0), (A, z(A)), (B, z(B)), (-2.0, 0.0), (C, z(C)))
        opA = A.T if ta == "T" else A
        opB = B.T if tb == "T" else B
        assert np.array_equal(got[0], 3.0 * (opA @ opB) - 2.0 * C) and not got[1].any()


def test_quick_returns_and_beta_zero_does_not_read_c():
    c = datagen.gemm_case(40, "N", "N", 4, 3, 5)
    Cn = (np.full((4, 3), np.nan), np.full((4, 3), np.nan))
    got = oracle.dd_gemm("N", "N", c.alpha, c.A, c.B, (0.0, 0.0), Cn)
    assert np.isfinite(got[0]).all() and np.isfinite(got[1]).all()
    # (alpha == 0 or k == 0) and beta == 1: no-op, even on NaN
    same = oracle.dd_gemm("N", "N", (0.0, 0.0), c.A, c.B, (1.0, 0.0), Cn)
    assert np.isnan(same[0]).all()
    same = oracle.dd_gemm("N", "N", c.alpha, c.A, c.B, (1.0, 0.0), Cn, 4, 3, 0)
    assert np.isnan(same[0]).all()


# ---------------------------------------------------------------------------
# scalar dd Rsyrk
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("uplo,trans", [("U", "N"), ("L", "N"), ("U", "T"), ("l", "t")])
def test_syrk_matches_gemm_triangle_and_exact(uplo, trans):
    n, k = 6, 9
    g = datagen.rng(50)
    A = datagen.dd_matrix(g, k if trans.upper() == "T" else n, n if trans.upper() == "T" else k)
    C = datagen.dd_matrix(g, n, n)
    al, be = datagen.dd_scalar(g), datagen.dd_scalar(g)
    got = oracle.dd_syrk(uplo, trans, al, A, be, C)
    t = trans.upper() == "T"
    ref = oracle.dd_gemm("T" if t else "N", "N" if t else "T", al, A, A, be, C)
    tri = np.triu(np.ones((n, n), bool)) if uplo.upper() == "U" else np.tril(
        np.ones((n, n), bool))
    assert np.array_equal(got[0][tri], ref[0][tri]) and np.array_equal(got[1][tri], ref[1][tri])
    assert np.array_equal(got[0][~tri], C[0][~tri])
    ex = fr.syrk_exact(uplo, trans, n, k, al, A, be, C)
    bound = gemm_bound("T" if t else "N", "N" if t else "T", n, n, k, al, A, A, be, C)
    for i in range(n):
        for j in range(n):
            if tri[i, j]:
                d = abs(F(got[0][i, j], got[1][i, j]) - ex[i][j])
                assert d <= Fraction(bound[i, j])


# ---------------------------------------------------------------------------
# Rpotrf / Rpotrs
# ---------------------------------------------------------------------------

def test_potrf_recovers_exact_integer_factor():
    g = datagen.rng(60)
    n = 12
    Ui = np.triu(g.integers(-4, 5, (n, n))).astype(np.float64)
    np.fill_diagonal(Ui, g.integers(1, 6, n))
    Fm = Ui.T @ Ui                      # exact in binary64 (small integers)
    fh, fl, info = oracle.dd_potrf("U", (Fm, np.zeros_like(Fm)))
    assert info == 0
    assert np.array_equal(np.triu(fh), Ui) and not np.triu(fl).any()
    lh, ll, info = oracle.dd_potrf("L", (Fm, np.zeros_like(Fm)))
    assert info == 0 and np.array_equal(np.tril(lh), Ui.T)


def test_potrf_reports_first_non_positive_minor():
    Fm = np.diag([4.0, 9.0, -1.0, 16.0])
    assert oracle.dd_potrf("U", (Fm, np.zeros_like(Fm)))[2] == 3
    Fm = np.array([[1.0, 2.0], [2.0, 4.0]])   # singular: second minor is 0
    assert oracle.dd_potrf("U", (Fm, np.zeros_like(Fm)))[2] == 2


def exact_residual_norm_ratio_potrf(Fd, Ud, n):
    """||U^T U - F||_1 / (n ||F||_1 eps) with U^T U - F evaluated exactly."""
    Ut = (np.triu(Ud[0]), np.triu(Ud[1]))
    rr, cc = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    R = oracle.exact_gemm_entries("T", "N", n, (1.0, 0.0), Ut, Ut, (-1.0, 0.0), Fd, rr.ravel(),
                                  cc.ravel())
    Rm = np.abs(R[0].reshape(n, n))
    Fn = np.abs(Fd[0]).sum(axis=0).max()
    return Rm.sum(axis=0).max() / (n * Fn * EPS_DD)


def test_potrf_potrs_lapack_ratios_on_ill_conditioned_spd():
    n = 24
    G, B = datagen.spd_request(61, n)
    Fd = oracle.dd_syrk("U", "N", (1.0, 0.0), G, (0.0, 0.0),
                        (np.zeros((n, n), order="F"), np.zeros((n, n), order="F")))
    # symmetrise (lower from upper) for the residual evaluation
    Fs = tuple(np.triu(P) + np.triu(P, 1).T for P in Fd)
    fh, fl, info = oracle.dd_potrf("U", Fd)
    assert info == 0
    assert exact_residual_norm_ratio_potrf(Fs, (fh, fl), n) < 30  # LAPACK threshold
    X = oracle.dd_potrs("U", (fh, fl), B)
    rr, cc = np.meshgrid(np.arange(n), np.arange(B[0].shape[1]), indexing="ij")
    R = oracle.exact_gemm_entries("N", "N", n, (-1.0, 0.0), Fs, X, (1.0, 0.0), B, rr.ravel(),
                                  cc.ravel())
    Fn = np.abs(Fs[0]).sum(axis=0).max()
    Xn = np.abs(X[0]).sum(axis=0).max()
    ratio = np.abs(R[0]).reshape(rr.shape).sum(axis=0).max() / (Fn * Xn * EPS_DD)
    assert ratio < 30
    # binary64 Cholesky cannot factor the same matrix reliably (cond ~ 1e20)
    try:
        L = np.linalg.cholesky(Fs[0])
        rel = np.abs(L @ L.T - Fs[0]).max() / np.abs(Fs[0]).max()
        x64 = np.linalg.solve(L.T, np.linalg.solve(L, B[0]))
        xdd = X[0]
        assert np.abs(x64 - xdd).max() / np.abs(xdd).max() > 1e-6 or rel > 0
    except np.linalg.LinAlgError:
        pass


def test_potrf_matches_numpy_on_well_conditioned_spd():
    g = datagen.rng(62)
    n = 20
    M = g.uniform(-1, 1, (n, n))
    Fm = M @ M.T + n * np.eye(n)
    fh, fl, info = oracle.dd_potrf("L", (Fm, np.zeros_like(Fm)))
    assert info == 0
    L = np.linalg.cholesky(Fm)
    assert np.abs(np.tril(fh) - L).max() <= 1e-13 * np.abs(L).max()


# ---------------------------------------------------------------------------
# quad-double exact tier
# ---------------------------------------------------------------------------

def round_qd_fraction(v):
    """Four components by repeated correct rounding of the rational v (Python's
    float(Fraction) rounds to nearest, ties to even)."""
    out = []
    for _ in range(4):
        x = float(v)
        out.append(x)
        v -= Fraction(x)
    return out


def qd_frac(c, idx):
    return sum((Fraction(float(P[idx])) for P in c), Fraction(0))


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
def test_exact_qd_tier_equals_fraction_rounding(ta, tb):
    g = datagen.rng(140)
    m, n, k = 3, 4, 5
    A = datagen.qd_matrix(g, k if ta == "T" else m, m if ta == "T" else k)
    B = datagen.qd_matrix(g, n if tb == "T" else k, k if tb == "T" else n)
    C = datagen.qd_matrix(g, m, n)
    al, be = datagen.qd_scalar(g), datagen.qd_scalar(g)
    rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    got = oracle.exact_qd_gemm_entries(ta, tb, k, al, A, B, be, C, rr.ravel(), cc.ravel())
    fa, fb = sum(map(Fraction, al)), sum(map(Fraction, be))
    for q, (i, j) in enumerate(zip(rr.ravel(), cc.ravel())):
        v = fb * qd_frac(C, (i, j))
        for l in range(k):
            a = qd_frac(A, (l, i) if ta == "T" else (i, l))
            b = qd_frac(B, (j, l) if tb == "T" else (l, j))
            v += fa * a * b
        assert [got[t][q] for t in range(4)] == round_qd_fraction(v)


def test_exact_qd_tier_matches_dd_tier_on_dd_inputs():
    """With zero third and fourth components, the first two components of
    the qd rounding are the dd rounding of the same exact value."""
    g = datagen.rng(141)
    m, n, k = 6, 5, 33
    A = datagen.dd_matrix(g, m, k)
    B = datagen.dd_matrix(g, k, n)
    C = datagen.dd_matrix(g, m, n)
    al, be = datagen.dd_scalar(g), datagen.dd_scalar(g)
    z = lambda P: np.zeros_like(P)
    A4, B4, C4 = ((P[0], P[1], z(P[0]), z(P[0])) for P in (A, B, C))
    rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    q = oracle.exact_qd_gemm_entries("N", "N", k, (*al, 0.0, 0.0), A4, B4, (*be, 0.0, 0.0),
                                     C4, rr.ravel(), cc.ravel())
    d = oracle.exact_gemm_entries("N", "N", k, al, A, B, be, C, rr.ravel(), cc.ravel())
    assert np.array_equal(q[0], d[0]) and np.array_equal(q[1], d[1])


def test_exact_qd_tier_integer_inputs():
    g = datagen.rng(142)
    A = g.integers(-50, 51, (7, 9)).astype(np.float64)
    B = g.integers(-50, 51, (9, 6)).astype(np.float64)
    z = lambda P: np.zeros_like(P)
    rr, cc = np.meshgrid(np.arange(7), np.arange(6), indexing="ij")
    q = oracle.exact_qd_gemm_entries("N", "N", 9, (2.0, 0, 0, 0),
                                     (np.asfortranarray(A), z(A), z(A), z(A)),
                                     (np.asfortranarray(B), z(B), z(B), z(B)), (0, 0, 0, 0),
                                     None, rr.ravel(), cc.ravel())
    assert np.array_equal(q[0].reshape(7, 6), 2 * A @ B)
    assert not q[1].any() and not q[2].any() and not q[3].any()


# ---------------------------------------------------------------------------
# Rsyr2k / Rsymm
# ---------------------------------------------------------------------------

def syr2k_case(seed, trans, n, k, pad=2):
    g = datagen.rng(seed)
    ar, ac = (n, k) if trans == "N" else (k, n)
    A = datagen.dd_matrix(g, ar, ac, ar + pad)
    B = datagen.dd_matrix(g, ar, ac, ar + pad)
    C = datagen.dd_matrix(g, n, n, n + pad)
    return A, B, C, datagen.dd_scalar(g), datagen.dd_scalar(g)


@pytest.mark.parametrize("uplo", ["U", "L"])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_syr2k_within_bound_of_exact_concatenated_gemm(uplo, trans):
    n, k = 11, 9
    A, B, C, al, be = syr2k_case(90, trans, n, k)
    got = oracle.dd_syr2k(uplo, trans, al, A, B, be, C, n, k)
    rows, cols = b3.triangle_entries(n, uplo)
    ex, bound = b3.exact_and_bound(b3.syr2k_as_gemm(trans, n, k, A, B), n, n, al, be, C,
                                   rows, cols)
    g = (got[0][rows, cols], got[1][rows, cols])
    assert err_over_bound(g, ex, bound) <= 1.0
    # the other triangle and the padding are untouched
    other = np.ones((n + 2, n), bool)
    other[rows, cols] = False
    assert np.array_equal(got[0][other], C[0][other], equal_nan=True)


def test_syr2k_integer_inputs_match_binary64():
    g = datagen.rng(91)
    n, k = 10, 6
    A = g.integers(-9, 10, (k, n)).astype(np.float64)
    B = g.integers(-9, 10, (k, n)).astype(np.float64)
    C = g.integers(-9, 10, (n, n)).astype(np.float64)
    z = np.zeros((k, n))
    got = oracle.dd_syr2k("L", "T", (3.0, 0.0), (A, z), (B, z), (-2.0, 0.0), (C, np.zeros((n, n))))
    ref = 3.0 * (A.T @ B + B.T @ A) - 2.0 * C
    rows, cols = b3.triangle_entries(n, "L")
    assert np.array_equal(got[0][rows, cols], ref[rows, cols]) and not got[1].any()


def test_syr2k_fraction_brute_force():
    n, k = 4, 3
    A, B, C, al, be = syr2k_case(92, "N", n, k, pad=0)
    got = oracle.dd_syr2k("U", "N", al, A, B, be, C)
    for j in range(n):
        for i in range(j + 1):
            v = F(*al) * sum(F(A[0][i, l], A[1][i, l]) * F(B[0][j, l], B[1][j, l]) +
                             F(B[0][i, l], B[1][i, l]) * F(A[0][j, l], A[1][j, l])
                             for l in range(k)) + F(*be) * F(C[0][i, j], C[1][i, j])
            assert abs(F(got[0][i, j], got[1][i, j]) - v) <= Fraction(2) ** -100 * abs(v)


@pytest.mark.parametrize("side", ["L", "R"])
@pytest.mark.parametrize("uplo", ["U", "L"])
def test_symm_within_bound_of_exact_symmetrised_gemm(side, uplo):
    m, n = 9, 7
    g = datagen.rng(93)
    order = m if side == "L" else n
    A = datagen.dd_matrix(g, order, order, order + 2)
    r, c = np.meshgrid(np.arange(order), np.arange(order), indexing="ij")
    unused = (r > c) if uplo == "U" else (r < c)
    for P in A:
        P[:order][unused] = np.nan                 # must never be read
    B = datagen.dd_matrix(g, m, n, m + 1)
    C = datagen.dd_matrix(g, m, n, m + 3)
    al, be = datagen.dd_scalar(g), datagen.dd_scalar(g)
    got = oracle.dd_symm(side, uplo, al, A, B, be, C, m, n)
    rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    rows, cols = rr.ravel(), cc.ravel()
    ex, bound = b3.exact_and_bound(b3.symm_as_gemm(side, uplo, m, n, A, B), m, n, al, be, C,
                                   rows, cols)
    assert err_over_bound((got[0][rows, cols], got[1][rows, cols]), ex, bound) <= 1.0


def test_symm_integer_inputs_match_binary64():
    g = datagen.rng(94)
    m, n = 8, 11
    S = g.integers(-9, 10, (n, n)).astype(np.float64)
    S = np.triu(S) + np.triu(S, 1).T
    B = g.integers(-9, 10, (m, n)).astype(np.float64)
    C = g.integers(-9, 10, (m, n)).astype(np.float64)
    stored = np.where(np.tril(np.ones((n, n))) > 0, S, np.nan)
    got = oracle.dd_symm("R", "L", (2.0, 0.0), (stored, np.zeros((n, n))), (B, np.zeros((m, n))),
                         (1.0, 0.0), (C, np.zeros((m, n))))
    assert np.array_equal(got[0], 2.0 * B @ S + C) and not got[1].any()


# ---------------------------------------------------------------------------
# Rgetrf / Rgetrs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m,n", [(12, 12), (15, 9), (8, 13)])
def test_getrf_recovers_dyadic_factorisation(m, n):
    A, L, U, ipiv = dyadic_lu_case(100 + m, m, n)
    lh, ll, piv, info = oracle.dd_getrf((A, np.zeros_like(A)))
    assert info == 0 and np.array_equal(piv, ipiv) and not ll.any()
    mn = min(m, n)
    assert np.array_equal(np.tril(lh[:, :mn], -1), np.tril(L, -1))
    assert np.array_equal(np.triu(lh[:mn, :]), U)


@pytest.mark.parametrize("m,n", [(40, 40), (47, 31), (29, 44)])
def test_getrf_lapack_ratio(m, n):
    g = datagen.rng(110 + m)
    A = datagen.dd_matrix(g, m, n)
    lh, ll, piv, info = oracle.dd_getrf(A)
    assert info == 0
    assert lu_residual_ratio(A, (lh, ll), piv, m, n) < 30


def test_getrf_matches_scipy_on_binary64_input():
    sla = pytest.importorskip("scipy.linalg")
    g = datagen.rng(120)
    A = g.standard_normal((30, 30))
    lh, _, piv, info = oracle.dd_getrf((np.asfortranarray(A), np.zeros((30, 30), order="F")))
    lu, p = sla.lu_factor(A)
    assert info == 0 and np.array_equal(piv, p + 1)
    assert np.abs(lh - lu).max() <= 1e-12 * np.abs(lu).max()


def test_getrf_info_on_singular_input():
    A = np.array([[1.0, 2.0, 0.0, 3.0], [2.0, 1.0, 0.0, 1.0], [0.0, 1.0, 0.0, 5.0],
                  [1.0, 1.0, 0.0, 2.0]])
    z = np.zeros_like(A)
    assert oracle.dd_getrf((np.asfortranarray(A), z))[3] == 3
    B = np.array([[1.0, 2.0], [1.0, 2.0]])
    assert oracle.dd_getrf((np.asfortranarray(B), np.zeros((2, 2))))[3] == 2


@pytest.mark.parametrize("trans", ["N", "T"])
def test_getrs_lapack_ratio(trans):
    n = 36
    g = datagen.rng(130)
    A = datagen.dd_matrix(g, n, n)
    B = datagen.dd_matrix(g, n, 4)
    lh, ll, piv, info = oracle.dd_getrf(A)
    X = oracle.dd_getrs(trans, (lh, ll), piv, B)
    rr, cc = np.meshgrid(np.arange(n), np.arange(4), indexing="ij")
    R = oracle.exact_gemm_entries(trans, "N", n, (-1.0, 0.0), A, X, (1.0, 0.0), B, rr.ravel(),
                                  cc.ravel())
    An = np.abs(A[0]).sum(axis=0).max()
    Xn = np.abs(X[0]).sum(axis=0).max()
    ratio = np.abs(R[0]).reshape(n, 4).sum(axis=0).max() / (An * Xn * EPS_DD)
    assert ratio < 30


# ---------------------------------------------------------------------------
# Rtrsm
# ---------------------------------------------------------------------------



@pytest.mark.parametrize("side,uplo,transa,diag", TRSM_VARIANTS)
def test_trsm_recovers_exact_integer_solution(side, uplo, transa, diag):
    """Integer X, triangular integer A with power-of-two diagonal, alpha = 2:
    B = op(A) X / 2 (or X op(A) / 2) is exact in binary64, and every step of
    the substitution is exact in dd, so the solve must return X bit for bit.
    The unused triangle (and a unit diagonal) hold NaN and must not be read."""
    g = datagen.rng(70)
    m, n = 9, 7
    order = m if side == "L" else n
    A = g.integers(-6, 7, (order, order)).astype(np.float64)
    np.fill_diagonal(A, g.choice([-4.0, -2.0, -1.0, 1.0, 2.0, 4.0], order))
    X = g.integers(-20, 21, (m, n)).astype(np.float64)
    T = op_triangle(A, uplo, transa, diag, order)
    Bx = (T @ X if side == "L" else X @ T) / 2.0
    stored = A.copy()
    r, c = np.meshgrid(np.arange(order), np.arange(order), indexing="ij")
    unused = (r > c) if uplo == "U" else (r < c)
    if diag == "U":
        unused |= r == c
    stored[unused] = np.nan
    Ad = (np.asfortranarray(stored), np.zeros((order, order), order="F"))
    xh, xl = oracle.dd_trsm(side, uplo, transa, diag, (2.0, 0.0), Ad,
                            (np.asfortranarray(Bx), np.zeros((m, n), order="F")))
    assert np.array_equal(xh, X) and not xl.any()


@pytest.mark.parametrize("side,uplo,transa,diag", TRSM_VARIANTS[::3])
def test_trsm_matches_fraction_solve(side, uplo, transa, diag):
    """Tiny dd systems against the exact rational solution."""
    c = datagen.trsm_case(71, side, uplo, transa, diag, 5, 4)
    order = c.m if side == "L" else c.n
    T = [[Fraction(0)] * order for _ in range(order)]
    for i in range(order):
        for j in range(order):
            inside = (i <= j) if uplo == "U" else (i >= j)
            if i == j and diag == "U":
                v = Fraction(1)
            elif inside:
                v = F(c.A[0][i, j], c.A[1][i, j])
            else:
                v = Fraction(0)
            if transa == "T":
                T[j][i] = v
            else:
                T[i][j] = v
    al = F(*c.alpha)
    Bf = [[al * F(c.B[0][i, j], c.B[1][i, j]) for j in range(c.n)] for i in range(c.m)]
    # side R: X T = B  <=>  T^T X^T = B^T
    Ts = T if side == "L" else [list(r) for r in zip(*T)]
    rhs = Bf if side == "L" else [list(r) for r in zip(*Bf)]
    lower = all(Ts[i][j] == 0 for i in range(order) for j in range(i + 1, order))
    cols = len(rhs[0])
    Xs = [[Fraction(0)] * cols for _ in range(order)]
    rows = range(order) if lower else range(order - 1, -1, -1)
    for q in range(cols):
        for i in rows:
            s = rhs[i][q] - sum(Ts[i][k] * Xs[k][q] for k in range(order) if k != i)
            Xs[i][q] = s / Ts[i][i]
    X = Xs if side == "L" else [list(r) for r in zip(*Xs)]
    xh, xl = oracle.dd_trsm(side, uplo, transa, diag, c.alpha, c.A, c.B)
    for i in range(c.m):
        for j in range(c.n):
            err = abs(F(xh[i, j], xl[i, j]) - X[i][j])
            assert err <= Fraction(2) ** -96 * abs(X[i][j]) + Fraction(2) ** -200


@pytest.mark.parametrize("side,uplo,transa,diag", TRSM_VARIANTS)
def test_trsm_backward_error_within_bound(side, uplo, transa, diag):
    c = datagen.trsm_case(72, side, uplo, transa, diag, 37, 29, pad=3)
    X = oracle.dd_trsm(side, uplo, transa, diag, c.alpha, c.A, c.B, c.m, c.n)
    X = (X[0][:c.m, :c.n], X[1][:c.m, :c.n])
    assert trsm_residual_over_bound(c, X) <= 1.0
    assert is_normalised(*X)


@pytest.mark.parametrize("side,uplo,transa,diag", TRSM_VARIANTS[1::3])
def test_trsm_matches_scipy_on_binary64_inputs(side, uplo, transa, diag):
    """With lo planes zero the dd solve agrees with scipy's binary64 one to
    binary64 accuracy (the matrices are diagonally dominant)."""
    sla = pytest.importorskip("scipy.linalg")
    c = datagen.trsm_case(73, side, uplo, transa, diag, 23, 31)
    order = c.m if side == "L" else c.n
    A0 = np.nan_to_num(c.A[0], nan=0.0)
    B0 = c.B[0]
    xh, _ = oracle.dd_trsm(side, uplo, transa, diag, (2.0, 0.0),
                           (c.A[0], np.zeros_like(c.A[0])), (B0, np.zeros_like(B0)))
    lower, trans = uplo == "L", 1 if transa == "T" else 0
    if side == "L":
        ref = sla.solve_triangular(A0, 2.0 * B0, trans=trans, lower=lower,
                                   unit_diagonal=diag == "U")
    else:   # X op(A) = 2B  <=>  op(A)^T X^T = 2B^T
        ref = sla.solve_triangular(A0, 2.0 * B0.T, trans=1 - trans, lower=lower,
                                   unit_diagonal=diag == "U").T
    assert np.abs(xh - ref).max() <= 1e-13 * np.abs(ref).max()


def test_trsm_alpha_zero_and_empty():
    c = datagen.trsm_case(74, "L", "U", "N", "N", 6, 5)
    B = (c.B[0].copy(order="F"), c.B[1].copy(order="F"))
    Anan = (np.full_like(c.A[0], np.nan), np.full_like(c.A[1], np.nan))
    xh, xl = oracle.dd_trsm("L", "U", "N", "N", (0.0, 0.0), Anan, B)
    assert not xh.any() and not xl.any()
    xh, xl = oracle.dd_trsm("L", "U", "N", "N", c.alpha, c.A, B, 0, 5)
    assert np.array_equal(xh, B[0]) and np.array_equal(xl, B[1])


# ---------------------------------------------------------------------------
# planted mistakes: every broken copy of the oracle must fail this file
# ---------------------------------------------------------------------------

MUTANTS = {
    "dropped_cross_term": ("e += a.hi * b.lo + a.lo * b.hi + a.lo * b.lo;",
                           "e += a.lo * b.hi + a.lo * b.lo;"),
    "two_sum_wrong_sign": ("*e = (a - av) + (b - bv);", "*e = (a - av) - (b - bv);"),
    "transposed_operand": ("int64_t idx = trans ? (c + r * ld) : (r + c * ld);",
                           "int64_t idx = trans ? (r + c * ld) : (c + r * ld);"),
    "dropped_beta_term": ("return dd_add(acc, dd_mul(beta, cin));", "return acc;"),
    "no_sticky_rounding": ("if (round_bit && (sticky || (mant & 1))) mant += 1;",
                           "if (round_bit && (mant & 1)) mant += 1;"),
    "sqrt_without_newton": ("fast_two_sum(x, corr, &s, &e);", "fast_two_sum(x, 0.0, &s, &e);"),
    "trsm_transposed_triangle": (
        "#define TIDX(r, c) ((right ^ ta) ? ((c) + (r) * lda) : ((r) + (c) * lda))",
        "#define TIDX(r, c) ((right ^ ta) ? ((r) + (c) * lda) : ((c) + (r) * lda))"),
    "trsm_wrong_sweep": ("const int t_lower = right ? op_upper : !op_upper;",
                         "const int t_lower = right ? !op_upper : op_upper;"),
    "trsm_alpha_ignored": ("b = dd_mul(alpha, b);", "b = dd_add(b, (odd){0.0, 0.0});"),
    "trsm_unit_diag_read": ("if (!unit) x = dd_div(", "x = dd_div("),
    "syr2k_second_product_sign": (
        "acc = dd_add(acc, dd_mul(op_elem(bh, bl, ldb, t, i, l),",
        "acc = dd_sub(acc, dd_mul(op_elem(bh, bl, ldb, t, i, l),"),
    "getrf_wrong_pivot": ("            if (dd_abs_greater((odd){ah[i + j * lda], al[i + j * lda]},",
                          "            if (!dd_abs_greater((odd){ah[i + j * lda], al[i + j * lda]},"),
    "getrf_left_columns_not_swapped": ("        if (p != j)\n            for (int64_t c = 0; c < n; ++c) {",
                                       "        if (p != j)\n            for (int64_t c = j; c < n; ++c) {"),
    "getrs_no_unpivot": ("            for (int64_t j = n - 1; j >= 0; --j)\n                if (ipiv[j] - 1 != j) SWAPROW(j, ipiv[j] - 1);",
                         ""),
    "qd_tier_drops_fourth_component": (
        "                    for (int z = 0; z < 4; ++z)\n                        if (alpha[x] != 0.0 && A[y][ia] != 0.0 && B[z][ib] != 0.0)",
        "                    for (int z = 0; z < 3; ++z)\n                        if (alpha[x] != 0.0 && A[y][ia] != 0.0 && B[z][ib] != 0.0)"),
    "symm_wrong_triangle": (
        "#define SYM(r, c) ((upper ? (r) <= (c) : (r) >= (c))",
        "#define SYM(r, c) ((upper ? (r) >= (c) : (r) <= (c))"),
}


@pytest.mark.skipif(os.environ.get("DD_ORACLE_LIB") is not None,
                    reason="already running against a planted mistake")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_are_caught(name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "dd_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "mutant.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        so = oracle.compile_source(path, os.path.join(d, "libmutant.so"))
        env = dict(os.environ, DD_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.abspath(__file__)], env=env, capture_output=True, text=True,
                           cwd=os.path.dirname(HERE))
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
