"""Pins for the split-precision oracle (oracle/ozaki_ref.py), CPU only."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import datagen
from oracle import ozaki_ref as oz
from oracle import fraction_ref as fr


def test_scale_exponent_is_tight():
    for v in [1.0, 0.999, 0.5, 0.4999, 3e-7, 2.0 ** -1000, 1e300, 5e-324]:
        e = oz.scale_exponent([v, -v / 3])
        assert Fraction(2) ** (e - 1) > Fraction(v) >= Fraction(2) ** (e - 2)
    assert oz.scale_exponent([0.0, -0.0]) == 0


def test_digits_reproduce_the_integer_and_stay_in_range():
    g = datagen.rng(1)
    for S in (2, 5, 14, 15):
        for _ in range(300):
            X = int(g.integers(-2 ** 62, 2 ** 62)) * int(g.integers(1, 2 ** 40)) % (2 ** (8 * S - 1))
            X = X if g.random() < 0.5 else -X
            d = oz.digits_of(X, S)
            assert sum(dt * 256 ** (S - 1 - t) for t, dt in enumerate(d)) == X
            assert all(-128 <= dt <= 127 for dt in d[1:]) and -128 <= d[0] <= 128
    assert oz.digits_of(2 ** 111, 14)[0] == 128 and oz.digits_of(-2 ** 111, 14)[0] == -128


def test_split_rounds_within_one_unit():
    g = datagen.rng(2)
    h, l = datagen.dd_matrix(g, 5, 40)
    f = np.ldexp(1.0, g.integers(-30, 30, (5, 1)))   # per-row powers of two (exact)
    h, l = h * f, l * f
    S = 14
    for r in range(5):
        D, e = oz.split_row(h[r], l[r], S)
        for c in range(40):
            x = Fraction(float(h[r, c])) + Fraction(float(l[r, c]))
            assert abs(x * Fraction(2) ** -e) < Fraction(1, 2)
            X = sum(int(D[t, c]) * 256 ** (S - 1 - t) for t in range(S))
            assert abs(X - x * Fraction(2) ** (8 * S - e)) <= 1


def test_integer_inputs_recombine_exactly():
    g = datagen.rng(3)
    m, n, k, S = 6, 5, 9, 14
    A = g.integers(-100, 100, (m, k)).astype(float)
    B = g.integers(-100, 100, (k, n)).astype(float)
    DA, ea = oz.split_matrix(A, np.zeros_like(A), S)
    DB, fb = oz.split_matrix(B.T.copy(), np.zeros_like(B.T), S)
    V = oz.recombine_exact(oz.band_products(DA, DB), ea, fb)
    ref = A @ B
    assert all(V[i][j] == Fraction(ref[i, j]) for i in range(m) for j in range(n))


@pytest.mark.parametrize("ill", [None, "outer"])
def test_truncation_error_within_documented_bound(ill):
    m, n, k = 4, 3, 50
    c = datagen.gemm_case(4, "N", "N", m, n, k, alpha=(1.0, 0.0), beta=(0.0, 0.0), ill=ill)
    exact = fr.gemm_exact("N", "N", m, n, k, (1.0, 0.0), c.A, c.B, (0.0, 0.0), c.C)
    errs = {}
    for S in (10, 11, 14):
        DA, ea = oz.split_matrix(*oz.op_rows(c.A, False, m, k), S)
        DB, fb = oz.split_matrix(*oz.op_cols(c.B, False, k, n), S)
        V = oz.recombine_exact(oz.band_products(DA, DB), ea, fb)
        worst = 0.0
        for i in range(m):
            for j in range(n):
                err = abs(V[i][j] - exact[i][j])
                doc = Fraction(43, 10) * k * Fraction(2) ** (int(ea[i]) + int(fb[j]) - 8 * S)
                assert err <= doc
                ab = sum(abs(Fraction(float(c.A[0][i, l]))) * abs(Fraction(float(c.B[0][l, j])))
                         for l in range(k))
                worst = max(worst, float(err / (4 * k * Fraction(2) ** -104 * ab)))
        errs[S] = worst
    # S = 14 meets the accuracy bound with margin; fewer slices do not, and
    # each slice buys 8 bits
    assert errs[14] < 0.25
    assert errs[10] > 1.0
    assert 30 < errs[10] / max(errs[11], 1e-300) < 2000


# ---------------------------------------------------------------------------
# residue (CRT) form
# ---------------------------------------------------------------------------

def test_crt_moduli_pairwise_coprime():
    import math

    mods = oz.crt_moduli()
    assert len(mods) == 40 and mods == sorted(mods, reverse=True) and max(mods) == 256
    for i in range(len(mods)):
        for j in range(i):
            assert math.gcd(mods[i], mods[j]) == 1
    assert [oz.sym_residue(x, 256) for x in (127, 128, -128, 255)] == [127, -128, -128, -1]
    assert [oz.sym_residue(x, 255) for x in (127, 128, -127)] == [127, -127, -127]


def test_crt_reconstruction_equals_integer_product():
    g = datagen.rng(7)
    mods = oz.crt_moduli(32)
    P = 1
    for p in mods:
        P *= p
    k = 9
    A = [[int(g.integers(-2 ** 62, 2 ** 62)) * 2 ** 49 + int(g.integers(0, 2 ** 49))
          for _ in range(k)] for _ in range(3)]
    B = [[int(g.integers(-2 ** 62, 2 ** 62)) * 2 ** 49 + int(g.integers(0, 2 ** 49))
          for _ in range(k)] for _ in range(4)]
    exact = [[sum(a * b for a, b in zip(ra, rb)) for rb in B] for ra in A]
    assert P > 2 * max(abs(v) for r in exact for v in r)
    RA = np.array([[[oz.sym_residue(x, p) for x in r] for r in A] for p in mods])
    RB = np.array([[[oz.sym_residue(x, p) for x in r] for r in B] for p in mods])
    assert np.abs(RA).max() <= 128 and np.abs(RB).max() <= 128
    rec = oz.crt_reconstruct(oz.crt_products(RA, RB, mods), mods)
    assert [[int(v) for v in r] for r in rec] == exact


def test_crt_form_error_is_the_operand_rounding_only():
    m, n, k = 3, 3, 40
    c = datagen.gemm_case(8, "N", "N", m, n, k, alpha=(1.0, 0.0), beta=(0.0, 0.0))
    mods = oz.crt_moduli(32)
    RA, ea = oz.residue_planes(*oz.op_rows(c.A, False, m, k), mods)
    RB, fb = oz.residue_planes(*oz.op_cols(c.B, False, k, n), mods)
    rec = oz.crt_reconstruct(oz.crt_products(RA, RB, mods), mods)
    exact = fr.gemm_exact("N", "N", m, n, k, (1.0, 0.0), c.A, c.B, (0.0, 0.0), c.C)
    for i in range(m):
        for j in range(n):
            v = Fraction(int(rec[i, j])) * Fraction(2) ** (int(ea[i]) + int(fb[j]) - 224)
            assert abs(v - exact[i][j]) <= k * Fraction(2) ** (int(ea[i]) + int(fb[j]) - 112)


# ---------------------------------------------------------------------------
# per-call certificate
# ---------------------------------------------------------------------------

def _bf16_neighbours(y: Fraction):
    """y as a float32 bit pattern (asserting it is a bf16) and the next bf16 above."""
    f = np.float32(float(y))
    assert Fraction(float(f)) == y, "not a float32"
    bits = int(np.array(f).view(np.uint32))
    assert bits & 0xFFFF == 0, "not a bf16"
    up = np.array(bits + 0x10000, dtype=np.uint32).view(np.float32)
    return bits, Fraction(float(up))


def test_bf16_floor_is_the_largest_bf16_not_above():
    """Brute force over the neighbouring bf16 values (numpy's float32 bits)."""
    g = datagen.rng(40)
    xs = [Fraction(0), Fraction(1, 3), Fraction(1, 2) - Fraction(1, 2 ** 60),
          Fraction(2) ** -126, Fraction(2) ** -133, Fraction(3, 2) * Fraction(2) ** -134,
          Fraction(2) ** -127 * Fraction(5, 3)]
    for _ in range(400):
        xs.append(Fraction(float(g.uniform(0.0, 0.5))) * Fraction(2) ** int(g.integers(-140, 0)))
    for x in xs:
        y = oz.bf16_floor(x)
        assert 0 <= y <= x
        if x == 0:
            continue
        bits, nxt = _bf16_neighbours(y)
        assert nxt > x
    # exact bf16 values map to themselves
    for v in (0.25, 0.1875, 2.0 ** -126, 2.0 ** -133, 3 * 2.0 ** -133):
        assert oz.bf16_floor(Fraction(v)) == Fraction(v)


def _stress_rows(seed, rows, k, spread):
    """dd rows whose entries spread over 2^-spread .. 1 of the row maximum."""
    g = datagen.rng(seed)
    h = g.uniform(-1, 1, (rows, k)) * np.ldexp(1.0, g.integers(-spread, 1, (rows, k)))
    h, l = datagen.dd_lo_for(h, g)
    return h, l


@pytest.mark.parametrize("W", [112, 120, 128])
def test_crt_product_error_within_its_constant(W):
    """|a b - a' b'| <= (1 + 2^-W) 2^(e + f - W) for every product of the
    rounded operands of the residue form, entries over 60 binades."""
    ah, al = _stress_rows(41, 3, 40, 60)
    bh, bl = _stress_rows(42, 3, 40, 60)
    cst = oz.product_error_constant("crt", W)
    for i in range(3):
        XA, e = oz.scaled_integers(ah[i], al[i], W // 8)
        for j in range(3):
            XB, f = oz.scaled_integers(bh[j], bl[j], W // 8)
            for l in range(40):
                a = Fraction(float(ah[i, l])) + Fraction(float(al[i, l]))
                b = Fraction(float(bh[j, l])) + Fraction(float(bl[j, l]))
                ap = XA[l] * Fraction(2) ** (e - W)
                bp = XB[l] * Fraction(2) ** (f - W)
                assert abs(a * b - ap * bp) <= cst * Fraction(2) ** (e + f - W)


@pytest.mark.parametrize("S", [10, 14, 15])
def test_sliced_product_error_within_its_constant(S):
    """One product through the digit bands (pairs t + u < S only) stays within
    product_error_constant("sliced", 8S) 2^(e + f - 8S)."""
    ah, al = _stress_rows(43, 40, 1, 0)
    bh, bl = _stress_rows(44, 40, 1, 0)
    cst = oz.product_error_constant("sliced", 8 * S)
    for q in range(40):
        DA, ea = oz.split_matrix(ah[q:q + 1], al[q:q + 1], S)
        DB, fb = oz.split_matrix(bh[q:q + 1], bl[q:q + 1], S)
        V = oz.recombine_exact(oz.band_products(DA, DB), ea, fb)[0][0]
        a = Fraction(float(ah[q, 0])) + Fraction(float(al[q, 0]))
        b = Fraction(float(bh[q, 0])) + Fraction(float(bl[q, 0]))
        unit = Fraction(2) ** (int(ea[0]) + int(fb[0]) - 8 * S)
        assert abs(a * b - V) <= cst * unit


def _crt_error_ratio(c, W, m, n, k):
    """max over entries of |alpha| |sum a'b' - sum ab| / (12 k 2^-106 (|alpha||A||B| +
    |beta||C|)): at most 1 is what a certified width promises."""
    ah, al = oz.op_rows(c.A, c.transa == "T", m, k)
    bh, bl = oz.op_cols(c.B, c.transb == "T", k, n)
    alpha = abs(Fraction(c.alpha[0]) + Fraction(c.alpha[1]))
    beta = abs(Fraction(c.beta[0]) + Fraction(c.beta[1]))
    worst = Fraction(0)
    for i in range(m):
        XA, e = oz.scaled_integers(ah[i], al[i], W // 8)
        for j in range(n):
            XB, f = oz.scaled_integers(bh[j], bl[j], W // 8)
            err, ab = Fraction(0), Fraction(0)
            for l in range(k):
                a = Fraction(float(ah[i, l])) + Fraction(float(al[i, l]))
                b = Fraction(float(bh[j, l])) + Fraction(float(bl[j, l]))
                err += a * b - XA[l] * XB[l] * Fraction(2) ** (e + f - 2 * W)
                ab += abs(a) * abs(b)
            cc = abs(Fraction(float(c.C[0][i, j])) + Fraction(float(c.C[1][i, j])))
            worst = max(worst, alpha * abs(err) /
                        (12 * k * Fraction(2) ** -106 * (alpha * ab + beta * cc)))
    return worst


def test_certified_width_keeps_the_error_within_the_bound():
    """Inner-scaled operands (exponents spread along k): the rule picks 128
    bits, and the exact error of the rounded product then stays within three
    quarters of the bound; at the default 112 bits it does not."""
    m, n, k = 3, 3, 400
    c = datagen.gemm_case(45, "N", "N", m, n, k, ill="inner")
    d = oz.exact_margins(oz.op_rows(c.A, False, m, k), oz.op_cols(c.B, False, k, n), c.alpha,
                         c.beta, c.C)
    W = oz.certified_width(min(d.values()), "crt", [112, 120, 128])
    assert W == 128
    assert _crt_error_ratio(c, 128, m, n, k) <= 1
    assert _crt_error_ratio(c, 112, m, n, k) > 1


def test_adversarial_operands_certify_no_width():
    """Rows of A with 0.9 in column 0 and entries of size 2^-40 elsewhere, row 0
    of B zero: the
    margin is the closed form sum_{l >= 1} |a_l||b_l| 2^-(e+f), no width up to
    128 bits qualifies, and at 128 bits the error does exceed the bound."""
    k = 64
    g = datagen.rng(46)
    ah = g.uniform(0.5, 1.0, (2, k)) * 2.0 ** -40
    ah[:, 0] = 0.9
    bh = g.uniform(-1, 1, (k, 2))
    bh[0, :] = 0.0
    ah, al = datagen.dd_lo_for(ah, g)        # full dd entries: 106-bit values
    bh, bl = datagen.dd_lo_for(bh, g)
    A = (np.asfortranarray(ah), np.asfortranarray(al))
    B = (np.asfortranarray(bh), np.asfortranarray(bl))
    C = (np.zeros((2, 2), order="F"), np.zeros((2, 2), order="F"))
    c = datagen.GemmCase("N", "N", 2, 2, k, (1.0, 0.0), A, B, (0.0, 0.0), C)
    d = oz.exact_margins(oz.op_rows(A, False, 2, k), oz.op_cols(B, False, k, 2), c.alpha,
                         c.beta)
    for (i, j), v in d.items():
        e, f = oz.scale_exponent(ah[i]), oz.scale_exponent(bh[:, j])
        want = sum((Fraction(float(ah[i, l])) + Fraction(float(al[i, l]))) *
                   abs(Fraction(float(bh[l, j])) + Fraction(float(bl[l, j])))
                   for l in range(1, k))
        assert v == want * Fraction(2) ** -(e + f)
    assert oz.certified_width(min(d.values()), "crt", [112, 120, 128]) == 0
    assert oz.certified_width(min(d.values()), "sliced", [112, 120]) == 0
    assert _crt_error_ratio(c, 128, 2, 2, k) > 1


def test_margins_cover_beta_c_and_skip_zero_rows():
    g = datagen.rng(47)
    A = datagen.dd_matrix(g, 3, 5)
    B = datagen.dd_matrix(g, 5, 2)
    A[0][1, :] = 0.0
    A[1][1, :] = 0.0
    C = datagen.dd_matrix(g, 3, 2)
    d0 = oz.exact_margins(oz.op_rows(A, False, 3, 5), oz.op_cols(B, False, 5, 2), (1.0, 0.0),
                          (0.0, 0.0))
    d1 = oz.exact_margins(oz.op_rows(A, False, 3, 5), oz.op_cols(B, False, 5, 2), (2.0, 0.0),
                          (1.0, 0.0), C)
    assert (1, 0) not in d0 and (1, 1) not in d0 and len(d0) == 4
    for key, v in d0.items():
        i, j = key
        e, f = oz.scale_exponent(A[0][i]), oz.scale_exponent(B[0][:, j])
        cc = abs(Fraction(float(C[0][i, j])) + Fraction(float(C[1][i, j])))
        assert d1[key] == v + Fraction(1, 2) * cc * Fraction(2) ** -(e + f)
    up = oz.exact_margins(oz.op_rows(A, False, 3, 5), oz.op_rows(A, False, 3, 5), (1.0, 0.0),
                          (0.0, 0.0), tri=1)
    assert all(i <= j for i, j in up)
