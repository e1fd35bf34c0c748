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
