"""The dd scalar operations of the kernels, one at a time (GPU).

Through ``mp_dd_elementwise``: on dd operands spread over 2^-60 .. 2^60
(lo parts drawn as in every workload), each result is compared with the
exact rational result: the relative error stays within the bound stated
for the operation (accurate add 3u^2 + 13u^3 <= 2^-104.3; product with the
low-by-low term dropped 8u^2 = 2^-103; two-digit division ~11u^2 < 2^-102;
division with the reciprocal digit ~20u^2 < 2^-101.6; square root 2^-103;
reciprocal ~6u^2 < 2^-102.5), with u = 2^-53.  Exact
results (integer quotients, perfect squares, powers of two) come out exact,
with a zero lo part; sqrt of 0 and of a negative number is 0; argument
errors.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest
import torch

import datagen
from gpucase import dev

pytestmark = pytest.mark.gpu

BOUND = {"add": 2.0 ** -104.3, "mul": 2.0 ** -103, "div": 2.0 ** -102, "divr": 2.0 ** -101.6,
         "sqrt": 2.0 ** -103, "rcp": 2.0 ** -102.5}


def operands(seed, n):
    g = datagen.rng(seed)
    e = g.integers(-60, 61, size=n).astype(np.float64)
    hi = g.uniform(0.5, 1.0, size=n) * np.where(g.random(n) < 0.5, -1.0, 1.0) * 2.0 ** e
    hi, lo = datagen.dd_lo_for(hi, g)
    return np.ascontiguousarray(hi), np.ascontiguousarray(lo)


def run(mp, op, x, y=None):
    n = x[0].shape[0]
    dx = dev(x)
    dy = dev(y) if y is not None else None
    z = (torch.empty(n, dtype=torch.float64, device="cuda"),
         torch.empty(n, dtype=torch.float64, device="cuda"))
    mp.mp_dd_elementwise(op, n, dx, dy, z)
    torch.cuda.synchronize()
    return z[0].cpu().numpy(), z[1].cpu().numpy()


def exact(op, xh, xl, yh=None, yl=None):
    x = Fraction(float(xh)) + Fraction(float(xl))
    y = None if yh is None else Fraction(float(yh)) + Fraction(float(yl))
    if op == "add":
        return x + y
    if op == "mul":
        return x * y
    if op in ("div", "divr"):
        return x / y
    if op == "rcp":
        return 1 / x
    return None


def rel_err_sqrt(zh, zl, xh, xl):
    # |z - sqrt(x)| / sqrt(x) <= |z^2 - x| / x (for z near sqrt(x)), exactly
    x = Fraction(float(xh)) + Fraction(float(xl))
    z = Fraction(float(zh)) + Fraction(float(zl))
    return float(abs(z * z - x) / x)


@pytest.mark.parametrize("op", ["add", "mul", "div", "divr", "rcp"])
def test_binary_ops_within_bound(cuda_lib, op):
    n = 3000
    x = operands(901, n)
    y = operands(902, n) if op != "rcp" else None
    zh, zl = run(cuda_lib, op, x, y)
    worst = 0.0
    for i in range(n):
        ex = exact(op, x[0][i], x[1][i], *( (y[0][i], y[1][i]) if y is not None else ()))
        got = Fraction(float(zh[i])) + Fraction(float(zl[i]))
        worst = max(worst, float(abs(got - ex) / abs(ex)))
        assert abs(zl[i]) <= abs(np.spacing(zh[i])) / 2 + 0.0   # normalised
    assert worst <= BOUND[op], (op, np.log2(worst))


def test_sqrt_within_bound(cuda_lib):
    n = 3000
    xh, xl = operands(903, n)
    x = (np.abs(xh), np.where(xh < 0, -xl, xl))
    zh, zl = run(cuda_lib, "sqrt", x)
    worst = max(rel_err_sqrt(zh[i], zl[i], x[0][i], x[1][i]) for i in range(n))
    # |z - r| / r ~ |z^2 - x| / (2x)
    assert worst / 2 <= BOUND["sqrt"], np.log2(worst / 2)


def test_exact_results_are_exact(cuda_lib):
    mp = cuda_lib
    g = datagen.rng(904)
    q = g.integers(-2 ** 26, 2 ** 26, size=500).astype(np.float64)
    b = g.integers(1, 2 ** 26, size=500).astype(np.float64) * np.where(g.random(500) < 0.5,
                                                                         -1.0, 1.0)
    a = q * b                      # exact: |a| < 2^52
    z0 = np.zeros(500)
    for op in ("div", "divr"):
        zh, zl = run(mp, op, (a, z0), (b, z0))
        assert np.array_equal(zh, q) and not zl.any(), op
    r = g.integers(1, 2 ** 26, size=500).astype(np.float64)
    zh, zl = run(mp, "sqrt", (r * r, z0))
    assert np.array_equal(zh, r) and not zl.any()
    p2 = 2.0 ** g.integers(-500, 500, size=500).astype(np.float64)
    zh, zl = run(mp, "rcp", (p2, z0))
    assert np.array_equal(zh, 1.0 / p2) and not zl.any()
    zh, zl = run(mp, "sqrt", (np.array([0.0, -4.0, -1e-300]), np.zeros(3)))
    assert not zh.any() and not zl.any()


def test_errors(cuda_lib):
    mp = cuda_lib
    x = dev((np.ones(4), np.zeros(4)))
    z = dev((np.zeros(4), np.zeros(4)))
    assert mp.mp_dd_elementwise("pow", 4, x, x, z, check=False) == -1
    assert mp.mp_dd_elementwise("add", -1, x, x, z, check=False) == -2
    assert mp.mp_dd_elementwise("add", 4, (None, None), x, z, check=False) == -3
    assert mp.mp_dd_elementwise("div", 4, x, None, z, check=False) == -4
    assert mp.mp_dd_elementwise("sqrt", 4, x, None, (None, None), check=False) == -5
    assert mp.mp_dd_elementwise("sqrt", 4, x, None, z, check=False) == 0
    assert mp.mp_dd_elementwise("add", 0, x, x, z, check=False) == 0
