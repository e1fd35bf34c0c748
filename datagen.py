"""Seeded synthetic inputs for the dd Rgemm / Rsyrk / Rpotrf / Rpotrs workloads.

This module is shared by the tests, the benchmark and the oracle checks.  It
holds only the input recipes (random numbers, shapes, scalings); none of the
method's arithmetic.  All generators draw from numpy's PCG64 with an explicit
seed, so both sides of every comparison see identical bits.

Recipes (the manual benchmarks on random matrices; its dd format is a pair
hi + lo of binary64 numbers with |lo| <= ulp(hi)/2):

* dd entries: hi ~ U(-1, 1); lo' = hi * 2^-53 * U(-1, 1); then (hi, lo) is
  renormalised so that hi == fl(hi + lo) (one binary64 addition and one
  subtraction, the standard renormalisation of a two-term sum).
* dd scalars alpha, beta: hi ~ U(0.5, 2), lo as above.
* ill-scaled operands: A = D_r * A0, B = B0 * D_c with power-of-two diagonal
  scalings whose integer exponents are uniform on {-30..30} ("outer"); the
  "inner" stress variant also scales the shared dimension.
* grouped problems: m, n, k each round(exp(U(ln 16, ln 512))).
* SPD requests: G (n x 2n) = U [diag(s) 0] V^T with s geometric from 1 to
  1e-10 and random orthogonal U, V (products of Householder reflectors with
  Gaussian vectors), formed in binary64; G's lo plane follows the dd entry
  recipe.  F = G G^T then has condition ~1e20.  ``spd_request`` draws it
  with numpy on the host; ``spd_request_device`` with torch's seeded
  generator on the GPU (the served benchmark, so that admission never waits
  for host-side generation), the same construction with other random bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def rng(seed: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _renormalise(hi: np.ndarray, lo: np.ndarray):
    s = hi + lo
    return s, lo - (s - hi)


def dd_lo_for(hi: np.ndarray, g: np.random.Generator):
    """Return (hi', lo) with lo drawn as hi * 2^-53 * U(-1, 1), renormalised."""
    lo = hi * 2.0 ** -53 * g.uniform(-1.0, 1.0, size=hi.shape)
    return _renormalise(hi, lo)


def qd_tail_for(x0: np.ndarray, g: np.random.Generator):
    """Four components (x0', x1, x2, x3) with x_{t+1} drawn as x_t 2^-53
    U(-1, 1) and the four renormalised (each component within half an ulp
    of the one above)."""
    x = [np.asarray(x0, dtype=np.float64)]
    for _ in range(3):
        x.append(x[-1] * 2.0 ** -53 * g.uniform(-1.0, 1.0, size=x[-1].shape))
    for t in (0, 1, 2):   # top-down, twice: |x_{t+1}| <= ulp(x_t) / 2
        x[t], x[t + 1] = _renormalise(x[t], x[t + 1])
    for t in (0, 1, 2):
        x[t], x[t + 1] = _renormalise(x[t], x[t + 1])
    return tuple(x)


def qd_matrix(g: np.random.Generator, rows: int, cols: int, ld: int | None = None,
              low: float = -1.0, high: float = 1.0):
    """A rows x cols quad-double matrix: four column-major planes of leading
    dimension ld (padding rows NaN), x0 ~ U(low, high) and the lower
    components as ``qd_tail_for``."""
    ld = max(1, rows if ld is None else ld)
    comps = qd_tail_for(g.uniform(low, high, size=(rows, cols)), g)
    out = []
    for c in comps:
        P = np.full((ld, cols), np.nan, order="F")
        P[:rows, :] = c
        out.append(P)
    return tuple(out)


def qd_scalar(g: np.random.Generator, low: float = 0.5, high: float = 2.0):
    return tuple(float(c[0]) for c in qd_tail_for(np.array([g.uniform(low, high)]), g))


def dd_matrix(g: np.random.Generator, rows: int, cols: int, ld: int | None = None,
              low: float = -1.0, high: float = 1.0):
    """A rows x cols dd matrix in column-major planes of leading dimension ld.

    Padding rows (ld > rows) are filled with NaN so that a kernel that reads
    outside the logical matrix is caught by the comparison."""
    ld = max(1, rows if ld is None else ld)
    hi = g.uniform(low, high, size=(rows, cols))
    hi, lo = dd_lo_for(hi, g)
    H = np.full((ld, cols), np.nan, order="F")
    L = np.full((ld, cols), np.nan, order="F")
    H[:rows, :] = hi
    L[:rows, :] = lo
    return H, L


def dd_scalar(g: np.random.Generator, low: float = 0.5, high: float = 2.0):
    hi = np.array([g.uniform(low, high)])
    hi, lo = dd_lo_for(hi, g)
    return float(hi[0]), float(lo[0])


def pow2_exponents(g: np.random.Generator, count: int, lo: int = -30, hi: int = 30):
    return g.integers(lo, hi + 1, size=count)


def scale_rows(M, exps):
    """Multiply row r of both planes by 2^exps[r] (exact)."""
    f = np.ldexp(1.0, np.asarray(exps))[:, None]
    return M[0] * f, M[1] * f


def scale_cols(M, exps):
    f = np.ldexp(1.0, np.asarray(exps))[None, :]
    return M[0] * f, M[1] * f


@dataclass
class GemmCase:
    transa: str
    transb: str
    m: int
    n: int
    k: int
    alpha: tuple
    A: tuple
    B: tuple
    beta: tuple
    C: tuple


def gemm_case(seed: int, transa: str, transb: str, m: int, n: int, k: int,
              alpha=None, beta=None, pad: int = 0, ill: str | None = None) -> GemmCase:
    """Draw A, then B, then C, then alpha, then beta (column-major order).

    ``alpha``/``beta`` None means "random dd in [0.5, 2]".  ``pad`` extra rows
    make every leading dimension non-tight.  ``ill`` is None, "outer" or
    "inner" (the ill-scaled recipes above)."""
    g = rng(seed)
    ta, tb = transa.upper() in "TC", transb.upper() in "TC"
    ar, ac = (k, m) if ta else (m, k)
    br, bc = (n, k) if tb else (k, n)
    A = dd_matrix(g, ar, ac, ar + pad)
    B = dd_matrix(g, br, bc, br + pad)
    C = dd_matrix(g, m, n, m + pad)
    al = dd_scalar(g) if alpha is None else alpha
    be = dd_scalar(g) if beta is None else beta
    if ill is not None:
        er = pow2_exponents(g, m)
        ec = pow2_exponents(g, n)
        # op(A) row i scaled by 2^er[i]; op(B) column j by 2^ec[j]
        A = scale_cols(A, er) if ta else _scale_rows_padded(A, er)
        B = _scale_rows_padded(B, ec) if tb else scale_cols(B, ec)
        if ill == "inner":
            ek = pow2_exponents(g, k, -15, 15)
            A = _scale_rows_padded(A, ek) if ta else scale_cols(A, ek)
            B = scale_cols(B, -ek) if tb else _scale_rows_padded(B, -ek)
    return GemmCase(transa, transb, m, n, k, al, A, B, be, C)


def _scale_rows_padded(M, exps):
    exps = np.asarray(exps)
    f = np.ones(M[0].shape[0])
    f[: exps.size] = np.ldexp(1.0, exps)
    return M[0] * f[:, None], M[1] * f[:, None]


@dataclass
class TrsmCase:
    side: str
    uplo: str
    transa: str
    diag: str
    m: int
    n: int
    alpha: tuple
    A: tuple
    B: tuple


def triangular_dd(g: np.random.Generator, order: int, uplo: str, diag: str,
                  ld: int | None = None):
    """An order x order triangular dd matrix in column-major planes: the uplo
    triangle U(-1, 1) off the diagonal, diagonal entries of magnitude
    order * U(1, 2) with random sign (strictly diagonally dominant, so the
    solve is well conditioned at every order).  The other triangle, padding
    rows and -- for diag = 'U' -- the diagonal are NaN: only entries a solve
    may read are finite."""
    ld = max(1, order if ld is None else ld)
    H, L = dd_matrix(g, order, order, ld)
    d = order * g.uniform(1.0, 2.0, order) * g.choice([-1.0, 1.0], order)
    dh, dl = dd_lo_for(d, g)
    idx = np.arange(order)
    H[idx, idx], L[idx, idx] = dh, dl
    r, c = np.meshgrid(idx, idx, indexing="ij")
    unused = (r > c) if uplo.upper() == "U" else (r < c)
    if diag.upper() == "U":
        unused |= r == c
    H[:order, :order][unused] = np.nan
    L[:order, :order][unused] = np.nan
    return H, L


def trsm_case(seed: int, side: str, uplo: str, transa: str, diag: str, m: int, n: int,
              alpha=None, pad: int = 0) -> TrsmCase:
    """Draw A (order m for side 'L', n for side 'R'; ``triangular_dd``), then
    B (m x n, U(-1, 1) dd), then alpha (random dd in [0.5, 2] when None).
    ``pad`` extra rows make both leading dimensions non-tight."""
    g = rng(seed)
    order = m if side.upper() == "L" else n
    A = triangular_dd(g, order, uplo, diag, order + pad)
    B = dd_matrix(g, m, n, m + pad)
    al = dd_scalar(g) if alpha is None else alpha
    return TrsmCase(side, uplo, transa, diag, m, n, al, A, B)


def grouped_problems(seed: int, count: int = 4096, lo: int = 16, hi: int = 512):
    """m, n, k per problem, each round(exp(U(ln lo, ln hi)))."""
    g = rng(seed)
    u = g.uniform(math.log(lo), math.log(hi), size=(count, 3))
    return np.rint(np.exp(u)).astype(np.int64)


def householder_orthogonal_apply(g: np.random.Generator, X: np.ndarray, side: str,
                                 reflectors: int = 3) -> np.ndarray:
    """Apply a random orthogonal Q = H_1 ... H_r (Householder reflectors with
    Gaussian vectors) to X from the left (Q X) or the right (X Q^T)."""
    X = np.array(X, dtype=np.float64, order="F")
    dim = X.shape[0] if side == "left" else X.shape[1]
    for _ in range(reflectors):
        v = g.standard_normal(dim)
        v /= np.linalg.norm(v)
        if side == "left":
            X -= 2.0 * np.outer(v, v @ X)
        else:
            X -= 2.0 * np.outer(X @ v, v)
    return X


def spd_request(seed: int, n: int, nrhs: int = 4, smin: float = 1e-10):
    """One served-solve request: G (n x 2n) dd and B (n x nrhs) dd."""
    g = rng(seed)
    s = np.geomspace(1.0, smin, n)
    G = np.zeros((n, 2 * n), order="F")
    G[np.arange(n), np.arange(n)] = s
    G = householder_orthogonal_apply(g, G, "left")
    G = householder_orthogonal_apply(g, G, "right")
    gh, gl = dd_lo_for(G, g)
    Bh = g.uniform(-1.0, 1.0, size=(n, nrhs))
    Bh, Bl = dd_lo_for(Bh, g)
    return (np.asfortranarray(gh), np.asfortranarray(gl)), (np.asfortranarray(Bh),
                                                            np.asfortranarray(Bl))


def request_sizes(seed: int, count: int = 2000, lo: int = 64, hi: int = 2048):
    g = rng(seed)
    return np.rint(np.exp(g.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def poisson_arrivals(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps."""
    g = rng(seed)
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=count))


def spd_request_device(seed: int, n: int, nrhs: int = 4, smin: float = 1e-10):
    """The served-solve recipe of ``spd_request`` generated on the current
    CUDA device with torch's seeded generator: G = U [diag(s) 0] V^T (s
    geometric from 1 to smin, U and V products of three Householder
    reflectors with Gaussian vectors), lo planes hi 2^-53 U(-1, 1)
    renormalised, B entries U(-1, 1) dd.  Returns ((G_hi, G_lo), (B_hi,
    B_lo)) as column-major float64 device tensors."""
    import torch

    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    dev = "cuda"
    s = torch.logspace(0.0, float(np.log10(smin)), n, dtype=torch.float64, device=dev)
    G = torch.zeros((n, 2 * n), dtype=torch.float64, device=dev)
    G[torch.arange(n), torch.arange(n)] = s
    for side in ("left", "right"):
        for _ in range(3):
            dim = n if side == "left" else 2 * n
            v = torch.randn(dim, dtype=torch.float64, device=dev, generator=gen)
            v /= torch.linalg.norm(v)
            if side == "left":
                G -= 2.0 * torch.outer(v, v @ G)
            else:
                G -= 2.0 * torch.outer(G @ v, v)

    def dd_pair(H):
        lo = H * 2.0 ** -53 * (2 * torch.rand(H.shape, dtype=torch.float64, device=dev,
                                               generator=gen) - 1)
        hi = H + lo
        lo = lo - (hi - H)
        # column-major (shape rows x cols, strides (1, rows))
        return hi.t().contiguous().t(), lo.t().contiguous().t()

    Bh = 2 * torch.rand((n, nrhs), dtype=torch.float64, device=dev, generator=gen) - 1
    return dd_pair(G), dd_pair(Bh)

