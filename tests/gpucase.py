"""Helpers for the GPU parity tests: move a seeded case to the device, run
the library through its C ABI binding, bring results back, and compare with
the oracle (exact tier or scalar dd tier) against the accuracy bound."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from ddcheck import err_over_bound, gemm_bound_entries, is_normalised


def dev(pair):
    import paper_2109_13406_gb300 as mp

    return tuple(mp.to_device(x) for x in pair)


def host(pair, rows=None, cols=None):
    import paper_2109_13406_gb300 as mp

    torch.cuda.synchronize()
    out = tuple(mp.to_numpy(x) for x in pair)
    if rows is not None:
        out = tuple(x[:rows, :cols] for x in out)
    return out


def run_gemm(c, fn=None):
    """Run case ``c`` (datagen.GemmCase) on the GPU; returns (hi, lo) m x n."""
    import paper_2109_13406_gb300 as mp

    A, B, C = dev(c.A), dev(c.B), dev(c.C)
    fn = fn or mp.mp_dd_Rgemm
    fn(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, c.A[0].shape[0], B, c.B[0].shape[0],
       c.beta, C, c.C[0].shape[0])
    return host(C, c.m, c.n)


def sample_blocks(m, n, bs=64, count=8, seed=0):
    """Row/col index arrays of ``count`` bs x bs blocks: the four corners, the
    diagonal start/end and random interior blocks (clipped to the matrix)."""
    g = np.random.Generator(np.random.PCG64(seed))
    starts = [(0, 0), (max(0, m - bs), max(0, n - bs)), (0, max(0, n - bs)), (max(0, m - bs), 0)]
    d = min(m, n)
    starts.append((max(0, d // 2 - bs // 2), max(0, d // 2 - bs // 2)))
    while len(starts) < count:
        starts.append((int(g.integers(0, max(1, m - bs + 1))), int(g.integers(0, max(1, n - bs + 1)))))
    rows, cols = [], []
    for (r0, c0) in starts:
        rr, cc = np.meshgrid(np.arange(r0, min(m, r0 + bs)), np.arange(c0, min(n, c0 + bs)),
                             indexing="ij")
        rows.append(rr.ravel())
        cols.append(cc.ravel())
    return np.concatenate(rows), np.concatenate(cols)


def check_against_exact(c, got, rows=None, cols=None):
    """max err/bound of ``got`` (full m x n result) against the exact tier at
    the given entries (all entries when rows is None)."""
    if rows is None:
        rr, cc = np.meshgrid(np.arange(c.m), np.arange(c.n), indexing="ij")
        rows, cols = rr.ravel(), cc.ravel()
    ex = oracle.exact_gemm_entries(c.transa, c.transb, c.k, c.alpha, c.A, c.B, c.beta, c.C,
                                   rows, cols)
    bound = gemm_bound_entries(c.transa, c.transb, c.m, c.n, c.k, c.alpha, c.A, c.B, c.beta,
                               c.C, rows, cols)
    g = (got[0][rows, cols], got[1][rows, cols])
    assert is_normalised(*g)
    return err_over_bound(g, ex, bound)


def check_against_scalar(c, got, rows, cols):
    """max err/bound against the oracle's scalar dd tier (itself within the
    bound of the exact result, so the comparison allows twice the bound)."""
    ref = oracle.dd_gemm_entries(c.transa, c.transb, c.k, c.alpha, c.A, c.B, c.beta, c.C, rows,
                                 cols)
    bound = gemm_bound_entries(c.transa, c.transb, c.m, c.n, c.k, c.alpha, c.A, c.B, c.beta,
                               c.C, rows, cols)
    g = (got[0][rows, cols], got[1][rows, cols])
    return err_over_bound(g, ref, 2.0 * bound)
