"""Grouped dd Rgemm (one persistent launch over many uneven problems), GPU.

Every problem's result must be bitwise equal to mp_dd_Rgemm on that problem
alone, for every tile shape (the per-entry operation order does not depend
on the tiling), including when the group is replayed from a CUDA graph; a
sample is also checked against the oracle's exact tier within the bound.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import datagen
import oracle
from ddcheck import err_over_bound, gemm_bound_entries
from gpucase import dev, host

pytestmark = pytest.mark.gpu


def make_group(seed, count, lo=1, hi=200):
    g = datagen.rng(seed)
    cases = []
    for i in range(count):
        m, n, k = (int(x) for x in g.integers(lo, hi + 1, 3))
        ta, tb = "NT"[int(g.integers(0, 2))], "NT"[int(g.integers(0, 2))]
        c = datagen.gemm_case(seed * 10000 + i, ta, tb, m, n, k, pad=int(g.integers(0, 3)))
        if i % 17 == 3:
            c.alpha, c.beta = (0.0, 0.0), (1.0, 0.0)        # BLAS quick return
        if i % 13 == 5:
            c.beta = (0.0, 0.0)
            c.C = (np.full_like(c.C[0], np.nan), np.full_like(c.C[1], np.nan))
        cases.append(c)
    return cases


def run_group(mp, cases, tile, use_graph=False):
    from paper_2109_13406_gb300 import grouped as gr

    devs = [(dev(c.A), dev(c.B), dev(c.C)) for c in cases]
    problems = [(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, B, c.beta, C)
                for c, (A, B, C) in zip(cases, devs)]
    table = None if tile is None else {f"{a},{b}": tile for a in range(4, 10)
                                        for b in range(4, 10)}
    G = gr.GroupedGemm(problems, table)
    if use_graph:
        G.capture()   # the capture's warm-up run computes once ...
        for (_, _, C), c in zip(devs, cases):   # ... so restore C and replay
            C[0].copy_(mp.to_device(c.C[0]))
            C[1].copy_(mp.to_device(c.C[1]))
        G.replay()
    else:
        G.run()
    torch.cuda.synchronize()
    return [host(C, c.m, c.n) for c, (_, _, C) in zip(cases, devs)]


def per_problem(mp, cases):
    out = []
    for c in cases:
        A, B, C = dev(c.A), dev(c.B), dev(c.C)
        mp.mp_dd_Rgemm(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, c.A[0].shape[0], B,
                       c.B[0].shape[0], c.beta, C, c.C[0].shape[0])
        out.append(host(C, c.m, c.n))
    return out


def same(a, b):
    return all(np.array_equal(x[0], y[0], equal_nan=True) and
               np.array_equal(x[1], y[1], equal_nan=True) for x, y in zip(a, b))


@pytest.mark.parametrize("tile", [None, 0, 1, 2, 3])
def test_grouped_bitwise_equals_per_problem(cuda_lib, tile):
    cases = make_group(11, 60)
    assert same(run_group(cuda_lib, cases, tile), per_problem(cuda_lib, cases))


def test_grouped_graph_replay_bitwise(cuda_lib):
    cases = make_group(12, 40)
    assert same(run_group(cuda_lib, cases, None, use_graph=True), per_problem(cuda_lib, cases))


def test_grouped_against_exact_tier(cuda_lib):
    cases = make_group(13, 12, lo=16, hi=120)
    got = run_group(cuda_lib, cases, None)
    for c, r in zip(cases, got):
        if c.alpha == (0.0, 0.0):
            continue
        g = datagen.rng(1)
        rows = g.integers(0, c.m, 40)
        cols = g.integers(0, c.n, 40)
        ex = oracle.exact_gemm_entries(c.transa, c.transb, c.k, c.alpha, c.A, c.B, c.beta,
                                       c.C, rows, cols)
        b = gemm_bound_entries(c.transa, c.transb, c.m, c.n, c.k, c.alpha, c.A, c.B, c.beta,
                               c.C, rows, cols)
        assert err_over_bound((r[0][rows, cols], r[1][rows, cols]), ex, b) <= 1.0


def test_grouped_descriptor_errors(cuda_lib):
    from paper_2109_13406_gb300 import grouped as gr

    c = datagen.gemm_case(14, "N", "N", 20, 20, 20)
    A, B, C = dev(c.A), dev(c.B), dev(c.C)
    d = gr.desc("N", "N", 20, 20, 20, (1.0, 0.0), A, B, (0.0, 0.0), C)
    d.lda = 3
    arr = gr.descs_array([d])
    ws = cuda_lib.workspace(1 << 16)
    assert gr.mp_dd_Rgemm_grouped_prepare(1, arr, ws, ws.numel(), check=False) == -2
    assert "descriptor 0" in cuda_lib.mp_dd_last_error()
    d.lda, d.transa = 20, 7
    arr = gr.descs_array([d])
    assert gr.mp_dd_Rgemm_grouped_prepare(1, arr, ws, ws.numel(), check=False) == -2
    d.transa = 0
    arr = gr.descs_array([d])
    assert gr.mp_dd_Rgemm_grouped_prepare(1, arr, ws, 10, check=False) == 2003


def test_autotuner_table_is_valid(cuda_lib, tmp_path):
    from paper_2109_13406_gb300 import grouped as gr

    table = gr.autotune(per_class=4, k=32, reps=1, cache_path=str(tmp_path / "t.json"),
                        force=True)
    assert len(table) == 36 and set(table.values()) <= {0, 1, 2, 3}
    again = gr.autotune(per_class=4, k=32, reps=1, cache_path=str(tmp_path / "t.json"))
    assert again == table   # served from the cache
