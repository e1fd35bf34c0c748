"""The server's per-request operation lists, checked on the CPU.

A request's work is a list of scheduler steps; inside a step the operations
run as launches in a fixed order: the tensor-core products (in list order),
then one grouped Rgemm launch, one batched diagonal factorisation and one
batched triangular solve, the operations of each batch at the same time.
This test runs the lists that ``SpdServer._plan`` builds with plain binary64
numpy arithmetic and exactly those semantics -- each batch reads the state
as it was when the batch began and writes afterwards, and two operations of
one batch may not write the same entries -- for every combination of group
size (rank-64 right-looking updates, or groups of 4 blocks with row-block
and depth-256 updates), FP64 or residue-form updates, and ragged orders.  A
list whose order or regions were wrong would not solve F X = B.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch


def _mat(T):
    return T.numpy()


def _op(M, t):
    return M.T if t in "TC" else M


def _gemm(args):
    ta, tb, m, n, k, al, A, B, be, C, uplo = args
    a, b, c = _op(_mat(A[0]), ta), _op(_mat(B[0]), tb), _mat(C[0])
    new = al[0] * (a[:m, :k] @ b[:k, :n]) + (be[0] * c[:m, :n] if be[0] != 0 else 0.0)
    mask = np.ones((m, n), bool)
    if uplo == 1:
        mask = np.triu(mask)
    elif uplo == 2:
        mask = np.tril(mask)
    return c, mask, np.where(mask, new, c[:m, :n])


def _diag(args):
    P, b, _ = args
    p = _mat(P[0])
    u = np.linalg.cholesky(np.triu(p[:b, :b]) + np.triu(p[:b, :b], 1).T).T
    mask = np.triu(np.ones((b, b), bool))
    return p, mask, np.where(mask, u, p[:b, :b])


def _trsm(args):
    U, Bm, b, cols, trans = args
    u, x = np.triu(_mat(U[0])[:b, :b]), _mat(Bm[0])
    sol = np.linalg.solve(u.T if trans else u, x[:b, :cols])
    return x, np.ones((b, cols), bool), sol


def _crt(args):
    P, Ct, rest, k = args
    p, c = _mat(P[0]), _mat(Ct[0])
    mask = np.triu(np.ones((rest, rest), bool))
    return c, mask, np.where(mask, c[:rest, :rest] - p[:k, :rest].T @ p[:k, :rest], c[:rest, :rest])


def _crt_gemm(args):
    Ut, Pr, Cr, b, cols, k = args
    u, p, c = _mat(Ut[0]), _mat(Pr[0]), _mat(Cr[0])
    return c, np.ones((b, cols), bool), c[:b, :cols] - u[:k, :b].T @ p[:k, :cols]


def _sliced(args):
    G, F = args
    g, f = _mat(G[0]), _mat(F[0])
    n = f.shape[0]
    mask = np.triu(np.ones((n, n), bool))
    return f, mask, np.where(mask, g @ g.T, f)


KERNELS = {"gemm": _gemm, "diag": _diag, "trsm": _trsm, "crt": _crt,
           "crt_gemm": _crt_gemm, "sliced": _sliced}


def _apply_batch(ops):
    """Every op computed from the state before the batch, then written; two
    ops of the batch must not write the same entry."""
    results = [KERNELS[kind](args) for kind, args in ops]
    written = {}
    for (kind, _), (target, mask, new) in zip(ops, results):
        base = target.__array_interface__["data"][0]
        rows, cols = mask.shape
        rr, cc = np.nonzero(mask)
        addr = base + (rr * target.strides[0] + cc * target.strides[1])
        for a in addr.tolist():
            assert a not in written, f"two {kind} operations of one batch write the same entry"
            written[a] = kind
        block = target[:rows, :cols]
        block[mask] = new[mask]


def run_plan(steps):
    for ops in steps:
        # tensor-core products at collection, one at a time in list order
        for kind, args in ops:
            if kind in ("sliced", "crt", "crt_gemm"):
                _apply_batch([(kind, args)])
        for kind in ("gemm", "diag", "trsm"):
            batch = [(k, a) for k, a in ops if k == kind]
            if batch:
                _apply_batch(batch)


@pytest.fixture(scope="module")
def built():
    """The package loads libmpdd.so on import: build it first (nvcc
    cross-compiles; nothing here touches a GPU)."""
    import __graft_entry__

    __graft_entry__._build_module().build()


@pytest.mark.parametrize("n", [64, 100, 300, 600])
@pytest.mark.parametrize("group", [1, 4])
@pytest.mark.parametrize("tensor_cores", [False, True])
def test_plan_solves_the_system(built, n, group, tensor_cores):
    from paper_2109_13406_gb300.server import Request, SpdServer

    g = np.random.Generator(np.random.PCG64(800 + n))
    nrhs = 4
    G = g.standard_normal((n, 2 * n)) / np.sqrt(2 * n) + np.hstack([np.eye(n), np.zeros((n, n))])
    B = g.standard_normal((n, nrhs))
    cpu = lambda a: torch.from_numpy(np.asfortranarray(a)).t().contiguous().t()
    zeros = lambda r, c: torch.zeros((c, r), dtype=torch.float64).t()
    r = Request(rid=0, n=n, G=None, B=None, nrhs_=nrhs)
    r.dev = {"G": (cpu(G), cpu(np.zeros_like(G))), "F": (zeros(n, n), zeros(n, n)),
             "X": (cpu(B), cpu(np.zeros_like(B))), "info": torch.zeros(1, dtype=torch.int64)}
    r.sliced_ws = 1 if tensor_cores else 0
    srv = SpdServer(group=group, crt_min_rest=64 if tensor_cores else 10 ** 9)
    steps = srv._plan(r)
    assert len(steps) <= 2 * ((n + 63) // 64) + 2
    kinds = {k for ops in steps for k, _ in ops}
    if tensor_cores and n - 64 >= 64:
        assert "crt" in kinds or "crt_gemm" in kinds
    if not tensor_cores:
        assert not kinds & {"sliced", "crt", "crt_gemm"}
    run_plan(steps)
    F = G @ G.T
    X = r.dev["X"][0].numpy()
    assert np.abs(F @ X - B).max() <= 1e-10 * np.abs(B).max()
