"""Grouped dd Rgemm: descriptors, the tile-shape autotuner, graph capture.

``mp_dd_Rgemm_grouped_prepare`` / ``mp_dd_Rgemm_grouped_run`` (C ABI) run
thousands of independent dd GEMMs in one persistent kernel launch.  This
module builds the descriptor array from torch tensors, chooses each
problem's output tile shape from a table measured on the device by
``autotune`` (cached as JSON), and wraps the run in a CUDA graph so that the
whole group is one graph launch.  Every entry of every problem is bitwise
equal to what ``mp_dd_Rgemm`` gives for that problem alone, whatever the
shapes, so the tuner changes speed only.
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import numpy as np
import torch

from . import _abi, _check, _dd, _ld, _sync_stream, lib, workspace
from ._abi import MpDDGemmDesc

SHAPES = {0: (32, 32), 1: (64, 32), 2: (32, 64), 3: (16, 16)}


def desc(transa, transb, m, n, k, alpha, A, B, beta, C, tile=-1, uplo=0,
         info=None) -> MpDDGemmDesc:
    """Descriptor of one problem on column-major dd tensors (hi, lo)."""
    d = MpDDGemmDesc()
    d.m, d.n, d.k = int(m), int(n), int(k)
    d.alpha, d.beta = _dd(alpha), _dd(beta)
    d.a_hi, d.a_lo, d.lda = A[0].data_ptr(), A[1].data_ptr(), _ld(A[0])
    d.b_hi, d.b_lo, d.ldb = B[0].data_ptr(), B[1].data_ptr(), _ld(B[0])
    d.c_hi, d.c_lo, d.ldc = C[0].data_ptr(), C[1].data_ptr(), _ld(C[0])
    d.transa = 1 if transa.upper() in "TC" else 0
    d.transb = 1 if transb.upper() in "TC" else 0
    d.tile = int(tile)
    d.uplo = int(uplo)
    d.info = None if info is None else info.data_ptr()
    return d


def descs_array(descs) -> ctypes.Array:
    arr = (MpDDGemmDesc * len(descs))()
    for i, d in enumerate(descs):
        arr[i] = d
    return arr


def mp_dd_Rgemm_grouped_workspace(count, descs) -> int:
    return int(lib().mp_dd_Rgemm_grouped_workspace(count, descs))


def mp_dd_Rgemm_grouped_prepare(count, descs, ws, nbytes, check=True):
    _sync_stream()
    rc = lib().mp_dd_Rgemm_grouped_prepare(count, descs, ws.data_ptr(), nbytes)
    return _check(rc, "mp_dd_Rgemm_grouped_prepare") if check else rc


def mp_dd_Rgemm_grouped_run(ws, check=True):
    _sync_stream()
    rc = lib().mp_dd_Rgemm_grouped_run(ws.data_ptr())
    return _check(rc, "mp_dd_Rgemm_grouped_run") if check else rc


# ----------------------------------------------------------------------------
# autotuner
# ----------------------------------------------------------------------------

def size_class(x: int) -> int:
    """Power-of-two class of a dimension: 16 -> 4, 17..32 -> 5, ..., 257..512 -> 9."""
    return max(4, min(9, int(math.ceil(math.log2(max(int(x), 1))))))


def _default_cache_path() -> str:
    return os.environ.get("MPDD_TUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                       "_build", "grouped_tiles.json"))


def autotune(shapes=(0, 1, 2, 3), per_class: int = 48, k: int = 128, reps: int = 3,
             seed: int = 7, cache_path: str | None = None, force: bool = False) -> dict:
    """Measure, for every (m class, n class) of 16..512, which tile shape runs a
    group of ``per_class`` problems of that class fastest, and return the
    table {"mc,nc": shape}.  Problems use sizes drawn uniformly inside the
    class and the given k; timing is CUDA events around the group run, best
    of ``reps``.  The table is cached per device name."""
    path = cache_path or _default_cache_path()
    devname = torch.cuda.get_device_name()
    if not force and os.path.exists(path):
        try:
            cached = json.load(open(path))
            if cached.get("device") == devname and cached.get("k") == k:
                return cached["table"]
        except (OSError, ValueError, KeyError):
            pass
    g = np.random.Generator(np.random.PCG64(seed))
    table = {}
    timings = {}
    for mc in range(4, 10):
        for nc in range(4, 10):
            lo_m, hi_m = 2 ** (mc - 1) + 1 if mc > 4 else 1, 2 ** mc
            lo_n, hi_n = 2 ** (nc - 1) + 1 if nc > 4 else 1, 2 ** nc
            ms = g.integers(lo_m, hi_m + 1, per_class)
            ns = g.integers(lo_n, hi_n + 1, per_class)
            mats = []
            for m_, n_ in zip(ms, ns):
                A = tuple(torch.rand(int(k), int(m_), dtype=torch.float64, device="cuda").t()
                          for _ in range(2))
                B = tuple(torch.rand(int(n_), int(k), dtype=torch.float64, device="cuda").t()
                          for _ in range(2))
                C = tuple(torch.zeros(int(n_), int(m_), dtype=torch.float64, device="cuda").t()
                          for _ in range(2))
                mats.append((int(m_), int(n_), A, B, C))
            best, best_ms = None, None
            for s in shapes:
                ds = descs_array([desc("N", "N", m_, n_, k, (1.0, 0.0), A, B, (0.0, 0.0), C, s)
                                  for (m_, n_, A, B, C) in mats])
                need = mp_dd_Rgemm_grouped_workspace(len(ds), ds)
                ws = workspace(need)
                mp_dd_Rgemm_grouped_prepare(len(ds), ds, ws, ws.numel())
                mp_dd_Rgemm_grouped_run(ws)
                torch.cuda.synchronize()
                t = []
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    mp_dd_Rgemm_grouped_run(ws)
                    e1.record()
                    torch.cuda.synchronize()
                    t.append(e0.elapsed_time(e1))
                ms_ = min(t)
                timings[f"{mc},{nc},{s}"] = ms_
                if best_ms is None or ms_ < best_ms:
                    best, best_ms = s, ms_
            table[f"{mc},{nc}"] = int(best)
            del mats
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump({"device": devname, "k": k, "table": table, "timings_ms": timings}, f,
                  indent=1)
    return table


def shape_for(table: dict | None, m: int, n: int) -> int:
    if not table:
        return -1
    return int(table.get(f"{size_class(m)},{size_class(n)}", -1))


# ----------------------------------------------------------------------------
# a prepared group, optionally replayed from a CUDA graph
# ----------------------------------------------------------------------------

class GroupedGemm:
    """A group of dd Rgemm problems on column-major dd tensors.

    ``problems`` is a list of (transa, transb, m, n, k, alpha, A, B, beta, C).
    ``table`` maps size classes to tile shapes (``autotune``); None lets the
    library choose.  ``run()`` launches the group; ``capture()`` records the
    run in a CUDA graph and ``replay()`` launches the graph."""

    def __init__(self, problems, table: dict | None = None):
        self.descs = descs_array([
            desc(ta, tb, m, n, k, al, A, B, be, C, shape_for(table, m, n))
            for (ta, tb, m, n, k, al, A, B, be, C) in problems])
        self.count = len(problems)
        need = mp_dd_Rgemm_grouped_workspace(self.count, self.descs)
        self.ws = workspace(need)
        mp_dd_Rgemm_grouped_prepare(self.count, self.descs, self.ws, self.ws.numel())
        self.graph = None
        self.flops = sum(2.0 * m * n * k for (_, _, m, n, k, *_rest) in problems)

    def run(self):
        mp_dd_Rgemm_grouped_run(self.ws)

    def capture(self):
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run()           # warm-up outside the graph
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self.graph

    def replay(self):
        self.graph.replay()

    def padded_macs(self) -> float:
        """Multiply-adds the kernel issues: partial tiles are zero-padded, and
        k runs in groups of 4 steps."""
        tot = 0.0
        for d in self.descs:
            s = d.tile
            bm, bn = SHAPES.get(s, (64, 64))
            tot += math.ceil(d.m / bm) * bm * math.ceil(d.n / bn) * bn * (4 * math.ceil(d.k / 4))
        return tot
