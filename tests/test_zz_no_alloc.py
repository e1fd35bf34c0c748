"""The allocation-free sliced Rgemm (mp_dd_Rgemm_sliced_noalloc), GPU.

It serves callers that cannot hand the library a workspace or let it
allocate (the MPBLAS argument list has no workspace argument, and some host
programs own all device memory or must never reach cudaMalloc).  Its
scratch is a fixed array inside the library, shared by every call.  The
test makes calls in a row on different problems -- a small one, the largest
the array holds, then the small one again on an array that still holds the
larger call's contents -- and checks through the C ABI that each result is
bitwise equal to the workspace form mp_dd_Rgemm_sliced (the same kernels on
the same inputs) and so within the accuracy bound the other tests use, that
the repeated call reproduces the first bit for bit, that the first meets the
bound against the oracle's exact tier, and that the array's status word and
certificate read back through mp_dd_noalloc_report.  A problem too large for
the array is refused before any device work.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import datagen
from ddcheck import err_over_bound, gemm_bound
from gpucase import check_against_exact, dev, host

pytestmark = pytest.mark.gpu


def _noalloc(mp, c, A, B):
    lda, ldb, ldc = c.A[0].shape[0], c.B[0].shape[0], c.C[0].shape[0]
    C1 = dev(c.C)
    mp.mp_dd_Rgemm_sliced_noalloc(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, lda, B, ldb,
                                  c.beta, C1, ldc, 0)
    got = host(C1, c.m, c.n)
    return got, mp.mp_dd_noalloc_report()


def _workspace_form(mp, c, A, B):
    lda, ldb, ldc = c.A[0].shape[0], c.B[0].shape[0], c.C[0].shape[0]
    C2 = dev(c.C)
    ws = mp.workspace(mp.mp_dd_Rgemm_sliced_workspace(c.m, c.n, c.k, 0))
    mp.mp_dd_Rgemm_sliced(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, lda, B, ldb, c.beta,
                          C2, ldc, 0, ws, ws.numel())
    ref = host(C2, c.m, c.n)
    return ref, mp.mp_dd_split_report(ws)


def test_noalloc_matches_workspace_form_on_calls_in_a_row(cuda_lib):
    mp = cuda_lib
    first = datagen.gemm_case(900, "N", "T", 300, 200, 250, pad=2)
    second = datagen.gemm_case(901, "T", "N", 512, 512, 512)   # the largest default size
    results = []
    for c in (first, second, first):
        A, B = dev(c.A), dev(c.B)
        got, rep = _noalloc(mp, c, A, B)
        ref, rep_ws = _workspace_form(mp, c, A, B)
        assert rep["status"] == 0 and rep_ws["status"] == 0
        assert rep["width_bits"] == rep_ws["width_bits"] == 112
        assert rep["dmin"] == rep_ws["dmin"] and rep["max_err_est"] <= 1.0
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        bound = gemm_bound(c.transa, c.transb, c.m, c.n, c.k, c.alpha, c.A, c.B, c.beta, c.C)
        assert err_over_bound(got, ref, bound) <= 1.0
        assert np.isfinite(got[0]).all()
        results.append(got)
    # the repeat after the larger problem: the shared array's leftovers do not matter
    assert np.array_equal(results[0][0], results[2][0])
    assert np.array_equal(results[0][1], results[2][1])
    assert check_against_exact(first, results[0]) <= 1.0


def test_noalloc_rejects_problems_beyond_the_scratch_array(cuda_lib):
    """Real 1024 x 1024 operands, so that a refusal that came too late would
    show up as a wrong result, not as an access outside the buffers."""
    mp = cuda_lib
    assert mp.mp_dd_Rgemm_sliced_workspace(1024, 1024, 1024, 0) > mp.NOALLOC_SCRATCH_BYTES
    c = datagen.gemm_case(902, "N", "N", 1024, 1024, 1024)
    A, B, C = dev(c.A), dev(c.B), dev(c.C)
    rc = mp.mp_dd_Rgemm_sliced_noalloc("N", "N", 1024, 1024, 1024, (1.0, 0.0), A, 1024, B,
                                       1024, (0.0, 0.0), C, 1024, 0, check=False)
    assert rc == 2002 and "scratch" in mp.mp_dd_last_error()
    torch.cuda.synchronize()
    got = host(C)
    assert np.array_equal(got[0], c.C[0]) and np.array_equal(got[1], c.C[1])
