"""The allocation-free sliced Rgemm (mp_dd_Rgemm_sliced_noalloc), GPU.

It serves callers that cannot hand the library a workspace or let it
allocate (the MPBLAS argument list has no workspace argument, and some host
programs own all device memory or must never reach cudaMalloc).  Its
scratch is a fixed array inside the library, shared by every call, so the
test makes two calls in a row on different problems and checks each
against the workspace form mp_dd_Rgemm_sliced, through the C ABI, within
the accuracy bound the other tests use.  It also checks that a problem too
large for the array is refused before any device work.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import datagen
from ddcheck import err_over_bound, gemm_bound
from gpucase import dev, host

pytestmark = pytest.mark.gpu


def _both(mp, c):
    """Run case c through the no-allocation form and the workspace form."""
    A, B = dev(c.A), dev(c.B)
    lda, ldb, ldc = c.A[0].shape[0], c.B[0].shape[0], c.C[0].shape[0]
    C1 = dev(c.C)
    mp.mp_dd_Rgemm_sliced_noalloc(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, lda, B, ldb,
                                  c.beta, C1, ldc, 0)
    got = host(C1, c.m, c.n)
    C2 = dev(c.C)
    ws = mp.workspace(mp.mp_dd_Rgemm_sliced_workspace(c.m, c.n, c.k, 0))
    mp.mp_dd_Rgemm_sliced(c.transa, c.transb, c.m, c.n, c.k, c.alpha, A, lda, B, ldb, c.beta,
                          C2, ldc, 0, ws, ws.numel())
    ref = host(C2, c.m, c.n)
    return got, ref


def test_noalloc_matches_workspace_form_on_two_calls_in_a_row(cuda_lib):
    first = datagen.gemm_case(900, "N", "T", 300, 200, 250, pad=2)
    second = datagen.gemm_case(901, "T", "N", 512, 512, 512)   # the largest default size
    for c in (first, second):
        got, ref = _both(cuda_lib, c)
        bound = gemm_bound(c.transa, c.transb, c.m, c.n, c.k, c.alpha, c.A, c.B, c.beta, c.C)
        assert err_over_bound(got, ref, bound) <= 1.0
        assert np.isfinite(got[0]).all()


def test_noalloc_rejects_problems_beyond_the_scratch_array(cuda_lib):
    assert cuda_lib.mp_dd_Rgemm_sliced_workspace(1024, 1024, 1024, 0) > \
        cuda_lib.NOALLOC_SCRATCH_BYTES
    c = datagen.gemm_case(902, "N", "N", 4, 4, 4)
    A, B, C = dev(c.A), dev(c.B), dev(c.C)
    rc = cuda_lib.mp_dd_Rgemm_sliced_noalloc("N", "N", 1024, 1024, 1024, (1.0, 0.0), A, 1024,
                                             B, 1024, (0.0, 0.0), C, 1024, 0, check=False)
    assert rc == 2002 and "scratch" in cuda_lib.mp_dd_last_error()
    torch.cuda.synchronize()
