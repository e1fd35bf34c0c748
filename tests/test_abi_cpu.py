"""The C ABI without a GPU: the library builds and loads, exports every
symbol the header declares, and rejects illegal arguments with the BLAS
argument numbering (the xerbla codes the manual's MPBLAS tests compare,
Sec. 8.1) before touching the device."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mp():
    import __graft_entry__

    __graft_entry__._build_module().build()
    import paper_2109_13406_gb300 as mp

    return mp


def header_functions():
    txt = open(os.path.join(ROOT, "include", "mpdd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mp_(?:dd|qd)_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(mp):
    names = header_functions()
    assert "mp_dd_Rgemm" in names and "mp_dd_Rsyrk" in names
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2109_13406_gb300", "libmpdd.so"))
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2109_13406_gb300 import _abi

    assert sorted(_abi.SIGNATURES) == names, "binding and header disagree"


def test_library_is_built_for_sm_103a_only():
    src = open(os.path.join(ROOT, "paper_2109_13406_gb300", "build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in src


def test_rgemm_illegal_arguments(mp):
    z = np.zeros((4, 4))
    A = (z, z)

    def call(ta="N", tb="N", m=2, n=2, k=2, lda=4, ldb=4, ldc=4, a=A, b=A, c=A):
        return mp.mp_dd_Rgemm(ta, tb, m, n, k, (1.0, 0.0), a, lda, b, ldb, (0.0, 0.0), c, ldc,
                              check=False)

    assert call(ta="X") == -1
    assert call(tb="q") == -2
    assert call(m=-1) == -3
    assert call(n=-1) == -4
    assert call(k=-1) == -5
    assert call(a=(None, None)) == -7
    assert call(m=5, lda=4) == -8
    assert call(ta="T", k=5, lda=4) == -8
    assert call(k=5, ldb=4) == -10
    assert call(tb="t", n=5, ldb=4, ldc=5) == -10
    assert call(b=(None, None)) == -9
    assert call(c=(None, None)) == -12
    assert call(m=5, lda=5, ldc=4) == -13
    assert "ldc" in mp.mp_dd_last_error()
    # checks come in DGEMM order: transa before m
    assert call(ta="X", m=-1) == -1
    # quick returns never touch the device
    assert call(m=0) == 0 and call(n=0) == 0
    assert mp.mp_dd_Rgemm("N", "N", 2, 2, 2, (0.0, 0.0), (None, None), 4, (None, None), 4,
                          (1.0, 0.0), A, 4, check=False) == 0
    assert mp.mp_dd_Rgemm("n", "c", 2, 2, 0, (1.0, 0.0), (None, None), 4, (None, None), 4,
                          (1.0, 0.0), A, 4, check=False) == 0


def test_rsyrk_illegal_arguments(mp):
    z = np.zeros((4, 4))
    A = (z, z)

    def call(uplo="U", trans="N", n=2, k=2, lda=4, ldc=4, a=A, c=A):
        return mp.mp_dd_Rsyrk(uplo, trans, n, k, (1.0, 0.0), a, lda, (0.0, 0.0), c, ldc,
                              check=False)

    assert call(uplo="X") == -1
    assert call(trans="Z") == -2
    assert call(n=-1) == -3
    assert call(k=-1) == -4
    assert call(a=(None, None)) == -6
    assert call(n=5, lda=4, ldc=5) == -7
    assert call(trans="T", k=5, lda=4) == -7
    assert call(c=(None, None)) == -9
    assert call(n=5, lda=5, ldc=4) == -10
    assert call(n=0) == 0


def test_host_variants_check_arguments(mp):
    z = np.zeros((4, 4))
    A = (z, z)
    assert mp.mp_dd_Rgemm_host("N", "N", 2, 2, 2, (1.0, 0.0), A, 1, A, 4, (0.0, 0.0), A, 4,
                               check=False) == -8
    assert mp.mp_dd_Rsyrk_host("U", "N", 2, 2, (1.0, 0.0), A, 4, (0.0, 0.0), A, 1,
                               check=False) == -10
