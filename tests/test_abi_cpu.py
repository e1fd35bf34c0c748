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


def test_header_and_library_serve_a_plain_c_program(mp, tmp_path):
    """The boundary is a C ABI: a C99 program that includes only mpdd.h
    compiles warning-free, links against libmpdd.so and gets DGEMM / DSYRK
    argument errors and messages back without a GPU."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_mpdd.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "mpdd.h"
int main(void) {
    mp_dd one = {1.0, 0.0};
    mp_dd_cmat A = {0, 0};
    mp_dd_mat C = {0, 0};
    if (mp_dd_Rgemm("X", "N", 2, 2, 2, one, A, 2, A, 2, one, C, 2) != -1) return 1;
    if (strstr(mp_dd_last_error(), "transa") == NULL) return 2;
    if (mp_dd_Rsyrk("U", "N", -1, 2, one, A, 2, one, C, 2) != -3) return 3;
    if (mp_dd_Rgemm("N", "N", 0, 2, 2, one, A, 2, A, 2, one, C, 2) != 0) return 4;
    if (mp_dd_version() <= 0) return 5;
    printf("ok\n");
    return 0;
}
''')
    exe = tmp_path / "use_mpdd"
    pkg = os.path.join(ROOT, "paper_2109_13406_gb300")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", pkg, "-lmpdd", f"-Wl,-rpath,{pkg}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
