"""Oracle for the double-double (dd) Rgemm / Rsyrk / Rpotrf / Rpotrs hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2109_13406_gb300``) and neither imports the
other; both take their inputs from the seeded generators in ``datagen.py``.

Contents
--------
* ``dd_oracle.c`` -- plain C, compiled here with gcc:
    - scalar dd arithmetic (TwoSum, FastTwoSum, FMA-based exact product, the
      accurate dd add, the full dd product, division, square root), after the
      manual's description of the dd format (Sec. 5: a dd is hi + lo of two
      binary64 numbers, arithmetic from Knuth's and Dekker's error-free
      transformations);
    - scalar dd Rgemm / Rsyrk / Rsyr2k / Rsymm / Rtrsm / Rpotrf / Rpotrs /
      Rgetrf / Rgetrs: plain loops with the argument semantics of the BLAS /
      LAPACK routine of the same name (Sec. 7.3 maps every MPBLAS argument
      list onto the BLAS one);
    - an exact tier: alpha*op(A)*op(B) + beta*C evaluated exactly in a
      superaccumulator and rounded once to the nearest dd.
* ``fraction_ref.py`` -- the same definitions in pure Python ``fractions``,
  independent of the C code, for tiny pins.

Parity status of each function (how it is pinned, see ``tests/test_oracle.py``):
scalar ops -- against Fraction arithmetic and their error bounds; Rgemm /
Rsyrk -- the manual's worked examples (Sec. 7.3), the exact tier, Fraction
brute force, closed forms and integer special cases; exact tier -- Fraction
brute force and known exact sums; Rpotrf / Rpotrs -- exact integer factors,
LAPACK test ratios (Sec. 8.2) and numpy's binary64 Cholesky on well
conditioned matrices; Rtrsm -- exact integer solutions for all sixteen
side/uplo/trans/diag variants, Fraction solves of tiny systems, the
componentwise backward-error bound of substitution evaluated by the exact
tier, and scipy's binary64 triangular solve; Rsyr2k / Rsymm -- the exact
tier on the equivalent Rgemm of concatenated or symmetrised operands,
integer inputs against binary64 matmul and Fraction brute force; Rgetrf / Rgetrs -- exact
recovery of a dyadic L U factorisation with a known permutation, LAPACK test
ratios with exact-tier residuals, scipy's binary64 LU (same pivots) and
LAPACK's info on singular input.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libddoracle.so")
_lib = None
_lock = threading.Lock()

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)


def compile_source(src: str, out: str) -> str:
    """Compile one C source of the oracle into a shared library.

    Flags: ``-O2 -ffp-contract=off`` (no silent FMA contraction, which would
    break TwoSum) and no fast-math; OpenMP when the compiler supports it."""
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11", "-fPIC",
            "-shared", src, "-o", out + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    """Compile ``dd_oracle.c`` into ``oracle/_build/libddoracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # DD_ORACLE_LIB names another build of dd_oracle.c; the planted-
            # mistake tests use it to load a deliberately broken copy.
            path = os.environ.get("DD_ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            c, i64, d = ctypes.c_char, ctypes.c_int64, ctypes.c_double
            L.oracle_two_sum.argtypes = [i64, _D, _D, _D, _D]
            L.oracle_two_prod.argtypes = [i64, _D, _D, _D, _D]
            for name in ("oracle_dd_add", "oracle_dd_mul", "oracle_dd_div"):
                getattr(L, name).argtypes = [i64, _D, _D, _D, _D, _D, _D]
            L.oracle_dd_sqrt.argtypes = [i64, _D, _D, _D, _D]
            L.oracle_dd_gemm.argtypes = [c, c, i64, i64, i64, d, d, _D, _D, i64, _D, _D, i64,
                                         d, d, _D, _D, i64]
            L.oracle_dd_gemm_entries.argtypes = [c, c, i64, d, d, _D, _D, i64, _D, _D, i64,
                                                 d, d, _D, _D, i64, i64, _I64, _I64, _D, _D]
            L.oracle_exact_gemm_entries.argtypes = L.oracle_dd_gemm_entries.argtypes
            L.oracle_dd_syrk.argtypes = [c, c, i64, i64, d, d, _D, _D, i64, d, d, _D, _D, i64]
            L.oracle_dd_potrf.argtypes = [c, i64, _D, _D, i64]
            L.oracle_dd_potrf.restype = i64
            L.oracle_dd_potrs.argtypes = [c, i64, i64, _D, _D, i64, _D, _D, i64]
            L.oracle_dd_trsm.argtypes = [c, c, c, c, i64, i64, d, d, _D, _D, i64, _D, _D, i64]
            L.oracle_dd_syr2k.argtypes = [c, c, i64, i64, d, d, _D, _D, i64, _D, _D, i64, d, d,
                                          _D, _D, i64]
            L.oracle_dd_getrf.argtypes = [i64, i64, _D, _D, i64, _I64]
            L.oracle_dd_getrf.restype = i64
            L.oracle_dd_getrs.argtypes = [c, i64, i64, _D, _D, i64, _I64, _D, _D, i64]
            L.oracle_dd_symm.argtypes = [c, c, i64, i64, d, d, _D, _D, i64, _D, _D, i64, d, d,
                                         _D, _D, i64]
            L.oracle_exact_sum.argtypes = [i64, _D, _D, _D]
            _P4 = ctypes.POINTER(_D)
            L.oracle_exact_qd_gemm_entries.argtypes = [c, c, i64, _D, _P4, i64, _P4, i64, _D,
                                                       _P4, i64, i64, _I64, _I64, _P4]
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_set_num_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def _f64(a) -> np.ndarray:
    """A float64 array in column-major (Fortran) order, without copying when possible."""
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _ch(s: str) -> ctypes.c_char:
    return ctypes.c_char(s.encode()[:1])


def _ld(a: np.ndarray) -> int:
    """Leading dimension of a column-major 2-D array (its row count)."""
    return max(1, a.shape[0])


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


# ----------------------------------------------------------------------------
# scalar dd layer (vectorised over arrays)
# ----------------------------------------------------------------------------

def two_sum(a, b):
    a, b = np.ascontiguousarray(a, np.float64), np.ascontiguousarray(b, np.float64)
    s, e = np.empty_like(a), np.empty_like(a)
    lib().oracle_two_sum(a.size, _p(a), _p(b), _p(s), _p(e))
    return s, e


def two_prod(a, b):
    a, b = np.ascontiguousarray(a, np.float64), np.ascontiguousarray(b, np.float64)
    p, e = np.empty_like(a), np.empty_like(a)
    lib().oracle_two_prod(a.size, _p(a), _p(b), _p(p), _p(e))
    return p, e


def _binop(name, a, b):
    ah, al = (np.ascontiguousarray(x, np.float64) for x in a)
    bh, bl = (np.ascontiguousarray(x, np.float64) for x in b)
    rh, rl = np.empty_like(ah), np.empty_like(ah)
    getattr(lib(), name)(ah.size, _p(ah), _p(al), _p(bh), _p(bl), _p(rh), _p(rl))
    return rh, rl


def dd_add(a, b):
    return _binop("oracle_dd_add", a, b)


def dd_mul(a, b):
    return _binop("oracle_dd_mul", a, b)


def dd_div(a, b):
    return _binop("oracle_dd_div", a, b)


def dd_sqrt(a):
    ah, al = (np.ascontiguousarray(x, np.float64) for x in a)
    rh, rl = np.empty_like(ah), np.empty_like(ah)
    lib().oracle_dd_sqrt(ah.size, _p(ah), _p(al), _p(rh), _p(rl))
    return rh, rl


# ----------------------------------------------------------------------------
# Rgemm / Rsyrk / Rpotrf / Rpotrs
# ----------------------------------------------------------------------------

def dd_gemm(transa, transb, alpha, A, B, beta, C, m=None, n=None, k=None):
    """Scalar dd Rgemm.  ``A``, ``B``, ``C`` are (hi, lo) pairs of column-major
    arrays whose row counts are the leading dimensions; ``alpha``/``beta`` are
    (hi, lo) tuples.  Returns a new (hi, lo) pair for C."""
    ah, al = _f64(A[0]), _f64(A[1])
    bh, bl = _f64(B[0]), _f64(B[1])
    ch, cl = _f64(C[0]).copy(order="F"), _f64(C[1]).copy(order="F")
    ta = transa.upper() in "TC"
    tb = transb.upper() in "TC"
    if m is None:
        m = ah.shape[1] if ta else ah.shape[0]
    if k is None:
        k = ah.shape[0] if ta else ah.shape[1]
    if n is None:
        n = bh.shape[0] if tb else bh.shape[1]
    lib().oracle_dd_gemm(_ch(transa), _ch(transb), m, n, k, alpha[0], alpha[1], _p(ah),
                         _p(al), _ld(ah), _p(bh), _p(bl), _ld(bh), beta[0], beta[1], _p(ch),
                         _p(cl), _ld(ch))
    return ch, cl


def _entries(fn, transa, transb, k, alpha, A, B, beta, C, rows, cols):
    ah, al = _f64(A[0]), _f64(A[1])
    bh, bl = _f64(B[0]), _f64(B[1])
    if C is None:
        ch = cl = np.zeros((1, 1), order="F")
    else:
        ch, cl = _f64(C[0]), _f64(C[1])
    rows = np.ascontiguousarray(rows, np.int64)
    cols = np.ascontiguousarray(cols, np.int64)
    oh, ol = np.empty(rows.size), np.empty(rows.size)
    fn(_ch(transa), _ch(transb), k, alpha[0], alpha[1], _p(ah), _p(al), _ld(ah), _p(bh),
       _p(bl), _ld(bh), beta[0], beta[1], _p(ch), _p(cl), _ld(ch), rows.size,
       rows.ctypes.data_as(_I64), cols.ctypes.data_as(_I64), _p(oh), _p(ol))
    return oh, ol


def dd_gemm_entries(transa, transb, k, alpha, A, B, beta, C, rows, cols):
    """Scalar dd Rgemm, only the entries (rows[q], cols[q])."""
    return _entries(lib().oracle_dd_gemm_entries, transa, transb, k, alpha, A, B, beta, C,
                    rows, cols)


def exact_gemm_entries(transa, transb, k, alpha, A, B, beta, C, rows, cols):
    """Exact alpha*op(A)*op(B) + beta*C at the given entries, rounded to the nearest dd."""
    return _entries(lib().oracle_exact_gemm_entries, transa, transb, k, alpha, A, B, beta, C,
                    rows, cols)


def dd_syrk(uplo, trans, alpha, A, beta, C, n=None, k=None):
    ah, al = _f64(A[0]), _f64(A[1])
    ch, cl = _f64(C[0]).copy(order="F"), _f64(C[1]).copy(order="F")
    t = trans.upper() in "TC"
    if n is None:
        n = ah.shape[1] if t else ah.shape[0]
    if k is None:
        k = ah.shape[0] if t else ah.shape[1]
    lib().oracle_dd_syrk(_ch(uplo), _ch(trans), n, k, alpha[0], alpha[1], _p(ah), _p(al),
                         _ld(ah), beta[0], beta[1], _p(ch), _p(cl), _ld(ch))
    return ch, cl


def dd_potrf(uplo, A, n=None):
    """Returns (factor_hi, factor_lo, info)."""
    ah, al = _f64(A[0]).copy(order="F"), _f64(A[1]).copy(order="F")
    if n is None:
        n = ah.shape[1]
    info = lib().oracle_dd_potrf(_ch(uplo), n, _p(ah), _p(al), _ld(ah))
    return ah, al, int(info)


def dd_potrs(uplo, F, B, n=None):
    fh, fl = _f64(F[0]), _f64(F[1])
    bh, bl = _f64(B[0]).copy(order="F"), _f64(B[1]).copy(order="F")
    if n is None:
        n = fh.shape[1]
    nrhs = bh.shape[1]
    lib().oracle_dd_potrs(_ch(uplo), n, nrhs, _p(fh), _p(fl), _ld(fh), _p(bh), _p(bl),
                          _ld(bh))
    return bh, bl


def dd_syr2k(uplo, trans, alpha, A, B, beta, C, n=None, k=None):
    """Rsyr2k (DSYR2K semantics): returns C (hi, lo); only the uplo triangle
    changes."""
    ah, al, bh_, bl_ = _f64(A[0]), _f64(A[1]), _f64(B[0]), _f64(B[1])
    ch, cl = _f64(C[0]).copy(order="F"), _f64(C[1]).copy(order="F")
    t = trans.upper() in "TC"
    n = (ah.shape[1] if t else ah.shape[0]) if n is None else n
    k = (ah.shape[0] if t else ah.shape[1]) if k is None else k
    lib().oracle_dd_syr2k(_ch(uplo), _ch(trans), n, k, float(alpha[0]), float(alpha[1]),
                          _p(ah), _p(al), _ld(ah), _p(bh_), _p(bl_), _ld(bh_),
                          float(beta[0]), float(beta[1]), _p(ch), _p(cl), _ld(ch))
    return ch, cl


def dd_symm(side, uplo, alpha, A, B, beta, C, m=None, n=None):
    """Rsymm (DSYMM semantics): returns C (hi, lo)."""
    ah, al, bh_, bl_ = _f64(A[0]), _f64(A[1]), _f64(B[0]), _f64(B[1])
    ch, cl = _f64(C[0]).copy(order="F"), _f64(C[1]).copy(order="F")
    m = ch.shape[0] if m is None else m
    n = ch.shape[1] if n is None else n
    lib().oracle_dd_symm(_ch(side), _ch(uplo), m, n, float(alpha[0]), float(alpha[1]),
                         _p(ah), _p(al), _ld(ah), _p(bh_), _p(bl_), _ld(bh_), float(beta[0]),
                         float(beta[1]), _p(ch), _p(cl), _ld(ch))
    return ch, cl


def dd_getrf(A, m=None, n=None):
    """Rgetrf (DGETRF semantics): returns (hi, lo, ipiv, info); ipiv one-based."""
    ah, al = _f64(A[0]).copy(order="F"), _f64(A[1]).copy(order="F")
    m = ah.shape[0] if m is None else m
    n = ah.shape[1] if n is None else n
    ipiv = np.zeros(max(1, min(m, n)), dtype=np.int64)
    info = lib().oracle_dd_getrf(m, n, _p(ah), _p(al), _ld(ah),
                                 ipiv.ctypes.data_as(_I64))
    return ah, al, ipiv[:min(m, n)], int(info)


def dd_getrs(trans, LU, ipiv, B, n=None):
    """Rgetrs (DGETRS semantics): X (hi, lo) with A X = B or A^T X = B."""
    ah, al = _f64(LU[0]), _f64(LU[1])
    bh, bl = _f64(B[0]).copy(order="F"), _f64(B[1]).copy(order="F")
    n = ah.shape[1] if n is None else n
    piv = np.ascontiguousarray(ipiv, dtype=np.int64)
    lib().oracle_dd_getrs(_ch(trans), n, bh.shape[1], _p(ah), _p(al), _ld(ah),
                          piv.ctypes.data_as(_I64), _p(bh), _p(bl), _ld(bh))
    return bh, bl


def dd_trsm(side, uplo, transa, diag, alpha, A, B, m=None, n=None):
    """Rtrsm (DTRSM semantics): returns X (hi, lo) with op(A) X = alpha B
    (side 'L') or X op(A) = alpha B (side 'R'); B is m x n."""
    ah, al = _f64(A[0]), _f64(A[1])
    bh, bl = _f64(B[0]).copy(order="F"), _f64(B[1]).copy(order="F")
    m = bh.shape[0] if m is None else m
    n = bh.shape[1] if n is None else n
    lib().oracle_dd_trsm(_ch(side), _ch(uplo), _ch(transa), _ch(diag), m, n,
                         float(alpha[0]), float(alpha[1]), _p(ah), _p(al), _ld(ah), _p(bh),
                         _p(bl), _ld(bh))
    return bh, bl


def _planes4(X):
    """Four float64 column-major planes and a C array of their pointers."""
    planes = [_f64(P) for P in X]
    arr = (_D * 4)(*[_p(P) for P in planes])
    return planes, arr


def exact_qd_gemm_entries(transa, transb, k, alpha, A, B, beta, C, rows, cols):
    """Selected entries of RN_qd(alpha op(A) op(B) + beta C), exactly: a tuple
    of four component arrays.  alpha, beta: 4-tuples; A, B, C: 4 planes each."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    count = rows.size
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    be = np.ascontiguousarray(beta, dtype=np.float64)
    pa, aa = _planes4(A)
    pb, ab = _planes4(B)
    if C is None:
        C = [np.zeros((1, 1), order="F")] * 4
    pc, ac = _planes4(C)
    out = [np.zeros(count) for _ in range(4)]
    ao = (_D * 4)(*[_p(o) for o in out])
    lib().oracle_exact_qd_gemm_entries(_ch(transa), _ch(transb), k, _p(al), aa, _ld(pa[0]),
                                       ab, _ld(pb[0]), _p(be), ac, _ld(pc[0]), count,
                                       rows.ctypes.data_as(_I64), cols.ctypes.data_as(_I64),
                                       ao)
    return tuple(out)


def exact_sum(x):
    x = np.ascontiguousarray(x, np.float64)
    h, l = ctypes.c_double(), ctypes.c_double()
    lib().oracle_exact_sum(x.size, _p(x), ctypes.byref(h), ctypes.byref(l))
    return h.value, l.value
