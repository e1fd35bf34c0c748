"""ctypes declarations of the C ABI in ``include/mpdd.h`` (argument marshalling only).

Every function of the header is bound here under its own name with its C
argument types; nothing here computes.  ``load()`` fails loudly when the
compiled library is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmpdd.so")


class MpDD(ctypes.Structure):
    """``mp_dd``: dd scalar hi + lo, passed by value."""
    _fields_ = [("hi", ctypes.c_double), ("lo", ctypes.c_double)]


class MpDDCMat(ctypes.Structure):
    """``mp_dd_cmat``: read-only hi/lo plane pointers."""
    _fields_ = [("hi", ctypes.c_void_p), ("lo", ctypes.c_void_p)]


class MpDDMat(ctypes.Structure):
    """``mp_dd_mat``: writable hi/lo plane pointers."""
    _fields_ = [("hi", ctypes.c_void_p), ("lo", ctypes.c_void_p)]


class MpDDGemmDesc(ctypes.Structure):
    """``mp_dd_gemm_desc``: one problem of a grouped Rgemm (144 bytes)."""
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("alpha", MpDD), ("beta", MpDD),
                ("a_hi", ctypes.c_void_p), ("a_lo", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("b_hi", ctypes.c_void_p), ("b_lo", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("c_hi", ctypes.c_void_p), ("c_lo", ctypes.c_void_p), ("ldc", ctypes.c_int64),
                ("transa", ctypes.c_int32), ("transb", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("uplo", ctypes.c_int32),
                ("info", ctypes.c_void_p)]


assert ctypes.sizeof(MpDDGemmDesc) == 152


class MpDDPotrfDiagDesc(ctypes.Structure):
    """``mp_dd_potrf_diag_desc``."""
    _fields_ = [("a_hi", ctypes.c_void_p), ("a_lo", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("n", ctypes.c_int64), ("offset", ctypes.c_int64), ("info", ctypes.c_void_p),
                ("lower", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class MpQD(ctypes.Structure):
    """``mp_qd``: four components."""
    _fields_ = [("x", ctypes.c_double * 4)]


class MpQDCMat(ctypes.Structure):
    """``mp_qd_cmat``: four device plane pointers."""
    _fields_ = [("x", ctypes.c_void_p * 4)]


MpQDMat = MpQDCMat  # same layout (``mp_qd_mat``)


class MpDDTrsmDesc(ctypes.Structure):
    """``mp_dd_trsm_desc``."""
    _fields_ = [("u_hi", ctypes.c_void_p), ("u_lo", ctypes.c_void_p), ("ldu", ctypes.c_int64),
                ("b_hi", ctypes.c_void_p), ("b_lo", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("n", ctypes.c_int64), ("nrhs", ctypes.c_int64), ("info", ctypes.c_void_p),
                ("trans", ctypes.c_int32), ("lower_u", ctypes.c_int32),
                ("lower_b", ctypes.c_int32), ("unit_diag", ctypes.c_int32)]

class MpDDSplitInfo(ctypes.Structure):
    """``mp_dd_split_info``: outcome of a split-precision call's certificate."""
    _fields_ = [("status", ctypes.c_int), ("form", ctypes.c_int),
                ("width_bits", ctypes.c_int), ("count", ctypes.c_int),
                ("max_err_est", ctypes.c_double), ("dmin", ctypes.c_double)]


_c = ctypes.c_char_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_dp = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); the order and types follow include/mpdd.h
SIGNATURES = {
    "mp_dd_set_stream": (_int, [_vp]),
    "mp_dd_get_stream": (_vp, []),
    "mp_dd_last_error": (ctypes.c_char_p, []),
    "mp_dd_version": (_int, []),
    "mp_dd_Rgemm": (_int, [_c, _c, _i64, _i64, _i64, MpDD, MpDDCMat, _i64, MpDDCMat, _i64, MpDD,
                           MpDDMat, _i64]),
    "mp_dd_Rsyrk": (_int, [_c, _c, _i64, _i64, MpDD, MpDDCMat, _i64, MpDD, MpDDMat, _i64]),
    "mp_dd_Rgemm_host": (_int, [_c, _c, _i64, _i64, _i64, MpDD, MpDDCMat, _i64, MpDDCMat, _i64,
                                MpDD, MpDDMat, _i64]),
    "mp_dd_Rsyrk_host": (_int, [_c, _c, _i64, _i64, MpDD, MpDDCMat, _i64, MpDD, MpDDMat, _i64]),
    "mp_dd_peak_fp64": (_int, [_dp]),
    "mp_dd_set_plain_staging": (_int, [_int]),
    "mp_dd_set_band_pairs": (_int, [_int]),
    "mp_dd_peak_imma": (_int, [_dp]),
    "mp_dd_peak_ddmac": (_int, [_dp]),
    "mp_dd_elementwise": (_int, [_c, _i64, MpDDCMat, MpDDCMat, MpDDMat]),
    "mp_dd_Rgemm_sliced_workspace": (_sz, [_i64, _i64, _i64, _int]),
    "mp_dd_Rgemm_sliced": (_int, [_c, _c, _i64, _i64, _i64, MpDD, MpDDCMat, _i64, MpDDCMat, _i64,
                                  MpDD, MpDDMat, _i64, _int, _vp, _sz]),
    "mp_dd_Rgemm_sliced_noalloc": (_int, [_c, _c, _i64, _i64, _i64, MpDD, MpDDCMat, _i64,
                                          MpDDCMat, _i64, MpDD, MpDDMat, _i64, _int]),
    "mp_dd_sliced_layout": (_int, [_i64, _i64, _i64, _int, ctypes.POINTER(ctypes.c_size_t)]),
    "mp_dd_Rgemm_crt_workspace": (_sz, [_i64, _i64, _i64]),
    "mp_dd_Rgemm_crt": (_int, [_c, _c, _i64, _i64, _i64, MpDD, MpDDCMat, _i64, MpDDCMat, _i64,
                               MpDD, MpDDMat, _i64, _vp, _sz]),
    "mp_dd_crt_layout": (_int, [_i64, _i64, _i64, ctypes.POINTER(ctypes.c_size_t),
                                ctypes.POINTER(ctypes.c_int)]),
    "mp_dd_workspace_status": (_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "mp_dd_split_report": (_int, [_vp, ctypes.POINTER(MpDDSplitInfo)]),
    "mp_dd_noalloc_report": (_int, [ctypes.POINTER(MpDDSplitInfo)]),
    "mp_dd_magnitude_layout": (_int, [_int, _i64, _i64, _i64, _int,
                                      ctypes.POINTER(ctypes.c_size_t)]),
    "mp_dd_sliced_timing": (_int, [_int]),
    "mp_dd_Rpotrf": (_int, [_c, _i64, MpDDMat, _i64, _vp]),
    "mp_dd_Rpotrs": (_int, [_c, _i64, _i64, MpDDCMat, _i64, MpDDMat, _i64, _vp]),
    "mp_dd_potrf_diag_batch": (_int, [_i64, _vp]),
    "mp_dd_trsm_batch": (_int, [_i64, _vp, _i64]),
    "mp_dd_Rtrsm": (_int, [_c, _c, _c, _c, _i64, _i64, MpDD, MpDDCMat, _i64, MpDDMat, _i64]),
    "mp_dd_Rsyrk_crt_workspace": (_sz, [_i64, _i64]),
    "mp_dd_Rpotrf_crt_workspace": (_sz, [_i64]),
    "mp_dd_Rpotrf_crt": (_int, [_c, _i64, MpDDMat, _i64, _vp, _vp, _sz]),
    "mp_dd_Rsyrk_crt": (_int, [_c, _c, _i64, _i64, MpDD, MpDDCMat, _i64, MpDD, MpDDMat, _i64, _vp,
                               _sz]),
    "mp_qd_Rgemm": (_int, [_c, _c, _i64, _i64, _i64, MpQD, MpQDCMat, _i64, MpQDCMat, _i64, MpQD,
                           MpQDMat, _i64]),
    "mp_dd_Rgetrf": (_int, [_i64, _i64, MpDDMat, _i64, _vp, _vp]),
    "mp_dd_Rgetrs": (_int, [_c, _i64, _i64, MpDDCMat, _i64, _vp, MpDDMat, _i64]),
    "mp_dd_Rsyr2k": (_int, [_c, _c, _i64, _i64, MpDD, MpDDCMat, _i64, MpDDCMat, _i64, MpDD,
                            MpDDMat, _i64]),
    "mp_dd_Rsymm": (_int, [_c, _c, _i64, _i64, MpDD, MpDDCMat, _i64, MpDDCMat, _i64, MpDD,
                           MpDDMat, _i64]),
    "mp_dd_Rgemm_grouped_workspace": (_sz, [_i64, ctypes.POINTER(MpDDGemmDesc)]),
    "mp_dd_Rgemm_grouped_prepare": (_int, [_i64, ctypes.POINTER(MpDDGemmDesc), _vp, _sz]),
    "mp_dd_Rgemm_grouped_run": (_int, [_vp]),
    "mp_dd_sliced_phase_ms": (_int, [ctypes.POINTER(ctypes.c_float)]),
    "mp_dd_sliced_phase_log": (_int, [ctypes.POINTER(ctypes.c_float), _int,
                                      ctypes.POINTER(ctypes.c_int)]),
}

_lib = None


def load():
    """Load ``libmpdd.so`` and declare every entry point.  Raises if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"libmpdd.so not found at {LIB_PATH}: the CUDA library must be built "
                "(python -c 'import __graft_entry__ as g; g.build()'); there is no "
                "fallback implementation")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
