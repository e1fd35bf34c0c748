"""GB300-native double-double (dd) Rgemm / Rsyrk: the MPBLAS hot path.

A thin Python binding over the C ABI of ``libmpdd.so`` (``include/mpdd.h``).
Each ``mp_dd_*`` function here has the C name and argument list and only
marshals arguments: device pointers from torch tensors, dd scalars as
``(hi, lo)`` tuples, the current torch stream.  Every step of the
computation runs in the library's CUDA kernels; if the library is missing
the import fails.

Matrices follow the manual's convention (MPLAPACK 2.0.1, Sec. 7.3): column
major with a leading dimension.  A dd matrix is a pair ``(hi, lo)`` of
float64 tensors with strides ``(1, ld)`` (a column-major view); see
``dd_empty`` and ``to_device``.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from ._abi import MpDD, MpDDCMat, MpDDMat

__all__ = [
    "MpddError", "mp_dd_Rgemm", "mp_dd_Rsyrk", "mp_dd_Rgemm_host", "mp_dd_Rsyrk_host",
    "mp_dd_peak_fp64", "mp_dd_peak_imma", "mp_dd_peak_ddmac", "mp_dd_set_plain_staging", "mp_dd_set_band_pairs", "mp_dd_elementwise", "mp_dd_set_stream", "mp_dd_last_error",
    "mp_dd_Rgemm_sliced",
    "mp_dd_Rgemm_sliced_workspace", "mp_dd_Rgemm_sliced_noalloc", "mp_dd_sliced_layout",
    "mp_dd_Rgemm_crt", "mp_dd_Rgemm_crt_workspace", "mp_dd_Rsyrk_crt",
    "mp_dd_Rsyrk_crt_workspace", "mp_dd_crt_layout", "mp_dd_workspace_status",
    "mp_dd_split_report", "mp_dd_noalloc_report", "mp_dd_magnitude_layout",
    "mp_dd_Rtrsm", "mp_dd_Rsyr2k", "mp_dd_Rsymm", "mp_qd_Rgemm", "mp_dd_Rgetrf", "mp_dd_Rgetrs", "mp_dd_Rpotrf", "mp_dd_Rpotrf_crt",
    "mp_dd_Rpotrs", "Rgemm", "Rsyrk", "Rtrsm", "Rgemm_sliced",
    "workspace", "dd_empty", "to_device", "to_numpy", "lib",
]

_LIB = _abi.load()


class MpddError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def lib():
    return _LIB


def mp_dd_last_error() -> str:
    return (_LIB.mp_dd_last_error() or b"").decode()


def _check(rc: int, name: str) -> int:
    if rc != 0:
        raise MpddError(rc, f"{name}: {mp_dd_last_error()}")
    return rc


def mp_dd_set_stream(stream=None) -> None:
    """Use ``stream`` (a torch.cuda.Stream, a raw handle, or None for torch's
    current stream) for later calls from this thread."""
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
    _LIB.mp_dd_set_stream(ctypes.c_void_p(handle))


def _sync_stream():
    # calls run on torch's current stream; without a CUDA device (argument
    # checks only) the legacy default stream handle is passed
    if torch.cuda.is_available():
        mp_dd_set_stream(torch.cuda.current_stream())
    else:
        _LIB.mp_dd_set_stream(None)


def _flag(c: str) -> bytes:
    return c.encode()[:1]


def _dd(x) -> MpDD:
    if isinstance(x, MpDD):
        return x
    if isinstance(x, (int, float)):
        return MpDD(float(x), 0.0)
    return MpDD(float(x[0]), float(x[1]))


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _cm(pair) -> MpDDCMat:
    return MpDDCMat(_ptr(pair[0]), _ptr(pair[1]))


def _m(pair) -> MpDDMat:
    return MpDDMat(_ptr(pair[0]), _ptr(pair[1]))


# ----------------------------------------------------------------------------
# raw entry points: same names and argument lists as include/mpdd.h
# (matrix arguments are (hi, lo) pairs of tensors, arrays or raw addresses)
# ----------------------------------------------------------------------------

def mp_dd_Rgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rgemm(_flag(transa), _flag(transb), m, n, k, _dd(alpha), _cm(A), lda,
                          _cm(B), ldb, _dd(beta), _m(C), ldc)
    return _check(rc, "mp_dd_Rgemm") if check else rc


def mp_dd_Rsyrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rsyrk(_flag(uplo), _flag(trans), n, k, _dd(alpha), _cm(A), lda, _dd(beta),
                          _m(C), ldc)
    return _check(rc, "mp_dd_Rsyrk") if check else rc


def mp_dd_Rgemm_host(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rgemm_host(_flag(transa), _flag(transb), m, n, k, _dd(alpha), _cm(A), lda,
                               _cm(B), ldb, _dd(beta), _m(C), ldc)
    return _check(rc, "mp_dd_Rgemm_host") if check else rc


def mp_dd_Rsyrk_host(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rsyrk_host(_flag(uplo), _flag(trans), n, k, _dd(alpha), _cm(A), lda,
                               _dd(beta), _m(C), ldc)
    return _check(rc, "mp_dd_Rsyrk_host") if check else rc


def mp_dd_Rgemm_sliced_workspace(m, n, k, slices=0) -> int:
    return int(_LIB.mp_dd_Rgemm_sliced_workspace(m, n, k, slices))


def mp_dd_Rgemm_sliced(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices,
                       workspace, workspace_bytes, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rgemm_sliced(_flag(transa), _flag(transb), m, n, k, _dd(alpha), _cm(A), lda,
                                 _cm(B), ldb, _dd(beta), _m(C), ldc, slices, _ptr(workspace),
                                 workspace_bytes)
    return _check(rc, "mp_dd_Rgemm_sliced") if check else rc


def mp_dd_Rgemm_sliced_noalloc(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                               slices=0, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rgemm_sliced_noalloc(_flag(transa), _flag(transb), m, n, k, _dd(alpha),
                                         _cm(A), lda, _cm(B), ldb, _dd(beta), _m(C), ldc, slices)
    return _check(rc, "mp_dd_Rgemm_sliced_noalloc") if check else rc


NOALLOC_SCRATCH_BYTES = 32 << 20   # MP_DD_NOALLOC_SCRATCH_BYTES in include/mpdd.h


def mp_dd_Rgemm_crt_workspace(m, n, k) -> int:
    return int(_LIB.mp_dd_Rgemm_crt_workspace(m, n, k))


def mp_dd_Rgemm_crt(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, workspace,
                    workspace_bytes, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rgemm_crt(_flag(transa), _flag(transb), m, n, k, _dd(alpha), _cm(A), lda,
                              _cm(B), ldb, _dd(beta), _m(C), ldc, _ptr(workspace),
                              workspace_bytes)
    return _check(rc, "mp_dd_Rgemm_crt") if check else rc


def mp_dd_Rsyrk_crt_workspace(n, k) -> int:
    return int(_LIB.mp_dd_Rsyrk_crt_workspace(n, k))


def mp_dd_Rsyrk_crt(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, workspace, workspace_bytes,
                    check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rsyrk_crt(_flag(uplo), _flag(trans), n, k, _dd(alpha), _cm(A), lda,
                              _dd(beta), _m(C), ldc, _ptr(workspace), workspace_bytes)
    return _check(rc, "mp_dd_Rsyrk_crt") if check else rc


def mp_dd_crt_layout(m, n, k) -> dict:
    off = (ctypes.c_size_t * 48)()
    cnt = ctypes.c_int()
    _check(_LIB.mp_dd_crt_layout(m, n, k, off, ctypes.byref(cnt)), "mp_dd_crt_layout")
    keys = ["rowmax", "colmax", "residues_a", "residues_b", "products", "m_pad", "n_pad",
            "k_pad"]
    d = dict(zip(keys, [int(x) for x in off[:8]]))
    d["moduli"] = [int(x) for x in off[8:8 + cnt.value]]
    return d


def mp_dd_sliced_layout(m, n, k, slices=0) -> dict:
    off = (ctypes.c_size_t * 8)()
    _check(_LIB.mp_dd_sliced_layout(m, n, k, slices, off), "mp_dd_sliced_layout")
    keys = ["rowmax", "colmax", "digits_a", "digits_b", "bands", "m_pad", "n_pad", "k_pad"]
    return dict(zip(keys, [int(x) for x in off]))


def mp_dd_workspace_status(workspace) -> int:
    _sync_stream()
    st = ctypes.c_int()
    _check(_LIB.mp_dd_workspace_status(_ptr(workspace), ctypes.byref(st)),
           "mp_dd_workspace_status")
    return st.value


def _split_info(info) -> dict:
    return {"status": info.status, "form": info.form, "width_bits": info.width_bits,
            "count": info.count, "max_err_est": info.max_err_est, "dmin": info.dmin}


def mp_dd_split_report(workspace) -> dict:
    """The certificate of the last split-precision call on ``workspace``:
    status, form, width_bits (0: the plain kernel computed C), count,
    max_err_est (guaranteed bound of max err / bound) and dmin."""
    _sync_stream()
    info = _abi.MpDDSplitInfo()
    _check(_LIB.mp_dd_split_report(_ptr(workspace), ctypes.byref(info)), "mp_dd_split_report")
    return _split_info(info)


def mp_dd_noalloc_report() -> dict:
    """mp_dd_split_report for the built-in scratch array of the current device."""
    _sync_stream()
    info = _abi.MpDDSplitInfo()
    _check(_LIB.mp_dd_noalloc_report(ctypes.byref(info)), "mp_dd_noalloc_report")
    return _split_info(info)


def mp_dd_magnitude_layout(form, m, n, k, slices=0) -> dict:
    off = (ctypes.c_size_t * 2)()
    _check(_LIB.mp_dd_magnitude_layout(form, m, n, k, slices, off), "mp_dd_magnitude_layout")
    return {"magnitude_a": off[0], "magnitude_b": off[1]}


def mp_dd_sliced_timing(enable: bool) -> None:
    _LIB.mp_dd_sliced_timing(1 if enable else 0)


def mp_dd_sliced_phase_ms() -> list:
    """[scaling + slicing, band products, recombination] of the last timed call (ms)."""
    ms = (ctypes.c_float * 3)()
    _check(_LIB.mp_dd_sliced_phase_ms(ms), "mp_dd_sliced_phase_ms")
    return [float(x) for x in ms]


def mp_dd_sliced_phase_log(max_calls: int = 4096) -> list:
    """Per-call phase times [[scale_split, products, recombine], ...] of the
    calls timed since mp_dd_sliced_timing(True)."""
    ms = (ctypes.c_float * (3 * max_calls))()
    n = ctypes.c_int()
    _check(_LIB.mp_dd_sliced_phase_log(ms, max_calls, ctypes.byref(n)), "mp_dd_sliced_phase_log")
    k = min(n.value, max_calls)
    return [[ms[3 * c], ms[3 * c + 1], ms[3 * c + 2]] for c in range(k)]


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """A device byte buffer for the calls that take a workspace."""
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def Rgemm_sliced(transa, transb, alpha, A, B, beta, C, m=None, n=None, k=None, slices=0,
                 ws=None):
    """Sliced Rgemm on column-major dd tensors; allocates a workspace when
    none is given and returns it (reuse it for later calls)."""
    ta, tb = transa.upper() in "TC", transb.upper() in "TC"
    if m is None:
        m = A[0].shape[1] if ta else A[0].shape[0]
    if k is None:
        k = A[0].shape[0] if ta else A[0].shape[1]
    if n is None:
        n = B[0].shape[0] if tb else B[0].shape[1]
    need = mp_dd_Rgemm_sliced_workspace(m, n, k, slices)
    if ws is None or ws.numel() < need:
        ws = workspace(need, C[0].device)
    mp_dd_Rgemm_sliced(transa, transb, m, n, k, alpha, A, _ld(A[0]), B, _ld(B[0]), beta, C,
                       _ld(C[0]), slices, ws, ws.numel())
    return ws


def mp_dd_Rpotrf(uplo, n, A, lda, info, check=True):
    """info: a device int64 tensor (one element) that receives LAPACK's info."""
    _sync_stream()
    rc = _LIB.mp_dd_Rpotrf(_flag(uplo), n, _m(A), lda, _ptr(info))
    return _check(rc, "mp_dd_Rpotrf") if check else rc


def _qd(x) -> _abi.MpQD:
    v = _abi.MpQD()
    comps = list(x) + [0.0] * (4 - len(x))
    for t in range(4):
        v.x[t] = float(comps[t])
    return v


def _qm(planes) -> _abi.MpQDCMat:
    if len(planes) != 4:
        raise ValueError("a qd matrix is four planes")
    m = _abi.MpQDCMat()
    for t in range(4):
        m.x[t] = _ptr(planes[t])
    return m


def mp_qd_Rgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, check=True):
    """Quad-double Rgemm; alpha/beta 4-tuples, A/B/C four device planes each."""
    _sync_stream()
    rc = _LIB.mp_qd_Rgemm(_flag(transa), _flag(transb), m, n, k, _qd(alpha), _qm(A), lda,
                          _qm(B), ldb, _qd(beta), _qm(C), ldc)
    return _check(rc, "mp_qd_Rgemm") if check else rc


def mp_dd_Rgetrf(m, n, A, lda, ipiv, info, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rgetrf(m, n, _m(A), lda, _ptr(ipiv), _ptr(info))
    return _check(rc, "mp_dd_Rgetrf") if check else rc


def mp_dd_Rgetrs(trans, n, nrhs, A, lda, ipiv, B, ldb, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rgetrs(_flag(trans), n, nrhs, _cm(A), lda, _ptr(ipiv), _m(B), ldb)
    return _check(rc, "mp_dd_Rgetrs") if check else rc


def mp_dd_Rsyr2k(uplo, trans, n, k, alpha, A, lda, B, ldb, beta, C, ldc, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rsyr2k(_flag(uplo), _flag(trans), n, k, _dd(alpha), _cm(A), lda, _cm(B),
                           ldb, _dd(beta), _m(C), ldc)
    return _check(rc, "mp_dd_Rsyr2k") if check else rc


def mp_dd_Rsymm(side, uplo, m, n, alpha, A, lda, B, ldb, beta, C, ldc, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rsymm(_flag(side), _flag(uplo), m, n, _dd(alpha), _cm(A), lda, _cm(B), ldb,
                          _dd(beta), _m(C), ldc)
    return _check(rc, "mp_dd_Rsymm") if check else rc


def mp_dd_Rtrsm(side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rtrsm(_flag(side), _flag(uplo), _flag(transa), _flag(diag), m, n,
                          _dd(alpha), _cm(A), lda, _m(B), ldb)
    return _check(rc, "mp_dd_Rtrsm") if check else rc


def mp_dd_Rpotrf_crt_workspace(n) -> int:
    return int(_LIB.mp_dd_Rpotrf_crt_workspace(n))


def mp_dd_Rpotrf_crt(uplo, n, A, lda, info, workspace, workspace_bytes, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rpotrf_crt(_flag(uplo), n, _m(A), lda, _ptr(info), _ptr(workspace),
                               workspace_bytes)
    return _check(rc, "mp_dd_Rpotrf_crt") if check else rc


def mp_dd_Rpotrs(uplo, n, nrhs, A, lda, B, ldb, factor_info=None, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_Rpotrs(_flag(uplo), n, nrhs, _cm(A), lda, _m(B), ldb, _ptr(factor_info))
    return _check(rc, "mp_dd_Rpotrs") if check else rc


def mp_dd_potrf_diag_batch(count, descs_dev, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_potrf_diag_batch(count, _ptr(descs_dev))
    return _check(rc, "mp_dd_potrf_diag_batch") if check else rc


def mp_dd_trsm_batch(count, descs_dev, max_nrhs, check=True):
    _sync_stream()
    rc = _LIB.mp_dd_trsm_batch(count, _ptr(descs_dev), max_nrhs)
    return _check(rc, "mp_dd_trsm_batch") if check else rc


def mp_dd_elementwise(op, n, x, y, z, check=True):
    _sync_stream()
    yy = y if y is not None else (None, None)
    rc = _LIB.mp_dd_elementwise(op.encode() if isinstance(op, str) else op, n, _cm(x), _cm(yy),
                                _m(z))
    return _check(rc, "mp_dd_elementwise") if check else rc


def mp_dd_peak_fp64() -> float:
    _sync_stream()
    r = ctypes.c_double()
    _check(_LIB.mp_dd_peak_fp64(ctypes.byref(r)), "mp_dd_peak_fp64")
    return r.value


def mp_dd_set_plain_staging(mode: int) -> None:
    """0 automatic, 1 register staging only, 2 TMA staging where it applies."""
    _check(_LIB.mp_dd_set_plain_staging(int(mode)), "mp_dd_set_plain_staging")


def mp_dd_set_band_pairs(mode: int) -> None:
    """CTA pairs (2-SM MMA) for 256-wide band products: 0 for the Rsyrk
    triangle (the default), 1 wherever they apply, 2 never."""
    _check(_LIB.mp_dd_set_band_pairs(int(mode)), "mp_dd_set_band_pairs")


def mp_dd_peak_ddmac() -> float:
    _sync_stream()
    r = ctypes.c_double()
    _check(_LIB.mp_dd_peak_ddmac(ctypes.byref(r)), "mp_dd_peak_ddmac")
    return r.value


def mp_dd_peak_imma() -> float:
    _sync_stream()
    r = ctypes.c_double()
    _check(_LIB.mp_dd_peak_imma(ctypes.byref(r)), "mp_dd_peak_imma")
    return r.value


# ----------------------------------------------------------------------------
# column-major dd tensors
# ----------------------------------------------------------------------------

def dd_empty(rows: int, cols: int, ld: int | None = None, device="cuda", fill=None):
    """(hi, lo) float64 tensors of shape (rows, cols), strides (1, ld)."""
    ld = max(1, rows if ld is None else ld)
    out = []
    for _ in range(2):
        store = torch.empty((max(cols, 1), ld), dtype=torch.float64, device=device)
        if fill is not None:
            store.fill_(fill)
        out.append(store.t()[:rows, :cols])
    return tuple(out)


def to_device(plane: np.ndarray, device="cuda") -> torch.Tensor:
    """A column-major numpy plane (ld x cols, Fortran order) -> device tensor
    with the same leading dimension; shape (ld, cols), strides (1, ld)."""
    a = np.asfortranarray(plane, dtype=np.float64)
    store = torch.from_numpy(np.ascontiguousarray(a.T)).to(device)
    return store.t()


def to_numpy(t: torch.Tensor) -> np.ndarray:
    """Device column-major tensor -> Fortran-order numpy array of the same shape."""
    return np.asfortranarray(t.detach().t().contiguous().cpu().numpy().T)


def _ld(t: torch.Tensor) -> int:
    if t.dim() != 2 or t.dtype != torch.float64:
        raise ValueError("dd planes must be 2-D float64 tensors")
    if t.shape[0] > 1 and t.stride(0) != 1:
        raise ValueError("dd planes must be column-major (stride(0) == 1)")
    if t.shape[1] > 1:
        return max(1, t.stride(1))
    return max(1, t.shape[0], t.stride(1))


def Rgemm(transa, transb, alpha, A, B, beta, C, m=None, n=None, k=None):
    """C := alpha op(A) op(B) + beta C on column-major dd tensors (in place)."""
    ta, tb = transa.upper() in "TC", transb.upper() in "TC"
    if m is None:
        m = A[0].shape[1] if ta else A[0].shape[0]
    if k is None:
        k = A[0].shape[0] if ta else A[0].shape[1]
    if n is None:
        n = B[0].shape[0] if tb else B[0].shape[1]
    return mp_dd_Rgemm(transa, transb, m, n, k, alpha, A, _ld(A[0]), B, _ld(B[0]), beta, C,
                       _ld(C[0]))


def Rtrsm(side, uplo, transa, diag, alpha, A, B, m=None, n=None):
    """mp_dd_Rtrsm on (hi, lo) device tensors; B (m x n) is overwritten by X."""
    m = B[0].shape[0] if m is None else m
    n = B[0].shape[1] if n is None else n
    return mp_dd_Rtrsm(side, uplo, transa, diag, m, n, alpha, A, _ld(A[0]), B, _ld(B[0]))


def Rsyrk(uplo, trans, alpha, A, beta, C, n=None, k=None):
    t = trans.upper() in "TC"
    if n is None:
        n = A[0].shape[1] if t else A[0].shape[0]
    if k is None:
        k = A[0].shape[0] if t else A[0].shape[1]
    return mp_dd_Rsyrk(uplo, trans, n, k, alpha, A, _ld(A[0]), beta, C, _ld(C[0]))
