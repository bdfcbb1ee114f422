"""GB300 tall-and-skinny matrix multiplication (TSM2R / TSM2L).

A thin ctypes binding over the C ABI in ``include/tsm2.h``; every step of the
multiply runs in the CUDA library ``_build/libtsm2.so`` (built by
``paper_2002_03258_gb300.build``).  There is no CPU fallback: if the library
is missing, every entry point raises.

Low-level functions carry the C names and arguments (device pointers as
ints, ``stream`` as an int handle, 0 = default stream) and return the integer
status.  ``tsm2r`` / ``tsm2l`` accept torch CUDA tensors that are column-major
views (shape ``(rows, cols)``, strides ``(1, ld)``), e.g. ``X.t()`` of a
contiguous row-major ``(cols, ld)`` tensor.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# TSM2_DEBUG=1 selects the bounds-checking build (build(debug=True)).
DEBUG = os.environ.get("TSM2_DEBUG", "0") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "_build", "libtsm2_debug.so" if DEBUG else "libtsm2.so")

SUCCESS = 0
ERR_INVALID_VALUE = 1
ERR_UNSUPPORTED = 2
ERR_CUDA = 3
ERR_TIMEOUT = 4
ERR_BOUNDS = 5

_lock = threading.Lock()
_lib = None


class TSM2Error(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"tsm2 status {status}: {message}")
        self.status = status


def _load():
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"CUDA library not built ({LIB_PATH} missing); run "
                    + ("`python -m paper_2002_03258_gb300.build --debug`" if DEBUG else
                       "`python -c \"import __graft_entry__ as g; g.build()\"`"))
            lib = ctypes.CDLL(LIB_PATH)
            i64, vp, u64 = ctypes.c_int64, ctypes.c_void_p, ctypes.c_uint64
            gemm_sig = [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp]
            for name in ("tsm2r_d", "tsm2r_s", "tsm2l_d", "tsm2l_s", "tsm2x_d", "tsm2x_s", "tsm2r_s_noalloc",
                         "tsm2r_s_host", "tsm2r_d_host", "tsm2l_s_host", "tsm2l_d_host",
                         "tsm2r_t_d", "tsm2r_t_s", "tsm2_rankk_d", "tsm2_rankk_s"):
                f = getattr(lib, name)
                f.argtypes = gemm_sig
                f.restype = ctypes.c_int
            lib.tsm2x_choice.argtypes = [ctypes.c_int, i64, i64, i64]
            lib.tsm2x_choice.restype = ctypes.c_char
            lib.tsm2r_bf16.argtypes = [i64, i64, i64, vp, vp, i64, vp, i64, vp, i64, vp]
            lib.tsm2r_bf16.restype = ctypes.c_int
            lib.tsm2_split_bf16.argtypes = [i64, i64, vp, i64, vp, vp, i64, vp]
            lib.tsm2_split_bf16.restype = ctypes.c_int
            i32 = ctypes.c_int
            lib.tsm2_batch_plan_create_s.argtypes = [i32, vp, i32, ctypes.POINTER(vp)]
            lib.tsm2_batch_plan_create_s.restype = i32
            for name in ("tsm2_batch_plan_execute", "tsm2_batch_plan_graph_launch"):
                f = getattr(lib, name)
                f.argtypes = [vp, vp]
                f.restype = i32
            lib.tsm2_batch_plan_execute_class.argtypes = [vp, i32, vp]
            lib.tsm2_batch_plan_execute_class.restype = i32
            lib.tsm2_batch_plan_num_classes.argtypes = [vp]
            lib.tsm2_batch_plan_num_classes.restype = i32
            lib.tsm2_batch_plan_class_info.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_char_p),
                                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32),
                                                       ctypes.POINTER(i32)]
            lib.tsm2_batch_plan_class_info.restype = i32
            lib.tsm2_batch_plan_set_grids.argtypes = [vp, i32, ctypes.POINTER(i32)]
            lib.tsm2_batch_plan_set_grids.restype = i32
            lib.tsm2_batch_plan_set_serial.argtypes = [vp, i32]
            lib.tsm2_batch_plan_set_serial.restype = i32
            lib.tsm2_batch_plan_set_mode.argtypes = [vp, i32]
            lib.tsm2_batch_plan_set_mode.restype = i32
            lib.tsm2_batch_plan_set_single_grid.argtypes = [vp, i32]
            lib.tsm2_batch_plan_set_single_grid.restype = i32
            lib.tsm2_batch_plan_num_launches.argtypes = [vp]
            lib.tsm2_batch_plan_num_launches.restype = i32
            lib.tsm2_batch_num_variants.argtypes = []
            lib.tsm2_batch_num_variants.restype = i32
            lib.tsm2_batch_variant_info.argtypes = [i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(i32),
                                                    ctypes.POINTER(i32), ctypes.POINTER(i32)]
            lib.tsm2_batch_variant_info.restype = i32
            lib.tsm2_batch_plan_destroy.argtypes = [vp]
            lib.tsm2_batch_plan_destroy.restype = None
            lib.tsm2_get_last_error_string.restype = ctypes.c_char_p
            lib.tsm2_last_config.restype = ctypes.c_char_p
            lib.tsm2_last_host_copy.restype = ctypes.c_char_p
            lib.tsm2_get_device_status.argtypes = [vp]
            lib.tsm2_get_device_status.restype = ctypes.c_int
            lib.tsm2_shutdown.restype = None
            lib.tsm2_set_wait_budget_ns.argtypes = [i64]
            lib.tsm2_set_path.argtypes = [ctypes.c_int]
            lib.tsm2_set_grid.argtypes = [ctypes.c_int]
            lib.tsm2_set_host_copy.argtypes = [ctypes.c_int]
            lib.tsm2_set_host_copy.restype = None
            lib.tsm2_set_balance.argtypes = [ctypes.c_int]
            lib.tsm2_set_balance.restype = None
            lib.tsm2_set_trace.argtypes = [vp, i64]
            lib.tsm2_set_trace.restype = None
            for name in ("tsm2_fill_uniform_d", "tsm2_fill_uniform_s", "tsm2_fill_int_small_d",
                         "tsm2_fill_int_small_s", "tsm2_fill_logmag_s"):
                f = getattr(lib, name)
                f.argtypes = [i64, i64, u64, u64, vp, i64, vp]
                f.restype = ctypes.c_int
            lib.tsm2_debug_checks.argtypes = []
            lib.tsm2_debug_checks.restype = ctypes.c_int
            lib.tsm2_fma_probe.argtypes = [ctypes.c_int, ctypes.c_int, i64, vp, vp]
            lib.tsm2_fma_probe.restype = ctypes.c_int
            for name in ("tsm2_fill_normal_ih_d", "tsm2_fill_normal_ih_s"):
                f = getattr(lib, name)
                f.argtypes = [i64, i64, u64, u64, ctypes.c_double, vp, i64, vp]
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def lib():
    """The loaded ctypes library (raises if it has not been built)."""
    return _load()


# ---- C-named entry points (argument marshalling only) ----------------------

def tsm2r_d(m, n, k, A, lda, B, ldb, C, ldc, stream=0):
    return _load().tsm2r_d(m, n, k, A, lda, B, ldb, C, ldc, stream)


def tsm2r_s(m, n, k, A, lda, B, ldb, C, ldc, stream=0):
    return _load().tsm2r_s(m, n, k, A, lda, B, ldb, C, ldc, stream)


def tsm2l_d(m, n, k, A, lda, B, ldb, C, ldc, stream=0):
    return _load().tsm2l_d(m, n, k, A, lda, B, ldb, C, ldc, stream)


def tsm2l_s(m, n, k, A, lda, B, ldb, C, ldc, stream=0):
    return _load().tsm2l_s(m, n, k, A, lda, B, ldb, C, ldc, stream)


def tsm2r_s_noalloc(m, n, k, A, lda, B, ldb, C, ldc, stream=0):
    return _load().tsm2r_s_noalloc(m, n, k, A, lda, B, ldb, C, ldc, stream)


def tsm2x_s(m, n, k, A, lda, B, ldb, C, ldc, stream=0):
    return _load().tsm2x_s(m, n, k, A, lda, B, ldb, C, ldc, stream)


def tsm2x_d(m, n, k, A, lda, B, ldb, C, ldc, stream=0):
    return _load().tsm2x_d(m, n, k, A, lda, B, ldb, C, ldc, stream)


def tsm2x_choice(elem_bytes, m, n, k) -> str:
    """'r' or 'l': the schedule tsm2x_s (4) / tsm2x_d (8) picks for the shape."""
    c = _load().tsm2x_choice(elem_bytes, m, n, k)
    return "" if c in (b"\x00", b"") else c.decode()


def tsm2r_s_host(m, n, k, A, lda, B, ldb, C, ldc, stream=0):
    return _load().tsm2r_s_host(m, n, k, A, lda, B, ldb, C, ldc, stream)


def tsm2r_d_host(m, n, k, A, lda, B, ldb, C, ldc, stream=0):
    return _load().tsm2r_d_host(m, n, k, A, lda, B, ldb, C, ldc, stream)


def tsm2l_s_host(m, n, k, A, lda, B, ldb, C, ldc, stream=0):
    return _load().tsm2l_s_host(m, n, k, A, lda, B, ldb, C, ldc, stream)


def tsm2l_d_host(m, n, k, A, lda, B, ldb, C, ldc, stream=0):
    return _load().tsm2l_d_host(m, n, k, A, lda, B, ldb, C, ldc, stream)


def tsm2r_t_d(m, n, k, A, lda, dC, lddc, dB, lddb, stream=0):
    return _load().tsm2r_t_d(m, n, k, A, lda, dC, lddc, dB, lddb, stream)


def tsm2r_t_s(m, n, k, A, lda, dC, lddc, dB, lddb, stream=0):
    return _load().tsm2r_t_s(m, n, k, A, lda, dC, lddc, dB, lddb, stream)


def tsm2_rankk_d(m, n, k, dC, lddc, B, ldb, dA, ldda, stream=0):
    return _load().tsm2_rankk_d(m, n, k, dC, lddc, B, ldb, dA, ldda, stream)


def tsm2_rankk_s(m, n, k, dC, lddc, B, ldb, dA, ldda, stream=0):
    return _load().tsm2_rankk_s(m, n, k, dC, lddc, B, ldb, dA, ldda, stream)


def tsm2r_bf16(m, n, k, A_hi, A_lo, lda, B, ldb, C, ldc, stream=0):
    return _load().tsm2r_bf16(m, n, k, A_hi, A_lo, lda, B, ldb, C, ldc, stream)


def tsm2_split_bf16(rows, cols, X, ldx, hi, lo, ldh, stream=0):
    return _load().tsm2_split_bf16(rows, cols, X, ldx, hi, lo, ldh, stream)


def tsm2_get_last_error_string() -> str:
    return _load().tsm2_get_last_error_string().decode()


def tsm2_last_config() -> str:
    return _load().tsm2_last_config().decode()


def tsm2_last_host_copy() -> str:
    return _load().tsm2_last_host_copy().decode()


def tsm2_get_device_status(stream=0) -> int:
    return _load().tsm2_get_device_status(stream)


def tsm2_shutdown() -> None:
    _load().tsm2_shutdown()


def tsm2_set_wait_budget_ns(ns: int) -> None:
    _load().tsm2_set_wait_budget_ns(int(ns))


def tsm2_set_path(path: int) -> None:
    _load().tsm2_set_path(int(path))


def tsm2_set_grid(blocks: int) -> None:
    _load().tsm2_set_grid(int(blocks))


def tsm2_set_host_copy(mode: int) -> None:
    _load().tsm2_set_host_copy(int(mode))


def tsm2_set_balance(mode: int) -> None:
    _load().tsm2_set_balance(int(mode))


def tsm2_set_trace(device_words, blocks: int) -> None:
    _load().tsm2_set_trace(device_words, int(blocks))


def check(status: int) -> None:
    """Raise :class:`TSM2Error` for a non-zero status."""
    if status != SUCCESS:
        raise TSM2Error(status, tsm2_get_last_error_string())


# ---- torch convenience -------------------------------------------------------

def _colmajor(t, name):
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    rows, cols = t.shape
    if t.stride(0) != 1 and rows > 1:
        raise ValueError(f"{name} must be a column-major view (stride(0) == 1), got strides {t.stride()}")
    ld = t.stride(1) if cols > 1 else max(rows, 1)
    return rows, cols, max(ld, rows, 1)


def empty_colmajor(rows, cols, dtype, device, ld=None):
    """Uninitialised column-major ``rows x cols`` tensor with leading dim ``ld``."""
    import torch
    ld = max(rows, 1) if ld is None else ld
    return torch.empty((cols, ld), dtype=dtype, device=device).t()[:rows]


def _stream_of(t):
    import torch
    return torch.cuda.current_stream(t.device).cuda_stream


def _matmul(op, A, B, out=None):
    import torch
    if A.dtype != B.dtype or A.dtype not in (torch.float32, torch.float64):
        raise TypeError("A and B must both be float32 or both float64")
    if not (A.is_cuda and B.is_cuda):
        raise ValueError("tensors must be on a CUDA device")
    m, n, lda = _colmajor(A, "A")
    n2, k, ldb = _colmajor(B, "B")
    if n != n2:
        raise ValueError(f"inner dimensions differ: {A.shape} x {B.shape}")
    if out is None:
        out = empty_colmajor(m, k, A.dtype, A.device)
    mc, kc, ldc = _colmajor(out, "out")
    if (mc, kc) != (m, k) or out.dtype != A.dtype:
        raise ValueError("out has the wrong shape or dtype")
    fn = {("r", torch.float64): tsm2r_d, ("r", torch.float32): tsm2r_s,
          ("l", torch.float64): tsm2l_d, ("l", torch.float32): tsm2l_s}[(op, A.dtype)]
    check(fn(m, n, k, A.data_ptr(), lda, B.data_ptr(), ldb, out.data_ptr(), ldc, _stream_of(A)))
    return out


def tsm2r_t(A, dC, out=None):
    """dB = A^T @ dC (A m x n, dC m x k; column-major views), the transposed TSM2R."""
    import torch
    if A.dtype != dC.dtype or A.dtype not in (torch.float32, torch.float64):
        raise TypeError("A and dC must both be float32 or both float64")
    m, n, lda = _colmajor(A, "A")
    m2, k, lddc = _colmajor(dC, "dC")
    if m != m2:
        raise ValueError(f"row counts differ: {A.shape} vs {dC.shape}")
    if out is None:
        out = empty_colmajor(n, k, A.dtype, A.device)
    _, _, lddb = _colmajor(out, "out")
    fn = tsm2r_t_d if A.dtype == torch.float64 else tsm2r_t_s
    check(fn(m, n, k, A.data_ptr(), lda, dC.data_ptr(), lddc, out.data_ptr(), lddb, _stream_of(A)))
    return out


def rankk(dC, B, out=None):
    """dA = dC @ B^T (dC m x k, B n x k; column-major views), a rank-k update."""
    import torch
    if dC.dtype != B.dtype or dC.dtype not in (torch.float32, torch.float64):
        raise TypeError("dC and B must both be float32 or both float64")
    m, k, lddc = _colmajor(dC, "dC")
    n, k2, ldb = _colmajor(B, "B")
    if k != k2:
        raise ValueError(f"column counts differ: {dC.shape} vs {B.shape}")
    if out is None:
        out = empty_colmajor(m, n, dC.dtype, dC.device)
    _, _, ldda = _colmajor(out, "out")
    fn = tsm2_rankk_d if dC.dtype == torch.float64 else tsm2_rankk_s
    check(fn(m, n, k, dC.data_ptr(), lddc, B.data_ptr(), ldb, out.data_ptr(), ldda, _stream_of(dC)))
    return out


def tsm2r(A, B, out=None):
    """C = A @ B with the TSM2R schedule (large A, tall-and-skinny B)."""
    return _matmul("r", A, B, out)


def tsm2l(A, B, out=None):
    """C = A @ B with the TSM2L schedule (tall-and-skinny A, small B)."""
    return _matmul("l", A, B, out)


__all__ = [
    "tsm2r_d", "tsm2r_s", "tsm2l_d", "tsm2l_s", "tsm2r_s_noalloc", "tsm2_get_last_error_string", "tsm2_last_config",
    "tsm2r_s_host", "tsm2r_d_host", "tsm2l_s_host", "tsm2l_d_host", "tsm2x_s", "tsm2x_d", "tsm2x_choice",
    "tsm2_get_device_status", "tsm2_shutdown", "tsm2_set_wait_budget_ns", "tsm2_set_path", "tsm2_set_grid", "tsm2_set_trace",
    "tsm2_set_host_copy", "tsm2_last_host_copy", "tsm2_set_balance",
    "check", "tsm2r", "tsm2l", "tsm2r_t", "rankk", "empty_colmajor", "TSM2Error", "lib", "LIB_PATH",
    "tsm2r_t_d", "tsm2r_t_s", "tsm2_rankk_d", "tsm2_rankk_s", "tsm2r_bf16", "tsm2_split_bf16",
]
