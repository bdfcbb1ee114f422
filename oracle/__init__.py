"""CPU oracle for TSM2R / TSM2L: the plain matrix-product definition in C.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_2002_03258_gb300``) and never imports it.

The arithmetic lives in ``tsm2_oracle.c`` (see its header for what is
computed and which passage of the paper it follows); this module compiles it
with gcc into ``oracle/_build/liboracle.so`` and wraps it for numpy arrays of
any strides.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsm2_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Flags: no fast-math and no contraction into fused multiply-adds, so every
# product is rounded and then added, on x86-64 and AArch64 alike.
CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc); returns its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, vp = ctypes.c_int64, ctypes.c_void_p
            sig = [i64, i64, i64, vp, i64, i64, vp, i64, i64, vp, i64, i64]
            for name in ("oracle_gemm_d", "oracle_gemm_s", "oracle_absgemm_d",
                         "oracle_absgemm_s", "oracle_gemm_ld"):
                f = getattr(lib, name)
                f.argtypes = sig
                f.restype = None
            lib.oracle_long_double_mant_dig.restype = ctypes.c_int
            lib.oracle_bf16_rne.argtypes = [i64, vp, vp]
            lib.oracle_bf16_to_float_n.argtypes = [i64, vp, vp]
            _lib = lib
    return _lib


def _strides(a: np.ndarray):
    rs, cs = a.strides
    return rs // a.itemsize, cs // a.itemsize


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(A: np.ndarray, B: np.ndarray):
    if A.ndim != 2 or B.ndim != 2 or A.shape[1] != B.shape[0]:
        raise ValueError(f"shape mismatch {A.shape} x {B.shape}")
    if A.dtype != B.dtype or A.dtype not in (np.float64, np.float32):
        raise ValueError(f"dtypes must match and be float32/float64, got {A.dtype}, {B.dtype}")


def _call(fname_d, fname_s, A, B, out_dtype=np.float64):
    _check(A, B)
    lib = _load()
    m, n = A.shape
    k = B.shape[1]
    C = np.zeros((m, k), dtype=out_dtype, order="F")
    if m == 0 or k == 0:
        return C
    fn = getattr(lib, fname_d if A.dtype == np.float64 else fname_s)
    ars, acs = _strides(A)
    brs, bcs = _strides(B)
    crs, ccs = _strides(C)
    fn(m, n, k, _ptr(A), ars, acs, _ptr(B), brs, bcs, _ptr(C), crs, ccs)
    return C


def gemm(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """C = A B, every entry a left-to-right binary64 sum over the inner index.

    float32 inputs are widened exactly; the result is always float64.
    """
    return _call("oracle_gemm_d", "oracle_gemm_s", A, B)


def absgemm(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """S = |A| |B| in binary64 (the error-bound magnitude matrix)."""
    return _call("oracle_absgemm_d", "oracle_absgemm_s", A, B)


def gemm_ld(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """C = A B accumulated in long double (binary64 inputs only)."""
    if A.dtype != np.float64:
        raise ValueError("gemm_ld takes float64 inputs")
    _check(A, B)
    lib = _load()
    m, n = A.shape
    k = B.shape[1]
    C = np.zeros((m, k), dtype=np.longdouble, order="F")
    if m and k:
        ars, acs = _strides(A)
        brs, bcs = _strides(B)
        crs, ccs = _strides(C)
        lib.oracle_gemm_ld(m, n, k, _ptr(A), ars, acs, _ptr(B), brs, bcs, _ptr(C), crs, ccs)
    return C


def long_double_mant_dig() -> int:
    return int(_load().oracle_long_double_mant_dig())


def gemm_threaded(A: np.ndarray, B: np.ndarray, threads: int) -> np.ndarray:
    """:func:`gemm` with the rows of A split over ``threads`` host threads.

    Each entry is still the same left-to-right sum, so the result is
    bitwise identical to :func:`gemm`; only wall time changes.  (ctypes
    releases the GIL during the foreign call.)
    """
    _check(A, B)
    m = A.shape[0]
    C = np.zeros((m, B.shape[1]), dtype=np.float64, order="F")
    if m == 0:
        return C
    threads = max(1, min(threads, m))
    bounds = np.linspace(0, m, threads + 1).astype(int)

    def work(t):
        lo, hi = bounds[t], bounds[t + 1]
        if hi > lo:
            C[lo:hi, :] = gemm(A[lo:hi, :], B)

    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(work, range(threads)))
    return C


def bf16_rne(x: np.ndarray) -> np.ndarray:
    """binary32 -> bfloat16 bit patterns (uint16), round to nearest even."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    _load().oracle_bf16_rne(x.size, _ptr(x), _ptr(out))
    return out


def bf16_to_float(h: np.ndarray) -> np.ndarray:
    """bfloat16 bit patterns -> binary32 (exact)."""
    h = np.ascontiguousarray(h, dtype=np.uint16)
    out = np.empty(h.shape, dtype=np.float32)
    _load().oracle_bf16_to_float_n(h.size, _ptr(h), _ptr(out))
    return out


def gamma(n: int, u: float) -> float:
    """gamma_n = n u / (1 - n u) (Higham, Accuracy and Stability, Sec. 3.1)."""
    nu = n * u
    if nu >= 1.0:
        return float("inf")
    return nu / (1.0 - nu)


U_FP64 = 2.0 ** -53
U_FP32 = 2.0 ** -24
