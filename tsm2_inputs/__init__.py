"""Seeded, counter-based synthetic inputs for the TSM2R / TSM2L workloads.

This module holds no matrix-multiply arithmetic.  It is the single definition
of the synthetic inputs; the CPU oracle side calls these numpy functions, and
the CUDA library carries its own implementation of the same definition
(``tsm2_fill_*`` in ``csrc/synth.cu``).  The two are cross-checked bit for bit
by the test-suite.

Generator
---------
splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; output constants as published in Vigna's
``splitmix64.c``).  With ``G = 0x9E3779B97F4A7C15`` and the finaliser

    fmix(z): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
             z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31

the stream for ``(seed, matrix_id)`` has the key
``key = fmix(fmix(seed + G) + matrix_id * G)`` and its ``idx``-th draw is
``fmix(key + (idx + 1) * G)`` (all arithmetic mod 2**64): the ``idx+1``-th
output of a splitmix64 generator started in state ``key``.  Being
counter-based, any element can be drawn on its own, which lets the oracle
regenerate single rows of a matrix that is far too large for the host.

Element index
-------------
A logical ``rows x cols`` matrix is indexed column-major over its logical
extent: element ``(i, j)`` is draw number ``i + j * rows``.  Leading-dimension
padding is never drawn.

Distributions (each exact in IEEE binary64, so host and device agree bitwise)
----------------------------------------------------------------------------
* ``uniform_pm1``: ``(x >> 11) * 2**-52 - 1`` in [-1, 1) (the paper draws
  from [0, 1), Sec. 4.1; the workloads here use [-1, 1]).
* ``int_small``: ``((x >> 32) mod 9) - 4`` in {-4..4}; every product and
  partial sum of these is an integer, so GEMM on them is exact.
* ``normal_ih``: Irwin-Hall with twelve uniforms ``u_t = (x_t >> 11) * 2**-53``
  (draws ``12*idx + t``) summed left to right in binary64, minus 6, times a
  caller-given ``scale``: mean 0, variance ``scale**2``.
* ``logmag``: sign from bit 0, significand ``1 + ((x >> 1) & (2**31-1)) *
  2**-31``, binade ``e = ((x >> 32) mod 20) - 10``; magnitudes are
  log-uniform over the twenty binades [2**-10, 2**10) and uniform inside
  each binade.

Binary32 variants are the binary64 value rounded to nearest-even.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Matrix identifiers used by the workloads (stream ids).
MID_A = 1
MID_B = 2
MID_DC = 3
MID_A_LO = 4
MID_BATCH = 5


def fmix(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, matrix_id: int) -> int:
    """Key of the stream ``(seed, matrix_id)``."""
    with np.errstate(over="ignore"):
        s = fmix(np.array([seed], dtype=np.uint64) + GOLDEN)
        k = fmix(s + np.array([matrix_id], dtype=np.uint64) * GOLDEN)
    return int(k[0])


def draws(key: int, idx: np.ndarray) -> np.ndarray:
    """Raw 64-bit draws number ``idx`` of the stream with key ``key``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return fmix(np.uint64(key) + (idx + np.uint64(1)) * GOLDEN)


def _index_grid(rows: int, cols: int, row_idx=None, col_idx=None) -> np.ndarray:
    r = np.arange(rows, dtype=np.uint64) if row_idx is None else np.asarray(row_idx, dtype=np.uint64)
    c = np.arange(cols, dtype=np.uint64) if col_idx is None else np.asarray(col_idx, dtype=np.uint64)
    return r[:, None] + c[None, :] * np.uint64(rows)


def _finish(v64: np.ndarray, dtype) -> np.ndarray:
    dtype = np.dtype(dtype)
    if dtype == np.float64:
        out = v64
    elif dtype == np.float32:
        out = v64.astype(np.float32)  # IEEE round-to-nearest-even
    else:
        raise ValueError(f"unsupported dtype {dtype}")
    return np.asfortranarray(out)


def uniform_pm1(seed: int, matrix_id: int, rows: int, cols: int, dtype=np.float64,
                row_idx=None, col_idx=None) -> np.ndarray:
    """Column-major (Fortran-ordered) ``rows x cols`` matrix, entries in [-1, 1).

    ``row_idx`` / ``col_idx`` select a sub-block of the logical matrix (the
    indices still refer to the full ``rows x cols`` matrix).
    """
    x = draws(stream_key(seed, matrix_id), _index_grid(rows, cols, row_idx, col_idx))
    v = (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -52 - 1.0
    return _finish(v, dtype)


def int_small(seed: int, matrix_id: int, rows: int, cols: int, dtype=np.float64,
              row_idx=None, col_idx=None) -> np.ndarray:
    """Integers in {-4, ..., 4} stored as floating point."""
    x = draws(stream_key(seed, matrix_id), _index_grid(rows, cols, row_idx, col_idx))
    v = ((x >> np.uint64(32)) % np.uint64(9)).astype(np.float64) - 4.0
    return _finish(v, dtype)


def normal_ih(seed: int, matrix_id: int, rows: int, cols: int, scale: float, dtype=np.float64,
              row_idx=None, col_idx=None) -> np.ndarray:
    """Irwin-Hall(12) approximate normal, mean 0, standard deviation ``scale``."""
    key = stream_key(seed, matrix_id)
    base = _index_grid(rows, cols, row_idx, col_idx) * np.uint64(12)
    s = np.zeros(base.shape, dtype=np.float64)
    for t in range(12):  # left-to-right binary64 sum, same order as the device
        u = (draws(key, base + np.uint64(t)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        s = s + u
    v = (s - 6.0) * np.float64(scale)
    return _finish(v, dtype)


def logmag(seed: int, matrix_id: int, rows: int, cols: int, dtype=np.float64,
           row_idx=None, col_idx=None) -> np.ndarray:
    """Random sign, magnitude log-uniform over the binades [2**-10, 2**10).

    From one draw ``x``: sign = bit 0 (1 means negative); binade
    ``e = ((x >> 32) mod 20) - 10``; significand ``1 + f * 2**-31`` with
    ``f = (x >> 1) & (2**31 - 1)``; value ``sign * significand * 2**e``.
    """
    x = draws(stream_key(seed, matrix_id), _index_grid(rows, cols, row_idx, col_idx))
    e = ((x >> np.uint64(32)) % np.uint64(20)).astype(np.int64) - 10
    f = ((x >> np.uint64(1)) & np.uint64(0x7FFFFFFF)).astype(np.float64)
    mag = np.ldexp(1.0 + f * 2.0 ** -31, e)
    sign = np.where((x & np.uint64(1)) == np.uint64(1), -1.0, 1.0)
    return _finish(sign * mag, dtype)


def uniform_int(seed: int, matrix_id: int, idx, lo: int, hi: int) -> np.ndarray:
    """Inclusive discrete uniform integers in [lo, hi] from draws ``idx``."""
    x = draws(stream_key(seed, matrix_id), np.asarray(idx, dtype=np.uint64))
    span = np.uint64(hi - lo + 1)
    return (x % span).astype(np.int64) + lo


def padded(a: np.ndarray, ld: int, fill=np.nan) -> np.ndarray:
    """Copy a column-major matrix into a column-major buffer with leading
    dimension ``ld`` (rows ``a.shape[0]..ld-1`` set to ``fill``).  Returns the
    full ``ld x cols`` Fortran-ordered buffer."""
    rows, cols = a.shape
    assert ld >= rows
    buf = np.full((ld, cols), fill, dtype=a.dtype, order="F")
    buf[:rows, :] = a
    return buf


def batch_shapes(seed: int = 0, n_r: int = 256, n_l: int = 256,
                 r_n=(512, 8192), r_k=(2, 16), l_m=(2 ** 14, 2 ** 20), l_n=(4, 32)):
    """Shapes of the uneven batch workload (draws of stream ``MID_BATCH``).

    TSM2R problem i (i < n_r): square A, n = m from draw 2i, k from draw 2i+1.
    TSM2L problem i: m from draw 2*n_r + 2i, n = k from draw 2*n_r + 2i + 1.
    All bounds inclusive.  The list (R problems, then L problems) is then put
    in the order of the argsort of draws 2*(n_r+n_l) + position.
    Returns a list of (op, m, n, k).
    """
    out = []
    for i in range(n_r):
        n = int(uniform_int(seed, MID_BATCH, [2 * i], *r_n)[0])
        k = int(uniform_int(seed, MID_BATCH, [2 * i + 1], *r_k)[0])
        out.append(("r", n, n, k))
    base = 2 * n_r
    for i in range(n_l):
        m = int(uniform_int(seed, MID_BATCH, [base + 2 * i], *l_m)[0])
        n = int(uniform_int(seed, MID_BATCH, [base + 2 * i + 1], *l_n)[0])
        out.append(("l", m, n, n))
    keys = draws(stream_key(seed, MID_BATCH), np.arange(len(out)) + 2 * (n_r + n_l))
    order = np.argsort(keys, kind="stable")
    return [out[i] for i in order]
