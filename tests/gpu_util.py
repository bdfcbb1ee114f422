"""Helpers for the GPU parity tests: column-major device buffers with padding
and offsets, and the componentwise comparison against the oracle."""
import numpy as np
import torch

import oracle

DT = {np.float64: torch.float64, np.float32: torch.float32}
FN = {("r", np.float64): "tsm2r_d", ("r", np.float32): "tsm2r_s",
      ("l", np.float64): "tsm2l_d", ("l", np.float32): "tsm2l_s",
      ("x", np.float64): "tsm2x_d", ("x", np.float32): "tsm2x_s"}


class DevMat:
    """Column-major device matrix inside a NaN-filled buffer.

    ``ld`` is the leading dimension, ``offset`` shifts the base pointer by that
    many elements (to break 16-byte alignment)."""

    def __init__(self, a: np.ndarray, ld=None, offset=0, fill=np.nan):
        rows, cols = a.shape
        self.rows, self.cols = rows, cols
        self.ld = max(rows, 1) if ld is None else ld
        self.offset = offset
        tdt = DT[a.dtype.type]
        self.buf = torch.full((max(cols, 1) * self.ld + offset + 8,), fill, dtype=tdt, device="cuda")
        self.view = self.buf[offset:offset + cols * self.ld].view(cols, self.ld).t()[:rows] if cols else None
        if rows and cols:
            self.view.copy_(torch.from_numpy(np.ascontiguousarray(a)).cuda())

    @property
    def ptr(self):
        return self.buf.data_ptr() + self.offset * self.buf.element_size()

    def numpy(self):
        if not self.rows or not self.cols:
            return np.zeros((self.rows, self.cols))
        return self.view.cpu().numpy()

    def padding(self):
        """Everything in the buffer outside the logical matrix."""
        full = self.buf.cpu().numpy()
        mask = np.ones(full.shape, bool)
        for j in range(self.cols):
            s = self.offset + j * self.ld
            mask[s:s + self.rows] = False
        return full[mask]


def call(op, dtype, m, n, k, dA, dB, dC, stream=0):
    import paper_2002_03258_gb300 as pkg
    fn = getattr(pkg, FN[(op, dtype)])
    return fn(m, n, k, dA.ptr, dA.ld, dB.ptr, dB.ld, dC.ptr, dC.ld, stream)


def assert_parity(got: np.ndarray, A: np.ndarray, B: np.ndarray, dtype, exact=False):
    """|C_gpu - C_oracle| <= 2 gamma_n(u) |A||B| elementwise (both sides carry
    at most gamma_n |A||B| of rounding error); NaN/Inf positions must match."""
    ref = oracle.gemm(A, B)
    got = got.astype(np.float64)
    assert got.shape == ref.shape
    fin = np.isfinite(ref)
    assert np.array_equal(np.isnan(got), np.isnan(ref)), "NaN positions differ"
    assert np.array_equal(got[~fin & ~np.isnan(ref)], ref[~fin & ~np.isnan(ref)]), "Inf values differ"
    if exact:
        assert np.array_equal(got[fin], ref[fin])
        return 0.0
    n = A.shape[1]
    u = oracle.U_FP64 if dtype == np.float64 else oracle.U_FP32
    S = oracle.absgemm(A, B)
    bound = 2.0 * oracle.gamma(n, u) * S
    err = np.abs(got - ref)
    bad = fin & ~(err <= bound)
    assert not bad.any(), (f"{bad.sum()} entries outside the bound; worst at {np.argwhere(bad)[0]}: "
                           f"err={err[bad].max():.3e} bound={bound[bad].min():.3e}")
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(bound > 0, err / bound, 0.0)
    return float(np.max(r[fin])) if fin.any() else 0.0
