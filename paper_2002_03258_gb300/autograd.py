"""Differentiable TSM2R: ``C = A @ B`` with a hand-written backward.

    forward   C  = A B          tsm2r_{s,d}      (A read once)
    backward  dB = A^T dC       tsm2r_t_{s,d}    (A read once more)
              dA = dC B^T       tsm2_rankk_{s,d} (dA written once)

All three run in the CUDA library; torch only supplies memory, streams and
the autograd graph.  Operands and gradients are column-major views (strides
``(1, ld)``), the layout of the C ABI.
"""
from __future__ import annotations

import torch

from . import rankk, tsm2r, tsm2r_t


def _colmajor(t: torch.Tensor) -> torch.Tensor:
    if t.dim() == 2 and (t.stride(0) == 1 or t.shape[0] <= 1) and t.stride(1) >= max(t.shape[0], 1):
        return t
    return t.t().contiguous().t()


class TSM2RFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B):
        A = _colmajor(A)
        B = _colmajor(B)
        ctx.save_for_backward(A, B)
        return tsm2r(A, B)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dC = _colmajor(dC)
        dA = rankk(dC, B) if ctx.needs_input_grad[0] else None
        dB = tsm2r_t(A, dC) if ctx.needs_input_grad[1] else None
        return dA, dB


def tsm2r_mm(A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """Differentiable ``A @ B`` on the TSM2R kernels."""
    return TSM2RFunction.apply(A, B)
