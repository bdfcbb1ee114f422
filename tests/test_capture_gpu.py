"""Stream capture and the per-stream workspace (include/tsm2.h, "Scratch").

The split-reduction workspace of a stream grows with cudaMalloc after a
synchronise, neither of which may run while the stream is captured into a
CUDA graph.  A call that would grow it during capture must return
TSM2_ERR_UNSUPPORTED and leave the capture valid; once the stream has run
the largest shape, the same call captures and replays correctly.
"""
import numpy as np
import pytest

import tsm2_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import DevMat, assert_parity  # noqa: E402


def test_workspace_growth_refused_during_capture_then_captures():
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    lib = pkg.lib()
    m, n, k = 4096, 4096, 16  # row blocks split between blocks: needs the workspace
    A = ti.uniform_pm1(8, ti.MID_A, m, n, np.float32)
    B = ti.uniform_pm1(8, ti.MID_B, n, k, np.float32)
    dA, dB, dC = DevMat(A), DevMat(B), DevMat(np.zeros((m, k), np.float32))
    # library state initialised outside any capture (device attributes, status word)
    assert lib.tsm2r_s(m, n, k, dA.ptr, m, dB.ptr, n, dC.ptr, m, 0) == 0
    torch.cuda.synchronize()

    s = torch.cuda.Stream()  # a stream the library has no workspace for
    x = torch.zeros(1, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        st = lib.tsm2r_s(m, n, k, dA.ptr, m, dB.ptr, n, dC.ptr, m, s.cuda_stream)
        x.add_(1.0)
    assert st == pkg.ERR_UNSUPPORTED
    assert "capture" in pkg.tsm2_get_last_error_string()
    g.replay()  # the capture itself stayed valid
    torch.cuda.synchronize()
    assert x.item() == 1.0

    # the largest shape once on the stream, then the call captures
    assert lib.tsm2r_s(m, n, k, dA.ptr, m, dB.ptr, n, dC.ptr, m, s.cuda_stream) == 0
    s.synchronize()
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=s):
        st2 = lib.tsm2r_s(m, n, k, dA.ptr, m, dB.ptr, n, dC.ptr, m, s.cuda_stream)
    assert st2 == 0, pkg.tsm2_get_last_error_string()
    dC.view.fill_(float("nan"))
    torch.cuda.synchronize()
    g2.replay()
    torch.cuda.synchronize()
    assert pkg.tsm2_get_device_status(0) == 0
    assert_parity(dC.numpy(), A, B, np.float32)
