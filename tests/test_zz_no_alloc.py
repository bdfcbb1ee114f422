"""The allocation-free binary32 TSM2R entry point, tsm2r_s_noalloc.

It serves callers that cannot call cudaMalloc (device memory wholly owned by
another allocator, or a loop that cannot afford cudaMalloc's cost and
synchronisation): its scratch is a fixed device array inside the library.
Through the C ABI, two calls in a row must give what tsm2r_s gives, within
the componentwise bound of the other parity tests (in fact bit for bit: same
kernel, same grid, same summation order).  Collected last, so that a failing
run that stops at the first failure has already run everything else; it must
pass alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

import tsm2_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import DevMat, assert_parity  # noqa: E402


def test_noalloc_matches_tsm2r_s_twice():
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    lib = pkg.lib()
    # several row blocks split between thread blocks, ragged m and k > 16
    for (m, n, k) in [(3000, 9000, 16), (10240, 10240, 20), (777, 5000, 3)]:
        ld = (m + 3) // 4 * 4
        A = ti.uniform_pm1(1, ti.MID_A, m, n, np.float32)
        B = ti.uniform_pm1(1, ti.MID_B, n, k, np.float32)
        dA, dB = DevMat(A, ld), DevMat(B)
        ref = DevMat(np.zeros((m, k), np.float32), ld)
        assert lib.tsm2r_s(m, n, k, dA.ptr, ld, dB.ptr, n, ref.ptr, ld, 0) == 0, pkg.tsm2_get_last_error_string()
        want = ref.numpy()
        for call in range(2):
            out = DevMat(np.full((m, k), np.nan, np.float32), ld, fill=-3.0)
            st = lib.tsm2r_s_noalloc(m, n, k, dA.ptr, ld, dB.ptr, n, out.ptr, ld, 0)
            assert st == 0, pkg.tsm2_get_last_error_string()
            assert not pkg.tsm2_last_config().startswith("simple")
            torch.cuda.synchronize()
            assert pkg.tsm2_get_device_status(0) == 0
            got = out.numpy()
            assert_parity(got, A, B, np.float32)
            assert_parity(want, A, B, np.float32)
            np.testing.assert_array_equal(got, want)
            assert np.all(out.padding() == -3.0)


def test_noalloc_rejects_problems_beyond_its_scratch():
    import paper_2002_03258_gb300 as pkg
    lib = pkg.lib()
    m, n, k = 4_000_000, 64, 16
    a = torch.empty(16, device="cuda")  # 16-byte aligned, never read: the call is rejected first
    fake = a.data_ptr()
    st = lib.tsm2r_s_noalloc(m, n, k, fake, m, fake + (1 << 32), n, fake + (1 << 34), m, 0)
    assert st == pkg.ERR_UNSUPPORTED
    assert "static scratch" in pkg.tsm2_get_last_error_string()


def test_noalloc_allocates_no_device_memory():
    """The defining property: after one warm-up call has loaded the library's
    device code, calls on a stream the library has never seen (tsm2r_s would
    allocate a workspace for it) leave the device's free memory unchanged."""
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    lib = pkg.lib()
    m, n, k = 10240, 10240, 16  # row blocks split between thread blocks: scratch needed
    A = ti.uniform_pm1(2, ti.MID_A, m, n, np.float32)
    B = ti.uniform_pm1(2, ti.MID_B, n, k, np.float32)
    dA, dB = DevMat(A), DevMat(B)
    out = DevMat(np.zeros((m, k), np.float32))
    assert lib.tsm2r_s_noalloc(m, n, k, dA.ptr, m, dB.ptr, n, out.ptr, m, 0) == 0
    torch.cuda.synchronize()
    fresh = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        st = lib.tsm2r_s_noalloc(m, n, k, dA.ptr, m, dB.ptr, n, out.ptr, m, fresh.cuda_stream)
        assert st == 0, pkg.tsm2_get_last_error_string()
    fresh.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    assert pkg.tsm2_get_device_status(0) == 0
    assert_parity(out.numpy(), A, B, np.float32)
