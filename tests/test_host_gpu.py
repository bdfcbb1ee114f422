"""Host-resident operands (tsm2r_*_host, tsm2l_*_host): the row-chunk
pipeline against the CPU oracle, with pinned and pageable host buffers,
padded leading dimensions, several chunks and a ragged last chunk."""
import ctypes

import numpy as np
import pytest

import oracle
import tsm2_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import assert_parity  # noqa: E402


def host_colmajor(a, ld, pinned, fill=np.nan):
    """Column-major host buffer (ld x cols) holding `a`; returns (tensor, ptr)."""
    rows, cols = a.shape
    t = torch.empty((cols, ld), dtype=torch.from_numpy(a[:1, :1].copy()).dtype, pin_memory=pinned)
    t.fill_(fill)
    t.t()[:rows].copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t, t.data_ptr()


@pytest.fixture
def copy_mode(request):
    """Selects the host copy path (0: SM copy kernels, 1: copy engines) for
    one test and restores the default afterwards."""
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_host_copy(request.param)
    yield request.param
    pkg.tsm2_set_host_copy(0)


def run_host(op, dtype, m, n, k, lda=None, ldb=None, ldc=None, pinned=True, rows=None, expect_copy=None):
    import paper_2002_03258_gb300 as pkg
    lda, ldb, ldc = lda or m, ldb or n, ldc or m
    full = rows is None
    ridx = None if full else np.asarray(rows)
    B = ti.uniform_pm1(7, ti.MID_B, n, k, dtype)
    tB, pB = host_colmajor(B, ldb, pinned)
    if full:
        A = ti.uniform_pm1(7, ti.MID_A, m, n, dtype)
        tA, pA = host_colmajor(A, lda, pinned)
    else:
        # Large A: generated by the device fill (same definition), copied to
        # the host buffer; the oracle regenerates the sampled rows itself.
        tdt = torch.float32 if dtype == np.float32 else torch.float64
        dA = torch.empty((n, lda), dtype=tdt, device="cuda")
        fill = getattr(pkg.lib(), "tsm2_fill_uniform_" + ("s" if dtype == np.float32 else "d"))
        assert fill(m, n, 7, ti.MID_A, dA.data_ptr(), lda, 0) == 0
        tA = torch.empty((n, lda), dtype=tdt, pin_memory=pinned)
        tA.copy_(dA)
        del dA
        pA = tA.data_ptr()
        A = ti.uniform_pm1(7, ti.MID_A, m, n, dtype, row_idx=ridx)
    tC = torch.full((k, ldc), -7.0, dtype=tA.dtype, pin_memory=pinned)
    suf = "s" if dtype == np.float32 else "d"
    fn = getattr(pkg, f"tsm2{op}_{suf}_host")
    s = torch.cuda.Stream()
    st = fn(m, n, k, pA, lda, pB, ldb, tC.data_ptr(), ldc, s.cuda_stream)
    assert st == 0, pkg.tsm2_get_last_error_string()
    if expect_copy is not None:
        assert pkg.tsm2_last_host_copy() == expect_copy
    s.synchronize()
    assert pkg.tsm2_get_device_status(0) == 0
    C = tC.numpy().T  # ldc x k
    assert np.all(C[m:] == -7.0), "rows beyond m of C must stay untouched"
    if full:
        return C[:m], A, B
    return C[ridx], A, B


SM = "A:sm B:sm C:sm"
ENGINE = "A:engine B:engine C:engine"


@pytest.mark.parametrize("pinned,copy_mode", [(True, 0), (True, 1), (False, 0)], indirect=["copy_mode"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("op,m,n,k", [("r", 1000, 777, 5), ("r", 4099, 2048, 16), ("r", 300, 4100, 20),
                                      ("l", 100003, 16, 16), ("l", 5000, 33, 7)])
def test_host_entry_single_chunk(op, m, n, k, dtype, pinned, copy_mode):
    # Page-locked buffers take the SM copy kernels unless the copy engines
    # are selected; pageable ones always take the copy engines.
    C, A, B = run_host(op, dtype, m, n, k, pinned=pinned, expect_copy=SM if pinned and copy_mode == 0 else ENGINE)
    assert_parity(C, A, B, dtype)


@pytest.mark.parametrize("copy_mode", [0, 1], indirect=True)
def test_host_entry_padded_leading_dimensions(copy_mode):
    # Leading dimensions that are not multiples of 16 bytes: the copy kernels'
    # 4-byte path.
    C, A, B = run_host("r", np.float32, 1500, 900, 9, lda=1537, ldb=901, ldc=1503,
                       expect_copy=SM if copy_mode == 0 else ENGINE)
    assert_parity(C, A, B, np.float32)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("m,lda", [(1001, 1004), (1003, 1004), (5, 8), (1, 4)])
def test_host_entry_vector_copy_with_tail(m, lda, dtype):
    # 16-byte aligned columns whose height is not a multiple of 16 bytes: the
    # copy kernels' 16-byte body plus 4-byte tail, in A, B and C.
    es = np.dtype(dtype).itemsize
    lda = lda if es == 4 else (m + 1) // 2 * 2
    for op, n, k in (("r", 2047, 13), ("l", 31, 31)):
        C, A, B = run_host(op, dtype, m, n, k, lda=lda, ldb=(n + 3) // 4 * 4 if es == 4 else (n + 1) // 2 * 2,
                           ldc=lda, expect_copy=SM)
        assert_parity(C, A, B, dtype)


@pytest.mark.parametrize("copy_mode", [1], indirect=True)
def test_host_copy_mode_selects_copy_engines(copy_mode):
    C, A, B = run_host("l", np.float32, 70001, 24, 24, expect_copy=ENGINE)
    assert_parity(C, A, B, np.float32)


def test_host_entry_several_chunks_tsm2r():
    # 40000 x 8192 binary32: chunks of 16384 rows (64 KiB column pieces), the
    # last one ragged (7232 rows); sampled rows from every chunk.
    rows = [0, 1, 16383, 16384, 20000, 32767, 32768, 39999]
    C, Ar, B = run_host("r", np.float32, 40000, 8192, 16, rows=rows)
    assert_parity(C, Ar, B, np.float32)


def test_host_entry_several_chunks_tsm2l():
    # 3000001 x 32 binary32: chunks of 2^21 rows, the last one ragged.
    rows = [0, 5, 2097151, 2097152, 2999999, 3000000]
    C, Ar, B = run_host("l", np.float32, 3000001, 32, 32, rows=rows)
    assert_parity(C, Ar, B, np.float32)


def test_host_entry_integers_exact_and_repeatable():
    import paper_2002_03258_gb300 as pkg
    m, n, k = 20000, 3000, 16
    A = ti.int_small(3, ti.MID_A, m, n, np.float32)
    B = ti.int_small(3, ti.MID_B, n, k, np.float32)
    tA, pA = host_colmajor(A, m, True)
    tB, pB = host_colmajor(B, n, True)
    outs = []
    for _ in range(2):
        tC = torch.empty((k, m), dtype=torch.float32, pin_memory=True)
        assert pkg.tsm2r_s_host(m, n, k, pA, m, pB, n, tC.data_ptr(), m, 0) == 0
        torch.cuda.synchronize()
        outs.append(tC.numpy().T.copy())
    ref = oracle.gemm(A.astype(np.float64), B.astype(np.float64))
    assert np.array_equal(outs[0].astype(np.float64), ref)
    assert np.array_equal(outs[0], outs[1])


def test_host_entry_edge_cases():
    import paper_2002_03258_gb300 as pkg
    tC = torch.full((3, 10), 5.0, dtype=torch.float32, pin_memory=True)
    tA = torch.ones(16, dtype=torch.float32, pin_memory=True)
    # n == 0: C = 0 (empty sum)
    assert pkg.tsm2r_s_host(10, 0, 3, tA.data_ptr(), 10, tA.data_ptr(), 1, tC.data_ptr(), 10, 0) == 0
    assert np.all(tC.numpy() == 0.0)
    # m == 0, k == 0: nothing touched
    tC.fill_(5.0)
    assert pkg.tsm2r_s_host(0, 4, 3, tA.data_ptr(), 1, tA.data_ptr(), 4, tC.data_ptr(), 1, 0) == 0
    assert pkg.tsm2r_s_host(10, 4, 0, tA.data_ptr(), 10, tA.data_ptr(), 4, tC.data_ptr(), 10, 0) == 0
    assert np.all(tC.numpy() == 5.0)
    # TSM2L with n > 64: B staged with A
    C, A, B = run_host("l", np.float32, 50000, 100, 20)
    assert_parity(C, A, B, np.float32)
