"""GPU parity: every kernel path against the CPU oracle, through the C ABI.

Sizes span several row blocks and pipeline stages with ragged tails in every
dimension; the bound is the componentwise 2 gamma_n(u) |A||B| (both sides'
rounding), exact equality where the inputs make the product exact.
"""
import numpy as np
import pytest

import oracle
import tsm2_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import DevMat, assert_parity, call  # noqa: E402


@pytest.fixture(autouse=True)
def _defaults():
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    pkg.tsm2_set_wait_budget_ns(1_000_000_000)
    yield
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    pkg.tsm2_set_wait_budget_ns(1_000_000_000)


def run(op, dtype, m, n, k, lda=None, ldb=None, ldc=None, offA=0, offB=0, offC=0, gen=ti.uniform_pm1, seed=0):
    import paper_2002_03258_gb300 as pkg
    A = gen(seed, ti.MID_A, m, n, dtype)
    B = gen(seed, ti.MID_B, n, k, dtype)
    dA = DevMat(A, lda, offA)
    dB = DevMat(B, ldb, offB)
    dC = DevMat(np.full((m, k), np.nan, dtype=dtype), ldc, offC, fill=-7.0)
    st = call(op, dtype, m, n, k, dA, dB, dC)
    assert st == 0, pkg.tsm2_get_last_error_string()
    torch.cuda.synchronize()
    assert pkg.tsm2_get_device_status(0) == 0
    got = dC.numpy()
    # rows m..ldc-1 and everything around C untouched
    pad = dC.padding()
    assert np.all(pad == -7.0), "C written outside its m x k extent"
    return got, A, B, pkg.tsm2_last_config()


R_SHAPES = [
    (1, 1, 1), (31, 33, 3), (257, 100, 2), (1000, 1023, 8), (1023, 1000, 16), (2049, 777, 5),
    (300, 5000, 4), (4097, 300, 17), (10241, 64, 7), (128, 4096, 16), (5000, 31, 33),
    (3001, 2000, 12), (1000, 777, 10), (2500, 1500, 28),
]
L_SHAPES = [
    (100003, 8, 8), (65537, 16, 16), (33333, 32, 32), (1000, 3, 5), (5000, 64, 64), (777, 33, 40),
    (1, 1, 1), (4096, 24, 2), (70001, 17, 9),
    (500001, 24, 24), (300000, 20, 20), (30000, 12, 12), (40000, 11, 9), (2000001, 12, 12),
    (1000005, 32, 29),
]


def pad16(x, dtype):
    v = 16 // np.dtype(dtype).itemsize
    return (max(x, 1) + v - 1) // v * v


@pytest.mark.parametrize("padded", [False, True])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("m,n,k", R_SHAPES)
def test_tsm2r_parity(m, n, k, dtype, padded):
    if padded:  # 16-byte row strides: the bulk-copy path, with ragged tails in m, n, k
        got, A, B, cfg = run("r", dtype, m, n, k, lda=pad16(m, dtype), ldb=pad16(n, dtype), ldc=pad16(m, dtype))
        assert not cfg.startswith("simple"), cfg
    else:
        got, A, B, cfg = run("r", dtype, m, n, k)
    assert_parity(got, A, B, dtype)


@pytest.mark.parametrize("padded", [False, True])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("m,n,k", L_SHAPES)
def test_tsm2l_parity(m, n, k, dtype, padded):
    if padded:
        got, A, B, cfg = run("l", dtype, m, n, k, lda=pad16(m, dtype), ldc=pad16(m, dtype))
        assert not cfg.startswith("simple"), cfg
    else:
        got, A, B, cfg = run("l", dtype, m, n, k)
    assert_parity(got, A, B, dtype)


@pytest.mark.parametrize("op", ["r", "l"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_padded_leading_dimensions(op, dtype):
    m, n, k = (3001, 45, 12) if op == "l" else (1500, 1300, 12)
    got, A, B, cfg = run(op, dtype, m, n, k, lda=pad16(m, dtype) + 8, ldb=pad16(n, dtype) + 4, ldc=m + 12)
    assert_parity(got, A, B, dtype)
    assert not cfg.startswith("simple"), cfg


@pytest.mark.parametrize("op", ["r", "l"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_misaligned_operands_take_elementwise_path(op, dtype):
    m, n, k = (1001, 37, 6) if op == "l" else (1001, 999, 6)
    got, A, B, cfg = run(op, dtype, m, n, k, lda=m + 1, ldb=n + 1, ldc=m + 3, offA=1, offB=1, offC=1)
    assert_parity(got, A, B, dtype)
    assert cfg.startswith("simple"), cfg


@pytest.mark.parametrize("op", ["r", "l"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_unaligned_c_only(op, dtype):
    m, n, k = 2003, 40, 9
    got, A, B, cfg = run(op, dtype, m, n, k, lda=pad16(m, dtype), ldb=pad16(n, dtype), ldc=m + 1, offC=1)
    assert_parity(got, A, B, dtype)
    assert not cfg.startswith("simple"), cfg  # only C unaligned: scalar stores on the bulk path


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_forced_paths(path, dtype):
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(path)
    got, A, B, cfg = run("r", dtype, 777, 1500, 10, lda=pad16(777, dtype), ldb=1500, ldc=777)
    assert_parity(got, A, B, dtype)
    assert cfg.startswith("simple") == (path == 1)


@pytest.mark.parametrize("op", ["r", "l"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_identity_gives_b_exactly(op, dtype):
    import paper_2002_03258_gb300 as pkg
    n, k = (32, 32) if op == "l" else (1100, 16)
    A = np.eye(n, dtype=dtype, order="F")
    B = ti.uniform_pm1(3, ti.MID_B, n, k, dtype)
    dA, dB = DevMat(A), DevMat(B)
    dC = DevMat(np.full((n, k), np.nan, dtype))
    assert call(op, dtype, n, n, k, dA, dB, dC) == 0, pkg.tsm2_get_last_error_string()
    assert np.array_equal(dC.numpy(), B)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_all_ones_rows_bitwise_equal(dtype):
    import paper_2002_03258_gb300 as pkg
    m, n, k = 700, 5003, 16
    A = np.ones((m, n), dtype=dtype, order="F")
    B = ti.uniform_pm1(4, ti.MID_B, n, k, dtype)
    dA, dB, dC = DevMat(A), DevMat(B), DevMat(np.zeros((m, k), dtype))
    assert call("r", dtype, m, n, k, dA, dB, dC) == 0, pkg.tsm2_get_last_error_string()
    got = dC.numpy()
    assert np.all(got == got[0:1, :])
    assert_parity(got, A, B, dtype)


@pytest.mark.parametrize("op", ["r", "l"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_small_integers_bit_exact(op, dtype):
    m, n, k = (50001, 32, 32) if op == "l" else (3001, 4099, 16)
    got, A, B, cfg = run(op, dtype, m, n, k, lda=pad16(m, dtype), ldb=pad16(n, dtype), ldc=pad16(m, dtype),
                         gen=ti.int_small, seed=5)
    assert not cfg.startswith("simple"), cfg
    assert_parity(got, A, B, dtype, exact=True)


def test_permutation_rows():
    import paper_2002_03258_gb300 as pkg
    n, k = 2048, 8
    perm = np.argsort(ti.uniform_pm1(9, 99, n, 1)[:, 0])
    P = np.zeros((n, n), order="F")
    P[np.arange(n), perm] = 1.0
    B = ti.uniform_pm1(9, ti.MID_B, n, k)
    dA, dB, dC = DevMat(P), DevMat(B), DevMat(np.zeros((n, k)))
    assert call("r", np.float64, n, n, k, dA, dB, dC) == 0, pkg.tsm2_get_last_error_string()
    assert np.array_equal(dC.numpy(), B[perm, :])


@pytest.mark.parametrize("op", ["r", "l"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_deterministic(op, dtype):
    m, n, k = (40000, 32, 16) if op == "l" else (2500, 20000, 16)
    g1, A, B, _ = run(op, dtype, m, n, k)
    g2, _, _, _ = run(op, dtype, m, n, k)
    assert g1.tobytes() == g2.tobytes()


@pytest.mark.parametrize("grid", [1, 3, 7, 40, 151])
def test_any_grid_size(grid):
    """The stream-K partition must cover every unit once for any block count."""
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_grid(grid)
    got, A, B, cfg = run("r", np.float32, 1537, 3001, 16, lda=1540, ldb=3004, ldc=1540)
    assert not cfg.startswith("simple"), cfg
    assert_parity(got, A, B, np.float32)
    got, A, B, cfg = run("r", np.float64, 1537, 3001, 13, lda=1538, ldb=3002, ldc=1537)
    assert not cfg.startswith("simple"), cfg
    assert_parity(got, A, B, np.float64)
    got, A, B, cfg = run("l", np.float64, 20001, 24, 24, lda=20002)
    assert not cfg.startswith("simple"), cfg
    assert_parity(got, A, B, np.float64)


def test_nan_and_inf_propagate():
    import paper_2002_03258_gb300 as pkg
    m, n, k = 600, 900, 4
    A = ti.uniform_pm1(1, ti.MID_A, m, n)
    B = ti.uniform_pm1(1, ti.MID_B, n, k)
    A[17, 400] = np.nan
    B[3, 2] = np.inf
    dA, dB, dC = DevMat(A), DevMat(B), DevMat(np.zeros((m, k)))
    assert call("r", np.float64, m, n, k, dA, dB, dC) == 0, pkg.tsm2_get_last_error_string()
    assert_parity(dC.numpy(), A, B, np.float64)


@pytest.mark.parametrize("op", ["r", "l"])
def test_empty_inner_dimension_zero_fills(op):
    import paper_2002_03258_gb300 as pkg
    m, k = 100, 5
    dA = DevMat(np.zeros((m, 1)))
    dB = DevMat(np.zeros((1, k)))
    dC = DevMat(np.full((m, k), np.nan))
    fn = getattr(pkg, "tsm2r_d" if op == "r" else "tsm2l_d")
    assert fn(m, 0, k, dA.ptr, m, dB.ptr, 1, dC.ptr, m, 0) == 0
    torch.cuda.synchronize()
    assert np.all(dC.numpy() == 0.0)


def test_timeout_path_reports_and_recovers():
    """Force every pipeline wait to a single attempt: the kernel must give up,
    flag the status word and return; the next normal call must be correct."""
    import paper_2002_03258_gb300 as pkg
    m, n, k = 4096, 8192, 16
    A = ti.uniform_pm1(2, ti.MID_A, m, n, np.float32)
    B = ti.uniform_pm1(2, ti.MID_B, n, k, np.float32)
    dA, dB, dC = DevMat(A), DevMat(B), DevMat(np.zeros((m, k), np.float32))
    pkg.tsm2_set_wait_budget_ns(0)
    assert call("r", np.float32, m, n, k, dA, dB, dC) == 0
    st = pkg.tsm2_get_device_status(0)
    pkg.tsm2_set_wait_budget_ns(1_000_000_000)
    assert st == pkg.ERR_TIMEOUT
    assert pkg.tsm2_get_device_status(0) == 0  # cleared
    assert call("r", np.float32, m, n, k, dA, dB, dC) == 0
    assert pkg.tsm2_get_device_status(0) == 0
    assert_parity(dC.numpy(), A, B, np.float32)


def test_streams_and_torch_wrappers():
    import paper_2002_03258_gb300 as pkg
    s = torch.cuda.Stream()
    A = ti.uniform_pm1(6, ti.MID_A, 3000, 2000, np.float32)
    B = ti.uniform_pm1(6, ti.MID_B, 2000, 8, np.float32)
    tA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    tB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()
    with torch.cuda.stream(s):
        C = pkg.tsm2r(tA, tB)
    s.synchronize()
    assert_parity(C.cpu().numpy(), A, B, np.float32)
    with pytest.raises(ValueError):
        pkg.tsm2r(tA.t().contiguous(), tB)  # row-major operand rejected


@pytest.mark.parametrize("dist", ["uniform", "int_small", "normal_ih"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_device_generator_matches_host_bitwise(dist, dtype):
    import ctypes
    import paper_2002_03258_gb300 as pkg
    rows, cols, ld = 1001, 37, 1003
    host = {"uniform": ti.uniform_pm1, "int_small": ti.int_small,
            "normal_ih": lambda s, mid, r, c, d: ti.normal_ih(s, mid, r, c, 0.25, d)}[dist](7, 11, rows, cols, dtype)
    d = DevMat(np.zeros((rows, cols), dtype), ld)
    suffix = "d" if dtype == np.float64 else "s"
    fn = getattr(pkg.lib(), f"tsm2_fill_{dist}_{suffix}")
    if dist == "normal_ih":
        st = fn(rows, cols, 7, 11, ctypes.c_double(0.25), d.ptr, ld, 0)
    else:
        st = fn(rows, cols, 7, 11, d.ptr, ld, 0)
    assert st == 0
    torch.cuda.synchronize()
    assert np.array_equal(d.numpy(), host)
    assert np.all(np.isnan(d.padding()[:5]))  # padding untouched


def test_device_logmag_matches_host_bitwise():
    import paper_2002_03258_gb300 as pkg
    rows, cols = 513, 29
    host = ti.logmag(3, 4, rows, cols, np.float32)
    d = DevMat(np.zeros((rows, cols), np.float32))
    assert pkg.lib().tsm2_fill_logmag_s(rows, cols, 3, 4, d.ptr, rows, 0) == 0
    torch.cuda.synchronize()
    assert np.array_equal(d.numpy(), host)
