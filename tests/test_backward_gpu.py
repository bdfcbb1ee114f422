"""Backward products of C = A B on the GPU: dB = A^T dC (tsm2r_t) and
dA = dC B^T (tsm2_rankk), against the CPU oracle (the plain product
definition applied to transposed views), finite differences and torch."""
import numpy as np
import pytest

import oracle
import tsm2_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import DevMat, assert_parity  # noqa: E402

MID_DC = ti.MID_DC


@pytest.fixture(autouse=True)
def _defaults():
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    yield
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)


def pad16(x, dtype):
    v = 16 // np.dtype(dtype).itemsize
    return (max(x, 1) + v - 1) // v * v


def run_t(dtype, m, n, k, lda=None, lddc=None, lddb=None, offA=0, gen=ti.uniform_pm1):
    import paper_2002_03258_gb300 as pkg
    A = gen(1, ti.MID_A, m, n, dtype)
    dC = gen(1, MID_DC, m, k, dtype)
    dA_, dD = DevMat(A, lda, offA), DevMat(dC, lddc)
    out = DevMat(np.full((n, k), np.nan, dtype), lddb, fill=-5.0)
    fn = pkg.tsm2r_t_d if dtype == np.float64 else pkg.tsm2r_t_s
    st = fn(m, n, k, dA_.ptr, dA_.ld, dD.ptr, dD.ld, out.ptr, out.ld, 0)
    assert st == 0, pkg.tsm2_get_last_error_string()
    torch.cuda.synchronize()
    assert pkg.tsm2_get_device_status(0) == 0
    assert np.all(out.padding() == -5.0)
    return out.numpy(), A, dC, pkg.tsm2_last_config()


T_SHAPES = [(1, 1, 1), (100, 37, 3), (1000, 1023, 8), (4097, 300, 16), (2048, 64, 17), (30000, 100, 8),
            (257, 4000, 2), (5000, 31, 33)]


@pytest.mark.parametrize("padded", [False, True])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("m,n,k", T_SHAPES)
def test_tsm2r_t_parity(m, n, k, dtype, padded):
    if padded:
        got, A, dC, cfg = run_t(dtype, m, n, k, lda=pad16(m, dtype), lddc=pad16(m, dtype), lddb=pad16(n, dtype))
        assert cfg.startswith("t_"), cfg
    else:
        got, A, dC, cfg = run_t(dtype, m, n, k)
    assert_parity(got, A.T, dC, dtype)  # oracle on the transposed view


@pytest.mark.parametrize("grid", [1, 5, 77])
def test_tsm2r_t_any_grid(grid):
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_grid(grid)
    got, A, dC, cfg = run_t(np.float32, 6000, 700, 8, lda=6000, lddc=6000)
    assert cfg.startswith("t_")
    assert_parity(got, A.T, dC, np.float32)


def test_tsm2r_t_misaligned_elementwise_path():
    got, A, dC, cfg = run_t(np.float64, 999, 77, 5, lda=1001, lddc=1003, offA=1)
    assert cfg.startswith("simple_t"), cfg
    assert_parity(got, A.T, dC, np.float64)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_tsm2r_t_identity_and_integers(dtype):
    import paper_2002_03258_gb300 as pkg
    n, k = 1024, 8
    A = np.eye(n, dtype=dtype, order="F")
    dC = ti.uniform_pm1(2, MID_DC, n, k, dtype)
    dA_, dD, out = DevMat(A), DevMat(dC), DevMat(np.zeros((n, k), dtype))
    fn = pkg.tsm2r_t_d if dtype == np.float64 else pkg.tsm2r_t_s
    assert fn(n, n, k, dA_.ptr, n, dD.ptr, n, out.ptr, n, 0) == 0
    assert np.array_equal(out.numpy(), dC)  # A = I gives dB = dC exactly
    got, A, dC, _ = run_t(dtype, 8192, 520, 16, lda=8192, lddc=8192, gen=ti.int_small)
    assert_parity(got, A.T, dC, dtype, exact=True)


def run_rankk(dtype, m, n, k, lddc=None, ldb=None, ldda=None, gen=ti.uniform_pm1):
    import paper_2002_03258_gb300 as pkg
    dC = gen(3, MID_DC, m, k, dtype)
    B = gen(3, ti.MID_B, n, k, dtype)
    dD, dB_ = DevMat(dC, lddc), DevMat(B, ldb)
    out = DevMat(np.full((m, n), np.nan, dtype), ldda, fill=-5.0)
    fn = pkg.tsm2_rankk_d if dtype == np.float64 else pkg.tsm2_rankk_s
    st = fn(m, n, k, dD.ptr, dD.ld, dB_.ptr, dB_.ld, out.ptr, out.ld, 0)
    assert st == 0, pkg.tsm2_get_last_error_string()
    torch.cuda.synchronize()
    assert np.all(out.padding() == -5.0)
    return out.numpy(), dC, B


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("m,n,k,ld", [(1, 1, 1, None), (1000, 300, 8, None), (1025, 67, 16, 1032),
                                      (4099, 129, 3, None), (777, 65, 40, 780), (2048, 2048, 8, None)])
def test_rankk_parity(m, n, k, ld, dtype):
    got, dC, B = run_rankk(dtype, m, n, k, ldda=ld)
    assert_parity(got, dC, B.T, dtype)


def test_rankk_integers_exact_and_zero_k():
    import paper_2002_03258_gb300 as pkg
    got, dC, B = run_rankk(np.float32, 3000, 500, 12, gen=ti.int_small)
    assert_parity(got, dC, B.T, np.float32, exact=True)
    out = DevMat(np.full((10, 7), np.nan))
    assert pkg.tsm2_rankk_d(10, 7, 0, out.ptr, 10, out.ptr, 7, out.ptr, 10, 0) == 0
    torch.cuda.synchronize()
    assert np.all(out.numpy() == 0.0)


def test_finite_differences_fp64():
    """L = <dC, A B> is bilinear, so central differences have no truncation
    error: dL/dB and dL/dA must match the backward kernels to rounding."""
    import paper_2002_03258_gb300 as pkg
    m = n = 256
    k = 8
    h = 1e-6
    scale = 1.0 / np.sqrt(n)
    A = ti.normal_ih(0, ti.MID_A, m, n, scale)
    B = ti.normal_ih(0, ti.MID_B, n, k, scale)
    dC = ti.normal_ih(0, MID_DC, m, k, 1.0)
    tA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    tB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()
    tdC = torch.from_numpy(np.ascontiguousarray(dC.T)).cuda().t()
    C = pkg.empty_colmajor(m, k, torch.float64, "cuda")

    def loss():
        pkg.check(pkg.tsm2r_d(m, n, k, tA.data_ptr(), m, tB.data_ptr(), n, C.data_ptr(), m, 0))
        return float((C * tdC).sum())

    dB = pkg.tsm2r_t(tA, tdC).cpu().numpy()
    dA = pkg.rankk(tdC, tB).cpu().numpy()
    # every entry of B
    for j in range(n):
        for c in range(k):
            old = tB[j, c].item()
            tB[j, c] = old + h
            lp = loss()
            tB[j, c] = old - h
            lm = loss()
            tB[j, c] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - dB[j, c]) <= 1e-7 * (1 + abs(dB[j, c])), (j, c, fd, dB[j, c])
    # 4096 sampled entries of A
    rng = np.random.default_rng(7)
    for idx in rng.integers(0, m * n, 4096):
        i, j = int(idx % m), int(idx // m)
        old = tA[i, j].item()
        tA[i, j] = old + h
        lp = loss()
        tA[i, j] = old - h
        lm = loss()
        tA[i, j] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - dA[i, j]) <= 1e-7 * (1 + abs(dA[i, j])), (i, j, fd, dA[i, j])


def test_autograd_function_matches_torch():
    from paper_2002_03258_gb300.autograd import tsm2r_mm
    m, n, k = 3000, 2000, 8
    A64 = torch.from_numpy(np.ascontiguousarray(ti.uniform_pm1(4, ti.MID_A, m, n).T)).cuda().t()
    B64 = torch.from_numpy(np.ascontiguousarray(ti.uniform_pm1(4, ti.MID_B, n, k).T)).cuda().t()
    W = torch.from_numpy(ti.uniform_pm1(4, MID_DC, m, k)).cuda()
    for dt, tol in ((torch.float64, 1e-10), (torch.float32, 1e-3)):
        A = A64.detach().clone().to(dt).requires_grad_(True)  # clone keeps the column-major strides
        B = B64.detach().clone().to(dt).requires_grad_(True)
        assert A.is_leaf and A.stride(0) == 1
        (tsm2r_mm(A, B) * W.to(dt)).sum().backward()
        Ar = A64.detach().clone().requires_grad_(True)
        Br = B64.detach().clone().requires_grad_(True)
        (Ar @ Br * W).sum().backward()
        torch.testing.assert_close(A.grad.double(), Ar.grad, rtol=tol, atol=tol)
        torch.testing.assert_close(B.grad.double(), Br.grad, rtol=tol, atol=tol)


def test_config3_fullsize_sampled():
    """16384 x 16384 x 8 binary32, N(0, 1/n) inputs generated on the device:
    sampled rows of dB and dA against the oracle (host-regenerated inputs)."""
    import paper_2002_03258_gb300 as pkg
    lib = pkg.lib()
    m = n = 16384
    k = 8
    scale = 1.0 / np.sqrt(n)
    A = torch.empty((n, m), dtype=torch.float32, device="cuda").t()
    B = torch.empty((k, n), dtype=torch.float32, device="cuda").t()
    dC = torch.empty((k, m), dtype=torch.float32, device="cuda").t()
    assert lib.tsm2_fill_normal_ih_s(m, n, 0, ti.MID_A, scale, A.data_ptr(), m, 0) == 0
    assert lib.tsm2_fill_normal_ih_s(n, k, 0, ti.MID_B, scale, B.data_ptr(), n, 0) == 0
    assert lib.tsm2_fill_normal_ih_s(m, k, 0, MID_DC, 1.0, dC.data_ptr(), m, 0) == 0
    dB = pkg.tsm2r_t(A, dC)
    dA = pkg.rankk(dC, B)
    torch.cuda.synchronize()
    assert pkg.tsm2_get_device_status(0) == 0
    Bh = ti.normal_ih(0, ti.MID_B, n, k, scale, np.float32)
    dCh = ti.normal_ih(0, MID_DC, m, k, 1.0, np.float32)
    assert np.array_equal(B.cpu().numpy(), Bh)
    cols = np.array([0, 1, 255, 256, 8191, 16383, 777, 12345])
    Acols = ti.normal_ih(0, ti.MID_A, m, n, scale, np.float32, col_idx=cols)  # m x len(cols)
    assert_parity(dB.cpu().numpy()[cols], Acols.T, dCh, np.float32)
    rows = np.array([0, 5, 1023, 1024, 16383, 9999])
    assert_parity(dA.cpu().numpy()[rows], dCh[rows], Bh.T, np.float32)
