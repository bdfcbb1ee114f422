"""Parity at the benchmark's full sizes, in the configuration the benchmark
times: inputs are generated in device memory by the library's generator, and
the oracle recomputes sampled rows of C from the host-side generator (the
counter-based stream lets it draw any row of A on its own).  Sampled rows
include the first and last rows and rows on both sides of row-block edges."""
import numpy as np
import pytest

import tsm2_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import assert_parity  # noqa: E402

TDT = {np.float64: torch.float64, np.float32: torch.float32}


def sample_rows(m, count=40, seed=123):
    rng = np.random.default_rng(seed)
    rows = set(int(x) for x in rng.integers(0, m, count))
    for edge in (0, 127, 128, 255, 256, 511, 512, 1023, 1024, m - 1, m - 2, m // 2):
        if 0 <= edge < m:
            rows.add(edge)
    return np.array(sorted(rows))


def device_matrix(rows, cols, dtype, seed, mid, dist="uniform"):
    import paper_2002_03258_gb300 as pkg
    t = torch.empty((cols, rows), dtype=TDT[dtype], device="cuda").t()
    suffix = "d" if dtype == np.float64 else "s"
    fn = getattr(pkg.lib(), f"tsm2_fill_{dist}_{suffix}")
    assert fn(rows, cols, seed, mid, t.data_ptr(), rows, 0) == 0
    return t


@pytest.mark.parametrize("op,dtype,m,n,k,dist", [
    ("r", np.float32, 30720, 30720, 16, "uniform"),
    ("r", np.float32, 10240, 10240, 2, "uniform"),
    ("r", np.float32, 20480, 20480, 8, "int_small"),
    ("r", np.float64, 30720, 30720, 16, "uniform"),
    ("r", np.float64, 10240, 10240, 4, "int_small"),
    ("l", np.float32, 2 ** 23, 32, 32, "uniform"),
    ("l", np.float32, 2 ** 20, 8, 8, "int_small"),
    ("l", np.float64, 2 ** 23, 16, 16, "uniform"),
    ("l", np.float64, 2 ** 20, 32, 32, "uniform"),
    # tall A: the 8-rows-per-lane TSM2L schedule for k chunks of 17..32
    # columns, row blocks claimed at run time for narrower ones
    ("l", np.float32, 3_000_000, 8, 8, "uniform"),
    ("l", np.float32, 3_000_000, 16, 16, "uniform"),
    ("l", np.float32, 3_000_000, 20, 20, "int_small"),
    ("l", np.float32, 3_000_000, 32, 32, "uniform"),
    # 16 C columns per lane (k chunk 25..32): ragged rows, inner dimension
    # and columns, so the second column warp stores through the predicated path
    ("l", np.float32, 1_000_004, 30, 29, "uniform"),
])
def test_fullsize_sampled_rows(op, dtype, m, n, k, dist):
    import paper_2002_03258_gb300 as pkg
    seed = 0
    A = device_matrix(m, n, dtype, seed, ti.MID_A, dist)
    B = device_matrix(n, k, dtype, seed, ti.MID_B, dist)
    C = torch.full((k, m), float("nan"), dtype=TDT[dtype], device="cuda").t()
    fn = getattr(pkg, {("r", np.float64): "tsm2r_d", ("r", np.float32): "tsm2r_s",
                       ("l", np.float64): "tsm2l_d", ("l", np.float32): "tsm2l_s"}[(op, dtype)])
    st = fn(m, n, k, A.data_ptr(), m, B.data_ptr(), n, C.data_ptr(), m, 0)
    assert st == 0, pkg.tsm2_get_last_error_string()
    assert pkg.tsm2_get_device_status(0) == 0
    cfg = pkg.tsm2_last_config()
    assert not cfg.startswith("simple")
    if op == "l" and dtype == np.float32 and m in (3_000_000, 1_000_004):
        assert cfg.startswith("lw_" if k > 16 else "l_f32"), cfg
    rows = sample_rows(m)
    got = C[torch.from_numpy(rows).cuda()].cpu().numpy()
    gen = {"uniform": ti.uniform_pm1, "int_small": ti.int_small}[dist]
    A_rows = gen(seed, ti.MID_A, m, n, dtype, row_idx=rows)
    B_host = gen(seed, ti.MID_B, n, k, dtype)
    assert np.array_equal(B.cpu().numpy(), B_host)  # the two generators agree
    assert_parity(got, A_rows, B_host, dtype, exact=(dist == "int_small"))
    # whole-C property at any size: every entry finite and within |A||B| <= n max|a| max|b|
    assert bool(torch.isfinite(C).all())
    assert float(C.abs().max()) <= n * 1.0 * 1.0 * (4 * 4 if dist == "int_small" else 1)
