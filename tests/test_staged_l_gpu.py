"""TSM2L with B staged instead of resident (n > 64; the setting of Alg. 6):
parity with the CPU oracle, exactness on small integers, any grid size,
column chunks for k > 32, determinism."""
import numpy as np
import pytest

import tsm2_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import assert_parity  # noqa: E402
from test_parity_gpu import pad16, run  # noqa: E402


@pytest.fixture(autouse=True)
def _defaults():
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    yield
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)


STAGED_SHAPES = [
    (5000, 65, 8), (100003, 100, 16), (30001, 300, 32), (2049, 1000, 3), (70001, 129, 33), (10, 200, 64),
    (4096, 96, 1), (50000, 80, 100), (1, 65, 2), (30001, 300, 24), (5000, 100, 12),
]


@pytest.mark.parametrize("padded", [False, True])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("m,n,k", STAGED_SHAPES)
def test_staged_tsm2l_parity(m, n, k, dtype, padded):
    if padded:  # 16-byte strides: the staged bulk-copy schedule
        got, A, B, cfg = run("l", dtype, m, n, k, lda=pad16(m, dtype), ldb=pad16(n, dtype), ldc=pad16(m, dtype))
        assert cfg.startswith("lt_"), cfg
    else:
        got, A, B, cfg = run("l", dtype, m, n, k)
    assert_parity(got, A, B, dtype)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_staged_tsm2l_small_integers_exact(dtype):
    m, n, k = 40001, 200, 32
    got, A, B, cfg = run("l", dtype, m, n, k, lda=pad16(m, dtype), ldb=pad16(n, dtype), ldc=pad16(m, dtype),
                         gen=ti.int_small, seed=11)
    assert cfg.startswith("lt_"), cfg
    assert_parity(got, A, B, dtype, exact=True)


@pytest.mark.parametrize("grid", [1, 5, 151])
def test_staged_tsm2l_any_grid(grid):
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_grid(grid)
    got, A, B, cfg = run("l", np.float32, 20001, 150, 24, lda=20004, ldb=152, ldc=20004)
    assert cfg.startswith("lt_"), cfg
    assert_parity(got, A, B, np.float32)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_staged_tsm2l_deterministic(dtype):
    m, n, k = 30000, 256, 16
    g1, _, _, _ = run("l", dtype, m, n, k, lda=m, ldb=n, ldc=m)
    g2, _, _, _ = run("l", dtype, m, n, k, lda=m, ldb=n, ldc=m)
    assert g1.tobytes() == g2.tobytes()
