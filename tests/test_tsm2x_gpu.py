"""TSM2X (tsm2x_s / tsm2x_d): the shape-chosen schedule runs, and its
result agrees with the CPU oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import assert_parity  # noqa: E402
from test_parity_gpu import pad16, run  # noqa: E402


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("m,n,k", [(15360, 16, 16), (15360, 1024, 16), (300000, 8, 4), (300000, 200, 16),
                                   (4000, 3000, 20), (150000, 300, 33), (1, 1, 1)])
def test_tsm2x_parity_and_choice(m, n, k, dtype):
    import paper_2002_03258_gb300 as pkg
    es = np.dtype(dtype).itemsize
    want = pkg.tsm2x_choice(es, m, n, k)
    got, A, B, cfg = run("x", dtype, m, n, k, lda=pad16(m, dtype), ldb=pad16(n, dtype), ldc=pad16(m, dtype))
    assert_parity(got, A, B, dtype)
    if want == "r":
        assert cfg.startswith("r_"), (want, cfg)
    else:
        assert cfg.startswith("l"), (want, cfg)
