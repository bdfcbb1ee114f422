"""The derived bfloat16 bound is tight enough to see a lost pipeline stage.

A planted mistake lives in the oracle, on the CPU: for the sampled rows of
the 32768 x 32768 x 16 workload (log-uniform A magnitudes, uniform B), drop
one stage's inner columns from the oracle's product and check that some
sampled output then moves by more than the bound the GPU test asserts.
Every stage position is tried, for plain and hi+lo A.
"""
import numpy as np
import pytest

import bf16_bound as bb
import oracle
import tsm2_inputs as ti

SM_COUNT = 152  # a larger grid only loosens the bound; GB300 has 152 SMs


def split_host(X32):
    hi = oracle.bf16_rne(X32)
    r = (X32 - oracle.bf16_to_float(hi)).astype(np.float32)
    return hi, oracle.bf16_rne(r)


def test_bound_values_at_full_size():
    m = n = 32768
    plain = bb.tc_factor(m, n, False, SM_COUNT)
    hilo = bb.tc_factor(m, n, True, SM_COUNT)
    # the structure, not n, sets the tensor-core term; the carry grows with n/G
    assert 3e-5 < plain < 6e-5, plain
    assert 5e-5 < hilo < 9e-5, hilo
    # the old n-proportional bounds were hundreds of times looser
    assert plain < (2.0 ** -16 + 4 * n * 2.0 ** -23) / 200
    assert hilo < (2.0 ** -24 + 10 * n * 2.0 ** -23) / 400


def test_partials_bound():
    # one block per row block or more: at most two partials per row block
    assert bb.max_partials(32768, 32768, False, 152) <= 4
    assert bb.max_partials(512, 64, False, 1) == 1
    # a single-block grid: one partial
    assert bb.max_partials(10 ** 5, 10 ** 4, True, 1) == 1
    # more blocks than units: every unit its own partial
    assert bb.max_partials(512, 640, False, 1000) == 10


@pytest.mark.parametrize("hilo", [False, True])
def test_dropped_stage_exceeds_bound_config5(hilo):
    m = n = 32768
    k = 16
    rows = np.array(bb.CONFIG5_ROWS)
    X = ti.logmag(0, ti.MID_A, m, n, np.float32, row_idx=rows)
    B = ti.uniform_pm1(0, ti.MID_B, n, k, np.float32).astype(np.float64)
    hi, lo = split_host(np.asfortranarray(X))
    A = oracle.bf16_to_float(hi).astype(np.float64)
    if hilo:
        A = A + oracle.bf16_to_float(lo)
    A = np.asfortranarray(A)
    S = oracle.absgemm(A, B)
    bound = bb.tc_factor(m, n, hilo, SM_COUNT) * S
    worst = np.inf
    for j0, j1 in bb.stage_columns(n, hilo):
        lost = oracle.gemm(np.asfortranarray(A[:, j0:j1]), np.asfortranarray(B[j0:j1]))
        ratio = float(np.max(np.abs(lost) / bound))
        worst = min(worst, ratio)
        assert ratio > 1.0, (j0, ratio)
    # and with room to spare
    assert worst > 2.0, worst


def test_simple_path_bound_is_gamma_n():
    assert bb.simple_factor(1000) == pytest.approx(1000 * 2.0 ** -24, rel=1e-4)
    with pytest.raises(ValueError):
        bb.factor("tc_f32", 1, 1, False, 1)
