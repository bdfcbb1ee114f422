"""Pins for the paper's performance model against the values the paper prints."""
import os

import pytest

from paper_2002_03258_gb300 import perfmodel as pm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "t2_threshold_paper.txt")


def _rows():
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, perf, bw, printed = line.split()
            yield name, float(perf), float(bw), float(printed)


@pytest.mark.parametrize("name,perf,bw,printed", list(_rows()))
def test_t2_threshold_matches_printed(name, perf, bw, printed):
    t = pm.t2_threshold(perf, bw, 8)
    # The paper rounds to one significant figure ("~40", "~6", "~70").
    step = 10.0 if printed >= 10 else 1.0
    assert round(t / step) * step == printed, (name, t)
    # the table's peaks are the ones stored in the model
    g = pm.PAPER_GPUS_DOUBLE[name]
    assert (g.peak_gflops, g.bw_gbs) == (perf, bw)


def test_classifier_directions():
    # K40c, n = 2..16 all memory-bound (Sec. 4.2.1); M40 n = 16 compute-bound (Sec. 4.2.2)
    k40 = pm.PAPER_GPUS_DOUBLE["K40c"]
    m40 = pm.PAPER_GPUS_DOUBLE["M40"]
    for k in (2, 4, 8, 16):
        assert not pm.is_compute_bound(k, k40.peak_gflops, k40.bw_gbs, 8)
    assert pm.is_compute_bound(16, m40.peak_gflops, m40.bw_gbs, 8)
    # r = 1 exactly at the threshold
    t = pm.t2_threshold(m40.peak_gflops, m40.bw_gbs, 8)
    assert abs(pm.time_ratio(t, m40.peak_gflops, m40.bw_gbs, 8) - 1.0) < 1e-12


def test_a100_bandwidth_ratio_prediction():
    # Sec. 4.2.5: memory-bound everywhere on A100, so the predicted speed-up
    # over V100 is the bandwidth ratio, ~1.7x.
    a, v = pm.PAPER_GPUS_DOUBLE["A100"], pm.PAPER_GPUS_DOUBLE["V100"]
    assert round(a.bw_gbs / v.bw_gbs, 1) == 1.7
    for k in (2, 4, 8, 16):
        assert not pm.is_compute_bound(k, a.peak_gflops, a.bw_gbs, 8)


def test_register_and_occupancy_formulas():
    # R_thread = (3 t2 + 2 t3) * bytes/4 + C ; S_thread = t2 * bytes
    assert pm.regs_per_thread(16, 4, 8, c_setup=10) == (48 + 8) * 2 + 10
    assert pm.smem_per_thread(16, 8) == 128
    g = pm.Gpu("x", 1.0, 1.0, sms=1, clock_ghz=1.0, regs_per_sm=65536, smem_per_sm=98304, hw_max_threads=2048)
    assert pm.max_occupancy(g, 16, 4, 8) == min(2048, 65536 / 112, 98304 / 128)
