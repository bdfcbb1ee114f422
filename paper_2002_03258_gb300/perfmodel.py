"""The paper's analytic performance model for TSM2R (Sec. 3.1.8, "Performance
Metrics Estimation", and Algorithm 7), restated for use on any GPU.

Symbols follow the paper: t2 is the number of C columns a thread accumulates
at a time (``tile_size_C``), t3 the number of A elements fetched at a time
(``tile_size_A``), ``bytes`` the element size.  Peak performance is in
GFLOP/s and bandwidth in GB/s, as in the paper's platform table.

Two parts feed the library's batched tuner (``autotune.seed_candidate``):
the Little's-law estimate of bytes in flight per SM picks the seed tile
variant (the pipeline must keep that much of A in flight), and the
compute/memory classifier ``t2_threshold`` decides whether padding C columns
up to a wider class costs time in the model.  The occupancy estimate
(``max_occupancy``, ``util_mem``) is the paper's formula for thread-per-row
kernels and is kept for reference; the library's persistent kernels run one
block per SM by construction.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Gpu:
    name: str
    peak_gflops: float      # arithmetic peak in the precision considered
    bw_gbs: float           # peak DRAM bandwidth
    sms: int = 0
    clock_ghz: float = 0.0
    regs_per_sm: int = 65536
    smem_per_sm: int = 0
    hw_max_threads: int = 2048


def t2_threshold(peak_gflops: float, bw_gbs: float, bytes_per_elem: int) -> float:
    """Boundary value of t2 between memory- and compute-bound (Sec. 3.1.8):
    t2_threshold = PeakPerf / PeakBand * bytes_per_elem."""
    return peak_gflops / bw_gbs * bytes_per_elem


def time_ratio(t2: float, peak_gflops: float, bw_gbs: float, bytes_per_elem: int) -> float:
    """r = time_comp / time_mem = t2 / bytes * PeakBand / PeakPerf; r > 1 means
    the inner loop is compute-bound."""
    return t2 / bytes_per_elem * bw_gbs / peak_gflops


def is_compute_bound(k: int, peak_gflops: float, bw_gbs: float, bytes_per_elem: int) -> bool:
    """Whole-problem classification: with t2 fixed to the skinny width k, the
    problem is compute-bound when k exceeds the threshold."""
    return k > t2_threshold(peak_gflops, bw_gbs, bytes_per_elem)


def regs_per_thread(t2: int, t3: int, bytes_per_elem: int, bytes_per_reg: int = 4, c_setup: int = 0) -> float:
    """R_thread = (3 t2 + 2 t3) * bytes_per_elem / bytes_per_reg + C."""
    return (3 * t2 + 2 * t3) * bytes_per_elem / bytes_per_reg + c_setup


def smem_per_thread(t2: int, bytes_per_elem: int) -> float:
    """S_thread = t2 * bytes_per_elem."""
    return t2 * bytes_per_elem


def max_occupancy(gpu: Gpu, t2: int, t3: int, bytes_per_elem: int, c_setup: int = 0) -> float:
    """MaxOccup_SM = min(HW_MAX, R_SM / R_thread, S_SM / S_thread) (threads/SM)."""
    r = regs_per_thread(t2, t3, bytes_per_elem, c_setup=c_setup)
    s = smem_per_thread(t2, bytes_per_elem)
    cands = [gpu.hw_max_threads, gpu.regs_per_sm / r]
    if gpu.smem_per_sm:
        cands.append(gpu.smem_per_sm / s)
    return min(cands)


def util_mem(gpu: Gpu, t2: int, t3: int, bytes_per_elem: int, latency_cycles: float) -> float:
    """Little's-law estimate of bandwidth utilisation:
    Concurrent_mem = MaxOccup * t3 (elements in flight per SM);
    Concurrent_max_mem = latency * PeakBand / (#SM * clock) (bytes per SM)."""
    conc = max_occupancy(gpu, t2, t3, bytes_per_elem) * t3 * bytes_per_elem
    need = latency_cycles * (gpu.bw_gbs * 1e9) / (gpu.sms * gpu.clock_ghz * 1e9)
    return min(1.0, conc / need)


def bytes_in_flight_per_sm(bw_gbs: float, sms: int, clock_ghz: float, latency_cycles: float) -> float:
    """Concurrent_max_mem in bytes: what each SM must keep in flight to reach
    the bandwidth peak.  Used to size the shared-memory ring."""
    return latency_cycles * bw_gbs / (sms * clock_ghz)


# Platform table of the paper (Table "Experimental platforms"), double
# precision peaks, used by the tests that pin the classifier.
PAPER_GPUS_DOUBLE = {
    "K40c": Gpu("K40c", 1430.0, 288.0),
    "M40": Gpu("M40", 213.0, 288.0),
    "P100": Gpu("P100", 4600.0, 720.0),
    "V100": Gpu("V100", 7500.0, 900.0),
    # Sec. 4.2.5: the A100 figures used for the paper's prediction.
    "A100": Gpu("A100", 9700.0, 1555.0),
}
