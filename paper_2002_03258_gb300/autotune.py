"""Measurement-driven tuning of batched plans, seeded by the paper's model.

The paper chooses its tile parameters t1, t3 (and tcf for TSM2L) by offline
profiling and t2 with its analytic model (Algorithm 7, Sec. 3.1.8-3.1.9;
tcf in Sec. 3.2.2).  The free choices of a batch here are:

* the tile variant: one of the compiled kernels, which differ in pipeline
  stages, rows of C per lane and inner columns per warp and stage;
* the class set: every column chunk in the narrowest class that holds it, or
  all TSM2R chunks in the 16-column class and all TSM2L chunks in the
  32-column class (fewer classes, padded columns);
* the execution mode: one persistent launch for the whole batch, one launch
  per class on all SMs, or the classes concurrently on SM shares.

The first candidate timed is the model's choice (``seed_candidate``): the
variant whose pipeline keeps Little's-law bytes in flight per SM with the
most rows per lane, the merged class set when every merged width stays below
the paper's t2 threshold taken at the FMA rate the kernels sustain (so
padding costs no time in the model), and the single launch.  Then every
candidate is timed (CUDA events, median of `reps` after a warm-up, L2
flushed before each), the fastest is kept and cached as JSON keyed by device
and problem set.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
import tempfile

from . import perfmodel
from .batched import MERGE_L, MERGE_R, BatchPlan, num_variants, variant_flag, variant_info

FLAG_CHOICES = (0, MERGE_R | MERGE_L)
MODE_CHOICES = ("single", "serial")
WIDEST = {"r": 16, "l": 32}  # widest TSM2R / TSM2L class of every variant
# Assumed DRAM round-trip latency (SM cycles) for the Little's-law estimate;
# the paper leaves it a platform constant (Sec. 3.1.8).
LATENCY_CYCLES = 1000.0
# Latency (SM cycles) of a dependent FMA, for the model's compute
# utilisation in Algorithm 7 (reported only).
FMA_LATENCY_CYCLES = 4.0
# Fraction of the binary32 FMA peak the kernels sustain at their on-chip
# limit (ncu: 65-69% FMA-pipe activity for TSM2R k = 16 and TSM2L
# n = k = 32).  The paper's threshold assumes the full peak; the seed uses
# the sustained rate.
FMA_SUSTAINED = 0.65


def _time(fn, torch, stream, reps, flush=None):
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def shares_from_times(times, sm_count):
    """Blocks per class proportional to the class's time alone, >= 1 each."""
    n = len(times)
    left = max(sm_count - n, 0)
    tot = sum(times) or 1.0
    return [1 + int(left * t / tot) for t in times]


def stage_bytes(info) -> int:
    """Bytes of A per pipeline stage of the TSM2R classes of a variant:
    (32 lanes x rows per lane) rows x (8 warps x inner columns) x 4 bytes."""
    return 32 * info["rows_per_lane"] * 8 * info["inner_per_warp"] * 4


def in_flight_bytes(info) -> int:
    """Bytes of A a block keeps in flight: every stage but the one consumed."""
    return (info["stages"] - 1) * stage_bytes(info)


def seed_candidate(infos, gpu: perfmodel.Gpu, latency_cycles: float = LATENCY_CYCLES,
                   fma_sustained: float = FMA_SUSTAINED):
    """The model's choice (variant, flags, mode) among ``infos`` (variant_info
    dicts) for a binary32 batch on ``gpu``: t2 threshold of Sec. 3.1.8 with
    the sustained FMA rate (``fma_sustained`` x peak)."""
    need = perfmodel.bytes_in_flight_per_sm(gpu.bw_gbs, gpu.sms, gpu.clock_ghz, latency_cycles)
    ok = [i for i in infos if in_flight_bytes(i) >= need]
    if ok:
        best = max(ok, key=lambda i: (i["rows_per_lane"], i["stages"], -i["variant"]))
    else:
        best = max(infos, key=lambda i: (in_flight_bytes(i), -i["variant"]))
    thr = perfmodel.t2_threshold(gpu.peak_gflops * fma_sustained, gpu.bw_gbs, 4)
    flags = MERGE_R | MERGE_L if max(WIDEST.values()) <= thr else 0
    return best["variant"], flags, "single"


def candidates(nvariants, seed=None):
    """Every (variant, flags, mode), the seed first."""
    out = [(v, f, m) for v in range(nvariants) for f in FLAG_CHOICES for m in MODE_CHOICES]
    if seed is not None and seed in out:
        out.remove(seed)
        out.insert(0, seed)
    return out


def load_cache(path):
    """The tuning cache at `path` as a dict ({} when absent or unreadable)."""
    if not path or not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        return {}
    return cache if isinstance(cache, dict) else {}


def store_cache(path, key, rec):
    """Adds `rec` under `key` to the cache at `path`.  The file is replaced
    atomically, so a concurrent reader sees the old or the new cache, never a
    partial one."""
    cache = load_cache(path)
    cache[key] = rec
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".tsm2_tune_", suffix=".json", dir=d)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def problem_set_key(problems) -> str:
    h = hashlib.sha256()
    for p in problems:
        h.update(f"{p.op}{p.m},{p.n},{p.k},{p.lda},{p.ldb},{p.ldc};".encode())
    return h.hexdigest()[:16]


def device_model(torch, dev, hbm_gbs=None, fp32_gflops=None) -> perfmodel.Gpu:
    """The model's platform constants for this GPU: SMs and clock from the
    device, bandwidth and binary32 FMA peak measured (or, if not given, the
    nominal 152 SMs x 128 lanes x 2 flops x clock and 8 TB/s)."""
    props = torch.cuda.get_device_properties(dev)
    clock_ghz = (getattr(props, "clock_rate", 0) or 2070000) / 1e6
    sms = props.multi_processor_count
    peak = fp32_gflops or sms * 128 * 2 * clock_ghz
    return perfmodel.Gpu(props.name, peak, hbm_gbs or 8000.0, sms=sms, clock_ghz=clock_ghz)


def alg7_record(gpu: perfmodel.Gpu, ks=(2, 8, 16, 32)):
    """Algorithm 7's (t2, t3) for binary32 TSM2R with an 8192 x 8192 A on
    this GPU, for several skinny widths: what the paper's procedure would
    pick for a thread-per-row kernel, reported beside the measured choice
    (the library's tiles are compiled variants, chosen by measurement)."""
    out = {}
    for k in ks:
        c = perfmodel.optimize_tiles(gpu, 8192, 8192, k, 4, LATENCY_CYCLES, FMA_LATENCY_CYCLES)
        out[f"k{k}"] = {"t2": c.t2, "t3": c.t3, "bound": c.bound, "model_ms": round(c.time_s * 1e3, 4)}
    return out


def make_plan(problems, variant, flags, mode):
    plan = BatchPlan(problems, flags | variant_flag(variant))
    plan.set_mode(mode)
    return plan


def autotune(problems, reps=3, flush=None, cache_path=None, log=None, hbm_gbs=None, fp32_gflops=None,
             candidate_list=None):
    """Returns (plan, record): the fastest plan found and what was measured."""
    import torch
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    key = f"{props.name}|{problem_set_key(problems)}"
    cache = load_cache(cache_path)
    if key in cache:
        rec = cache[key]
        return make_plan(problems, rec["variant"], rec["flags"], rec["mode"]), dict(rec, cached=True)
    infos = [variant_info(v) for v in range(num_variants())]
    gpu = device_model(torch, dev, hbm_gbs, fp32_gflops)
    seed = seed_candidate(infos, gpu)
    best = None
    trials = []
    for (v, flags, mode) in (candidate_list or candidates(len(infos), seed)):
        plan = make_plan(problems, v, flags, mode)
        plan.graph_launch(sh)  # warm-up: module load, attributes, graph capture
        torch.cuda.synchronize()
        t = _time(lambda: plan.graph_launch(sh), torch, stream, reps, flush)
        trial = {"variant": v, "stages": infos[v]["stages"], "rows_per_lane": infos[v]["rows_per_lane"],
                 "inner_per_warp": infos[v]["inner_per_warp"], "flags": flags, "mode": mode,
                 "launches": plan.num_launches(), "classes": [c["name"] for c in plan.classes()],
                 "ms": round(t, 4), "seed": (v, flags, mode) == seed}
        trials.append(trial)
        if log:
            log(trial)
        if best is None or t < best[0]:
            if best is not None:
                best[1].close()
            best = (t, plan, trial)
        else:
            plan.close()
    t, plan, trial = best
    rank = sorted(x["ms"] for x in trials).index(next(x["ms"] for x in trials if x["seed"])) + 1 \
        if any(x["seed"] for x in trials) else None
    rec = {"variant": trial["variant"], "flags": trial["flags"], "mode": trial["mode"], "ms": round(t, 4),
           "launches": trial["launches"], "seed": {"variant": seed[0], "flags": seed[1], "mode": seed[2],
                                                   "rank": rank},
           "model": {"bytes_in_flight_per_sm": round(perfmodel.bytes_in_flight_per_sm(
               gpu.bw_gbs, gpu.sms, gpu.clock_ghz, LATENCY_CYCLES)), "t2_threshold_fp32": round(
               perfmodel.t2_threshold(gpu.peak_gflops, gpu.bw_gbs, 4), 2), "t2_threshold_fp32_sustained": round(
               perfmodel.t2_threshold(gpu.peak_gflops * FMA_SUSTAINED, gpu.bw_gbs, 4), 2),
               "fma_sustained": FMA_SUSTAINED, "latency_cycles": LATENCY_CYCLES,
               "alg7_tsm2r_8192": alg7_record(gpu)},
           "trials": trials}
    if cache_path:
        store_cache(cache_path, key, {k: rec[k] for k in ("variant", "flags", "mode", "ms", "launches")})
    return plan, rec
