"""Measurement-driven tuning of batched plans.

The paper chooses t1 and tcf by offline profiling and t2, t3 with its model
(Algorithm 7, Sec. 3.1.9; tcf in Sec. 3.2.2).  Here the free choices of a
batch are (a) the tile classes -- 4 or 8 rows per lane for TSM2L problems,
one merged or one class per C-column width -- and (b) the SM share of every
class kernel (the classes run concurrently).  The tuner measures each class
alone on the whole GPU (time t_c), sets the shares proportional to t_c (so
all classes finish together if their time scales inversely with their SMs),
compares that against the byte-proportional default, repeats for every tile
choice and keeps the fastest, caching the result as JSON keyed by device and
problem set.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
import tempfile

from .batched import MERGE_L, MERGE_R, WIDE_L, BatchPlan

FLAG_CHOICES = (0, WIDE_L, MERGE_R | MERGE_L, WIDE_L | MERGE_R | MERGE_L)


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


def autotune(problems, flags_choices=FLAG_CHOICES, reps=3, flush=None, cache_path=None, log=None):
    """Returns (plan, record): the fastest plan found and what was measured."""
    import torch
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    sm = props.multi_processor_count
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    key = f"{props.name}|{problem_set_key(problems)}"
    cache = load_cache(cache_path)
    if key in cache:
        rec = cache[key]
        plan = BatchPlan(problems, rec["flags"])
        plan.set_grids(rec["grids"])
        plan.set_serial(rec.get("serial", False))
        return plan, dict(rec, cached=True)
    best = None
    trials = []
    for flags in flags_choices:
        plan = BatchPlan(problems, flags)
        plan.execute(sh)  # warm-up (module load, attributes)
        torch.cuda.synchronize()
        cls = plan.classes()
        times = [_time(lambda i=i: plan.execute_class(i, sh), torch, stream, reps, flush) for i in range(len(cls))]
        for label, grids in (("bytes", [c["grid"] for c in cls]), ("measured", shares_from_times(times, sm)),
                             ("serial", [c["grid"] for c in cls])):
            plan.set_serial(label == "serial")
            plan.set_grids(grids)
            plan.graph_launch(sh)
            torch.cuda.synchronize()
            t = _time(lambda: plan.graph_launch(sh), torch, stream, reps, flush)
            trials.append({"flags": flags, "shares": label, "grids": grids, "ms": round(t, 4),
                           "class_alone_ms": [round(x, 4) for x in times], "classes": [c["name"] for c in cls]})
            if log:
                log(trials[-1])
            if best is None or t < best[0]:
                if best is not None and best[1] is not plan:
                    best[1].close()
                best = (t, plan, flags, grids, label == "serial")
        if best[1] is not plan:
            plan.close()
    t, plan, flags, grids, serial = best
    plan.set_grids(grids)
    plan.set_serial(serial)
    rec = {"flags": flags, "grids": grids, "serial": serial, "ms": round(t, 4), "trials": trials}
    if cache_path:
        store_cache(cache_path, key, {"flags": flags, "grids": grids, "serial": serial, "ms": round(t, 4)})
    return plan, rec
