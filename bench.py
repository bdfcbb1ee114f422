#!/usr/bin/env python3
"""Benchmark of the TSM2R / TSM2L library on GB300.

Workload (one "step"): the binary32 sweep of the paper's shapes (Sec. 4.1):
TSM2R with A n x n, n in {10240, 20480, 30720}, times B n x k, k in
{2, 4, 8, 16}; and TSM2L with A m x n, m in {2^20, 2^23}, n in {8, 16, 32},
times B n x n.  Entries are uniform in [-1, 1) from the splitmix64 generator,
generated in device memory.  Every launch is preceded by an L2 flush (a
memset of twice the L2 size, then a read of another buffer of that size, so
no operand and no dirty line is left in L2) and timed on its stream with CUDA
events; the step time is the sum of the 18 kernel durations.  The same sweep
behind the memset alone is reported beside it (``flush_write_only``).

Metric: achieved HBM bandwidth, algorithmic bytes s*(m n + n k + m k) per
multiply divided by kernel time, in GB/s (whole job: summed over ranks).

Also reported on the same line: the binary64 sweep (compute-bound on GB300's
FP64 units, so reported against the FP64 roof), cuBLAS GEMM on the same
operands (comparator), an end-to-end figure through the public C ABI with
host buffers, SM clocks sampled during the timed region, the roofline of the
dominant kernel, and the CPU oracle timed on the host cores.

``--impl reference`` times the CPU oracle (the reference implementation of
the definition) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

R_SIZES = [10240, 20480, 30720]
R_KS = [2, 4, 8, 16]
L_MS = [2 ** 20, 2 ** 23]
L_NS = [8, 16, 32]
WORKLOAD = ("tsm2 sweep: TSM2R n x n * n x k, n in {10240,20480,30720}, k in {2,4,8,16}; "
            "TSM2L m x n * n x n, m in {2^20,2^23}, n in {8,16,32}; uniform[-1,1) seed 0")
BATCH_PITCH_BYTES = 512     # batched workload: leading dimensions rounded up to 512 bytes (pitched allocation)
FP64_NOMINAL_TFLOPS = 1.25   # GB300 nominal FP64 (no FP64 tensor-core speed-up)
NOMINAL_HBM_GBS = 8000.0     # GB300 HBM3e, nominal (~8 TB/s)
FALLBACK_HBM_GBS = 6800.0


def make_l2_flush(torch, device):
    """(flush, write_only_flush) for the timed loops.  `flush` writes a buffer
    of twice the L2 size (evicting every operand line) and then reads another
    one, so the lines left in L2 are clean: after a write alone the timed
    kernel would also pay for writing the flush's dirty lines back to DRAM
    (measured: up to ~30 us on a 0.53 ms kernel).  `write_only_flush` is the
    memset alone, reported beside the headline for comparison."""
    l2 = getattr(torch.cuda.get_device_properties(device), "L2_cache_size", 128 << 20) or (128 << 20)
    wbuf = torch.empty(2 * l2, dtype=torch.uint8, device=device)
    rbuf = torch.ones(2 * l2 // 4, dtype=torch.float32, device=device)
    sink = torch.zeros((), dtype=torch.float32, device=device)

    def flush():
        wbuf.zero_()
        torch.sum(rbuf, dim=(0,), out=sink)

    def write_only_flush():
        wbuf.zero_()
    return flush, write_only_flush


def cases(dtype_bytes):
    out = []
    for n in R_SIZES:
        for k in R_KS:
            out.append(("r", n, n, k))
    for m in L_MS:
        for n in L_NS:
            out.append(("l", m, n, n))
    return [(op, m, n, k, dtype_bytes) for (op, m, n, k) in out]


def alg_bytes(m, n, k, es):
    return es * (m * n + n * k + m * k)


def launches_per_call(op, n, k):
    """Kernels one tsm2r_s / tsm2l_s call launches (binary32, bulk-copy path):
    one per column chunk (16 columns for TSM2R, 32 for TSM2L).  B reaches the
    kernels as it is (row-major configurations transpose it on chip)."""
    kc = 32 if op == "l" else 16
    return -(-k // kc) if k > 0 else 0


# Device sources of the bulk-copy kernels (the dominant kernel's
# DRAM-traffic record is tied to these).
KERNEL_SOURCES = ("common.cuh", "internal.h", "tsm2_cfg.cuh", "tsm2_stream.cu")


def src_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2002_03258_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def traffic_record(config_name, workload_key):
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None
    try:
        j = json.load(open(p))
    except Exception:
        return None
    rec = j.get(config_name, {}).get(workload_key)
    if not rec or rec.get("src_hash") != src_hash():
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"tsm2_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.t0 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            rec = parse_clock_samples(f)
        os.unlink(self.path)
        return rec


def parse_clock_samples(lines):
    """Summary of `nvidia-smi --query-gpu=<ClockSampler.FIELDS> --format=csv,
    noheader,nounits` lines: median SM clock over the samples above half the
    maximum (the loaded ones), the maximum, and the throttle reasons seen
    active in any sample.  None without a valid sample."""
    sm, smax, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax = max(smax, float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    loaded = [x for x in sm if x > 0.5 * smax] or sm
    return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": sorted(reasons),
            "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def ranks_max(x, dev, world):
    """Largest value of x over all ranks (a step time: the slowest rank sets
    the job's time).  One rank: x itself, no collective."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbs(world, step_bytes, ms):
    """Whole-job throughput: every rank moves step_bytes per step (weak
    scaling, replicas), the step takes the slowest rank's ms."""
    return world * step_bytes / (ms * 1e-3) / 1e9


# ---------------------------------------------------------------------------
# CPU oracle arm (reference arm and cpu_baseline)

def measure_fma_peak(elem, target_ms=20.0, reps=5):
    """FMA throughput of this GPU from the library's probe kernel
    (tsm2_fma_probe): 8 blocks of 256 threads per SM, independent chains,
    sized to run about `target_ms` (as long as the FP64 kernels it is
    compared with, so both see the clocks of a loaded GPU).  Best of `reps`
    CUDA-event timings after one warm-up."""
    import torch

    import paper_2002_03258_gb300 as pkg
    lib = pkg.lib()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = 8 * sms
    threads = blocks * 256
    per_iter = 16 if elem == 8 else 32  # flops per thread per step
    guess = 1.25e12 if elem == 8 else 80e12
    iters = max(100, int(guess * target_ms * 1e-3 / (per_iter * threads)))
    sink = torch.empty(threads, dtype=torch.float64 if elem == 8 else torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    best = float("inf")
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pkg.check(lib.tsm2_fma_probe(elem, blocks, iters, sink.data_ptr(), stream.cuda_stream))
        e1.record(stream)
        torch.cuda.synchronize()
        if r > 0:
            best = min(best, e0.elapsed_time(e1))
    flops = float(per_iter) * iters * threads
    return {"tflops": round(flops / (best * 1e-3) / 1e12, 4), "ms": round(best, 3), "blocks": blocks,
            "iters": iters, "kind": "DFMA chains" if elem == 8 else "FFMA2 chains"}


def host_cores():
    """Cores this process may run on (its CPU affinity set), not every core
    of the host."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_sample_run(dtype_name, steps, warmup, budget_s=20.0):
    """Time the CPU oracle on a bounded row sample of every case of the sweep.

    Returns (GB/s, description, cores, seconds per step)."""
    import numpy as np

    import oracle
    import tsm2_inputs as ti
    dt = np.float32 if dtype_name == "f32" else np.float64
    es = 4 if dt == np.float32 else 8
    cores = host_cores()
    samples = []
    for op, m, n, k, _ in cases(es):
        rows = max(64, min(m, (1 << 21) // n))  # about 2M elements of A per case
        ridx = np.arange(rows)
        A = ti.uniform_pm1(0, ti.MID_A, m, n, dt, row_idx=ridx)
        B = ti.uniform_pm1(0, ti.MID_B, n, k, dt)
        samples.append((A, B, alg_bytes(rows, n, k, es)))
    tot_bytes = sum(s[2] for s in samples)
    for _ in range(max(0, warmup)):
        for A, B, _ in samples[:1]:
            oracle.gemm_threaded(A, B, cores)
    times = []
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        for A, B, _ in samples:
            oracle.gemm_threaded(A, B, cores)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    desc = (f"first max(64, 2^21/n) rows of A for each of the {len(samples)} sweep cases "
            f"({tot_bytes / 1e6:.0f} MB algorithmic per step), oracle.gemm_threaded on {cores} threads")
    return tot_bytes / t / 1e9, desc, cores, t


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    steps = max(1, args.steps)
    value, desc, cores, t = oracle_sample_run("f32", steps, min(args.warmup, 1))
    line = {
        "impl": "reference", "metric": "TSM2R/TSM2L achieved HBM GB/s (binary32 sweep)", "value": round(value, 4),
        "unit": "GB/s", "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
        "ms_per_step": round(t * 1e3, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "accumulate": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (row sample, CPU)", "sample": desc,
                   "arithmetic": "binary32 inputs widened exactly, products and sums in binary64"},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm

def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__ as ge
    world, rank, local = dist_setup()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ge.build()
    import paper_2002_03258_gb300 as pkg
    import tsm2_inputs as ti
    lib = pkg.lib()
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream

    props = torch.cuda.get_device_properties(dev)
    l2_flush, l2_flush_write_only = make_l2_flush(torch, dev)

    def make_sweep(es, seed):
        tdt = torch.float32 if es == 4 else torch.float64
        suf = "s" if es == 4 else "d"
        fill = getattr(lib, f"tsm2_fill_uniform_{suf}")
        bufs = {}
        work = []
        for op, m, n, k, _ in cases(es):
            keyA = ("A", op, m, n)
            if keyA not in bufs:
                t = torch.empty((n, m), dtype=tdt, device=dev).t()
                pkg.check(fill(m, n, seed, ti.MID_A, t.data_ptr(), m, sh))
                bufs[keyA] = t
            kmax = 16 if op == "r" else n
            keyB = ("B", op, n, kmax)
            if keyB not in bufs:
                t = torch.empty((kmax, n), dtype=tdt, device=dev).t()
                pkg.check(fill(n, kmax, seed, ti.MID_B, t.data_ptr(), n, sh))
                bufs[keyB] = t
            keyC = ("C", op, m, kmax)
            if keyC not in bufs:
                bufs[keyC] = torch.empty((kmax, m), dtype=tdt, device=dev).t()
            fn = getattr(pkg, f"tsm2{op}_{suf}")
            work.append(dict(op=op, m=m, n=n, k=k, es=es, fn=fn, A=bufs[keyA], B=bufs[keyB], C=bufs[keyC],
                             bytes=alg_bytes(m, n, k, es), flops=2 * m * n * k))
        return work, bufs

    def call(w, s=sh):
        return w["fn"](w["m"], w["n"], w["k"], w["A"].data_ptr(), w["m"], w["B"].data_ptr(), w["n"],
                       w["C"].data_ptr(), w["m"], s)

    def timed_steps(work, steps, warmup, flush_fn=None):
        flush_fn = flush_fn or l2_flush
        for _ in range(warmup):
            for w in work:
                flush_fn()
                pkg.check(call(w))
        torch.cuda.synchronize()
        pkg.check(pkg.tsm2_get_device_status(sh))
        evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in work]
               for _ in range(steps)]
        case_cfg = {}
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_region0 = time.perf_counter()
        for s in range(steps):
            for i, w in enumerate(work):
                flush_fn()
                evs[s][i][0].record(stream)
                pkg.check(call(w))
                evs[s][i][1].record(stream)
                case_cfg[i] = pkg.tsm2_last_config()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        wall = time.perf_counter() - t_region0
        pkg.check(pkg.tsm2_get_device_status(sh))
        per = [[evs[s][i][0].elapsed_time(evs[s][i][1]) for i in range(len(work))] for s in range(steps)]
        return per, case_cfg, wall

    peak_hbm, peak_kind = measured_peaks()
    clocks = ClockSampler(local)

    # ---- binary32 sweep: the headline -------------------------------------------------
    work32, bufs32 = make_sweep(4, 0)
    torch.cuda.synchronize()
    clocks.start()
    per, case_cfg, wall = timed_steps(work32, args.steps, args.warmup)
    clock_rec = clocks.stop()
    step_ms = [sum(row) for row in per]
    mean_step_ms = ranks_max(statistics.mean(step_ms), dev, world)
    step_bytes = sum(w["bytes"] for w in work32)
    value = job_gbs(world, step_bytes, mean_step_ms)
    case_rows = []
    for i, w in enumerate(work32):
        ts = [per[s][i] for s in range(args.steps)]
        ms = statistics.mean(ts)
        case_rows.append({"op": "tsm2" + w["op"], "m": w["m"], "n": w["n"], "k": w["k"], "ms": round(ms, 4),
                          "ms_median": round(statistics.median(ts), 4), "ms_min": round(min(ts), 4),
                          "gbs": round(w["bytes"] / (ms * 1e-3) / 1e9, 1),
                          "frac_hbm": round(w["bytes"] / (ms * 1e-3) / 1e9 / peak_hbm, 3),
                          "frac_nominal": round(w["bytes"] / (ms * 1e-3) / 1e9 / NOMINAL_HBM_GBS, 3),
                          "gflops": round(w["flops"] / (ms * 1e-3) / 1e9, 1),
                          "config": case_cfg.get(i)})
    dom = max(range(len(work32)), key=lambda i: case_rows[i]["ms"])
    dw = work32[dom]
    dom_ms = case_rows[dom]["ms"]
    achieved = dw["bytes"] / (dom_ms * 1e-3) / 1e9
    wkey = f"{dw['op']}_{dw['m']}x{dw['n']}x{dw['k']}_f32"
    traffic = traffic_record(case_cfg.get(dom), wkey)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak_hbm, "unit": "GB/s",
                "frac": round(achieved / peak_hbm, 4), "traffic": traffic,
                "kernel": case_cfg.get(dom), "workload": wkey, "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": dw["bytes"]}

    # ---- the launch floor: the same flush and event pair around a trivial kernel ------
    def floor_us(fn, reps=30):
        ts = []
        for _ in range(reps + 5):
            l2_flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        return round(statistics.median(ts[5:]), 2)
    one = torch.zeros(1, device=dev)
    launch_floor = {"events_only_us": floor_us(lambda: None), "trivial_kernel_us": floor_us(lambda: one.add_(1.0)),
                    "note": "CUDA-event time of an empty region and of a one-element kernel after the same L2 "
                            "flush: the part of every timed call that is launch and completion"}

    # ---- the same sweep behind the write-only flush (comparison) -----------------------
    wo_steps = max(1, min(args.steps, 3))
    per_wo, _, _ = timed_steps(work32, wo_steps, 1, l2_flush_write_only)
    wo_ms = ranks_max(statistics.mean(sum(row) for row in per_wo), dev, world)
    wo_dom = statistics.mean(per_wo[s_][dom] for s_ in range(wo_steps))
    flush_write_only = {"value": round(job_gbs(world, step_bytes, wo_ms), 2), "unit": "GB/s",
                        "ms_per_step": round(wo_ms, 4), "steps": wo_steps,
                        "dominant_kernel_ms": round(wo_dom, 4),
                        "dominant_kernel_frac": round(dw["bytes"] / (wo_dom * 1e-3) / 1e9 / peak_hbm, 4),
                        "l2": "memset of 2x L2 before every launch, no read pass"}

    # ---- end to end through the C ABI with host buffers --------------------------------------
    # tsm2r_s_host / tsm2l_s_host: A, B, C in page-locked host memory; each
    # call streams A to the device in row chunks, overlapping copy-in, the
    # product and the copy-out of C (all inside the timed region).
    h_in, h_out, h_shared = [], [], {}
    for w in work32:
        key = w["A"].data_ptr()  # cases that share a device A share its host copy
        if key not in h_shared:
            h_shared[key] = torch.empty((w["n"], w["m"]), dtype=w["A"].dtype, pin_memory=True).t()
            h_shared[key].copy_(w["A"])
        hA = h_shared[key]
        hB = torch.empty((w["k"], w["n"]), dtype=w["A"].dtype, pin_memory=True).t()
        hB.copy_(w["B"][:, :w["k"]])
        hC = torch.empty((w["k"], w["m"]), dtype=w["A"].dtype, pin_memory=True).t()
        h_in.append((hA, hB))
        h_out.append(hC)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 5))
    h2d = sum(w["A"].numel() * w["es"] + w["n"] * w["k"] * w["es"] for w in work32)
    d2h = sum(w["m"] * w["k"] * w["es"] for w in work32)
    host_fn = {"r": pkg.tsm2r_s_host, "l": pkg.tsm2l_s_host}

    def e2e_step():
        for (hA, hB), hC, w in zip(h_in, h_out, work32):
            pkg.check(host_fn[w["op"]](w["m"], w["n"], w["k"], hA.data_ptr(), w["m"], hB.data_ptr(), w["n"],
                                       hC.data_ptr(), w["m"], sh))

    e2e_step()  # staging buffers allocated outside the timed region
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e_end.record(stream)
    torch.cuda.synchronize()
    e2e_ms = ranks_max(e_start.elapsed_time(e_end) / e2e_steps, dev, world)
    e2e = {"value": round(job_gbs(world, step_bytes, e2e_ms), 2), "unit": "GB/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3),
           "host_copy": pkg.tsm2_last_host_copy()}
    del h_in, h_out, h_shared

    # ---- cuBLAS comparator on the same operands (not timed in the step) -----------------
    def cublas_ms(w):
        """Median of 3 L2-flushed torch.matmul calls (cuBLAS GEMM) on the case's
        column-major operands."""
        A, B = w["A"], w["B"][:, :w["k"]]
        out = torch.empty((w["k"], w["m"]), dtype=A.dtype, device=dev).t()
        torch.matmul(A, B, out=out)
        ts = []
        for _ in range(3):
            l2_flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch.matmul(A, B, out=out)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        del out
        return statistics.median(ts)

    if not args.no_cublas:
        for i, w in enumerate(work32):
            ms = cublas_ms(w)
            case_rows[i]["cublas_ms"] = round(ms, 4)
            case_rows[i]["speedup_vs_cublas"] = round(ms / case_rows[i]["ms"], 3)

    # ---- binary64 sweep (FP64 ALU bound) ----------------------------------------------------
    fp64 = None
    if not args.no_fp64:
        fma64 = measure_fma_peak(8)
        work64, bufs64 = make_sweep(8, 0)
        per64, case_cfg64, _ = timed_steps(work64, max(1, min(args.steps, 3)), min(args.warmup, 3))
        ms64 = statistics.mean(sum(r) for r in per64)
        bytes64 = sum(w["bytes"] for w in work64)
        flops64 = sum(w["flops"] for w in work64)
        d64 = max(range(len(work64)), key=lambda i: per64[0][i])
        d64_ms = statistics.mean(r[d64] for r in per64)
        tfl = work64[d64]["flops"] / (d64_ms * 1e-3) / 1e12
        fp64 = {"value": round(bytes64 / (ms64 * 1e-3) / 1e9, 1), "unit": "GB/s", "ms_per_step": round(ms64, 3),
                "tflops": round(flops64 / (ms64 * 1e-3) / 1e12, 3),
                "roofline": {"bound": "alu", "achieved": round(tfl, 3), "peak": fma64["tflops"],
                             "unit": "TFLOP/s", "frac": round(tfl / fma64["tflops"], 4),
                             "kernel": case_cfg64.get(d64), "peak_kind": "measured (DFMA probe, this run)",
                             "peak_probe": fma64, "nominal_peak": FP64_NOMINAL_TFLOPS,
                             "frac_nominal": round(tfl / FP64_NOMINAL_TFLOPS, 4),
                             "workload": f"{work64[d64]['op']}_{work64[d64]['m']}x{work64[d64]['n']}x{work64[d64]['k']}_f64"},
                "cases": [{"op": "tsm2" + w["op"], "m": w["m"], "n": w["n"], "k": w["k"],
                           "ms": round(statistics.mean(r[i] for r in per64), 4),
                           "tflops": round(w["flops"] / (statistics.mean(r[i] for r in per64) * 1e-3) / 1e12, 3)}
                          for i, w in enumerate(work64)]}
        if not args.no_cublas:
            for i, w in enumerate(work64):
                ms = cublas_ms(w)
                row = fp64["cases"][i]
                row["cublas_ms"] = round(ms, 4)
                row["speedup_vs_cublas"] = round(ms / row["ms"], 3)
        del bufs64, work64
        torch.cuda.empty_cache()

    # ---- differentiable TSM2R: forward + backward (binary32, 16384^2, k = 8) -------------------
    fwd_bwd = None
    if not args.no_fwdbwd:
        m = n = 16384
        k = 8
        sc = 1.0 / (n ** 0.5)
        A = torch.empty((n, m), dtype=torch.float32, device=dev).t()
        B = torch.empty((k, n), dtype=torch.float32, device=dev).t()
        dC = torch.empty((k, m), dtype=torch.float32, device=dev).t()
        C = torch.empty((k, m), dtype=torch.float32, device=dev).t()
        dB = torch.empty((k, n), dtype=torch.float32, device=dev).t()
        dA = torch.empty((n, m), dtype=torch.float32, device=dev).t()
        pkg.check(lib.tsm2_fill_normal_ih_s(m, n, 0, ti.MID_A, sc, A.data_ptr(), m, sh))
        pkg.check(lib.tsm2_fill_normal_ih_s(n, k, 0, ti.MID_B, sc, B.data_ptr(), n, sh))
        pkg.check(lib.tsm2_fill_normal_ih_s(m, k, 0, ti.MID_DC, 1.0, dC.data_ptr(), m, sh))
        legs = {
            "fwd": lambda: pkg.tsm2r_s(m, n, k, A.data_ptr(), m, B.data_ptr(), n, C.data_ptr(), m, sh),
            "dB": lambda: pkg.tsm2r_t_s(m, n, k, A.data_ptr(), m, dC.data_ptr(), m, dB.data_ptr(), n, sh),
            "dA": lambda: pkg.tsm2_rankk_s(m, n, k, dC.data_ptr(), m, B.data_ptr(), n, dA.data_ptr(), m, sh),
        }
        leg_bytes = 4 * (m * n + n * k + m * k)
        times = {}
        for name, f in legs.items():
            ts = []
            for r in range(args.warmup + max(3, min(args.steps, 10))):
                l2_flush()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pkg.check(f())
                e1.record(stream)
                torch.cuda.synchronize()
                if r >= args.warmup:
                    ts.append(e0.elapsed_time(e1))
            times[name] = statistics.median(ts)
        pkg.check(pkg.tsm2_get_device_status(sh))
        tot = sum(times.values())
        fwd_bwd = {"workload": "16384 x 16384 x 8 binary32, N(0,1/n) inputs, dC N(0,1)",
                   "ms": {kk: round(v, 4) for kk, v in times.items()}, "total_ms": round(tot, 4),
                   "gbs": {kk: round(leg_bytes / (v * 1e-3) / 1e9, 1) for kk, v in times.items()},
                   "frac_hbm": {kk: round(leg_bytes / (v * 1e-3) / 1e9 / peak_hbm, 3) for kk, v in times.items()},
                   "fwd_bwd_over_fwd": round(tot / times["fwd"], 3)}
        del A, B, dC, C, dB, dA

    # ---- mixed precision: A in binary32, bfloat16, bfloat16 hi+lo (32768^2, k = 16) -----------
    mixed = None
    if not args.no_mixed:
        import numpy as np

        import oracle
        m = n = 32768
        k = 16
        X = torch.empty((n, m), dtype=torch.float32, device=dev).t()
        pkg.check(lib.tsm2_fill_logmag_s(m, n, 0, ti.MID_A, X.data_ptr(), m, sh))
        Bm = torch.empty((k, n), dtype=torch.float32, device=dev).t()
        pkg.check(lib.tsm2_fill_uniform_s(n, k, 0, ti.MID_B, Bm.data_ptr(), n, sh))
        hi = torch.empty((n, m), dtype=torch.int16, device=dev)
        lo = torch.empty((n, m), dtype=torch.int16, device=dev)
        pkg.check(pkg.tsm2_split_bf16(m, n, X.data_ptr(), m, hi.data_ptr(), lo.data_ptr(), m, sh))
        Cm = torch.empty((k, m), dtype=torch.float32, device=dev).t()
        variants = {
            "fp32": (lambda: pkg.tsm2r_s(m, n, k, X.data_ptr(), m, Bm.data_ptr(), n, Cm.data_ptr(), m, sh),
                     4 * m * n + 4 * n * k + 4 * m * k),
            "bf16": (lambda: pkg.tsm2r_bf16(m, n, k, hi.data_ptr(), None, m, Bm.data_ptr(), n, Cm.data_ptr(), m, sh),
                     2 * m * n + 4 * n * k + 4 * m * k),
            "bf16_hilo": (lambda: pkg.tsm2r_bf16(m, n, k, hi.data_ptr(), lo.data_ptr(), m, Bm.data_ptr(), n,
                                                 Cm.data_ptr(), m, sh),
                          4 * m * n + 4 * n * k + 4 * m * k),
        }
        rows = np.linspace(0, m - 1, 24).astype(np.int64)
        Xr = ti.logmag(0, ti.MID_A, m, n, np.float32, row_idx=rows).astype(np.float64)
        Bh = ti.uniform_pm1(0, ti.MID_B, n, k, np.float32).astype(np.float64)
        ref = oracle.gemm(np.asfortranarray(Xr), Bh)
        S = oracle.absgemm(np.asfortranarray(Xr), Bh)
        mixed = {"workload": "32768 x 32768 A, magnitudes log-uniform over [2^-10, 2^10), random sign; "
                             "B 32768 x 16 uniform[-1,1); error vs binary64 oracle on 24 sampled rows",
                 "variants": {}}
        for name, (f, nbytes) in variants.items():
            ts = []
            for r in range(args.warmup + max(3, min(args.steps, 10))):
                l2_flush()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pkg.check(f())
                e1.record(stream)
                torch.cuda.synchronize()
                if r >= args.warmup:
                    ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            cfgname = pkg.tsm2_last_config()
            got = Cm.cpu().numpy()[rows].astype(np.float64)
            err = np.abs(got - ref)
            big = np.abs(ref) > 1e-6 * S
            mixed["variants"][name] = {
                "config": cfgname, "ms": round(ms, 4), "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                "frac_hbm": round(nbytes / (ms * 1e-3) / 1e9 / peak_hbm, 3),
                "max_err_over_absAB": float(f"{float(np.max(err / S)):.3e}"),
                "normwise_rel_err": float(f"{float(np.linalg.norm(got - ref) / np.linalg.norm(ref)):.3e}"),
                "max_rel_err": float(f"{float(np.max(err[big] / np.abs(ref[big]))):.3e}")}
        pkg.check(pkg.tsm2_get_device_status(sh))
        f32ms = mixed["variants"]["fp32"]["ms"]
        for v in mixed["variants"].values():
            v["speedup_vs_fp32"] = round(f32ms / v["ms"], 3)
        del X, Bm, hi, lo, Cm
        torch.cuda.empty_cache()

    # ---- batched uneven problems: one persistent launch vs a loop of plain launches ----------
    batched = None
    if not args.no_batched:
        import paper_2002_03258_gb300.batched as bt
        from paper_2002_03258_gb300.autotune import autotune, make_plan
        shapes = ti.batch_shapes(0)

        def build_batch(pitch_bytes):
            """Device buffers of the 512 problems, leading dimensions rounded
            up to `pitch_bytes`; returns (problems, buffers, plain calls, bytes)."""
            pe = max(1, pitch_bytes // 4)
            probs_, keep_, calls_, tot = [], [], [], 0
            for idx, (op, m, n, k) in enumerate(shapes):
                lda = (m + pe - 1) // pe * pe
                ldb = (n + pe - 1) // pe * pe
                tA = torch.empty((n, lda), dtype=torch.float32, device=dev)
                tB = torch.empty((k, ldb), dtype=torch.float32, device=dev)
                tC = torch.empty((k, lda), dtype=torch.float32, device=dev)
                pkg.check(lib.tsm2_fill_uniform_s(m, n, idx, ti.MID_A, tA.data_ptr(), lda, sh))
                pkg.check(lib.tsm2_fill_uniform_s(n, k, idx, ti.MID_B, tB.data_ptr(), ldb, sh))
                keep_ += [tA, tB, tC]
                probs_.append(bt.problem(op, m, n, k, tA.data_ptr(), lda, tB.data_ptr(), ldb, tC.data_ptr(), lda))
                fn = pkg.tsm2r_s if op == "r" else pkg.tsm2l_s
                calls_.append((fn, (m, n, k, tA.data_ptr(), lda, tB.data_ptr(), ldb, tC.data_ptr(), lda, sh)))
                tot += 4 * (m * n + n * k + m * k)
            torch.cuda.synchronize()
            return probs_, keep_, calls_, tot

        def timed(fn, reps):
            ts = []
            for _ in range(reps):
                l2_flush()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return statistics.median(ts)

        reps = max(3, min(args.steps, 5))
        probs, keep, loop_calls, total = build_batch(BATCH_PITCH_BYTES)

        def loop():
            for fn, a in loop_calls:
                pkg.check(fn(*a))

        loop()
        t_loop = timed(loop, reps)
        plan0 = make_plan(probs, 0, 0, "single")
        plan0.graph_launch(sh)
        t_default = timed(lambda: plan0.graph_launch(sh), reps)
        classes0 = plan0.classes()
        launches0 = plan0.num_launches()
        plan0.close()
        tuned, rec = autotune(probs, reps=3, flush=l2_flush, hbm_gbs=peak_hbm)
        t_tuned = timed(lambda: tuned.graph_launch(sh), reps)
        pkg.check(pkg.tsm2_get_device_status(sh))
        best_single = min((t for t in rec["trials"] if t["mode"] == "single"), key=lambda t: t["ms"])
        best_serial = min((t for t in rec["trials"] if t["mode"] == "serial"), key=lambda t: t["ms"])
        batched = {
            "workload": "512 problems: 256 TSM2R (n = m uniform in [512, 8192], k in {2..16}), 256 TSM2L "
                        "(m in [2^14, 2^20], n = k in {4..32}), binary32 uniform[-1,1), seed 0; leading "
                        f"dimensions rounded up to {BATCH_PITCH_BYTES} bytes",
            "algorithmic_bytes": total,
            "loop_of_plain_launches_ms": round(t_loop, 4),
            "graph_single_launch_default_ms": round(t_default, 4),
            "graph_autotuned_ms": round(t_tuned, 4),
            "gbs": {"loop": round(total / (t_loop * 1e-3) / 1e9, 1),
                    "single_launch_default": round(total / (t_default * 1e-3) / 1e9, 1),
                    "best_single_launch": round(total / (best_single["ms"] * 1e-3) / 1e9, 1),
                    "best_serial_classes": round(total / (best_serial["ms"] * 1e-3) / 1e9, 1),
                    "graph_autotuned": round(total / (t_tuned * 1e-3) / 1e9, 1)},
            "frac_hbm_autotuned": round(total / (t_tuned * 1e-3) / 1e9 / peak_hbm, 3),
            "speedup_autotuned_vs_loop": round(t_loop / t_tuned, 3),
            "launches": {"loop": sum(launches_per_call(o, n, k) for o, m, n, k in shapes),
                         "single_launch": launches0, "autotuned": tuned.num_launches()},
            "autotuned": {k2: rec[k2] for k2 in ("variant", "flags", "mode", "launches", "seed", "model")}
            | {"classes": [c["name"] for c in tuned.classes()],
               "tile": {k2: v2 for k2, v2 in rec["trials"][[t["variant"] == rec["variant"] and t["flags"] == rec["flags"]
                                                            and t["mode"] == rec["mode"] for t in rec["trials"]].index(True)].items()
                        if k2 in ("stages", "rows_per_lane", "inner_per_warp")}},
            "default_classes": [(c["name"], c["nprob"]) for c in classes0],
            "trials": [(t["variant"], t["flags"], t["mode"], t["launches"], t["ms"]) for t in rec["trials"]],
            "trial_fields": ["variant", "flags", "mode", "launches", "ms"],
        }
        tuned.close()
        del keep, probs, loop_calls
        torch.cuda.empty_cache()
        # Same batch with leading dimensions only 16-byte aligned: 1 KB column
        # runs of A then straddle DRAM lines (the tuned choice, re-timed).
        probs, keep, _, _ = build_batch(16)
        p16 = make_plan(probs, rec["variant"], rec["flags"], rec["mode"])
        p16.graph_launch(sh)
        t16 = timed(lambda: p16.graph_launch(sh), reps)
        pkg.check(pkg.tsm2_get_device_status(sh))
        p16.close()
        batched["pitch16_autotuned_ms"] = round(t16, 4)
        batched["gbs"]["pitch16_autotuned"] = round(total / (t16 * 1e-3) / 1e9, 1)
        del keep, probs
        torch.cuda.empty_cache()

    # ---- TSM2R / TSM2L crossover and the TSM2X choice -------------------------------------------
    crossover = None
    if not args.no_crossover:
        rows_x = []
        worst = 1.0
        picked = 0
        for m in (15360, 1 << 20):
            for n in (4, 16, 64, 256, 1024):
                k = 16
                A = torch.empty((n, m), dtype=torch.float32, device=dev).t()
                B = torch.empty((k, n), dtype=torch.float32, device=dev).t()
                C = torch.empty((k, m), dtype=torch.float32, device=dev).t()
                pkg.check(lib.tsm2_fill_uniform_s(m, n, 0, ti.MID_A, A.data_ptr(), m, sh))
                pkg.check(lib.tsm2_fill_uniform_s(n, k, 0, ti.MID_B, B.data_ptr(), n, sh))
                nbytes = 4 * (m * n + n * k + m * k)
                rec = {"m": m, "n": n, "k": k}
                cands = (("tsm2r", pkg.tsm2r_s), ("tsm2l", pkg.tsm2l_s), ("tsm2x", pkg.tsm2x_s))
                cfg, ts = {}, {name: [] for name, _ in cands}
                for name, fn in cands:
                    pkg.check(fn(m, n, k, A.data_ptr(), m, B.data_ptr(), n, C.data_ptr(), m, sh))
                    cfg[name] = pkg.tsm2_last_config()
                # The three candidates take turns within each repeat, so that a
                # slow phase of the box hits all of them; small cases (a few us)
                # get more repeats.
                reps = 15 if nbytes < (64 << 20) else max(5, min(args.steps, 9))
                for _ in range(reps):
                    for name, fn in cands:
                        l2_flush()
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        pkg.check(fn(m, n, k, A.data_ptr(), m, B.data_ptr(), n, C.data_ptr(), m, sh))
                        e1.record(stream)
                        torch.cuda.synchronize()
                        ts[name].append(e0.elapsed_time(e1))
                for name, _ in cands:
                    ms = statistics.median(ts[name])
                    rec[name] = {"gbs": round(nbytes / (ms * 1e-3) / 1e9, 1), "config": cfg[name]}
                best = max(rec["tsm2r"]["gbs"], rec["tsm2l"]["gbs"])
                best_op = "tsm2r" if rec["tsm2r"]["gbs"] >= rec["tsm2l"]["gbs"] else "tsm2l"
                rec["tsm2x_over_best"] = round(rec["tsm2x"]["gbs"] / best, 3)
                # The choice itself, free of timing noise on the small cases:
                # TSM2X ran the configuration of the faster schedule.
                rec["tsm2x_picked_faster"] = rec["tsm2x"]["config"] == rec[best_op]["config"]
                picked += int(rec["tsm2x_picked_faster"])
                worst = min(worst, rec["tsm2x_over_best"])
                rows_x.append(rec)
                del A, B, C
        pkg.check(pkg.tsm2_get_device_status(sh))
        crossover = {"workload": "binary32 A m x n (m in {15360, 2^20}, inner n in {4..1024}), B n x 16, "
                                 "uniform[-1,1) seed 0; TSM2R vs TSM2L (B resident n <= 64, staged above) vs the "
                                 "TSM2X choice", "worst_tsm2x_over_best": worst,
                     "tsm2x_picked_faster": f"{picked}/{len(rows_x)}", "cases": rows_x}

    # ---- CPU oracle baseline (rank 0, N = 1) --------------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, desc, cores, _ = oracle_sample_run("f32", 1, 0)
        cpu = {"value": round(v, 4), "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc}

    n_launch = args.steps * sum(launches_per_call(w["op"], w["n"], w["k"]) for w in work32)
    line = {
        "metric": "TSM2R/TSM2L achieved HBM GB/s (binary32 sweep)", "value": round(value, 2), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(mean_step_ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (device-generated splitmix64 uniform[-1,1))",
        "config": {"workload": WORKLOAD,
                   "l2": "flushed before every launch: memset of 2x L2, then a read of another 2x L2 buffer "
                         "(no operand and no dirty line of the flush left in L2)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "step_wall_s": round(wall / args.steps, 4)},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": n_launch,
        "clocks": clock_rec, "fp64": fp64, "fwd_bwd": fwd_bwd, "mixed_precision": mixed, "batched": batched,
        "crossover": crossover, "cases": case_rows, "flush_write_only": flush_write_only,
        "launch_floor": launch_floor,
        "src_hash": src_hash(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_case(args):
    """One multiply, timed like the sweep (for profiling single kernels)."""
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_2002_03258_gb300 as pkg
    import tsm2_inputs as ti
    op, dt, m, n, k = args.case.split(":")
    m, n, k = int(m), int(n), int(k)
    bf16 = dt in ("bf16", "bf16hilo")  # TSM2R with A in bfloat16 (hi, or hi + lo), B and C binary32
    if bf16 and op != "r":
        raise SystemExit("bfloat16 A is a TSM2R variant: use op r")
    tdt = torch.float64 if dt == "f64" else torch.float32
    suf = "d" if dt == "f64" else "s"
    es = 8 if dt == "f64" else 4
    lib = pkg.lib()
    A = torch.empty((n, m), dtype=tdt, device="cuda").t()
    B = torch.empty((k, n), dtype=tdt, device="cuda").t()
    C = torch.empty((k, m), dtype=tdt, device="cuda").t()
    fill = getattr(lib, f"tsm2_fill_uniform_{suf}")
    pkg.check(fill(m, n, 0, ti.MID_A, A.data_ptr(), m, 0))
    pkg.check(fill(n, k, 0, ti.MID_B, B.data_ptr(), n, 0))
    if bf16:
        hi = torch.empty((n, m), dtype=torch.int16, device="cuda")
        lo = torch.empty((n, m), dtype=torch.int16, device="cuda") if dt == "bf16hilo" else None
        pkg.check(pkg.tsm2_split_bf16(m, n, A.data_ptr(), m, hi.data_ptr(), lo.data_ptr() if lo is not None else None,
                                      m, 0))
        del A
        es_a = 4 if dt == "bf16hilo" else 2

        def fn(m_, n_, k_, _a, lda, b, ldb, c, ldc, st):
            return pkg.tsm2r_bf16(m_, n_, k_, hi.data_ptr(), lo.data_ptr() if lo is not None else None, lda, b, ldb,
                                  c, ldc, st)
        A_ptr = 0
        nbytes = es_a * m * n + 4 * (n * k + m * k)
    else:
        fn = getattr(pkg, f"tsm2{op}_{suf}")
        A_ptr = A.data_ptr()
        nbytes = alg_bytes(m, n, k, es)
    l2_flush, _ = make_l2_flush(torch, 0)
    ts = []
    for r in range(args.warmup + args.steps):
        l2_flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pkg.check(fn(m, n, k, A_ptr, m, B.data_ptr(), n, C.data_ptr(), m, 0))
        e1.record()
        torch.cuda.synchronize()
        if r >= args.warmup:
            ts.append(e0.elapsed_time(e1))
    pkg.check(pkg.tsm2_get_device_status(0))
    ms = statistics.median(ts)
    print(json.dumps({"case": args.case, "config": pkg.tsm2_last_config(), "ms": round(ms, 4),
                      "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                      "algorithmic_bytes": nbytes, "src_hash": src_hash()}), flush=True)
    return 0


def run_host_case(args):
    """One host-operand multiply (tsm2r_s_host / tsm2l_s_host, binary32): A,
    B and C in page-locked host memory, the copies inside the timed region
    (for profiling the host pipeline and its copy kernels).  `mode` 0 moves
    the buffers with the SM copy kernels, 1 with the copy engines."""
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_2002_03258_gb300 as pkg
    import tsm2_inputs as ti
    op, m, n, k, mode = args.host_case.split(":")
    m, n, k, mode = int(m), int(n), int(k), int(mode)
    if op not in ("r", "l"):
        raise SystemExit("op must be r or l")
    lib = pkg.lib()
    dA = torch.empty((n, m), dtype=torch.float32, device="cuda")
    pkg.check(lib.tsm2_fill_uniform_s(m, n, 0, ti.MID_A, dA.data_ptr(), m, 0))
    hA = torch.empty((n, m), dtype=torch.float32, pin_memory=True)
    hA.copy_(dA)
    del dA
    hB = torch.empty((k, n), dtype=torch.float32, pin_memory=True).uniform_(-1, 1)
    hC = torch.empty((k, m), dtype=torch.float32, pin_memory=True)
    fn = pkg.tsm2r_s_host if op == "r" else pkg.tsm2l_s_host
    pkg.tsm2_set_host_copy(mode)
    ts = []
    for r in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pkg.check(fn(m, n, k, hA.data_ptr(), m, hB.data_ptr(), n, hC.data_ptr(), m, 0))
        e1.record()
        torch.cuda.synchronize()
        if r >= args.warmup:
            ts.append(e0.elapsed_time(e1))
    pkg.check(pkg.tsm2_get_device_status(0))
    path = pkg.tsm2_last_host_copy()
    pkg.tsm2_set_host_copy(0)
    ms = statistics.median(ts)
    print(json.dumps({"host_case": args.host_case, "config": pkg.tsm2_last_config(), "host_copy": path,
                      "ms": round(ms, 3), "gbs": round(alg_bytes(m, n, k, 4) / (ms * 1e-3) / 1e9, 1),
                      "h2d_gbs": round(4 * (m * n + n * k) / (ms * 1e-3) / 1e9, 1),
                      "d2h_gbs": round(4 * m * k / (ms * 1e-3) / 1e9, 1), "src_hash": src_hash()}), flush=True)
    return 0


def run_batch_case(args):
    """One tile class of the batched workload: the first `count` problems of
    the 512-problem batch whose op is `op` and whose k chunk uses the C-column
    width `kc` (op "x": the first `count` problems, any class), as one plan
    (flags; default mode, one launch), executed like the batched leg (for the
    ncu captures of the batched kernel)."""
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_2002_03258_gb300 as pkg
    import paper_2002_03258_gb300.batched as bt
    import tsm2_inputs as ti
    parts = args.batch_case.split(":")
    op, kc, count, flags = parts[:4]
    kc, count, flags = int(kc), int(count), int(flags)
    pitch = int(parts[4]) if len(parts) > 4 else 16  # bytes: leading dimensions rounded up to this
    pe = max(1, pitch // 4)
    widths = (2, 4, 8, 12, 16, 24, 32)
    lib = pkg.lib()
    probs, keep, total = [], [], 0
    for idx, (o, m, n, k) in enumerate(ti.batch_shapes(0)):
        if len(probs) >= count:
            break
        # op "x", kc 0: the first `count` problems of the batch, any class
        if op != "x" and (o != op or next(w for w in widths if w >= min(k, 32 if o == "l" else 16)) != kc):
            continue
        lda, ldb = (m + pe - 1) // pe * pe, (n + pe - 1) // pe * pe
        tA = torch.empty((n, lda), dtype=torch.float32, device="cuda")
        tB = torch.empty((k, ldb), dtype=torch.float32, device="cuda")
        tC = torch.empty((k, lda), dtype=torch.float32, device="cuda")
        pkg.check(lib.tsm2_fill_uniform_s(m, n, idx, ti.MID_A, tA.data_ptr(), lda, 0))
        pkg.check(lib.tsm2_fill_uniform_s(n, k, idx, ti.MID_B, tB.data_ptr(), ldb, 0))
        keep += [tA, tB, tC]
        probs.append(bt.problem(o, m, n, k, tA.data_ptr(), lda, tB.data_ptr(), ldb, tC.data_ptr(), lda))
        total += 4 * (m * n + n * k + m * k)
    plan = bt.BatchPlan(probs, flags)
    l2_flush, _ = make_l2_flush(torch, 0)
    ts = []
    for r in range(args.warmup + args.steps):
        l2_flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.execute(0)
        e1.record()
        torch.cuda.synchronize()
        if r >= args.warmup:
            ts.append(e0.elapsed_time(e1))
    pkg.check(pkg.tsm2_get_device_status(0))
    ms = statistics.median(ts)
    print(json.dumps({"batch_case": args.batch_case, "problems": len(probs), "launches": plan.num_launches(),
                      "classes": [c["name"] for c in plan.classes()],
                      "ms": round(ms, 4), "gbs": round(total / (ms * 1e-3) / 1e9, 1), "algorithmic_bytes": total}),
          flush=True)
    plan.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cublas", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fwdbwd", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-crossover", action="store_true")
    ap.add_argument("--case", default=None, help="op:dtype:m:n:k, e.g. r:f32:8192:8192:16 -- time one multiply only (op r, l or x; dtype "
                         "f32, f64, or for op r bf16 / bf16hilo)")
    ap.add_argument("--batch-case", default=None, help="op:kc:count:flags[:pitch], e.g. l:32:20:1 -- time one tile class of the "
                    "batched workload (its first `count` problems) as one plan")
    ap.add_argument("--host-case", default=None, help="op:m:n:k:mode, e.g. r:30720:30720:16:0 -- time one host-operand "
                    "multiply (binary32; mode 0 SM copy kernels, 1 copy engines)")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.host_case:
        return run_host_case(args)
    if args.batch_case:
        return run_batch_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
