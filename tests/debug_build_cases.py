"""Parity cases run against the bounds-checking build (TSM2_DEBUG=1).

Executed in a child process by tests/test_debug_build_gpu.py, so that the
parent keeps the release library.  Every case must match the oracle and leave
the device status clean: no kernel computed an address outside its operand.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import torch  # noqa: E402

import paper_2002_03258_gb300 as pkg  # noqa: E402
import tsm2_inputs as ti  # noqa: E402
from gpu_util import DevMat, assert_parity, call  # noqa: E402


def check_status():
    st = pkg.tsm2_get_device_status(0)
    assert st == 0, (st, pkg.tsm2_get_last_error_string())


def products():
    cases = [("r", np.float32, 1031, 777, 5), ("r", np.float32, 4096, 8192, 16), ("r", np.float32, 3000, 9000, 12),
             ("r", np.float32, 2049, 4097, 20), ("r", np.float64, 1000, 1000, 8), ("l", np.float32, 100001, 32, 32),
             ("l", np.float32, 70001, 64, 64), ("l", np.float32, 30000, 200, 16), ("l", np.float64, 50000, 16, 16),
             ("r", np.float32, 33, 10241, 16)]
    for op, dt, m, n, k in cases:
        A = ti.uniform_pm1(1, ti.MID_A, m, n, dt)
        B = ti.uniform_pm1(1, ti.MID_B, n, k, dt)
        ld = (m + 3) // 4 * 4 + 4  # padded, still 16-byte rows
        dA, dB, dC = DevMat(A, ld), DevMat(B, (n + 3) // 4 * 4), DevMat(np.zeros((m, k), dt), ld, fill=-3.0)
        assert call(op, dt, m, n, k, dA, dB, dC) == 0, pkg.tsm2_get_last_error_string()
        check_status()
        assert not pkg.tsm2_last_config().startswith("simple"), pkg.tsm2_last_config()
        assert_parity(dC.numpy(), A, B, dt)
        assert np.all(dC.padding() == -3.0)
    return len(cases)


def noalloc_and_backward():
    lib = pkg.lib()
    m, n, k = 3000, 9000, 16
    A = ti.uniform_pm1(2, ti.MID_A, m, n, np.float32)
    B = ti.uniform_pm1(2, ti.MID_B, n, k, np.float32)
    dA, dB, dC = DevMat(A), DevMat(B), DevMat(np.zeros((m, k), np.float32))
    assert lib.tsm2r_s_noalloc(m, n, k, dA.ptr, m, dB.ptr, n, dC.ptr, m, 0) == 0
    assert not pkg.tsm2_last_config().startswith("simple")
    check_status()
    assert_parity(dC.numpy(), A, B, np.float32)
    m, n, k = 20000, 3000, 8
    A = ti.uniform_pm1(3, ti.MID_A, m, n, np.float32)
    D = ti.uniform_pm1(3, ti.MID_B, m, k, np.float32)
    dA, dD, dBt = DevMat(A), DevMat(D), DevMat(np.zeros((n, k), np.float32))
    assert pkg.tsm2r_t_s(m, n, k, dA.ptr, dA.ld, dD.ptr, dD.ld, dBt.ptr, dBt.ld, 0) == 0
    check_status()
    assert_parity(dBt.numpy(), np.asfortranarray(A.T), D, np.float32)
    return 2


def batched():
    import paper_2002_03258_gb300.batched as bt
    shapes = [("r", 3000, 3000, 16), ("r", 2500, 2500, 5), ("r", 777, 777, 11), ("l", 200001, 24, 24),
              ("l", 90000, 8, 8), ("l", 5000, 32, 32)]
    items = []
    for idx, (op, m, n, k) in enumerate(shapes):
        A = ti.uniform_pm1(idx, ti.MID_A, m, n, np.float32)
        B = ti.uniform_pm1(idx, ti.MID_B, n, k, np.float32)
        ld = (m + 3) // 4 * 4
        dA, dB, dC = DevMat(A, ld), DevMat(B, (n + 3) // 4 * 4), DevMat(np.zeros((m, k), np.float32), ld)
        items.append((A, B, dA, dB, dC, bt.problem(op, m, n, k, dA.ptr, ld, dB.ptr, dB.ld, dC.ptr, ld)))
    n = 0
    for v in range(bt.num_variants()):
        plan = bt.BatchPlan([it[5] for it in items], bt.variant_flag(v))
        for mode in ("single", "serial"):
            plan.set_mode(mode)
            for _, _, _, _, dC, _ in items:
                dC.view.fill_(float("nan"))
            plan.execute(0)
            check_status()
            for i, (A, B, _, _, dC, _) in enumerate(items):
                try:
                    assert_parity(dC.numpy(), A, B, np.float32)
                except AssertionError as e:
                    raise AssertionError(f"variant {v} mode {mode} problem {i} {shapes[i]} "
                                         f"classes {[c['name'] for c in plan.classes()]}: {e}") from None
            n += 1
        plan.close()
    return n


def main():
    # ALLOW_RELEASE=1: the same cases against the release build (for comparison)
    if os.environ.get("ALLOW_RELEASE") != "1":
        assert pkg.DEBUG and pkg.lib().tsm2_debug_checks() == 1, "not the debug build"
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    n = products() + noalloc_and_backward() + batched()
    torch.cuda.synchronize()
    print(f"DEBUG-BUILD-OK {n}", flush=True)


if __name__ == "__main__":
    main()
