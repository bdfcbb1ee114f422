"""Bounded waits of every pipelined kernel: with the waits forced to give up
(a negative wait budget: no barrier is tested, so every kernel takes its
timeout path whatever its timing), each kernel must stop instead of spinning,
record the timeout in the device status word and return; tsm2_get_device_status
then reports TSM2_ERR_TIMEOUT once (and resets the arrival counters), and the
next normal call must give a correct result.  (The real timer, a zero budget
that runs out, is exercised by test_parity_gpu.py.)

The kernels covered: TSM2R (binary64; binary32 with the on-chip B transpose),
TSM2L with resident B (binary32 and binary64) and with staged B, the
transposed TSM2R of the backward pass, the batched kernel (one persistent
launch and one launch per class) and the tensor-core bfloat16 kernel (plain
and hi+lo), whose early exit must still free its tensor memory -- a second
launch on the same SMs would otherwise wait for it.
"""
import numpy as np
import pytest

import tsm2_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import DevMat, assert_parity, call  # noqa: E402


def expect_timeout_then_recover(run, check):
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_wait_budget_ns(-1)
    try:
        assert run() == 0, pkg.tsm2_get_last_error_string()
        st = pkg.tsm2_get_device_status(0)
    finally:
        pkg.tsm2_set_wait_budget_ns(1_000_000_000)
    assert st == pkg.ERR_TIMEOUT
    assert "wait" in pkg.tsm2_get_last_error_string()
    assert pkg.tsm2_get_device_status(0) == 0  # reported once, then cleared
    assert run() == 0, pkg.tsm2_get_last_error_string()
    assert pkg.tsm2_get_device_status(0) == 0
    check()


# Sizes where every block runs dozens of stages, so the producer lane must
# wait for released stages (a single attempt then fails); TSM2L results are
# checked on sampled rows.
@pytest.mark.parametrize("op,dtype,m,n,k,cfg", [
    ("r", np.float64, 3000, 6000, 8, "r_f64"),
    ("r", np.float32, 4096, 8192, 12, "r_f32_kc12"),
    ("l", np.float32, 1 << 21, 32, 32, "l"),
    ("l", np.float32, 1 << 21, 16, 16, "l_f32_kc16"),
    ("l", np.float64, 1 << 21, 16, 16, "l"),
    ("l", np.float32, 1 << 19, 200, 16, "lt_f32"),
])
def test_single_problem_kernels(op, dtype, m, n, k, cfg):
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    A = ti.uniform_pm1(4, ti.MID_A, m, n, dtype)
    B = ti.uniform_pm1(4, ti.MID_B, n, k, dtype)
    dA, dB, dC = DevMat(A), DevMat(B), DevMat(np.zeros((m, k), dtype))

    def run():
        st = call(op, dtype, m, n, k, dA, dB, dC)
        assert pkg.tsm2_last_config().startswith(cfg), pkg.tsm2_last_config()
        return st

    def check():
        if m <= 10000:
            assert_parity(dC.numpy(), A, B, dtype)
            return
        rows = np.unique(np.concatenate([np.random.default_rng(1).integers(0, m, 3000), [0, m - 1]]))
        got = dC.view[torch.from_numpy(rows).cuda()].cpu().numpy()
        assert_parity(got, np.ascontiguousarray(A[rows]), B, dtype)

    expect_timeout_then_recover(run, check)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_transposed_tsm2r(dtype):
    import paper_2002_03258_gb300 as pkg
    m, n, k = 20000, 3000, 8
    A = ti.uniform_pm1(6, ti.MID_A, m, n, dtype)
    D = ti.uniform_pm1(6, ti.MID_B, m, k, dtype)
    dA, dD, dB = DevMat(A), DevMat(D), DevMat(np.zeros((n, k), dtype))
    fn = pkg.tsm2r_t_s if dtype == np.float32 else pkg.tsm2r_t_d

    def run():
        st = fn(m, n, k, dA.ptr, dA.ld, dD.ptr, dD.ld, dB.ptr, dB.ld, 0)
        assert not pkg.tsm2_last_config().startswith("simple")
        return st

    expect_timeout_then_recover(run, lambda: assert_parity(dB.numpy(), np.asfortranarray(A.T), D, dtype))


@pytest.mark.parametrize("mode", ["single", "serial"])
def test_batched_kernel(mode):
    import paper_2002_03258_gb300 as pkg
    import paper_2002_03258_gb300.batched as bt
    shapes = [("r", 3000, 3000, 16), ("r", 2500, 2500, 5), ("l", 200000, 24, 24), ("l", 90000, 8, 8)]
    items = []
    for idx, (op, m, n, k) in enumerate(shapes):
        A = ti.uniform_pm1(idx, ti.MID_A, m, n, np.float32)
        B = ti.uniform_pm1(idx, ti.MID_B, n, k, np.float32)
        ld = (m + 127) // 128 * 128
        dA, dB, dC = DevMat(A, ld), DevMat(B), DevMat(np.zeros((m, k), np.float32), ld)
        items.append((A, B, dA, dB, dC, bt.problem(op, m, n, k, dA.ptr, ld, dB.ptr, dB.ld, dC.ptr, ld)))
    plan = bt.BatchPlan([it[5] for it in items], 0)
    plan.set_mode(mode)

    def run():
        plan.execute(0)
        return 0

    def check():
        for A, B, dA, dB, dC, _ in items:
            assert_parity(dC.numpy(), A, B, np.float32)

    expect_timeout_then_recover(run, check)
    plan.close()


@pytest.mark.parametrize("hilo", [False, True])
def test_bf16_tensor_core_kernel(hilo):
    import oracle
    import paper_2002_03258_gb300 as pkg
    from test_bf16_gpu import check, dev_colmajor, split_host
    m, n, k = 4096, 8192, 16
    X = ti.logmag(3, ti.MID_A, m, n, np.float32)
    B = ti.uniform_pm1(3, ti.MID_B, n, k, np.float32)
    hi, lo = split_host(np.asfortranarray(X))
    thi, _ = dev_colmajor(hi, m, torch.int16)
    tlo, _ = dev_colmajor(lo, m, torch.int16)
    tB, vB = dev_colmajor(B)
    tC = torch.full((k, m), -9.0, device="cuda")

    def run():
        st = pkg.tsm2r_bf16(m, n, k, thi.data_ptr(), tlo.data_ptr() if hilo else None, m, vB.data_ptr(), n,
                            tC.data_ptr(), m, 0)
        assert pkg.tsm2_last_config().startswith("tc_bf16")
        return st

    def verify():
        Aeff = oracle.bf16_to_float(hi).astype(np.float64)
        if hilo:
            Aeff = Aeff + oracle.bf16_to_float(lo)
        check(tC.t().cpu().numpy().astype(np.float64), np.asfortranarray(Aeff), B.astype(np.float64), hilo,
              pkg.tsm2_last_config())

    # A launch that gave up, then (same SMs, same tensor memory) normal ones.
    expect_timeout_then_recover(run, verify)
