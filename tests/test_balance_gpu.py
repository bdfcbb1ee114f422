"""Run-time row-block claiming of TSM2L with B on chip (Algorithm 5's
persistent grid, Sec. 3.2.2, with the row blocks handed out from an atomic
counter instead of in equal static runs).

Checked: the oracle's bound in both partitions; the two partitions give the
same bits (every row block is computed whole by one thread block in a fixed
order, whoever claims it); repeated calls stay identical (the kernel rearms
its counters); every row block is claimed exactly once (the per-block trace
counts units); any grid size; a stream captured before it has a workspace
falls back to the static partition and replays correctly.
"""
import numpy as np
import pytest

import tsm2_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import DevMat, assert_parity, call  # noqa: E402

# (dtype, m, n, k, configuration prefix): resident-B shapes of every kind.
SHAPES = [
    (np.float32, 300001, 8, 8, "l_f32_kc8"),
    (np.float32, 2000003, 16, 16, "l_f32_kc16"),
    (np.float32, 1 << 20, 32, 32, "lw_f32_kc32"),
    (np.float32, 2000003, 12, 10, "l_f32_kc12"),
    (np.float32, 3000001, 3, 2, "l_f32_kc2"),
    (np.float32, 200000, 24, 20, "lw_f32_kc24"),
    (np.float32, 99999, 64, 5, "l_f32_kc8"),
    (np.float64, 500001, 16, 16, "l_f64_kc16"),
]


def sample_rows(m, count=2500, seed=2):
    rows = np.random.default_rng(seed).integers(0, m, count)
    return np.unique(np.concatenate([rows, [0, 1, m // 2, m - 2, m - 1]]))


def run_both(dtype, m, n, k, prefix, grid=0):
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(grid)
    A = ti.uniform_pm1(6, ti.MID_A, m, n, dtype)
    B = ti.uniform_pm1(6, ti.MID_B, n, k, dtype)
    ld = (m + 3) // 4 * 4
    dA, dB, dC = DevMat(A, ld), DevMat(B), DevMat(np.zeros((m, k), dtype), ld)
    out = {}
    try:
        for mode in (1, 0):
            pkg.tsm2_set_balance(mode)
            dC.view.fill_(float("nan"))
            assert call("l", dtype, m, n, k, dA, dB, dC) == 0, pkg.tsm2_get_last_error_string()
            assert pkg.tsm2_last_config().startswith(prefix), pkg.tsm2_last_config()
            assert pkg.tsm2_get_device_status(0) == 0
            out[mode] = dC.view.clone()
    finally:
        pkg.tsm2_set_balance(0)
        pkg.tsm2_set_grid(0)
    return A, B, dA, dB, dC, out


@pytest.mark.parametrize("dtype,m,n,k,prefix", SHAPES)
def test_claimed_row_blocks_match_oracle_and_static_bits(dtype, m, n, k, prefix):
    A, B, dA, dB, dC, out = run_both(dtype, m, n, k, prefix)
    assert torch.equal(out[0], out[1]), "run-time and static partitions differ"
    assert not torch.isnan(out[0]).any(), "a row block was never computed"
    rows = sample_rows(m)
    got = out[0][torch.from_numpy(rows).cuda()].cpu().numpy()
    assert_parity(got, np.ascontiguousarray(A[rows]), B, dtype)


@pytest.mark.parametrize("grid", [1, 3, 7, 40, 151])
def test_any_grid(grid):
    dtype, m, n, k, prefix = np.float32, 123457, 16, 16, "l_f32_kc16"
    A, B, dA, dB, dC, out = run_both(dtype, m, n, k, prefix, grid=grid)
    assert torch.equal(out[0], out[1])
    assert not torch.isnan(out[0]).any()
    rows = sample_rows(m, 1500, seed=grid)
    got = out[0][torch.from_numpy(rows).cuda()].cpu().numpy()
    assert_parity(got, np.ascontiguousarray(A[rows]), B, dtype)


def test_repeated_calls_rearm_the_counters():
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    m, n, k = 1 << 19, 8, 8
    A = ti.uniform_pm1(7, ti.MID_A, m, n, np.float32)
    B = ti.uniform_pm1(7, ti.MID_B, n, k, np.float32)
    dA, dB, dC = DevMat(A), DevMat(B), DevMat(np.zeros((m, k), np.float32))
    first = None
    for r in range(6):
        dC.view.fill_(float("nan"))
        assert call("l", np.float32, m, n, k, dA, dB, dC) == 0
        if first is None:
            first = dC.view.clone()
        else:
            assert torch.equal(dC.view, first), f"call {r} differs"
    assert pkg.tsm2_get_device_status(0) == 0
    rows = sample_rows(m)
    assert_parity(first[torch.from_numpy(rows).cuda()].cpu().numpy(), np.ascontiguousarray(A[rows]), B, np.float32)


def test_trace_counts_every_unit_once():
    """The per-block trace: units over all blocks = row blocks x stages per
    row block, each block's SM id below the SM count, times ordered."""
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    m, n, k = 1 << 20, 32, 32  # lw_f32_kc32: 1024-row blocks, 8 inner columns per stage
    A = ti.uniform_pm1(8, ti.MID_A, m, n, np.float32)
    B = ti.uniform_pm1(8, ti.MID_B, n, k, np.float32)
    dA, dB, dC = DevMat(A), DevMat(B), DevMat(np.zeros((m, k), np.float32))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    words = torch.zeros(4 * 1024, dtype=torch.int64, device="cuda")
    pkg.tsm2_set_trace(words.data_ptr(), 1024)
    try:
        assert call("l", np.float32, m, n, k, dA, dB, dC) == 0
        torch.cuda.synchronize()
    finally:
        pkg.tsm2_set_trace(None, 0)
    assert pkg.tsm2_last_config() == "lw_f32_kc32"
    t = words.view(-1, 4).cpu().numpy().astype(np.uint64)
    used = t[:, 0] > 0
    assert used.sum() == min(sms, m // 1024)
    t = t[used]
    units = (t[:, 3] & np.uint64(0xffffffff)).astype(np.int64)
    sm = (t[:, 3] >> np.uint64(32)).astype(np.int64)
    assert units.sum() == (m // 1024) * (32 // 8)
    assert np.all(units % 4 == 0)  # whole row blocks
    assert np.all(sm < sms)
    assert np.all(t[:, 0] <= t[:, 1]) and np.all(t[:, 1] <= t[:, 2])


def test_capture_without_workspace_uses_static_partition():
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    lib = pkg.lib()
    m, n, k = 300000, 16, 16
    A = ti.uniform_pm1(9, ti.MID_A, m, n, np.float32)
    B = ti.uniform_pm1(9, ti.MID_B, n, k, np.float32)
    dA, dB, dC = DevMat(A), DevMat(B), DevMat(np.zeros((m, k), np.float32))
    assert lib.tsm2l_s(m, n, k, dA.ptr, m, dB.ptr, n, dC.ptr, m, 0) == 0  # library state outside capture
    ref = dC.view.clone()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()  # no workspace yet on this stream
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        st = lib.tsm2l_s(m, n, k, dA.ptr, m, dB.ptr, n, dC.ptr, m, s.cuda_stream)
    assert st == 0, pkg.tsm2_get_last_error_string()
    for _ in range(3):
        dC.view.fill_(float("nan"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(dC.view, ref)
    assert pkg.tsm2_get_device_status(0) == 0
    # once the stream has a workspace, captured calls claim row blocks
    assert lib.tsm2l_s(m, n, k, dA.ptr, m, dB.ptr, n, dC.ptr, m, s.cuda_stream) == 0
    s.synchronize()
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=s):
        assert lib.tsm2l_s(m, n, k, dA.ptr, m, dB.ptr, n, dC.ptr, m, s.cuda_stream) == 0
    for _ in range(3):
        dC.view.fill_(float("nan"))
        torch.cuda.synchronize()
        g2.replay()
        torch.cuda.synchronize()
        assert torch.equal(dC.view, ref)
    assert pkg.tsm2_get_device_status(0) == 0



def test_several_column_passes():
    """k = 80: three launches (32 + 32 + 16 columns of C), each claiming the
    row blocks afresh from the rearmed counters."""
    dtype, m, n, k = np.float32, 500001, 24, 80
    A, B, dA, dB, dC, out = run_both(dtype, m, n, k, "l_f32_kc16")
    assert torch.equal(out[0], out[1])
    assert not torch.isnan(out[0]).any()
    rows = sample_rows(m, 1500, seed=5)
    got = out[0][torch.from_numpy(rows).cuda()].cpu().numpy()
    assert_parity(got, np.ascontiguousarray(A[rows]), B, dtype)


def test_timeout_while_claiming_then_recover():
    """Single-attempt waits on a tall shape: blocks give up part-way through
    their claims; the status reports the timeout once, the host clears the
    counters, and the next calls give the static partition's bits again."""
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    m, n, k = 1 << 22, 16, 16
    A = ti.uniform_pm1(10, ti.MID_A, m, n, np.float32)
    B = ti.uniform_pm1(10, ti.MID_B, n, k, np.float32)
    dA, dB, dC = DevMat(A), DevMat(B), DevMat(np.zeros((m, k), np.float32))
    pkg.tsm2_set_wait_budget_ns(0)
    try:
        assert call("l", np.float32, m, n, k, dA, dB, dC) == 0
        st = pkg.tsm2_get_device_status(0)
    finally:
        pkg.tsm2_set_wait_budget_ns(1_000_000_000)
    assert pkg.tsm2_last_config() == "l_f32_kc16"
    assert st in (0, pkg.ERR_TIMEOUT)
    assert pkg.tsm2_get_device_status(0) == 0
    outs = {}
    try:
        for mode in (1, 0, 0):
            pkg.tsm2_set_balance(mode)
            dC.view.fill_(float("nan"))
            assert call("l", np.float32, m, n, k, dA, dB, dC) == 0
            assert pkg.tsm2_get_device_status(0) == 0
            outs.setdefault(mode, []).append(dC.view.clone())
    finally:
        pkg.tsm2_set_balance(0)
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][0])
    rows = sample_rows(m, 1500, seed=6)
    got = outs[0][0][torch.from_numpy(rows).cuda()].cpu().numpy()
    assert_parity(got, np.ascontiguousarray(A[rows]), B, np.float32)


def test_two_streams_claim_independently():
    """Each stream has its own claim counters: two tall TSM2L products in
    flight at once on two streams (repeatedly, without synchronising between
    them) give the same bits as alone."""
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_path(0)
    pkg.tsm2_set_grid(0)
    lib = pkg.lib()
    shapes = [(1 << 21, 16, 16), (1500001, 8, 8)]
    mats = []
    for i, (m, n, k) in enumerate(shapes):
        A = ti.uniform_pm1(20 + i, ti.MID_A, m, n, np.float32)
        B = ti.uniform_pm1(20 + i, ti.MID_B, n, k, np.float32)
        ld = (m + 3) // 4 * 4
        mats.append((m, n, k, A, B, DevMat(A, ld), DevMat(B), DevMat(np.zeros((m, k), np.float32), ld)))
    ref = []
    for (m, n, k, A, B, dA, dB, dC) in mats:
        assert lib.tsm2l_s(m, n, k, dA.ptr, dA.ld, dB.ptr, dB.ld, dC.ptr, dC.ld, 0) == 0
        torch.cuda.synchronize()
        ref.append(dC.view.clone())
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for (m, n, k, A, B, dA, dB, dC), s in zip(mats, streams):  # workspaces outside the loop's timing
        assert lib.tsm2l_s(m, n, k, dA.ptr, dA.ld, dB.ptr, dB.ld, dC.ptr, dC.ld, s.cuda_stream) == 0
    torch.cuda.synchronize()
    for _ in range(5):
        for (m, n, k, A, B, dA, dB, dC), s in zip(mats, streams):
            dC.view.fill_(float("nan"))
        torch.cuda.synchronize()
        for (m, n, k, A, B, dA, dB, dC), s in zip(mats, streams):
            assert lib.tsm2l_s(m, n, k, dA.ptr, dA.ld, dB.ptr, dB.ld, dC.ptr, dC.ld, s.cuda_stream) == 0
        torch.cuda.synchronize()
        assert pkg.tsm2_get_device_status(0) == 0
        for r, (m, n, k, A, B, dA, dB, dC) in zip(ref, mats):
            assert torch.equal(dC.view, r)
    for r, (m, n, k, A, B, dA, dB, dC) in zip(ref, mats):
        rows = sample_rows(m, 1000, seed=m % 97)
        assert_parity(r[torch.from_numpy(rows).cuda()].cpu().numpy(), np.ascontiguousarray(A[rows]), B, np.float32)
