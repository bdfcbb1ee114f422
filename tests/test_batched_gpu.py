"""Batched plans (tsm2_batch_plan_*): every problem of an uneven batch against
the CPU oracle, for every tile variant, class set, grid and launch mode (one
persistent launch, one launch per class, classes concurrently)."""
import numpy as np
import pytest

import tsm2_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import assert_parity  # noqa: E402


def make_batch(seed=3):
    import paper_2002_03258_gb300.batched as bt
    shapes = ti.batch_shapes(seed, n_r=18, n_l=18, r_n=(1, 1500), r_k=(1, 20), l_m=(1, 60000), l_n=(1, 40))
    shapes += [("r", 300, 0, 4), ("l", 0, 8, 8), ("r", 2000, 2000, 16), ("l", 70001, 64, 64)]
    items = []
    for idx, (op, m, n, k) in enumerate(shapes):
        lda = (max(m, 1) + 3) // 4 * 4
        ldb = (max(n, 1) + 3) // 4 * 4
        ldc = lda + 4
        A = ti.uniform_pm1(seed + idx, ti.MID_A, m, n, np.float32)
        B = ti.uniform_pm1(seed + idx, ti.MID_B, n, k, np.float32)
        tA = torch.zeros((max(n, 1), lda), device="cuda")
        tB = torch.zeros((max(k, 1), ldb), device="cuda")
        tC = torch.full((max(k, 1), ldc), float("nan"), device="cuda")
        if m and n:
            tA.t()[:m, :n].copy_(torch.from_numpy(np.ascontiguousarray(A)))
        if n and k:
            tB.t()[:n, :k].copy_(torch.from_numpy(np.ascontiguousarray(B)))
        items.append(dict(op=op, m=m, n=n, k=k, A=A, B=B, tA=tA, tB=tB, tC=tC,
                          p=bt.problem(op, m, n, k, tA.data_ptr(), lda, tB.data_ptr(), ldb, tC.data_ptr(), ldc)))
    return items


def check_all(items):
    torch.cuda.synchronize()
    for it in items:
        m, k = it["m"], it["k"]
        if m == 0 or k == 0:
            continue
        got = it["tC"].t()[:m, :k].cpu().numpy()
        assert_parity(got, it["A"], it["B"], np.float32)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("merge", [False, True])
def test_batch_plan_parity(variant, merge):
    import paper_2002_03258_gb300 as pkg
    import paper_2002_03258_gb300.batched as bt
    items = make_batch()
    flags = bt.variant_flag(variant) | ((bt.MERGE_R | bt.MERGE_L) if merge else 0)
    plan = bt.BatchPlan([it["p"] for it in items], flags)
    ncls = len(plan.classes())
    assert plan.num_launches() == 1  # default: the whole batch in one persistent launch
    assert all(c["name"].startswith(f"v{variant}_") for c in plan.classes())
    if merge:
        assert {c["name"].split("_kc")[1] for c in plan.classes()} <= {"16", "32"}
    plan.execute(0)
    assert pkg.tsm2_get_device_status(0) == 0
    check_all(items)
    first = [it["tC"].clone() for it in items]
    # same plan as a CUDA graph: same bits (same grid, same split points)
    for it in items:
        it["tC"].fill_(float("nan"))
    plan.graph_launch(0)
    torch.cuda.synchronize()
    for a, it in zip(first, items):
        assert torch.equal(torch.nan_to_num(a, 7.0), torch.nan_to_num(it["tC"], 7.0))
    # other grids of the single launch, then the per-class modes (other split
    # points: parity, not bits)
    for g in (1, 37):
        plan.set_single_grid(g)
        for it in items:
            it["tC"].fill_(float("nan"))
        plan.graph_launch(0)
        assert pkg.tsm2_get_device_status(0) == 0
        check_all(items)
    plan.set_mode("concurrent")
    assert plan.num_launches() == ncls
    for grids in ([1] * ncls, [3] * ncls, [37] * ncls):
        plan.set_grids(grids)
        for it in items:
            it["tC"].fill_(float("nan"))
        plan.graph_launch(0)
        assert pkg.tsm2_get_device_status(0) == 0
        check_all(items)
    plan.set_mode("serial")
    assert plan.num_launches() == ncls
    for it in items:
        it["tC"].fill_(float("nan"))
    plan.graph_launch(0)
    assert pkg.tsm2_get_device_status(0) == 0
    check_all(items)
    for c in range(ncls):  # one class alone touches only its own problems' C
        plan.execute_class(c, 0)
    assert pkg.tsm2_get_device_status(0) == 0
    check_all(items)
    plan.close()


def test_variant_info_and_bad_variant():
    import paper_2002_03258_gb300 as pkg
    import paper_2002_03258_gb300.batched as bt
    n = bt.num_variants()
    assert n == 4
    infos = [bt.variant_info(v) for v in range(n)]
    assert {i["stages"] for i in infos} >= {4, 5}
    assert {i["rows_per_lane"] for i in infos} >= {4, 8}
    assert {i["inner_per_warp"] for i in infos} >= {4, 8}
    with pytest.raises(pkg.TSM2Error) as e:
        bt.variant_info(n)
    assert e.value.status == pkg.ERR_INVALID_VALUE
    items = make_batch(seed=9)[:3]
    with pytest.raises(pkg.TSM2Error) as e:
        bt.BatchPlan([it["p"] for it in items], bt.variant_flag(n))
    assert e.value.status == pkg.ERR_INVALID_VALUE
    plan = bt.BatchPlan([it["p"] for it in items], 0)
    with pytest.raises(pkg.TSM2Error):
        plan.set_mode(7)
    with pytest.raises(pkg.TSM2Error):
        plan.set_single_grid(0)
    plan.close()


def test_batch_rejects_unaligned_and_bad_args():
    import paper_2002_03258_gb300 as pkg
    import paper_2002_03258_gb300.batched as bt
    t = torch.zeros(3 << 16, device="cuda")
    base = t.data_ptr()
    b_off, c_off = 1 << 18, 2 << 18  # bytes: A, B and C never overlap
    with pytest.raises(pkg.TSM2Error) as e:  # lda * 4 not a multiple of 16 bytes
        bt.BatchPlan([bt.problem("r", 33, 33, 4, base, 33, base + b_off, 36, base + c_off, 36)])
    assert e.value.status == pkg.ERR_UNSUPPORTED
    with pytest.raises(pkg.TSM2Error) as e:  # TSM2L with n > 64
        bt.BatchPlan([bt.problem("l", 100, 65, 4, base, 100, base + b_off, 68, base + c_off, 100)])
    assert e.value.status == pkg.ERR_UNSUPPORTED
    with pytest.raises(pkg.TSM2Error) as e:
        bt.BatchPlan([bt.problem("r", 10, 10, 2, base, 8, base + b_off, 12, base + c_off, 12)])  # lda < m
    assert e.value.status == pkg.ERR_INVALID_VALUE


def test_autotuner_picks_a_valid_plan(tmp_path):
    from paper_2002_03258_gb300.autotune import autotune
    items = make_batch(seed=5)
    plan, rec = autotune([it["p"] for it in items], reps=2, cache_path=str(tmp_path / "tune.json"))
    assert rec["ms"] > 0 and len(rec["trials"]) == 16
    assert rec["trials"][0]["seed"] and rec["seed"]["rank"] >= 1
    assert {t["variant"] for t in rec["trials"]} == {0, 1, 2, 3}
    assert {(t["stages"], t["rows_per_lane"], t["inner_per_warp"]) for t in rec["trials"]} >= {(5, 8, 4), (4, 8, 4)}
    for it in items:
        it["tC"].fill_(float("nan"))
    plan.graph_launch(0)
    check_all(items)
    plan2, rec2 = autotune([it["p"] for it in items], cache_path=str(tmp_path / "tune.json"))
    assert rec2.get("cached") and (rec2["flags"], rec2["variant"], rec2["mode"]) == (rec["flags"], rec["variant"],
                                                                                  rec["mode"])
    plan.close()
    plan2.close()


@pytest.mark.parametrize("variant,merge,mode,pitch", [(0, False, "single", 512), (3, True, "serial", 16),
                                                      (1, False, "single", 16)])
def test_batch_fullsize_workload_sampled(variant, merge, mode, pitch):
    """The benchmark's 512-problem workload (256 TSM2R n^2 x k, n in [512,
    8192]; 256 TSM2L, m in [2^14, 2^20], n = k in 4..32; about 43 GB of A and
    C), inputs generated on the device exactly as the benchmark makes them,
    one CUDA-graph launch of the plan; sampled rows of every fourth problem
    (128 of them, across the classes) against the oracle on rows regenerated
    on the host, and every entry of every C finite."""
    import paper_2002_03258_gb300 as pkg
    import paper_2002_03258_gb300.batched as bt
    lib = pkg.lib()
    shapes = ti.batch_shapes(0)
    probs, bufs = [], []
    pe = pitch // 4
    for idx, (op, m, n, k) in enumerate(shapes):
        lda = (m + pe - 1) // pe * pe
        ldb = (n + pe - 1) // pe * pe
        tA = torch.empty((n, lda), dtype=torch.float32, device="cuda")
        tB = torch.empty((k, ldb), dtype=torch.float32, device="cuda")
        tC = torch.full((k, lda), float("nan"), dtype=torch.float32, device="cuda")
        assert lib.tsm2_fill_uniform_s(m, n, idx, ti.MID_A, tA.data_ptr(), lda, 0) == 0
        assert lib.tsm2_fill_uniform_s(n, k, idx, ti.MID_B, tB.data_ptr(), ldb, 0) == 0
        bufs.append((tA, tB, tC))
        probs.append(bt.problem(op, m, n, k, tA.data_ptr(), lda, tB.data_ptr(), ldb, tC.data_ptr(), lda))
    plan = bt.BatchPlan(probs, bt.variant_flag(variant) | ((bt.MERGE_R | bt.MERGE_L) if merge else 0))
    plan.set_mode(mode)
    plan.graph_launch(0)
    assert pkg.tsm2_get_device_status(0) == 0
    # every fourth problem of the (shuffled) batch, 10 random rows plus the
    # first and the last
    rng = np.random.default_rng(11)
    checked = 0
    for idx, (op, m, n, k) in enumerate(shapes):
        if idx % 4:
            continue
        tA, tB, tC = bufs[idx]
        rows = np.unique(np.concatenate([rng.integers(0, m, 10), [0, m - 1]]))
        got = tC.t()[torch.from_numpy(rows).cuda(), :k].cpu().numpy()
        A_rows = ti.uniform_pm1(idx, ti.MID_A, m, n, np.float32, row_idx=rows)
        B = ti.uniform_pm1(idx, ti.MID_B, n, k, np.float32)
        assert_parity(got, A_rows, B, np.float32)
        checked += 1
    assert checked == 128
    # whole-C property at any size: every C entry of every problem finite
    for (tA, tB, tC), (op, m, n, k) in zip(bufs, shapes):
        assert bool(torch.isfinite(tC.t()[:m, :k]).all()), (op, m, n, k)
    plan.close()
    del bufs
    torch.cuda.empty_cache()


@pytest.mark.parametrize("mode", ["single", "serial"])
def test_class_with_fewer_groups_than_blocks(mode):
    """A TSM2R class whose work groups are fewer than the grid's blocks (one
    777^2 problem with 12 columns: 100 stages) beside larger classes: in one
    launch the class is shared by only as many blocks as it has groups, so
    every partial sum its fix-up adds was written."""
    import paper_2002_03258_gb300 as pkg
    import paper_2002_03258_gb300.batched as bt
    shapes = [("r", 3000, 3000, 16), ("r", 777, 777, 11), ("r", 300, 300, 3), ("l", 200001, 24, 24)]
    items = []
    for idx, (op, m, n, k) in enumerate(shapes):
        A = ti.uniform_pm1(idx, ti.MID_A, m, n, np.float32)
        B = ti.uniform_pm1(idx, ti.MID_B, n, k, np.float32)
        lda, ldb = (m + 3) // 4 * 4, (n + 3) // 4 * 4
        tA = torch.zeros((n, lda), device="cuda")
        tB = torch.zeros((k, ldb), device="cuda")
        tC = torch.full((k, lda), float("nan"), device="cuda")
        tA.t()[:m].copy_(torch.from_numpy(np.ascontiguousarray(A)))
        tB.t()[:n].copy_(torch.from_numpy(np.ascontiguousarray(B)))
        items.append(dict(op=op, m=m, n=n, k=k, A=A, B=B, tA=tA, tB=tB, tC=tC,
                          p=bt.problem(op, m, n, k, tA.data_ptr(), lda, tB.data_ptr(), ldb, tC.data_ptr(), lda)))
    for v in range(bt.num_variants()):
        plan = bt.BatchPlan([it["p"] for it in items], bt.variant_flag(v))
        plan.set_mode(mode)
        for it in items:
            it["tC"].fill_(float("nan"))
        plan.graph_launch(0)
        assert pkg.tsm2_get_device_status(0) == 0
        check_all(items)
        plan.close()


def test_adaptive_tsm2l_shares_keep_the_bits():
    """The single launch moves TSM2L row blocks between blocks from launch to
    launch (weights adapted to each block's measured rate); whole row blocks
    are computed alike whoever owns them, so every launch, the graph replay
    and the equal-share launch give the same bits."""
    import paper_2002_03258_gb300 as pkg
    import paper_2002_03258_gb300.batched as bt
    items = make_batch(seed=11)
    plan = bt.BatchPlan([it["p"] for it in items], bt.variant_flag(1))
    pkg.tsm2_set_balance(2)  # adapt although the plan is small
    try:
        plan.execute(0)
        assert pkg.tsm2_get_device_status(0) == 0
        check_all(items)
        first = [it["tC"].clone() for it in items]
        for r in range(6):
            for it in items:
                it["tC"].fill_(float("nan"))
            if r % 2:
                plan.graph_launch(0)
            else:
                plan.execute(0)
            torch.cuda.synchronize()
            assert pkg.tsm2_get_device_status(0) == 0
            for a, it in zip(first, items):
                assert torch.equal(torch.nan_to_num(a, 7.0), torch.nan_to_num(it["tC"], 7.0)), f"launch {r}"
        pkg.tsm2_set_balance(1)  # equal shares
        plan.close()
        plan = bt.BatchPlan([it["p"] for it in items], bt.variant_flag(1))  # a fresh graph
        for it in items:
            it["tC"].fill_(float("nan"))
        plan.execute(0)
        torch.cuda.synchronize()
        for a, it in zip(first, items):
            assert torch.equal(torch.nan_to_num(a, 7.0), torch.nan_to_num(it["tC"], 7.0))
    finally:
        pkg.tsm2_set_balance(0)
        plan.close()
