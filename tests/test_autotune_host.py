"""Host-side logic of the batched-plan tuner (no GPU): SM shares, the
problem-set key and the JSON cache."""
import json
import multiprocessing as mp
import os

from paper_2002_03258_gb300.autotune import load_cache, problem_set_key, shares_from_times, store_cache
from paper_2002_03258_gb300.batched import problem


def test_shares_proportional_to_class_time():
    g = shares_from_times([1.0, 3.0], 152)
    assert g == [1 + int(150 * 0.25), 1 + int(150 * 0.75)]
    assert sum(g) <= 152
    # Every class keeps at least one block, even with more classes than SMs.
    assert shares_from_times([0.0, 0.0, 5.0], 2) == [1, 1, 1]
    assert shares_from_times([0.0, 0.0], 10) == [1, 1]


def test_problem_set_key_depends_on_every_shape_field():
    base = [problem("r", 100, 200, 4, 0, 100, 0, 200, 0, 100), problem("l", 1 << 16, 8, 8, 0, 1 << 16, 0, 8, 0, 1 << 16)]
    k0 = problem_set_key(base)
    assert k0 == problem_set_key(list(base))
    variants = [
        [problem("l", 100, 200, 4, 0, 100, 0, 200, 0, 100), base[1]],
        [problem("r", 101, 200, 4, 0, 101, 0, 200, 0, 101), base[1]],
        [problem("r", 100, 200, 5, 0, 100, 0, 200, 0, 100), base[1]],
        [problem("r", 100, 200, 4, 0, 104, 0, 200, 0, 100), base[1]],
        [base[1], base[0]],
    ]
    assert len({k0} | {problem_set_key(v) for v in variants}) == 1 + len(variants)
    # Pointers are not part of the key: the same shapes reuse the tuning.
    moved = [problem("r", 100, 200, 4, 4096, 100, 8192, 200, 16384, 100), base[1]]
    assert problem_set_key(moved) == k0


def test_cache_roundtrip_and_bad_files(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    assert load_cache(p) == {}
    store_cache(p, "a", {"flags": 1, "grids": [3, 4], "serial": False, "ms": 1.5})
    store_cache(p, "b", {"flags": 0, "grids": [7], "serial": True, "ms": 2.0})
    c = load_cache(p)
    assert c["a"]["grids"] == [3, 4] and c["b"]["serial"] is True
    assert [f.name for f in (tmp_path / "sub").iterdir()] == ["tune.json"]  # no temporary left behind
    with open(p, "w") as f:
        f.write("{ truncated")
    assert load_cache(p) == {}
    with open(p, "w") as f:
        json.dump([1, 2], f)
    assert load_cache(p) == {}
    store_cache(p, "c", {"ms": 1.0})
    assert load_cache(p) == {"c": {"ms": 1.0}}


def _writer(path, i, n):
    for j in range(n):
        store_cache(path, f"w{i}_{j}", {"ms": float(j)})


def test_concurrent_writers_never_leave_a_partial_file(tmp_path):
    # Concurrent tuners may drop each other's entries (last writer wins), but a
    # reader must always find a whole JSON object.
    p = str(tmp_path / "tune.json")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_writer, args=(p, i, 20)) for i in range(3)]
    for q in procs:
        q.start()
    while any(q.is_alive() for q in procs):
        if os.path.exists(p):
            with open(p) as f:
                assert isinstance(json.load(f), dict)
    for q in procs:
        q.join()
        assert q.exitcode == 0
    with open(p) as f:
        final = json.load(f)
    assert final and all(isinstance(v, dict) and "ms" in v for v in final.values())
    assert not [f for f in os.listdir(tmp_path) if f != "tune.json"]


from paper_2002_03258_gb300 import perfmodel  # noqa: E402
from paper_2002_03258_gb300.autotune import (  # noqa: E402
    MERGE_L, MERGE_R, candidates, in_flight_bytes, seed_candidate, stage_bytes)

INFOS = [  # the compiled variants' parameters (tsm2_batch_v*.cu)
    {"variant": 0, "stages": 5, "rows_per_lane": 8, "inner_per_warp": 4},
    {"variant": 1, "stages": 4, "rows_per_lane": 8, "inner_per_warp": 4},
    {"variant": 2, "stages": 5, "rows_per_lane": 4, "inner_per_warp": 4},
    {"variant": 3, "stages": 5, "rows_per_lane": 4, "inner_per_warp": 8},
]
GB300 = perfmodel.Gpu("GB300", 79500.0, 6785.0, sms=152, clock_ghz=2.07)


def test_stage_and_in_flight_bytes():
    assert stage_bytes(INFOS[0]) == 256 * 32 * 4      # 256 rows x 32 inner columns, binary32
    assert stage_bytes(INFOS[2]) == 128 * 32 * 4
    assert stage_bytes(INFOS[3]) == 128 * 64 * 4
    assert in_flight_bytes(INFOS[0]) == 4 * 32768
    assert in_flight_bytes(INFOS[1]) == 3 * 32768


def test_seed_follows_the_model():
    # Little's law on GB300: ~21.6 KB per SM at 1000 cycles; every variant
    # covers it, so the most rows per lane (then stages) wins: variant 0.
    need = perfmodel.bytes_in_flight_per_sm(6785.0, 152, 2.07, 1000.0)
    assert 20000 < need < 23000
    # t2 threshold at the sustained FMA rate: 79.5 TF x 0.65 / 6.785 TB/s x 4
    # = 30.5 columns < 32, so the seed keeps the classes apart; at the full
    # peak (the paper's assumption) it would merge them.
    assert seed_candidate(INFOS, GB300) == (0, 0, "single")
    assert seed_candidate(INFOS, GB300, fma_sustained=1.0) == (0, MERGE_R | MERGE_L, "single")
    # a latency so long that only the deepest rings qualify
    deep = seed_candidate(INFOS, GB300, latency_cycles=4 * 2.07 * 152 * 98304 / 6785.0 / 4)
    assert deep[0] in (0, 2, 3)
    # nothing qualifies: the largest in-flight volume
    assert seed_candidate(INFOS, GB300, latency_cycles=1e9)[0] == 0
    # a GPU whose t2 threshold is below 32 columns: no merging (padding costs)
    slow = perfmodel.Gpu("x", 1000.0, 6785.0, sms=152, clock_ghz=2.07)
    assert seed_candidate(INFOS, slow)[1] == 0


def test_candidates_cover_the_space_seed_first():
    c = candidates(4, seed=(2, 0, "serial"))
    assert c[0] == (2, 0, "serial")
    assert len(c) == 4 * 2 * 2 and len(set(c)) == len(c)
    assert {v for v, _, _ in c} == {0, 1, 2, 3}
    assert {m for _, _, m in c} == {"single", "serial"}
