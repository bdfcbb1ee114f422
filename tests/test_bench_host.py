"""Host-side arithmetic of bench.py (no GPU): launch counting, algorithmic
bytes, the sweep's case list, the DRAM-traffic record's hash gate and the
clock-sample summary."""
import json

import bench


def test_algorithmic_bytes():
    # A read once, B read once, C written once.
    assert bench.alg_bytes(30720, 30720, 16, 4) == 4 * (30720 * 30720 + 30720 * 16 + 30720 * 16)
    assert bench.alg_bytes(1 << 23, 32, 32, 4) == 4 * ((1 << 23) * 32 + 32 * 32 + (1 << 23) * 32)
    assert bench.alg_bytes(0, 5, 5, 8) == 8 * 25


def test_launches_per_call():
    # One launch per column chunk: 16 columns for TSM2R, 32 for TSM2L; B is
    # transposed on chip, so no packing launches.
    assert bench.launches_per_call("r", 30720, 2) == 1
    assert bench.launches_per_call("r", 30720, 8) == 1
    assert bench.launches_per_call("r", 30720, 9) == 1
    assert bench.launches_per_call("r", 30720, 16) == 1
    assert bench.launches_per_call("r", 30720, 20) == 2   # 16 + 4
    assert bench.launches_per_call("r", 30720, 33) == 3   # 16 + 16 + 1
    assert bench.launches_per_call("l", 32, 32) == 1      # (op, inner n, k)
    assert bench.launches_per_call("l", 100, 100) == 4    # 32, 32, 32, 4
    assert bench.launches_per_call("l", 64, 40) == 2
    assert bench.launches_per_call("r", 100, 0) == 0


def test_sweep_cases():
    c = bench.cases(4)
    assert len(c) == 18
    r = [x for x in c if x[0] == "r"]
    l = [x for x in c if x[0] == "l"]
    assert sorted({(m, n) for _, m, n, _, _ in r}) == [(n, n) for n in bench.R_SIZES]
    assert sorted({k for *_, k, _ in r}) == bench.R_KS
    assert all(n == k for _, _, n, k, _ in l) and sorted({m for _, m, *_ in l}) == bench.L_MS
    assert all(es == 4 for *_, es in c)


def test_traffic_record_is_tied_to_the_kernel_sources(tmp_path, monkeypatch):
    rec = {"r_f32_kc16": {"r_30720x30720x16_f32": {"dram_bytes_per_launch": 123, "src_hash": "abc"}}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.txt").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "src_hash", lambda: "abc")
    assert bench.traffic_record("r_f32_kc16", "r_30720x30720x16_f32") == 123
    assert bench.traffic_record("r_f32_kc16", "r_20480x20480x16_f32") is None
    assert bench.traffic_record("r_f32_kc8", "r_30720x30720x16_f32") is None
    monkeypatch.setattr(bench, "src_hash", lambda: "changed")
    assert bench.traffic_record("r_f32_kc16", "r_30720x30720x16_f32") is None
    (tmp_path / "profiles" / "dram_traffic.txt").write_text("{ not json")
    monkeypatch.setattr(bench, "src_hash", lambda: "abc")
    assert bench.traffic_record("r_f32_kc16", "r_30720x30720x16_f32") is None


def test_committed_traffic_record_matches_the_sources():
    # The committed record must describe the kernel sources as they stand.
    v = bench.traffic_record("r_f32_kc16", "r_30720x30720x16_f32")
    alg = bench.alg_bytes(30720, 30720, 16, 4)
    assert v is not None and alg <= v < 1.05 * alg


def test_clock_sample_summary():
    idle = "0, 345, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    busy = "0, {}, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, {}"
    lines = [idle, busy.format(2070, "Not Active"), busy.format(1980, "Active"), busy.format(2070, "Not Active"),
             "garbage", "0, N/A, 2070, 0, 0, a, b, c, d"]
    r = bench.parse_clock_samples(lines)
    assert r["samples"] == 4
    assert r["sm_max_mhz"] == 2070.0
    assert r["sm_mhz"] == 2070.0          # median of the loaded samples (the idle one is left out)
    assert r["reasons"] == ["sw_power_cap"]
    hot = busy.format(1500, "Not Active").split(", ")
    hot[5] = "Active"                     # hw_slowdown
    assert bench.parse_clock_samples([", ".join(hot)])["reasons"] == ["hw_slowdown"]
    assert bench.parse_clock_samples(["x"]) is None
