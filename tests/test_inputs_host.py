"""The batched workload's shape generator (no GPU): counts, inclusive
bounds, determinism, the shuffle being a permutation, and the seed-0 byte
total that the benchmark's batched leg reports."""
from collections import Counter

import tsm2_inputs as ti


def alg_bytes(op, m, n, k):
    return 4 * (m * n + n * k + m * k)


def test_counts_shapes_and_bounds():
    shapes = ti.batch_shapes(0)
    assert len(shapes) == 512
    r = [s for s in shapes if s[0] == "r"]
    l = [s for s in shapes if s[0] == "l"]
    assert len(r) == 256 and len(l) == 256
    assert all(m == n and 512 <= n <= 8192 and 2 <= k <= 16 for _, m, n, k in r)   # square A, B n x k
    assert all(n == k and 4 <= n <= 32 and 2 ** 14 <= m <= 2 ** 20 for _, m, n, k in l)  # B n x n


def test_bounds_are_inclusive():
    shapes = ti.batch_shapes(3, n_r=400, n_l=400, r_n=(10, 12), r_k=(2, 3), l_m=(5, 6), l_n=(4, 5))
    assert {n for op, _, n, _ in shapes if op == "r"} == {10, 11, 12}
    assert {k for op, _, _, k in shapes if op == "r"} == {2, 3}
    assert {m for op, m, _, _ in shapes if op == "l"} == {5, 6}
    assert {n for op, _, n, _ in shapes if op == "l"} == {4, 5}


def test_deterministic_and_seeded():
    assert ti.batch_shapes(0) == ti.batch_shapes(0)
    assert ti.batch_shapes(0) != ti.batch_shapes(1)


def test_shuffle_is_a_permutation_of_the_drawn_problems():
    # The drawn problems (R then L) before the shuffle, rebuilt from the
    # generator's documented draw positions.
    n_r = n_l = 256
    drawn = []
    for i in range(n_r):
        n = int(ti.uniform_int(0, ti.MID_BATCH, [2 * i], 512, 8192)[0])
        k = int(ti.uniform_int(0, ti.MID_BATCH, [2 * i + 1], 2, 16)[0])
        drawn.append(("r", n, n, k))
    for i in range(n_l):
        m = int(ti.uniform_int(0, ti.MID_BATCH, [2 * n_r + 2 * i], 2 ** 14, 2 ** 20)[0])
        n = int(ti.uniform_int(0, ti.MID_BATCH, [2 * n_r + 2 * i + 1], 4, 32)[0])
        drawn.append(("l", m, n, n))
    shuffled = ti.batch_shapes(0)
    assert Counter(shuffled) == Counter(drawn)
    assert shuffled != drawn  # the order did change
    assert [s[0] for s in shuffled].count("r") == 256


def test_seed0_bytes_match_the_benchmark_workload():
    shapes = ti.batch_shapes(0)
    r = sum(alg_bytes(*s) for s in shapes if s[0] == "r")
    l = sum(alg_bytes(*s) for s in shapes if s[0] == "l")
    assert r + l == 42847462136          # the batched leg's algorithmic_bytes
    assert round(r / 1e9, 1) == 24.8 and round(l / 1e9, 1) == 18.0
