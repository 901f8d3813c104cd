"""Pins of the oracle's format planning: degree order (Section 3.1 Solution 2),
Algorithm 1 (tile count), Algorithms 2-3 (workload size, performance model)
and the composite packing of Solution 3; bitonic partition (Section 3.2).

Pinned by the worked example of Figure 1 (tests/golden/fig1_composite.txt),
hand-computed model times, exhaustive search over WL under the same model,
and coverage invariants of the packing."""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _const_table(v=1.0, nlog=21):
    return nlog, np.full(2 * nlog * nlog, v)


def _major_table(row_perf, col_perf, nlog=21):
    perf = np.empty(2 * nlog * nlog)
    perf[: nlog * nlog] = row_perf
    perf[nlog * nlog:] = col_perf
    return nlog, perf


def _fixture():
    d = {"workload": []}
    for line in open(os.path.join(GOLD, "fig1_composite.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "workload":
            d["workload"].append(tuple(int(v) for v in line[1:]))
        else:
            d[line[0]] = [int(v) for v in line[1:]]
    return d


def test_fig1_tiles_and_composite_partition():
    g = _fixture()
    assert oracle.alg1_tiles(g["sorted_col_len"], g["tile_width"][0]) == g["expect_ntile"][0]
    rl = np.array(g["tile0_row_len"])
    part = oracle.partition_tile(np.arange(rl.size), rl, heavy=0, wl=g["wl"][0],
                                 max_warps=1000, rule=0, table=_const_table())
    got = list(zip(part["wl_first"], part["wl_h"], part["wl_w"], part["wl_major"]))
    assert got == g["workload"]


def test_degree_order_is_stable_descending_bijection():
    rng = np.random.default_rng(0)
    length = rng.integers(0, 6, 200)
    pi, inv = oracle.degree_order(length)
    assert sorted(inv.tolist()) == list(range(200))
    assert np.all(pi[inv] == np.arange(200))
    s = length[inv]
    assert np.all(np.diff(s) <= 0)
    for k in range(199):       # ties by ascending id
        if s[k] == s[k + 1]:
            assert inv[k] < inv[k + 1]


def test_alg1_hand_cases():
    assert oracle.alg1_tiles([5, 4, 3, 2, 2, 1, 1, 1], 2) == 3   # stops at a length-1 start
    assert oracle.alg1_tiles([5, 4, 3, 3, 2, 2, 2, 2], 2) == 4   # stops at n / tile_width
    assert oracle.alg1_tiles([5, 4, 3, 3, 2, 2, 2, 2, 9], 2) == 4  # floor(9/2) = 4
    assert oracle.alg1_tiles([1, 1, 1, 1], 2) == 0
    assert oracle.alg1_tiles([3, 3, 3], 4) == 0                  # n < tile width


def test_alg3_hand_computed():
    # lengths [4,3,2,1,1,1,1,1], WL=4, paper rule: workloads
    #   (4 x 1, row) -> 32 x 1;  (3 x 1, row) -> 32 x 1;
    #   (2 x 2, row: rows of length 2 and 1) -> 32 x 2;  (1 x 4, col) -> 1 x 32
    rl = np.array([4, 3, 2, 1, 1, 1, 1, 1])
    assert oracle.alg3_model(rl, 4, 1000, 0, _const_table(1.0)) == 160.0
    # row-major perf 2, column-major perf 1, 2 warps per iteration:
    # iter 0 = {32, 32} with P = 2 -> 32;  iter 1 = {64, 32} with P = 1.5 -> 64
    assert abs(oracle.alg3_model(rl, 4, 2, 0, _major_table(2.0, 1.0)) - 96.0) < 1e-12
    # size-independent performance: one iteration, t = total padded slots / P
    assert abs(oracle.alg3_model(rl, 4, 1000, 0, _const_table(4.0)) - 40.0) < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_alg2_equals_exhaustive_search(seed):
    rng = np.random.default_rng(seed)
    rl = np.sort(rng.zipf(1.8, 3000).clip(1, 400))[::-1].astype(np.int64)
    nlog = 21
    table = (nlog, rng.uniform(0.5, 2.0, 2 * nlog * nlog))
    nnz = int(rl.sum())
    max_warps = int(rng.integers(2, 40))
    wl, t = oracle.alg2_partition(rl, nnz, max_warps, 1, table)
    cands = [w for w in range(int(rl[0]), nnz // max_warps + 1, int(rl[0]))]
    if not cands:
        assert wl == rl[0]
    else:
        times = [oracle.alg3_model(rl, w, max_warps, 1, table) for w in cands]
        assert wl == cands[int(np.argmin(times))]
        assert t == min(times)


def test_partition_covers_every_nonzero_once_with_heavy_split():
    rng = np.random.default_rng(7)
    n = 500
    rl = rng.zipf(1.6, n).clip(0, 3000).astype(np.int64)
    rl[rng.random(n) < 0.2] = 0
    ids = rng.permutation(n).astype(np.int64)
    H = 64
    part = oracle.partition_tile(ids, rl, heavy=H, wl=0, max_warps=37, rule=1,
                                 table=_const_table())
    # every row's chunks add up to its length, each chunk <= H
    tot = {}
    for r, ch, L in zip(part["rank_row"], part["rank_chunk"], part["rank_len"]):
        assert 0 < L <= H
        tot[r] = tot.get(r, 0) + L
    assert tot == {int(i): int(L) for i, L in zip(ids, rl) if L > 0}
    # ranking: lengths non-increasing
    assert np.all(np.diff(part["rank_len"]) <= 0)
    # workloads tile the ranking contiguously, w = first row length
    pos = 0
    for f, h, w, mj in zip(part["wl_first"], part["wl_h"], part["wl_w"], part["wl_major"]):
        assert f == pos and h >= 1
        assert w == part["rank_len"][f]
        assert h == min(max(1, part["WL"] // w), len(part["rank_len"]) - f)
        rs, cs = h * ((w + 31) // 32 * 32), (h + 31) // 32 * 32 * w
        assert mj == (0 if rs < cs else 1)
        pos += h
    assert pos == len(part["rank_len"])


def test_tune_heavy_picks_min_cost_candidate():
    rng = np.random.default_rng(11)
    rl = rng.zipf(1.5, 4000).clip(0, 20000).astype(np.int64)
    ids = np.arange(rl.size, dtype=np.int64)
    table = _const_table()
    max_warps = 50
    H, wl = oracle.tune_heavy(ids, rl, max_warps, 1, table, split_cost=0.0)
    nnz = int(rl.sum())
    base = max(32, -(-nnz // max_warps))
    base = -(-base // 32) * 32
    costs = []
    for k in range(4):
        Hk = max(32, -(-(-(-base // (1 << k))) // 32) * 32)
        part = oracle.partition_tile(ids, rl, Hk, 0, max_warps, 1, table)
        costs.append((oracle.alg3_model(part["rank_len"], part["WL"], max_warps, 1, table),
                      Hk, part["WL"]))
    best = min(costs, key=lambda c: c[0])
    assert (H, wl) == (best[1], best[2])


def test_bitonic_partition_deals_back_and_forth():
    rl = np.array([9, 8, 7, 6, 5, 4, 3, 2, 1])
    part = oracle.bitonic_partition(rl, 3)
    assert part.tolist() == [0, 1, 2, 2, 1, 0, 0, 1, 2]
    rng = np.random.default_rng(1)
    rl = rng.zipf(1.7, 10000).clip(1, 10 ** 5)
    part = oracle.bitonic_partition(rl, 4)
    counts = np.bincount(part, minlength=4)
    assert counts.max() - counts.min() <= 1
    loads = np.bincount(part, weights=rl, minlength=4)
    # the largest row bounds the imbalance of a bitonic deal
    assert loads.max() - loads.min() <= rl.max()


def test_plan_format_small_rmat():
    import graphgen
    rp, col = graphgen.rmat(10, 8, seed=1)
    n = rp.shape[0] - 1
    plan = oracle.plan_format(rp, col, tile_width=64, max_warps=300, table=_const_table())
    outdeg = np.diff(rp)
    assert plan["ntile"] == oracle.alg1_tiles(outdeg[plan["inv"]], 64)
    # every non-zero of M lands in exactly one tile: in-tile lengths add up
    M = oracle.build_M(rp, col)
    indeg = np.diff(M[0])
    total = np.zeros(n, np.int64)
    for c0, c1, H, part in plan["tiles"]:
        for r, L in zip(part["rank_row"], part["rank_len"]):
            total[r] += L
    assert np.array_equal(total, indeg[plan["inv"]])
    assert np.array_equal(np.sort(plan["zero_rows"]), np.flatnonzero(indeg[plan["inv"]] == 0))


@pytest.mark.parametrize("rule,major", [(2, 0), (3, 1)])
def test_forced_storage_rules_are_the_special_cases(rule, major):
    # rule 2: every workload row-major (CSR-vector); rule 3: every workload
    # column-major (ELL); the ranking and the rectangles do not depend on
    # the rule, only the storage major (and so the padded size) does
    rng = np.random.default_rng(11)
    n = 400
    rl = rng.zipf(1.7, n).clip(0, 2000).astype(np.int64)
    ids = rng.permutation(n).astype(np.int64)
    base = oracle.partition_tile(ids, rl, heavy=0, wl=96, max_warps=29, rule=1, table=_const_table())
    part = oracle.partition_tile(ids, rl, heavy=0, wl=96, max_warps=29, rule=rule, table=_const_table())
    assert np.all(np.asarray(part["wl_major"]) == major)
    for k in ("rank_row", "rank_len", "wl_first", "wl_h", "wl_w"):
        assert np.array_equal(np.asarray(part[k]), np.asarray(base[k]))


@pytest.mark.parametrize("w,h", [(32, 32), (64, 32), (16, 16)])
def test_rule1_tie_goes_to_column_major(w, h):
    # h rows of w entries and WL = w * h: one w x h workload whose row-major
    # and column-major forms pad to the same number of slots; rule 1 then
    # stores it column-major (its rows side by side), the paper's rule
    # (w >= h) row-major
    ids = np.arange(h, dtype=np.int64)
    rl = np.full(h, w, np.int64)
    for rule, major in ((1, 1), (0, 0)):
        part = oracle.partition_tile(ids, rl, heavy=0, wl=w * h, max_warps=8, rule=rule,
                                     table=_const_table())
        assert list(part["wl_h"]) == [h] and list(part["wl_w"]) == [w]
        assert list(part["wl_major"]) == [major]


# ---- the row cap (at most max_rows rows per workload, GB300 reading of the
# packing step) and the per-chunk split cost of the heavy-row tuning, pinned
# by cases worked out by hand below (not by the builder)

def _cap_case():
    # 40 rows of 64 entries, then 70 rows of 1 entry; WL = 2560 = 40 * 64
    return np.array([64] * 40 + [1] * 70, np.int64)


def test_row_cap_packing_hand_computed():
    rl = _cap_case()
    ids = np.arange(rl.size, dtype=np.int64)
    # cap 32 (rule 1):
    #   rank 0:  w = 64, h = min(2560/64 = 40, 32) = 32: row-major 32 * 64 =
    #            2048 slots, column-major 32 * 64 = 2048 -> tie -> column-major
    #   rank 32: w = 64 (rows 32..39 have 64 entries), h = 32 -> column-major
    #   rank 64: w = 1,  h = min(2560, 32, 46 left) = 32 -> column-major
    #   rank 96: w = 1,  h = 14 (the rows left) -> column-major
    capped = oracle.partition_tile(ids, rl, heavy=0, wl=2560, max_warps=1000, rule=1,
                                   table=_const_table(), max_rows=32)
    assert list(capped["wl_first"]) == [0, 32, 64, 96]
    assert list(capped["wl_h"]) == [32, 32, 32, 14]
    assert list(capped["wl_w"]) == [64, 64, 1, 1]
    assert list(capped["wl_major"]) == [1, 1, 1, 1]
    # no cap: rank 0 takes all 40 rows of 64 (row-major 40 * 64 = 2560 <
    # column-major 64 * 64 = 4096), rank 40 the 70 one-entry rows
    # (column-major, h padded to 96)
    free = oracle.partition_tile(ids, rl, heavy=0, wl=2560, max_warps=1000, rule=1,
                                 table=_const_table(), max_rows=0)
    assert list(free["wl_first"]) == [0, 40]
    assert list(free["wl_h"]) == [40, 70]
    assert list(free["wl_major"]) == [0, 1]


def test_row_cap_model_hand_computed():
    rl = _cap_case()
    # padded sizes with the cap: 64 * 32 + 64 * 32 + 1 * 32 + 1 * 32 = 4160
    # slots, all column-major; without it: 64 * 40 (row-major) + 1 * 96
    # (column-major) = 2656
    assert oracle.alg3_model(rl, 2560, 1000, 1, _const_table(1.0), max_rows=32) == 4160.0
    assert oracle.alg3_model(rl, 2560, 1000, 1, _const_table(1.0), max_rows=0) == 2656.0
    # row-major table 2, column-major 1, one warp per iteration (Eq. 1):
    # capped: four column-major iterations, 2048 + 2048 + 32 + 32 = 4160;
    # uncapped: 2560 / 2 + 96 / 1 = 1376
    t = _major_table(2.0, 1.0)
    assert abs(oracle.alg3_model(rl, 2560, 1, 1, t, max_rows=32) - 4160.0) < 1e-9
    assert abs(oracle.alg3_model(rl, 2560, 1, 1, t, max_rows=0) - 1376.0) < 1e-9
    # two warps per iteration, table by column-major height bucket: h_pad 32
    # (log2 5) runs at 4, everything else at 1 -> capped iterations
    # {2048, 2048} at P = 4 and {32, 32} at P = 4: 1024 + 16 = 1040
    nlog = 21
    perf = np.ones(2 * nlog * nlog)
    for lw in range(nlog):
        perf[(1 * nlog + lw) * nlog + 5] = 4.0
    assert abs(oracle.alg3_model(rl, 2560, 2, 1, (nlog, perf), max_rows=32) - 1040.0) < 1e-9
    # the cap bounds rows, not WL: a cap of 40 leaves this plan as uncapped
    assert oracle.alg3_model(rl, 2560, 1000, 1, _const_table(1.0), max_rows=40) == 2656.0


def test_row_cap_one_entry_rows():
    # 100 one-entry rows, cap 32: workloads of 32, 32, 32 and 4 rows, each
    # a 1 x 32 column-major rectangle (128 padded slots in all)
    rl = np.ones(100, np.int64)
    part = oracle.partition_tile(np.arange(100, dtype=np.int64), rl, heavy=0, wl=1000,
                                 max_warps=1000, rule=1, table=_const_table(), max_rows=32)
    assert list(part["wl_h"]) == [32, 32, 32, 4]
    assert list(part["wl_major"]) == [1, 1, 1, 1]
    assert oracle.alg3_model(rl, 1000, 1000, 1, _const_table(1.0), max_rows=32) == 128.0
    # by height bucket: h_pad 32 at 2 and h_pad 128 (log2 7) at 1: capped
    # 128 / 2 = 64, uncapped one 1 x 128 rectangle 128 / 1 = 128
    nlog = 21
    perf = np.ones(2 * nlog * nlog)
    perf[(1 * nlog + 0) * nlog + 5] = 2.0
    assert abs(oracle.alg3_model(rl, 1000, 1000, 1, (nlog, perf), max_rows=32) - 64.0) < 1e-12
    assert abs(oracle.alg3_model(rl, 1000, 1000, 1, (nlog, perf), max_rows=0) - 128.0) < 1e-12


def _split_table():
    # every shape at 1 except row-major rectangles 64..127 slots wide (w_pad
    # 128 -> log2 7), which run at 0.5
    nlog = 21
    perf = np.ones(2 * nlog * nlog)
    for lh in range(nlog):
        perf[(0 * nlog + 7) * nlog + lh] = 0.5
    return nlog, perf


@pytest.mark.parametrize("split_cost,H,wl", [(0.0, 64, 64), (10.0, 64, 64), (42.0, 64, 64),
                                             (43.0, 128, 128), (50.0, 128, 128)])
def test_tune_heavy_split_cost_hand_computed(split_cost, H, wl):
    # One row of 128 entries and four of 32; nnz = 256, max_warps = 2:
    # base = 128, candidates H = 128, 64, 32 (k = 3 gives 32 again, skipped).
    #   H = 128: no split; Algorithm 2 range WL in {128}: workloads 128 x 1
    #            (row-major, w_pad 128 -> 0.5) and 32 x 4 (1) in one
    #            iteration: 256 / 0.75 = 341.33; no chunk
    #   H = 64:  virtual rows 64, 64, 32 x 4; WL in {64, 128} both model 256
    #            (every rectangle at 1), the first is kept: WL = 64; 2 chunks
    #   H = 32:  eight 32-entry virtual rows, model 256 for every WL; 4 chunks
    # cost = model + split_cost * chunks: H = 64 wins while
    # 256 + 2 s < 341.33, i.e. s < 42.67; above that H = 128 (cost 341.33)
    rl = np.array([128, 32, 32, 32, 32], np.int64)
    ids = np.arange(5, dtype=np.int64)
    got = oracle.tune_heavy(ids, rl, 2, 1, _split_table(), split_cost=split_cost)
    assert got == (H, wl)
    # the same with the row cap on (no workload here exceeds 32 rows)
    assert oracle.tune_heavy(ids, rl, 2, 1, _split_table(), split_cost, max_rows=32) == (H, wl)


def test_split_chunk_count_hand_computed():
    rl = np.array([128, 32, 32, 32, 32, 0, 65], np.int64)
    # rows longer than H are counted by their chunks, the others not at all
    assert oracle.split_cost_chunks(rl, 128) == 0.0
    assert oracle.split_cost_chunks(rl, 64) == 2.0 + 2.0      # 128 -> 2, 65 -> 2
    assert oracle.split_cost_chunks(rl, 32) == 4.0 + 3.0      # 128 -> 4, 65 -> 3


def test_choose_rule_hand_cases():
    # 64 rows of 4 entries, WL = 128 -> two 4 x 32 workloads.  Constant
    # table: rules 0, 1, 3 store them column-major (4 x 32 = 128 slots
    # each), rule 2 row-major (32 x 32 = 1024 each): costs 256, 256, 2048,
    # 256 -> the first of the cheapest in the order 1, 0, 2, 3 is rule 1
    ids = np.arange(64, dtype=np.int64)
    rl = np.full(64, 4, np.int64)
    costs = [oracle.plan_cost(ids, rl, 0, 128, 1000, r, _const_table(), 0.0) for r in (0, 1, 2, 3)]
    assert costs == [256.0, 256.0, 2048.0, 256.0]
    assert oracle.choose_rule(ids, rl, 0, 128, 1000, _const_table(), 0.0) == 1
    # 32 rows of 32 entries, WL = 1024 -> one 32 x 32 workload: rules 0 and
    # 2 store it row-major, 1 (tie) and 3 column-major.  Row-major table 2,
    # column-major 1: 512 for rules 0 and 2, 1024 for 1 and 3 -> rule 0
    # (before 2 in the order)
    ids = np.arange(32, dtype=np.int64)
    rl = np.full(32, 32, np.int64)
    t = _major_table(2.0, 1.0)
    assert [oracle.plan_cost(ids, rl, 0, 1024, 1000, r, t, 0.0) for r in (0, 1, 2, 3)] == \
        [512.0, 1024.0, 512.0, 1024.0]
    assert oracle.choose_rule(ids, rl, 0, 1024, 1000, t, 0.0) == 0
    # 10 rows of 64 entries, WL = 64 -> ten 64 x 1 workloads: rules 0, 1, 2
    # row-major (64 slots each), rule 3 column-major (64 x 32 = 2048 each).
    # Row-major table 0.001, column-major 1: 640 / 0.001 = 640000 against
    # 20480 -> rule 3
    ids = np.arange(10, dtype=np.int64)
    rl = np.full(10, 64, np.int64)
    t = _major_table(0.001, 1.0)
    costs = [oracle.plan_cost(ids, rl, 0, 64, 1000, r, t, 0.0) for r in (0, 1, 2, 3)]
    assert np.allclose(costs, [640000.0, 640000.0, 640000.0, 20480.0])
    assert oracle.choose_rule(ids, rl, 0, 64, 1000, t, 0.0) == 3
