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
