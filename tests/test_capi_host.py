"""C-ABI library on the CPU: it loads, exports every symbol include/spg.h
declares, rejects malformed input, and its host builder reproduces the
oracle's format plan exactly (integer work, bit-exact): degree order,
Algorithm 1 tiles, heavy-row threshold, Algorithm 2 workload size, row
ranking and workloads (Section 3.1 Solutions 2-3, Section 3.3), and the
packed slots hold exactly the non-zeros of M = W^T."""
import ctypes
import os
import re
import tempfile

import numpy as np
import pytest

import graphgen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def spg():
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_1103_2405_gb300 as m
    return m


def _header_symbols():
    text = open(os.path.join(ROOT, "include", "spg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spg_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(spg):
    L = spg.lib()
    syms = _header_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(spg.EXPORTS) == syms
    assert spg.version().startswith("spg")


def _table_file(perf, nlog=21):
    fd, path = tempfile.mkstemp(suffix=".txt")
    os.close(fd)
    with open(path, "w") as f:
        for mj in range(2):
            for lw in range(nlog):
                for lh in range(nlog):
                    f.write(f"{mj} {lw} {lh} {float(perf[(mj * nlog + lw) * nlog + lh])!r}\n")
    return path


CASES = [  # (scale, ef, tile_width, heavy, rule, max_warps, max_rows)
    (12, 8, 256, -1, 1, 300, -1),
    (12, 8, 64, 0, 0, 97, -1),
    (12, 8, -1, -1, 1, 9728, -1),
    (12, 8, 1024, 64, 1, 50, -1),
    (10, 16, 128, -1, 0, 13, -1),
    (12, 8, -1, -1, 1, 9728, 256),
    (12, 8, 512, -1, 1, 40, 37),
    (12, 8, 1024, -1, 2, 300, -1),
    (12, 8, -1, 64, 3, 9728, -1),
    (12, 8, 256, -1, 4, 300, -1),     # automatic storage rule per part
    (10, 16, 128, 0, 4, 13, 37),
    (12, 8, -1, -1, 4, 9728, -1),
]


@pytest.mark.parametrize("scale,ef,tw,heavy,rule,mw,mr", CASES)
def test_host_plan_matches_oracle(spg, scale, ef, tw, heavy, rule, mw, mr):
    nlog = 21
    perf = np.random.default_rng(scale * 7 + mw).uniform(1e9, 5e9, 2 * nlog * nlog)
    path = _table_file(perf)
    try:
        rp, col = graphgen.rmat(scale, ef, seed=1)
        f = spg.Format(rp, col, kind="pagerank", tile_width=tw, heavy_row=heavy, layout_rule=rule,
                       max_warps=mw, keep_plan=True, host_only=True, table=path, max_rows=mr)
        plan = oracle.plan_format(rp, col, tile_width=max(tw, 0), max_warps=mw,
                                  table=(nlog, perf), heavy=heavy, rule=rule, split_cost=2e-7,
                                  max_rows=max(mr, 0))
    finally:
        spg.load_table(None)
        os.unlink(path)
    pi, inv = f.perm()
    assert np.array_equal(pi, plan["pi"]) and np.array_equal(inv, plan["inv"])
    assert f.info()["ntile"] == plan["ntile"]
    for p, (c0, c1, H, part) in enumerate(plan["tiles"]):
        ti = f.tile_info(p)
        ex = f.export_plan(p)
        assert (ti["col_begin"], ti["col_end"]) == (c0, c1)
        assert ex["heavy"] == H and ex["WL"] == part["WL"]
        for k in ("rank_row", "rank_chunk", "rank_len", "wl_first", "wl_h", "wl_w", "wl_major"):
            assert np.array_equal(ex[k], part[k]), (p, k)
        assert ex["rule"] == part["rule"] == (rule if rule != 4 else ex["rule"])
    assert np.array_equal(f.zero_rows(), plan["zero_rows"])
    # the packed slots hold exactly M's entries (values bit-exact)
    r, c, v = f.export_entries()
    mrp, mcol, mval = oracle.build_M(rp, col)
    n = rp.shape[0] - 1
    got = np.lexsort((c, r))
    want = np.lexsort((mcol, np.repeat(np.arange(n), np.diff(mrp))))
    assert np.array_equal(r[got], np.repeat(np.arange(n), np.diff(mrp))[want])
    assert np.array_equal(c[got], mcol[want])
    assert np.array_equal(v[got].view(np.uint32), mval[want].view(np.uint32))


def test_pattern_only_layout_holds_the_same_matrix(spg):
    # column indices only; each column's value fl32(1/outdeg) comes back from
    # the per-column table, so the stored matrix is still exactly M
    rp, col = graphgen.rmat(11, 8, seed=3)
    f = spg.Format(rp, col, kind="pagerank", pattern_only=True, host_only=True, max_warps=200,
                   keep_plan=True)
    r, c, v = f.export_entries()
    mrp, mcol, mval = oracle.build_M(rp, col)
    n = rp.shape[0] - 1
    got = np.lexsort((c, r))
    want = np.lexsort((mcol, np.repeat(np.arange(n), np.diff(mrp))))
    assert np.array_equal(c[got], mcol[want])
    assert np.array_equal(v[got].view(np.uint32), mval[want].view(np.uint32))
    with pytest.raises(spg.SpgError):
        spg.Format(rp, col, kind="hits", pattern_only=True, host_only=True)


def test_hits_block_matrix_entries(spg):
    rp, col = graphgen.rmat(9, 8, seed=2)
    n = rp.shape[0] - 1
    f = spg.Format(rp, col, kind="hits", host_only=True, max_warps=64)
    r, c, v = f.export_entries()
    assert f.n == 2 * n and np.all(v == 1.0)
    src = np.repeat(np.arange(n), np.diff(rp))
    # Eq. 8: rows v < n hold (v, n+u) for u->v; rows n+u hold (n+u, v)
    want = set(zip(col.tolist(), (n + src).tolist())) | set(zip((n + src).tolist(), col.tolist()))
    assert set(zip(r.tolist(), c.tolist())) == want and len(r) == 2 * len(col)


@pytest.mark.parametrize("bad", ["nonsquare", "rowptr0", "decreasing", "colrange", "nnz"])
def test_malformed_csr_rejected(spg, bad):
    rp = np.array([0, 2, 3, 3], np.int64)
    col = np.array([1, 2, 0], np.int32)
    L = spg.lib()
    n, nc, nnz = 3, 3, 3
    if bad == "nonsquare":
        nc = 4
    elif bad == "rowptr0":
        rp = np.array([1, 2, 3, 3], np.int64)
    elif bad == "decreasing":
        rp = np.array([0, 2, 1, 3], np.int64)
    elif bad == "colrange":
        col = np.array([1, 3, 0], np.int32)
    elif bad == "nnz":
        nnz = 4
        col = np.array([1, 2, 0, 0], np.int32)
    csr = spg._Csr(n, nc, nnz, ctypes.c_void_p(rp.ctypes.data), ctypes.c_void_p(col.ctypes.data),
                   None, 0)
    opts = spg._Opts(0, 0, -1, 1, 64, 1, 0, 0, 0, -1, 0.0, None, 0, 0, 0, 0, 0, 0, None, 0, 0, 0, 0)
    h = ctypes.c_void_p()
    st = L.spg_build_format(ctypes.byref(csr), 1, ctypes.byref(opts), None, ctypes.byref(h))
    assert st == -1 and not h.value
    assert len(L.spg_last_error()) > 0


def test_degenerate_graphs_build(spg):
    # no edges at all; a single node; every row a zero row
    for rp, col in [(np.zeros(5, np.int64), np.zeros(0, np.int32)),
                    (np.zeros(2, np.int64), np.zeros(0, np.int32))]:
        f = spg.Format(rp, col, kind="pagerank", host_only=True, max_warps=64)
        info = f.info()
        assert info["nnz"] == 0 and info["zero_rows"] == rp.shape[0] - 1
        assert info["dangling_start"] == 0
        r, c, v = f.export_entries()
        assert r.size == 0


def test_batch_host_build_orders_within_each_graph(spg):
    graphs = [graphgen.chung_lu(n, 12 * n, 2.3, n / 4, seed=5 + i) for i, n in enumerate((300, 77, 1000))]
    b = spg.BatchFormat(graphs, host_only=True, max_warps=64)
    off = b.offsets
    assert off.tolist() == [0, 300, 377, 1377]
    pi = np.empty(b.n, np.int32)
    inv = np.empty(b.n, np.int32)
    spg._check(spg.lib().spg_format_perm(b._h, spg._ptr(pi)[0], spg._ptr(inv)[0]))
    for g, (rp, col) in enumerate(graphs):
        seg = inv[off[g]:off[g + 1]] - off[g]
        p_ref, inv_ref = oracle.degree_order(np.diff(rp))
        assert np.array_equal(seg, inv_ref)       # Solution 2 order within each graph


def test_batch_claim_order_only_reorders(spg):
    # graph-by-graph claim order (claim_order 0) against the ranking order
    # (claim_order 1): same plan, same stored entries; claim units never
    # span two graphs, so there are at least as many
    sizes = [40, 300, 77, 1000, 2500, 60, 90, 700, 1500, 33, 5000, 128]
    graphs = [graphgen.chung_lu(n, 12 * n, 2.3, n / 4, seed=50 + i) for i, n in enumerate(sizes)]
    b = spg.BatchFormat(graphs, host_only=True, max_warps=64, keep_plan=True)
    ref = spg.BatchFormat(graphs, host_only=True, max_warps=64, keep_plan=True, claim_order=1)
    pa, pb = b.export_plan(0), ref.export_plan(0)
    for k in ("rank_row", "rank_chunk", "rank_len", "wl_first", "wl_h", "wl_w", "wl_major"):
        assert np.array_equal(pa[k], pb[k]), k
    ea, eb = b.export_entries(), ref.export_entries()
    oa, ob = np.lexsort((ea[1], ea[0])), np.lexsort((eb[1], eb[0]))
    for x, y in zip(ea, eb):
        assert np.array_equal(x[oa], y[ob])
    assert b.tile_info(0)["nunits"] >= ref.tile_info(0)["nunits"]
    one = spg.BatchFormat(graphs, host_only=True, max_warps=64, unit_slots=1)
    assert one.tile_info(0)["nunits"] == one.tile_info(0)["nwl"] + -(-one.info()["zero_rows"] // 1024)


def test_bad_table_rejected(spg):
    fd, path = tempfile.mkstemp(suffix=".txt")
    with os.fdopen(fd, "w") as f:
        f.write("0 3 4 -1.0\n")
    with pytest.raises(spg.SpgError):
        spg.load_table(path)
    os.unlink(path)
    spg.load_table(None)


@pytest.mark.parametrize("P", [1, 2, 3, 7])
def test_partition_rows_matches_oracle(spg, P):
    rp, col = graphgen.rmat(12, 8, seed=2)
    mrp, _, _ = oracle.build_M(rp, col)
    rl = np.diff(mrp)
    part = spg.partition_rows(rl, P)
    assert np.array_equal(part, oracle.bitonic_partition(rl, P))
    assert np.array_equal(spg.partition_rows(np.zeros(0, np.int64), P), np.zeros(0, np.int32))
    with pytest.raises(spg.SpgError):
        spg.partition_rows(rl, 0)


def test_rank_formats_hold_their_rows(spg):
    # every rank holds exactly its rows of M, over all columns, in the order
    # of the whole matrix: the union of the ranks' entries is M
    rp, col = graphgen.rmat(11, 8, seed=3)
    n = rp.shape[0] - 1
    mrp, mcol, mval = oracle.build_M(rp, col)
    P = 3
    part = spg.partition_rows(np.diff(mrp), P)
    whole = spg.Format(rp, col, kind="pagerank", host_only=True, max_warps=200)
    pi, _ = whole.perm()
    got = []
    for r in range(P):
        f = spg.Format(rp, col, kind="pagerank", host_only=True, max_warps=200, row_part=part,
                       part_id=r, nparts=P)
        assert np.array_equal(f.perm()[0], pi)
        rr, cc, vv = f.export_entries()
        assert np.all(part[rr] == r)
        assert f.info()["zero_rows"] == int(np.sum((part == r) & (np.diff(mrp) == 0)))
        got.append((rr, cc, vv))
    r = np.concatenate([g[0] for g in got]); c = np.concatenate([g[1] for g in got])
    v = np.concatenate([g[2] for g in got])
    o = np.lexsort((c, r))
    mr = np.repeat(np.arange(n), np.diff(mrp))
    assert np.array_equal(r[o], mr) and np.array_equal(c[o], mcol)
    assert np.array_equal(v[o].view(np.uint32), mval.view(np.uint32))
    for bad in (dict(kind="hits"), dict(part_id=3), dict(keep_csr=True)):
        kw = dict(kind="pagerank", host_only=True, row_part=part, part_id=0, nparts=P)
        kw.update(bad)
        with pytest.raises(spg.SpgError):
            spg.Format(rp, col, **kw)


def test_claim_order_option_keeps_the_stored_entries(spg):
    # the claim order permutes whole workloads: the stored entries, their
    # values and the zero rows are the same in both orders; other values
    # are refused
    rp, col = graphgen.rmat(12, 8, seed=4)
    keys = []
    for order in (0, 1):
        f = spg.Format(rp, col, kind="pagerank", host_only=True, max_warps=200, claim_order=order)
        r, c, v = f.export_entries()
        o = np.lexsort((c, r))
        keys.append((r[o], c[o], v[o].view(np.uint32), f.zero_rows(), f.info()["padded_slots"]))
    for other in keys[1:]:
        for a, b in zip(keys[0], other):
            assert np.array_equal(a, b)
    with pytest.raises(spg.SpgError):
        spg.Format(rp, col, kind="pagerank", host_only=True, claim_order=2)


def test_claim_order_puts_the_longest_latency_chain_first(spg):
    # every workload row-major (rule 2), WL = 64: the rows of length 64 form
    # one-row workloads (a 2-step row: few round trips), the rows of length
    # 2 form 32-row workloads (32 rows walked one after another: many).
    # Ranking order stores the long rows first; longest-first stores the
    # 32-row workloads first.  Entries are exported in storage order.
    n = 200
    edges = [(u, v) for v in range(4) for u in range(100, 164)]
    edges += [(u, v) for v in range(4, 68) for u in (100, 101)]
    edges.sort()
    src = np.array([e[0] for e in edges], np.int64)
    col = np.array([e[1] for e in edges], np.int32)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp)
    first = {}
    for order in (0, 1):
        f = spg.Format(rp, col, kind="pagerank", host_only=True, wl=64, heavy_row=0, layout_rule=2,
                       max_warps=64, claim_order=order)
        r, c, v = f.export_entries()
        first[order] = int(r[0])
    assert first[1] in range(4)          # ranking order: a row of length 64
    assert first[0] in range(4, 68)      # longest first: a 32-row workload of 2-entry rows


def test_tile_coo_option_builds_on_the_host(spg):
    # the TILE-COO list is an addition: the composite format is unchanged,
    # and a host-only handle refuses the GPU call
    rp, col = graphgen.rmat(11, 8, seed=2)
    a = spg.Format(rp, col, kind="pagerank", host_only=True, max_warps=200, tile_width=512)
    b = spg.Format(rp, col, kind="pagerank", host_only=True, max_warps=200, tile_width=512, tile_coo=True)
    for k in ("n", "nnz", "ntile", "nworkloads", "padded_slots", "zero_rows"):
        assert a.info()[k] == b.info()[k]
    n = rp.shape[0] - 1
    x = np.zeros(n, np.float32)
    with pytest.raises(spg.SpgError):
        b.spmv_tile_coo(x, np.zeros(n, np.float32))


def test_automatic_rule_is_the_argmin_of_the_model(spg):
    # rule 4: each part's storage rule is the first (in the order 1, 0, 2, 3)
    # whose plan the Algorithm 3 model prices lowest -- checked against the
    # oracle's model cost of every rule's plan, part by part
    nlog = 21
    rng = np.random.default_rng(5)
    for trial in range(3):
        perf = rng.uniform(1e9, 5e9, 2 * nlog * nlog)
        if trial == 1:
            perf[: nlog * nlog] *= 0.05     # row-major slow: ELL-leaning plans
        path = _table_file(perf)
        try:
            rp, col = graphgen.rmat(11, 8, seed=1 + trial)
            f = spg.Format(rp, col, kind="pagerank", tile_width=256, max_warps=64, keep_plan=True,
                           host_only=True, table=path, layout_rule=4)
        finally:
            spg.load_table(None)
            os.unlink(path)
        n = rp.shape[0] - 1
        pi, inv = f.perm()
        M = oracle.build_M(rp, col)
        rows_p = pi[np.repeat(np.arange(n), np.diff(M[0]))]
        cols_p = pi[M[1]]
        ids = np.arange(n, dtype=np.int64)
        for p in range(f.nparts()):
            ti = f.tile_info(p)
            m = (cols_p >= ti["col_begin"]) & (cols_p < ti["col_end"])
            rl = np.bincount(rows_p[m], minlength=n).astype(np.int64)
            costs = {r: oracle.plan_cost(ids, rl, -1, 0, 64, r, (nlog, perf), 2e-7, 32)
                     for r in (1, 0, 2, 3)}
            best = min(costs.values())
            want = next(r for r in (1, 0, 2, 3) if costs[r] == best)
            assert ti["layout_rule"] == want, (trial, p, costs)


def test_slice_share_is_the_densest_columns_share_of_entries(spg):
    # the first x_stage_cols columns of a part (decreasing column length)
    # hold this share of its entries; option 1 stages the slice only where
    # it is >= 0.10 -- recomputed here from the out-degrees (the column
    # lengths of M)
    rp, col = graphgen.rmat(14, 8, seed=1)
    deg = np.sort(np.diff(rp))[::-1].astype(np.int64)
    for S, tw in ((1024, -1), (4096, -1), (512, 2048)):
        f = spg.Format(rp, col, kind="pagerank", host_only=True, x_stage_cols=S, tile_width=tw)
        for p in range(f.nparts()):
            ti = f.tile_info(p)
            seg = deg[ti["col_begin"]:ti["col_end"]]
            want = seg[:S].sum() / seg.sum() if seg.sum() > 0 else 0.0
            assert abs(ti["slice_share"] - want) <= 1e-12, (S, p)
    # a directed star: every entry of M lies in the centre's column
    n = 1000
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = n - 1
    col = np.arange(1, n, dtype=np.int32)
    f = spg.Format(rp, col, kind="pagerank", host_only=True, x_stage_cols=1, tile_width=-1)
    assert f.tile_info(0)["slice_share"] == 1.0
