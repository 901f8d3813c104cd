"""FP64 oracle of the tiled-composite SpMV method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg may import this package.  The product path
(``paper_1103_2405_gb300``) never imports it, and it imports nothing from the
product: the two share only the seeded inputs of ``graphgen``.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, FP64), each
function citing the passage of the paper it follows; this module only
marshals numpy arrays through ctypes and, for the format plan, composes the
C steps in the paper's order (Section 3.1 Solutions 2-3, Algorithms 1-3).

Parity unpinned: none.  Every function is pinned by a ``-m "not gpu"`` test
against dense brute force, closed forms, invariants or exhaustive search
(tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so with gcc (no threads, -O2, strict FP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-shared",
                               "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            sig = {
                "orc_build_M": ([i64, P, P, P, P, P], i64),
                "orc_spmv": ([i64, P, P, P, P, dbl, dbl, P], None),
                "orc_spmv_rows": ([i64, P, P, P, P, P, P], None),
                "orc_pagerank": ([i64, P, P, P, P, dbl, dbl, i32, P, P, P], i32),
                "orc_rwr": ([i64, P, P, P, P, i64, dbl, dbl, i32, P, P, P], i32),
                "orc_hits": ([i64, P, P, i32, i32, P, P], None),
                "orc_edge_softmax": ([i64, P, P, P], None),
                "orc_rwr_weighted": ([i64, P, P, P, i64, dbl, dbl, i32, P], i32),
                "orc_rwr_adjoint": ([i64, P, P, P, i64, dbl, P, P, dbl, i32, P, P], i32),
                "orc_degree_order": ([i64, P, P, P], None),
                "orc_alg1_tiles": ([i64, P, i64], i64),
                "orc_alg3_model": ([i64, P, i64, i64, i32, i32, P, i64], dbl),
                "orc_alg2_partition": ([i64, P, i64, i64, i32, i32, P, P, i64], i64),
                "orc_partition_tile": ([i64, P, P, i64, i64, i64, i32, i32, P, P, P, P, P, P,
                                        P, P, P, P, i64], i64),
                "orc_tune_heavy": ([i64, P, P, i64, i32, i32, P, dbl, P, i64], i64),
                "orc_split_cost_chunks": ([i64, P, i64], dbl),
                "orc_bitonic_partition": ([i64, P, i32, P], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ----------------------------------------------------------------- transform --

def build_M(a_rowptr, a_col):
    """M = W^T with FP32 values fl32(1/outdeg(u)) (Appendix F, Eq. 6).

    Returns (m_rowptr int64[n+1], m_col int32[nnz], m_val float32[nnz])."""
    a_rowptr = _c(a_rowptr, np.int64)
    a_col = _c(a_col, np.int32)
    n = a_rowptr.shape[0] - 1
    nnz = int(a_rowptr[-1])
    m_rowptr = np.empty(n + 1, np.int64)
    m_col = np.empty(max(nnz, 1), np.int32)
    m_val = np.empty(max(nnz, 1), np.float32)
    if _load().orc_build_M(n, _p(a_rowptr), _p(a_col), _p(m_rowptr), _p(m_col), _p(m_val)) < 0:
        raise MemoryError("orc_build_M")
    return m_rowptr, m_col[:nnz], m_val[:nnz]


def spmv(M, x, alpha=1.0, beta=0.0, y=None):
    """y = alpha M x + beta y in FP64 (inputs promoted from their stored type)."""
    rp, col, val = M
    rp, col, val = _c(rp, np.int64), _c(col, np.int32), _c(val, np.float32)
    n = rp.shape[0] - 1
    xd = _c(x, np.float64)
    yd = np.zeros(n, np.float64) if y is None else np.array(y, dtype=np.float64)
    _load().orc_spmv(n, _p(rp), _p(col), _p(val), _p(xd), float(alpha), float(beta), _p(yd))
    return yd


def spmv_rows(M, rows, x):
    """(M x)[rows] in FP64 -- sampled checks on matrices too big to multiply whole."""
    rp, col, val = M
    rows = _c(rows, np.int64)
    xd = _c(x, np.float64)
    out = np.empty(rows.shape[0], np.float64)
    _load().orc_spmv_rows(rows.shape[0], _p(rows), _p(_c(rp, np.int64)), _p(_c(col, np.int32)),
                          _p(_c(val, np.float32)), _p(xd), _p(out))
    return out


# ---------------------------------------------------------- power iterations --

def pagerank(a_rowptr, a_col, c=0.85, tol=1e-13, max_iter=10000, p_init=None, M=None):
    """PageRank by Eq. 6 with uniform dangling redistribution.

    Returns (p float64[n], iterations, last L1 change)."""
    a_rowptr = _c(a_rowptr, np.int64)
    n = a_rowptr.shape[0] - 1
    if M is None:
        M = build_M(a_rowptr, a_col)
    rp, col, val = M
    outdeg = np.diff(a_rowptr).astype(np.int64)
    p = np.empty(n, np.float64)
    l1 = ctypes.c_double(0)
    pi = None if p_init is None else _c(p_init, np.float64)
    it = _load().orc_pagerank(n, _p(_c(rp, np.int64)), _p(_c(col, np.int32)),
                              _p(_c(val, np.float32)), _p(outdeg), float(c), float(tol),
                              int(max_iter), _p(pi), _p(p), ctypes.byref(l1))
    return p, int(it), float(l1.value)


def rwr(a_rowptr, a_col, s, c=0.85, tol=1e-13, max_iter=10000, M=None, r_init=None):
    """RWR by Eq. 9 on M with dangling mass returned to s.  Returns (r, iters, l1)."""
    a_rowptr = _c(a_rowptr, np.int64)
    n = a_rowptr.shape[0] - 1
    if M is None:
        M = build_M(a_rowptr, a_col)
    rp, col, val = M
    outdeg = np.diff(a_rowptr).astype(np.int64)
    r = np.empty(n, np.float64)
    l1 = ctypes.c_double(0)
    ri = None if r_init is None else _c(r_init, np.float64)
    it = _load().orc_rwr(n, _p(_c(rp, np.int64)), _p(_c(col, np.int32)), _p(_c(val, np.float32)),
                         _p(outdeg), int(s), float(c), float(tol), int(max_iter), _p(ri), _p(r),
                         ctypes.byref(l1))
    return r, int(it), float(l1.value)


def hits(a_rowptr, a_col, iters=50, norm=2):
    """HITS by Eq. 7 (Jacobi), each half normalised (norm=1: sum, norm=2: L2)."""
    a_rowptr = _c(a_rowptr, np.int64)
    n = a_rowptr.shape[0] - 1
    a = np.empty(n, np.float64)
    h = np.empty(n, np.float64)
    _load().orc_hits(n, _p(a_rowptr), _p(_c(a_col, np.int32)), int(iters), int(norm), _p(a), _p(h))
    return a, h


# ----------------------------------------------------- differentiable RWR --

def edge_softmax(a_rowptr, theta):
    a_rowptr = _c(a_rowptr, np.int64)
    n = a_rowptr.shape[0] - 1
    P = np.zeros(int(a_rowptr[-1]), np.float64)
    _load().orc_edge_softmax(n, _p(a_rowptr), _p(_c(theta, np.float32)), _p(P))
    return P


def rwr_weighted(a_rowptr, a_col, P, s, c=0.85, tol=1e-14, max_iter=100000):
    a_rowptr = _c(a_rowptr, np.int64)
    n = a_rowptr.shape[0] - 1
    r = np.empty(n, np.float64)
    it = _load().orc_rwr_weighted(n, _p(a_rowptr), _p(_c(a_col, np.int32)), _p(_c(P, np.float64)),
                                  int(s), float(c), float(tol), int(max_iter), _p(r))
    return r, int(it)


def rwr_adjoint(a_rowptr, a_col, P, s, c, r, g, tol=1e-14, max_iter=100000):
    a_rowptr = _c(a_rowptr, np.int64)
    n = a_rowptr.shape[0] - 1
    lam = np.empty(n, np.float64)
    dth = np.zeros(int(a_rowptr[-1]), np.float64)
    it = _load().orc_rwr_adjoint(n, _p(a_rowptr), _p(_c(a_col, np.int32)), _p(_c(P, np.float64)),
                                 int(s), float(c), _p(_c(r, np.float64)), _p(_c(g, np.float64)),
                                 float(tol), int(max_iter), _p(lam), _p(dth))
    return lam, dth, int(it)


def rwr_loss(a_rowptr, a_col, theta, s, targets, c=0.85):
    """L(theta) = -sum_t log r_t with r the weighted-RWR fixed point."""
    P = edge_softmax(a_rowptr, theta)
    r, _ = rwr_weighted(a_rowptr, a_col, P, s, c)
    return float(-np.sum(np.log(r[np.asarray(targets)]))), r, P


def rwr_loss_grad(a_rowptr, a_col, theta, s, targets, c=0.85):
    """(loss, dL/dtheta float64[nnz], r, lambda) by the adjoint fixed point."""
    loss, r, P = rwr_loss(a_rowptr, a_col, theta, s, targets, c)
    n = r.shape[0]
    g = np.zeros(n, np.float64)
    np.add.at(g, np.asarray(targets), -1.0 / r[np.asarray(targets)])
    lam, dth, _ = rwr_adjoint(a_rowptr, a_col, P, s, c, r, g)
    return loss, dth, r, lam


# --------------------------------------------------------------- format plan --

def degree_order(length):
    """(pi, inv): positions by decreasing length, ties by ascending id."""
    length = _c(length, np.int64)
    n = length.shape[0]
    pi = np.empty(n, np.int32)
    inv = np.empty(n, np.int32)
    _load().orc_degree_order(n, _p(length), _p(pi), _p(inv))
    return pi, inv


def alg1_tiles(sorted_col_len, tile_width):
    s = _c(sorted_col_len, np.int64)
    return int(_load().orc_alg1_tiles(s.shape[0], _p(s), int(tile_width)))


def alg3_model(row_len, WL, max_warps, rule, table, max_rows=0):
    nlog, perf = table
    rl = _c(row_len, np.int64)
    return float(_load().orc_alg3_model(rl.shape[0], _p(rl), int(WL), int(max_warps), int(rule),
                                        int(nlog), _p(_c(perf, np.float64)), int(max_rows)))


def alg2_partition(row_len, nnz, max_warps, rule, table, max_rows=0):
    nlog, perf = table
    rl = _c(row_len, np.int64)
    t = ctypes.c_double(0)
    wl = _load().orc_alg2_partition(rl.shape[0], _p(rl), int(nnz), int(max_warps), int(rule),
                                    int(nlog), _p(_c(perf, np.float64)), ctypes.byref(t),
                                    int(max_rows))
    return int(wl), float(t.value)


def partition_tile(row_id, row_len, heavy, wl, max_warps, rule, table, max_rows=0):
    """Composite partition of one tile (Solution 3 + Algorithms 2-3).

    Returns dict(WL, rank_row, rank_chunk, rank_len, wl_first, wl_h, wl_w, wl_major)."""
    nlog, perf = table
    row_id = _c(row_id, np.int64)
    row_len = _c(row_len, np.int64)
    nnz = int(row_len[row_len > 0].sum())
    cap = int(row_id.shape[0] + nnz // 32 + 1)
    rr, rc, rl = (np.empty(cap, np.int64) for _ in range(3))
    f, h, w, mj = (np.empty(cap, np.int64) for _ in range(4))
    nv = ctypes.c_int64(0)
    nw = ctypes.c_int64(0)
    WL = _load().orc_partition_tile(row_id.shape[0], _p(row_id), _p(row_len), int(heavy), int(wl),
                                    int(max_warps), int(rule), int(nlog),
                                    _p(_c(perf, np.float64)), ctypes.byref(nv), _p(rr), _p(rc),
                                    _p(rl), ctypes.byref(nw), _p(f), _p(h), _p(w), _p(mj),
                                    int(max_rows))
    k, j = nv.value, nw.value
    return dict(WL=int(WL), rank_row=rr[:k].copy(), rank_chunk=rc[:k].copy(),
                rank_len=rl[:k].copy(), wl_first=f[:j].copy(), wl_h=h[:j].copy(),
                wl_w=w[:j].copy(), wl_major=mj[:j].copy())


def tune_heavy(row_id, row_len, max_warps, rule, table, split_cost, max_rows=0):
    nlog, perf = table
    row_id = _c(row_id, np.int64)
    row_len = _c(row_len, np.int64)
    wl = ctypes.c_int64(0)
    H = _load().orc_tune_heavy(row_id.shape[0], _p(row_id), _p(row_len), int(max_warps),
                               int(rule), int(nlog), _p(_c(perf, np.float64)), float(split_cost),
                               ctypes.byref(wl), int(max_rows))
    return int(H), int(wl.value)


def split_cost_chunks(row_len, H):
    """Chunks of the rows longer than H (the count the split cost multiplies)."""
    rl = _c(row_len, np.int64)
    return float(_load().orc_split_cost_chunks(rl.shape[0], _p(rl), int(H)))


AUTO_RULE = 4


def plan_cost(row_id, row_len, heavy, wl, max_warps, rule, table, split_cost, max_rows=0):
    """Modelled cost of one tile's plan under storage rule `rule`: split
    threshold (tuned when heavy < 0), Algorithm 2 workload size (wl = 0) and
    the Algorithm 3 time of that plan, plus split_cost per chunk of a split
    row."""
    rl = _c(row_len, np.int64)
    if int(rl[rl > 0].sum()) == 0:
        return 0.0
    H = tune_heavy(row_id, rl, max_warps, rule, table, split_cost, max_rows)[0] if heavy < 0 else heavy
    part = partition_tile(row_id, rl, H, wl, max_warps, rule, table, max_rows)
    t = alg3_model(part["rank_len"], part["WL"], max_warps, rule, table, max_rows)
    return t + split_cost * (split_cost_chunks(rl, H) if H > 0 else 0.0)


def choose_rule(row_id, row_len, heavy, wl, max_warps, table, split_cost, max_rows=0):
    """Section 5 reading: CSR-vector (rule 2) and ELL (rule 3) are special
    cases of the composite format, as are the paper's w >= h rule (0) and
    the fewer-padded-slots rule (1); the automatic storage rule takes, per
    tile, the one whose plan Algorithm 3 prices lowest (first of 1, 0, 2, 3
    on a tie)."""
    best, best_r = np.inf, 1
    for r in (1, 0, 2, 3):
        c = plan_cost(row_id, row_len, heavy, wl, max_warps, r, table, split_cost, max_rows)
        if c < best:
            best, best_r = c, r
    return best_r


def plan_format(a_rowptr, a_col, tile_width, max_warps, table, heavy=-1, wl=0, rule=1,
                split_cost=0.0, M=None, max_rows=0):
    """The tiled composite layout of M = W^T, step by step in the paper's order.

    1. column lengths of M (= out-degrees), symmetric order by decreasing
       length (Solution 2);
    2. Algorithm 1 tile count with ``tile_width``; tiles are
       [t*tw, (t+1)*tw) and the sparse part is the rest (Solutions 2-3);
    3. per tile, in-tile row lengths; split threshold (heavy=-1: tuned,
       0: off, >0: fixed) and Algorithm 2 WL (wl=0) and packing.
    Returns dict(pi, inv, ntile, tiles=[(c0, c1, H, part_dict)], zero_rows)."""
    a_rowptr = _c(a_rowptr, np.int64)
    n = a_rowptr.shape[0] - 1
    outdeg = np.diff(a_rowptr).astype(np.int64)
    pi, inv = degree_order(outdeg)
    sorted_len = outdeg[inv]
    ntile = alg1_tiles(sorted_len, tile_width) if tile_width > 0 else 0
    if M is None:
        M = build_M(a_rowptr, a_col)
    rp, col, _ = M
    rows_p = pi[np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))].astype(np.int64)
    cols_p = pi[col].astype(np.int64)
    bounds = [t * tile_width for t in range(ntile)] + [ntile * tile_width if ntile else 0, n]
    if ntile == 0:
        bounds = [0, n]
    tiles = []
    touched = np.zeros(n, dtype=bool)
    for t in range(len(bounds) - 1):
        c0, c1 = bounds[t], bounds[t + 1]
        m = (cols_p >= c0) & (cols_p < c1)
        rl = np.bincount(rows_p[m], minlength=n).astype(np.int64)
        touched |= rl > 0
        ids = np.arange(n, dtype=np.int64)
        r = choose_rule(ids, rl, heavy, wl, max_warps, table, split_cost, max_rows) \
            if rule == AUTO_RULE else rule
        if heavy < 0:
            H, _ = tune_heavy(ids, rl, max_warps, r, table, split_cost, max_rows)
        else:
            H = heavy
        part = partition_tile(ids, rl, H, wl, max_warps, r, table, max_rows)
        part["rule"] = r
        tiles.append((c0, c1, H, part))
    zero_rows = np.flatnonzero(~touched).astype(np.int64)
    return dict(pi=pi, inv=inv, ntile=ntile, tiles=tiles, zero_rows=zero_rows)


def bitonic_partition(row_len, P):
    """Section 3.2 bitonic assignment of rows to P parts."""
    rl = _c(row_len, np.int64)
    part = np.empty(rl.shape[0], np.int32)
    _load().orc_bitonic_partition(rl.shape[0], _p(rl), int(P), _p(part))
    return part
