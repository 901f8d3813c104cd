"""Seeded synthetic inputs: R-MAT and Chung-Lu graphs, random vectors, seed picks.

Input generation only.  The graphs come back as the adjacency structure of A
(CSR by source node: ``rowptr`` int64[n+1], ``col`` int32[nnz], columns sorted,
duplicates and self-loops removed) -- no matrix values, no reordering.  Both the
CUDA path and the FP64 oracle consume these arrays; neither shares any other
code with the other.

The C core (``graphgen.c``) is compiled on first use with the system C compiler
(``build()``); every draw comes from a counter-based SplitMix64 stream, so the
results do not depend on the thread count or the machine.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "_graphgen.so")
_lock = threading.Lock()
_lib = None

# R-MAT quadrant probabilities of the workloads (a, b, c; d = 1 - a - b - c).
RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile graphgen.c into _graphgen.so (gcc, plain C11 + pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, u64, i32, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
            lib.gg_rmat_edges.argtypes = [i32, i64, dbl, dbl, dbl, u64, i32, P, P]
            lib.gg_rmat_edges.restype = i32
            lib.gg_chung_lu_weights.argtypes = [i64, dbl, dbl, dbl, P]
            lib.gg_chung_lu_weights.restype = dbl
            lib.gg_alias_table.argtypes = [i64, P, P, P]
            lib.gg_alias_table.restype = i32
            lib.gg_chung_lu_edges.argtypes = [i64, i64, P, P, u64, i32, P, P]
            lib.gg_chung_lu_edges.restype = i32
            lib.gg_random_permutation.argtypes = [i64, u64, P]
            lib.gg_random_permutation.restype = i32
            lib.gg_edges_to_csr.argtypes = [i64, i64, P, P, P, i32, P, P]
            lib.gg_edges_to_csr.restype = i64
            lib.gg_uniform_f32.argtypes = [u64, i64, P]
            lib.gg_uniform_f32.restype = None
            lib.gg_normal_f32.argtypes = [u64, i64, P]
            lib.gg_normal_f32.restype = None
            lib.gg_rand64_export.argtypes = [u64, u64, u64]
            lib.gg_rand64_export.restype = u64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _threads(nthreads):
    return int(nthreads or min(32, os.cpu_count() or 1))


def rand64(seed: int, stream: int, ctr: int) -> int:
    """One raw 64-bit counter-based draw (exposed for tests)."""
    return int(_load().gg_rand64_export(seed, stream, ctr))


def random_permutation(n: int, seed: int) -> np.ndarray:
    perm = np.empty(n, dtype=np.uint32)
    if _load().gg_random_permutation(n, seed, _ptr(perm)) != 0:
        raise ValueError("bad permutation size")
    return perm


def edges_to_csr(n: int, src: np.ndarray, dst: np.ndarray, relabel=None, nthreads=None):
    """Edge list -> (rowptr int64[n+1], col int32[nnz]); dedup, no self-loops."""
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    m = src.shape[0]
    rowptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(max(m, 1), dtype=np.uint32)
    if relabel is not None:
        relabel = np.ascontiguousarray(relabel, dtype=np.uint32)
    nnz = _load().gg_edges_to_csr(n, m, _ptr(src), _ptr(dst), _ptr(relabel),
                                  _threads(nthreads), _ptr(rowptr), _ptr(col))
    if nnz < 0:
        raise ValueError("edges_to_csr failed (%d)" % nnz)
    col = col[:nnz].view(np.int32).copy() if nnz < col.shape[0] else col.view(np.int32)
    return rowptr, col


def rmat_edges(scale: int, m: int, seed: int = 1, abc=RMAT_ABC, nthreads=None):
    """Raw R-MAT edge list (duplicates and self-loops still present)."""
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    a, b, c = abc
    if _load().gg_rmat_edges(scale, m, a, b, c, seed, _threads(nthreads), _ptr(src), _ptr(dst)) != 0:
        raise ValueError("bad R-MAT parameters")
    return src, dst


def rmat(scale: int, edge_factor: int, seed: int = 1, abc=RMAT_ABC, relabel: bool = True,
         nthreads=None):
    """R-MAT graph with 2^scale nodes and edge_factor*2^scale generated edges.

    Duplicates and self-loops are removed, so the returned nnz is below the
    generated count.  With ``relabel`` the node ids go through a seeded random
    permutation (seed + 0x5eed), so that low ids are not the hubs.
    """
    n = 1 << scale
    m = edge_factor * n
    src, dst = rmat_edges(scale, m, seed, abc, nthreads)
    perm = random_permutation(n, seed + 0x5EED) if relabel else None
    return edges_to_csr(n, src, dst, perm, nthreads)


def chung_lu_weights(n: int, m: float, gamma: float, dmax: float) -> np.ndarray:
    w = np.empty(n, dtype=np.float64)
    if _load().gg_chung_lu_weights(n, float(m), float(gamma), float(dmax), _ptr(w)) < 0:
        raise ValueError("bad Chung-Lu parameters")
    return w


def chung_lu(n: int, m: int, gamma: float, dmax: float, seed: int = 1, relabel: bool = True,
             nthreads=None):
    """Chung-Lu graph: expected degrees w_i = min(dmax, C (i+1)^(-1/(gamma-1))),
    sum w = m; m edges with source and destination drawn independently
    proportional to w; dedup and self-loop removal; seeded relabel."""
    w = chung_lu_weights(n, m, gamma, dmax)
    prob = np.empty(n, dtype=np.float64)
    alias = np.empty(n, dtype=np.uint32)
    lib = _load()
    if lib.gg_alias_table(n, _ptr(w), _ptr(prob), _ptr(alias)) != 0:
        raise ValueError("alias table failed")
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    if lib.gg_chung_lu_edges(n, m, _ptr(prob), _ptr(alias), seed, _threads(nthreads),
                             _ptr(src), _ptr(dst)) != 0:
        raise ValueError("Chung-Lu edge draw failed")
    del w, prob, alias
    perm = random_permutation(n, seed + 0x5EED) if relabel else None
    return edges_to_csr(n, src, dst, perm, nthreads)


def uniform(n: int, seed: int) -> np.ndarray:
    """x ~ U[0,1) float32 (24-bit mantissa draws)."""
    out = np.empty(n, dtype=np.float32)
    _load().gg_uniform_f32(seed, n, _ptr(out))
    return out


def normal(n: int, seed: int) -> np.ndarray:
    """N(0,1) float32 (Box-Muller)."""
    out = np.empty(n, dtype=np.float32)
    _load().gg_normal_f32(seed, n, _ptr(out))
    return out


def outdeg(rowptr: np.ndarray) -> np.ndarray:
    return np.diff(rowptr)


def pick_source(rowptr: np.ndarray, seed: int = 3) -> int:
    """RWR source node: a seeded pick among the top 1% of nodes by out-degree
    (ties broken by ascending id), so it has outgoing mass to spread."""
    d = outdeg(rowptr)
    n = d.shape[0]
    top = max(1, n // 100)
    order = np.lexsort((np.arange(n), -d))[:top]
    return int(order[rand64(seed, 8, 0) % top])


def pick_seeds(rowptr: np.ndarray, k: int, seed: int = 4) -> np.ndarray:
    """k distinct nodes with out-degree > 0, seeded (restart nodes of batched RWR)."""
    d = outdeg(rowptr)
    cand = np.flatnonzero(d > 0)
    if cand.shape[0] < k:
        raise ValueError("not enough nodes with out-degree > 0")
    keys = _keys_fast(cand.shape[0], seed, 9)
    return cand[np.argsort(keys, kind="stable")[:k]].astype(np.int32)


def _keys_fast(n: int, seed: int, stream: int) -> np.ndarray:
    # vectorised uniform draws through the same counter stream as uniform()
    out = np.empty(n, dtype=np.float32)
    _load().gg_uniform_f32(seed * 1000003 + stream, n, _ptr(out))
    return out


def reachable_from(rowptr: np.ndarray, col: np.ndarray, s: int) -> np.ndarray:
    """Boolean mask of nodes reachable from s along directed edges (BFS)."""
    n = rowptr.shape[0] - 1
    seen = np.zeros(n, dtype=bool)
    seen[s] = True
    frontier = np.array([s], dtype=np.int64)
    while frontier.size:
        starts, ends = rowptr[frontier], rowptr[frontier + 1]
        lens = ends - starts
        if lens.sum() == 0:
            break
        idx = np.repeat(starts - np.cumsum(np.concatenate(([0], lens[:-1]))), lens) + \
            np.arange(lens.sum())
        nb = np.unique(col[idx])
        nb = nb[~seen[nb]]
        seen[nb] = True
        frontier = nb.astype(np.int64)
    return seen


def pick_targets(rowptr: np.ndarray, col: np.ndarray, s: int, k: int, seed: int = 5) -> np.ndarray:
    """k distinct target nodes reachable from s (so their RWR score is > 0)."""
    cand = np.flatnonzero(reachable_from(rowptr, col, s))
    if cand.shape[0] < k:
        raise ValueError("not enough reachable targets")
    keys = _keys_fast(cand.shape[0], seed, 10)
    return np.sort(cand[np.argsort(keys, kind="stable")[:k]]).astype(np.int32)


def pick_edges(nnz: int, k: int, seed: int = 6) -> np.ndarray:
    """k distinct edge ids (finite-difference probes)."""
    keys = _keys_fast(nnz, seed, 11)
    return np.sort(np.argsort(keys, kind="stable")[:k]).astype(np.int64)


def chung_lu_batch_sizes(count: int, lo_log2: int = 10, hi_log2: int = 17, seed: int = 1000):
    """Node counts log-uniform in [2^lo, 2^hi] for a batch of small graphs."""
    u = _keys_fast(count, seed, 12).astype(np.float64)
    return np.floor(2.0 ** (lo_log2 + u * (hi_log2 - lo_log2))).astype(np.int64)


# ------------------------------------------- non-power-law sanity matrices --
#
# Matrices with the shapes of the paper's unstructured comparison set (its
# dense 2K x 2K case and banded / finite-element-like sparsity); values are
# U[0,1) draws of the counter generator (seeded), so every entry is a
# positive FP32 and the tolerance bound |M| |x| is simply M x.

def _csr_from_rows(n: int, row_len: np.ndarray, cols: np.ndarray, seed: int):
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(row_len, out=rowptr[1:])
    val = uniform(int(rowptr[-1]), seed)
    return rowptr, np.ascontiguousarray(cols, dtype=np.int32), val


def dense_matrix(n: int, seed: int = 21):
    """Every entry of an n x n matrix stored (the paper's dense 2K x 2K case)."""
    cols = np.tile(np.arange(n, dtype=np.int32), n)
    return _csr_from_rows(n, np.full(n, n, dtype=np.int64), cols, seed)


def banded(n: int, half_width: int, seed: int = 22):
    """Row i holds columns max(0, i-b) .. min(n-1, i+b)."""
    i = np.arange(n, dtype=np.int64)
    lo = np.maximum(0, i - half_width)
    hi = np.minimum(n - 1, i + half_width)
    row_len = hi - lo + 1
    start = np.repeat(lo, row_len)
    offs = np.arange(int(row_len.sum()), dtype=np.int64) - np.repeat(np.cumsum(row_len) - row_len, row_len)
    return _csr_from_rows(n, row_len, (start + offs).astype(np.int32), seed)


def stencil_3d(nx: int, ny: int, nz: int, seed: int = 23):
    """27-point stencil of an nx x ny x nz grid (a trilinear finite-element
    pattern): node (x, y, z) couples to every node within one step along
    each axis; columns ascending."""
    n = nx * ny * nz
    g = np.arange(n, dtype=np.int64)
    x, y, z = g % nx, (g // nx) % ny, g // (nx * ny)
    cols = []
    ok_all = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                xx, yy, zz = x + dx, y + dy, z + dz
                ok = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
                cols.append(np.where(ok, xx + nx * (yy + ny * zz), -1))
                ok_all.append(ok)
    C = np.stack(cols, axis=1)            # n x 27, ascending within a row
    K = np.stack(ok_all, axis=1)
    row_len = K.sum(axis=1).astype(np.int64)
    return _csr_from_rows(n, row_len, C[K], seed)
