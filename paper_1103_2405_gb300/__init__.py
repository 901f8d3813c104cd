"""Tiled composite SpMV for power-law graphs on GB300 -- Python binding.

Thin ctypes layer over the C ABI of ``include/spg.h`` (``lib/libspg.so``):
argument marshalling only; every step runs in the library's C++ builder and
sm_103a kernels.  Vectors may be torch tensors (CUDA or CPU) or numpy arrays;
device tensors are passed by pointer, host arrays are staged by the library.

The library must have been built (``__graft_entry__.build()`` or
``python paper_1103_2405_gb300/build.py``); importing the binding without it
raises immediately -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libspg.so")
TABLE_PATH = os.path.join(_HERE, "perf_table_gb300.txt")

KIND = {"matrix": 0, "pagerank": 1, "hits": 2, "weighted": 3}
CSR_SCALAR, CSR_VECTOR = 0, 1
NOT_CONVERGED = 1


class SpgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"spg status {status}: {msg}")
        self.status = status


class _Csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("on_device", ctypes.c_int)]


class _Opts(ctypes.Structure):
    _fields_ = [("tile_width", ctypes.c_int64), ("wl", ctypes.c_int64), ("heavy_row", ctypes.c_int64),
                ("layout_rule", ctypes.c_int), ("max_warps", ctypes.c_int), ("vec_width", ctypes.c_int),
                ("build_transpose", ctypes.c_int), ("keep_plan", ctypes.c_int),
                ("keep_csr", ctypes.c_int), ("device", ctypes.c_int), ("split_cost", ctypes.c_double),
                ("tune_table_path", ctypes.c_char_p), ("x_stage_cols", ctypes.c_int64),
                ("slab_prefetch", ctypes.c_int64), ("loop_mode", ctypes.c_int),
                ("max_rows", ctypes.c_int64), ("kernel", ctypes.c_int), ("pattern_only", ctypes.c_int),
                ("row_part", ctypes.c_void_p), ("part_id", ctypes.c_int32), ("nparts", ctypes.c_int32),
                ("unit_slots", ctypes.c_int64), ("separate_check", ctypes.c_int32),
                ("claim_order", ctypes.c_int32), ("tile_coo", ctypes.c_int32)]


class IterInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("last_l1", ctypes.c_double),
                ("dangling", ctypes.c_double), ("ms", ctypes.c_float)]

    def as_dict(self):
        return dict(iters=self.iters, last_l1=self.last_l1, dangling=self.dangling, ms=self.ms)


class _Info(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in
                ("n", "nnz", "ntile", "tile_width", "nworkloads", "padded_slots", "split_rows",
                 "split_chunks", "zero_rows", "device_bytes", "max_warps")] + \
               [("predicted_ms", ctypes.c_double), ("dangling_start", ctypes.c_int64)]


class _TileInfo(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in
                ("col_begin", "col_end", "heavy", "wl", "nvirt", "nwl", "nnz")] + \
               [("predicted_ms", ctypes.c_double), ("layout_rule", ctypes.c_int64),
                ("slice_share", ctypes.c_double), ("nunits", ctypes.c_int64)]


# Every symbol include/spg.h declares.
EXPORTS = ["spg_build_format", "spg_destroy", "spg_format_info", "spg_tile_info", "spg_format_perm",
           "spg_format_export_plan", "spg_format_export_entries", "spg_format_zero_rows",
           "spg_spmv", "spg_spmv_permuted", "spg_spmm", "spg_pagerank", "spg_rwr", "spg_hits",
           "spg_set_edge_logits", "spg_rwr_weighted", "spg_rwr_adjoint", "spg_build_batch",
           "spg_batch_offsets", "spg_batch_pagerank",
           "spg_baseline_spmv", "spg_baseline_pagerank", "spg_time_parts", "spg_load_table", "spg_launch_count",
           "spg_status_string", "spg_last_error", "spg_version", "spg_spmv_permuted_noalloc",
           "spg_partition_rows", "spg_pagerank_ranks", "spg_spmv_tile_coo", "spg_pagerank_rank_step",
           "spg_pack_slice", "spg_unpack_slice"]

_lib = None


def lib():
    """The loaded libspg.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32, f32, f64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float,
                                 ctypes.c_double)
        sig = {
            "spg_build_format": [ctypes.POINTER(_Csr), i32, ctypes.POINTER(_Opts), P, ctypes.POINTER(P)],
            "spg_destroy": [P],
            "spg_format_info": [P, ctypes.POINTER(_Info)],
            "spg_tile_info": [P, i64, ctypes.POINTER(_TileInfo)],
            "spg_format_perm": [P, P, P],
            "spg_format_export_plan": [P, i64, P, P, P, P, P, P, P],
            "spg_format_export_entries": [P, P, P, P],
            "spg_format_zero_rows": [P, P],
            "spg_spmv": [P, P, P, f32, f32, P],
            "spg_spmv_permuted": [P, P, P, P],
            "spg_spmv_tile_coo": [P, P, P, P],
            "spg_spmm": [P, P, i64, P, i64, i32, f32, f32, P],
            "spg_pagerank": [P, f32, f64, i32, P, P, ctypes.POINTER(IterInfo), P],
            "spg_rwr": [P, f32, P, i32, f64, i32, P, ctypes.POINTER(IterInfo), P],
            "spg_hits": [P, i32, f64, i32, P, P, ctypes.POINTER(IterInfo), P],
            "spg_set_edge_logits": [P, P, P],
            "spg_rwr_weighted": [P, f32, i32, f64, i32, P, ctypes.POINTER(IterInfo), P],
            "spg_rwr_adjoint": [P, f32, i32, P, P, f64, i32, P, P, ctypes.POINTER(IterInfo), P],
            "spg_build_batch": [P, i32, ctypes.POINTER(_Opts), P, ctypes.POINTER(P)],
            "spg_batch_offsets": [P, P],
            "spg_batch_pagerank": [P, f32, f64, i32, P, P, P],
            "spg_baseline_spmv": [P, i32, P, P, f32, f32, P],
            "spg_baseline_pagerank": [P, i32, f32, f64, i32, P, ctypes.POINTER(IterInfo), P],
            "spg_time_parts": [P, i32, i32, P, P],
            "spg_spmv_permuted_noalloc": [P, P, P, P],
            "spg_load_table": [ctypes.c_char_p],
            "spg_partition_rows": [i64, P, i32, P],
            "spg_pagerank_ranks": [P, i32, f32, f64, i32, P, P, ctypes.POINTER(IterInfo), P],
            "spg_pagerank_rank_step": [P, f32, f64, P, P, P, P],
            "spg_pack_slice": [i64, P, P, P, P],
            "spg_unpack_slice": [i64, P, P, P, P],
        }
        for name, args in sig.items():
            getattr(L, name).argtypes = args
            getattr(L, name).restype = ctypes.c_int
        L.spg_launch_count.restype = ctypes.c_int64
        L.spg_launch_count.argtypes = []
        for name in ("spg_status_string", "spg_last_error", "spg_version"):
            getattr(L, name).restype = ctypes.c_char_p
        L.spg_status_string.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _check(status, allow_not_converged=False):
    if status == 0 or (allow_not_converged and status == NOT_CONVERGED):
        return status
    L = lib()
    raise SpgError(status, f"{L.spg_status_string(status).decode()}: {L.spg_last_error().decode()}")


def launch_count() -> int:
    return int(lib().spg_launch_count())


def version() -> str:
    return lib().spg_version().decode()


def load_table(path=None):
    _check(lib().spg_load_table(None if path is None else str(path).encode()))


# --------------------------------------------------------------- marshalling --

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(pointer, keepalive) of a torch tensor or numpy array (contiguous)."""
    if a is None:
        return None, None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), a
    a = np.ascontiguousarray(a)
    return ctypes.c_void_p(a.ctypes.data), a


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _empty_like_vec(ref, n, k=1):
    if _is_torch(ref):
        import torch
        shape = (n,) if k == 1 else (n, k)
        return torch.empty(shape, dtype=torch.float32, device=ref.device)
    return np.empty(n if k == 1 else (n, k), dtype=np.float32)


class Format:
    """A built tiled composite format (one handle of the C ABI).

    rowptr (int64[n+1]), col (int32[nnz]) describe the CSR given to
    spg_build_format; ``val`` is the matrix values (kind 'matrix') or edge
    logits (kind 'weighted').  Build options map 1:1 to spg_build_opts."""

    def __init__(self, rowptr, col, val=None, kind="pagerank", tile_width=0, wl=0, heavy_row=-1,
                 layout_rule=1, max_warps=0, vec_width=1, build_transpose=False, keep_plan=False,
                 keep_csr=False, host_only=False, split_cost=0.0, table=None, x_stage_cols=0,
                 slab_prefetch=0, loop_mode=0, max_rows=0, kernel=0, pattern_only=False,
                 row_part=None, part_id=0, nparts=None, unit_slots=0, separate_check=False,
                 claim_order=0, tile_coo=False, stream=None):
        L = lib()
        self._h = ctypes.c_void_p(None)
        on_dev = _is_torch(rowptr) and rowptr.is_cuda
        if not on_dev:
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
            if val is not None:
                val = np.ascontiguousarray(val, dtype=np.float32)
        n = int(rowptr.shape[0]) - 1
        nnz = int(col.shape[0])
        prp, k1 = _ptr(rowptr)
        pcol, k2 = _ptr(col)
        pval, k3 = _ptr(val)
        csr = _Csr(n, n, nnz, prp, pcol, pval, 1 if on_dev else 0)
        tpath = table if table is not None else (TABLE_PATH if os.path.exists(TABLE_PATH) else None)
        opts = _Opts(int(tile_width), int(wl), int(heavy_row), int(layout_rule), int(max_warps),
                     int(vec_width), int(bool(build_transpose)), int(bool(keep_plan)),
                     int(bool(keep_csr)), -1 if host_only else 0, float(split_cost),
                     None if tpath is None else str(tpath).encode(), int(x_stage_cols),
                     int(slab_prefetch), int(loop_mode), int(max_rows), int(kernel),
                     int(bool(pattern_only)))
        opts.unit_slots = int(unit_slots)
        opts.separate_check = int(bool(separate_check))
        opts.claim_order = int(claim_order)
        opts.tile_coo = int(bool(tile_coo))
        if row_part is not None:
            row_part = np.ascontiguousarray(row_part, dtype=np.int32)
            opts.row_part = row_part.ctypes.data
            opts.part_id = int(part_id)
            opts.nparts = int(nparts) if nparts is not None else (int(row_part.max()) + 1 if row_part.size else 1)
            self.part_id, self.nparts = int(part_id), int(opts.nparts)
        _check(L.spg_build_format(ctypes.byref(csr), KIND[kind], ctypes.byref(opts),
                                  _stream(stream), ctypes.byref(self._h)))
        self.kind = kind
        self.n_graph = n
        self.nnz_in = nnz
        info = self.info()
        self.n = info["n"]
        self.nnz = info["nnz"]

    def close(self):
        if self._h is not None and self._h.value:
            lib().spg_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- inspection --
    def info(self):
        i = _Info()
        _check(lib().spg_format_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in _Info._fields_}

    def tile_info(self, part):
        t = _TileInfo()
        _check(lib().spg_tile_info(self._h, int(part), ctypes.byref(t)))
        return {k: getattr(t, k) for k, _ in _TileInfo._fields_}

    def nparts(self):
        return self.info()["ntile"] + 1

    def perm(self):
        pi = np.empty(self.n, np.int32)
        inv = np.empty(self.n, np.int32)
        _check(lib().spg_format_perm(self._h, _ptr(pi)[0], _ptr(inv)[0]))
        return pi, inv

    def export_plan(self, part):
        t = self.tile_info(part)
        rr, rc, rl = (np.empty(t["nvirt"], np.int64) for _ in range(3))
        f, h, w, m = (np.empty(t["nwl"], np.int64) for _ in range(4))
        _check(lib().spg_format_export_plan(self._h, int(part), *(_ptr(a)[0] for a in
                                                                    (rr, rc, rl, f, h, w, m))))
        return dict(WL=t["wl"], heavy=t["heavy"], rule=t["layout_rule"], rank_row=rr, rank_chunk=rc, rank_len=rl,
                    wl_first=f, wl_h=h, wl_w=w, wl_major=m)

    def export_entries(self):
        nnz = self.nnz
        r = np.empty(nnz, np.int64)
        c = np.empty(nnz, np.int32)
        v = np.empty(nnz, np.float32)
        _check(lib().spg_format_export_entries(self._h, _ptr(r)[0], _ptr(c)[0], _ptr(v)[0]))
        return r, c, v

    def zero_rows(self):
        z = np.empty(self.info()["zero_rows"], np.int64)
        _check(lib().spg_format_zero_rows(self._h, _ptr(z)[0]))
        return z

    # ---------------------------------------------------------------- compute --
    def spmv(self, x, y=None, alpha=1.0, beta=0.0, stream=None):
        if y is None:
            y = _empty_like_vec(x, self.n)
        px, kx = _ptr(x)
        py, ky = _ptr(y)
        _check(lib().spg_spmv(self._h, px, py, float(alpha), float(beta), _stream(stream)))
        return y

    def spmv_permuted(self, xp, yp, stream=None):
        _check(lib().spg_spmv_permuted(self._h, _ptr(xp)[0], _ptr(yp)[0], _stream(stream)))
        return yp

    def spmv_tile_coo(self, xp, yp, stream=None):
        """TILE-COO SpMV on permuted device vectors (handle built with tile_coo)."""
        _check(lib().spg_spmv_tile_coo(self._h, _ptr(xp)[0], _ptr(yp)[0], _stream(stream)))
        return yp

    def spmm(self, X, Y=None, alpha=1.0, beta=0.0, stream=None):
        k = int(X.shape[1])
        if Y is None:
            Y = _empty_like_vec(X, self.n, k)
        _check(lib().spg_spmm(self._h, _ptr(X)[0], int(X.stride(0) if _is_torch(X) else k),
                              _ptr(Y)[0], int(Y.stride(0) if _is_torch(Y) else k), k,
                              float(alpha), float(beta), _stream(stream)))
        return Y

    def pagerank(self, damping=0.85, tol=1e-8, max_iter=1000, p0=None, out=None, like=None,
                 stream=None):
        if out is None:
            out = _empty_like_vec(like if like is not None else (p0 if p0 is not None else np.empty(0)),
                                  self.n)
        info = IterInfo()
        _check(lib().spg_pagerank(self._h, float(damping), float(tol), int(max_iter), _ptr(p0)[0],
                                  _ptr(out)[0], ctypes.byref(info), _stream(stream)),
               allow_not_converged=True)
        return out, info.as_dict()

    def hits(self, norm=2, iters=50, auth=None, hub=None, like=None, stream=None):
        n = self.n_graph
        ref = like if like is not None else np.empty(0)
        auth = _empty_like_vec(ref, n) if auth is None else auth
        hub = _empty_like_vec(ref, n) if hub is None else hub
        info = IterInfo()
        _check(lib().spg_hits(self._h, int(norm), 0.0, int(iters), _ptr(auth)[0], _ptr(hub)[0],
                              ctypes.byref(info), _stream(stream)))
        return auth, hub, info.as_dict()

    def rwr(self, seeds, restart=0.15, tol=1e-8, max_iter=1000, out=None, like=None, stream=None):
        seeds = np.ascontiguousarray(np.atleast_1d(seeds), dtype=np.int32)
        k = int(seeds.shape[0])
        if out is None:
            out = _empty_like_vec(like if like is not None else np.empty(0), self.n, k)
        info = IterInfo()
        _check(lib().spg_rwr(self._h, float(restart), _ptr(seeds)[0], k, float(tol), int(max_iter),
                             _ptr(out)[0], ctypes.byref(info), _stream(stream)),
               allow_not_converged=True)
        return out, info.as_dict()

    # ------------------------------------------------------ differentiable RWR --
    def set_edge_logits(self, theta, stream=None):
        """P = softmax over each node's out-edges of theta (nnz, A's CSR order)."""
        _check(lib().spg_set_edge_logits(self._h, _ptr(theta)[0], _stream(stream)))

    def rwr_weighted(self, seed, restart=0.15, tol=1e-10, max_iter=2000, out=None, like=None,
                     stream=None):
        out = _empty_like_vec(like if like is not None else np.empty(0), self.n) if out is None else out
        info = IterInfo()
        _check(lib().spg_rwr_weighted(self._h, float(restart), int(seed), float(tol), int(max_iter),
                                      _ptr(out)[0], ctypes.byref(info), _stream(stream)),
               allow_not_converged=True)
        return out, info.as_dict()

    def rwr_adjoint(self, seed, r, g, restart=0.15, tol=1e-10, max_iter=2000, lam=None, dtheta=None,
                    stream=None):
        """lambda = c K^T lambda + g and dL/dtheta (see spg_rwr_adjoint)."""
        lam = _empty_like_vec(r, self.n) if lam is None else lam
        dtheta = _empty_like_vec(r, self.nnz_in) if dtheta is None else dtheta
        info = IterInfo()
        _check(lib().spg_rwr_adjoint(self._h, float(restart), int(seed), _ptr(r)[0], _ptr(g)[0],
                                     float(tol), int(max_iter), _ptr(lam)[0], _ptr(dtheta)[0],
                                     ctypes.byref(info), _stream(stream)), allow_not_converged=True)
        return lam, dtheta, info.as_dict()

    def baseline_spmv(self, which, x, y=None, alpha=1.0, beta=0.0, stream=None):
        if y is None:
            y = _empty_like_vec(x, self.n)
        _check(lib().spg_baseline_spmv(self._h, int(which), _ptr(x)[0], _ptr(y)[0], float(alpha),
                                       float(beta), _stream(stream)))
        return y

    def rank_step(self, damping, delta, xp, yp, stream=None):
        """One Eq. 6 iteration of this rank's rows (spg_pagerank_rank_step):
        returns (L1 change over the rank's rows, dangling mass of its rows)."""
        part = (ctypes.c_double * 2)()
        _check(lib().spg_pagerank_rank_step(self._h, float(damping), float(delta), _ptr(xp)[0],
                                            _ptr(yp)[0], part, _stream(stream)))
        return float(part[0]), float(part[1])

    def time_parts(self, mode=0, reps=20, stream=None):
        """Mean launch duration (ms) of each part's kernel (CUDA events)."""
        ms = np.zeros(self.nparts(), np.float32)
        _check(lib().spg_time_parts(self._h, int(mode), int(reps), _ptr(ms)[0], _stream(stream)))
        return ms

    def baseline_pagerank(self, which, damping=0.85, tol=1e-8, max_iter=1000, out=None, like=None,
                          stream=None):
        if out is None:
            out = _empty_like_vec(like if like is not None else np.empty(0), self.n)
        info = IterInfo()
        _check(lib().spg_baseline_pagerank(self._h, int(which), float(damping), float(tol),
                                           int(max_iter), _ptr(out)[0], ctypes.byref(info),
                                           _stream(stream)), allow_not_converged=True)
        return out, info.as_dict()


def _autograd():
    import torch

    class RWRStationary(torch.autograd.Function):
        """r(theta): stationary RWR vector with softmax edge weights.

        forward: P = edge softmax of theta written into the format, r = the
        RWR fixed point (spg_rwr_weighted).  backward: the adjoint fixed point
        lambda = c K^T lambda + dL/dr on the stored transposed layout and the
        softmax chain rule (spg_rwr_adjoint); no iterate is checkpointed."""

        @staticmethod
        def forward(ctx, theta, fmt, seed, restart=0.15, tol=1e-10, max_iter=2000):
            fmt.set_edge_logits(theta.detach().contiguous())
            r, _ = fmt.rwr_weighted(seed, restart, tol, max_iter, like=theta)
            ctx.fmt, ctx.seed, ctx.restart, ctx.tol, ctx.max_iter = fmt, seed, restart, tol, max_iter
            ctx.save_for_backward(r)
            return r

        @staticmethod
        def backward(ctx, grad_r):
            (r,) = ctx.saved_tensors
            _, dth, _ = ctx.fmt.rwr_adjoint(ctx.seed, r, grad_r.contiguous(), ctx.restart, ctx.tol,
                                            ctx.max_iter)
            return dth, None, None, None, None, None

    return RWRStationary


def partition_rows(row_len, P):
    """Section 3.2 bitonic row partition (spg_partition_rows): part of each
    row (int32[n]) for P parts, rows dealt by decreasing length."""
    rl = np.ascontiguousarray(row_len, dtype=np.int64)
    part = np.empty(rl.shape[0], np.int32)
    _check(lib().spg_partition_rows(rl.shape[0], _ptr(rl)[0], int(P), _ptr(part)[0]))
    return part


def pack_slice(idx, full, slice_, stream=None):
    """slice[i] = full[idx[i]] on the device (spg_pack_slice)."""
    _check(lib().spg_pack_slice(int(idx.shape[0]), _ptr(idx)[0], _ptr(full)[0], _ptr(slice_)[0],
                                _stream(stream)))
    return slice_


def unpack_slice(idx, slice_, full, stream=None):
    """full[idx[i]] = slice[i] on the device (spg_unpack_slice)."""
    _check(lib().spg_unpack_slice(int(idx.shape[0]), _ptr(idx)[0], _ptr(slice_)[0], _ptr(full)[0],
                                  _stream(stream)))
    return full


def pagerank_ranks(ranks, damping=0.85, tol=1e-8, max_iter=1000, p0=None, out=None, like=None,
                   stream=None):
    """Row-partitioned PageRank over the rank formats (spg_pagerank_ranks):
    ranks[r] built with the same row_part and part_id = r."""
    n = ranks[0].n_graph
    if out is None:
        out = _empty_like_vec(like if like is not None else (p0 if p0 is not None else np.empty(0)), n)
    arr = (ctypes.c_void_p * len(ranks))(*[f._h.value for f in ranks])
    info = IterInfo()
    _check(lib().spg_pagerank_ranks(ctypes.cast(arr, ctypes.c_void_p), len(ranks), float(damping),
                                    float(tol), int(max_iter), _ptr(p0)[0], _ptr(out)[0],
                                    ctypes.byref(info), _stream(stream)), allow_not_converged=True)
    return out, info.as_dict()


class BatchFormat:
    """Many independent graphs in one handle (spg_build_batch): one
    tiled-composite sweep per iteration over all of them."""

    def __init__(self, graphs, heavy_row=-1, layout_rule=1, max_warps=0, x_stage_cols=0,
                 slab_prefetch=0, loop_mode=0, max_rows=0, kernel=0, host_only=False, table=None,
                 claim_order=0, keep_plan=False, unit_slots=0, stream=None):
        L = lib()
        keep = []
        arr = (_Csr * len(graphs))()
        for g, (rp, col) in enumerate(graphs):
            rp = np.ascontiguousarray(rp, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
            keep += [rp, col]
            n = rp.shape[0] - 1
            arr[g] = _Csr(n, n, int(col.shape[0]), ctypes.c_void_p(rp.ctypes.data),
                          ctypes.c_void_p(col.ctypes.data), None, 0)
        tpath = table if table is not None else (TABLE_PATH if os.path.exists(TABLE_PATH) else None)
        opts = _Opts(0, 0, int(heavy_row), int(layout_rule), int(max_warps), 1, 0, 0, 0,
                     -1 if host_only else 0, 0.0, None if tpath is None else str(tpath).encode(),
                     int(x_stage_cols), int(slab_prefetch), int(loop_mode), int(max_rows),
                     int(kernel), 0)
        opts.claim_order = int(claim_order)
        opts.keep_plan = int(bool(keep_plan))
        opts.unit_slots = int(unit_slots)
        self._h = ctypes.c_void_p(None)
        _check(L.spg_build_batch(ctypes.cast(arr, ctypes.c_void_p), len(graphs), ctypes.byref(opts),
                                 _stream(stream), ctypes.byref(self._h)))
        self.count = len(graphs)
        self.offsets = np.empty(self.count + 1, np.int64)
        _check(L.spg_batch_offsets(self._h, _ptr(self.offsets)[0]))
        self.n = int(self.offsets[-1])

    def close(self):
        if self._h is not None and self._h.value:
            lib().spg_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        i = _Info()
        _check(lib().spg_format_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in _Info._fields_}

    tile_info = Format.tile_info
    export_plan = Format.export_plan
    perm = Format.perm

    def export_entries(self):
        nnz = self.info()["nnz"]
        r = np.empty(nnz, np.int64)
        c = np.empty(nnz, np.int32)
        v = np.empty(nnz, np.float32)
        _check(lib().spg_format_export_entries(self._h, _ptr(r)[0], _ptr(c)[0], _ptr(v)[0]))
        return r, c, v

    def pagerank(self, damping=0.85, tol=1e-8, max_iter=1000, out=None, like=None, stream=None):
        """Concatenated PageRank vectors and one info dict per graph."""
        out = _empty_like_vec(like if like is not None else np.empty(0), self.n) if out is None else out
        infos = (IterInfo * self.count)()
        _check(lib().spg_batch_pagerank(self._h, float(damping), float(tol), int(max_iter),
                                        _ptr(out)[0], ctypes.cast(infos, ctypes.c_void_p),
                                        _stream(stream)), allow_not_converged=True)
        return out, [x.as_dict() for x in infos]

    def split(self, vec):
        return [vec[self.offsets[g]:self.offsets[g + 1]] for g in range(self.count)]


_rwr_fn = None


def __getattr__(name):
    global _rwr_fn
    if name == "RWRStationary":
        if _rwr_fn is None:
            _rwr_fn = _autograd()
        return _rwr_fn
    raise AttributeError(name)
