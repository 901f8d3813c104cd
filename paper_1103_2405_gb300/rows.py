"""Row-partitioned PageRank across ranks (Section 3.2), one driver for any
number of processes.

Each rank holds its own rows of M -- a handle built with ``row_part`` /
``part_id`` (rows dealt bitonically by ``partition_rows``) over all columns
in the column order of the whole matrix, so that every rank's iterate lives
in one permuted index space -- and per iteration:

1. computes its rows of y' = c M' x' + (c delta + 1 - c) / n and its partial
   sums (L1 change over its rows, dangling mass of its rows) with its own
   kernels (``spg_pagerank_rank_step``);
2. packs its rows of y' into a contiguous slice (``spg_pack_slice``);
3. all-gathers every rank's slice and scatters them into its whole x'
   (``spg_unpack_slice``), so every rank holds the new iterate;
4. all-reduces the partials, summed in rank order (the same order, hence
   the same FP64 result and the same stop decision, on every rank);
5. stops when the L1 change is below tol, or after max_iter iterations.

The exchange of steps 3-4 is an interface with two implementations:
``LocalExchange`` (every rank in this process, e.g. several handles on one
device) and ``DistExchange`` (torch.distributed, one rank per process:
``all_gather`` of the slices and of the partials).  The rank's computation
is an interface too (``step``, ``pack``, ``unpack``): ``DeviceRank`` runs
the library's kernels; anything with the same three methods can stand in
for it.
"""
from __future__ import annotations

import numpy as np

from . import Format, pack_slice, partition_rows, unpack_slice


def rank_positions(row_part, pi, nparts):
    """Permuted positions owned by each rank, ascending: rank r owns the
    positions pi[v] of the nodes v with row_part[v] == r."""
    row_part = np.asarray(row_part)
    pi = np.asarray(pi)
    return [np.sort(pi[np.flatnonzero(row_part == r)]).astype(np.int32) for r in range(nparts)]


def uniform_start(n, dangling_start):
    """x' = 1/n everywhere and its dangling mass (positions >= dangling_start
    are the dangling nodes in the degree order)."""
    return 1.0 / n, float(n - dangling_start) / n


class DeviceRank:
    """One rank's iterate, scratch and index lists on a CUDA device, stepped
    by the library's kernels."""

    def __init__(self, fmt: Format, rank: int, positions, device):
        import torch
        self.fmt, self.rank = fmt, rank
        info = fmt.info()
        self.n, self.dangling_start = info["n"], info["dangling_start"]
        v0, self.delta0 = uniform_start(self.n, self.dangling_start)
        self.x = torch.full((self.n,), v0, dtype=torch.float32, device=device)
        self.y = torch.empty(self.n, dtype=torch.float32, device=device)
        self.idx = [torch.from_numpy(p).to(device) for p in positions]
        self.slice = torch.empty(len(positions[rank]), dtype=torch.float32, device=device)

    def step(self, damping, delta):
        return self.fmt.rank_step(damping, delta, self.x, self.y)

    def pack(self):
        return pack_slice(self.idx[self.rank], self.y, self.slice)

    def unpack(self, slices):
        for r, sl in enumerate(slices):
            unpack_slice(self.idx[r], sl, self.x)


class LocalExchange:
    """Every rank in this process: the slices and partials are already here."""

    def allgather(self, slices):
        return list(slices)

    def sum_ranks(self, partials):
        l1 = delta = 0.0
        for a, b in partials:          # rank order
            l1 += a
            delta += b
        return l1, delta


class DistExchange:
    """One rank per process over torch.distributed (NCCL between GPUs, gloo
    on CPU): slices of unequal length travel padded to the longest."""

    def __init__(self, lengths, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.lengths = [int(x) for x in lengths]
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def allgather(self, slices):
        import torch
        (mine,) = slices
        width = max(self.lengths)
        pad = torch.zeros(width, dtype=mine.dtype, device=mine.device)
        pad[: mine.shape[0]] = mine
        out = [torch.empty_like(pad) for _ in range(self.world)]
        self.dist.all_gather(out, pad, group=self.group)
        return [o[:n] for o, n in zip(out, self.lengths)]

    def sum_ranks(self, partials):
        import torch
        (mine,) = partials
        t = torch.tensor(mine, dtype=torch.float64)
        if self.dist.get_backend(self.group) == "nccl":
            t = t.cuda()
        out = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t, group=self.group)
        l1 = delta = 0.0
        for o in out:                  # rank order, on every rank
            a, b = o.tolist()
            l1 += a
            delta += b
        return l1, delta


def pagerank_rows(ranks, exchange, damping=0.85, tol=1e-8, max_iter=1000):
    """Run the row-partitioned iteration over this process's ranks (all of
    them with LocalExchange, one with DistExchange).  Returns (iterations,
    last L1 change, dangling mass of the final iterate); every rank's x then
    holds the final iterate in permuted order."""
    delta = ranks[0].delta0
    l1 = float("inf")
    it = 0
    while it < max_iter:
        partials = [r.step(damping, delta) for r in ranks]
        slices = exchange.allgather([r.pack() for r in ranks])
        for r in ranks:
            r.unpack(slices)
        l1, delta = exchange.sum_ranks(partials)
        it += 1
        if tol > 0 and l1 < tol:
            break
    return it, l1, delta


def build_rank(rowptr, col, rank, nparts, **opts):
    """The rank's handle and the row partition: rows of M (nodes by
    in-degree) dealt bitonically to nparts ranks (Section 3.2)."""
    n = int(np.asarray(rowptr).shape[0]) - 1
    indeg = np.bincount(np.asarray(col), minlength=n).astype(np.int64)
    row_part = partition_rows(indeg, nparts)
    fmt = Format(rowptr, col, kind="pagerank", row_part=row_part, part_id=rank, nparts=nparts, **opts)
    pi, inv = fmt.perm()
    return fmt, row_part, rank_positions(row_part, pi, nparts), inv
