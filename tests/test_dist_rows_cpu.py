"""The row-partitioned driver (Section 3.2) across processes, on CPU ranks:
two gloo processes each hold one rank of the bitonic row partition of a
small R-MAT graph and run paper_1103_2405_gb300.rows.pagerank_rows with the
torch.distributed exchange -- slice packing by permuted position, all-gather
of unequal slices, partials summed in rank order, the stop rule.  Each
rank's own rows are computed by a float64 NumPy stand-in for the library's
kernels (there is no GPU here); the result must be the oracle's fixed point
and both ranks must end with the same iterate and iteration count."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C = 0.85


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class HostRank:
    """A rank stepped in float64 NumPy (test stand-in for DeviceRank)."""

    def __init__(self, M, pi, inv, rank, positions, dangling_start):
        self.rank, self.positions = rank, positions
        self.n = pi.shape[0]
        self.dangling_start = dangling_start
        self.x = np.full(self.n, 1.0 / self.n)
        self.y = np.zeros(self.n)
        self.delta0 = float(self.n - dangling_start) / self.n
        rp, col, val = M
        own = positions[rank]
        self.rows = [(k, pi[col[rp[inv[k]]:rp[inv[k] + 1]]], val[rp[inv[k]]:rp[inv[k] + 1]].astype(np.float64))
                     for k in own]

    def step(self, damping, delta):
        base = (damping * delta + 1.0 - damping) / self.n
        l1 = dang = 0.0
        for k, cols, vals in self.rows:
            f = damping * float(np.dot(vals, self.x[cols])) + base
            self.y[k] = f
            l1 += abs(f - self.x[k])
            if k >= self.dangling_start:
                dang += f
        return l1, dang

    def pack(self):
        import torch
        return torch.from_numpy(self.y[self.positions[self.rank]].copy())

    def unpack(self, slices):
        for r, sl in enumerate(slices):
            self.x[self.positions[r]] = sl.numpy()


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import graphgen
    import oracle
    from paper_1103_2405_gb300 import rows
    rp, col = graphgen.rmat(10, 8, seed=1)
    fmt, row_part, positions, inv = rows.build_rank(rp, col, rank, world, host_only=True)
    pi, _ = fmt.perm()
    M = oracle.build_M(rp, col)
    me = HostRank(M, pi, inv, rank, positions, fmt.info()["dangling_start"])
    ex = rows.DistExchange([len(p) for p in positions])
    it, l1, delta = rows.pagerank_rows([me], ex, damping=C, tol=1e-10, max_iter=500)
    out[rank] = (it, l1, me.x[pi].copy(), [len(p) for p in positions])
    dist.barrier()
    dist.destroy_process_group()


def test_two_process_row_partition_reaches_the_fixed_point():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import graphgen
    import oracle
    rp, col = graphgen.rmat(10, 8, seed=1)
    p_star, it_ref, _ = oracle.pagerank(rp, col, C, tol=1e-13)
    _, it_tol, _ = oracle.pagerank(rp, col, C, tol=1e-10)
    (it0, l10, x0, lens), (it1, l11, x1, _) = out[0], out[1]
    n = rp.shape[0] - 1
    assert sum(lens) == n and min(lens) > 0            # every row owned once
    assert it0 == it1 and l10 == l11                    # same stop decision
    assert np.array_equal(x0, x1)                       # same iterate everywhere
    assert l10 < 1e-10 and abs(it0 - it_tol) <= 1
    assert np.abs(x0 - p_star).sum() <= 1e-9
