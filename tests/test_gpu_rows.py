"""The row-partitioned driver (Section 3.2) on the GPU: each rank's rows
stepped by the library's kernels (spg_pagerank_rank_step), its slice packed
and unpacked by spg_pack_slice / spg_unpack_slice, exchanged through the
driver's exchange interface -- in one process (P = 1, 2, 3 ranks on one
device) and through torch.distributed with NCCL at world size 1.  The result
must be the oracle's fixed point (L1 <= 1e-6)."""
import socket

import numpy as np
import pytest
import torch

import graphgen
import oracle
from paper_1103_2405_gb300 import rows

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
C = 0.85


@pytest.fixture(scope="module")
def g13():
    rp, col = graphgen.rmat(13, 8, seed=2)
    p_star, _, _ = oracle.pagerank(rp, col, C, tol=1e-13)
    _, it_ref, _ = oracle.pagerank(rp, col, C, tol=1e-8)
    return rp, col, p_star, it_ref


@pytest.mark.parametrize("P", [1, 2, 3])
def test_local_ranks_reach_the_fixed_point(g13, P):
    rp, col, p_star, it_ref = g13
    ranks = []
    for r in range(P):
        fmt, row_part, positions, inv = rows.build_rank(rp, col, r, P, tile_width=2048)
        ranks.append(rows.DeviceRank(fmt, r, positions, DEV))
    it, l1, delta = rows.pagerank_rows(ranks, rows.LocalExchange(), damping=C, tol=1e-8, max_iter=1000)
    torch.cuda.synchronize()
    pi, _ = ranks[0].fmt.perm()
    for rk in ranks:       # every rank holds the whole final iterate
        assert torch.equal(rk.x, ranks[0].x)
    p = ranks[0].x.cpu().numpy().astype(np.float64)[pi]
    assert l1 < 1e-8 and abs(it - it_ref) <= 2
    assert abs(p.sum() - 1.0) <= 1e-5
    assert np.abs(p - p_star).sum() <= 1e-6


def test_distributed_exchange_world_size_one(g13):
    import torch.distributed as dist
    rp, col, p_star, it_ref = g13
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        fmt, row_part, positions, inv = rows.build_rank(rp, col, 0, 1)
        me = rows.DeviceRank(fmt, 0, positions, DEV)
        ex = rows.DistExchange([len(p) for p in positions])
        it, l1, delta = rows.pagerank_rows([me], ex, damping=C, tol=1e-8, max_iter=1000)
        torch.cuda.synchronize()
    finally:
        dist.destroy_process_group()
    pi, _ = fmt.perm()
    p = me.x.cpu().numpy().astype(np.float64)[pi]
    assert np.abs(p - p_star).sum() <= 1e-6 and abs(it - it_ref) <= 2
