"""Row-partitioned PageRank (Section 3.2) emulated on one GPU: P rank
formats built from the bitonic row partition, each computing its own rows
into its own iterate buffers, an all-gather step and an all-reduce of the
(L1, dangling) partials per iteration.  The result must equal the FP64
oracle's fixed point within the PageRank tolerance, for any P."""
import numpy as np
import pytest
import torch

import graphgen
import oracle
import paper_1103_2405_gb300 as spg

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
C = 0.85


@pytest.fixture(scope="module")
def g14():
    rp, col = graphgen.rmat(14, 8, seed=1)
    M = oracle.build_M(rp, col)
    p_star, _, _ = oracle.pagerank(rp, col, C, tol=1e-13, M=M)
    _, it_ref, _ = oracle.pagerank(rp, col, C, tol=1e-8, M=M)
    return rp, col, M, p_star, it_ref


@pytest.mark.parametrize("P,opts", [(1, {}), (2, {}), (3, dict(tile_width=4096)), (4, {}),
                                    (8, dict(heavy_row=64)), (3, dict(pattern_only=True))])
def test_ranks_pagerank_matches_oracle(g14, P, opts):
    rp, col, M, p_star, it_ref = g14
    part = spg.partition_rows(np.diff(M[0]), P)
    ranks = [spg.Format(rp, col, kind="pagerank", row_part=part, part_id=r, nparts=P, **opts)
             for r in range(P)]
    p, info = spg.pagerank_ranks(ranks, C, tol=1e-8, max_iter=1000, like=torch.empty(0, device=DEV))
    p = p.cpu().numpy().astype(np.float64)
    assert np.abs(p - p_star).sum() <= 1e-6
    assert abs(p.sum() - 1.0) <= 1e-5
    assert abs(info["iters"] - it_ref) <= 2 and info["last_l1"] < 1e-8


def test_ranks_agree_with_one_handle_and_reject_mismatches(g14):
    rp, col, M, p_star, _ = g14
    P = 2
    part = spg.partition_rows(np.diff(M[0]), P)
    ranks = [spg.Format(rp, col, kind="pagerank", row_part=part, part_id=r, nparts=P) for r in range(P)]
    like = torch.empty(0, device=DEV)
    p5, info = spg.pagerank_ranks(ranks, C, tol=0.0, max_iter=5, like=like)
    assert info["iters"] == 5
    q5, _ = spg.Format(rp, col, kind="pagerank").pagerank(C, tol=0.0, max_iter=5, like=like)
    assert np.abs(p5.cpu().numpy() - q5.cpu().numpy()).sum() <= 1e-6
    with pytest.raises(spg.SpgError):
        spg.pagerank_ranks(ranks[::-1], C, like=like)           # part ids out of order
    other = spg.Format(rp, col, kind="pagerank")
    with pytest.raises(spg.SpgError):
        spg.pagerank_ranks([ranks[0], other], C, like=like)     # not a rank format
