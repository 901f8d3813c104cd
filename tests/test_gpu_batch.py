"""GPU parity of the batched PageRank over many independent Chung-Lu graphs
(block-diagonal union, per-graph degree order, one sweep per iteration),
against the oracle's fixed point of every graph: ||p_g - p_g*||_1 <= 1e-6."""
import numpy as np
import pytest
import torch

import graphgen
import oracle
import paper_1103_2405_gb300 as spg

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _batch(count, lo, hi, seed=1000):
    sizes = graphgen.chung_lu_batch_sizes(count, lo, hi, seed)
    graphs = []
    for g, n in enumerate(sizes):
        n = int(n)
        graphs.append(graphgen.chung_lu(n, 12 * n, 2.3, max(2.0, n / 4), seed=seed + g))
    return graphs


@pytest.mark.parametrize("opts", [dict(), dict(x_stage_cols=-1, heavy_row=0),
                                  dict(claim_order=1), dict(kernel=1, unit_slots=1)])
def test_batch_pagerank_matches_oracle(opts):
    graphs = _batch(24, 6, 12)
    graphs.append((np.zeros(4, np.int64), np.zeros(0, np.int32)))    # edgeless graph
    b = spg.BatchFormat(graphs, **opts)
    p, infos = b.pagerank(0.85, tol=1e-8, max_iter=1000, like=torch.empty(0, device=DEV))
    p = p.cpu().numpy()
    assert len(infos) == len(graphs)
    for g, ((rp, col), pg) in enumerate(zip(graphs, b.split(p))):
        p_star, it_ref, _ = oracle.pagerank(rp, col, 0.85, tol=1e-13)
        assert np.abs(pg - p_star).sum() <= 1e-6, g
    # per-graph convergence iterations, at a tolerance well above the FP32
    # noise floor of the L1 change of small graphs (n_g * ulp(p) ~ 1e-8)
    _, infos6 = b.pagerank(0.85, tol=1e-6, max_iter=1000, like=torch.empty(0, device=DEV))
    for g, (rp, col) in enumerate(graphs):
        _, it6, _ = oracle.pagerank(rp, col, 0.85, tol=1e-6)
        assert abs(infos6[g]["iters"] - it6) <= 1, (g, infos6[g], it6)


def test_batch_fixed_iterations_equal_single_graph_runs():
    graphs = _batch(6, 8, 10, seed=77)
    b = spg.BatchFormat(graphs)
    p, _ = b.pagerank(0.85, tol=0.0, max_iter=7, like=torch.empty(0, device=DEV))
    for (rp, col), pg in zip(graphs, b.split(p.cpu().numpy())):
        ref, _, _ = oracle.pagerank(rp, col, 0.85, tol=0.0, max_iter=7)
        assert np.abs(pg - ref).sum() <= 1e-6


@pytest.mark.parametrize("opts", [dict(), dict(x_stage_cols=-1)])
def test_claim_orders_agree_bit_for_bit(opts):
    # graph-by-graph and ranking claim orders, persistent and plain kernels:
    # every row is summed in the same order, so the iterates are identical
    graphs = _batch(40, 6, 12, seed=31)
    like = torch.empty(0, device=DEV)
    p, _ = spg.BatchFormat(graphs, **opts).pagerank(0.85, tol=0.0, max_iter=9, like=like)
    q, _ = spg.BatchFormat(graphs, claim_order=1).pagerank(0.85, tol=0.0, max_iter=9, like=like)
    assert torch.equal(p, q)
