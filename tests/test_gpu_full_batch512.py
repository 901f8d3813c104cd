"""Full-size parity of the batching workload: 512 independent Chung-Lu
graphs (node counts log-uniform in [2^10, 2^17], exponent 2.3, average
degree 12, seeds 1000 + g), PageRank (Eq. 6, d = 0.85, tol 1e-8) on all of
them in one batched handle; every graph's result against the oracle's fixed
point of that graph (tol 1e-13, computed in spawned worker processes):
||p_g - p_g*||_1 <= 1e-6."""
import numpy as np
import pytest
import torch

import graphgen
import paper_1103_2405_gb300 as spg
import _fullsize_refs as refs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def test_batch512_every_graph_matches_oracle():
    sizes = graphgen.chung_lu_batch_sizes(512, 10, 17, 1000)
    graphs = [refs.batch_graph(g, n) for g, n in enumerate(sizes)]
    assert sum(int(g[0].shape[0] - 1) for g in graphs) > 10_000_000
    b = spg.BatchFormat(graphs)
    p, infos = b.pagerank(0.85, tol=1e-8, max_iter=1000, like=torch.empty(0, device=DEV))
    assert len(infos) == 512 and all(i["iters"] > 0 for i in infos)
    p = p.cpu().numpy()
    ref = refs.pool_map(refs.batch_pagerank, [(g, n, 1e-13) for g, n in enumerate(sizes)], 16)
    worst = 0.0
    for g, (pg, pr) in enumerate(zip(b.split(p), ref)):
        err = np.abs(pg.astype(np.float64) - pr).sum()
        worst = max(worst, err)
        assert err <= 1e-6, (g, err)
    print(f"worst per-graph L1 {worst:.2e}")
