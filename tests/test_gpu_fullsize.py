"""Full-size parity on the R-MAT scale-22 workload (4,194,304 nodes, edge
factor 16), in the launch configuration bench.py times (default build
options).  SpMV: sampled rows -- random ones plus the heaviest (split) rows
-- against the oracle computed row by row.  PageRank: the oracle's fixed
point computed in full (FP64, single thread, tens of seconds), L1 <= 1e-6."""
import numpy as np
import pytest
import torch

import graphgen
import oracle
import paper_1103_2405_gb300 as spg

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def g22():
    rp, col = graphgen.rmat(22, 16, seed=1)
    return rp, col, oracle.build_M(rp, col)


def test_spmv_sampled_rows_scale22(g22):
    rp, col, M = g22
    n = rp.shape[0] - 1
    f = spg.Format(rp, col, kind="pagerank")
    x = graphgen.uniform(n, 2)
    y = f.spmv(torch.from_numpy(x).to(DEV))
    torch.cuda.synchronize()
    y = y.cpu().numpy()
    indeg = np.diff(M[0])
    heavy = np.argsort(-indeg, kind="stable")[:256]
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([heavy, rng.integers(0, n, 8192), [0, n - 1]]))
    ref = oracle.spmv_rows(M, rows, x)
    bound = oracle.spmv_rows((M[0], M[1], np.abs(M[2])), rows, x)
    assert np.all(np.abs(y[rows] - ref) <= 1e-5 * bound + 1e-30)
    assert np.linalg.norm(y[rows] - ref) / np.linalg.norm(ref) <= 1e-5
    assert f.info()["split_rows"] > 0


def test_pagerank_scale22(g22):
    rp, col, M = g22
    f = spg.Format(rp, col, kind="pagerank")
    p, info = f.pagerank(0.85, tol=1e-8, max_iter=1000, like=torch.empty(0, device=DEV))
    p = p.cpu().numpy().astype(np.float64)
    assert abs(p.sum() - 1.0) <= 1e-5
    p_star, _, _ = oracle.pagerank(rp, col, 0.85, tol=1e-11, M=M)
    assert np.abs(p - p_star).sum() <= 1e-6
