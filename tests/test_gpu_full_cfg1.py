"""Full-size parity on the R-MAT scale-22 workload (4,194,304 nodes, edge
factor 16, 65,243,428 edges after dedup), default build options -- the
iterations of Appendix F beyond PageRank, each against the FP64 oracle run
in full:

* HITS (Eqs. 7-8, Jacobi form, L2-normalised halves) at iteration 50:
  relative L2 <= 1e-5 per half against the oracle's iteration 50;
* single-source RWR (Eq. 9 on M, restart 0.15): ||r - r*||_1 <= 1e-6
  against the oracle's fixed point;
* RWR with 64 restart vectors as one SpMM per iteration: the fixed point of
  four sampled columns against the oracle's (computed side by side in
  spawned worker processes), plus one plain SpMM (k = 64) on sampled rows of
  every column against the oracle's row sums (relative L2 <= 1e-5 per
  column)."""
import numpy as np
import pytest
import torch

import graphgen
import oracle
import paper_1103_2405_gb300 as spg
import _fullsize_refs as refs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
C = 0.85


@pytest.fixture(scope="module")
def g22():
    rp, col = graphgen.rmat(22, 16, seed=1)
    return rp, col, oracle.build_M(rp, col)


def test_hits_iteration50_scale22(g22):
    rp, col, M = g22
    f = spg.Format(rp, col, kind="hits")
    a, h, info = f.hits(norm=2, iters=50, like=torch.empty(0, device=DEV))
    assert info["iters"] == 50
    a_ref, h_ref = oracle.hits(rp, col, iters=50, norm=2)
    for got, ref in ((a, a_ref), (h, h_ref)):
        got = got.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_rwr_single_source_scale22(g22):
    rp, col, M = g22
    s = graphgen.pick_source(rp, 3)
    f = spg.Format(rp, col, kind="pagerank")
    r, info = f.rwr([s], 1 - C, tol=1e-9, max_iter=2000, like=torch.empty(0, device=DEV))
    r = r.cpu().numpy().astype(np.float64)
    r_ref, _, _ = oracle.rwr(rp, col, s, C, tol=1e-12, M=M)
    assert abs(r.sum() - 1.0) <= 1e-5
    assert np.abs(r - r_ref).sum() <= 1e-6


def test_rwr64_spmm_scale22(g22):
    rp, col, M = g22
    n = rp.shape[0] - 1
    seeds = graphgen.pick_seeds(rp, 64, 4)
    f = spg.Format(rp, col, kind="pagerank", vec_width=64)
    # plain SpMM first: Y = M X on sampled rows, every column
    X = torch.from_numpy(graphgen.uniform(n * 64, 2).reshape(n, 64)).to(DEV)
    Y = f.spmm(X).cpu().numpy()
    Xh = X.cpu().numpy()
    rng = np.random.default_rng(2)
    indeg = np.diff(M[0])
    rows = np.unique(np.concatenate([np.argsort(-indeg, kind="stable")[:64],
                                     rng.integers(0, n, 512)]))
    for j in range(64):
        ref = oracle.spmv_rows(M, rows, Xh[:, j])
        bound = oracle.spmv_rows((M[0], M[1], np.abs(M[2])), rows, np.abs(Xh[:, j]))
        # relative L2 per column over the sampled rows (the SpMV tolerance);
        # each element within 1e-4 of its |M||x| bound (long rows are summed
        # serially per lane in FP32)
        assert np.linalg.norm(Y[rows, j] - ref) <= 1e-5 * np.linalg.norm(ref), j
        assert np.all(np.abs(Y[rows, j] - ref) <= 1e-4 * bound + 1e-30), j
    del X, Y, Xh
    # the 64-seed RWR solve, four sampled columns against the oracle
    R, info = f.rwr(seeds, 1 - C, tol=1e-9, max_iter=2000, like=torch.empty(0, device=DEV))
    R = R.cpu().numpy().astype(np.float64)
    cols = [0, 21, 42, 63]
    ref = refs.pool_map(refs.rwr_column, [(22, 16, int(seeds[j]), 1e-12) for j in cols], 4)
    for j, rj in zip(cols, ref):
        assert abs(R[:, j].sum() - 1.0) <= 1e-5, j
        assert np.abs(R[:, j] - rj).sum() <= 1e-6, j
