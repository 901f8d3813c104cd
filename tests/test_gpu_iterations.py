"""GPU parity of the fused power iterations (Appendix F) against the oracle.

PageRank (Eq. 6) and RWR (Eq. 9) are compared with the oracle's converged
fixed point p* (tol 1e-13): ||p - p*||_1 <= 1e-6 (the target).  HITS (Eqs.
7-8) is compared iterate for iterate at iteration 50: relative L2 <= 1e-5 per
half.  Closed forms check the tiny graphs end to end."""
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
    return rp, col, M, p_star


@pytest.mark.parametrize("opts", [dict(), dict(tile_width=2048), dict(tile_width=512, heavy_row=0),
                                  dict(pattern_only=True), dict(pattern_only=True, tile_width=1024),
                                  dict(kernel=2), dict(kernel=3), dict(kernel=1),
                                  dict(kernel=1, pattern_only=True, tile_width=4096)])
def test_pagerank_matches_oracle(g14, opts):
    rp, col, M, p_star = g14
    f = spg.Format(rp, col, kind="pagerank", **opts)
    p, info = f.pagerank(C, tol=1e-8, max_iter=1000, like=torch.empty(0, device=DEV))
    p = p.cpu().numpy().astype(np.float64)
    assert np.abs(p - p_star).sum() <= 1e-6
    assert abs(p.sum() - 1.0) <= 1e-5
    _, it_ref, _ = oracle.pagerank(rp, col, C, tol=1e-8, M=M)
    assert abs(info["iters"] - it_ref) <= 2
    assert info["last_l1"] < 1e-8


@pytest.mark.parametrize("opts", [dict(), dict(tile_width=2048, heavy_row=32), dict(unit_slots=1)])
def test_claim_order_does_not_change_the_result(g14, opts):
    # longest-first and ranking-order claims: every row has one writer and
    # split rows combine in chunk order, so the iterates agree bit for bit
    rp, col, M, p_star = g14
    like = torch.empty(0, device=DEV)
    got = []
    for order in (0, 1):
        f = spg.Format(rp, col, kind="pagerank", claim_order=order, **opts)
        p, info = f.pagerank(C, tol=1e-8, max_iter=1000, like=like)
        x = torch.from_numpy(graphgen.uniform(rp.shape[0] - 1, 3)).to(DEV)
        got.append((p.cpu(), info["iters"], f.spmv(x).cpu()))
    for other in got[1:]:
        assert torch.equal(got[0][0], other[0]) and got[0][1] == other[1]
        assert torch.equal(got[0][2], other[2])
    assert np.abs(got[0][0].numpy().astype(np.float64) - p_star).sum() <= 1e-6


def test_pagerank_warm_start_and_limits(g14):
    rp, col, M, p_star = g14
    f = spg.Format(rp, col, kind="pagerank")
    n = rp.shape[0] - 1
    p0 = torch.from_numpy(p_star.astype(np.float32)).to(DEV)
    p, info = f.pagerank(C, tol=1e-6, max_iter=100, p0=p0)
    assert info["iters"] <= 2
    # max_iter = 0 returns the start vector; an unreachable tol reports not converged
    p, info = f.pagerank(C, tol=1e-8, max_iter=0, like=p0)
    assert info["iters"] == 0 and np.allclose(p.cpu().numpy(), 1.0 / n)
    p, info = f.pagerank(C, tol=1e-30, max_iter=5, like=p0)
    assert info["iters"] == 5
    # exactly K iterations equal K oracle iterations
    p5_ref, _, _ = oracle.pagerank(rp, col, C, tol=0.0, max_iter=5, M=M)
    assert np.abs(p.cpu().numpy() - p5_ref).sum() <= 1e-6


@pytest.mark.parametrize("which", [spg.CSR_SCALAR, spg.CSR_VECTOR])
def test_baseline_pagerank(g14, which):
    rp, col, M, p_star = g14
    f = spg.Format(rp, col, kind="pagerank", keep_csr=True)
    p, info = f.baseline_pagerank(which, C, tol=1e-8, max_iter=1000, like=torch.empty(0, device=DEV))
    assert np.abs(p.cpu().numpy() - p_star).sum() <= 1e-6


def test_pagerank_closed_forms():
    for n in (5, 33, 1000):
        edges = [(i, 0) for i in range(1, n)]              # in-star, dangling centre
        rp, col = graphgen.edges_to_csr(n, [e[0] for e in edges], [e[1] for e in edges])
        f = spg.Format(rp, col, kind="pagerank")
        p, _ = f.pagerank(C, tol=1e-9, max_iter=1000, like=torch.empty(0, device=DEV))
        p = p.cpu().numpy()
        centre = (1 + C * (n - 1)) / (n + C * (n - 1))
        assert abs(p[0] - centre) <= 1e-6
        cyc_rp, cyc_col = graphgen.edges_to_csr(n, np.arange(n), (np.arange(n) + 1) % n)
        q, _ = spg.Format(cyc_rp, cyc_col).pagerank(C, tol=1e-9, max_iter=100,
                                                    like=torch.empty(0, device=DEV))
        assert np.allclose(q.cpu().numpy(), 1.0 / n, rtol=1e-6)


@pytest.mark.parametrize("norm", [2, 1])
@pytest.mark.parametrize("opts", [dict(), dict(tile_width=4096, heavy_row=64), dict(kernel=1)])
def test_hits_matches_oracle(norm, opts):
    rp, col = graphgen.rmat(13, 8, seed=1)
    a_ref, h_ref = oracle.hits(rp, col, iters=50, norm=norm)
    f = spg.Format(rp, col, kind="hits", **opts)
    a, h, info = f.hits(norm=norm, iters=50, like=torch.empty(0, device=DEV))
    a, h = a.cpu().numpy(), h.cpu().numpy()
    assert info["iters"] == 50
    assert np.linalg.norm(a - a_ref) / np.linalg.norm(a_ref) <= 1e-5
    assert np.linalg.norm(h - h_ref) / np.linalg.norm(h_ref) <= 1e-5


def test_hits_golden_ratio():
    rp, col = graphgen.edges_to_csr(4, [0, 0, 1], [2, 3, 3])
    a, h, _ = spg.Format(rp, col, kind="hits").hits(norm=2, iters=50, like=torch.empty(0, device=DEV))
    a, h = a.cpu().numpy(), h.cpu().numpy()
    phi = (1 + 5 ** 0.5) / 2
    assert abs(a[3] / a[2] - phi) <= 1e-5 and abs(h[0] / h[1] - phi) <= 1e-5


@pytest.mark.parametrize("opts", [dict(), dict(tile_width=1024, heavy_row=32), dict(kernel=1)])
def test_rwr_single_seed(g14, opts):
    rp, col, M, _ = g14
    s = graphgen.pick_source(rp, 3)
    r_star, _, _ = oracle.rwr(rp, col, s, C, tol=1e-13, M=M)
    f = spg.Format(rp, col, kind="pagerank", **opts)
    r, info = f.rwr([s], restart=0.15, tol=1e-8, max_iter=1000, like=torch.empty(0, device=DEV))
    r = r.cpu().numpy()
    assert np.abs(r - r_star).sum() <= 1e-6 and abs(r.sum() - 1) <= 1e-5


@pytest.mark.parametrize("k,opts", [(64, dict(vec_width=64)), (7, dict(tile_width=2048, heavy_row=64))])
def test_rwr_batched_seeds(g14, k, opts):
    rp, col, M, _ = g14
    seeds = graphgen.pick_seeds(rp, k, 4)
    f = spg.Format(rp, col, kind="pagerank", **opts)
    R, info = f.rwr(seeds, restart=0.15, tol=1e-8, max_iter=1000, like=torch.empty(0, device=DEV))
    R = R.cpu().numpy()
    assert R.shape == (rp.shape[0] - 1, k)
    for j in list(range(0, k, max(1, k // 8))) + [k - 1]:
        r_star, _, _ = oracle.rwr(rp, col, int(seeds[j]), C, tol=1e-13, M=M)
        assert np.abs(R[:, j] - r_star).sum() <= 1e-6, j


def test_rwr_refuses_more_than_64_seeds(g14):
    rp, col, M, _ = g14
    f = spg.Format(rp, col, kind="pagerank")
    with pytest.raises(spg.SpgError) as e:
        f.rwr(graphgen.pick_seeds(rp, 65, 4), restart=0.15, tol=1e-8, max_iter=10,
              like=torch.empty(0, device=DEV))
    assert e.value.status == -1
