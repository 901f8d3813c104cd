"""Pins of the oracle's HITS (Eq. 7, Jacobi, per-half normalisation) and RWR
(Eq. 9 on M, dangling mass to the restart node).

HITS: complete bipartite graphs (uniform scores), the two-hub graph whose
authority/hub ratio is the golden ratio, and the principal eigenvector of
A^T A from a dense eigensolver.  RWR: dense linear solve, sum(r) = 1 and the
reversibility identity deg(s) r_s(t) = deg(t) r_t(s) on undirected graphs."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from _helpers import dense_M, csr_from_edges  # noqa: E402

import oracle  # noqa: E402

C = 0.85
PHI = (1 + 5 ** 0.5) / 2


def test_hits_complete_bipartite_uniform():
    hubs, auths = [0, 1, 2], [3, 4, 5, 6]
    edges = [(h, a) for h in hubs for a in auths]
    rp, col = csr_from_edges(7, edges)
    for norm in (1, 2):
        a, h = oracle.hits(rp, col, iters=50, norm=norm)
        expect_a = 1 / len(auths) if norm == 1 else 1 / len(auths) ** 0.5
        expect_h = 1 / len(hubs) if norm == 1 else 1 / len(hubs) ** 0.5
        np.testing.assert_allclose(a[auths], expect_a, rtol=1e-14)
        np.testing.assert_allclose(a[hubs], 0.0, atol=0)
        np.testing.assert_allclose(h[hubs], expect_h, rtol=1e-14)
        np.testing.assert_allclose(h[auths], 0.0, atol=0)


def test_hits_two_hub_golden_ratio():
    # h1 -> {a1, a2}, h2 -> {a2}: A^T A = [[1,1],[1,2]], a2/a1 = h1/h2 = phi
    h1, h2, a1, a2 = 0, 1, 2, 3
    rp, col = csr_from_edges(4, [(h1, a1), (h1, a2), (h2, a2)])
    a, h = oracle.hits(rp, col, iters=50, norm=2)
    assert abs(a[a2] / a[a1] - PHI) < 1e-12
    assert abs(h[h1] / h[h2] - PHI) < 1e-12
    a1n, _ = oracle.hits(rp, col, iters=50, norm=1)
    assert abs(a1n[a2] / a1n[a1] - PHI) < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hits_dense_eigenvector(seed):
    n = 30
    rng = np.random.default_rng(seed)
    edges = [(u, v) for u in range(n) for v in range(n) if u != v and rng.random() < 0.15]
    rp, col = csr_from_edges(n, edges)
    A, _ = dense_M(n, edges)
    w, V = np.linalg.eigh(A.T @ A)
    assert w[-1] - w[-2] > 0.5  # well separated
    v = np.abs(V[:, -1])
    a, _ = oracle.hits(rp, col, iters=400, norm=2)
    np.testing.assert_allclose(a, v, atol=1e-10)
    # 50 Jacobi steps equal the same steps taken with dense products
    ad = np.full(n, 1 / n)
    hd = np.full(n, 1 / n)
    for _ in range(50):
        ad, hd = A.T @ hd, A @ ad
        ad, hd = ad / np.linalg.norm(ad), hd / np.linalg.norm(hd)
    a50, h50 = oracle.hits(rp, col, iters=50, norm=2)
    np.testing.assert_allclose(a50, ad, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(h50, hd, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("n,prob,seed", [(10, 0.25, 0), (45, 0.06, 1)])
def test_rwr_dense_solve(n, prob, seed):
    rng = np.random.default_rng(seed)
    edges = [(u, v) for u in range(n) for v in range(n) if u != v and rng.random() < prob]
    rp, col = csr_from_edges(n, edges)
    A, Md = dense_M(n, edges)
    D = (A.sum(axis=1) == 0).astype(float)
    for s in (0, n - 1):
        e = np.zeros(n)
        e[s] = 1
        K = Md + np.outer(e, D)
        r_star = (1 - C) * np.linalg.solve(np.eye(n) - C * K, e)
        r, _, l1 = oracle.rwr(rp, col, s, C, tol=1e-15)
        np.testing.assert_allclose(r, r_star, rtol=1e-11, atol=1e-15)
        assert abs(r.sum() - 1) < 1e-6


def test_rwr_reversibility_on_undirected_graph():
    n = 25
    rng = np.random.default_rng(3)
    und = set()
    for u in range(n):                      # a ring keeps it connected, no dangling
        und.add((u, (u + 1) % n))
    for _ in range(40):
        u, v = rng.integers(0, n, 2)
        if u != v:
            und.add((int(u), int(v)))
    edges = sorted(set(und) | {(v, u) for (u, v) in und})
    rp, col = csr_from_edges(n, edges)
    deg = np.diff(rp)
    R = np.stack([oracle.rwr(rp, col, s, C, tol=1e-15)[0] for s in range(n)])
    # R[s, t] = r_s(t); exact in real arithmetic, here up to the FP32 rounding
    # of the stored 1/deg values (relative 2^-24 each, amplified by <= 1/(1-c))
    lhs = deg[:, None] * R
    np.testing.assert_allclose(lhs, lhs.T, rtol=1e-6, atol=1e-14)
