"""Pins of the oracle's PageRank (Appendix F, Eq. 6 + uniform dangling mass).

Closed forms: the directed n-cycle (uniform), the undirected star and the
in-star (leaves -> dangling centre), derived from the fixed-point equations;
the dense linear solve of the fixed point on random graphs; sum(p) = 1."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from _helpers import dense_M, csr_from_edges  # noqa: E402

import oracle  # noqa: E402

C = 0.85


def _tol(deg):
    # closed forms hold for exact 1/deg; the stored values are fl32(1/deg), so
    # when 1/deg is not a float32 the bound is that rounding (2^-24 relative)
    # amplified by at most 1/(1-c)
    return 1e-12 if float(np.float32(1.0 / deg)) == 1.0 / deg else 1e-6


def test_directed_cycle_is_uniform():
    n = 7
    rp, col = csr_from_edges(n, [(i, (i + 1) % n) for i in range(n)])
    p, it, _ = oracle.pagerank(rp, col, C, tol=1e-15)
    np.testing.assert_allclose(p, 1.0 / n, rtol=0, atol=1e-16)
    assert it == 1  # p(0) is already the fixed point


@pytest.mark.parametrize("n", [2, 5, 10, 33])
def test_undirected_star_centre(n):
    edges = [(0, i) for i in range(1, n)] + [(i, 0) for i in range(1, n)]
    rp, col = csr_from_edges(n, edges)
    p, _, _ = oracle.pagerank(rp, col, C, tol=1e-15)
    centre = (1 + C * (n - 1)) / (n * (1 + C))
    assert abs(p[0] - centre) < _tol(n - 1)
    np.testing.assert_allclose(p[1:], (1 - centre) / (n - 1), rtol=10 * _tol(n - 1))


@pytest.mark.parametrize("n", [2, 5, 10, 33])
def test_in_star_with_dangling_centre(n):
    edges = [(i, 0) for i in range(1, n)]
    rp, col = csr_from_edges(n, edges)
    p, _, _ = oracle.pagerank(rp, col, C, tol=1e-15)
    centre = (1 + C * (n - 1)) / (n + C * (n - 1))
    assert abs(p[0] - centre) < 1e-12
    np.testing.assert_allclose(p[1:], 1.0 / (n + C * (n - 1)), rtol=1e-11)


@pytest.mark.parametrize("n,prob,seed", [(12, 0.2, 0), (50, 0.05, 1), (90, 0.02, 2)])
def test_dense_fixed_point_solve(n, prob, seed):
    rng = np.random.default_rng(seed)
    edges = [(u, v) for u in range(n) for v in range(n) if u != v and rng.random() < prob]
    rp, col = csr_from_edges(n, edges)
    A, Md = dense_M(n, edges)
    dangling = (A.sum(axis=1) == 0).astype(float)
    # (I - c M - (c/n) 1 1_D^T) p = (1-c)/n 1
    K = np.eye(n) - C * Md - (C / n) * np.outer(np.ones(n), dangling)
    p_star = np.linalg.solve(K, np.full(n, (1 - C) / n))
    p, it, l1 = oracle.pagerank(rp, col, C, tol=1e-14)
    assert l1 < 1e-14
    np.testing.assert_allclose(p, p_star, rtol=1e-11, atol=1e-14)
    assert abs(p.sum() - 1.0) < 1e-6


def test_iteration_count_and_warm_start():
    n = 60
    rng = np.random.default_rng(5)
    edges = [(u, v) for u in range(n) for v in range(n) if u != v and rng.random() < 0.1]
    rp, col = csr_from_edges(n, edges)
    p, it, _ = oracle.pagerank(rp, col, C, tol=1e-8)
    # the error contracts by at most c per step
    assert it <= int(np.ceil(np.log(1e-8 / 2) / np.log(C))) + 1
    # warm start from the answer converges in one step
    p2, it2, _ = oracle.pagerank(rp, col, C, tol=1e-6, p_init=p)
    assert it2 == 1
    np.testing.assert_allclose(p2, p, atol=1e-7)


def test_iteration_is_an_l1_contraction_and_certifies_the_error():
    # G(p) = c M p + (c * sum_{u dangling} p_u + 1 - c)/n contracts L1
    # distances by c (M's non-dangling columns sum to 1, dangling mass is
    # spread): ||G p - G q||_1 <= c ||p - q||_1 for any p, q; hence for any
    # p, ||p - p*||_1 <= ||p - G^k p||_1 / (1 - c^k) (used to certify the
    # billion-edge GPU result without converging the oracle there)
    import graphgen
    rp, col = graphgen.rmat(11, 8, seed=3)
    n = rp.shape[0] - 1
    M = oracle.build_M(rp, col)
    c = 0.85
    rng = np.random.default_rng(0)
    c_eff = c * (1.0 + 2.0 ** -23)
    for _ in range(5):
        p = rng.random(n)
        q = rng.random(n) * rng.integers(0, 2, n)
        Gp, _, _ = oracle.pagerank(rp, col, c, tol=0.0, max_iter=1, p_init=p, M=M)
        Gq, _, _ = oracle.pagerank(rp, col, c, tol=0.0, max_iter=1, p_init=q, M=M)
        assert np.abs(Gp - Gq).sum() <= c_eff * np.abs(p - q).sum() * (1 + 1e-12)
    p_star, _, _ = oracle.pagerank(rp, col, c, tol=1e-14, M=M)
    for scale in (1e-3, 1e-6):
        p = p_star + scale * rng.standard_normal(n) / n
        for k in (1, 3, 6):
            qk, _, _ = oracle.pagerank(rp, col, c, tol=0.0, max_iter=k, p_init=p, M=M)
            cert = np.abs(p - qk).sum() / (1.0 - c_eff ** k)
            true = np.abs(p - p_star).sum()
            assert true <= cert * (1 + 1e-9)
            # and never loose by more than (1 + c^k) / (1 - c^k)
            assert cert <= (1.0 + c_eff ** k) / (1.0 - c_eff ** k) * true * (1 + 1e-9)
