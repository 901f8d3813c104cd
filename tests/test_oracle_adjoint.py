"""Pins of the oracle's differentiable RWR: softmax edge weights, the weighted
RWR fixed point and the adjoint gradient of L = -sum_t log r_t.

The forward is checked against a dense linear solve; the gradient against a
dense adjoint with the softmax Jacobian written out, and against FP64 central
finite differences of the forward (h = 1e-3)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from _helpers import csr_from_edges  # noqa: E402

import oracle  # noqa: E402

C = 0.85


def _graph(n, prob, seed):
    rng = np.random.default_rng(seed)
    edges = [(u, v) for u in range(n) for v in range(n) if u != v and rng.random() < prob]
    return csr_from_edges(n, edges)


def _dense_K(rp, col, P, s):
    n = rp.shape[0] - 1
    K = np.zeros((n, n))
    for u in range(n):
        if rp[u] == rp[u + 1]:
            K[s, u] += 1.0
        for e in range(rp[u], rp[u + 1]):
            K[col[e], u] += P[e]
    return K


def test_softmax_rows_sum_to_one():
    rp, col = _graph(20, 0.2, 0)
    theta = np.random.default_rng(1).standard_normal(rp[-1]).astype(np.float32)
    P = oracle.edge_softmax(rp, theta)
    for u in range(20):
        if rp[u + 1] > rp[u]:
            seg = P[rp[u]:rp[u + 1]]
            assert abs(seg.sum() - 1) < 1e-14
            t = theta[rp[u]:rp[u + 1]].astype(np.float64)
            np.testing.assert_allclose(seg, np.exp(t) / np.exp(t).sum(), rtol=1e-13)


def test_weighted_rwr_dense_and_gradient():
    import graphgen
    n, s = 16, 3
    rp, col = _graph(n, 0.2, 2)
    theta = np.random.default_rng(3).standard_normal(rp[-1]).astype(np.float32)
    reach = np.flatnonzero(graphgen.reachable_from(rp, col, s))
    targets = reach[[0, 2, len(reach) // 2, -1]]
    loss, grad, r, lam = oracle.rwr_loss_grad(rp, col, theta, s, targets, C)
    P = oracle.edge_softmax(rp, theta)
    K = _dense_K(rp, col, P, s)
    e = np.zeros(n)
    e[s] = 1
    r_star = (1 - C) * np.linalg.solve(np.eye(n) - C * K, e)
    np.testing.assert_allclose(r, r_star, rtol=1e-12, atol=1e-15)
    # dense adjoint: lambda = (I - c K^T)^-1 g, dL/dP_e = c lambda_v r_u,
    # then the softmax Jacobian diag(P) - P P^T per source node
    g = np.zeros(n)
    g[targets] = -1.0 / r_star[targets]
    lam_star = np.linalg.solve(np.eye(n) - C * K.T, g)
    np.testing.assert_allclose(lam, lam_star, rtol=1e-10, atol=1e-12)
    gP = np.array([C * lam_star[col[e]] * r_star[u] for u in range(n)
                   for e in range(rp[u], rp[u + 1])])
    expect = np.zeros(rp[-1])
    for u in range(n):
        b, e1 = rp[u], rp[u + 1]
        if b == e1:
            continue
        p = P[b:e1]
        J = np.diag(p) - np.outer(p, p)
        expect[b:e1] = J @ gP[b:e1]
    np.testing.assert_allclose(grad, expect, rtol=1e-9, atol=1e-12)


def test_gradient_matches_central_differences():
    import graphgen
    n, s = 24, 0
    rp, col = _graph(n, 0.15, 4)
    theta = np.random.default_rng(5).standard_normal(rp[-1]).astype(np.float32).astype(np.float64)
    reach = np.flatnonzero(graphgen.reachable_from(rp, col, s))
    targets = reach[[1, len(reach) // 3, len(reach) // 2, -1]]
    assert len(reach) > 8
    _, grad, _, _ = oracle.rwr_loss_grad(rp, col, theta, s, targets, C)
    h = 1e-3
    fd = np.zeros(rp[-1])
    for e in range(rp[-1]):
        tp = theta.copy()
        tm = theta.copy()
        tp[e] += h
        tm[e] -= h
        lp = _loss64(rp, col, tp, s, targets)
        lm = _loss64(rp, col, tm, s, targets)
        fd[e] = (lp - lm) / (2 * h)
    assert np.linalg.norm(grad - fd) <= 1e-5 * np.linalg.norm(fd)


def _loss64(rp, col, theta, s, targets):
    # FP64 logits (finite differences of an FP32-rounded logit would be noise)
    n = rp.shape[0] - 1
    P = np.zeros(rp[-1])
    for u in range(n):
        b, e1 = rp[u], rp[u + 1]
        if b < e1:
            t = theta[b:e1] - theta[b:e1].max()
            P[b:e1] = np.exp(t) / np.exp(t).sum()
    r, _ = oracle.rwr_weighted(rp, col, P, s, C)
    return -np.sum(np.log(r[targets]))
