"""Pins of the oracle's transform and SpMV (Appendix F Eq. 6; Appendix B).

The oracle's CSR pull product is checked against a dense matrix built
independently from the edge list (brute force), exhaustively over every
3-node digraph and on random graphs up to 64 nodes, and against the
column-sum invariant of a column-stochastic matrix."""
import itertools
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from _helpers import dense_M, csr_from_edges  # noqa: E402

import oracle  # noqa: E402


def _random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    return [(u, v) for u in range(n) for v in range(n) if u != v and rng.random() < p]


def test_all_3node_digraphs_match_dense():
    pairs = [(u, v) for u in range(3) for v in range(3) if u != v]
    x = np.array([0.3, -1.7, 2.25])
    for mask in range(1 << len(pairs)):
        edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        rp, col = csr_from_edges(3, edges)
        M = oracle.build_M(rp, col)
        _, Md = dense_M(3, edges)
        np.testing.assert_allclose(oracle.spmv(M, x), Md @ x, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("n,p,seed", [(2, 0.9, 0), (17, 0.2, 1), (40, 0.08, 2), (64, 0.05, 3)])
def test_random_graphs_match_dense(n, p, seed):
    edges = _random_graph(n, p, seed)
    rp, col = csr_from_edges(n, edges)
    M = oracle.build_M(rp, col)
    _, Md = dense_M(n, edges)
    x = np.random.default_rng(seed + 100).random(n)
    np.testing.assert_allclose(oracle.spmv(M, x), Md @ x, rtol=1e-13, atol=1e-15)
    # alpha / beta: y = a M x + b y
    y0 = np.random.default_rng(seed + 200).random(n)
    np.testing.assert_allclose(oracle.spmv(M, x, alpha=-0.5, beta=2.0, y=y0),
                               -0.5 * (Md @ x) + 2.0 * y0, rtol=1e-13, atol=1e-15)
    # beta = 0 never reads y (NaN must not propagate)
    assert np.all(np.isfinite(oracle.spmv(M, x, alpha=1.0, beta=0.0, y=np.full(n, np.nan))))
    rows = np.array([n - 1, 0, n // 2])
    np.testing.assert_allclose(oracle.spmv_rows(M, rows, x), (Md @ x)[rows], rtol=1e-13)


def test_transform_is_transposed_row_normalisation():
    # edge u->v lands in row v, column u, with value fl32(1/outdeg(u))
    edges = [(0, 1), (0, 2), (0, 3), (2, 1), (3, 0)]
    rp, col = csr_from_edges(4, edges)
    mrp, mcol, mval = oracle.build_M(rp, col)
    assert list(mrp) == [0, 1, 3, 4, 5]
    assert list(mcol) == [3, 0, 2, 0, 0]
    assert mval[0] == np.float32(1.0) and mval[1] == np.float32(1 / 3)
    assert mval[2] == np.float32(1.0) and mval[3] == np.float32(1 / 3)


def test_column_sums_invariant():
    # 1^T M x = sum over non-dangling u of x_u (each column of M sums to 1 up to
    # the FP32 rounding of 1/outdeg, |deg*fl32(1/deg) - 1| <= deg*2^-24)
    n = 300
    edges = _random_graph(n, 0.03, 7)
    rp, col = csr_from_edges(n, edges)
    M = oracle.build_M(rp, col)
    x = np.random.default_rng(8).random(n)
    deg = np.diff(rp)
    lhs = oracle.spmv(M, x).sum()
    rhs = x[deg > 0].sum()
    assert abs(lhs - rhs) <= 1e-6 * rhs


def test_ones_vector_gives_inverse_outdegree_sums():
    edges = [(0, 2), (1, 2), (1, 3), (3, 2), (2, 0)]
    rp, col = csr_from_edges(4, edges)
    y = oracle.spmv(oracle.build_M(rp, col), np.ones(4))
    # y_2 = 1/1 (from 0) + 1/2 (from 1) + 1/1 (from 3)
    np.testing.assert_allclose(y, [1.0, 0.0, 2.5, 0.5], rtol=1e-7)
