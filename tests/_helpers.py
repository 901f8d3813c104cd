"""Test-only helpers: dense brute-force matrices and tiny edge-list graphs."""
import numpy as np


def dense_M(n, edges):
    """Dense M = W^T from an edge list, FP32-rounded 1/outdeg values (test helper)."""
    A = np.zeros((n, n))
    for u, v in edges:
        A[u, v] = 1.0
    deg = A.sum(axis=1)
    W = np.zeros_like(A)
    for u in range(n):
        if deg[u] > 0:
            W[u] = A[u] * float(np.float32(1.0 / deg[u]))
    return A, W.T.copy()


def csr_from_edges(n, edges):
    """Adjacency CSR (rows = source, sorted, unique) from an edge list (test helper)."""
    adj = [sorted(set(v for (u, v) in edges if u == w and v != w)) for w in range(n)]
    rowptr = np.zeros(n + 1, np.int64)
    for u in range(n):
        rowptr[u + 1] = rowptr[u] + len(adj[u])
    col = np.array([v for u in range(n) for v in adj[u]], dtype=np.int32)
    return rowptr, col
