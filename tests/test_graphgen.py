"""Input generator checks: determinism across thread counts, R-MAT quadrant
statistics, Chung-Lu degree totals, dedup/self-loop removal against a set-based
brute force, and the range/moments of the random vectors."""
import numpy as np

import graphgen


def test_thread_count_independent():
    a = graphgen.rmat(12, 8, seed=3, nthreads=1)
    b = graphgen.rmat(12, 8, seed=3, nthreads=7)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = graphgen.chung_lu(5000, 40000, 2.1, 500, seed=2, nthreads=1)
    d = graphgen.chung_lu(5000, 40000, 2.1, 500, seed=2, nthreads=5)
    assert np.array_equal(c[0], d[0]) and np.array_equal(c[1], d[1])


def test_rmat_quadrant_frequencies():
    # top-level bit of (src, dst) follows (a, b, c, d)
    scale, m = 10, 400000
    src, dst = graphgen.rmat_edges(scale, m, seed=9)
    top = 1 << (scale - 1)
    s1, d1 = src >= top, dst >= top
    freq = [np.mean(~s1 & ~d1), np.mean(~s1 & d1), np.mean(s1 & ~d1), np.mean(s1 & d1)]
    np.testing.assert_allclose(freq, [0.57, 0.19, 0.19, 0.05], atol=4e-3)
    # every level follows the same law: popcount of src ~ Binomial(scale, 0.24)
    pc = np.array([bin(int(v)).count("1") for v in src[:20000]])
    assert abs(pc.mean() - scale * 0.24) < 0.05


def test_edges_to_csr_dedup_matches_sets():
    rng = np.random.default_rng(0)
    n, m = 300, 5000
    src = rng.integers(0, n, m).astype(np.uint32)
    dst = rng.integers(0, n, m).astype(np.uint32)
    rp, col = graphgen.edges_to_csr(n, src, dst, nthreads=3)
    expect = sorted({(int(u), int(v)) for u, v in zip(src, dst) if u != v})
    got = [(u, int(col[k])) for u in range(n) for k in range(rp[u], rp[u + 1])]
    assert got == expect
    perm = graphgen.random_permutation(n, 4)
    assert sorted(perm.tolist()) == list(range(n))
    rp2, col2 = graphgen.edges_to_csr(n, src, dst, relabel=perm)
    expect2 = sorted({(int(perm[u]), int(perm[v])) for u, v in expect})
    got2 = [(u, int(col2[k])) for u in range(n) for k in range(rp2[u], rp2[u + 1])]
    assert got2 == expect2


def test_chung_lu_weights_and_degrees():
    n, m = 20000, 200000
    w = graphgen.chung_lu_weights(n, m, 2.1, 800.0)
    assert abs(w.sum() - m) < 1e-6 * m
    assert w.max() <= 800.0 + 1e-9 and np.all(np.diff(w) <= 1e-12)
    rp, col = graphgen.chung_lu(n, m, 2.1, 800.0, seed=1, relabel=False)
    outdeg = np.diff(rp)
    # hubs keep most of their expected degree (dedup only trims them)
    assert 0.6 * w[0] < outdeg[0] <= w[0] * 1.2
    assert rp[-1] > 0.85 * m


def test_vectors():
    x = graphgen.uniform(100000, 2)
    assert x.dtype == np.float32 and x.min() >= 0 and x.max() < 1
    assert abs(x.mean() - 0.5) < 5e-3
    assert np.array_equal(x, graphgen.uniform(100000, 2))
    z = graphgen.normal(200000, 7)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1) < 1e-2


def test_seed_picks():
    rp, col = graphgen.rmat(12, 8, seed=1)
    s = graphgen.pick_source(rp, 3)
    d = np.diff(rp)
    assert d[s] >= np.sort(d)[::-1][len(d) // 100 - 1]
    seeds = graphgen.pick_seeds(rp, 64, 4)
    assert len(set(seeds.tolist())) == 64 and np.all(d[seeds] > 0)
    t = graphgen.pick_targets(rp, col, s, 100, 5)
    assert len(set(t.tolist())) == 100 and graphgen.reachable_from(rp, col, s)[t].all()


def test_unstructured_generators_closed_forms():
    rp, col, val = graphgen.dense_matrix(37)
    assert rp[-1] == 37 * 37 and np.array_equal(col[:37], np.arange(37))
    n, b = 1000, 7
    rp, col, val = graphgen.banded(n, b)
    assert rp[-1] == n * (2 * b + 1) - b * (b + 1)
    i = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(np.abs(col - i) <= b)
    nx, ny, nz = 5, 4, 3
    rp, col, val = graphgen.stencil_3d(nx, ny, nz)
    assert rp[-1] == (3 * nx - 2) * (3 * ny - 2) * (3 * nz - 2)
    assert np.all(np.diff(rp) <= 27) and np.diff(rp).max() == 27
    for r in range(nx * ny * nz):
        seg = col[rp[r]:rp[r + 1]]
        assert np.all(np.diff(seg) > 0) and r in seg
    assert val.dtype == np.float32 and np.all((val >= 0) & (val < 1))
