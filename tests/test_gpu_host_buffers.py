"""Caller vectors in host memory: pinned (mapped) host buffers are read and
written by the permutation kernels straight over the host link, pageable
ones go through a staging copy.  Every path runs the same arithmetic, so the
results must equal the device-buffer results bit for bit; one case is also
checked against the oracle's fixed point."""
import numpy as np
import pytest
import torch

import graphgen
import oracle
import paper_1103_2405_gb300 as spg

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def graph():
    return graphgen.rmat(14, 8, seed=3)


def _host(t, pinned):
    h = t.cpu()
    return h.pin_memory() if pinned else h.numpy().copy()


@pytest.mark.parametrize("pattern", [False, True])
@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_spmv_host_vectors_equal_device_vectors(graph, pattern, beta):
    rp, col = graph
    n = rp.shape[0] - 1
    f = spg.Format(rp, col, kind="pagerank", pattern_only=pattern, tile_width=4096)
    g = torch.Generator().manual_seed(5)
    x = torch.rand(n, generator=g).to(DEV)
    y0 = torch.rand(n, generator=g).to(DEV)
    ref = f.spmv(x, y0.clone(), alpha=1.5, beta=beta).cpu()
    for pinned in (True, False):
        xh, yh = _host(x, pinned), _host(y0, pinned)
        out = f.spmv(xh, yh, alpha=1.5, beta=beta)
        got = out if isinstance(out, torch.Tensor) else torch.from_numpy(out)
        assert torch.equal(got, ref), pinned


def test_pagerank_host_buffers(graph):
    rp, col = graph
    n = rp.shape[0] - 1
    f = spg.Format(rp, col, kind="pagerank")
    p0 = torch.full((n,), 1.0 / n, device=DEV)
    ref, _ = f.pagerank(0.85, tol=0.0, max_iter=30, p0=p0, like=p0)
    ref = ref.cpu()
    for pinned in (True, False):
        out = torch.empty(n).pin_memory() if pinned else np.empty(n, np.float32)
        got, _ = f.pagerank(0.85, tol=0.0, max_iter=30, p0=_host(p0, pinned), out=out)
        got = got if isinstance(got, torch.Tensor) else torch.from_numpy(got)
        assert torch.equal(got, ref), pinned
    # and the converged vector through pinned buffers against the oracle
    out = torch.empty(n).pin_memory()
    p, _ = f.pagerank(0.85, tol=1e-8, max_iter=1000, p0=_host(p0, True), out=out)
    p_star, _, _ = oracle.pagerank(rp, col, 0.85, tol=1e-13)
    assert np.abs(p.numpy().astype(np.float64) - p_star).sum() <= 1e-6


def test_rwr_hits_batch_outputs_in_pinned_memory(graph):
    rp, col = graph
    n = rp.shape[0] - 1
    like = torch.empty(0, device=DEV)
    f = spg.Format(rp, col, kind="pagerank")
    s = int(graphgen.pick_source(rp, 3))
    ref, _ = f.rwr([s], 0.15, tol=0.0, max_iter=20, like=like)
    got, _ = f.rwr([s], 0.15, tol=0.0, max_iter=20, out=torch.empty(n).pin_memory())
    assert torch.equal(got, ref.cpu())
    seeds = graphgen.pick_seeds(rp, 3, 4)
    Rd, _ = f.rwr(seeds, 0.15, tol=0.0, max_iter=20, like=like)
    Rp, _ = f.rwr(seeds, 0.15, tol=0.0, max_iter=20, out=torch.empty(n, 3).pin_memory())
    Rn, _ = f.rwr(seeds, 0.15, tol=0.0, max_iter=20, out=np.empty((n, 3), np.float32))
    assert torch.equal(Rp, Rd.cpu()) and np.array_equal(Rn, Rd.cpu().numpy())
    fh = spg.Format(rp, col, kind="hits")
    a, h, _ = fh.hits(norm=2, iters=15, like=like)
    ap, hp, _ = fh.hits(norm=2, iters=15, auth=torch.empty(n).pin_memory(), hub=torch.empty(n).pin_memory())
    assert torch.equal(ap, a.cpu()) and torch.equal(hp, h.cpu())
    graphs = [graphgen.chung_lu(m, 12 * m, 2.3, m / 4, seed=9 + i) for i, m in enumerate((300, 1000, 77))]
    b = spg.BatchFormat(graphs)
    q, _ = b.pagerank(0.85, tol=0.0, max_iter=12, like=like)
    qp, _ = b.pagerank(0.85, tol=0.0, max_iter=12, out=torch.empty(b.n).pin_memory())
    assert torch.equal(qp, q.cpu())
