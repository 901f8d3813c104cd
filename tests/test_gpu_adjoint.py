"""GPU parity of the differentiation workload: softmax edge weights written
into the packed layout, the weighted RWR fixed point, and the adjoint
gradient of L = -sum_t log r_t by transposed-SpMV iterations on the stored
transposed layout.  Checked against the FP64 oracle gradient (all edges,
relative L2 <= 1e-3) and FP64 central finite differences (h = 1e-3, 64
sampled edges, relative L2 <= 1e-3)."""
import numpy as np
import pytest
import torch

import graphgen
import oracle
import paper_1103_2405_gb300 as spg

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
C = 0.85


def _setup(scale, ef, ntargets, opts=None):
    rp, col = graphgen.rmat(scale, ef, seed=1)
    theta = graphgen.normal(int(rp[-1]), 7)
    s = graphgen.pick_source(rp, 3)
    t = graphgen.pick_targets(rp, col, s, ntargets, 5)
    f = spg.Format(rp, col, val=theta, kind="weighted", build_transpose=True, **(opts or {}))
    return rp, col, theta, s, t, f


def _gpu_grad(f, theta, s, t):
    th = torch.from_numpy(theta).to(DEV)
    f.set_edge_logits(th)
    r, info = f.rwr_weighted(s, restart=1 - C, tol=1e-10, max_iter=5000, like=th)
    g = torch.zeros_like(r)
    tt = torch.from_numpy(t.astype(np.int64)).to(DEV)
    g[tt] = -1.0 / r[tt]
    lam, dth, ainfo = f.rwr_adjoint(s, r, g, restart=1 - C, tol=1e-10, max_iter=5000)
    torch.cuda.synchronize()
    return r.cpu().numpy(), dth.cpu().numpy(), info, ainfo


@pytest.mark.parametrize("opts", [dict(), dict(tile_width=1024, heavy_row=32), dict(kernel=1)])
def test_weighted_rwr_and_gradient_vs_oracle(opts):
    rp, col, theta, s, t, f = _setup(11, 8, 30, opts)
    r, dth, info, ainfo = _gpu_grad(f, theta, s, t)
    loss, dth_ref, r_ref, _ = oracle.rwr_loss_grad(rp, col, theta, s, t, C)
    assert np.abs(r - r_ref).sum() <= 1e-6
    assert np.linalg.norm(dth - dth_ref) / np.linalg.norm(dth_ref) <= 1e-3
    assert ainfo["last_l1"] < 1e-10


def test_gradient_vs_central_differences():
    rp, col, theta, s, t, f = _setup(14, 8, 100)
    _, dth, _, _ = _gpu_grad(f, theta, s, t)
    edges = graphgen.pick_edges(int(rp[-1]), 64, 6)
    th64 = theta.astype(np.float64)
    h = 1e-3
    fd = np.empty(edges.size)
    for i, e in enumerate(edges):
        tp, tm = th64.copy(), th64.copy()
        tp[e] += h
        tm[e] -= h
        fd[i] = (_loss64(rp, col, tp, s, t) - _loss64(rp, col, tm, s, t)) / (2 * h)
    assert np.linalg.norm(dth[edges] - fd) <= 1e-3 * np.linalg.norm(fd)


def _loss64(rp, col, theta, s, t):
    P = np.zeros(theta.size)
    for u in range(rp.size - 1):
        b, e = rp[u], rp[u + 1]
        if b < e:
            z = theta[b:e] - theta[b:e].max()
            P[b:e] = np.exp(z) / np.exp(z).sum()
    r, _ = oracle.rwr_weighted(rp, col, P, s, C)
    return -np.sum(np.log(r[t]))


def test_autograd_function_and_logit_rewrite():
    rp, col, theta, s, t, f = _setup(12, 8, 40)
    th = torch.from_numpy(theta).to(DEV).requires_grad_(True)
    r = spg.RWRStationary.apply(th, f, s)
    loss = -torch.log(r[torch.from_numpy(t.astype(np.int64)).to(DEV)]).sum()
    loss.backward()
    loss_ref, dth_ref, _, _ = oracle.rwr_loss_grad(rp, col, theta, s, t, C)
    assert abs(loss.item() - loss_ref) <= 1e-4 * abs(loss_ref)
    g = th.grad.cpu().numpy()
    assert np.linalg.norm(g - dth_ref) / np.linalg.norm(dth_ref) <= 1e-3
    # new logits rewrite the packed weights in place
    theta2 = (theta * 0.5).astype(np.float32)
    f.set_edge_logits(torch.from_numpy(theta2).to(DEV))
    r2, _ = f.rwr_weighted(s, 1 - C, 1e-10, 5000, like=th)
    r2_ref, _ = oracle.rwr_weighted(rp, col, oracle.edge_softmax(rp, theta2), s, C)
    assert np.abs(r2.cpu().numpy() - r2_ref).sum() <= 1e-6
