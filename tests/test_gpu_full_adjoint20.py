"""Full-size parity of the differentiation workload: R-MAT scale 20
(1,048,576 nodes, edge factor 16), per-edge logits N(0,1) (seed 7),
softmax weights over each node's out-edges, RWR from the seeded source
(restart 0.15), loss = -sum over 1,000 seeded reachable targets of log r_t.
The GPU forward fixed point against the oracle's (L1 <= 1e-6) and the GPU
adjoint gradient against the FP64 oracle gradient over every edge (relative
L2 <= 1e-3)."""
import numpy as np
import pytest
import torch

import graphgen
import oracle
import paper_1103_2405_gb300 as spg

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
C = 0.85


def test_adjoint_gradient_scale20():
    rp, col = graphgen.rmat(20, 16, seed=1)
    theta = graphgen.normal(int(rp[-1]), 7)
    s = graphgen.pick_source(rp, 3)
    t = graphgen.pick_targets(rp, col, s, 1000, 5)
    f = spg.Format(rp, col, val=theta, kind="weighted", build_transpose=True)
    th = torch.from_numpy(theta).to(DEV)
    f.set_edge_logits(th)
    r, info = f.rwr_weighted(s, restart=1 - C, tol=1e-10, max_iter=5000, like=th)
    g = torch.zeros_like(r)
    tt = torch.from_numpy(t.astype(np.int64)).to(DEV)
    g[tt] = -1.0 / r[tt]
    lam, dth, ainfo = f.rwr_adjoint(s, r, g, restart=1 - C, tol=1e-10, max_iter=5000)
    torch.cuda.synchronize()
    r, dth = r.cpu().numpy().astype(np.float64), dth.cpu().numpy().astype(np.float64)
    loss, dth_ref, r_ref, _ = oracle.rwr_loss_grad(rp, col, theta, s, t, C)
    assert np.abs(r - r_ref).sum() <= 1e-6
    assert np.linalg.norm(dth - dth_ref) <= 1e-3 * np.linalg.norm(dth_ref)
