"""GPU parity of the tiled composite SpMV on the non-power-law sanity
matrices (the paper's dense 2K x 2K case, banded and finite-element-like
27-point stencil patterns) against the FP64 oracle, relative L2 <= 1e-5 and
the element-wise FP32 accumulation bound."""
import numpy as np
import pytest
import torch

import graphgen
import oracle
import paper_1103_2405_gb300 as spg

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _mat(kind):
    if kind == "dense2k":
        return graphgen.dense_matrix(2048)
    if kind == "banded":
        return graphgen.banded(200_000, 8)
    if kind == "stencil":
        return graphgen.stencil_3d(64, 64, 48)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["dense2k", "banded", "stencil"])
@pytest.mark.parametrize("opts", [dict(), dict(kernel=2), dict(tile_width="n/8")])
def test_unstructured_spmv(kind, opts):
    rp, col, val = _mat(kind)
    n = rp.shape[0] - 1
    if opts.get("tile_width") == "n/8":   # several dense tiles (at most 126 parts)
        opts = dict(tile_width=max(256, 1 << int(np.log2(n / 8))))
    f = spg.Format(rp, col, val, kind="matrix", **opts)
    x = graphgen.uniform(n, 2)
    y = f.spmv(torch.from_numpy(x).to(DEV))
    torch.cuda.synchronize()
    y = y.cpu().numpy().astype(np.float64)
    ref = oracle.spmv((rp, col, val), x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-5
    assert np.all(np.abs(y - ref) <= 1e-5 * ref + 1e-30)     # all terms >= 0: |M||x| = M x
