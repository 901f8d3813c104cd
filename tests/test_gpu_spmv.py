"""GPU parity of the tiled composite SpMV/SpMM against the FP64 oracle.

Seeded R-MAT graphs shaped like the paper's power-law inputs, built under
several tile widths (one part, several dense tiles with a ragged sparse
tail), heavy-row thresholds (split rows on and off) and both storage rules,
plus degenerate graphs.  Tolerance: relative L2 <= 1e-5 per SpMV (the
target), and element-wise |y - y*| <= 1e-5 * (|M| |x|)_v + 1e-30, the FP32
accumulation bound for rows of <= ~10^5 terms."""
import numpy as np
import pytest
import torch

import graphgen
import oracle
import paper_1103_2405_gb300 as spg

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _graph(kind):
    if kind == "rmat14":
        return graphgen.rmat(14, 8, seed=1)
    if kind == "rmat12":
        return graphgen.rmat(12, 16, seed=5)
    if kind == "hub":       # one row of 20000 entries (in-star) + a ring
        n = 20001
        src = np.concatenate([np.arange(1, n), np.arange(n)])
        dst = np.concatenate([np.zeros(n - 1, np.int64), (np.arange(n) + 1) % n])
        return graphgen.edges_to_csr(n, src, dst)
    if kind == "empty":
        return np.zeros(101, np.int64), np.zeros(0, np.int32)
    if kind == "single":
        return np.zeros(2, np.int64), np.zeros(0, np.int32)
    if kind == "varied":    # 2048 nodes, in-degrees spread over 0..1500: rows of every length
        rng = np.random.default_rng(11)
        n = 2048
        deg = rng.integers(0, 1501, size=n)
        dst = np.repeat(np.arange(n), deg)
        src = rng.integers(0, n, size=dst.shape[0])
        return graphgen.edges_to_csr(n, src, dst)
    if kind == "dense":     # dense 300 x 300 (every off-diagonal edge)
        n = 300
        u, v = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        m = u != v
        return graphgen.edges_to_csr(n, u[m], v[m])
    raise ValueError(kind)


def _check(y, yref, M, x, tol=1e-5):
    y = y.detach().cpu().numpy().astype(np.float64) if torch.is_tensor(y) else np.asarray(y, np.float64)
    nrm = np.linalg.norm(yref)
    if nrm > 0:
        assert np.linalg.norm(y - yref) / nrm <= tol
    bound = oracle.spmv((M[0], M[1], np.abs(M[2])), np.abs(np.asarray(x, np.float64)))
    assert np.all(np.abs(y - yref) <= tol * bound + 1e-30)


CONFIGS = [
    ("rmat14", dict()),                                        # auto: one composite part
    ("rmat14", dict(pattern_only=True, tile_width=2048)),      # 4-byte slots, values folded into x
    ("hub", dict(pattern_only=True)),
    ("rmat14", dict(kernel=2)),                                # plain 8-warp kernel
    ("rmat14", dict(kernel=3, tile_width=2048)),               # TMA ring kernel
    ("rmat14", dict(kernel=1)),                                # staged x-slice kernel
    ("rmat14", dict(kernel=4)),                                # slice-free persistent kernel
    ("rmat14", dict(layout_rule=4, tile_width=2048)),          # storage rule chosen by the model
    ("varied", dict(x_stage_cols=512, tile_width=1024)),       # slice on some parts only
    ("rmat14", dict(kernel=1, tile_width=2048, pattern_only=True)),
    ("varied", dict(kernel=1)),
    ("varied", dict(kernel=1, heavy_row=256, max_rows=-1)),
    ("varied", dict(kernel=1, pattern_only=True, max_rows=100)),
    ("varied", dict()),
    ("hub", dict(kernel=1)),
    ("rmat14", dict(tile_width=2048)),                         # dense tiles + sparse tail
    ("rmat14", dict(tile_width=256, heavy_row=0)),             # no split rows
    ("rmat14", dict(tile_width=4096, heavy_row=32, layout_rule=0)),
    ("rmat14", dict(tile_width=2048, layout_rule=2)),           # all CSR-vector
    ("rmat14", dict(layout_rule=3)),                            # all ELL
    ("rmat12", dict(tile_width=100, wl=96)),                   # ragged tile width, fixed WL
    ("hub", dict()),                                           # split hub row
    ("hub", dict(heavy_row=0)),                                # one warp for the hub row
    ("dense", dict(tile_width=64)),
    ("empty", dict()),
    ("single", dict()),
]


@pytest.mark.parametrize("gkind,opts", CONFIGS)
def test_spmv_matches_oracle(gkind, opts):
    rp, col = _graph(gkind)
    n = rp.shape[0] - 1
    M = oracle.build_M(rp, col)
    f = spg.Format(rp, col, kind="pagerank", **opts)
    x = graphgen.uniform(n, 2)
    xt = torch.from_numpy(x).to(DEV)
    y = f.spmv(xt)
    torch.cuda.synchronize()
    _check(y, oracle.spmv(M, x), M, x)
    # alpha / beta (BLAS semantics; beta = 0 never reads y)
    y0 = graphgen.uniform(n, 9) - 0.5
    yt = torch.from_numpy(y0).to(DEV)
    f.spmv(xt, yt, alpha=0.5, beta=-2.0)
    yref = oracle.spmv(M, x, alpha=0.5, beta=-2.0, y=y0)
    assert np.allclose(yt.cpu().numpy(), yref, rtol=1e-5, atol=1e-6)
    ynan = torch.full((n,), float("nan"), device=DEV)
    f.spmv(xt, ynan, alpha=1.0, beta=0.0)
    assert torch.isfinite(ynan).all()


def test_spmv_host_pointers_and_permuted_entry():
    rp, col = _graph("rmat14")
    n = rp.shape[0] - 1
    M = oracle.build_M(rp, col)
    f = spg.Format(rp, col, kind="pagerank", tile_width=1024)
    x = graphgen.uniform(n, 2)
    y = np.zeros(n, np.float32)
    f.spmv(x, y)                       # numpy in, numpy out (staged by the library)
    _check(y, oracle.spmv(M, x), M, x)
    pi, inv = f.perm()
    xp = torch.from_numpy(x[inv]).to(DEV)
    yp = torch.empty(n, device=DEV)
    f.spmv_permuted(xp, yp)
    torch.cuda.synchronize()
    assert np.array_equal(yp.cpu().numpy()[pi], y)


@pytest.mark.parametrize("gkind,opts", [("rmat14", dict()), ("rmat14", dict(tile_width=2048)),
                                         ("rmat12", dict(tile_width=100)), ("hub", dict()),
                                         ("varied", dict(tile_width=512)), ("dense", dict(tile_width=64)),
                                         ("empty", dict()), ("single", dict())])
def test_tile_coo_spmv_matches_oracle(gkind, opts):
    # the TILE-COO ablation (Section 5): same degree order and tiles, COO
    # storage, segmented warp sums with atomics at interval edges
    rp, col = _graph(gkind)
    n = rp.shape[0] - 1
    M = oracle.build_M(rp, col)
    f = spg.Format(rp, col, kind="pagerank", tile_coo=True, **opts)
    x = graphgen.uniform(n, 2)
    pi, inv = f.perm()
    xp = torch.from_numpy(x[inv]).to(DEV)
    yp = torch.full((n,), float("nan"), device=DEV)     # zeroed by the call
    f.spmv_tile_coo(xp, yp)
    torch.cuda.synchronize()
    _check(yp.cpu().numpy()[pi], oracle.spmv(M, x), M, x)


def test_tile_coo_needs_the_option():
    rp, col = _graph("rmat12")
    n = rp.shape[0] - 1
    f = spg.Format(rp, col, kind="pagerank")
    xp = torch.zeros(n, device=DEV)
    with pytest.raises(spg.SpgError):
        f.spmv_tile_coo(xp, torch.empty(n, device=DEV))


def test_spmv_deterministic():
    rp, col = _graph("hub")
    f = spg.Format(rp, col, kind="pagerank", heavy_row=64)
    assert f.info()["split_rows"] >= 1
    x = torch.from_numpy(graphgen.uniform(rp.shape[0] - 1, 3)).to(DEV)
    a = f.spmv(x).clone()
    b = f.spmv(x)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("which", [spg.CSR_SCALAR, spg.CSR_VECTOR])
def test_baselines_match_oracle(which):
    rp, col = _graph("rmat14")
    n = rp.shape[0] - 1
    M = oracle.build_M(rp, col)
    f = spg.Format(rp, col, kind="pagerank", keep_csr=True)
    x = graphgen.uniform(n, 2)
    y = f.baseline_spmv(which, torch.from_numpy(x).to(DEV))
    torch.cuda.synchronize()
    _check(y, oracle.spmv(M, x), M, x)


@pytest.mark.parametrize("k,opts", [(64, dict(tile_width=2048)), (3, dict()), (130, dict(heavy_row=64)),
                                    (64, dict(vec_width=64)), (128, dict(heavy_row=64, tile_width=2048)),
                                    (192, dict())])
def test_spmm_matches_oracle(k, opts):
    rp, col = _graph("rmat12")
    n = rp.shape[0] - 1
    M = oracle.build_M(rp, col)
    f = spg.Format(rp, col, kind="pagerank", **opts)
    X = np.stack([graphgen.uniform(n, 20 + j) for j in range(k)], axis=1).astype(np.float32)
    Y = f.spmm(torch.from_numpy(X).to(DEV))
    torch.cuda.synchronize()
    Y = Y.cpu().numpy()
    for j in range(k):
        _check(Y[:, j], oracle.spmv(M, X[:, j]), M, X[:, j])
