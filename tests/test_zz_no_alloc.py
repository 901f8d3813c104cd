"""spg_spmv_permuted_noalloc: the SpMV entry point for callers that must not
allocate device memory during a call (its scratch is a fixed array inside
the library).  Called through the C ABI, its output must match the
allocating entry point spg_spmv_permuted on the same format and input, on
two calls in a row (the shared array keeps the previous call's contents,
which the call must not depend on), and a format beyond the array's limits
must be refused with SPG_ERR_INVALID.

This file is collected last on purpose; it builds everything it uses, so it
also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

import graphgen
import paper_1103_2405_gb300 as spg

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _call_noalloc(f, xp, yp):
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    return spg.lib().spg_spmv_permuted_noalloc(f._h, ctypes.c_void_p(xp.data_ptr()),
                                               ctypes.c_void_p(yp.data_ptr()), stream)


def _close(y, ref):
    y, ref = y.double().cpu().numpy(), ref.double().cpu().numpy()
    assert np.linalg.norm(y - ref) <= 1e-5 * np.linalg.norm(ref)
    assert np.allclose(y, ref, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("opts", [dict(tile_width=2048, heavy_row=64), dict(x_stage_cols=-1),
                                  dict(tile_width=2048, heavy_row=64, kernel=1)])
def test_noalloc_matches_allocating_entry_point_twice(opts):
    rp, col = graphgen.rmat(14, 8, seed=1)
    f = spg.Format(rp, col, kind="pagerank", **opts)
    info = f.info()
    assert info["split_rows"] > 0
    n = f.n
    xp = torch.from_numpy(graphgen.uniform(n, 2)).to(DEV)
    ref = torch.empty(n, device=DEV)
    f.spmv_permuted(xp, ref)
    for _ in range(2):
        y = torch.full((n,), float("nan"), device=DEV)
        assert _call_noalloc(f, xp, y) == 0, spg.lib().spg_last_error()
        torch.cuda.synchronize()
        _close(y, ref)
    # a different input through the same (reused) scratch
    xp2 = torch.from_numpy(graphgen.uniform(n, 3)).to(DEV)
    ref2 = torch.empty(n, device=DEV)
    f.spmv_permuted(xp2, ref2)
    y2 = torch.empty(n, device=DEV)
    assert _call_noalloc(f, xp2, y2) == 0
    torch.cuda.synchronize()
    _close(y2, ref2)


def test_noalloc_refuses_formats_beyond_its_limits():
    # 70,000 rows with 33 entries each, cut at 32: 70,000 split rows > 65,536
    rows, deg = 70000, 33
    n = rows + deg
    src = np.repeat(np.arange(rows, rows + deg), rows)
    dst = np.tile(np.arange(rows), deg)
    rp, col = graphgen.edges_to_csr(n, src, dst)
    f = spg.Format(rp, col, kind="pagerank", heavy_row=32)
    assert f.info()["split_rows"] > 65536
    xp = torch.ones(f.n, device=DEV)
    yp = torch.empty(f.n, device=DEV)
    assert _call_noalloc(f, xp, yp) == -1
    assert b"split rows" in spg.lib().spg_last_error()


def test_noalloc_allocates_no_device_memory():
    # after a first call (which looks up the array's address and loads the
    # kernels), further calls leave the device's free memory unchanged
    rp, col = graphgen.rmat(14, 8, seed=1)
    f = spg.Format(rp, col, kind="pagerank", tile_width=2048, heavy_row=64)
    xp = torch.from_numpy(graphgen.uniform(f.n, 2)).to(DEV)
    y = torch.empty(f.n, device=DEV)
    assert _call_noalloc(f, xp, y) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(DEV)
    for _ in range(3):
        assert _call_noalloc(f, xp, y) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert free1 == free0


@pytest.mark.parametrize("kernel", [0, 1])
def test_noalloc_and_permuted_accept_an_unaligned_x_view(kernel):
    # x' as a slice one float into a buffer (4-byte aligned, not 16): the
    # shared-memory x slice must not use 16-byte loads there
    import oracle
    rp, col = graphgen.rmat(14, 8, seed=1)
    f = spg.Format(rp, col, kind="pagerank", tile_width=2048, kernel=kernel)
    n = f.n
    pi, inv = f.perm()
    x = graphgen.uniform(n, 2)
    big = torch.zeros(n + 1, device=DEV)
    big[1:] = torch.from_numpy(x[inv]).to(DEV)
    xp = big[1:]
    assert xp.data_ptr() % 16 != 0
    ref = oracle.spmv(oracle.build_M(rp, col), x)[inv]
    y1 = torch.empty(n, device=DEV)
    f.spmv_permuted(xp, y1)
    y2 = torch.empty(n, device=DEV)
    assert _call_noalloc(f, xp, y2) == 0
    torch.cuda.synchronize()
    for y in (y1, y2):
        y = y.double().cpu().numpy()
        assert np.linalg.norm(y - ref) <= 1e-5 * np.linalg.norm(ref)
