"""The boundary from C: a plain C99 program compiled with gcc against
include/spg.h and linked with libspg.so builds a host-only format of a small
graph, reads its summary, exports its entries and checks them against the
definition M[v][u] = 1/outdeg(u) (Eq. 6), and checks that malformed input is
refused with SPG_ERR_INVALID.  No GPU is touched (device = -1)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "spg.h"

/* 0->1, 0->2, 1->2, 2->0, 3->2 ; node 4 has no edges */
static const int64_t rp[6] = {0, 2, 3, 4, 5, 5};
static const int32_t col[5] = {1, 2, 2, 0, 2};

int main(void)
{
    spg_csr csr;
    spg_build_opts o;
    spg_handle h = NULL;
    spg_format_info_t info;
    int64_t rows[5];
    int32_t cols[5];
    float vals[5];
    int i, bad = 0;
    memset(&csr, 0, sizeof csr);
    memset(&o, 0, sizeof o);
    csr.n_rows = csr.n_cols = 5;
    csr.nnz = 5;
    csr.row_ptr = rp;
    csr.col = col;
    o.heavy_row = -1;
    o.layout_rule = 1;
    o.max_warps = 8;
    o.device = -1;
    if (spg_build_format(&csr, SPG_KIND_PAGERANK, &o, NULL, &h) != SPG_OK) {
        printf("build failed: %s\n", spg_last_error());
        return 1;
    }
    if (spg_format_info(h, &info) != SPG_OK) return 2;
    printf("n=%lld nnz=%lld zero_rows=%lld\n", (long long)info.n, (long long)info.nnz,
           (long long)info.zero_rows);
    if (spg_format_export_entries(h, rows, cols, vals) != SPG_OK) return 3;
    for (i = 0; i < 5; ++i) {
        /* entry (v, u) of M = W^T for the edge u -> v: value 1/outdeg(u) */
        int64_t u = cols[i], v = rows[i], k, found = 0, deg = rp[u + 1] - rp[u];
        for (k = rp[u]; k < rp[u + 1]; ++k) found |= col[k] == v;
        if (!found || vals[i] != 1.0f / (float)deg) bad = 1;
    }
    spg_destroy(h);
    /* a column index out of range must be refused */
    {
        int32_t badcol[5] = {1, 2, 2, 0, 9};
        spg_handle h2 = NULL;
        csr.col = badcol;
        if (spg_build_format(&csr, SPG_KIND_PAGERANK, &o, NULL, &h2) != SPG_ERR_INVALID) bad |= 2;
        if (h2) spg_destroy(h2);
    }
    printf("entries_ok=%d version=%s\n", bad == 0, spg_version());
    return bad;
}
"""


def test_c_program_builds_and_inspects_a_format():
    import __graft_entry__
    lib = __graft_entry__.build_library()
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    libdir = os.path.dirname(lib)
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "consumer.c")
        exe = os.path.join(d, "consumer")
        with open(src, "w") as fh:
            fh.write(PROGRAM)
        cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
               src, "-o", exe, "-L", libdir, "-l:" + os.path.basename(lib),
               "-Wl,-rpath," + libdir]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stdout + r.stderr
        assert "n=5 nnz=5 zero_rows=2" in r.stdout
        assert "entries_ok=1" in r.stdout
