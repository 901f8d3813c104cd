"""Offline shape benchmark: measure the performance lookup table of the
Section 3.3 model on the current GPU and write it as a text table.

For every workload shape (storage major, padded width w, padded height h)
the benchmark builds a synthetic matrix in which every workload has exactly
that shape -- rows of length w, workload size w*h, at most h rows per
workload, no row splitting -- with random columns over 4M columns (a 16 MB x,
like the R-MAT scale-22 workload), times the tiled-composite SpMV kernel
alone (CUDA events, `spg_time_parts`), and records stored slots per second.
Missing buckets are filled by the loader from the nearest measured one.

Usage:  python -m paper_1103_2405_gb300.tune_table [out.txt]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

N_COLS = 1 << 22
TARGET_NNZ = 1 << 24
MAX_NNZ = 1 << 27
MAX_WL = 1 << 15          # the paper's bound on the workload size of the table


def shapes():
    """(major, w, h) of the shapes the builder produces: row-major rows of
    w (multiple of 32) slots, up to 32 rows; column-major 32- or 64-row
    blocks of short rows."""
    out = []
    for lw in range(5, 14):
        for lh in range(0, 6):
            if (1 << (lw + lh)) <= MAX_WL:
                out.append((0, 1 << lw, 1 << lh))
    for lw in range(0, 5):
        for lh in (5, 6):
            out.append((1, 1 << lw, 1 << lh))
    return out


def shape_matrix(w, h, rng, max_warps):
    """Enough workloads of the shape to fill the GPU twice over (at
    least TARGET_NNZ slots, at most MAX_NNZ): R rows of exactly w entries
    with random columns over N_COLS (or R) columns, any other rows empty."""
    slots = min(MAX_NNZ, max(TARGET_NNZ, 2 * max_warps * w * h))
    rows = max(h, slots // w)
    rows -= rows % h
    n = max(N_COLS, rows)
    cols = rng.integers(0, n, size=(rows, w), dtype=np.int64)
    cols.sort(axis=1)
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:rows + 1] = np.arange(1, rows + 1) * w
    rowptr[rows + 1:] = rows * w
    vals = rng.random(rows * w, dtype=np.float32)
    return rowptr, cols.reshape(-1).astype(np.int32), vals, rows


def measure(out_path, reps=20, seed=0):
    import torch
    import paper_1103_2405_gb300 as spg
    rng = np.random.default_rng(seed)
    # time of the empty rows alone (every shape matrix pads to N_COLS rows
    # with empty ones, which the kernel still writes): subtracted pro rata
    empty = spg.Format(np.zeros(N_COLS + 1, np.int64), np.zeros(0, np.int32),
                       np.zeros(0, np.float32), kind="matrix", tile_width=-1)
    t_empty = float(empty.time_parts(mode=0, reps=reps).sum())
    del empty
    lines = ["# spg performance table: major log2(w_pad) log2(h_pad) slots_per_second",
             f"# measured {time.strftime('%Y-%m-%d %H:%M:%S')} on {torch.cuda.get_device_name(0)}"]
    max_warps = torch.cuda.get_device_properties(0).multi_processor_count * 32
    for major, w, h in shapes():
        rowptr, col, val, rows = shape_matrix(w, h, rng, max_warps)
        n = rowptr.shape[0] - 1
        f = spg.Format(rowptr, col, val, kind="matrix", tile_width=-1, wl=w * h, max_rows=h,
                       heavy_row=0, layout_rule=0, table=None)
        ms = float(f.time_parts(mode=0, reps=reps).sum())
        ms_work = max(ms - t_empty * (n - rows) / N_COLS, 0.05 * ms)
        slots = rows * w
        perf = slots / (ms_work * 1e-3)
        lines.append(f"{major} {int(np.log2(w))} {int(np.log2(h))} {perf:.6e}")
        print(lines[-1], f"# rows={rows} ms={ms:.4f} empty_ms={t_empty:.4f}", flush=True)
        del f
    with open(out_path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    return out_path


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(here, "perf_table_gb300.txt")
    print(measure(out))
