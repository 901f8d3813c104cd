// format.h -- host-side description of a built tiled composite layout.
#pragma once
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "spg_internal.h"

namespace spg {

// Performance lookup table of Section 3.3: slots/s for (major, log2 w_pad,
// log2 h_pad) buckets, each log clamped to [0, kTableLog).
constexpr int kTableLog = 21;
struct PerfTable {
    double perf[2][kTableLog][kTableLog];
    bool loaded = false;
};
PerfTable &perf_table();                // process-wide table
void perf_table_default(PerfTable &t);  // built-in analytic table
bool perf_table_load(const char *path, PerfTable &t, std::string &err);
double perf_lookup(const PerfTable &t, int major, int64_t wpad, int64_t hpad);

// Storage rule value that lets the Algorithm 3 model choose rule 0-3 per part.
constexpr int kAutoRule = 4;

struct BuildParams {
    int64_t tile_width = 0;   // resolved (> 0) or <= 0 for none
    int64_t wl = 0;
    int64_t heavy = -1;
    int layout_rule = 1;      // 0-3, or kAutoRule (chosen per part by the model)
    int64_t max_warps = 9728;
    int64_t max_rows = 0;     // > 0: at most this many rows per workload
    double split_cost = 2e-7;
    bool keep_plan = false;
    bool track_edges = false;
    // store column indices only (every column's entries share one value,
    // kept per column in inv_deg): 4 bytes per slot instead of 8
    bool pattern_only = false;
    // block-diagonal union of independent graphs: node segments
    // [seg_off[g], seg_off[g+1]); the degree order is taken within each segment
    const int64_t *seg_off = nullptr;
    int64_t nseg = 0;
    // columns of the shared-memory x slice the kernel would stage per part
    // (for PartHost::slice_share; 0 = none)
    int64_t stage_cols = 0;
    // block-diagonal unions (nseg > 0) of one part: store (and claim) the
    // part's workloads segment by segment, claim units within a segment
    bool segment_order = false;
    // claim units of the persistent kernels: consecutive workloads grouped
    // until their cost (padded slots + 4 per row) reaches this; <= 1 = one
    // workload per unit
    int64_t unit_slots = 0;
    // 0: workloads of a part stored (and claimed) longest first by
    // latency_rounds(); 1: in the ranking order
    int claim_order = 0;
    // also store every part as a row-sorted COO list (the TILE-COO format,
    // the ablation of the composite storage)
    bool build_coo = false;
};

// Dependent global-memory round trips of the warp that computes workload d
// in the SpMV kernels' loops: descriptor and row operands, then per
// 32-row block of a column-major workload two trips (slots, then gathers)
// per batch of 8 columns (4 when two blocks run together), per row of a
// row-major workload one trip per 4 pipelined 32-slot steps plus two for
// the rest; a row-free workload two trips per 128 rows.
double latency_rounds(const Workload &d);

struct PartHost {
    int64_t c0 = 0, c1 = 0;
    int64_t heavy = 0, wl = 0, nnz = 0, nvirt = 0;
    int32_t rule = 1;         // storage rule the part was built with (0-3)
    // share of the part's entries (all rows) in its first stage_cols columns:
    // what a shared-memory x slice of that many columns would serve
    double slice_share = 0.0;
    int64_t nwl = 0;          // regular workloads
    int64_t nwl_total = 0;    // + zero-row workloads
    int64_t unit_off = 0, nunits = 0;   // claim units: units[unit_off .. unit_off + nunits] (+ end)
    int64_t wl_off = 0;       // first workload in the concatenated array
    int32_t nblocks = 0, red_base = 0;
    double predicted_s = 0;
    // plan (keep_plan)
    std::vector<int32_t> rank_row, rank_chunk, rank_len;
    std::vector<int64_t> wl_first;
    std::vector<int32_t> wl_h, wl_w, wl_major;
};

struct Layout {
    int64_t n = 0, nnz = 0;
    int64_t tile_width = 0, ntile = 0;
    int64_t max_warps = 0;
    int64_t padded_slots = 0;
    int64_t nsplit = 0, nchunk_slots = 0, nred = 0;
    int64_t dangling_start = 0;
    std::vector<int32_t> perm, inv;
    std::vector<int64_t> seg_dstart;    // per segment: first position of its dangling tail
    std::vector<PartHost> parts;
    std::vector<int64_t> zero_rows;
    // packed arrays (host copy; released after upload unless kept)
    std::vector<Workload> wl;
    std::vector<int32_t> units;         // per part: first workload of each claim unit, then the end
    std::vector<uint32_t> rows;
    std::vector<uint2> slab;
    std::vector<uint32_t> slab4;        // pattern-only slots
    std::vector<float> inv_deg;         // pattern-only: column value, permuted order
    bool pattern = false;
    std::vector<SplitRow> split;
    std::vector<int32_t> slot_owner;
    std::vector<int64_t> edge_slot;     // edge id -> slab slot (track_edges)
    // TILE-COO (build_coo): part p's entries are [coo_off[p], coo_off[p+1])
    // of (row, column, value), sorted by row, then column
    std::vector<int64_t> coo_off;
    std::vector<int32_t> coo_row, coo_col;
    std::vector<float> coo_val;
    // device copies
    int32_t *d_perm = nullptr, *d_inv = nullptr;
    Workload *d_wl = nullptr;
    int32_t *d_units = nullptr;
    uint32_t *d_rows = nullptr;
    uint2 *d_slab = nullptr;
    uint32_t *d_slab4 = nullptr;
    float *d_inv_deg = nullptr;
    SplitRow *d_split = nullptr;
    int32_t *d_slot_owner = nullptr;
    float *d_partial = nullptr;
    uint32_t *d_counter = nullptr;
    int64_t *d_edge_slot = nullptr;
    int32_t *d_coo_row = nullptr, *d_coo_col = nullptr;
    float *d_coo_val = nullptr;
    int64_t device_bytes = 0;
    bool on_device = false;

    std::vector<PartView> part_views() const;
    SplitView split_view() const;
    void free_device();
};

// X given column by column (CSC of the matrix to format): column j holds
// entries (rowidx[k], val[k]) for k in [colptr[j], colptr[j+1]); eid[k] (or k
// when eid is null) names the entry for the edge map.  row_class (nullable)
// marks rows of the second HITS half.
struct ColumnSource {
    int64_t n = 0;
    const int64_t *colptr = nullptr;
    const int32_t *rowidx = nullptr;
    const float *val = nullptr;
    const int64_t *eid = nullptr;
    const uint8_t *row_class = nullptr;
    // rows to hold (by original row id, nullable = all): one rank's share of
    // a row partition; the column order is still that of the whole matrix
    const uint8_t *row_keep = nullptr;
};

// Host builder: order, tile, rank, tune, pack.  Fills `out` (host arrays).
bool build_layout(const ColumnSource &src, const BuildParams &prm, Layout &out,
                  std::string &err);
// Upload the packed arrays; release host copies unless keep_host.
cudaError_t upload_layout(Layout &L, bool keep_host, cudaStream_t stream);

// Algorithm 3 model (seconds) of one ranked part; Algorithm 2 search.
double model_time(const int32_t *vlen, int64_t nv, int64_t WL, int64_t max_warps, int rule,
                  int64_t max_rows, const PerfTable &t);
int64_t alg2_search(const int32_t *vlen, int64_t nv, int64_t nnz, int64_t max_warps,
                    int rule, int64_t max_rows, const PerfTable &t, double *best);

int hw_threads();

// Run fn(lo, hi) over [0, n) split into contiguous chunks on hw_threads()
// threads (serially below `grain` items).
template <class F> void parallel_for(int64_t n, int64_t grain, F fn)
{
    int nt = hw_threads();
    if (n <= grain || nt <= 1) { if (n > 0) fn((int64_t)0, n); return; }
    int64_t chunks = std::min<int64_t>(nt, (n + grain - 1) / grain);
    std::vector<std::thread> th;
    th.reserve((size_t)chunks);
    for (int64_t t = 1; t < chunks; ++t)
        th.emplace_back([=] { fn(n * t / chunks, n * (t + 1) / chunks); });
    fn((int64_t)0, n / chunks);
    for (auto &x : th) x.join();
}

// Dynamic version: items handed out in blocks of `block` (uneven work).
template <class F> void parallel_dynamic(int64_t n, int64_t block, F fn)
{
    int nt = hw_threads();
    if (n <= block || nt <= 1) { if (n > 0) fn((int64_t)0, n); return; }
    std::atomic<int64_t> next{0};
    auto worker = [&] {
        for (;;) {
            int64_t lo = next.fetch_add(block);
            if (lo >= n) break;
            fn(lo, std::min(n, lo + block));
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(worker);
    worker();
    for (auto &x : th) x.join();
}

}  // namespace spg
