// spg_internal.h -- layout of the tiled composite format shared by the host
// builder (builder.cpp), the kernels (kernels.cu) and the C ABI (capi.cu).
//
// Device layout of one format (all arrays in HBM, allocated once at build):
//   perm[n] / inv[n]   int32  symmetric order by decreasing column length
//                             (Section 3.1, Solution 2): perm[orig] = pos.
//   parts              ntile dense column tiles (Algorithm 1) + the sparse
//                      remainder, launched in order (Solution 1).
//   workloads[]        24-byte descriptors, one warp each (Solution 3).
//   rows[]             int32 row entry per (virtual) row of a workload:
//                      permuted row id | flag bits below.
//   slab[]             uint2 {col, float bits} slots; padding has col = -1.
//                      Row-major workload: row r at slab + r*w (w padded to
//                      32).  Column-major: 32-row blocks, slot of (row r,
//                      entry k) = slab + (r/32)*32*w + k*32 + r%32.
//   split tables       chunks of rows longer than the heavy threshold.
#pragma once
#include <cstdint>

namespace spg {

constexpr int kWarp = 32;
constexpr int kWarpsPerBlock = 8;          // 256-thread blocks
constexpr int kBlock = kWarp * kWarpsPerBlock;
constexpr int kZeroRowsPerWorkload = 1024; // rows of a w = 0 workload

// Flag bits of a row entry.
constexpr uint32_t kRowSplit = 0x80000000u;    // low 31 bits: chunk slot of a split row
constexpr uint32_t kRowNotFirst = 0x40000000u; // the row has entries in an earlier part
constexpr uint32_t kRowNotLast = 0x20000000u;  // the row has entries in a later part
constexpr uint32_t kRowClass = 0x10000000u;    // HITS: the row is in the hub half
constexpr uint32_t kRowIdMask = 0x0fffffffu;   // n < 2^28
constexpr int64_t kMaxN = (int64_t)1 << 28;

struct Workload {        // 24 bytes, one warp
    int64_t slab;        // first slot
    int32_t rows;        // first row entry
    int32_t w;           // row-major: padded width; column-major: width
    int32_t h;           // rows (unpadded)
    int32_t major;       // 0 row-major (CSR-vector), 1 column-major (ELL)
};
static_assert(sizeof(Workload) == 24, "Workload layout");

struct SplitRow {        // one row cut into nchunks chunks (consecutive slots)
    uint32_t row;        // permuted row id | kRowNotFirst/NotLast/Class flags
    int32_t first_slot;
    int32_t nchunks;
    int32_t red_slot;    // index of this split row (its reduction slot after the blocks')
};

// Per-part device view handed to the kernels.
struct PartView {
    const Workload *wl;
    const uint32_t *rows;
    const uint2 *slab;
    const uint32_t *slab4;   // pattern-only layout: column index per slot (value implied)
    uint32_t *sched;      // staged kernel: {next workload, warps done}, zero between launches
    uint32_t *status;     // TMA kernel: set non-zero when a bounded wait ran out
    int32_t nwl;          // workloads incl. zero-row ones
    int32_t nblocks;      // launch blocks
    int32_t red_base;     // first reduction slot of this part's blocks
    int32_t c0;           // first column of the part
    int32_t xs_cols;      // > 0: columns [c0, c0 + xs_cols) staged in shared memory
    int32_t pf_ahead;     // bytes of a workload's slots prefetched into L2 ahead of use (0 = off)
    int32_t tma;          // 1: slots streamed into shared memory by TMA bulk copies
    int32_t persist;      // 1: persistent 8-warp blocks without an x slice
    int32_t nunits;       // persistent kernels: claim units of this part
    const int32_t *units; // first workload of each claim unit (nunits + 1 entries)
};

// TMA-pipelined kernel: per warp a ring of kTmaStages chunks of kTmaChunk
// bytes (128 slots), and at most kTmaMaxCols floats of x in shared memory.
constexpr int kTmaChunk = 1024;
constexpr int kTmaStages = 4;
constexpr int kTmaMaxCols = 24576;

// Largest x slice staged in shared memory (floats): 192 KB.
constexpr int kStagedMaxCols = 49152;
// Default x slice of the staged kernel (floats): 96 KB, which with the
// kernel's 2 KB of static shared memory fits the 100 KB shared-memory
// carve-out and leaves about 156 KB of the SM's 256 KB to the L1 cache --
// the columns past the slice are gathered through L1, and a 192 KB slice
// (36 KB of L1 left) measured slower (R-MAT scale 24 PageRank iteration:
// 0.749 ms with 24K columns, 0.872 ms with 48K, 0.776 ms with none).
// Between 16K and 40K columns 24K is the fastest or within 1.1 % of it at
// R-MAT scales 22 and 24, and the fastest at scale 26 (3.376 ms against
// 3.440 with 28K and 3.412 with 32K).
constexpr int kStagedDefaultCols = 24576;
// Option 1 runs the slice kernel on a part only when the slice's columns
// hold at least this share of the part's entries (R-MAT 22-26: 37-23 % in
// the first part; R-MAT 26's second part 0.3 %, measured 0.119 ms with the
// slice against 0.110 ms without; banded and stencil matrices well under
// 1 %); the other parts run the slice-free persistent kernel (option 4).
constexpr double kSliceMinShare = 0.10;

// Split-row scratch shared by all parts of a format.
struct SplitView {
    const SplitRow *rows;      // by split row index
    const int32_t *slot_owner; // chunk slot -> split row index
    float *partial;            // chunk slot -> partial sum (scratch)
    uint32_t *counter;         // split row -> chunks done (scratch, kept at 0 between launches)
    int32_t red_split_base;    // split row s reduces into slot red_split_base + s
    int32_t pad_;
};

// Scalars of a power iteration, in device memory (FP64 where the sums need it).
struct IterState {
    double c;             // damping
    double tol;
    double delta;         // dangling mass of the current iterate
    double l1;            // L1 change of the last iteration
    double scale[2];      // HITS: factors that normalise the current iterate's halves
    double inv_n;
    int32_t iter;
    int32_t max_iter;
    int32_t parity;       // current iterate is buf[parity]
    int32_t done;
    int32_t seed;         // RWR restart node (permuted id)
    int32_t hits_norm;    // 1 or 2
    int64_t n;
    int64_t dangling_start;
    float *buf[2];        // ping-pong iterates (permuted order)
    const float *aux;     // adjoint: the loss gradient g in permuted order
    // pattern-only PageRank: z = p * inv_deg is the gathered vector
    float *zbuf[2];
    const float *inv_deg;
    // batch of independent graphs (block-diagonal union)
    const int32_t *gid;   // graph of each permuted position
    float *gbase;         // per graph: (c * dangling mass + 1 - c) / n_g of the current iterate
    double *gl1;          // per graph: L1 change of the last iteration
    double *gdelta;       // per graph: dangling mass of the current iterate
    int32_t *giters;      // per graph: iterations until its L1 change went below tol (0 = not yet)
    const int64_t *goff;  // per graph: first position (count + 1 entries)
    const int64_t *gdstart;  // per graph: first position of its dangling tail
    int32_t ngraph;
    int32_t nchunk;       // batch: fixed chunks of positions for the per-graph sums
    const int64_t *cstart;   // per chunk: first position (nchunk + 1 entries)
    const int32_t *cgraph;   // per chunk: its graph
    const int32_t *gchunk;   // per graph: first chunk (ngraph + 1 entries)
    double2 *cpart;          // per chunk: (L1 change, dangling mass) of the iteration
};

}  // namespace spg
