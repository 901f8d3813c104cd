/*
 * spg.h -- C ABI of the tiled composite SpMV library for power-law graphs
 * (GB300, sm_103a).
 *
 * The method is the one of Yang, Parthasarathy and Sadayappan, "Fast Sparse
 * Matrix-Vector Multiplication on GPUs: Implications for Graph Mining":
 * columns (and, symmetrically, rows) reordered by decreasing column length
 * (Section 3.1, Solution 2), the dense prefix cut into column tiles
 * (Solution 1, Algorithm 1), every tile stored as a composite of row-major
 * (CSR-vector) and column-major (ELL) rectangular workloads, one warp each
 * (Solution 3), with the workload size picked by a performance model
 * (Section 3.3, Algorithms 2-3), and the power iterations of Appendix F
 * (PageRank Eq. 6, HITS Eqs. 7-8, Random Walk with Restart Eq. 9) on top.
 *
 * Conventions shared by every entry point:
 *  - Every call returns an spg_status; no exception or longjmp crosses the
 *    ABI.  SPG_NOT_CONVERGED is a positive warning: outputs are written.
 *  - Vectors are FP32, in ORIGINAL node order, and may be device pointers or
 *    host pointers (pageable or pinned); the library detects which with
 *    cudaPointerGetAttributes.  Pinned (page-locked, mapped) host vectors
 *    are read (x of spg_spmv, p0 of spg_pagerank, g of spg_rwr_adjoint) and
 *    written (y of spg_spmv, the results of spg_pagerank, spg_rwr,
 *    spg_pagerank_ranks and spg_batch_pagerank) by the permutation
 *    kernels directly over the host link, in order, without a staging copy:
 *    the reordering between node order and the format's position order and
 *    the transfer are one pass.  Pageable host vectors, and the other host
 *    vectors, are staged through the library's own device workspace.  The caller owns
 *    every vector; the library keeps no caller pointer after a call
 *    returns.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls on
 *    device vectors are asynchronous on that stream; calls that take or
 *    return host vectors, and calls that report iteration counts, synchronise
 *    it before returning.  Errors of earlier asynchronous work surface as
 *    SPG_ERR_CUDA at the next synchronising call.
 *  - A handle owns its device format and one workspace.  It is
 *    thread-compatible, not thread-safe: concurrent calls on one handle race;
 *    use one handle per stream.
 */
#ifndef SPG_H
#define SPG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spg_format_t *spg_handle;

typedef enum {
    SPG_OK = 0,
    SPG_NOT_CONVERGED = 1,      /* max_iter reached before tol; outputs written */
    SPG_ERR_INVALID = -1,       /* bad argument or malformed CSR */
    SPG_ERR_OOM = -2,           /* host or device allocation failed */
    SPG_ERR_CUDA = -3,          /* a CUDA call failed (spg_last_error() has text) */
    SPG_ERR_TIMEOUT = -4,       /* a bounded device-side wait ran out */
    SPG_ERR_UNSUPPORTED = -5    /* operation not available for this matrix kind */
} spg_status;

/* What the CSR given to spg_build_format describes. */
typedef enum {
    /* The CSR is the square matrix itself (values used).  spmv/spmm only. */
    SPG_KIND_MATRIX = 0,
    /* The CSR is the adjacency A of a directed graph (rows = source; values
     * ignored).  The library builds M = W^T with W the row-normalised A,
     * M(v,u) = fl32(1/outdeg(u)) for every edge u->v (Appendix F, Eq. 6);
     * spmv multiplies by M; pagerank and rwr iterate on it. */
    SPG_KIND_PAGERANK = 1,
    /* The CSR is A; the library builds the 2n x 2n block matrix
     * [[0, A^T], [A, 0]] of Eq. 8 with unit values; hits iterates on it and
     * spmv multiplies by it (vectors of length 2n: authorities then hubs). */
    SPG_KIND_HITS = 2,
    /* The CSR is A and `val` holds per-edge logits theta (A's CSR order).
     * M(v,u) = softmax over u's out-edges of theta; rwr_weighted and
     * rwr_adjoint use it, and spg_set_edge_logits rewrites it in place. */
    SPG_KIND_WEIGHTED = 3,
    /* A batch of independent graphs (spg_build_batch only). */
    SPG_KIND_BATCH = 4
} spg_kind;

/* Compressed sparse rows: n_rows + 1 row offsets (int64), nnz column indices
 * (int32, each in [0, n_cols)), nnz values (FP32, may be NULL when the kind
 * ignores values).  Pointers are host memory unless on_device != 0.  The
 * builder copies what it needs; the arrays may be freed after the call. */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    const int64_t *row_ptr;
    const int32_t *col;
    const float *val;
    int on_device;
} spg_csr;

/* Build options.  Zero-initialise, then set what you need. */
typedef struct {
    /* Column tile width (Section 3.1, Solution 1; Algorithm 1).  0 = auto:
     * the largest power of two whose x slice (tile_width * 4 bytes) fits in
     * 60 % of the L2 (16M columns on GB300); < 0 = no dense tiles (the whole
     * matrix is one composite tile). */
    int64_t tile_width;
    /* Workload size per warp (Solution 3).  0 = Algorithm 2. */
    int64_t wl;
    /* Rows longer than this are cut into chunks of this many entries, each
     * its own warp, combined in fixed order (not in the paper; GB300).  -1 =
     * tuned by the performance model, 0 = never split, > 0 = fixed. */
    int64_t heavy_row;
    /* Storage rule of a workload: 0 = the paper's (row-major iff w >= h),
     * 1 = the major with fewer padded slots (column-major on a tie: its 32
     * rows proceed side by side, where a row-major warp walks them one
     * after another),
     * 2 = every workload row-major (the CSR-vector special case), 3 = every
     * workload column-major (the ELL special case; Section 5),
     * 4 = automatic: per part, the rule of 0-3 whose plan -- its own split
     * threshold and Algorithm 2 workload size -- the Algorithm 3 model
     * prices lowest (first of 1, 0, 2, 3 on a tie); spg_tile_info reports
     * the rule each part got.  Rule 1 is the default (opts NULL): the model
     * ranks the rules as measured at R-MAT scale 22, but at scale 26 it
     * picks rule 0 for the largest part, measured 3 % slower there.  A
     * zeroed options struct selects rule 0. */
    int layout_rule;
    /* Maximum resident warps of the whole GPU used by Algorithms 2-3.
     * 0 = query the current device (SMs x resident warps of the kernel). */
    int max_warps;
    /* Vector width the format is meant for (1 for spmv, k for spmm).  It
     * does not narrow the auto tiles: on GB300 a k = 64 SpMM ran fastest on
     * the SpMV tiles (R-MAT scale 22, RWR iteration: 3.57 ms with one part,
     * 3.69 ms with 1M-column tiles, 4.12 ms with the 128K-column tiles whose
     * 64-wide x slice fits the L2) -- each extra part re-reads and re-writes
     * the rows it continues, which costs more than the slice's L2 reuse
     * saves.  Kept for the ABI; 0 or 1 otherwise. */
    int vec_width;
    /* Also build the transposed layout (for spg_rwr_adjoint). */
    int build_transpose;
    /* Keep the host copy of the layout plan for spg_format_export_* calls. */
    int keep_plan;
    /* Keep the CSR of M in original order on the device for the plain
     * CSR-scalar / CSR-vector baselines (spg_baseline_*). */
    int keep_csr;
    /* -1 = build on the host only (no device upload; for inspecting the
     * layout on a machine without a GPU); otherwise the current device. */
    int device;
    /* Modelled cost, in seconds, of one chunk of a split row (added to the
     * Algorithm 3 time when tuning heavy_row).  0 = default. */
    double split_cost;
    /* Path of a performance table (text, see spg_load_table) or NULL for the
     * table built into the library. */
    const char *tune_table_path;
    /* Columns of x staged in shared memory per part by kernel option 1 (the
     * part's densest ones: columns are in decreasing-length order; the GB300
     * counterpart of the paper's texture-cache tile): 0 = auto (24576, i.e.
     * 96 KB, which leaves about 156 KB of the SM to the L1 cache that
     * gathers the other columns), at most 49152; < 0 = off (x gathered
     * through L1/L2 only). */
    int64_t x_stage_cols;
    /* Distance, in bytes, by which each warp's bulk L2 prefetch of its slots
     * runs ahead of their use (TMA cp.async.bulk.prefetch).  <= 0 = off (the
     * default: measured slower at R-MAT scale 22, the slot stream is not the
     * latency that limits the kernel). */
    int64_t slab_prefetch;
    /* 0 = power iterations inside one CUDA graph with a conditional WHILE
     * node (default); 1 = a host loop of direct launches that polls the
     * convergence flag every 16 iterations (the paper's structure; also what
     * a kernel profiler can attribute launch by launch). */
    int loop_mode;
    /* Most rows one workload may hold (not in the paper; GB300): a warp
     * walks its workload's 32-row blocks in sequence, so a tall workload of
     * one-entry rows is a long serial chain of dependent loads.  The
     * Algorithm 3 model sees the capped rectangles.  0 = auto (32),
     * < 0 = no cap (the paper's packing). */
    int64_t max_rows;
    /* SpMV kernel.  0 = auto (the default): option 1, or option 4 when
     * x_stage_cols < 0.  1: one persistent 32-warp block per SM (parts at
     * least 1024 columns wide) with the part's first x_stage_cols columns
     * of x in shared memory, gathered by predicated loads (shared inside the
     * slice, global past it); warps take claim units from a counter.
     * 4: persistent 8-warp blocks -- five per SM (40 warps) for plain SpMV,
     * four (32 warps) for the fused power-iteration epilogues -- with every
     * gather through L1/L2.  2: plain 8-warp blocks, one workload per warp.
     * 3: option 1 with each warp's slots streamed into a shared-memory ring
     * by TMA bulk copies.  Options 1 and 4 also compute up to four
     * consecutive short column-major workloads of a claim unit together.
     * Measured per PageRank iteration on GB300 (kernel time, options 1 vs
     * 4, before that change): R-MAT scale 22 0.170 vs 0.175 ms,
     * scale 24 0.757 vs 0.776 ms, scale 26 3.71 vs 3.77 ms; plain SpMV at
     * scale 22 0.157 vs 0.174 ms.  Scattered 4-byte gathers through L1 cost
     * one tag lookup per distinct line, which bounds the gather rate; the
     * slice moves the densest columns' gathers to shared memory. */
    int kernel;
    /* PAGERANK handles only: store column indices alone (4 bytes per slot
     * instead of 8).  M = A^T diag(1/outdeg), so the iteration gathers
     * z = p * (1/outdeg) and the epilogue writes both p and z; spmv scales x
     * first.  rwr and spmm need stored values and refuse such handles. */
    int pattern_only;
    /* Row partition (Section 3.2; PAGERANK handles only): when row_part is
     * non-NULL (int32[n], part of each node, 0 <= part < nparts, as written
     * by spg_partition_rows) the handle holds rank part_id's rows of M only
     * -- the rows v with row_part[v] == part_id -- over all columns, in the
     * column order of the whole matrix, so that every rank's iterate uses
     * one permuted order.  Its kernels write only those rows.  The array is
     * read during the call and not retained.  NULL = all rows. */
    const int32_t *row_part;
    int32_t part_id;
    int32_t nparts;
    /* Persistent SpMV kernels (options 0, 1, 4): warps take work from a
     * counter in claim units, runs of consecutive workloads grouped until
     * their cost (padded slots + 4 per row) reaches unit_slots; a workload
     * at least that large is a unit alone.  One atomic on one address per
     * claim bounds the claim rate, which small workloads would otherwise
     * hit.  0 = auto (2048), 1 = one workload per claim. */
    int64_t unit_slots;
    /* Power iterations: 0 = the convergence check (fixed-order sums of the
     * block partials, state update, graph condition) runs in the last block
     * of each iteration's last part kernel; 1 = in a one-block kernel of its
     * own after the parts (one more launch per iteration). */
    int32_t separate_check;
    /* Order in which the persistent kernels' warps claim the workloads of a
     * part: 0 = longest first (default), by the number of dependent
     * global-memory round trips the kernel's loops make for the workload,
     * so that no long workload starts near the end of the launch; 1 = the
     * ranking order of Algorithm 2 (row length descending).  Results are
     * the same bit for bit: every row has one writer and split rows are
     * combined in chunk order.  Measured on GB300 (PageRank iteration,
     * longest first vs ranking order): with row-major ties (an earlier
     * storage rule) R-MAT scale 22 0.176 vs 0.193 ms; with the current rule
     * the orders agree within 0.3 % (R-MAT 22 0.1755 vs 0.1760 ms, R-MAT 24
     * 0.798 vs 0.800 ms, Chung-Lu 4M 0.1661 vs 0.1657 ms).  Batch handles
     * (spg_build_batch): 0 = graph by graph, longest first within a graph. */
    int32_t claim_order;
    /* Non-zero: also store every part as a row-sorted (row, column, value)
     * list -- the paper's TILE-COO format (same degree order and column
     * tiles, COO storage instead of the composite one; Section 5 compares
     * the two) -- for spg_spmv_tile_coo.  12 more bytes per non-zero on the
     * device.  Ignored by spg_build_batch. */
    int32_t tile_coo;
} spg_build_opts;

/* Per-call results of the power iterations. */
typedef struct {
    int iters;          /* iterations run */
    double last_l1;     /* L1 change of the last iteration (max over columns for k > 1) */
    double dangling;    /* dangling mass of the final iterate */
    float ms;           /* device time of the solve (CUDA events) */
} spg_iter_info;

/* Summary of a built format. */
typedef struct {
    int64_t n, nnz;             /* matrix size and non-zeros */
    int64_t ntile;              /* dense tiles (Algorithm 1); parts = ntile + 1 */
    int64_t tile_width;
    int64_t nworkloads;         /* over all parts, zero-row workloads included */
    int64_t padded_slots;       /* stored slots (non-zeros + padding) */
    int64_t split_rows, split_chunks;
    int64_t zero_rows;          /* rows with no entry in any tile */
    int64_t device_bytes;       /* device memory held by the format */
    int64_t max_warps;          /* value used by the model */
    double predicted_ms;        /* Algorithm 3 time summed over parts */
    int64_t dangling_start;     /* first position of the dangling tail (kind PAGERANK/WEIGHTED) */
} spg_format_info_t;

/* One part (dense tile or the sparse remainder) of a format. */
typedef struct {
    int64_t col_begin, col_end; /* permuted column range */
    int64_t heavy;              /* split threshold used (0 = none) */
    int64_t wl;                 /* workload size (Algorithm 2) */
    int64_t nvirt;              /* ranked (virtual) rows */
    int64_t nwl;                /* workloads, zero-row workloads excluded */
    int64_t nnz;                /* non-zeros in the part */
    double predicted_ms;
    int64_t layout_rule;        /* storage rule the part was built with (0-3) */
    double slice_share;         /* share of the part's entries in its first x_stage_cols
                                   columns; kernel option 1 stages the x slice for the
                                   part only when it is at least 0.10 */
    int64_t nunits;             /* claim units of the persistent kernels */
} spg_tile_info_t;

/* ---------------------------------------------------------------- build -- */

/* Build the tiled composite format of the matrix the CSR describes (see
 * spg_kind), on the host (C++), and upload it to the current device.
 * Steps: transform (Appendix F), symmetric order by decreasing column length
 * with ties by ascending id (Solution 2, counting sort as in the "Sorting
 * Cost" paragraph), Algorithm 1 tiles, per part the in-tile row ranking,
 * heavy-row split, Algorithm 2 workload size and packing (Solution 3).
 * `opts` may be NULL (all defaults).  On success *out owns the format.
 * Errors: SPG_ERR_INVALID for a non-square matrix, row_ptr not starting at 0
 * or not non-decreasing, row_ptr[n] != nnz, a column out of range, n >= 2^28;
 * SPG_ERR_OOM; SPG_ERR_CUDA. */
spg_status spg_build_format(const spg_csr *csr, spg_kind kind, const spg_build_opts *opts,
                            void *stream, spg_handle *out);

/* Free a handle and everything it owns (device memory included).  NULL is ok. */
spg_status spg_destroy(spg_handle h);

spg_status spg_format_info(spg_handle h, spg_format_info_t *info);
spg_status spg_tile_info(spg_handle h, int64_t part, spg_tile_info_t *info);

/* Symmetric permutation: pi[orig] = position, inv[position] = orig (host
 * arrays of n int32; either may be NULL). */
spg_status spg_format_perm(spg_handle h, int32_t *pi, int32_t *inv);

/* Plan of one part (needs keep_plan): the ranking of its (virtual) rows --
 * permuted row id, chunk index, length -- and per workload its first rank,
 * height h, width w (length of its first row) and major (0 row, 1 column).
 * Host arrays sized nvirt and nwl from spg_tile_info; any may be NULL. */
spg_status spg_format_export_plan(spg_handle h, int64_t part, int64_t *rank_row,
                                  int64_t *rank_chunk, int64_t *rank_len,
                                  int64_t *wl_first, int64_t *wl_h, int64_t *wl_w,
                                  int64_t *wl_major);

/* Every stored non-zero as (row, col, value) in ORIGINAL ids, read back from
 * the packed device (or host-only) layout, padding skipped, split chunks
 * merged: nnz entries into host arrays, in storage order. */
spg_status spg_format_export_entries(spg_handle h, int64_t *rows, int32_t *cols, float *vals);

/* Rows (permuted ids) with no entry in any part, ascending (host, zero_rows). */
spg_status spg_format_zero_rows(spg_handle h, int64_t *rows);

/* ----------------------------------------------------------------- SpMV -- */

/* y = alpha * M x + beta * y (Appendix B's y = A x, on the matrix of the
 * handle's kind).  x, y: n FP32, original order.  beta == 0: y is not read.
 * The product runs one tiled-composite launch per part in order (Solution 1:
 * "we restart a kernel for each tile"), FP32 accumulation, no atomics on y;
 * x is taken into the permuted order before (gathered from device memory,
 * read in order from pinned host memory) and y gathered back into original
 * order after (y[j] = alpha y'[pi(j)] + beta y[j], written in order). */
spg_status spg_spmv(spg_handle h, const float *x, float *y, float alpha, float beta,
                    void *stream);

/* Same product with x and y already in the handle's permuted order (device
 * pointers only): y' = M' x', no permutation passes. */
spg_status spg_spmv_permuted(spg_handle h, const float *x_perm, float *y_perm, void *stream);

/* TILE-COO SpMV (Section 5: the tiled kernel with COO storage, the ablation
 * of the composite storage): y' = M' x' on PERMUTED device vectors of n
 * floats (x' = x[inv], as spg_spmv_permuted), one launch per part over its
 * row-sorted entry list: each warp takes 256 consecutive entries, sums
 * them per row with a segmented warp scan and adds rows that may continue
 * into a neighbouring warp's entries with atomicAdd (the summation order
 * of such rows is not fixed).  y' is zeroed first.  Needs a handle built
 * with tile_coo != 0 (else SPG_ERR_INVALID); x' and y' must be distinct. */
spg_status spg_spmv_tile_coo(spg_handle h, const float *x_perm, float *y_perm, void *stream);

/* Y = alpha * M X + beta * Y for k vectors: X (n x k) and Y (n x k) FP32,
 * row-major with leading dimensions ldx, ldy >= k, original row order.
 * One warp per workload; for k a multiple of 64 each half-warp gathers one
 * stored entry's X row (16 bytes per lane), otherwise each lane takes two of
 * every 64-column chunk; device pointers only.  k in [1, 1024]. */
spg_status spg_spmm(spg_handle h, const float *X, int64_t ldx, float *Y, int64_t ldy, int k,
                    float alpha, float beta, void *stream);

/* ------------------------------------------------------ power iterations -- */

/* PageRank, Appendix F Eq. 6: p <- c M p + (c * sum_{u dangling} p_u + 1 - c)/n,
 * from p0 (NULL = uniform 1/n), until ||p(k+1) - p(k)||_1 < tol or max_iter
 * (tol <= 0: exactly max_iter iterations).  The damping, dangling mass, L1
 * norm and the swap of iterates are fused into the last tile's epilogue; the
 * scalars are FP64; the loop runs inside one CUDA graph with a conditional
 * WHILE node (no host round trip per iteration).  p_out: n FP32, original
 * order.  Kind PAGERANK only.  Returns SPG_NOT_CONVERGED if tol > 0 was not
 * reached. */
spg_status spg_pagerank(spg_handle h, float damping, double tol, int max_iter,
                        const float *p0, float *p_out, spg_iter_info *info, void *stream);

/* Section 3.2: the bitonic row partition.  Rows of M (nodes, by in-degree
 * row_len[v], decreasing; ties ascending id) are dealt to P parts in rounds
 * of P, the dealing direction reversing every round, so that parts get
 * near-equal rows and entries.  part: int32[n] host output.  P in [1, 64];
 * SPG_ERR_INVALID otherwise. */
spg_status spg_partition_rows(int64_t n, const int64_t *row_len, int P, int32_t *part);

/* Row-partitioned PageRank (Section 3.2) over P rank handles, run on the
 * calling device: ranks[r] must be PAGERANK handles built from the same
 * graph with the same row_part, nparts = P and part_id = r.  Each
 * iteration, every rank's tiled-composite kernels produce its own rows of
 * the next iterate in its own x/y buffers; an all-gather step then gives
 * every rank the whole vector (on one device: a kernel copying each row
 * from its owner's buffer into the others', where several GPUs would
 * all-gather the ranks' row slices and scatter them locally); one check
 * kernel sums all ranks' (L1 change, dangling mass) partials in a fixed
 * order -- the all-reduce -- and updates every rank's state.  Same
 * arguments and result as spg_pagerank (p0 NULL = uniform start); the host
 * drives the iterations (no graph), P in [1, 8]. */
spg_status spg_pagerank_ranks(const spg_handle *ranks, int P, float damping, double tol,
                              int max_iter, const float *p0, float *p_out, spg_iter_info *info,
                              void *stream);

/* One PageRank iteration (Eq. 6) of ONE rank of the Section 3.2 row
 * partition, for a driver that runs every rank in its own process (or on its
 * own device) and exchanges row slices between iterations itself.  h: a
 * device PAGERANK handle built with row_part / part_id = this rank (or with
 * no row_part: every row); x_perm: the whole current iterate (n floats,
 * the handle's permuted order, device); y_perm: device output of n floats,
 * of which only this rank's rows are written.  delta: the dangling mass of
 * x over ALL rows (the sum over ranks of the previous step's partial[1];
 * for the uniform start, the sum over dangling nodes of 1/n).  Writes, in
 * partial (host double[2]): this rank's L1 change sum |y'_v - x'_v| and its
 * rows' dangling mass sum of y'_v over dangling v, each summed in a fixed
 * order.  Synchronises `stream`.  Errors: SPG_ERR_INVALID for a non-device
 * or aliased vector, bad damping or negative delta; SPG_ERR_UNSUPPORTED for
 * a pattern_only handle. */
spg_status spg_pagerank_rank_step(spg_handle h, float damping, double delta, const float *x_perm,
                                  float *y_perm, double *partial, void *stream);

/* Row slices of the Section 3.2 all-gather (device pointers, idx int32 of
 * count positions in [0, n)): pack slice[i] = full[idx[i]]; unpack
 * full[idx[i]] = slice[i].  Asynchronous on `stream`; count 0 is a no-op;
 * SPG_ERR_INVALID for a negative count or a host pointer. */
spg_status spg_pack_slice(int64_t count, const int32_t *idx, const float *full, float *slice,
                          void *stream);
spg_status spg_unpack_slice(int64_t count, const int32_t *idx, const float *slice, float *full,
                            void *stream);

/* Random Walk with Restart, Appendix F Eq. 9 on M (personalised PageRank):
 * r <- c M r + [v == s] (c * dangling mass + 1 - c), r(0) = e_s, for each of
 * the k restart nodes seeds[0..k) (host int32, original ids).  k == 1 runs
 * SpMV iterations; k > 1 runs them as one SpMM over the n x k block (R is
 * n x k row-major, original order); columns that converge keep iterating
 * until all have (their L1 stays below tol).  restart = 1 - c.  k in
 * [1, 64] (one 64-column chunk of per-column sums); SPG_ERR_INVALID
 * otherwise -- call again per group of 64 seeds.  Kind PAGERANK. */
spg_status spg_rwr(spg_handle h, float restart, const int32_t *seeds, int k, double tol,
                   int max_iter, float *R, spg_iter_info *info, void *stream);

/* HITS, Appendix F Eqs. 7-8 (Jacobi form) as one SpMV on [[0,A^T],[A,0]]:
 * a(0) = h(0) = 1/n, each half normalised separately every iteration
 * (norm = 2: Euclidean, the default; norm = 1: sum, as in the paper).
 * Exactly max_iter iterations (tol is reserved and must be <= 0).  auth,
 * hub: n FP32, original order.  Kind HITS. */
spg_status spg_hits(spg_handle h, int norm, double tol, int max_iter, float *auth, float *hub,
                    spg_iter_info *info, void *stream);

/* ------------------------------------------------- differentiable RWR -- */

/* Rewrite the transition weights of a WEIGHTED handle from per-edge logits
 * theta (nnz FP32, A's CSR order, device or host): P_e = softmax over the
 * out-edges of each node, written straight into the packed slots of the
 * forward (and transposed) layout through the stored edge map. */
spg_status spg_set_edge_logits(spg_handle h, const float *theta, void *stream);

/* RWR fixed point on a WEIGHTED handle: r = c K r + (1-c) e_s with
 * K = M + e_s 1_D^T (dangling mass returns to s); r: n FP32, original order. */
spg_status spg_rwr_weighted(spg_handle h, float restart, int32_t seed, double tol, int max_iter,
                            float *r, spg_iter_info *info, void *stream);

/* Adjoint of spg_rwr_weighted (not in the paper): given r and g = dL/dr
 * (n FP32 each, original order), solve lambda = c K^T lambda + g by
 * transposed-SpMV iterations on the stored transposed layout (needs
 * build_transpose), then dL/dtheta_e = P_e (G_e - sum_{e' in out(u)} P_e' G_e')
 * with G_e = c lambda_v r_u for e = u -> v.  lambda: n FP32; dtheta: nnz FP32
 * in A's CSR order.  No iterate checkpointing: the fixed point is
 * differentiated implicitly. */
spg_status spg_rwr_adjoint(spg_handle h, float restart, int32_t seed, const float *r,
                           const float *g, double tol, int max_iter, float *lambda,
                           float *dtheta, spg_iter_info *info, void *stream);

/* ------------------------------------------------------ batched graphs -- */

/* Build one handle over `count` independent graphs (adjacency CSRs, as for
 * SPG_KIND_PAGERANK; host or device pointers per csr).  The graphs become the
 * diagonal blocks of one matrix; the degree order of Section 3.1 Solution 2
 * is taken within each graph, the composite partition (Solution 3) over all
 * of them, so one launch sweeps every graph (not in the paper; batching of
 * many small graphs).  opts->tile_width is ignored (one part).  Graph g's
 * nodes occupy positions [offsets[g], offsets[g+1]) of the concatenated
 * vectors (spg_batch_offsets).
 * With claim_order 0 (the default) the workloads are stored, and claimed
 * by the persistent kernels' warps, graph by graph (longest first within a
 * graph, claim units within a graph), so that the warps running at any
 * moment share a few graphs' x and y lines in L1 and L2 (512 Chung-Lu
 * graphs, PageRank iteration: 0.625 ms against 0.677 ms longest first over
 * all graphs); claim_order 1 keeps the ranking order.  Either way the plan
 * (ranking, workload sizes, packing) is that of the whole union and the
 * results are the same bit for bit. */
spg_status spg_build_batch(const spg_csr *graphs, int count, const spg_build_opts *opts,
                           void *stream, spg_handle *out);

/* count + 1 node offsets of a batch handle (host int64 array). */
spg_status spg_batch_offsets(spg_handle h, int64_t *offsets);

/* PageRank (Eq. 6, uniform dangling redistribution per graph) on every graph
 * of a batch handle at once: per iteration one tiled-composite launch over
 * all graphs, one block per fixed chunk of at most 8192 positions for the
 * per-graph L1 change and dangling mass, one check block that adds each
 * graph's chunks in order; the whole solve is one CUDA graph with a WHILE
 * node.  Each
 * graph records the iteration at which its L1 change first went below tol;
 * the loop ends when all have (or at max_iter).  p_out: the concatenated
 * vectors, original node order within each graph.  info (nullable): count
 * entries, one per graph (iters = its convergence iteration, last_l1 = its
 * final L1 change, dangling = its final dangling mass). */
spg_status spg_batch_pagerank(spg_handle h, float damping, double tol, int max_iter,
                              float *p_out, spg_iter_info *info, void *stream);

/* ------------------------------------------------------------ baselines -- */

typedef enum { SPG_BASELINE_CSR_SCALAR = 0, SPG_BASELINE_CSR_VECTOR = 1 } spg_baseline;

/* The plain CSR kernels of Appendix B on the CSR of M in original order
 * (needs keep_csr): CSR-scalar (one thread per row) and CSR-vector (one warp
 * per row).  Same semantics as spg_spmv / spg_pagerank. */
spg_status spg_baseline_spmv(spg_handle h, spg_baseline which, const float *x, float *y,
                             float alpha, float beta, void *stream);
spg_status spg_baseline_pagerank(spg_handle h, spg_baseline which, float damping, double tol,
                                 int max_iter, float *p_out, spg_iter_info *info, void *stream);

/* ----------------------------------------------- allocation-free SpMV -- */

/* The paper has no counterpart to this entry point.
 *
 * Same product as spg_spmv_permuted (y' = M' x', device vectors in the
 * handle's permuted order), for callers that must not allocate device
 * memory during the call: a serving or real-time loop that reserved all of
 * its device memory up front, a process whose device memory belongs to an
 * allocator or pool it may not bypass, or one already at its memory limit,
 * where a cudaMalloc can fail or stall the device.  This call allocates
 * nothing (no cudaMalloc, no cudaFree, no allocating library routine):
 * the scratch its kernels need -- partial sums and arrival counters of rows
 * cut into chunks, work counters of the persistent kernels -- lives in one
 * fixed array of 1,311,744 bytes inside the library, which every GPU that
 * loads the library holds until the process exits.  It runs the kernel
 * option the handle was built with (spg_build_opts.kernel), as
 * spg_spmv_permuted does.
 *
 *  - Limits: formats with at most 128 parts, 65,536 split rows and 262,144
 *    split chunks (spg_format_info: ntile + 1, split_rows, split_chunks);
 *    larger ones get SPG_ERR_INVALID with a message naming the limits.
 *  - The handle's device must be the current device.  The first call on a
 *    device looks up the array's device address (cudaGetSymbolAddress) with
 *    that device current; make that first call before any stream capture.
 *    The address is kept for the life of the process: resetting the device
 *    (cudaDeviceReset) after that first call is not supported.
 *  - x_perm and y_perm need the alignment of a float (4 bytes); the kernels
 *    use 16-byte loads of x only where the address allows them.
 *  - Every call on a device shares the one array and it keeps the last
 *    call's contents: the call clears its counters on `stream` before its
 *    kernels, but calls whose work overlaps on the GPU (other streams,
 *    other threads) race on the array.  Order them on one stream.
 *  - The handle itself is built (and allocates) beforehand, once. */
spg_status spg_spmv_permuted_noalloc(spg_handle h, const float *x_perm, float *y_perm,
                                     void *stream);

/* -------------------------------------------------------------- misc -- */

/* Load a performance table (Section 3.3 lookup table) for the process: text
 * lines "major log2w log2h perf" (perf in slots/s); missing shapes take the
 * nearest measured bucket.  NULL restores the built-in table. */
spg_status spg_load_table(const char *path);

/* Measurement: time each part's tiled-composite kernel alone, `reps`
 * back-to-back launches per part between two CUDA events on `stream`, and
 * write the mean launch duration (ms) of part p to ms_out[p] (host array of
 * ntile + 1 floats).  mode 0: the plain SpMV kernel (x' and y' are the
 * handle's workspace, contents arbitrary); mode 1: the PageRank epilogue
 * kernel on the state of the last spg_pagerank call on this handle. */
spg_status spg_time_parts(spg_handle h, int mode, int reps, float *ms_out, void *stream);

/* Kernel launches this library issued since load (all entry points). */
int64_t spg_launch_count(void);

const char *spg_status_string(spg_status s);
/* Text of the last error on the calling thread ("" if none). */
const char *spg_last_error(void);
/* Library version string. */
const char *spg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPG_H */
