// kernels.h -- host launchers of the sm_103a kernels (kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "spg_internal.h"

namespace spg {

// Epilogue of the last part that touches a row (Appendix F).
enum EpiMode {
    EPI_RAW = 0,       // y' = (M' x')_v
    EPI_PAGERANK = 1,  // y' = c (M' x')_v + (c delta + 1 - c)/n;  sum |y'-x'|, dangling sum
    EPI_RWR = 2,       // y' = c (M' x')_v + [v == s](c delta + 1 - c); same sums
    EPI_HITS = 3,      // y' = (M' x')_v * scale[other half];  per-half sum or sum of squares
    EPI_ADJ = 4,       // y' = c (M'^T x')_v + [v dangling] c x'_s + g'_v;  sum |y'-x'|
    EPI_BATCH = 5,     // y' = c (M' x')_v + base[graph of v];  sums in a separate pass
    EPI_PR_PAT = 6,    // pattern-only PageRank: gathers z, writes p and z = p * inv_deg
    EPI_RAW_PAT = 7    // pattern-only SpMV: y' = A'^T x' (x' already scaled by inv_deg)
};

// One tiled-composite launch of one part (Solution 3: one warp per
// workload).  x/y come from st->buf[parity] when st != nullptr.
// Fused convergence check: when nred > 0, the last block of the launch runs
// the iteration's check over red[0, nred) on st (and the graph condition).
struct FuseCheck {
    unsigned long long cond = 0;
    unsigned *done = nullptr;     // arrival counter, zero between launches
    IterState *st = nullptr;
    int use_cond = 0;
    int nred = 0;
};

// Returns true if the launch also ran the check (fc.nred > 0 and a kernel
// that supports it).
bool launch_part(int mode, const PartView &pv, const SplitView &sv, const float *x, float *y,
                 const IterState *st, double2 *red, cudaStream_t s, const FuseCheck &fc = FuseCheck());

// SpMM over one part: Y' (n x k, ld k) += rows of M' X' (k <= 1024).  Modes
// EPI_RAW and EPI_RWR (per-column restart seeds, per-column sums into
// red[(slot * 2 + {0,1}) * k + j]).
void launch_part_spmm(int mode, const PartView &pv, const SplitView &sv, const float *X, float *Y,
                      int k, const IterState *st, const int32_t *seeds, const double *delta_k,
                      double *redk, cudaStream_t s);

// Sum the reduction slots and advance the iteration state (one block).
// mode EPI_PAGERANK / EPI_RWR: l1 = sum slot.x, delta = sum slot.y;
// EPI_HITS: scale[c] = 1/norm of half c.  Sets the graph conditional
// (when cond != 0) to "keep iterating".
void launch_check(int mode, IterState *st, const double2 *red, int nred,
                  unsigned long long cond, int use_cond, cudaStream_t s);
// Row-partitioned PageRank on one device: all-gather of the ranks' rows and
// the all-reduce / check over all ranks' partials.
void launch_allgather_rows(int64_t n, const int8_t *owner, IterState *const *states, int P, bool pat,
                           cudaStream_t s);
void launch_check_ranks(IterState *const *states, int P, const double2 *red, int nred, cudaStream_t s);
// The check for SpMM RWR: per-column l1_k / delta_k (two-stage column sums
// in `scratch`), l1 = max over columns.
void launch_check_k(IterState *st, const double *redk, int nred, int k, double *delta_k,
                    double *l1_k, double *scratch, unsigned long long cond, int use_cond,
                    cudaStream_t s);

// Dangling mass of buf[parity] (positions >= dangling_start, or the rows
// flagged in `dangling`) into st->delta; `scratch` holds init_delta_scratch()
// doubles.
void launch_init_delta(IterState *st, double *scratch, cudaStream_t s);
void launch_init_delta_flags(IterState *st, const uint8_t *dangling, double *scratch, cudaStream_t s);
int init_delta_scratch();
// p[idx[i]] = 1 for i < count
void launch_set_one(float *p, const int32_t *idx, int count, cudaStream_t s);
void launch_init_delta_k(int64_t dangling_start, int64_t n, const float *X, int k,
                         double *delta_k, double *scratch, cudaStream_t s);
// Doubles of scratch the two-stage column sums need (check_k, init_delta_k).
int colsum_scratch();

// z[i] = p[i] * inv_deg[i] (pattern-only start vectors)
void launch_scale(int64_t n, const float *p, const float *inv_deg, float *z, cudaStream_t s);
// xp[k] = x[inv[k]] * inv_deg[k]
void launch_gather_scaled(int64_t n, const int32_t *inv, const float *x, const float *inv_deg,
                          float *xp, cudaStream_t s);

// Permutation and vector helpers.
void launch_gather(int64_t n, const int32_t *inv, const float *x, float *xp, cudaStream_t s);
void launch_gather_rows(int64_t n, int k, const int32_t *inv, const float *X, int64_t ldx,
                        float *Xp, cudaStream_t s);
void launch_scatter_axpby(int64_t n, const int32_t *inv, const float *yp, float *y, float alpha,
                          float beta, cudaStream_t s);
void launch_scatter_rows(int64_t n, int k, const int32_t *inv, const float *Yp, float *Y,
                         int64_t ldy, float alpha, float beta, cudaStream_t s);
// Caller order <-> position order by perm (perm[j] = position of node j),
// the caller's side read or written in order (it may be mapped host memory):
// xp[perm[j]] = x[j] (* d[perm[j]] when d != nullptr);
void launch_permute_in(int64_t n, const int32_t *perm, const float *x, const float *d, float *xp,
                       cudaStream_t s);
// out[j] = buf[parity][perm[j]] (* the scale of its half when hits), from state;
void launch_unpermute_state(int64_t n, const int32_t *perm, const IterState *st, float *out,
                            const uint8_t *row_half, int hits, cudaStream_t s);
// y[j] = alpha yp[perm[j]] + beta y[j] (beta = 0: y not read);
void launch_unpermute_axpby(int64_t n, const int32_t *perm, const float *yp, float *y, float alpha,
                            float beta, cudaStream_t s);
// rows of an n x k block: Y[j] (leading dimension ldy) = alpha Yp[perm[j]] + beta Y[j].
void launch_unpermute_rows(int64_t n, int k, const int32_t *perm, const float *Yp, float *Y,
                           int64_t ldy, float alpha, float beta, cudaStream_t s);
void launch_fill(int64_t n, float v, float *p, cudaStream_t s);
void launch_onehot_rows(int64_t n, int k, const int32_t *seeds, float *X, cudaStream_t s);

// TILE-COO SpMV over entries [e0, e1) of a row-sorted (row, column, value)
// list: y[row] += val * x[col] (y zeroed by the caller before the first part).
void launch_tile_coo(const int32_t *row, const int32_t *col, const float *val, int64_t e0,
                     int64_t e1, const float *x, float *y, int num_sms, cudaStream_t s);

// Plain CSR baselines on M in original order.  mode EPI_RAW or EPI_PAGERANK
// (dangling flags per row; reductions into red[blockIdx]).
void launch_csr_scalar(int mode, int64_t n, const int64_t *rp, const int32_t *col,
                       const float *val, const uint8_t *dangling, const float *x, float *y,
                       const IterState *st, double2 *red, int *nblocks_out, cudaStream_t s);
void launch_csr_vector(int mode, int64_t n, const int64_t *rp, const int32_t *col,
                       const float *val, const uint8_t *dangling, const float *x, float *y,
                       const IterState *st, double2 *red, int *nblocks_out, cudaStream_t s);
int csr_scalar_blocks(int64_t n);
int csr_vector_blocks(int64_t n);

// Edge weights: P_e = softmax over out-edges of theta, written to the slab
// slots edge_slot[e] (forward) and edge_slot_t[e] (transposed, nullable).
// heavy: the nheavy nodes of more than edge_heavy_degree() out-edges (one
// block each); the others take 8-lane segments.
void launch_edge_softmax(int64_t n, const int64_t *a_rp, const float *theta,
                         const int64_t *edge_slot, uint2 *slab, const int64_t *edge_slot_t,
                         uint2 *slab_t, float *P_out, const int32_t *heavy, int nheavy,
                         cudaStream_t s);
int edge_heavy_degree();
// dtheta_e = P_e (G_e - sum_{e' in out(u)} P_e' G_e'), G_e = c lambda_v r_u.
void launch_edge_grad(int64_t n, const int64_t *a_rp, const int32_t *a_col, const float *P,
                      const float *lambda, const float *r, float c, float *dtheta,
                      const int32_t *heavy, int nheavy, cudaStream_t s);

// Resident blocks per SM of the persistent 8-warp SpMV kernel (options 0
// and 4) and of the plain one-warp-per-workload kernel (option 2) on this
// device.
int persist_blocks_per_sm();
int part_blocks_per_sm();

// Batch of graphs: L1 change and dangling mass per chunk of a graph's rows
// (nchunk chunks, one block each), then the per-graph sums of the chunks in
// order, the per-graph bases, convergence record and the loop condition
// (one block).
void launch_batch_reduce(IterState *st, int nchunk, cudaStream_t s);
void launch_batch_check(IterState *st, int ngraph, unsigned long long cond, int use_cond,
                        cudaStream_t s);
// x[v] = 1 / n_{graph of v}
void launch_batch_init(int64_t n, const IterState *st, float *x, cudaStream_t s);

// Launch counter of this library.
void count_launches(int64_t k);
int64_t launch_count();

}  // namespace spg
