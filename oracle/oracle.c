/*
 * oracle.c -- plain, slow, single-threaded FP64 reference of the method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link,
 * call or execute this file: only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference leg use it.  It shares no code with the
 * CUDA path (paper_1103_2405_gb300/csrc); the only common inputs are the
 * seeded graphs and vectors produced by graphgen/.
 *
 * Every function follows a definition from the paper (Yang, Parthasarathy,
 * Sadayappan, "Fast Sparse Matrix-Vector Multiplication on GPUs: Implications
 * for Graph Mining"), cited in its comment, written out with no blocking,
 * fusion or reordering beyond what that definition states.
 *
 *  - orc_build_M      Appendix F, Eq. 6: W = row-normalised A, matrix M = W^T.
 *  - orc_spmv         Appendix B: y = A x over CSR, rows in order, columns
 *                     ascending, FP64 accumulation.
 *  - orc_pagerank     Appendix F, Eq. 6 (+ uniform dangling redistribution).
 *  - orc_rwr          Appendix F, Eq. 9 on M (+ dangling mass to the source).
 *  - orc_hits         Appendix F, Eq. 7 (Jacobi form), per-half normalisation.
 *  - orc_edge_softmax / orc_rwr_weighted / orc_rwr_adjoint
 *                     RWR with per-edge softmax transition weights and the
 *                     gradient of -sum log r_t by the adjoint fixed point
 *                     (not in the paper; the differentiation workload).
 *  - orc_degree_order Section 3.1 Solution 2: columns by decreasing length.
 *  - orc_alg1_tiles   Algorithm 1 (tile count).
 *  - orc_alg3_model / orc_alg2_partition / orc_partition_tile
 *                     Algorithms 2 and 3, Section 3.1 Solution 3.
 *  - orc_bitonic_partition  Section 3.2 (bitonic row partition).
 *
 * Readings where the paper is silent or ambiguous are stated at each use.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------ transform -- */

/* Appendix F, Eq. 6: W(u,v) = A(u,v) / outdeg(u); the power iteration uses
 * W^T, so M(v,u) = 1/outdeg(u) for every edge u->v.  Each value is the FP64
 * quotient rounded once to FP32 (the precision the GPU stores).  Row v of M
 * lists its columns u in ascending order.  Returns nnz. */
int64_t orc_build_M(int64_t n, const int64_t *a_rowptr, const int32_t *a_col,
                    int64_t *m_rowptr, int32_t *m_col, float *m_val)
{
    int64_t nnz = a_rowptr[n];
    for (int64_t v = 0; v <= n; ++v) m_rowptr[v] = 0;
    for (int64_t e = 0; e < nnz; ++e) m_rowptr[a_col[e] + 1]++;
    for (int64_t v = 0; v < n; ++v) m_rowptr[v + 1] += m_rowptr[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!fill) return -1;
    for (int64_t v = 0; v <= n; ++v) fill[v] = m_rowptr[v];
    for (int64_t u = 0; u < n; ++u) {            /* ascending u => sorted rows */
        int64_t deg = a_rowptr[u + 1] - a_rowptr[u];
        for (int64_t e = a_rowptr[u]; e < a_rowptr[u + 1]; ++e) {
            int64_t v = a_col[e];
            m_col[fill[v]] = (int32_t)u;
            m_val[fill[v]] = (float)(1.0 / (double)deg);
            fill[v]++;
        }
    }
    free(fill);
    return nnz;
}

/* --------------------------------------------------------- SpMV -- */

/* Appendix B: y = alpha * A x + beta * y over CSR; beta == 0 means y is not
 * read.  FP64 throughout, columns in stored (ascending) order. */
void orc_spmv(int64_t nrows, const int64_t *rowptr, const int32_t *col,
              const float *val, const double *x, double alpha, double beta,
              double *y)
{
    for (int64_t v = 0; v < nrows; ++v) {
        double s = 0.0;
        for (int64_t k = rowptr[v]; k < rowptr[v + 1]; ++k)
            s += (double)val[k] * x[col[k]];
        y[v] = alpha * s + (beta != 0.0 ? beta * y[v] : 0.0);
    }
}

/* Same on a row subset: y[i] = (A x)[rows[i]] (sampled checks at full size). */
void orc_spmv_rows(int64_t nsel, const int64_t *rows, const int64_t *rowptr,
                   const int32_t *col, const float *val, const double *x,
                   double *y)
{
    for (int64_t i = 0; i < nsel; ++i) {
        int64_t v = rows[i];
        double s = 0.0;
        for (int64_t k = rowptr[v]; k < rowptr[v + 1]; ++k)
            s += (double)val[k] * x[col[k]];
        y[i] = s;
    }
}

/* ----------------------------------------------------- PageRank -- */

/* Appendix F, Eq. 6: p(k+1) = c M p(k) + (1-c) p(0), p(0) = 1/n.
 * Reading (the paper is silent on dangling nodes): the mass c * sum_{u in D}
 * p_u of nodes with no out-edges is spread uniformly, so every iterate sums
 * to 1:  p(k+1)_v = c (M p(k))_v + (c * sum_{u in D} p(k)_u + 1 - c) / n.
 * Reading (convergence is not stated): stop once ||p(k+1) - p(k)||_1 < tol,
 * or after max_iter iterations.  p_init (nullable) replaces p(0) as the start
 * (warm start); the teleport stays uniform.  Returns the iteration count. */
int orc_pagerank(int64_t n, const int64_t *rowptr, const int32_t *col,
                 const float *val, const int64_t *outdeg, double c, double tol,
                 int max_iter, const double *p_init, double *p, double *last_l1)
{
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    if (!q) return -1;
    for (int64_t v = 0; v < n; ++v) p[v] = p_init ? p_init[v] : 1.0 / (double)n;
    int it = 0;
    double l1 = INFINITY;
    while (it < max_iter) {
        double dangling = 0.0;
        for (int64_t u = 0; u < n; ++u)
            if (outdeg[u] == 0) dangling += p[u];
        double base = (c * dangling + (1.0 - c)) / (double)n;
        for (int64_t v = 0; v < n; ++v) {
            double s = 0.0;
            for (int64_t k = rowptr[v]; k < rowptr[v + 1]; ++k)
                s += (double)val[k] * p[col[k]];
            q[v] = c * s + base;
        }
        l1 = 0.0;
        for (int64_t v = 0; v < n; ++v) { l1 += fabs(q[v] - p[v]); p[v] = q[v]; }
        ++it;
        if (l1 < tol) break;
    }
    free(q);
    if (last_l1) *last_l1 = l1;
    return it;
}

/* ---------------------------------------------------------- RWR -- */

/* Appendix F, Eq. 9: r(k+1) = c W' r(k) + (1-c) e_s, here with the
 * column-stochastic M = W^T in place of W (reading: personalised PageRank on
 * the directed graph, so r stays a distribution).  Reading for dangling
 * nodes: their mass returns to the restart node s,
 *   r(k+1)_v = c (M r(k))_v + [v == s] (c * sum_{u in D} r(k)_u + 1 - c).
 * r(0) = e_s (or r_init when given).  Stops at ||r(k+1) - r(k)||_1 < tol or
 * max_iter.  Returns the iteration count. */
int orc_rwr(int64_t n, const int64_t *rowptr, const int32_t *col,
            const float *val, const int64_t *outdeg, int64_t s, double c,
            double tol, int max_iter, const double *r_init, double *r,
            double *last_l1)
{
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    if (!q) return -1;
    for (int64_t v = 0; v < n; ++v) r[v] = r_init ? r_init[v] : (v == s ? 1.0 : 0.0);
    int it = 0;
    double l1 = INFINITY;
    while (it < max_iter) {
        double dangling = 0.0;
        for (int64_t u = 0; u < n; ++u)
            if (outdeg[u] == 0) dangling += r[u];
        for (int64_t v = 0; v < n; ++v) {
            double acc = 0.0;
            for (int64_t k = rowptr[v]; k < rowptr[v + 1]; ++k)
                acc += (double)val[k] * r[col[k]];
            q[v] = c * acc + (v == s ? c * dangling + (1.0 - c) : 0.0);
        }
        l1 = 0.0;
        for (int64_t v = 0; v < n; ++v) { l1 += fabs(q[v] - r[v]); r[v] = q[v]; }
        ++it;
        if (l1 < tol) break;
    }
    free(q);
    if (last_l1) *last_l1 = l1;
    return it;
}

/* --------------------------------------------------------- HITS -- */

/* Appendix F, Eq. 7 (Jacobi form): a(k+1) = A^T h(k), h(k+1) = A a(k), with
 * a(0) = h(0) = 1/n.  After each step each half is normalised on its own:
 * norm == 1 divides by its sum (as the paper describes), norm == 2 by its
 * Euclidean length.  A half that comes out all-zero is left at zero.
 * Computed directly from A's adjacency lists (not via the block matrix of
 * Eq. 8).  Runs exactly `iters` iterations. */
void orc_hits(int64_t n, const int64_t *a_rowptr, const int32_t *a_col,
              int iters, int norm, double *a, double *h)
{
    double *na = (double *)malloc(sizeof(double) * (size_t)n);
    double *nh = (double *)malloc(sizeof(double) * (size_t)n);
    if (!na || !nh) { free(na); free(nh); return; }
    for (int64_t v = 0; v < n; ++v) { a[v] = 1.0 / (double)n; h[v] = 1.0 / (double)n; }
    for (int it = 0; it < iters; ++it) {
        for (int64_t v = 0; v < n; ++v) na[v] = 0.0;
        for (int64_t u = 0; u < n; ++u) {
            double hu = h[u], s = 0.0;
            for (int64_t e = a_rowptr[u]; e < a_rowptr[u + 1]; ++e) {
                na[a_col[e]] += hu;          /* (A^T h)_v = sum_{u->v} h_u */
                s += a[a_col[e]];            /* (A a)_u   = sum_{u->v} a_v */
            }
            nh[u] = s;
        }
        double sa = 0.0, sh = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            if (norm == 1) { sa += na[v]; sh += nh[v]; }
            else { sa += na[v] * na[v]; sh += nh[v] * nh[v]; }
        }
        if (norm != 1) { sa = sqrt(sa); sh = sqrt(sh); }
        for (int64_t v = 0; v < n; ++v) {
            a[v] = sa > 0 ? na[v] / sa : 0.0;
            h[v] = sh > 0 ? nh[v] / sh : 0.0;
        }
    }
    free(na); free(nh);
}

/* ------------------------------------- differentiable RWR (edge weights) -- */

/* Transition weights from per-edge logits: for every node u, P_e =
 * exp(theta_e) / sum_{e' in out(u)} exp(theta_e') over u's out-edges e
 * (A's CSR order).  Max-shifted for stability; FP64. */
void orc_edge_softmax(int64_t n, const int64_t *a_rowptr, const float *theta,
                      double *P)
{
    for (int64_t u = 0; u < n; ++u) {
        int64_t b = a_rowptr[u], e1 = a_rowptr[u + 1];
        if (b == e1) continue;
        double mx = -INFINITY, s = 0.0;
        for (int64_t e = b; e < e1; ++e) if (theta[e] > mx) mx = theta[e];
        for (int64_t e = b; e < e1; ++e) s += exp((double)theta[e] - mx);
        for (int64_t e = b; e < e1; ++e) P[e] = exp((double)theta[e] - mx) / s;
    }
}

/* RWR with M(v,u) = P_{u->v} (column-stochastic on non-dangling columns), in
 * push form over A: r(k+1) = c (M r(k) + (sum_{u in D} r(k)_u) e_s)
 * + (1-c) e_s, i.e. r = c K r + (1-c) e_s with K = M + e_s 1_D^T.
 * Stops at L1 change < tol or max_iter; returns the iteration count. */
int orc_rwr_weighted(int64_t n, const int64_t *a_rowptr, const int32_t *a_col,
                     const double *P, int64_t s, double c, double tol,
                     int max_iter, double *r)
{
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    if (!q) return -1;
    for (int64_t v = 0; v < n; ++v) r[v] = (v == s) ? 1.0 : 0.0;
    int it = 0;
    while (it < max_iter) {
        double dangling = 0.0;
        for (int64_t v = 0; v < n; ++v) q[v] = 0.0;
        for (int64_t u = 0; u < n; ++u) {
            if (a_rowptr[u] == a_rowptr[u + 1]) { dangling += r[u]; continue; }
            for (int64_t e = a_rowptr[u]; e < a_rowptr[u + 1]; ++e)
                q[a_col[e]] += P[e] * r[u];
        }
        double l1 = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            double nv = c * q[v] + (v == s ? c * dangling + (1.0 - c) : 0.0);
            l1 += fabs(nv - r[v]);
            r[v] = nv;
        }
        ++it;
        if (l1 < tol) break;
    }
    free(q);
    return it;
}

/* Gradient of L(theta) with r the RWR fixed point above and g = dL/dr given.
 * Adjoint fixed point: lambda = c K^T lambda + g, i.e.
 *   lambda_u = c (sum_{e=u->v} P_e lambda_v + [u in D] lambda_s) + g_u,
 * iterated from lambda = g until the L1 change < tol (contraction: K^T is
 * row-stochastic and c < 1).  Edge sensitivities G_e = c lambda_v r_u for
 * e = u->v, and through the softmax
 *   dL/dtheta_e = P_e (G_e - sum_{e' in out(u)} P_e' G_e').
 * Returns the adjoint iteration count. */
int orc_rwr_adjoint(int64_t n, const int64_t *a_rowptr, const int32_t *a_col,
                    const double *P, int64_t s, double c, const double *r,
                    const double *g, double tol, int max_iter, double *lambda,
                    double *dtheta)
{
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    if (!q) return -1;
    for (int64_t v = 0; v < n; ++v) lambda[v] = g[v];
    int it = 0;
    while (it < max_iter) {
        double ls = lambda[s], l1 = 0.0;
        for (int64_t u = 0; u < n; ++u) {
            double acc = 0.0;
            if (a_rowptr[u] == a_rowptr[u + 1]) acc = ls;
            else
                for (int64_t e = a_rowptr[u]; e < a_rowptr[u + 1]; ++e)
                    acc += P[e] * lambda[a_col[e]];
            q[u] = c * acc + g[u];
        }
        for (int64_t u = 0; u < n; ++u) { l1 += fabs(q[u] - lambda[u]); lambda[u] = q[u]; }
        ++it;
        if (l1 < tol) break;
    }
    free(q);
    for (int64_t u = 0; u < n; ++u) {
        double dot = 0.0;
        for (int64_t e = a_rowptr[u]; e < a_rowptr[u + 1]; ++e)
            dot += P[e] * (c * lambda[a_col[e]] * r[u]);
        for (int64_t e = a_rowptr[u]; e < a_rowptr[u + 1]; ++e)
            dtheta[e] = P[e] * (c * lambda[a_col[e]] * r[u] - dot);
    }
    return it;
}

/* ------------------------------------------------ degree reordering -- */

static const int64_t *g_len_for_cmp;

static int cmp_len_desc_id_asc(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    int64_t la = g_len_for_cmp[a], lb = g_len_for_cmp[b];
    if (la != lb) return la > lb ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Section 3.1, Solution 2: order columns by decreasing length.  Reading: ties
 * by ascending id, and the same permutation is applied to rows (symmetric),
 * so x and y share one index space.  inv[k] = node at position k;
 * pi[node] = its position. */
void orc_degree_order(int64_t n, const int64_t *len, int32_t *pi, int32_t *inv)
{
    for (int64_t i = 0; i < n; ++i) inv[i] = (int32_t)i;
    g_len_for_cmp = len;
    qsort(inv, (size_t)n, sizeof(int32_t), cmp_len_desc_id_asc);
    for (int64_t k = 0; k < n; ++k) pi[inv[k]] = (int32_t)k;
}

/* ----------------------------------------------------- Algorithm 1 -- */

/* Algorithm 1 (tile count): columns sorted by decreasing length; keep adding
 * tiles of tile_width columns while the tile count is below n / tile_width
 * (read as floor division, so a partial last tile stays in the sparse part)
 * and the first column of the next tile has length > 1.  Returns NTile; the
 * tiles are [t*tile_width, (t+1)*tile_width) and the sparse part is
 * [NTile*tile_width, n). */
int64_t orc_alg1_tiles(int64_t n, const int64_t *sorted_col_len, int64_t tile_width)
{
    int64_t ntile = 0;
    if (tile_width <= 0) return 0;
    while (ntile < n / tile_width) {
        int64_t start = ntile * tile_width;
        if (sorted_col_len[start] <= 1) break;
        ++ntile;
    }
    return ntile;
}

/* ---------------------------------------------- performance model -- */

/* Lookup table of the offline benchmark (Section 3.3): performance (nnz
 * slots per second with every warp running that shape) for each storage
 * major (0 = row-major, 1 = column-major) and padded shape, bucketed by
 * floor(log2(w_pad)) and floor(log2(h_pad)), each clamped to [0, nlog-1].
 * perf has 2 * nlog * nlog entries: perf[(major * nlog + lw) * nlog + lh]. */
typedef struct {
    int nlog;
    const double *perf;
} orc_table;

static int ilog2_floor(int64_t v)
{
    int l = 0;
    while (v > 1) { v >>= 1; ++l; }
    return l;
}

static double table_perf(const orc_table *t, int major, int64_t wpad, int64_t hpad)
{
    int lw = ilog2_floor(wpad), lh = ilog2_floor(hpad);
    if (lw > t->nlog - 1) lw = t->nlog - 1;
    if (lh > t->nlog - 1) lh = t->nlog - 1;
    return t->perf[((int64_t)major * t->nlog + lw) * t->nlog + lh];
}

static int64_t round_up32(int64_t v) { return (v + 31) / 32 * 32; }

/* Storage decision of Section 3.1, Solution 3 for a w x h workload:
 * rule 0 (the paper): row-major when w >= h, else column-major.
 * rule 1 (GB300 reading): the major with fewer padded slots, column-major
 * on a tie.  Row-major pads w to a multiple of 32, column-major pads h.
 * rules 2 and 3: every workload row-major (CSR-vector) or column-major
 * (ELL) -- the special cases of the composite format named in Section 5. */
static int pick_major(int rule, int64_t w, int64_t h)
{
    if (rule == 0) return w >= h ? 0 : 1;
    if (rule == 2) return 0;
    if (rule == 3) return 1;
    int64_t row_slots = h * round_up32(w), col_slots = round_up32(h) * w;
    return row_slots < col_slots ? 0 : 1;
}

/*
 * Algorithm 3, PM(T, WL): simulate the partition of one tile whose (virtual)
 * row lengths are given in decreasing order, group warps into "iterations"
 * of max_warps warps (Eq. 1), and return t = sum_i Size(i) / P_i (Eqs. 2-5)
 * with P_i the mean table performance of the warps of iteration i.
 * Readings: a workload starting at rank i takes h = max(1, floor(WL / w))
 * rows, w = length of row i, clipped at the rows left; Size and the table
 * lookup use the padded rectangle; the iteration count is that of the warps
 * actually formed.  [GB300 reading] with max_rows > 0 a workload also holds
 * at most max_rows rows (a warp walks its rows' 32-row blocks one after
 * another, so a tall workload of one-entry rows is a long serial chain).
 */
static int64_t wl_rows(int64_t WL, int64_t w, int64_t left, int64_t max_rows)
{
    int64_t h = WL / w;
    if (h < 1) h = 1;
    if (max_rows > 0 && h > max_rows) h = max_rows;
    if (h > left) h = left;
    return h;
}

double orc_alg3_model(int64_t nrows, const int64_t *row_len, int64_t WL,
                      int64_t max_warps, int rule, int nlog, const double *perf,
                      int64_t max_rows)
{
    orc_table t = { nlog, perf };
    if (nrows <= 0) return 0.0;
    int64_t nwarp = 0;
    for (int64_t i = 0; i < nrows; ) {
        i += wl_rows(WL, row_len[i], nrows - i, max_rows);
        ++nwarp;
    }
    int64_t iters = (nwarp + max_warps - 1) / max_warps;
    double *P = (double *)calloc((size_t)iters, sizeof(double));
    double *S = (double *)calloc((size_t)iters, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)iters, sizeof(int64_t));
    int64_t j = 0;
    for (int64_t i = 0; i < nrows; ++j) {
        int64_t w = row_len[i], h = wl_rows(WL, w, nrows - i, max_rows);
        int major = pick_major(rule, w, h);
        int64_t wp = major == 0 ? round_up32(w) : w;
        int64_t hp = major == 0 ? h : round_up32(h);
        int64_t it = j / max_warps;
        P[it] += table_perf(&t, major, wp, hp);
        S[it] += (double)(wp * hp);
        cnt[it] += 1;
        i += h;
    }
    double total = 0.0;
    for (int64_t it = 0; it < iters; ++it) {
        double pi = P[it] / (double)cnt[it];
        total += S[it] / pi;
    }
    free(P); free(S); free(cnt);
    return total;
}

/* Algorithm 2, Partition(T): WL runs from the longest row upward in steps of
 * the longest row while WL <= nnz / max_warps; keep the first WL with the
 * smallest modelled time.  Reading: if that range is empty, WL = the longest
 * row.  Returns WL; *best_time gets its modelled time. */
int64_t orc_alg2_partition(int64_t nrows, const int64_t *row_len, int64_t nnz,
                           int64_t max_warps, int rule, int nlog,
                           const double *perf, double *best_time, int64_t max_rows)
{
    if (nrows <= 0) { if (best_time) *best_time = 0.0; return 0; }
    int64_t low = row_len[0];
    int64_t opt = 0;
    double opt_t = INFINITY;
    for (int64_t WL = low; WL * max_warps <= nnz; WL += low) {
        double t = orc_alg3_model(nrows, row_len, WL, max_warps, rule, nlog, perf, max_rows);
        if (t < opt_t) { opt_t = t; opt = WL; }
    }
    if (opt == 0) {
        opt = low;
        opt_t = orc_alg3_model(nrows, row_len, low, max_warps, rule, nlog, perf, max_rows);
    }
    if (best_time) *best_time = opt_t;
    return opt;
}

/*
 * Section 3.1, Solution 3 on one tile, given the tile's rows as (row id,
 * length) pairs.  Steps, in the paper's order:
 *   1. rank rows by length, high to low (reading: ties by ascending row id);
 *   2. [GB300 reading] a row longer than `heavy` is cut into chunks of
 *      `heavy` entries (the last one shorter), which enter the ranking as
 *      virtual rows (ties: row id, then chunk index); heavy <= 0 disables it;
 *   3. WL = wl if wl > 0, else Algorithm 2 over the virtual row lengths;
 *   4. pack: a workload starting at rank i has w = length of row i and
 *      h = max(1, floor(WL / w)) rows (clipped at the rows left and, when
 *      max_rows > 0, at max_rows), stored by pick_major().
 * Rows of length 0 are not part of any workload.
 * Outputs: rank_row[k], rank_chunk[k], rank_len[k] for k < *nvirt, and per
 * workload wl_first[j] (rank of its first row), wl_h[j], wl_w[j],
 * wl_major[j] for j < *nwl.  Arrays must hold nnz-bounded sizes (callers
 * pass capacity >= number of virtual rows).  Returns the chosen WL.
 */
static const int64_t *g_vlen, *g_vrow, *g_vchunk;

static int cmp_virtual(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    if (g_vlen[a] != g_vlen[b]) return g_vlen[a] > g_vlen[b] ? -1 : 1;
    if (g_vrow[a] != g_vrow[b]) return g_vrow[a] < g_vrow[b] ? -1 : 1;
    if (g_vchunk[a] != g_vchunk[b]) return g_vchunk[a] < g_vchunk[b] ? -1 : 1;
    return 0;
}

int64_t orc_partition_tile(int64_t nrows, const int64_t *row_id,
                           const int64_t *row_len, int64_t heavy, int64_t wl,
                           int64_t max_warps, int rule, int nlog,
                           const double *perf, int64_t *nvirt_out,
                           int64_t *rank_row, int64_t *rank_chunk,
                           int64_t *rank_len, int64_t *nwl_out,
                           int64_t *wl_first, int64_t *wl_h, int64_t *wl_w,
                           int64_t *wl_major, int64_t max_rows)
{
    int64_t nv = 0, nnz = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t L = row_len[r];
        if (L <= 0) continue;
        nnz += L;
        nv += (heavy > 0 && L > heavy) ? (L + heavy - 1) / heavy : 1;
    }
    int64_t *vlen = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv + 1));
    int64_t *vrow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv + 1));
    int64_t *vchunk = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv + 1));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv + 1));
    int64_t k = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t L = row_len[r];
        if (L <= 0) continue;
        if (heavy > 0 && L > heavy) {
            int64_t nch = (L + heavy - 1) / heavy;
            for (int64_t ch = 0; ch < nch; ++ch) {
                vlen[k] = (ch < nch - 1) ? heavy : L - heavy * (nch - 1);
                vrow[k] = row_id[r]; vchunk[k] = ch; ++k;
            }
        } else {
            vlen[k] = L; vrow[k] = row_id[r]; vchunk[k] = 0; ++k;
        }
    }
    for (int64_t i = 0; i < nv; ++i) order[i] = i;
    g_vlen = vlen; g_vrow = vrow; g_vchunk = vchunk;
    qsort(order, (size_t)nv, sizeof(int64_t), cmp_virtual);
    for (int64_t i = 0; i < nv; ++i) {
        rank_row[i] = vrow[order[i]];
        rank_chunk[i] = vchunk[order[i]];
        rank_len[i] = vlen[order[i]];
    }
    *nvirt_out = nv;
    int64_t WL = wl > 0 ? wl
        : orc_alg2_partition(nv, rank_len, nnz, max_warps, rule, nlog, perf, NULL, max_rows);
    int64_t j = 0;
    for (int64_t i = 0; i < nv; ++j) {
        int64_t w = rank_len[i], h = wl_rows(WL, w, nv - i, max_rows);
        wl_first[j] = i; wl_h[j] = h; wl_w[j] = w;
        wl_major[j] = pick_major(rule, w, h);
        i += h;
    }
    *nwl_out = j;
    free(vlen); free(vrow); free(vchunk); free(order);
    return WL;
}

/* ------------------------------------------- bitonic row partition -- */

/* Section 3.2: rows sorted by length (decreasing; reading: ties by ascending
 * id) are dealt to P parts in rounds of P; the part that received the
 * longest row of one round receives the shortest row of the next, i.e. the
 * dealing direction alternates every round.  part[row] gets the part id. */
void orc_bitonic_partition(int64_t n, const int64_t *row_len, int P,
                           int32_t *part)
{
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *dummy = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    orc_degree_order(n, row_len, dummy, order);
    for (int64_t k = 0; k < n; ++k) {
        int64_t round = k / P, pos = k % P;
        int32_t p = (int32_t)((round % 2 == 0) ? pos : P - 1 - pos);
        part[order[k]] = p;
    }
    free(order); free(dummy);
}

/* ------------------------------------------- heavy-row threshold tuning -- */

/* [GB300 reading, not in the paper] The paper's lower bound WL >= longest row
 * leaves one warp with a whole hub row.  The split threshold H is picked by
 * the same model: base = max(32, ceil(nnz / max_warps)) rounded up to a
 * multiple of 32; candidates H_k = round_up32(ceil(base / 2^k)), k = 0..3
 * (duplicates skipped, never below 32).  For each, the tile's virtual rows
 * are ranked, WL comes from Algorithm 2, and the cost is the modelled time
 * plus split_cost seconds per chunk of a split row.  The first candidate with
 * the smallest cost wins.  Returns H; *wl_out gets its WL. */
double orc_split_cost_chunks(int64_t nrows, const int64_t *row_len, int64_t H)
{
    double chunks = 0.0;
    for (int64_t r = 0; r < nrows; ++r)
        if (row_len[r] > H) chunks += (double)((row_len[r] + H - 1) / H);
    return chunks;
}

int64_t orc_tune_heavy(int64_t nrows, const int64_t *row_id,
                       const int64_t *row_len, int64_t max_warps, int rule,
                       int nlog, const double *perf, double split_cost,
                       int64_t *wl_out, int64_t max_rows)
{
    int64_t nnz = 0, nv_cap = 0;
    for (int64_t r = 0; r < nrows; ++r)
        if (row_len[r] > 0) { nnz += row_len[r]; nv_cap += 1 + row_len[r] / 32; }
    if (nnz == 0) { if (wl_out) *wl_out = 0; return 32; }
    int64_t base = (nnz + max_warps - 1) / max_warps;
    if (base < 32) base = 32;
    base = round_up32(base);
    int64_t *rr = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv_cap);
    int64_t *rc = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv_cap);
    int64_t *rl = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv_cap);
    int64_t *f = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv_cap);
    int64_t *hh = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv_cap);
    int64_t *ww = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv_cap);
    int64_t *mm = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv_cap);
    int64_t bestH = base, bestWL = 0, prevH = -1;
    double best = INFINITY;
    for (int k = 0; k < 4; ++k) {
        int64_t div = (int64_t)1 << k;
        int64_t H = round_up32((base + div - 1) / div);
        if (H < 32) H = 32;
        if (H == prevH) continue;
        prevH = H;
        int64_t nv = 0, nwl = 0;
        int64_t WL = orc_partition_tile(nrows, row_id, row_len, H, 0, max_warps,
                                        rule, nlog, perf, &nv, rr, rc, rl, &nwl,
                                        f, hh, ww, mm, max_rows);
        double t = orc_alg3_model(nv, rl, WL, max_warps, rule, nlog, perf, max_rows) +
                   split_cost * orc_split_cost_chunks(nrows, row_len, H);
        if (t < best) { best = t; bestH = H; bestWL = WL; }
    }
    free(rr); free(rc); free(rl); free(f); free(hh); free(ww); free(mm);
    if (wl_out) *wl_out = bestWL;
    return bestH;
}
