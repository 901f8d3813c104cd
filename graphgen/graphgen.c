/*
 * graphgen.c -- seeded synthetic graph inputs (R-MAT, Chung-Lu) and seeded
 * random vectors.
 *
 * This module produces INPUTS only: the adjacency structure A of a directed
 * graph (CSR by source node, columns sorted, duplicates and self-loops
 * removed) and uniform / normal random vectors.  It holds none of the SpMV
 * method's arithmetic (no 1/outdeg values, no reordering, no tiling); both the
 * CUDA path and the FP64 oracle read what it produces.
 *
 * Random numbers come from a counter-based generator: the SplitMix64 output
 * function (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) applied to a key derived from (seed, stream,
 * counter).  Every draw depends only on its counter, so the output is
 * identical for any thread count.
 *
 * R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): every edge descends
 * `scale` levels of the adjacency matrix; at each level one quadrant is chosen
 * with probabilities (a, b, c, d), where the quadrant's row half gives the
 * source bit and its column half the destination bit.
 *
 * Chung-Lu (Chung and Lu 2002): node i carries an expected degree w_i; each of
 * m edges draws its source and its destination independently with
 * probability proportional to w (Walker/Vose alias method).
 *
 * Plain C11 + pthreads; no architecture-specific code, so it builds and gives
 * the same results on x86-64 and aarch64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

/* ------------------------------------------------------------------ RNG -- */

static inline uint64_t gg_mix64(uint64_t z)
{
    /* SplitMix64 output function (published constants). */
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* One 64-bit draw for (seed, stream, counter).  The SplitMix64 state after
 * `ctr+1` steps from a state keyed by (seed, stream) is
 * key + (ctr+1)*golden; the draw is the output function of that state. */
uint64_t gg_rand64(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    const uint64_t golden = 0x9e3779b97f4a7c15ULL;
    uint64_t key = gg_mix64(seed * golden + 0x632be59bd9b4e019ULL) ^
                   gg_mix64(stream + 0x3c6ef372fe94f82aULL);
    return gg_mix64(key + (ctr + 1) * golden);
}

/* Streams: each generator uses its own stream id so draws never collide. */
enum { ST_RMAT = 1, ST_CL_SRC = 2, ST_CL_DST = 3, ST_PERM = 4,
       ST_UNIFORM = 5, ST_NORMAL = 6 };

/* --------------------------------------------------------- threading -- */

typedef struct {
    void (*fn)(void *ctx, int64_t lo, int64_t hi, int tid);
    void *ctx;
    int64_t lo, hi;
    int tid;
} gg_job;

static void *gg_job_main(void *p)
{
    gg_job *j = (gg_job *)p;
    j->fn(j->ctx, j->lo, j->hi, j->tid);
    return NULL;
}

/* Split [0, n) into nthreads contiguous chunks and run fn on each. */
static void gg_parallel(int nthreads, int64_t n,
                        void (*fn)(void *, int64_t, int64_t, int), void *ctx)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < 65536 || nthreads == 1) { fn(ctx, 0, n, 0); return; }
    pthread_t th[256];
    gg_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].tid = t;
        jobs[t].lo = n * t / nthreads; jobs[t].hi = n * (t + 1) / nthreads;
    }
    int started[256];
    for (int t = 1; t < nthreads; ++t)
        started[t] = pthread_create(&th[t], NULL, gg_job_main, &jobs[t]) == 0;
    gg_job_main(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) {
        if (started[t]) pthread_join(th[t], NULL);
        else gg_job_main(&jobs[t]);          /* could not spawn: run inline */
    }
}

/* -------------------------------------------------------------- R-MAT -- */

typedef struct {
    int scale;
    uint32_t ta, tab, tabc;   /* cumulative thresholds on 32-bit draws */
    uint64_t seed;
    uint32_t *src, *dst;
} rmat_ctx;

static void rmat_body(void *p, int64_t lo, int64_t hi, int tid)
{
    (void)tid;
    rmat_ctx *c = (rmat_ctx *)p;
    for (int64_t e = lo; e < hi; ++e) {
        uint32_t s = 0, d = 0;
        uint64_t r = 0;
        for (int l = 0; l < c->scale; ++l) {
            uint32_t u;
            if ((l & 1) == 0) {
                r = gg_rand64(c->seed, ST_RMAT, (uint64_t)e * 32u + (uint64_t)(l >> 1));
                u = (uint32_t)(r >> 32);
            } else {
                u = (uint32_t)r;
            }
            uint32_t sb, db;
            if (u < c->ta)        { sb = 0; db = 0; }
            else if (u < c->tab)  { sb = 0; db = 1; }
            else if (u < c->tabc) { sb = 1; db = 0; }
            else                  { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        c->src[e] = s;
        c->dst[e] = d;
    }
}

/* Generate m R-MAT edges over 2^scale nodes (duplicates/self-loops kept). */
int gg_rmat_edges(int scale, int64_t m, double a, double b, double c,
                  uint64_t seed, int nthreads, uint32_t *src, uint32_t *dst)
{
    if (scale < 1 || scale > 31 || m < 0 || a < 0 || b < 0 || c < 0 ||
        a + b + c > 1.0)
        return -1;
    rmat_ctx ctx;
    ctx.scale = scale; ctx.seed = seed; ctx.src = src; ctx.dst = dst;
    const double two32 = 4294967296.0;
    double fa = a * two32, fab = (a + b) * two32, fabc = (a + b + c) * two32;
    ctx.ta = fa >= two32 ? 0xffffffffu : (uint32_t)fa;
    ctx.tab = fab >= two32 ? 0xffffffffu : (uint32_t)fab;
    ctx.tabc = fabc >= two32 ? 0xffffffffu : (uint32_t)fabc;
    gg_parallel(nthreads, m, rmat_body, &ctx);
    return 0;
}

/* ----------------------------------------------------------- Chung-Lu -- */

/* Expected degrees w_i = min(dmax, C*(i+1)^(-1/(gamma-1))), with C found by
 * bisection so that sum(w) = m.  Writes w[0..n).  Returns C, or -1. */
double gg_chung_lu_weights(int64_t n, double m, double gamma, double dmax,
                           double *w)
{
    if (n < 1 || !(gamma > 1.0) || !(dmax > 0) || !(m > 0)) return -1.0;
    const double beta = 1.0 / (gamma - 1.0);
    for (int64_t i = 0; i < n; ++i) w[i] = pow((double)(i + 1), -beta);
    double lo = 0.0, hi = 1.0;
    /* grow hi until the capped sum reaches m (or every weight is capped) */
    for (int it = 0; it < 200; ++it) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) { double v = hi * w[i]; s += v < dmax ? v : dmax; }
        if (s >= m || hi * w[n - 1] >= dmax) break;
        lo = hi; hi *= 2.0;
    }
    for (int it = 0; it < 100; ++it) {
        double mid = 0.5 * (lo + hi), s = 0.0;
        for (int64_t i = 0; i < n; ++i) { double v = mid * w[i]; s += v < dmax ? v : dmax; }
        if (s < m) lo = mid; else hi = mid;
        if (hi - lo <= 1e-12 * hi) break;
    }
    double C = 0.5 * (lo + hi);
    for (int64_t i = 0; i < n; ++i) { double v = C * w[i]; w[i] = v < dmax ? v : dmax; }
    return C;
}

/* Vose alias table over weights w[0..n): prob[i] in [0,1], alias[i]. */
int gg_alias_table(int64_t n, const double *w, double *prob, uint32_t *alias)
{
    if (n < 1) return -1;
    double sum = 0.0;
    for (int64_t i = 0; i < n; ++i) sum += w[i];
    if (!(sum > 0)) return -1;
    int64_t *small = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *large = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!small || !large) { free(small); free(large); return -2; }
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; ++i) {
        prob[i] = w[i] * (double)n / sum;
        alias[i] = (uint32_t)i;
        if (prob[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        int64_t s = small[--ns], l = large[--nl];
        alias[s] = (uint32_t)l;
        prob[l] = (prob[l] + prob[s]) - 1.0;
        if (prob[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) prob[large[--nl]] = 1.0;
    while (ns > 0) prob[small[--ns]] = 1.0;
    free(small); free(large);
    return 0;
}

typedef struct {
    int64_t n;
    const double *prob;
    const uint32_t *alias;
    uint64_t seed;
    uint32_t *src, *dst;
} cl_ctx;

static inline uint32_t cl_draw(const cl_ctx *c, uint64_t r)
{
    /* high 32 bits pick the column, low 32 bits the coin */
    uint64_t i = ((r >> 32) * (uint64_t)c->n) >> 32;
    double coin = (double)(uint32_t)r * (1.0 / 4294967296.0);
    return coin < c->prob[i] ? (uint32_t)i : c->alias[i];
}

static void cl_body(void *p, int64_t lo, int64_t hi, int tid)
{
    (void)tid;
    cl_ctx *c = (cl_ctx *)p;
    for (int64_t e = lo; e < hi; ++e) {
        c->src[e] = cl_draw(c, gg_rand64(c->seed, ST_CL_SRC, (uint64_t)e));
        c->dst[e] = cl_draw(c, gg_rand64(c->seed, ST_CL_DST, (uint64_t)e));
    }
}

int gg_chung_lu_edges(int64_t n, int64_t m, const double *prob,
                      const uint32_t *alias, uint64_t seed, int nthreads,
                      uint32_t *src, uint32_t *dst)
{
    if (n < 1 || n > 0xffffffffLL || m < 0) return -1;
    cl_ctx ctx = { n, prob, alias, seed, src, dst };
    gg_parallel(nthreads, m, cl_body, &ctx);
    return 0;
}

/* ------------------------------------------------------- permutation -- */

/* Seeded uniform random permutation of [0, n) (Fisher-Yates, Durstenfeld). */
int gg_random_permutation(int64_t n, uint64_t seed, uint32_t *perm)
{
    if (n < 0 || n > 0xffffffffLL) return -1;
    for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        uint64_t r = gg_rand64(seed, ST_PERM, (uint64_t)i);
        /* multiply-shift bounded draw in [0, i] */
        uint64_t j = (uint64_t)(((__uint128_t)r * (uint64_t)(i + 1)) >> 64);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    return 0;
}

/* ------------------------------------------- edges -> CSR (dedup) -- */

#define RADIX_BITS 11
#define RADIX_SIZE (1 << RADIX_BITS)

typedef struct {
    const uint32_t *src, *dst, *relabel;
    uint64_t *keys;
    int idbits;
} pack_ctx;

static void pack_body(void *p, int64_t lo, int64_t hi, int tid)
{
    (void)tid;
    pack_ctx *c = (pack_ctx *)p;
    for (int64_t e = lo; e < hi; ++e) {
        uint64_t s = c->src[e], d = c->dst[e];
        if (c->relabel) { s = c->relabel[s]; d = c->relabel[d]; }
        c->keys[e] = (s << c->idbits) | d;   /* source-major packed key */
    }
}

typedef struct {
    const uint64_t *in;
    uint64_t *out;
    int shift;
    int nthreads;
    int64_t n;
    int64_t (*hist)[RADIX_SIZE];
} radix_ctx;

static void radix_hist(void *p, int64_t lo, int64_t hi, int tid)
{
    radix_ctx *c = (radix_ctx *)p;
    int64_t *h = c->hist[tid];
    memset(h, 0, sizeof(int64_t) * RADIX_SIZE);
    for (int64_t i = lo; i < hi; ++i) h[(c->in[i] >> c->shift) & (RADIX_SIZE - 1)]++;
}

static void radix_scatter(void *p, int64_t lo, int64_t hi, int tid)
{
    radix_ctx *c = (radix_ctx *)p;
    int64_t *h = c->hist[tid];           /* holds start offsets now */
    for (int64_t i = lo; i < hi; ++i) {
        uint64_t k = c->in[i];
        c->out[h[(k >> c->shift) & (RADIX_SIZE - 1)]++] = k;
    }
}

/* Stable LSD radix sort of keys over their low `bits` bits; result in keys. */
static int gg_radix_sort(uint64_t *keys, int64_t n, int bits, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < 65536) nthreads = 1;
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    int64_t (*hist)[RADIX_SIZE] = malloc(sizeof(int64_t) * RADIX_SIZE * (size_t)nthreads);
    if (!tmp || !hist) { free(tmp); free(hist); return -2; }
    uint64_t *in = keys, *out = tmp;
    for (int shift = 0; shift < bits; shift += RADIX_BITS) {
        radix_ctx c = { in, out, shift, nthreads, n, hist };
        gg_parallel(nthreads, n, radix_hist, &c);
        int64_t run = 0;
        for (int d = 0; d < RADIX_SIZE; ++d)
            for (int t = 0; t < nthreads; ++t) {
                int64_t v = hist[t][d]; hist[t][d] = run; run += v;
            }
        gg_parallel(nthreads, n, radix_scatter, &c);
        uint64_t *sw = in; in = out; out = sw;
    }
    if (in != keys) memcpy(keys, in, sizeof(uint64_t) * (size_t)n);
    free(tmp); free(hist);
    return 0;
}

/*
 * Edge list -> CSR of A (rows = source).  Optionally relabels both endpoints
 * through `relabel` (new = relabel[old]).  Removes self-loops and duplicate
 * edges (one kept).  Columns within a row come out sorted ascending.
 * rowptr has n+1 entries; col must hold m entries.  Returns nnz, or <0.
 */
int64_t gg_edges_to_csr(int64_t n, int64_t m, const uint32_t *src,
                        const uint32_t *dst, const uint32_t *relabel,
                        int nthreads, int64_t *rowptr, uint32_t *col)
{
    if (n < 1 || n > 0xffffffffLL || m < 0) return -1;
    for (int64_t e = 0; e < m; ++e)
        if ((int64_t)src[e] >= n || (int64_t)dst[e] >= n) return -1;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
    if (!keys) return -2;
    int idbits = 1;
    while (((int64_t)1 << idbits) < n) ++idbits;
    /* sort the packed key (src << idbits | dst) over its 2*idbits bits */
    pack_ctx pc = { src, dst, relabel, keys, idbits };
    gg_parallel(nthreads, m, pack_body, &pc);
    int rc = gg_radix_sort(keys, m, 2 * idbits, nthreads);
    if (rc) { free(keys); return rc; }
    const uint64_t dmask = ((uint64_t)1 << idbits) - 1;
    for (int64_t i = 0; i <= n; ++i) rowptr[i] = 0;
    int64_t nnz = 0;
    uint64_t prev = ~(uint64_t)0;
    for (int64_t e = 0; e < m; ++e) {
        uint64_t k = keys[e];
        if (k == prev) continue;
        prev = k;
        uint64_t s = k >> idbits, d = k & dmask;
        if (s == d) continue;
        col[nnz++] = (uint32_t)d;
        rowptr[s + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
    free(keys);
    return nnz;
}

/* --------------------------------------------------------- vectors -- */

/* U[0,1) float32: 24 random bits, exactly representable. */
void gg_uniform_f32(uint64_t seed, int64_t n, float *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = (float)(gg_rand64(seed, ST_UNIFORM, (uint64_t)i) >> 40) *
                 (1.0f / 16777216.0f);
}

/* N(0,1) float32 by the Box-Muller transform on two 53-bit uniforms. */
void gg_normal_f32(uint64_t seed, int64_t n, float *out)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t r1 = gg_rand64(seed, ST_NORMAL, 2 * (uint64_t)i);
        uint64_t r2 = gg_rand64(seed, ST_NORMAL, 2 * (uint64_t)i + 1);
        double u1 = ((double)(r1 >> 11) + 1.0) * (1.0 / 9007199254740992.0); /* (0,1] */
        double u2 = (double)(r2 >> 11) * (1.0 / 9007199254740992.0);         /* [0,1) */
        out[i] = (float)(sqrt(-2.0 * log(u1)) * cos(two_pi * u2));
    }
}

uint64_t gg_rand64_export(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    return gg_rand64(seed, stream, ctr);
}
