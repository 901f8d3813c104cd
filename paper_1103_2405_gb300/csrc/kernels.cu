// kernels.cu -- sm_103a kernels of the tiled composite SpMV/SpMM and the
// power-iteration epilogues (Yang, Parthasarathy, Sadayappan: Section 3.1
// Solution 3 for the workload kernels, Appendix F Eqs. 6-9 for the epilogues,
// Appendix B for the plain CSR-scalar / CSR-vector baselines).
//
// Design on GB300: the gather of x is the only reused stream, so x goes
// through the read-only path (__ldg: L1 + L2) and the matrix slots stream
// with evict-first loads (__ldcs) so they do not displace x.  One warp owns
// one workload; row-major workloads reduce with warp shuffles (tree order),
// column-major ones keep one row per lane.  No atomics touch y: every row has
// exactly one writer per part; rows cut into chunks are combined by the last
// chunk to finish, summing the chunk partials in chunk order (deterministic).
// No tensor cores: the gather is not a dense contraction.
#include <atomic>
#include <climits>
#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#include "kernels.h"

namespace spg {

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t k) { g_launches.fetch_add(k); }
int64_t launch_count() { return g_launches.load(); }

constexpr unsigned kFull = 0xffffffffu;
// Grid of a grid-stride elementwise kernel: one thread per element up to
// 64 blocks of 256 per SM.
static inline int grid_for(int64_t n, int per = 256)
{
    int64_t g = (n + per - 1) / per;
    if (g > 152 * 64) g = 152 * 64;
    return (int)(g > 0 ? g : 1);
}
// Resident blocks per SM of the plain one-warp-per-workload kernel (option
// 2): the gather is latency bound, so occupancy is what keeps enough loads
// in flight.
#ifndef SPG_PART_MINB
#define SPG_PART_MINB 6
#endif
constexpr int kPartMinBlocks = SPG_PART_MINB;
// Staged variant: one 32-warp block per SM sharing up to kStagedMaxCols
// floats (192 KB) of x in shared memory.
constexpr int kStagedBlock = 1024;
// Persistent plain variant: 8-warp blocks, kPersistMinBlocks per SM, no x
// slice -- more resident warps (more slot loads in flight) than the staged
// kernel's one 32-warp block.
// Blocks per SM: 5 (48 registers) for the plain SpMV, whose loop needs no
// more; 4 (64 registers, no spills) for the power-iteration epilogues --
// measured best for each (R-MAT 22 PageRank iteration 0.192 ms at 4 vs
// 0.198 at 5; banded SpMV 0.230 ms at 5 vs 0.240 at 4).
constexpr int kPersistMinBlocks = 5;
__host__ __device__ constexpr int persist_minb(int mode)
{
    return (mode == EPI_RAW || mode == EPI_RAW_PAT) ? kPersistMinBlocks : 4;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Per-thread running sum of the epilogue terms (L1 change, dangling mass,
// HITS norms) as an unevaluated float pair s + c, each step Knuth's
// TwoSum: the rounding error of s + a is carried in c.  Accurate to about
// 2^-44 relative over the few thousand terms a thread adds, i.e. as good as
// an FP64 running sum here, in FP32 arithmetic: GB300's FP64 rate is a small
// fraction of its FP32 rate, and per-row FP64 adds and conversions were a
// visible part of the epilogue time.  Converted to FP64 once per thread for
// the warp / block reductions.
struct FSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a)
    {
        const float t = s + a;
        const float bp = t - s;
        c += (s - (t - bp)) + (a - bp);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};


// Uniform per-launch epilogue parameters, read once from the state.
struct Epi {
    float c, base, tele;
    int seed;
    int64_t dstart;
    float sc[2];
    int hnorm;
    const float *aux;
    const int32_t *gid;
    const float *gbase;
    float xs;            // adjoint: x[seed] of the current launch
    float *znew;         // pattern-only PageRank: z of the new iterate
    const float *invdeg;
};

template <int MODE>
__device__ __forceinline__ Epi load_epi(const IterState *st)
{
    Epi E;
    E.c = 1.f; E.base = 0.f; E.tele = 0.f; E.seed = -1; E.dstart = 0;
    E.sc[0] = E.sc[1] = 1.f; E.hnorm = 2; E.aux = nullptr; E.gid = nullptr; E.gbase = nullptr;
    E.xs = 0.f; E.znew = nullptr; E.invdeg = nullptr;
    if (MODE == EPI_BATCH) {
        E.c = (float)st->c;
        E.gid = st->gid;
        E.gbase = st->gbase;
    } else if (MODE == EPI_ADJ) {
        E.c = (float)st->c;
        E.seed = st->seed;
        E.aux = st->aux;
    } else if (MODE == EPI_PAGERANK || MODE == EPI_RWR || MODE == EPI_PR_PAT) {
        const double c = st->c, d = st->delta;
        E.c = (float)c;
        E.dstart = st->dangling_start;
        if (MODE == EPI_PR_PAT) {
            E.znew = st->zbuf[st->parity ^ 1];
            E.invdeg = st->inv_deg;
        }
        if (MODE != EPI_RWR) E.base = (float)((c * d + (1.0 - c)) * st->inv_n);
        else { E.tele = (float)(c * d + (1.0 - c)); E.seed = st->seed; }
    } else if (MODE == EPI_HITS) {
        E.sc[0] = (float)st->scale[0];
        E.sc[1] = (float)st->scale[1];
        E.hnorm = st->hits_norm;
    }
    return E;
}

// Final value of row v from its total, written to y; sums for the check.
template <int MODE>
__device__ __forceinline__ void epilogue(const Epi &E, uint32_t rid, float tot,
                                         const float *__restrict__ x, float *__restrict__ y,
                                         FSum &r0, FSum &r1)
{
    const uint32_t v = rid & kRowIdMask;
    if (rid & kRowNotFirst) tot += y[v];
    if (rid & kRowNotLast) { y[v] = tot; return; }
    if (MODE == EPI_RAW || MODE == EPI_RAW_PAT) {
        y[v] = tot;
    } else if (MODE == EPI_PAGERANK || MODE == EPI_RWR || MODE == EPI_PR_PAT) {
        float add = MODE != EPI_RWR ? E.base : ((int)v == E.seed ? E.tele : 0.f);
        float f = fmaf(E.c, tot, add);
        y[v] = f;
        if (MODE == EPI_PR_PAT) E.znew[v] = f * __ldg(E.invdeg + v);
        r0.add(fabsf(f - x[v]));
        if ((int64_t)v >= E.dstart) r1.add(f);
    } else if (MODE == EPI_BATCH) {
        y[v] = fmaf(E.c, tot, __ldg(E.gbase + __ldg(E.gid + v)));
    } else if (MODE == EPI_ADJ) {
        // lambda = c K^T lambda + g with K^T = M^T + 1_D e_s^T: dangling rows
        // (class bit) also receive c * lambda_s
        const float add = (rid & kRowClass) ? E.c * x[E.seed] : 0.f;
        const float f = fmaf(E.c, tot, add + __ldg(E.aux + v));
        y[v] = f;
        r0.add(fabsf(f - x[v]));
    } else {  // HITS: a-rows read the hub half and vice versa
        const int cls = (rid & kRowClass) ? 1 : 0;
        float f = tot * (cls ? E.sc[0] : E.sc[1]);
        y[v] = f;
        const float q = E.hnorm == 2 ? f * f : f;
        if (cls == 0) r0.add(q); else r1.add(q);
    }
}

// A chunk of a split row: publish the partial; the last chunk to arrive sums
// all partials in chunk order and finishes the row.
template <int MODE>
__device__ __forceinline__ void finish_split(const Epi &E, const SplitView &sv, double2 *red,
                                          uint32_t rid, float acc, const float *__restrict__ x,
                                          float *__restrict__ y)
{
    const int slot = (int)(rid & 0x7fffffffu);
    sv.partial[slot] = acc;
    __threadfence();
    const int s = sv.slot_owner[slot];
    const SplitRow sr = sv.rows[s];
    const unsigned prev = atomicAdd(sv.counter + s, 1u);
    if (prev != (unsigned)sr.nchunks - 1) return;
    __threadfence();
    float tot = 0.f;
    for (int k = 0; k < sr.nchunks; ++k) tot += __ldcg(sv.partial + sr.first_slot + k);
    sv.counter[s] = 0u;
    FSum r0, r1;
    epilogue<MODE>(E, sr.row, tot, x, y, r0, r1);
    if (MODE != EPI_RAW && MODE != EPI_RAW_PAT && MODE != EPI_BATCH)
        red[sv.red_split_base + sr.red_slot] = make_double2(r0.value(), r1.value());
}


// What a row's epilogue reads besides its sum, fetched before the sum is
// computed so the loads overlap the slot stream: the row entry, y_v (rows
// continued from an earlier part), x_v (the L1 change), and the per-row
// additive term of the adjoint / batch epilogues.
struct RowPre {
    uint32_t rid;
    float yv, xv, av;
};

template <int MODE>
__device__ __forceinline__ RowPre prefetch_row(const Epi &E, const uint32_t *__restrict__ rows,
                                               int i, bool valid, const float *__restrict__ x,
                                               const float *__restrict__ y)
{
    RowPre p{0u, 0.f, 0.f, 0.f};
    if (!valid) return p;
    p.rid = __ldg(rows + i);
    if (p.rid & kRowSplit) return p;
    const uint32_t v = p.rid & kRowIdMask;
    if (p.rid & kRowNotFirst) p.yv = y[v];
    if (!(p.rid & kRowNotLast)) {
        if (MODE == EPI_PAGERANK || MODE == EPI_RWR || MODE == EPI_ADJ || MODE == EPI_PR_PAT) p.xv = x[v];
        if (MODE == EPI_PR_PAT) p.av = __ldg(E.invdeg + v);
        if (MODE == EPI_ADJ) p.av = __ldg(E.aux + v);
        if (MODE == EPI_BATCH) p.av = __ldg(E.gbase + __ldg(E.gid + v));
    }
    return p;
}

__device__ __forceinline__ RowPre shfl_row(const RowPre &p, int src)
{
    RowPre q;
    q.rid = __shfl_sync(kFull, p.rid, src);
    q.yv = __shfl_sync(kFull, p.yv, src);
    q.xv = __shfl_sync(kFull, p.xv, src);
    q.av = __shfl_sync(kFull, p.av, src);
    return q;
}

// The epilogue of a row whose extra operands were prefetched (same
// arithmetic as epilogue()).
template <int MODE>
__device__ __forceinline__ void epilogue_pre(const Epi &E, const RowPre &p, float tot,
                                             float *__restrict__ y, FSum &r0, FSum &r1)
{
    const uint32_t rid = p.rid, v = rid & kRowIdMask;
    if (rid & kRowNotFirst) tot += p.yv;
    if (rid & kRowNotLast) { y[v] = tot; return; }
    if (MODE == EPI_RAW || MODE == EPI_RAW_PAT) {
        y[v] = tot;
    } else if (MODE == EPI_PAGERANK || MODE == EPI_RWR || MODE == EPI_PR_PAT) {
        float add = MODE != EPI_RWR ? E.base : ((int)v == E.seed ? E.tele : 0.f);
        float f = fmaf(E.c, tot, add);
        y[v] = f;
        if (MODE == EPI_PR_PAT) E.znew[v] = f * p.av;
        r0.add(fabsf(f - p.xv));
        if ((int64_t)v >= E.dstart) r1.add(f);
    } else if (MODE == EPI_BATCH) {
        y[v] = fmaf(E.c, tot, p.av);
    } else if (MODE == EPI_ADJ) {
        const float add = (rid & kRowClass) ? E.c * E.xs : 0.f;
        const float f = fmaf(E.c, tot, add + p.av);
        y[v] = f;
        r0.add(fabsf(f - p.xv));
    } else {
        const int cls = (rid & kRowClass) ? 1 : 0;
        float f = tot * (cls ? E.sc[0] : E.sc[1]);
        y[v] = f;
        const float q = E.hnorm == 2 ? f * f : f;
        if (cls == 0) r0.add(q); else r1.add(q);
    }
}

template <int MODE>
__device__ __forceinline__ void finish_row_pre(const Epi &E, const SplitView &sv, double2 *red,
                                               const RowPre &p, float acc,
                                               const float *__restrict__ x, float *__restrict__ y,
                                               FSum &r0, FSum &r1)
{
    if (p.rid & kRowSplit) finish_split<MODE>(E, sv, red, p.rid, acc, x, y);
    else epilogue_pre<MODE>(E, p, acc, y, r0, r1);
}

template <int MODE>
__device__ __forceinline__ void block_reduce_store(const FSum &f0, const FSum &f1, double2 *out)
{
    double r0 = f0.value(), r1 = f1.value();
    __shared__ double s0[32], s1[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    r0 = warp_sum_d(r0);
    r1 = warp_sum_d(r1);
    if (lane == 0) { s0[warp] = r0; s1[warp] = r1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        const int nw = blockDim.x >> 5;
        for (int w = 0; w < nw; ++w) { a += s0[w]; b += s1[w]; }
        *out = make_double2(a, b);
    }
}

__device__ __forceinline__ void block_sum2_1024(double &a, double &b)
{
    __shared__ double s0[32], s1[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    if (lane == 0) { s0[warp] = a; s1[warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) { x += s0[w]; y += s1[w]; }
        a = x;
        b = y;
    }
}

// The convergence check of one iteration (fixed-order sums of the block
// partials, then the state update and the graph loop's condition), run by
// one block: the check kernel, or the last block of the iteration's last
// part kernel (fused).
__device__ __forceinline__ void check_body(int mode, IterState *st, const double2 *red, int nred,
                                           cudaGraphConditionalHandle cond, int use_cond)
{
    if (st->done) return;   // host-loop mode may launch past convergence
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nred; i += blockDim.x) {
        const double2 v = red[i];
        a += v.x;
        b += v.y;
    }
    block_sum2_1024(a, b);
    if (threadIdx.x == 0) {
        if (mode == EPI_HITS) {
            const double na = st->hits_norm == 2 ? sqrt(a) : a;
            const double nh = st->hits_norm == 2 ? sqrt(b) : b;
            st->scale[0] = na > 0.0 ? 1.0 / na : 0.0;
            st->scale[1] = nh > 0.0 ? 1.0 / nh : 0.0;
            st->l1 = 0.0;
        } else {
            st->l1 = a;
            st->delta = b;
        }
        st->iter += 1;
        st->parity ^= 1;
        const int done = st->iter >= st->max_iter ||
                         (mode != EPI_HITS && st->tol > 0.0 && st->l1 < st->tol);
        st->done = done;
        if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
    }
}

// Fused check: after its block partial is stored, each block of the
// iteration's last part kernel counts itself out; the last one -- every
// other block of this launch and every earlier launch of the iteration has
// then written its partials -- runs the check and re-arms the counter.
template <int MODE>
__device__ __forceinline__ void fused_check(const FuseCheck &fc, const double2 *red)
{
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(fc.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    check_body(MODE == EPI_PR_PAT ? EPI_PAGERANK : MODE, fc.st, red, fc.nred,
               (cudaGraphConditionalHandle)fc.cond, fc.use_cond);
    if (threadIdx.x == 0) *fc.done = 0u;
}

// x gathers: straight from global memory through the read-only path, or
// from the shared-memory copy of the part's first `S` columns (its densest
// ones: columns are in decreasing-length order) with global fallback.
struct GatherGlobal {
    const float *__restrict__ x;
    __device__ __forceinline__ float operator()(int c) const { return __ldg(x + c); }
};
struct GatherStaged {
    const float *__restrict__ x;
    const float *xs;
    int c0;
    unsigned S;
    __device__ __forceinline__ float operator()(int c) const
    {
        const unsigned o = (unsigned)(c - c0);
        return o < S ? xs[o] : __ldg(x + c);
    }
};

// A slot against the shared-memory slice or global x, without a branch:
// both loads are predicated (shared when the column lies in the slice,
// global when it lies outside and is not padding), so a warp whose lanes
// split between the two issues both loads back to back and keeps its
// gathers in flight together.  Measured against the branching form (R-MAT
// scale 24 PageRank iteration, 24K-column slice): 0.749 vs 0.782 ms.
__device__ __forceinline__ float slot_fma_g(uint2 v, const GatherStaged &g, float acc)
{
    const int c = (int)v.x;
    const unsigned o = (unsigned)(c - g.c0);
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(g.xs) + 4u * o;
    const float *ga = g.x + c;
    float xv;
    asm("{\n\t.reg .pred ps, pg;\n\t"
        "setp.lt.u32 ps, %1, %2;\n\t"
        "setp.ge.and.s32 pg, %3, 0, !ps;\n\t"
        "mov.f32 %0, 0f00000000;\n\t"
        "@ps ld.shared.f32 %0, [%4];\n\t"
        "@pg ld.global.nc.f32 %0, [%5];\n\t}"
        : "=f"(xv) : "r"(o), "r"(g.S), "r"(c), "r"(sa), "l"(ga));
    return fmaf(__uint_as_float(v.y), xv, acc);
}

template <class G>
__device__ __forceinline__ float slot_fma_g(uint2 v, const G &g, float acc)
{
    const int c = (int)v.x;
    const float xv = c >= 0 ? g(c) : 0.0f;
    return fmaf(__uint_as_float(v.y), xv, acc);
}

// Bulk prefetch of a workload's slots into L2 (TMA, fire and forget): a
// workload's slab region is consumed front to back, so lane 0 keeps the
// prefetched frontier `ahead` bytes in front of the consumed position.  The
// region starts on a 256-byte boundary and spans a multiple of 256 bytes.
__device__ __forceinline__ void l2_prefetch(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

struct SlabPrefetch {
    const char *base;
    unsigned total, done, ahead;
    __device__ __forceinline__ void advance(unsigned consumed, int lane)
    {
        while (done < total && done < consumed + ahead) {
            const unsigned n = min(4096u, total - done);
            if (lane == 0) l2_prefetch(base + done, n);
            done += n;
        }
    }
};

// Slot loaders of a workload's region: the full layout stores {column,
// value} pairs (8 bytes); the pattern-only layout stores the column alone (4
// bytes) and every slot's value is 1 -- the column's value is folded into
// the gathered vector (z = p * inv_deg for PageRank).  Both hand back a
// {column, float bits} pair, padding as column -1.
__host__ __device__ constexpr bool is_pattern(int mode) { return mode == EPI_PR_PAT || mode == EPI_RAW_PAT; }

template <bool PAT> struct Slots;
template <> struct Slots<false> {
    static constexpr int kBytes = 8;
    const uint2 *__restrict__ p;
    __device__ __forceinline__ Slots(const PartView &pv, int64_t off) : p(pv.slab + off) {}
    __device__ __forceinline__ uint2 ld(int64_t i) const { return __ldcs(p + i); }
    __device__ __forceinline__ const char *bytes_at(int64_t i) const { return reinterpret_cast<const char *>(p + i); }
};
template <> struct Slots<true> {
    static constexpr int kBytes = 4;
    const uint32_t *__restrict__ p;
    __device__ __forceinline__ Slots(const PartView &pv, int64_t off) : p(pv.slab4 + off) {}
    __device__ __forceinline__ uint2 ld(int64_t i) const { return make_uint2(__ldcs(p + i), 0x3f800000u); }
    __device__ __forceinline__ const char *bytes_at(int64_t i) const { return reinterpret_cast<const char *>(p + i); }
};

// One workload (Solution 3) computed by the calling warp.
template <int MODE, class G>
__device__ __forceinline__ void do_workload(const Workload &d, const PartView &pv,
                                            const SplitView &sv, const G &g, const Epi &E,
                                            const float *__restrict__ x, float *__restrict__ y,
                                            double2 *red, int lane, FSum &r0, FSum &r1)
{
    const uint32_t *__restrict__ rows = pv.rows + d.rows;
    if (d.w == 0) {
        // rows without entries (the epilogue alone): kZeroBatch rows per lane
        // per pass, their operand loads all in flight together
        constexpr int kZeroBatch = 4;
        for (int i0 = 0; i0 < d.h; i0 += 32 * kZeroBatch) {
            RowPre p[kZeroBatch];
#pragma unroll
            for (int u = 0; u < kZeroBatch; ++u) {
                const int i = i0 + u * 32 + lane;
                p[u] = prefetch_row<MODE>(E, rows, i, i < d.h, x, y);
            }
#pragma unroll
            for (int u = 0; u < kZeroBatch; ++u)
                if (i0 + u * 32 + lane < d.h) finish_row_pre<MODE>(E, sv, red, p[u], 0.f, x, y, r0, r1);
        }
        return;
    }
    const Slots<is_pattern(MODE)> slab{pv, d.slab};
    const int hp = d.major == 0 ? d.h : (d.h + 31) & ~31;
    SlabPrefetch pf{slab.bytes_at(0), (unsigned)((int64_t)hp * d.w * Slots<is_pattern(MODE)>::kBytes),
                    0u, (unsigned)pv.pf_ahead};
    if (pf.ahead) pf.advance(0u, lane);
    if (d.major == 0) {
        // row-major (CSR-vector): the warp strides across one row at a time;
        // the next 4 slots per lane are in flight while the current 4 gather
        const int nst = d.w >> 5;   // 32-slot steps per row
        for (int g0 = 0; g0 < d.h; g0 += 32) {
            const RowPre mine = prefetch_row<MODE>(E, rows, g0 + lane, g0 + lane < d.h, x, y);
            const int gend = min(d.h, g0 + 32);
            for (int i = g0; i < gend; ++i) {
                const int64_t s = (int64_t)i * d.w + lane;
                float acc = 0.f;
                int st = 0;
                if (nst >= 4) {
                    uint2 a0 = slab.ld(s), a1 = slab.ld(s + 32), a2 = slab.ld(s + 64), a3 = slab.ld(s + 96);
                    for (st = 4; st + 4 <= nst; st += 4) {
                        if (pf.ahead) pf.advance((unsigned)(((int64_t)i * d.w + st * 32) * Slots<is_pattern(MODE)>::kBytes), lane);
                        const int64_t q = s + st * 32;
                        const uint2 b0 = slab.ld(q), b1 = slab.ld(q + 32), b2 = slab.ld(q + 64), b3 = slab.ld(q + 96);
                        acc = slot_fma_g(a0, g, acc);
                        acc = slot_fma_g(a1, g, acc);
                        acc = slot_fma_g(a2, g, acc);
                        acc = slot_fma_g(a3, g, acc);
                        a0 = b0; a1 = b1; a2 = b2; a3 = b3;
                    }
                    acc = slot_fma_g(a0, g, acc);
                    acc = slot_fma_g(a1, g, acc);
                    acc = slot_fma_g(a2, g, acc);
                    acc = slot_fma_g(a3, g, acc);
                }
                {   // the last < 4 steps (all of a short row): loads first
                    uint2 r[3];
#pragma unroll
                    for (int u = 0; u < 3; ++u)
                        r[u] = st + u < nst ? slab.ld(s + (st + u) * 32) : make_uint2(0xffffffffu, 0u);
#pragma unroll
                    for (int u = 0; u < 3; ++u) acc = slot_fma_g(r[u], g, acc);
                }
                acc = warp_sum(acc);
                const RowPre p = shfl_row(mine, i - g0);
                if (lane == 0) finish_row_pre<MODE>(E, sv, red, p, acc, x, y, r0, r1);
                if (pf.ahead) pf.advance((unsigned)((int64_t)(i + 1) * d.w * Slots<is_pattern(MODE)>::kBytes), lane);
            }
        }
    } else {
        // column-major (ELL): one row per lane; two 32-row blocks per pass so
        // each lane keeps two independent load chains in flight
        for (int b = 0; b < hp; b += 64) {
            const bool two = b + 32 < hp;
            const RowPre pa = prefetch_row<MODE>(E, rows, b + lane, b + lane < d.h, x, y);
            const RowPre pb = prefetch_row<MODE>(E, rows, b + 32 + lane, two && b + 32 + lane < d.h, x, y);
            const int64_t sa = (int64_t)b * d.w + lane;
            const int64_t sb = sa + (int64_t)32 * d.w;
            float acc_a = 0.f, acc_b = 0.f;
            int e = 0;
            if (two) {
                for (; e + 3 < d.w; e += 4) {
                    if (pf.ahead) pf.advance((unsigned)(((int64_t)b * d.w + (int64_t)e * 32) * Slots<is_pattern(MODE)>::kBytes), lane);
                    uint2 a[4], c[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        a[u] = slab.ld(sa + (int64_t)(e + u) * 32);
                        c[u] = slab.ld(sb + (int64_t)(e + u) * 32);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        acc_a = slot_fma_g(a[u], g, acc_a);
                        acc_b = slot_fma_g(c[u], g, acc_b);
                    }
                }
                for (; e < d.w; ++e) {
                    const uint2 a0 = slab.ld(sa + (int64_t)e * 32), c0 = slab.ld(sb + (int64_t)e * 32);
                    acc_a = slot_fma_g(a0, g, acc_a);
                    acc_b = slot_fma_g(c0, g, acc_b);
                }
            } else {
                for (; e + 7 < d.w; e += 8) {
                    if (pf.ahead) pf.advance((unsigned)(((int64_t)b * d.w + (int64_t)e * 32) * Slots<is_pattern(MODE)>::kBytes), lane);
                    uint2 a[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) a[u] = slab.ld(sa + (int64_t)(e + u) * 32);
#pragma unroll
                    for (int u = 0; u < 8; ++u) acc_a = slot_fma_g(a[u], g, acc_a);
                }
                {
                    uint2 r[7];
#pragma unroll
                    for (int u = 0; u < 7; ++u)
                        r[u] = e + u < d.w ? slab.ld(sa + (int64_t)(e + u) * 32) : make_uint2(0xffffffffu, 0u);
#pragma unroll
                    for (int u = 0; u < 7; ++u) acc_a = slot_fma_g(r[u], g, acc_a);
                }
            }
            if (b + lane < d.h) finish_row_pre<MODE>(E, sv, red, pa, acc_a, x, y, r0, r1);
            if (two && b + 32 + lane < d.h) finish_row_pre<MODE>(E, sv, red, pb, acc_b, x, y, r0, r1);
            if (pf.ahead) pf.advance((unsigned)((int64_t)(b + 64) * d.w * Slots<is_pattern(MODE)>::kBytes), lane);
        }
    }
}

// Up to four consecutive short column-major workloads of one claim unit
// (one 32-row block each, at most kShortW entries per row) computed
// together: each lane carries one row of each, so its four dependent
// chains -- row entry and operands, slots, gathers, epilogue -- overlap
// instead of running one after another (the row cap makes every ELL
// workload a single block, so a warp otherwise has one chain per lane).
// Each row's entries are summed in the same order as do_workload.
// Measured (PageRank kernel per iteration): R-MAT scale 22 0.1552 vs 0.1655
// ms, scale 24 0.7255 vs 0.7486 ms, scale 26 3.376 vs 3.468 ms; limits of
// 8, 16 and 32 entries per row measured 0.1561, 0.1615 and 0.1619 ms at
// scale 22.
constexpr int kShortW = 4;

__device__ __forceinline__ bool short_block(const Workload &d)
{
    return d.major == 1 && d.w > 0 && d.w <= kShortW && d.h <= 32;
}

template <int MODE, class G>
__device__ __forceinline__ void do_short4(const Workload *dd, const PartView &pv, const SplitView &sv,
                                          const G &g, const Epi &E, const float *__restrict__ x,
                                          float *__restrict__ y, double2 *red, int lane, FSum &r0,
                                          FSum &r1)
{
    RowPre pr[4];
    float ac[4];
    int wmax = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        pr[u] = prefetch_row<MODE>(E, pv.rows + dd[u].rows, lane, lane < dd[u].h, x, y);
        ac[u] = 0.f;
        wmax = max(wmax, (int)dd[u].w);
    }
    for (int e = 0; e < wmax; ++e) {
        uint2 sl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const Slots<is_pattern(MODE)> slab{pv, dd[u].slab};
            sl[u] = e < dd[u].w ? slab.ld((int64_t)e * 32 + lane) : make_uint2(0xffffffffu, 0u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) ac[u] = slot_fma_g(sl[u], g, ac[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (lane < dd[u].h) finish_row_pre<MODE>(E, sv, red, pr[u], ac[u], x, y, r0, r1);
}

template <int MODE>
__device__ __forceinline__ void resolve_xy(const IterState *st, const float *&x, float *&y)
{
    if (st) {
        const int par = st->parity;
        x = st->buf[par];
        y = st->buf[par ^ 1];
    }
}

// Tiled composite SpMV over one part (Solution 3), one warp per workload:
// warp `wid` computes workload `wid` (8-warp blocks, x gathered from L1/L2).
template <int MODE>
__global__ void __launch_bounds__(kBlock, kPartMinBlocks)
k_part(PartView pv, SplitView sv, const float *__restrict__ xin, float *__restrict__ yout,
       const IterState *__restrict__ st, double2 *__restrict__ red)
{
    const float *x = xin;
    float *y = yout;
    Epi E = load_epi<MODE>(st);
    resolve_xy<MODE>(st, x, y);
    if (MODE == EPI_ADJ) E.xs = x[E.seed];
    const float *gsrc = (MODE == EPI_PR_PAT) ? st->zbuf[st->parity] : x;
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    FSum r0, r1;
    if (wid < pv.nwl) {
        const GatherGlobal g{gsrc};
        do_workload<MODE>(pv.wl[wid], pv, sv, g, E, x, y, red, lane, r0, r1);
    }
    if (MODE != EPI_RAW && MODE != EPI_RAW_PAT && MODE != EPI_BATCH)
        block_reduce_store<MODE>(r0, r1, red + pv.red_base + blockIdx.x);
}

// The persistent form of the same computation, two instantiations:
// * NT = 256 (the default kernel): MINB 8-warp blocks per SM, x gathered
//   through L1/L2;
// * NT = 1024 (option 1): one 32-warp block per SM that first copies the
//   part's densest columns x[c0, c0 + S) into shared memory (the GB300
//   counterpart of the paper's texture-cache tile, Section 3.1 Solution 1).
// Warps take workloads in order from a counter (pv.sched[0]) in claim units
// -- runs of consecutive workloads grouped by the builder so that small
// workloads are claimed several at a time (one atomic on one address per
// claim bounds the claim rate) while large ones stay alone; the last warp
// out resets the counters for the next launch (pv.sched[1] counts finished
// warps).  No block waits on another; the fused check (fc.nred > 0) runs in
// whichever block finishes last.
template <int MODE, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_part_staged(PartView pv, SplitView sv, const float *__restrict__ xin,
              float *__restrict__ yout, const IterState *st, double2 *red, FuseCheck fc)
{
    extern __shared__ float xs[];
    const float *x = xin;
    float *y = yout;
    Epi E = load_epi<MODE>(st);
    resolve_xy<MODE>(st, x, y);
    if (MODE == EPI_ADJ) E.xs = x[E.seed];
    const float *gsrc = (MODE == EPI_PR_PAT) ? st->zbuf[st->parity] : x;
    // the 32-warp variant stages x[c0, c0 + S) in shared memory; the
    // several-blocks-per-SM variant gathers everything through L1/L2
    constexpr bool kStage = NT == kStagedBlock;
    const int S = kStage ? pv.xs_cols : 0, c0 = pv.c0;
    if (kStage) {
        // 16-byte copies only where the caller's x address allows them (x
        // may be any float-aligned device pointer, e.g. a tensor slice)
        if (((c0 | S) & 3) == 0 && (reinterpret_cast<uintptr_t>(gsrc + c0) & 15) == 0) {
            const float4 *src = reinterpret_cast<const float4 *>(gsrc + c0);
            float4 *dst = reinterpret_cast<float4 *>(xs);
            for (int i = threadIdx.x; i < (S >> 2); i += blockDim.x) dst[i] = __ldg(src + i);
        } else {
            for (int i = threadIdx.x; i < S; i += blockDim.x) xs[i] = __ldg(gsrc + c0 + i);
        }
        __syncthreads();
    }
    using Gather = typename std::conditional<kStage, GatherStaged, GatherGlobal>::type;
    Gather g;
    if constexpr (kStage) g = GatherStaged{gsrc, xs, c0, (unsigned)S};
    else g = GatherGlobal{gsrc};
    const int lane = threadIdx.x & 31;
    FSum r0, r1;
    for (;;) {
        unsigned u = 0;
        if (lane == 0) u = atomicAdd(pv.sched, 1u);
        u = __shfl_sync(kFull, u, 0);
        if (u >= (unsigned)pv.nunits) break;
        const int w0 = __ldg(pv.units + u), w1 = __ldg(pv.units + u + 1);
        for (int w = w0; w < w1;) {
            if (w + 3 < w1) {
                Workload dd[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) dd[u] = pv.wl[w + u];
                if (short_block(dd[0]) && short_block(dd[1]) && short_block(dd[2]) && short_block(dd[3])) {
                    do_short4<MODE>(dd, pv, sv, g, E, x, y, red, lane, r0, r1);
                    w += 4;
                    continue;
                }
            }
            do_workload<MODE>(pv.wl[w], pv, sv, g, E, x, y, red, lane, r0, r1);
            ++w;
        }
    }
    if (lane == 0) {
        const unsigned done = atomicAdd(pv.sched + 1, 1u);
        if (done == gridDim.x * (blockDim.x >> 5) - 1) {   // every warp has left the loop
            pv.sched[0] = 0u;
            pv.sched[1] = 0u;
        }
    }
    if (MODE != EPI_RAW && MODE != EPI_RAW_PAT && MODE != EPI_BATCH) {
        block_reduce_store<MODE>(r0, r1, red + pv.red_base + blockIdx.x);
        if (fc.nred > 0) fused_check<MODE>(fc, red);
    }
}

// ------------------------------------------------ TMA-pipelined kernel --
//
// The slot stream is the one large sequential stream of the SpMV, and a
// warp's workload occupies one contiguous, 256-byte aligned region of it
// consumed front to back (row-major: row after row; column-major: 32-slot
// columns of a 32-row block).  Each warp therefore streams its region into a
// ring of kTmaStages shared-memory chunks with TMA bulk copies
// (cp.async.bulk ... mbarrier::complete_tx): in-flight data holds no
// registers, so every warp keeps 4 KB of slots in flight, and slots are read
// from shared memory in batches of 4 steps whose x gathers are issued back
// to back.  Lane 0 is the producer of its own warp's ring; every wait is
// bounded and records a status flag instead of hanging.

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_copy_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

constexpr int kTmaSteps = kTmaChunk / 256;        // 32-slot steps per chunk
constexpr uint32_t kTmaWaitLimit = 1u << 22;      // try_wait rounds before giving up

struct TmaRing {
    char *buf;            // kTmaStages x kTmaChunk bytes of this warp
    uint64_t *bar;        // kTmaStages barriers of this warp
    uint32_t used;        // chunks this warp has consumed so far (all workloads)
    bool fail;
};

// Issue chunk c of the region `src` (bytes total) into its stage.
__device__ __forceinline__ void tma_issue(TmaRing &R, const char *src, uint32_t bytes, uint32_t c)
{
    const uint32_t k = R.used + c, st = k % kTmaStages;
    const uint32_t n = min((uint32_t)kTmaChunk, bytes - c * kTmaChunk);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(R.bar + st, n);
    tma_copy_1d(R.buf + st * kTmaChunk, src + (size_t)c * kTmaChunk, n, R.bar + st);
}

__device__ __forceinline__ bool tma_wait(TmaRing &R, uint32_t c)
{
    const uint32_t k = R.used + c, st = k % kTmaStages, parity = (k / kTmaStages) & 1u;
    for (uint32_t it = 0; it < kTmaWaitLimit; ++it)
        if (mbar_try_wait(R.bar + st, parity)) return true;
    return false;
}

template <int MODE, class G>
__device__ __forceinline__ void do_workload_tma(const Workload &d, const PartView &pv,
                                                const SplitView &sv, const G &g, const Epi &E,
                                                const float *__restrict__ x,
                                                float *__restrict__ y, double2 *red, int lane,
                                                TmaRing &R, FSum &r0, FSum &r1)
{
    const uint32_t *__restrict__ rows = pv.rows + d.rows;
    const int hp = d.major == 0 ? d.h : (d.h + 31) & ~31;
    const uint32_t bytes = (uint32_t)((int64_t)hp * d.w * 8);
    const uint32_t nch = (bytes + kTmaChunk - 1) / kTmaChunk;
    const char *src = reinterpret_cast<const char *>(pv.slab + d.slab);
    if (lane == 0)
        for (uint32_t c = 0; c < nch && c < (uint32_t)kTmaStages; ++c) tma_issue(R, src, bytes, c);
    // steps per row (row-major) or per 32-row block (column-major)
    const int per = d.major == 0 ? (d.w >> 5) : d.w;
    int left = per;                // steps left in the current row / block
    int unit = 0;                  // current row (row-major) or block (column-major)
    RowPre mine = prefetch_row<MODE>(E, rows, lane, lane < d.h, x, y);
    float acc = 0.f;
    if (nch == 0) {                // rows without entries (w = 0)
        for (int b = 0; b < hp; b += 32) {
            if (b > 0) mine = prefetch_row<MODE>(E, rows, b + lane, b + lane < d.h, x, y);
            if (b + lane < d.h) finish_row_pre<MODE>(E, sv, red, mine, 0.f, x, y, r0, r1);
        }
        return;
    }
    for (uint32_t c = 0; c < nch; ++c) {
        if (!tma_wait(R, c)) {
            // give up: record it, then let the copies still in flight land
            // (each wait bounded again) before the warp leaves its ring
            R.fail = true;
            for (uint32_t q = c + 1; q < nch && q < c + kTmaStages; ++q) tma_wait(R, q);
            break;
        }
        const uint32_t st = (R.used + c) % kTmaStages;
        const uint2 *ch = reinterpret_cast<const uint2 *>(R.buf + st * kTmaChunk);
        const int steps = (int)min((uint32_t)kTmaSteps, (bytes - c * kTmaChunk) / 256u);
        uint2 sl[kTmaSteps];
        float xv[kTmaSteps];
#pragma unroll
        for (int j = 0; j < kTmaSteps; ++j) sl[j] = j < steps ? ch[j * 32 + lane] : make_uint2(0xffffffffu, 0u);
        __syncwarp();
        if (lane == 0 && c + kTmaStages < nch) tma_issue(R, src, bytes, c + kTmaStages);
#pragma unroll
        for (int j = 0; j < kTmaSteps; ++j) xv[j] = (int)sl[j].x >= 0 ? g((int)sl[j].x) : 0.f;
#pragma unroll
        for (int j = 0; j < kTmaSteps; ++j) {
            if (j >= steps) break;
            acc = fmaf(__uint_as_float(sl[j].y), xv[j], acc);
            if (--left > 0) continue;
            left = per;
            if (d.major == 0) {
                const int i = unit++;
                const float tot = warp_sum(acc);
                if (i > 0 && (i & 31) == 0)
                    mine = prefetch_row<MODE>(E, rows, i + lane, i + lane < d.h, x, y);
                const RowPre p = shfl_row(mine, i & 31);
                if (lane == 0) finish_row_pre<MODE>(E, sv, red, p, tot, x, y, r0, r1);
            } else {
                const int b = unit++ * 32;
                if (b + lane < d.h) finish_row_pre<MODE>(E, sv, red, mine, acc, x, y, r0, r1);
                if (b + 32 < hp) mine = prefetch_row<MODE>(E, rows, b + 32 + lane, b + 32 + lane < d.h, x, y);
            }
            acc = 0.f;
        }
    }
    R.used += nch;
}

// One persistent 32-warp block per SM: x[c0, c0 + xs_cols) in shared memory
// as in k_part_staged, plus the per-warp TMA rings.  Shared memory:
// barriers (1 KB), rings (32 x 4 KB), x slice.
template <int MODE>
__global__ void __launch_bounds__(kStagedBlock, 1)
k_part_tma(PartView pv, SplitView sv, const float *__restrict__ xin, float *__restrict__ yout,
           const IterState *__restrict__ st, double2 *__restrict__ red)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int kWarps = kStagedBlock / 32;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    char *ring = reinterpret_cast<char *>(smem + 1024);
    float *xs = reinterpret_cast<float *>(smem + 1024 + kWarps * kTmaStages * kTmaChunk);
    const float *x = xin;
    float *y = yout;
    Epi E = load_epi<MODE>(st);
    resolve_xy<MODE>(st, x, y);
    if (MODE == EPI_ADJ) E.xs = x[E.seed];
    const int S = pv.xs_cols, c0 = pv.c0;
    if (((c0 | S) & 3) == 0 && (reinterpret_cast<uintptr_t>(x + c0) & 15) == 0) {
        const float4 *src4 = reinterpret_cast<const float4 *>(x + c0);
        float4 *dst4 = reinterpret_cast<float4 *>(xs);
        for (int i = threadIdx.x; i < (S >> 2); i += blockDim.x) dst4[i] = __ldg(src4 + i);
    } else {
        for (int i = threadIdx.x; i < S; i += blockDim.x) xs[i] = __ldg(x + c0 + i);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    TmaRing R{ring + warp * kTmaStages * kTmaChunk, bars + warp * kTmaStages, 0u, false};
    if (lane == 0) {
        for (int s2 = 0; s2 < kTmaStages; ++s2) mbar_init(R.bar + s2, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const GatherStaged g{x, xs, c0, (unsigned)S};
    FSum r0, r1;
    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(pv.sched, 1u);
        w = __shfl_sync(kFull, w, 0);
        if (w >= (unsigned)pv.nwl || R.fail) break;
        do_workload_tma<MODE>(pv.wl[w], pv, sv, g, E, x, y, red, lane, R, r0, r1);
    }
    if (lane == 0) {
        if (R.fail) atomicOr(pv.status, 1u);
        const unsigned done = atomicAdd(pv.sched + 1, 1u);
        if (done == gridDim.x * (blockDim.x >> 5) - 1) {   // every warp has left the loop
            pv.sched[0] = 0u;
            pv.sched[1] = 0u;
        }
    }
    if (MODE != EPI_RAW && MODE != EPI_RAW_PAT && MODE != EPI_BATCH)
        block_reduce_store<MODE>(r0, r1, red + pv.red_base + blockIdx.x);
}

constexpr size_t kTmaSmemFixed = 1024 + (size_t)(kStagedBlock / 32) * kTmaStages * kTmaChunk;

template <int MODE> static void launch_tma(const PartView &pv, const SplitView &sv, const float *x,
                                           float *y, const IterState *st, double2 *red,
                                           cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_part_tma<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kTmaSmemFixed + kTmaMaxCols * sizeof(float)));
        attr = true;
    }
    k_part_tma<MODE><<<pv.nblocks, kStagedBlock, kTmaSmemFixed + (size_t)pv.xs_cols * sizeof(float), s>>>(
        pv, sv, x, y, st, red);
}

int persist_blocks_per_sm()
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_part_staged<EPI_RAW, kBlock, kPersistMinBlocks>,
                                                      kBlock, 0) != cudaSuccess)
        return 0;
    return b;
}

int part_blocks_per_sm()
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_part<EPI_PAGERANK>, kBlock, 0) != cudaSuccess)
        return 0;
    return b;
}

template <int MODE> static void launch_staged(const PartView &pv, const SplitView &sv, const float *x,
                                              float *y, const IterState *st, double2 *red,
                                              const FuseCheck &fc, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_part_staged<MODE, kStagedBlock, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kStagedMaxCols * (int)sizeof(float));
        attr = true;
    }
    if (pv.persist)
        k_part_staged<MODE, kBlock, persist_minb(MODE)><<<pv.nblocks, kBlock, 0, s>>>(pv, sv, x, y, st, red, fc);
    else
        k_part_staged<MODE, kStagedBlock, 1><<<pv.nblocks, kStagedBlock, (size_t)pv.xs_cols * sizeof(float), s>>>(
            pv, sv, x, y, st, red, fc);
}

bool launch_part(int mode, const PartView &pv, const SplitView &sv, const float *x, float *y,
                 const IterState *st, double2 *red, cudaStream_t s, const FuseCheck &fc)
{
    if (pv.nblocks <= 0) return false;
    if (pv.tma) {
        switch (mode) {
        case EPI_RAW: launch_tma<EPI_RAW>(pv, sv, x, y, st, red, s); break;
        case EPI_PAGERANK: launch_tma<EPI_PAGERANK>(pv, sv, x, y, st, red, s); break;
        case EPI_RWR: launch_tma<EPI_RWR>(pv, sv, x, y, st, red, s); break;
        case EPI_ADJ: launch_tma<EPI_ADJ>(pv, sv, x, y, st, red, s); break;
        case EPI_BATCH: launch_tma<EPI_BATCH>(pv, sv, x, y, st, red, s); break;
        default: launch_tma<EPI_HITS>(pv, sv, x, y, st, red, s); break;
        }
        count_launches(1);
        return false;
    }
    if (pv.xs_cols > 0 || pv.persist) {
        switch (mode) {
        case EPI_RAW: launch_staged<EPI_RAW>(pv, sv, x, y, st, red, fc, s); break;
        case EPI_PAGERANK: launch_staged<EPI_PAGERANK>(pv, sv, x, y, st, red, fc, s); break;
        case EPI_RWR: launch_staged<EPI_RWR>(pv, sv, x, y, st, red, fc, s); break;
        case EPI_ADJ: launch_staged<EPI_ADJ>(pv, sv, x, y, st, red, fc, s); break;
        case EPI_BATCH: launch_staged<EPI_BATCH>(pv, sv, x, y, st, red, fc, s); break;
        case EPI_PR_PAT: launch_staged<EPI_PR_PAT>(pv, sv, x, y, st, red, fc, s); break;
        case EPI_RAW_PAT: launch_staged<EPI_RAW_PAT>(pv, sv, x, y, st, red, fc, s); break;
        default: launch_staged<EPI_HITS>(pv, sv, x, y, st, red, fc, s); break;
        }
        count_launches(1);
        return fc.nred > 0 && mode != EPI_RAW && mode != EPI_RAW_PAT && mode != EPI_BATCH;
    }
    dim3 g(pv.nblocks), b(kBlock);
    switch (mode) {
    case EPI_RAW: k_part<EPI_RAW><<<g, b, 0, s>>>(pv, sv, x, y, st, red); break;
    case EPI_PAGERANK: k_part<EPI_PAGERANK><<<g, b, 0, s>>>(pv, sv, x, y, st, red); break;
    case EPI_RWR: k_part<EPI_RWR><<<g, b, 0, s>>>(pv, sv, x, y, st, red); break;
    case EPI_ADJ: k_part<EPI_ADJ><<<g, b, 0, s>>>(pv, sv, x, y, st, red); break;
    case EPI_BATCH: k_part<EPI_BATCH><<<g, b, 0, s>>>(pv, sv, x, y, st, red); break;
    case EPI_PR_PAT: k_part<EPI_PR_PAT><<<g, b, 0, s>>>(pv, sv, x, y, st, red); break;
    case EPI_RAW_PAT: k_part<EPI_RAW_PAT><<<g, b, 0, s>>>(pv, sv, x, y, st, red); break;
    default: k_part<EPI_HITS><<<g, b, 0, s>>>(pv, sv, x, y, st, red); break;
    }
    count_launches(1);
    return false;
}

// ------------------------------------------------------------------ SpMM --
//
// Y' = M' X' for k vectors (X' n x k row-major).  One warp per workload, the
// k columns in chunks of 64: lane l owns columns c0 + 2l and c0 + 2l + 1, so
// every stored entry (c, v) costs one coalesced gather of 64 columns of X
// row c (256 bytes per warp) and two FMAs per lane.  The gather is the
// dominant traffic (4k bytes per entry against 8 for the slot), so the
// kernel keeps several entries' gathers in flight per lane:
// * row-major workload: a batch of 32 entries of the row is loaded one per
//   lane and broadcast by shuffles, all 32 gathered together (kSpmmRowU);
//   the next batch's slots are loaded before the current batch is consumed;
// * column-major block of 32 rows: step e holds entry e of all 32 rows, so
//   the warp keeps the 32 rows' partial sums in registers (acc[32], static
//   indices) and walks the block step by step -- short rows cost no
//   per-row latency chain.
// The epilogue (split rows, RWR terms, per-column sums) is per row with one
// lane per column pair.

constexpr int kSpmmU = 8;
// Row-major workloads: the whole 32-entry batch of a row gathered at once
// (32 X rows, 8 KB per warp, in flight) -- the row path does not hold the
// column-major path's 32 row sums, so its registers allow it (RWR k = 64 at
// R-MAT scale 22: 3.10 ms per iteration against 3.37 with 8 at a time).
// Same summation order as 8 at a time.
constexpr int kSpmmRowU = 32;
// Rows of a 32-row ELL block whose sums one pass keeps in registers (the
// block is walked 32 / rows times, its slots re-read each time) and resident
// blocks per SM, per mode: the plain SpMM trades register rows for a third
// block per SM (4.03 -> 3.76 ms at k = 64, R-MAT 22); the RWR epilogue needs
// the registers (3.40 ms at 32 rows and two blocks, 5.2 ms at 16 and three).
__host__ __device__ constexpr int spmm_rows(int mode) { return mode == EPI_RAW ? 16 : 32; }
__host__ __device__ constexpr int spmm_minb(int mode) { return mode == EPI_RAW ? 3 : 2; }
// Rows whose epilogue operands are fetched together.
constexpr int kSpmmEpi = 4;
// Blocks of the first stage of the deterministic column sums.
constexpr int kColsumBlocks = 152;
constexpr size_t kSpmmTileBytes = (size_t)kWarpsPerBlock * 32 * 32 * sizeof(float2);   // 64 KB

struct EpiK {
    float c;
    int64_t dstart;
};

// One stored entry's gather: X row c, the lane's two columns.
template <bool EVEN>
__device__ __forceinline__ float2 gather2(const float *__restrict__ X, int c, int k, int j0)
{
    float2 p = make_float2(0.f, 0.f);
    if (c < 0 || j0 >= k) return p;
    const float *r = X + (int64_t)c * k + j0;
    if (EVEN) return __ldg(reinterpret_cast<const float2 *>(r));
    p.x = __ldg(r);
    if (j0 + 1 < k) p.y = __ldg(r + 1);
    return p;
}

// Row epilogue for SpMM: RAW or RWR per column (restart seeds[j], dangling
// mass delta_k[j]).  Per-lane sums for its two columns.
template <int MODE>
__device__ __forceinline__ void epilogue_k(const EpiK &E, uint32_t rid, float t0, float t1,
                                           int j0, int k, const float *__restrict__ X,
                                           float *__restrict__ Y, const int32_t *seeds,
                                           const double *delta_k, FSum *acc4)
{
    const uint32_t v = rid & kRowIdMask;
    float *yr = Y + (int64_t)v * k;
    const float *xr = X + (int64_t)v * k;
    const bool h0 = j0 < k, h1 = j0 + 1 < k;
    if (rid & kRowNotFirst) { if (h0) t0 += yr[j0]; if (h1) t1 += yr[j0 + 1]; }
    if ((rid & kRowNotLast) || MODE == EPI_RAW) {
        if (h0) yr[j0] = t0;
        if (h1) yr[j0 + 1] = t1;
        return;
    }
    const double c = E.c;
    if (h0) {
        float add = (int)v == __ldg(seeds + j0) ? (float)(c * delta_k[j0] + (1.0 - c)) : 0.f;
        float f = fmaf(E.c, t0, add);
        yr[j0] = f;
        acc4[0].add(fabsf(f - xr[j0]));
        if ((int64_t)v >= E.dstart) acc4[2].add(f);
    }
    if (h1) {
        float add = (int)v == __ldg(seeds + j0 + 1) ? (float)(c * delta_k[j0 + 1] + (1.0 - c)) : 0.f;
        float f = fmaf(E.c, t1, add);
        yr[j0 + 1] = f;
        acc4[1].add(fabsf(f - xr[j0 + 1]));
        if ((int64_t)v >= E.dstart) acc4[3].add(f);
    }
}

// A finished row (chunk c0 of its columns) of the SpMM: either the epilogue,
// or -- for a chunk of a split row -- publish the partial; after the last
// column chunk the last chunk of the row to arrive sums all partials in chunk
// order and runs the epilogue for every column chunk.  Warp-uniform.
template <int MODE>
__device__ __noinline__ void spmm_finish_split(const EpiK &E, const SplitView &sv, uint32_t rid,
                                               float a0, float a1, int c0, int k, int lane,
                                               const float *__restrict__ X, float *__restrict__ Y,
                                               const int32_t *seeds, const double *delta_k,
                                               double *redk)
{
    const int j0 = c0 + 2 * lane;
    const int slot = (int)(rid & 0x7fffffffu);
    float *pp = sv.partial + (int64_t)slot * k;
    if (j0 < k) pp[j0] = a0;
    if (j0 + 1 < k) pp[j0 + 1] = a1;
    if (c0 + 64 < k) return;   // publish after the last column chunk
    __threadfence();
    __syncwarp();
    const int s = sv.slot_owner[slot];
    const SplitRow sr = sv.rows[s];
    unsigned prev = 0;
    if (lane == 0) prev = atomicAdd(sv.counter + s, 1u);
    prev = __shfl_sync(kFull, prev, 0);
    if (prev != (unsigned)sr.nchunks - 1) return;
    __threadfence();
    FSum sr4[4];
    for (int cc = 0; cc < k; cc += 64) {
        const int jj = cc + 2 * lane;
        float t0 = 0.f, t1 = 0.f;
        for (int q = 0; q < sr.nchunks; ++q) {
            const float *src = sv.partial + (int64_t)(sr.first_slot + q) * k;
            if (jj < k) t0 += __ldcg(src + jj);
            if (jj + 1 < k) t1 += __ldcg(src + jj + 1);
        }
        epilogue_k<MODE>(E, sr.row, t0, t1, jj, k, X, Y, seeds, delta_k, sr4);
    }
    if (lane == 0) sv.counter[s] = 0u;
    if (MODE != EPI_RAW && j0 < k) {
        double *o = redk + (int64_t)(sv.red_split_base + sr.red_slot) * 2 * k;
        o[j0] = sr4[0].value();
        o[k + j0] = sr4[2].value();
        if (j0 + 1 < k) { o[j0 + 1] = sr4[1].value(); o[k + j0 + 1] = sr4[3].value(); }
    }
}

template <int MODE>
__device__ __forceinline__ void spmm_finish(const EpiK &E, const SplitView &sv, uint32_t rid,
                                            float a0, float a1, int c0, int k, int lane,
                                            const float *__restrict__ X, float *__restrict__ Y,
                                            const int32_t *seeds, const double *delta_k,
                                            double *redk, FSum *acc4)
{
    if (rid & kRowSplit)
        spmm_finish_split<MODE>(E, sv, rid, a0, a1, c0, k, lane, X, Y, seeds, delta_k, redk);
    else
        epilogue_k<MODE>(E, rid, a0, a1, c0 + 2 * lane, k, X, Y, seeds, delta_k, acc4);
}

// The operands a row's SpMM epilogue reads besides its sums -- y' (rows
// continued from an earlier part) and x' (the L1 change) for the lane's two
// columns -- fetched ahead so that their latency overlaps other rows' work.
struct RowPreK {
    float2 yv, xv;
};

template <int MODE>
__device__ __forceinline__ RowPreK prefetch_row_k(uint32_t rid, bool ok, const float *__restrict__ X,
                                                  const float *__restrict__ Y, int k, int j0)
{
    RowPreK r{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (!ok || (rid & kRowSplit) || j0 >= k) return r;
    const int64_t o = (int64_t)(rid & kRowIdMask) * k + j0;
    const bool two = j0 + 1 < k;
    if (rid & kRowNotFirst) { r.yv.x = Y[o]; if (two) r.yv.y = Y[o + 1]; }
    if (MODE != EPI_RAW && !(rid & kRowNotLast)) { r.xv.x = X[o]; if (two) r.xv.y = X[o + 1]; }
    return r;
}

// epilogue_k with its row operands prefetched (same arithmetic).
template <int MODE>
__device__ __forceinline__ void epilogue_k_pre(const EpiK &E, uint32_t rid, float t0, float t1,
                                               const RowPreK &r, int j0, int k,
                                               float *__restrict__ Y, const int32_t *seeds,
                                               const double *delta_k, FSum *acc4)
{
    const uint32_t v = rid & kRowIdMask;
    float *yr = Y + (int64_t)v * k;
    const bool h0 = j0 < k, h1 = j0 + 1 < k;
    if (rid & kRowNotFirst) { t0 += r.yv.x; t1 += r.yv.y; }
    if ((rid & kRowNotLast) || MODE == EPI_RAW) {
        if (h0) yr[j0] = t0;
        if (h1) yr[j0 + 1] = t1;
        return;
    }
    const double c = E.c;
    if (h0) {
        float add = (int)v == __ldg(seeds + j0) ? (float)(c * delta_k[j0] + (1.0 - c)) : 0.f;
        float f = fmaf(E.c, t0, add);
        yr[j0] = f;
        acc4[0].add(fabsf(f - r.xv.x));
        if ((int64_t)v >= E.dstart) acc4[2].add(f);
    }
    if (h1) {
        float add = (int)v == __ldg(seeds + j0 + 1) ? (float)(c * delta_k[j0 + 1] + (1.0 - c)) : 0.f;
        float f = fmaf(E.c, t1, add);
        yr[j0 + 1] = f;
        acc4[1].add(fabsf(f - r.xv.y));
        if ((int64_t)v >= E.dstart) acc4[3].add(f);
    }
}

template <int MODE>
__device__ __forceinline__ void spmm_finish_pre(const EpiK &E, const SplitView &sv, uint32_t rid,
                                                float a0, float a1, const RowPreK &r, int c0, int k,
                                                int lane, const float *__restrict__ X,
                                                float *__restrict__ Y, const int32_t *seeds,
                                                const double *delta_k, double *redk, FSum *acc4)
{
    if (rid & kRowSplit)
        spmm_finish_split<MODE>(E, sv, rid, a0, a1, c0, k, lane, X, Y, seeds, delta_k, redk);
    else
        epilogue_k_pre<MODE>(E, rid, a0, a1, r, c0 + 2 * lane, k, Y, seeds, delta_k, acc4);
}

// Row-major workload: rows one after another, 32 entries per batch.
template <int MODE, bool EVEN>
__device__ __forceinline__ void spmm_rows(const Workload &d, const uint2 *__restrict__ slab,
                                          const uint32_t *__restrict__ rows, const EpiK &E,
                                          const SplitView &sv, const float *__restrict__ X,
                                          float *__restrict__ Y, int k, int lane,
                                          const int32_t *seeds, const double *delta_k,
                                          double *redk, FSum *acc4)
{
    const uint2 pad = make_uint2(0xffffffffu, 0u);
    for (int c0 = 0; c0 < k; c0 += 64) {
        const int j0 = c0 + 2 * lane;
        for (int i = 0; i < d.h; ++i) {
            const uint32_t rid = __ldg(rows + i);
            const RowPreK pre = prefetch_row_k<MODE>(rid, true, X, Y, k, j0);
            const uint2 *rs = slab + (int64_t)i * d.w;
            float a0 = 0.f, a1 = 0.f;
            uint2 nxt = d.w > 0 ? __ldcs(rs + lane) : pad;
            for (int e0 = 0; e0 < d.w; e0 += 32) {
                const uint2 ent = nxt;
                const int cnt = __popc(__ballot_sync(kFull, (int)ent.x >= 0));
                // entries are a prefix of the row's slots: a full batch may
                // have a successor, a partial one ends the row
                nxt = (cnt == 32 && e0 + 32 < d.w) ? __ldcs(rs + e0 + 32 + lane) : pad;
                for (int t = 0; t < cnt; t += kSpmmRowU) {
                    float2 p[kSpmmRowU];
                    float vv[kSpmmRowU];
#pragma unroll
                    for (int u = 0; u < kSpmmRowU; ++u) {
                        const int c = __shfl_sync(kFull, (int)ent.x, (t + u) & 31);
                        vv[u] = __shfl_sync(kFull, __uint_as_float(ent.y), (t + u) & 31);
                        p[u] = gather2<EVEN>(X, t + u < cnt ? c : -1, k, j0);
                    }
#pragma unroll
                    for (int u = 0; u < kSpmmRowU; ++u) {
                        const float w = t + u < cnt ? vv[u] : 0.f;
                        a0 = fmaf(w, p[u].x, a0);
                        a1 = fmaf(w, p[u].y, a1);
                    }
                }
                if (cnt < 32) break;
            }
            spmm_finish_pre<MODE>(E, sv, rid, a0, a1, pre, c0, k, lane, X, Y, seeds, delta_k, redk, acc4);
        }
    }
}

// Column-major workload: 32-row blocks, step e = entry e of each of the 32
// rows (one slot per lane); the 32 rows' sums stay in registers.
template <int MODE, bool EVEN>
__device__ __forceinline__ void spmm_block(const Workload &d, const uint2 *__restrict__ slab,
                                           const uint32_t *__restrict__ rows, const EpiK &E,
                                           const SplitView &sv, const float *__restrict__ X,
                                           float *__restrict__ Y, int k, int lane,
                                           const int32_t *seeds, const double *delta_k,
                                           double *redk, FSum *acc4, float2 *tile)
{
    const uint2 pad = make_uint2(0xffffffffu, 0u);
    const int hp = (d.h + 31) & ~31;
    constexpr int RB = spmm_rows(MODE);   // rows of the block summed per pass
    for (int b = 0; b < hp; b += 32) {
        const uint32_t my_rid = b + lane < d.h ? __ldg(rows + b + lane) : 0u;
        const uint2 *blk = slab + (int64_t)b * d.w;
        const int nr = min(32, d.h - b);
        for (int c0 = 0; c0 < k; c0 += 64) {
            const int j0 = c0 + 2 * lane;
            for (int r0 = 0; r0 < nr; r0 += RB) {
                float2 acc[RB];
#pragma unroll
                for (int t = 0; t < RB; ++t) acc[t] = make_float2(0.f, 0.f);
                uint2 nxt = d.w > 0 ? __ldcs(blk + lane) : pad;
                for (int e = 0; e < d.w; ++e) {
                    const uint2 ent = nxt;
                    nxt = e + 1 < d.w ? __ldcs(blk + (int64_t)(e + 1) * 32 + lane) : pad;
#pragma unroll
                    for (int t0 = 0; t0 < RB; t0 += kSpmmU) {
                        float2 p[kSpmmU];
                        float vv[kSpmmU];
#pragma unroll
                        for (int u = 0; u < kSpmmU; ++u) {
                            const int c = __shfl_sync(kFull, (int)ent.x, r0 + t0 + u);
                            vv[u] = __shfl_sync(kFull, __uint_as_float(ent.y), r0 + t0 + u);
                            p[u] = gather2<EVEN>(X, c, k, j0);
                        }
#pragma unroll
                        for (int u = 0; u < kSpmmU; ++u) {
                            acc[t0 + u].x = fmaf(vv[u], p[u].x, acc[t0 + u].x);
                            acc[t0 + u].y = fmaf(vv[u], p[u].y, acc[t0 + u].y);
                        }
                    }
                }
                // the epilogue reads the sums back row by row from the warp's
                // shared-memory tile (one 64-column row per step, lane l holds
                // columns 2l, 2l+1): a rolled loop, so the sums are not live
                // across inlined epilogues
#pragma unroll
                for (int t = 0; t < RB; ++t) tile[t * 32 + lane] = acc[t];
                __syncwarp();
                const int nrr = min(RB, nr - r0);
#pragma unroll 1
                for (int t0 = 0; t0 < nrr; t0 += kSpmmEpi) {
                    uint32_t rid[kSpmmEpi];
                    RowPreK pre[kSpmmEpi];
#pragma unroll
                    for (int u = 0; u < kSpmmEpi; ++u) {
                        rid[u] = __shfl_sync(kFull, my_rid, (r0 + t0 + u) & 31);
                        pre[u] = prefetch_row_k<MODE>(rid[u], t0 + u < nrr, X, Y, k, j0);
                    }
#pragma unroll
                    for (int u = 0; u < kSpmmEpi; ++u) {
                        if (t0 + u < nrr) {
                            const float2 a = tile[(t0 + u) * 32 + lane];
                            spmm_finish_pre<MODE>(E, sv, rid[u], a.x, a.y, pre[u], c0, k, lane, X, Y, seeds,
                                                  delta_k, redk, acc4);
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
}

// ---- k a multiple of 64: a half-warp per stored entry, 16 bytes per lane
// (the form every k % 64 == 0 call takes; the float2 form above serves the
// other k).  The SpMM is bound by instruction issue, not by the gather's
// memory latency (ncu: 1.62G warp instructions per RWR iteration at R-MAT
// scale 22 in the float2 form, issue 43 % busy, 4.2 long-scoreboard cycles
// per issue); this form measured 2.62 ms per RWR k = 64 iteration against
// 3.03 ms.
// Lane l serves half h = l / 16 and column quad q = l % 16 (columns
// c0 + 4q .. c0 + 4q + 3 of the 64-column chunk), so one warp instruction
// gathers the 256-byte X rows of two entries -- half the shuffles, address
// arithmetic and loads per entry of the float2 form, and no column bounds
// checks.  Sums go back to the float2-per-lane layout (columns c0 + 2l,
// c0 + 2l + 1) for the same row epilogue.

#ifndef SPG_SPMM4_ROWU
#define SPG_SPMM4_ROWU 8
#endif
#ifndef SPG_SPMM4_BLKU
#define SPG_SPMM4_BLKU 4
#endif
// Row pairs of a block summed per pass: two passes of 16 rows (the block's
// slots read twice) hold half the sums in registers and spill less than one
// pass of 32 (RWR k = 64 at R-MAT scale 22: 2.553 ms per iteration against
// 2.622 with one pass and 2.806 with four); a third resident block per SM
// (80 registers, all of the carve-out to shared memory) measured 3.40-4.24 ms.
#ifndef SPG_SPMM4_PASS
#define SPG_SPMM4_PASS 8
#endif
#ifndef SPG_SPMM4_MINB
#define SPG_SPMM4_MINB 2
#endif
constexpr int kSpmm4RowU = SPG_SPMM4_ROWU;   // entry pairs gathered together, row-major path
constexpr int kSpmm4BlkU = SPG_SPMM4_BLKU;   // row pairs gathered together per step, block path
constexpr int kSpmm4Pass = SPG_SPMM4_PASS;   // row pairs of a 32-row block summed per pass
constexpr int kSpmm4MinB = SPG_SPMM4_MINB;   // resident blocks per SM (register budget)
#ifndef SPG_SPMM4_EPI
#define SPG_SPMM4_EPI 4
#endif
constexpr int kSpmm4Epi = SPG_SPMM4_EPI;     // block rows whose epilogue operands are fetched together
static_assert(16 % kSpmm4Pass == 0 && kSpmm4Pass % kSpmm4BlkU == 0, "SpMM pass shape");

__device__ __forceinline__ float4 gather4q(const float *__restrict__ Xq, int c, int k)
{
    if (c < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
    return __ldg(reinterpret_cast<const float4 *>(Xq + (int64_t)c * k));
}

__device__ __forceinline__ void fma4(float4 &a, float v, const float4 &p)
{
    a.x = fmaf(v, p.x, a.x);
    a.y = fmaf(v, p.y, a.y);
    a.z = fmaf(v, p.z, a.z);
    a.w = fmaf(v, p.w, a.w);
}

// Row-major workload: entries 2t and 2t + 1 of each 32-entry batch go to the
// two halves; the halves' sums are added at the end of the row.
template <int MODE>
__device__ __forceinline__ void spmm_rows4(const Workload &d, const uint2 *__restrict__ slab,
                                           const uint32_t *__restrict__ rows, const EpiK &E,
                                           const SplitView &sv, const float *__restrict__ X,
                                           float *__restrict__ Y, int k, int lane,
                                           const int32_t *seeds, const double *delta_k,
                                           double *redk, FSum *acc4)
{
    const uint2 pad = make_uint2(0xffffffffu, 0u);
    const int h = lane >> 4, q = lane & 15;
    for (int c0 = 0; c0 < k; c0 += 64) {
        const float *Xq = X + c0 + 4 * q;
        const int j0 = c0 + 2 * lane;
        for (int i = 0; i < d.h; ++i) {
            const uint32_t rid = __ldg(rows + i);
            const RowPreK pre = prefetch_row_k<MODE>(rid, true, X, Y, k, j0);
            const uint2 *rs = slab + (int64_t)i * d.w;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            uint2 nxt = d.w > 0 ? __ldcs(rs + lane) : pad;
            for (int e0 = 0; e0 < d.w; e0 += 32) {
                const uint2 ent = nxt;
                const int cnt = __popc(__ballot_sync(kFull, (int)ent.x >= 0));
                nxt = (cnt == 32 && e0 + 32 < d.w) ? __ldcs(rs + e0 + 32 + lane) : pad;
#pragma unroll
                for (int t0 = 0; t0 < 16; t0 += kSpmm4RowU) {
                    float4 p[kSpmm4RowU];
#pragma unroll
                    for (int u = 0; u < kSpmm4RowU; ++u) {
                        const int e = 2 * (t0 + u) + h;
                        const int c = __shfl_sync(kFull, (int)ent.x, e);
                        p[u] = gather4q(Xq, e < cnt ? c : -1, k);
                    }
#pragma unroll
                    for (int u = 0; u < kSpmm4RowU; ++u) {
                        const int e = 2 * (t0 + u) + h;
                        const float v = __shfl_sync(kFull, __uint_as_float(ent.y), e);
                        fma4(a, e < cnt ? v : 0.f, p[u]);
                    }
                }
                if (cnt < 32) break;
            }
            a.x += __shfl_xor_sync(kFull, a.x, 16);
            a.y += __shfl_xor_sync(kFull, a.y, 16);
            a.z += __shfl_xor_sync(kFull, a.z, 16);
            a.w += __shfl_xor_sync(kFull, a.w, 16);
            // lane l takes columns 2l, 2l + 1: half of quad l / 2
            const float bx = __shfl_sync(kFull, a.x, lane >> 1), by = __shfl_sync(kFull, a.y, lane >> 1);
            const float bz = __shfl_sync(kFull, a.z, lane >> 1), bw = __shfl_sync(kFull, a.w, lane >> 1);
            const float a0 = (lane & 1) ? bz : bx, a1 = (lane & 1) ? bw : by;
            spmm_finish_pre<MODE>(E, sv, rid, a0, a1, pre, c0, k, lane, X, Y, seeds, delta_k, redk, acc4);
        }
    }
}

// Column-major block of 32 rows: half h sums rows 2t + h for its column
// quad, kSpmm4Pass row pairs t per pass over the block's slots, step by step
// (the same order of the row's entries as the float2 form), then writes the
// sums to the warp's tile in the float2-per-lane layout for the epilogue.
template <int MODE>
__device__ __forceinline__ void spmm_block4(const Workload &d, const uint2 *__restrict__ slab,
                                            const uint32_t *__restrict__ rows, const EpiK &E,
                                            const SplitView &sv, const float *__restrict__ X,
                                            float *__restrict__ Y, int k, int lane,
                                            const int32_t *seeds, const double *delta_k,
                                            double *redk, FSum *acc4, float2 *tile)
{
    const uint2 pad = make_uint2(0xffffffffu, 0u);
    const int hp = (d.h + 31) & ~31;
    const int h = lane >> 4, q = lane & 15;
    for (int b = 0; b < hp; b += 32) {
        const uint32_t my_rid = b + lane < d.h ? __ldg(rows + b + lane) : 0u;
        const uint2 *blk = slab + (int64_t)b * d.w;
        const int nr = min(32, d.h - b);
        for (int c0 = 0; c0 < k; c0 += 64) {
            const float *Xq = X + c0 + 4 * q;
            const int j0 = c0 + 2 * lane;
#pragma unroll 1
            for (int tp = 0; tp < 16 && 2 * tp < nr; tp += kSpmm4Pass) {
                // pass over row pairs tp .. tp + kSpmm4Pass - 1 (rows 2 tp .. 2 tp + 2 kSpmm4Pass - 1)
                float4 acc[kSpmm4Pass];
#pragma unroll
                for (int t = 0; t < kSpmm4Pass; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
                uint2 nxt = d.w > 0 ? __ldcs(blk + lane) : pad;
                for (int e = 0; e < d.w; ++e) {
                    const uint2 ent = nxt;
                    nxt = e + 1 < d.w ? __ldcs(blk + (int64_t)(e + 1) * 32 + lane) : pad;
#pragma unroll
                    for (int t0 = 0; t0 < kSpmm4Pass; t0 += kSpmm4BlkU) {
                        float4 p[kSpmm4BlkU];
#pragma unroll
                        for (int u = 0; u < kSpmm4BlkU; ++u) {
                            const int c = __shfl_sync(kFull, (int)ent.x, 2 * (tp + t0 + u) + h);
                            p[u] = gather4q(Xq, c, k);
                        }
#pragma unroll
                        for (int u = 0; u < kSpmm4BlkU; ++u) {
                            const float v = __shfl_sync(kFull, __uint_as_float(ent.y), 2 * (tp + t0 + u) + h);
                            fma4(acc[t0 + u], v, p[u]);
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < kSpmm4Pass; ++t) {
                    tile[(2 * (tp + t) + h) * 32 + 2 * q] = make_float2(acc[t].x, acc[t].y);
                    tile[(2 * (tp + t) + h) * 32 + 2 * q + 1] = make_float2(acc[t].z, acc[t].w);
                }
                __syncwarp();
                const int rend = min(nr, 2 * (tp + kSpmm4Pass));
#pragma unroll 1
                for (int t0 = 2 * tp; t0 < rend; t0 += kSpmm4Epi) {
                    uint32_t rid[kSpmm4Epi];
                    RowPreK pre[kSpmm4Epi];
#pragma unroll
                    for (int u = 0; u < kSpmm4Epi; ++u) {
                        rid[u] = __shfl_sync(kFull, my_rid, (t0 + u) & 31);
                        pre[u] = prefetch_row_k<MODE>(rid[u], t0 + u < rend, X, Y, k, j0);
                    }
#pragma unroll
                    for (int u = 0; u < kSpmm4Epi; ++u) {
                        if (t0 + u < rend) {
                            const float2 a = tile[(t0 + u) * 32 + lane];
                            spmm_finish_pre<MODE>(E, sv, rid[u], a.x, a.y, pre[u], c0, k, lane, X, Y, seeds,
                                                  delta_k, redk, acc4);
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
}

// The k % 64 == 0 form of k_part_spmm (same launch geometry and sums).
template <int MODE>
__global__ void __launch_bounds__(kBlock, kSpmm4MinB)
k_part_spmm4(PartView pv, SplitView sv, const float *__restrict__ Xin, float *__restrict__ Yout,
             int k, const IterState *__restrict__ st, const int32_t *__restrict__ seeds,
             const double *__restrict__ delta_k, double *__restrict__ redk)
{
    const float *X = Xin;
    float *Y = Yout;
    EpiK E;
    E.c = 1.f;
    E.dstart = 0;
    if (st) {
        const int par = st->parity;
        X = st->buf[par];
        Y = st->buf[par ^ 1];
        E.c = (float)st->c;
        E.dstart = st->dangling_start;
    }
    extern __shared__ float2 spmm_tile4[];   // per warp: 32 rows x 64 columns
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wid = blockIdx.x * kWarpsPerBlock + warp;
    FSum acc4[4];
    if (wid < pv.nwl) {
        const Workload d = pv.wl[wid];
        const uint2 *slab = pv.slab + d.slab;
        const uint32_t *rows = pv.rows + d.rows;
        if (d.major == 0)
            spmm_rows4<MODE>(d, slab, rows, E, sv, X, Y, k, lane, seeds, delta_k, redk, acc4);
        else
            spmm_block4<MODE>(d, slab, rows, E, sv, X, Y, k, lane, seeds, delta_k, redk, acc4,
                              spmm_tile4 + warp * 32 * 32);
    }
    if (MODE != EPI_RAW) {
        __shared__ double sm[kWarpsPerBlock][4][32];
        sm[warp][0][lane] = acc4[0].value(); sm[warp][1][lane] = acc4[1].value();
        sm[warp][2][lane] = acc4[2].value(); sm[warp][3][lane] = acc4[3].value();
        __syncthreads();
        if (threadIdx.x < 128) {
            const int qq = threadIdx.x >> 5, l = threadIdx.x & 31;
            double a = 0.0;
            for (int w = 0; w < kWarpsPerBlock; ++w) a += sm[w][qq][l];
            const int j = 2 * l + (qq & 1);
            if (j < k) {
                double *o = redk + (int64_t)(pv.red_base + blockIdx.x) * 2 * k;
                o[(qq >> 1) * k + j] = a;
            }
        }
    }
}

// SpMM over one part.  Split rows: chunk partials (k floats per chunk slot)
// in sv.partial, combined in chunk order by the last chunk.  Per-block
// column sums for RWR into redk[(slot * 2 + q) * k + j] (q = 0: L1, 1: dangling).
template <int MODE, bool EVEN>
__global__ void __launch_bounds__(kBlock, spmm_minb(MODE))
k_part_spmm(PartView pv, SplitView sv, const float *__restrict__ Xin, float *__restrict__ Yout,
            int k, const IterState *__restrict__ st, const int32_t *__restrict__ seeds,
            const double *__restrict__ delta_k, double *__restrict__ redk)
{
    const float *X = Xin;
    float *Y = Yout;
    EpiK E;
    E.c = 1.f;
    E.dstart = 0;
    if (st) {
        const int par = st->parity;
        X = st->buf[par];
        Y = st->buf[par ^ 1];
        E.c = (float)st->c;
        E.dstart = st->dangling_start;
    }
    extern __shared__ float2 spmm_tile[];   // per warp: 32 rows x 64 columns
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wid = blockIdx.x * kWarpsPerBlock + warp;
    FSum acc4[4];   // L1 j0, L1 j0+1, dangling j0, dangling j0+1
    if (wid < pv.nwl) {
        const Workload d = pv.wl[wid];
        const uint2 *slab = pv.slab + d.slab;
        const uint32_t *rows = pv.rows + d.rows;
        if (d.major == 0)
            spmm_rows<MODE, EVEN>(d, slab, rows, E, sv, X, Y, k, lane, seeds, delta_k, redk, acc4);
        else
            spmm_block<MODE, EVEN>(d, slab, rows, E, sv, X, Y, k, lane, seeds, delta_k, redk, acc4,
                                   spmm_tile + warp * 32 * 32);
    }
    if (MODE != EPI_RAW) {
        // per-block column sums (k <= 64 for the RWR epilogue)
        __shared__ double sm[kWarpsPerBlock][4][32];
        sm[warp][0][lane] = acc4[0].value(); sm[warp][1][lane] = acc4[1].value();
        sm[warp][2][lane] = acc4[2].value(); sm[warp][3][lane] = acc4[3].value();
        __syncthreads();
        if (threadIdx.x < 128) {
            const int q = threadIdx.x >> 5, l = threadIdx.x & 31;
            double a = 0.0;
            for (int w = 0; w < kWarpsPerBlock; ++w) a += sm[w][q][l];
            const int j = 2 * l + (q & 1);
            if (j < k) {
                double *o = redk + (int64_t)(pv.red_base + blockIdx.x) * 2 * k;
                o[(q >> 1) * k + j] = a;
            }
        }
    }
}

void launch_part_spmm(int mode, const PartView &pv, const SplitView &sv, const float *X, float *Y,
                      int k, const IterState *st, const int32_t *seeds, const double *delta_k,
                      double *redk, cudaStream_t s)
{
    if (pv.nblocks <= 0) return;
    dim3 g(pv.nblocks), b(kBlock);
    const size_t smem = kSpmmTileBytes;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_part_spmm<EPI_RAW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_part_spmm<EPI_RAW, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_part_spmm<EPI_RWR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_part_spmm<EPI_RWR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    static bool attr4 = false;
    if (!attr4) {
        cudaFuncSetAttribute(k_part_spmm4<EPI_RAW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_part_spmm4<EPI_RWR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (kSpmm4MinB > 2) {   // more than two 72 KB blocks per SM: all of the carve-out to shared memory
            cudaFuncSetAttribute(k_part_spmm4<EPI_RAW>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
            cudaFuncSetAttribute(k_part_spmm4<EPI_RWR>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        }
        attr4 = true;
    }
    if (k % 64 == 0) {
        if (mode == EPI_RAW) k_part_spmm4<EPI_RAW><<<g, b, smem, s>>>(pv, sv, X, Y, k, st, seeds, delta_k, redk);
        else k_part_spmm4<EPI_RWR><<<g, b, smem, s>>>(pv, sv, X, Y, k, st, seeds, delta_k, redk);
        count_launches(1);
        return;
    }
    const bool even = (k % 2) == 0;
    if (mode == EPI_RAW) {
        if (even) k_part_spmm<EPI_RAW, true><<<g, b, smem, s>>>(pv, sv, X, Y, k, st, seeds, delta_k, redk);
        else k_part_spmm<EPI_RAW, false><<<g, b, smem, s>>>(pv, sv, X, Y, k, st, seeds, delta_k, redk);
    } else {
        if (even) k_part_spmm<EPI_RWR, true><<<g, b, smem, s>>>(pv, sv, X, Y, k, st, seeds, delta_k, redk);
        else k_part_spmm<EPI_RWR, false><<<g, b, smem, s>>>(pv, sv, X, Y, k, st, seeds, delta_k, redk);
    }
    count_launches(1);
}

// ----------------------------------------------------------------- check --

__global__ void __launch_bounds__(1024)
k_check(int mode, IterState *st, const double2 *__restrict__ red, int nred,
        cudaGraphConditionalHandle cond, int use_cond)
{
    check_body(mode, st, red, nred, cond, use_cond);
}

void launch_check(int mode, IterState *st, const double2 *red, int nred,
                  unsigned long long cond, int use_cond, cudaStream_t s)
{
    k_check<<<1, 1024, 0, s>>>(mode, st, red, nred, (cudaGraphConditionalHandle)cond, use_cond);
    count_launches(1);
}

// Row-partitioned PageRank on one device (Section 3.2).  All-gather step:
// rank r has written the next iterate's rows it owns into its own buffer
// states[r]->buf[parity ^ 1]; every row is copied from its owner's buffer
// into the other ranks' (across GPUs: an all-gather of the ranks' row slices
// and a local scatter).  Pattern-only ranks also carry z = p * inv_deg.
__global__ void k_allgather_rows(int64_t n, const int8_t *__restrict__ owner,
                                 IterState *const *states, int P, int pat)
{
    __shared__ float *ybuf[8], *zbuf[8];
    if (threadIdx.x < P) {
        const IterState *st = states[threadIdx.x];
        ybuf[threadIdx.x] = st->buf[st->parity ^ 1];
        zbuf[threadIdx.x] = pat ? st->zbuf[st->parity ^ 1] : nullptr;
    }
    __syncthreads();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int o = owner[v];
        const float val = ybuf[o][v];
        const float zv = pat ? zbuf[o][v] : 0.f;
        for (int q = 0; q < P; ++q) {
            if (q == o) continue;
            ybuf[q][v] = val;
            if (pat) zbuf[q][v] = zv;
        }
    }
}

void launch_allgather_rows(int64_t n, const int8_t *owner, IterState *const *states, int P, bool pat,
                           cudaStream_t s)
{
    k_allgather_rows<<<grid_for(n), 256, 0, s>>>(n, owner, states, P, pat ? 1 : 0);
    count_launches(1);
}

// All-reduce step: the ranks' block partials of (L1 change, dangling mass)
// lie in one buffer; their fixed-order sum goes to every rank's state, which
// all advance together (the check of k_check, PageRank form).
__global__ void __launch_bounds__(1024)
k_check_ranks(IterState *const *states, int P, const double2 *__restrict__ red, int nred)
{
    if (states[0]->done) return;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nred; i += blockDim.x) {
        const double2 v = red[i];
        a += v.x;
        b += v.y;
    }
    block_sum2_1024(a, b);
    if (threadIdx.x == 0) {
        const IterState *s0 = states[0];
        const int iter = s0->iter + 1;
        const int done = iter >= s0->max_iter || (s0->tol > 0.0 && a < s0->tol);
        for (int r = 0; r < P; ++r) {
            IterState *st = states[r];
            st->l1 = a;
            st->delta = b;
            st->iter = iter;
            st->parity ^= 1;
            st->done = done;
        }
    }
}

void launch_check_ranks(IterState *const *states, int P, const double2 *red, int nred, cudaStream_t s)
{
    k_check_ranks<<<1, 1024, 0, s>>>(states, P, red, nred);
    count_launches(1);
}

// Per-column sums over slots for k columns (k <= 64): thread (q, part)
// sums slots part, part+P, ... of column q in order, then parts in order.
__global__ void __launch_bounds__(128)
k_check_k(IterState *st, const double *__restrict__ part, int nb, int k, double *delta_k,
          double *l1_k, cudaGraphConditionalHandle cond, int use_cond)
{
    __shared__ double colmax[64];
    if (st->done) return;   // host-loop mode may launch past convergence
    const int Q = 2 * k;
    if (threadIdx.x < Q) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += part[(int64_t)b * Q + threadIdx.x];
        if (threadIdx.x < k) { l1_k[threadIdx.x] = t; colmax[threadIdx.x] = t; }
        else delta_k[threadIdx.x - k] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int j = 0; j < k; ++j) m = fmax(m, colmax[j]);
        st->l1 = m;
        st->iter += 1;
        st->parity ^= 1;
        const int done = st->iter >= st->max_iter || (st->tol > 0.0 && m < st->tol);
        st->done = done;
        if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
    }
}

// Deterministic column sums of a row-major block src (rows [row0, row0 +
// nrows), row stride ld, first Q <= 128 columns), stage 1 of 2: block b sums
// a fixed contiguous range of rows; thread (p, q) takes every P-th row of it
// for column q (FP32 sources through a TwoSum pair, FP64 ones in FP64); the P
// partials are added in order into part[b * Q + q].
template <class T>
__global__ void __launch_bounds__(256)
k_colsum_part(const T *__restrict__ src, int64_t row0, int64_t nrows, int64_t ld, int Q,
              double *__restrict__ part)
{
    __shared__ double sm[256];
    const int P = 256 / Q;
    const int q = threadIdx.x % Q, p = threadIdx.x / Q;
    const int64_t per = (nrows + gridDim.x - 1) / gridDim.x;
    const int64_t lo = row0 + per * blockIdx.x, hi = min(row0 + nrows, lo + per);
    double a = 0.0;
    if (p < P) {
        if (sizeof(T) == sizeof(float)) {
            FSum f;
            for (int64_t v = lo + p; v < hi; v += P) f.add((float)src[v * ld + q]);
            a = f.value();
        } else {
            for (int64_t v = lo + p; v < hi; v += P) a += (double)src[v * ld + q];
        }
    }
    sm[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x < Q) {
        double t = 0.0;
        for (int pp = 0; pp < P; ++pp) t += sm[pp * Q + threadIdx.x];
        part[(int64_t)blockIdx.x * Q + threadIdx.x] = t;
    }
}

int colsum_scratch() { return kColsumBlocks * 128; }

void launch_check_k(IterState *st, const double *redk, int nred, int k, double *delta_k,
                    double *l1_k, double *scratch, unsigned long long cond, int use_cond,
                    cudaStream_t s)
{
    k_colsum_part<double><<<kColsumBlocks, 256, 0, s>>>(redk, 0, nred, 2 * k, 2 * k, scratch);
    k_check_k<<<1, 128, 0, s>>>(st, scratch, kColsumBlocks, k, delta_k, l1_k,
                                (cudaGraphConditionalHandle)cond, use_cond);
    count_launches(2);
}

// Dangling mass of the start vector: a deterministic two-stage sum (fixed
// per-block ranges, then one block adds the block partials in order).
constexpr int kInitBlocks = 304;

template <bool FLAGS>
__global__ void __launch_bounds__(256) k_init_delta_part(const IterState *st, const uint8_t *flags,
                                                        double *part)
{
    const float *x = st->buf[st->parity];
    const int64_t a = FLAGS ? 0 : st->dangling_start, n = st->n;
    const int64_t len = n - a, per = (len + gridDim.x - 1) / gridDim.x;
    const int64_t lo = a + per * blockIdx.x, hi = min(n, lo + per);
    double s = 0.0;
    for (int64_t v = lo + threadIdx.x; v < hi; v += blockDim.x)
        if (!FLAGS || flags[v]) s += (double)x[v];
    __shared__ double sm[8];
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sm[w];
        part[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) k_init_delta_final(IterState *st, const double *part, int nb)
{
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a += part[i];
    block_sum2_1024(a, b);
    if (threadIdx.x == 0) st->delta = a;
}

void launch_init_delta(IterState *st, double *scratch, cudaStream_t s)
{
    k_init_delta_part<false><<<kInitBlocks, 256, 0, s>>>(st, nullptr, scratch);
    k_init_delta_final<<<1, 1024, 0, s>>>(st, scratch, kInitBlocks);
    count_launches(2);
}

void launch_init_delta_flags(IterState *st, const uint8_t *dangling, double *scratch, cudaStream_t s)
{
    k_init_delta_part<true><<<kInitBlocks, 256, 0, s>>>(st, dangling, scratch);
    k_init_delta_final<<<1, 1024, 0, s>>>(st, scratch, kInitBlocks);
    count_launches(2);
}

int init_delta_scratch() { return kInitBlocks; }

__global__ void k_set_one(float *p, const int32_t *idx, int count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) p[idx[i]] = 1.f;
}

void launch_set_one(float *p, const int32_t *idx, int count, cudaStream_t s)
{
    k_set_one<<<(count + 255) / 256, 256, 0, s>>>(p, idx, count);
    count_launches(1);
}

__global__ void __launch_bounds__(128)
k_init_delta_k_final(const double *__restrict__ part, int nb, int k, double *delta_k)
{
    if (threadIdx.x < k) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += part[(int64_t)b * k + threadIdx.x];
        delta_k[threadIdx.x] = t;
    }
}

void launch_init_delta_k(int64_t dangling_start, int64_t n, const float *X, int k,
                         double *delta_k, double *scratch, cudaStream_t s)
{
    const int64_t a = dangling_start;
    k_colsum_part<float><<<kColsumBlocks, 256, 0, s>>>(X, a, n - a, k, k, scratch);
    k_init_delta_k_final<<<1, 128, 0, s>>>(scratch, kColsumBlocks, k, delta_k);
    count_launches(2);
}

// ------------------------------------------------------- batch of graphs --

// Block g: L1 change and dangling mass of graph g over its positions
// [goff[g], goff[g+1]) (its dangling tail starts at gdstart[g]); fixed order.
// Per-graph L1 change and dangling mass, stage 1: block c sums chunk c --
// a fixed range of at most kBatchChunk positions of one graph -- (each
// thread a fixed strided subset, TwoSum pairs, then the warps in order) into
// cpart[c].  The check adds each graph's chunks in order (stage 2).
__global__ void __launch_bounds__(256) k_batch_reduce(const IterState *st)
{
    const int c = blockIdx.x;
    const float *x = st->buf[st->parity];
    const float *y = st->buf[st->parity ^ 1];
    const int g = st->cgraph[c];
    const int64_t a = st->cstart[c], b = st->cstart[c + 1], ds = st->gdstart[g];
    FSum fl1, fdg;
#pragma unroll 4
    for (int64_t v = a + threadIdx.x; v < b; v += blockDim.x) {
        const float f = y[v];
        fl1.add(fabsf(f - x[v]));
        if (v >= ds) fdg.add(f);
    }
    __shared__ double s0[8], s1[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double l1 = warp_sum_d(fl1.value());
    const double dg = warp_sum_d(fdg.value());
    if (lane == 0) { s0[warp] = l1; s1[warp] = dg; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double p = 0.0, q = 0.0;
        for (int w = 0; w < 8; ++w) { p += s0[w]; q += s1[w]; }
        st->cpart[c] = make_double2(p, q);
    }
}

void launch_batch_reduce(IterState *st, int nchunk, cudaStream_t s)
{
    k_batch_reduce<<<nchunk, 256, 0, s>>>(st);
    count_launches(1);
}

// Per graph: the next base (c * dangling mass + 1 - c) / n_g and the
// iteration its L1 change first went below tol; the loop stops when every
// graph has converged (its L1 change has gone below tol once: an FP32
// iterate can settle into a rounding cycle whose change stays near tol) or
// at max_iter.
__global__ void __launch_bounds__(1024) k_batch_check(IterState *st, int ngraph,
                                                      cudaGraphConditionalHandle cond, int use_cond)
{
    if (st->done) return;
    __shared__ double smax[32];
    __shared__ int sall[32];
    const double c = st->c, tol = st->tol;
    const int it = st->iter + 1;
    double mx = 0.0;
    int all = 1;
    for (int g = threadIdx.x; g < ngraph; g += blockDim.x) {
        double l1 = 0.0, dg = 0.0;
        for (int q = st->gchunk[g]; q < st->gchunk[g + 1]; ++q) {
            const double2 v = st->cpart[q];
            l1 += v.x;
            dg += v.y;
        }
        st->gl1[g] = l1;
        st->gdelta[g] = dg;
        const double ng = (double)(st->goff[g + 1] - st->goff[g]);
        st->gbase[g] = (float)((c * dg + (1.0 - c)) / ng);
        if (tol > 0.0 && l1 < tol && st->giters[g] == 0) st->giters[g] = it;
        if (st->giters[g] == 0) all = 0;
        mx = fmax(mx, l1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
        all &= __shfl_xor_sync(kFull, all, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { smax[warp] = mx; sall[warp] = all; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        int a = 1;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { m = fmax(m, smax[w]); a &= sall[w]; }
        st->l1 = m;
        st->iter = it;
        st->parity ^= 1;
        const int done = it >= st->max_iter || (tol > 0.0 && a);
        st->done = done;
        if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
    }
}

void launch_batch_check(IterState *st, int ngraph, unsigned long long cond, int use_cond,
                        cudaStream_t s)
{
    k_batch_check<<<1, 1024, 0, s>>>(st, ngraph, (cudaGraphConditionalHandle)cond, use_cond);
    count_launches(1);
}

__global__ void k_batch_init(int64_t n, const IterState *__restrict__ st, float *__restrict__ x)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int g = st->gid[v];
        x[v] = (float)(1.0 / (double)(st->goff[g + 1] - st->goff[g]));
    }
}

// ------------------------------------------------------------- vectors --


__global__ void k_gather(int64_t n, const int32_t *__restrict__ inv, const float *__restrict__ x,
                         float *__restrict__ xp)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        xp[i] = __ldg(x + inv[i]);
}

void launch_gather(int64_t n, const int32_t *inv, const float *x, float *xp, cudaStream_t s)
{
    k_gather<<<grid_for(n), 256, 0, s>>>(n, inv, x, xp);
    count_launches(1);
}

__global__ void k_gather_rows(int64_t n, int k, const int32_t *__restrict__ inv,
                              const float *__restrict__ X, int64_t ldx, float *__restrict__ Xp)
{
    const int64_t total = n * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k, j = t % k;
        Xp[t] = __ldg(X + (int64_t)inv[i] * ldx + j);
    }
}

void launch_gather_rows(int64_t n, int k, const int32_t *inv, const float *X, int64_t ldx,
                        float *Xp, cudaStream_t s)
{
    k_gather_rows<<<grid_for(n * k), 256, 0, s>>>(n, k, inv, X, ldx, Xp);
    count_launches(1);
}

__global__ void k_scatter_axpby(int64_t n, const int32_t *__restrict__ inv,
                                const float *__restrict__ yp, float *__restrict__ y, float alpha,
                                float beta)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = inv ? (int64_t)inv[i] : i;
        const float v = alpha * yp[i];
        y[o] = beta != 0.f ? fmaf(beta, y[o], v) : v;
    }
}

void launch_scatter_axpby(int64_t n, const int32_t *inv, const float *yp, float *y, float alpha,
                          float beta, cudaStream_t s)
{
    k_scatter_axpby<<<grid_for(n), 256, 0, s>>>(n, inv, yp, y, alpha, beta);
    count_launches(1);
}

__global__ void k_scatter_rows(int64_t n, int k, const int32_t *__restrict__ inv,
                               const float *__restrict__ Yp, float *__restrict__ Y, int64_t ldy,
                               float alpha, float beta)
{
    const int64_t total = n * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k, j = t % k;
        float *dst = Y + (int64_t)inv[i] * ldy + j;
        const float v = alpha * Yp[t];
        *dst = beta != 0.f ? fmaf(beta, *dst, v) : v;
    }
}

void launch_scatter_rows(int64_t n, int k, const int32_t *inv, const float *Yp, float *Y,
                         int64_t ldy, float alpha, float beta, cudaStream_t s)
{
    k_scatter_rows<<<grid_for(n * k), 256, 0, s>>>(n, k, inv, Yp, Y, ldy, alpha, beta);
    count_launches(1);
}

// Vectors between the caller's order and the position order.  perm[j] is
// the position of node j.  Both directions read or write the caller's side
// in order: into positions, xp[perm[j]] = x[j] (* d[perm[j]]) reads x in
// order and scatters into xp; back, out[j] = (scaled) z[perm[j]] gathers
// from the positions and writes out in order.  The caller's side may be
// mapped (pinned) host memory, read or written straight over the host
// link in whole lines; on GB300 scattered 4-byte reads also cost less
// than scattered writes (67M floats: 1.04 ms gathering, 1.69-2.16 ms
// scattering).
__global__ void k_permute_in(int64_t n, const int32_t *__restrict__ perm, const float *__restrict__ x,
                             const float *__restrict__ d, float *__restrict__ xp)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = perm[j];
        xp[p] = d ? x[j] * __ldg(d + p) : x[j];
    }
}

void launch_permute_in(int64_t n, const int32_t *perm, const float *x, const float *d, float *xp,
                       cudaStream_t s)
{
    k_permute_in<<<grid_for(n), 256, 0, s>>>(n, perm, x, d, xp);
    count_launches(1);
}

__global__ void k_unpermute_state(int64_t n, const int32_t *__restrict__ perm,
                                  const IterState *__restrict__ st, float *__restrict__ out,
                                  const uint8_t *__restrict__ row_half, int hits)
{
    const float *z = st->buf[st->parity];
    float sc0 = 1.f, sc1 = 1.f;
    if (hits) { sc0 = (float)st->scale[0]; sc1 = (float)st->scale[1]; }
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = perm[j];
        float v = z[p];
        if (hits) v *= row_half[p] ? sc1 : sc0;
        out[j] = v;
    }
}

void launch_unpermute_state(int64_t n, const int32_t *perm, const IterState *st, float *out,
                            const uint8_t *row_half, int hits, cudaStream_t s)
{
    k_unpermute_state<<<grid_for(n), 256, 0, s>>>(n, perm, st, out, row_half, hits);
    count_launches(1);
}

__global__ void k_unpermute_axpby(int64_t n, const int32_t *__restrict__ perm,
                                  const float *__restrict__ yp, float *__restrict__ y, float alpha,
                                  float beta)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const float v = alpha * yp[perm[j]];
        y[j] = beta != 0.f ? fmaf(beta, y[j], v) : v;
    }
}

void launch_unpermute_axpby(int64_t n, const int32_t *perm, const float *yp, float *y, float alpha,
                            float beta, cudaStream_t s)
{
    k_unpermute_axpby<<<grid_for(n), 256, 0, s>>>(n, perm, yp, y, alpha, beta);
    count_launches(1);
}

// Rows of an n x k block back to original order: Y[j] = alpha Yp[pi(j)]
// (+ beta Y[j]), Y written row after row (it may be mapped host memory).
__global__ void k_unpermute_rows(int64_t n, int k, const int32_t *__restrict__ perm,
                                 const float *__restrict__ Yp, float *__restrict__ Y, int64_t ldy,
                                 float alpha, float beta)
{
    const int64_t total = n * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / k, c = t % k;
        float *dst = Y + j * ldy + c;
        const float v = alpha * __ldg(Yp + (int64_t)perm[j] * k + c);
        *dst = beta != 0.f ? fmaf(beta, *dst, v) : v;
    }
}

void launch_unpermute_rows(int64_t n, int k, const int32_t *perm, const float *Yp, float *Y,
                           int64_t ldy, float alpha, float beta, cudaStream_t s)
{
    k_unpermute_rows<<<grid_for(n * k), 256, 0, s>>>(n, k, perm, Yp, Y, ldy, alpha, beta);
    count_launches(1);
}

__global__ void k_fill(int64_t n, float v, float *__restrict__ p)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

void launch_batch_init(int64_t n, const IterState *st, float *x, cudaStream_t s)
{
    k_batch_init<<<grid_for(n), 256, 0, s>>>(n, st, x);
    count_launches(1);
}

__global__ void k_scale(int64_t n, const float *__restrict__ p, const float *__restrict__ d,
                        float *__restrict__ z)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        z[i] = p[i] * d[i];
}

void launch_scale(int64_t n, const float *p, const float *inv_deg, float *z, cudaStream_t s)
{
    k_scale<<<grid_for(n), 256, 0, s>>>(n, p, inv_deg, z);
    count_launches(1);
}

__global__ void k_gather_scaled(int64_t n, const int32_t *__restrict__ inv, const float *__restrict__ x,
                                const float *__restrict__ d, float *__restrict__ xp)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        xp[i] = __ldg(x + inv[i]) * d[i];
}

void launch_gather_scaled(int64_t n, const int32_t *inv, const float *x, const float *inv_deg,
                          float *xp, cudaStream_t s)
{
    k_gather_scaled<<<grid_for(n), 256, 0, s>>>(n, inv, x, inv_deg, xp);
    count_launches(1);
}

void launch_fill(int64_t n, float v, float *p, cudaStream_t s)
{
    k_fill<<<grid_for(n), 256, 0, s>>>(n, v, p);
    count_launches(1);
}

__global__ void k_onehot_rows(int64_t n, int k, const int32_t *__restrict__ seeds,
                              float *__restrict__ X)
{
    const int64_t total = n * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k, j = t % k;
        X[t] = (int64_t)seeds[j] == i ? 1.f : 0.f;
    }
}

void launch_onehot_rows(int64_t n, int k, const int32_t *seeds, float *X, cudaStream_t s)
{
    k_onehot_rows<<<grid_for(n * k), 256, 0, s>>>(n, k, seeds, X);
    count_launches(1);
}

// ------------------------------------------------------------- TILE-COO --
//
// The paper's TILE-COO kernel (Section 5: the tiled SpMV with COO storage,
// against which the composite storage is measured): the entries of one part
// as a (row, column, value) list sorted by row.  Warp w takes the intervals
// [a, a + kCooSpan) of the list (grid stride) in 32-entry coalesced steps.
// A step forms its 32 products, adds the segment left open by the step
// before to its first lane when the row continues, and runs an inclusive
// segmented scan over equal rows (rows are sorted, so equal neighbours form
// one segment).  A lane that ends a segment inside the step adds its sum to
// y; the last lane's segment stays open.  Only the first and the last row of
// an interval can continue into a neighbouring interval: those are added
// with atomicAdd, every other row with a plain read-add-write (its entries
// of this part lie in this interval alone, and parts run one after another).
constexpr int kCooSpan = 256;

__global__ void __launch_bounds__(256)
k_tile_coo(const int32_t *__restrict__ row, const int32_t *__restrict__ col,
           const float *__restrict__ val, int64_t e0, int64_t e1,
           const float *__restrict__ x, float *__restrict__ y)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = e0 + warp * kCooSpan; a < e1; a += nwarp * kCooSpan) {
        const int64_t b = min(a + (int64_t)kCooSpan, e1);
        const int first = __ldg(row + a);
        int crow = -1;       // row of the open segment (-1: none)
        float cval = 0.f;
        for (int64_t s = a; s < b; s += 32) {
            const int64_t e = s + lane;
            int r = -1;
            float v = 0.f;
            if (e < b) {
                r = __ldg(row + e);
                v = __ldg(val + e) * __ldg(x + __ldg(col + e));
            }
            const int r0 = __shfl_sync(kFull, r, 0);
            if (crow >= 0 && crow != r0) {      // the open segment ended with the last step
                if (lane == 0) {
                    if (crow == first) atomicAdd(y + crow, cval);
                    else y[crow] += cval;
                }
                crow = -1;
            }
            if (lane == 0 && crow >= 0) v += cval;
            for (int d = 1; d < 32; d <<= 1) {
                const float o = __shfl_up_sync(kFull, v, d);
                const int ro = __shfl_up_sync(kFull, r, d);
                if (lane >= d && ro == r) v += o;
            }
            const int rn = __shfl_down_sync(kFull, r, 1);
            if (lane < 31 && rn != r && r >= 0) {
                if (r == first) atomicAdd(y + r, v);
                else y[r] += v;
            }
            crow = __shfl_sync(kFull, r, 31);
            cval = __shfl_sync(kFull, v, 31);
        }
        if (lane == 0 && crow >= 0) atomicAdd(y + crow, cval);
    }
}

void launch_tile_coo(const int32_t *row, const int32_t *col, const float *val, int64_t e0,
                     int64_t e1, const float *x, float *y, int num_sms, cudaStream_t s)
{
    if (e1 <= e0) return;
    const int64_t spans = (e1 - e0 + kCooSpan - 1) / kCooSpan;
    int64_t blocks = (spans + 7) / 8;                    // one interval per warp
    const int64_t cap = (int64_t)(num_sms > 0 ? num_sms : 1) * 8;   // 64 warps per SM, grid stride
    if (blocks > cap) blocks = cap;
    k_tile_coo<<<(int)blocks, 256, 0, s>>>(row, col, val, e0, e1, x, y);
    count_launches(1);
}

// ------------------------------------------------------------ baselines --

template <int MODE>
__device__ __forceinline__ void csr_epilogue(const Epi &E, int64_t v, float acc,
                                             const uint8_t *dangling, const float *x, float *y,
                                             FSum &r0, FSum &r1)
{
    if (MODE == EPI_RAW) { y[v] = acc; return; }
    const float f = fmaf(E.c, acc, E.base);
    y[v] = f;
    r0.add(fabsf(f - x[v]));
    if (dangling[v]) r1.add(f);
}

// Appendix B CSR kernel: one thread per row.
template <int MODE>
__global__ void __launch_bounds__(kBlock)
k_csr_scalar(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
             const float *__restrict__ val, const uint8_t *__restrict__ dangling,
             const float *__restrict__ xin, float *__restrict__ yout,
             const IterState *__restrict__ st, double2 *__restrict__ red)
{
    const float *x = xin;
    float *y = yout;
    Epi E = load_epi<MODE>(st);
    if (st) { x = st->buf[st->parity]; y = st->buf[st->parity ^ 1]; }
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    FSum r0, r1;
    if (v < n) {
        float acc = 0.f;
        for (int64_t k = rp[v]; k < rp[v + 1]; ++k) acc = fmaf(val[k], __ldg(x + col[k]), acc);
        csr_epilogue<MODE>(E, v, acc, dangling, x, y, r0, r1);
    }
    if (MODE != EPI_RAW) block_reduce_store<MODE>(r0, r1, red + blockIdx.x);
}

// Appendix B CSR-vector kernel: one warp per row.
template <int MODE>
__global__ void __launch_bounds__(kBlock)
k_csr_vector(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
             const float *__restrict__ val, const uint8_t *__restrict__ dangling,
             const float *__restrict__ xin, float *__restrict__ yout,
             const IterState *__restrict__ st, double2 *__restrict__ red)
{
    const float *x = xin;
    float *y = yout;
    Epi E = load_epi<MODE>(st);
    if (st) { x = st->buf[st->parity]; y = st->buf[st->parity ^ 1]; }
    const int lane = threadIdx.x & 31;
    const int64_t v = blockIdx.x * (int64_t)kWarpsPerBlock + (threadIdx.x >> 5);
    FSum r0, r1;
    if (v < n) {
        float acc = 0.f;
        for (int64_t k = rp[v] + lane; k < rp[v + 1]; k += 32) acc = fmaf(val[k], __ldg(x + col[k]), acc);
        acc = warp_sum(acc);
        if (lane == 0) csr_epilogue<MODE>(E, v, acc, dangling, x, y, r0, r1);
    }
    if (MODE != EPI_RAW) block_reduce_store<MODE>(r0, r1, red + blockIdx.x);
}

int csr_scalar_blocks(int64_t n) { return (int)((n + kBlock - 1) / kBlock); }
int csr_vector_blocks(int64_t n) { return (int)((n + kWarpsPerBlock - 1) / kWarpsPerBlock); }

void launch_csr_scalar(int mode, int64_t n, const int64_t *rp, const int32_t *col,
                       const float *val, const uint8_t *dangling, const float *x, float *y,
                       const IterState *st, double2 *red, int *nblocks_out, cudaStream_t s)
{
    const int g = csr_scalar_blocks(n);
    if (nblocks_out) *nblocks_out = g;
    if (mode == EPI_RAW) k_csr_scalar<EPI_RAW><<<g, kBlock, 0, s>>>(n, rp, col, val, dangling, x, y, st, red);
    else k_csr_scalar<EPI_PAGERANK><<<g, kBlock, 0, s>>>(n, rp, col, val, dangling, x, y, st, red);
    count_launches(1);
}

void launch_csr_vector(int mode, int64_t n, const int64_t *rp, const int32_t *col,
                       const float *val, const uint8_t *dangling, const float *x, float *y,
                       const IterState *st, double2 *red, int *nblocks_out, cudaStream_t s)
{
    const int g = csr_vector_blocks(n);
    if (nblocks_out) *nblocks_out = g;
    if (mode == EPI_RAW) k_csr_vector<EPI_RAW><<<g, kBlock, 0, s>>>(n, rp, col, val, dangling, x, y, st, red);
    else k_csr_vector<EPI_PAGERANK><<<g, kBlock, 0, s>>>(n, rp, col, val, dangling, x, y, st, red);
    count_launches(1);
}

// ------------------------------------------------------ differentiable RWR --

// Softmax of the logits over each node's out-edges, written into the packed
// slots of the forward and transposed layouts.  Nodes of at most
// kEdgeHeavy out-edges take an 8-lane segment of a warp (four nodes per warp
// at once: the typical node has a few edges, so a whole warp per node would
// serialise the loads' latency node after node); the heavier ones (a short
// list built with the format) take a 256-thread block each, so that a hub's
// edges are not a long serial loop either.
constexpr int kEdgeLanes = 8;
constexpr int kEdgeHeavy = 64;

__device__ __forceinline__ unsigned seg_mask(int lane)
{
    return ((1u << kEdgeLanes) - 1u) << (lane & ~(kEdgeLanes - 1));
}

__device__ __forceinline__ float seg_max(float v, unsigned mask)
{
#pragma unroll
    for (int o = kEdgeLanes / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o, kEdgeLanes));
    return v;
}

__device__ __forceinline__ float seg_sum(float v, unsigned mask)
{
#pragma unroll
    for (int o = kEdgeLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, kEdgeLanes);
    return v;
}

// Block-wide max / sum of one value per thread (256 threads), result in
// every thread.
__device__ __forceinline__ float block_max256(float v, float *sm)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = sm[0];
    for (int w = 1; w < 8; ++w) r = fmaxf(r, sm[w]);
    __syncthreads();
    return r;
}

__device__ __forceinline__ float block_sum256(float v, float *sm)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = 0.f;
    for (int w = 0; w < 8; ++w) r += sm[w];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void store_weight(int64_t q, float p, const int64_t *es, uint2 *slab,
                                             const int64_t *est, uint2 *slab_t, float *P)
{
    if (P) P[q] = p;
    if (es) slab[es[q]].y = __float_as_uint(p);
    if (est) slab_t[est[q]].y = __float_as_uint(p);
}

__global__ void k_edge_softmax(int64_t n, const int64_t *__restrict__ rp,
                               const float *__restrict__ theta, const int64_t *__restrict__ es,
                               uint2 *slab, const int64_t *__restrict__ est, uint2 *slab_t,
                               float *__restrict__ P)
{
    const int sl = threadIdx.x & (kEdgeLanes - 1);
    const unsigned mask = seg_mask(threadIdx.x & 31);
    for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kEdgeLanes; u < n;
         u += ((int64_t)gridDim.x * blockDim.x) / kEdgeLanes) {
        const int64_t b = rp[u], e = rp[u + 1];
        if (b == e || e - b > kEdgeHeavy) continue;
        float m = -INFINITY;
        for (int64_t q = b + sl; q < e; q += kEdgeLanes) m = fmaxf(m, theta[q]);
        m = seg_max(m, mask);
        float sum = 0.f;
        for (int64_t q = b + sl; q < e; q += kEdgeLanes) sum += __expf(theta[q] - m);
        sum = seg_sum(sum, mask);
        const float inv = 1.f / sum;
        for (int64_t q = b + sl; q < e; q += kEdgeLanes)
            store_weight(q, __expf(theta[q] - m) * inv, es, slab, est, slab_t, P);
    }
}

__global__ void __launch_bounds__(256)
k_edge_softmax_heavy(const int32_t *__restrict__ heavy, const int64_t *__restrict__ rp,
                     const float *__restrict__ theta, const int64_t *__restrict__ es, uint2 *slab,
                     const int64_t *__restrict__ est, uint2 *slab_t, float *__restrict__ P)
{
    __shared__ float sm[8];
    const int64_t u = heavy[blockIdx.x];
    const int64_t b = rp[u], e = rp[u + 1];
    float m = -INFINITY;
    for (int64_t q = b + threadIdx.x; q < e; q += blockDim.x) m = fmaxf(m, theta[q]);
    m = block_max256(m, sm);
    float sum = 0.f;
    for (int64_t q = b + threadIdx.x; q < e; q += blockDim.x) sum += __expf(theta[q] - m);
    sum = block_sum256(sum, sm);
    const float inv = 1.f / sum;
    for (int64_t q = b + threadIdx.x; q < e; q += blockDim.x)
        store_weight(q, __expf(theta[q] - m) * inv, es, slab, est, slab_t, P);
}

void launch_edge_softmax(int64_t n, const int64_t *a_rp, const float *theta,
                         const int64_t *edge_slot, uint2 *slab, const int64_t *edge_slot_t,
                         uint2 *slab_t, float *P_out, const int32_t *heavy, int nheavy,
                         cudaStream_t s)
{
    k_edge_softmax<<<grid_for(n * kEdgeLanes), 256, 0, s>>>(n, a_rp, theta, edge_slot, slab,
                                                            edge_slot_t, slab_t, P_out);
    count_launches(1);
    if (nheavy > 0) {
        k_edge_softmax_heavy<<<nheavy, 256, 0, s>>>(heavy, a_rp, theta, edge_slot, slab,
                                                    edge_slot_t, slab_t, P_out);
        count_launches(1);
    }
}

// dL/dtheta over each node's out-edges (segments and heavy blocks as for
// the softmax).
__global__ void k_edge_grad(int64_t n, const int64_t *__restrict__ rp,
                            const int32_t *__restrict__ col, const float *__restrict__ P,
                            const float *__restrict__ lam, const float *__restrict__ r, float c,
                            float *__restrict__ dth)
{
    const int sl = threadIdx.x & (kEdgeLanes - 1);
    const unsigned mask = seg_mask(threadIdx.x & 31);
    for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kEdgeLanes; u < n;
         u += ((int64_t)gridDim.x * blockDim.x) / kEdgeLanes) {
        const int64_t b = rp[u], e = rp[u + 1];
        if (b == e || e - b > kEdgeHeavy) continue;
        const float cr = c * r[u];
        float dot = 0.f;
        for (int64_t q = b + sl; q < e; q += kEdgeLanes) dot = fmaf(P[q], cr * lam[col[q]], dot);
        dot = seg_sum(dot, mask);
        for (int64_t q = b + sl; q < e; q += kEdgeLanes) dth[q] = P[q] * (cr * lam[col[q]] - dot);
    }
}

__global__ void __launch_bounds__(256)
k_edge_grad_heavy(const int32_t *__restrict__ heavy, const int64_t *__restrict__ rp,
                  const int32_t *__restrict__ col, const float *__restrict__ P,
                  const float *__restrict__ lam, const float *__restrict__ r, float c,
                  float *__restrict__ dth)
{
    __shared__ float sm[8];
    const int64_t u = heavy[blockIdx.x];
    const int64_t b = rp[u], e = rp[u + 1];
    const float cr = c * r[u];
    float dot = 0.f;
    for (int64_t q = b + threadIdx.x; q < e; q += blockDim.x) dot = fmaf(P[q], cr * lam[col[q]], dot);
    dot = block_sum256(dot, sm);
    for (int64_t q = b + threadIdx.x; q < e; q += blockDim.x) dth[q] = P[q] * (cr * lam[col[q]] - dot);
}

void launch_edge_grad(int64_t n, const int64_t *a_rp, const int32_t *a_col, const float *P,
                      const float *lambda, const float *r, float c, float *dtheta,
                      const int32_t *heavy, int nheavy, cudaStream_t s)
{
    k_edge_grad<<<grid_for(n * kEdgeLanes), 256, 0, s>>>(n, a_rp, a_col, P, lambda, r, c, dtheta);
    count_launches(1);
    if (nheavy > 0) {
        k_edge_grad_heavy<<<nheavy, 256, 0, s>>>(heavy, a_rp, a_col, P, lambda, r, c, dtheta);
        count_launches(1);
    }
}

int edge_heavy_degree() { return kEdgeHeavy; }

}  // namespace spg
