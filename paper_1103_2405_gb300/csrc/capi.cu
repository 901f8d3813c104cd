// capi.cu -- the extern "C" boundary (include/spg.h): handles, workspace,
// the power-iteration drivers and the exports of the layout plan.
//
// Power iterations run entirely on the device: per iteration one launch per
// part with the fused epilogue (Appendix F) and one check kernel that sums
// the per-block FP64 partials in a fixed order, updates the scalars and the
// ping-pong parity, and sets the conditional of a CUDA-graph WHILE node, so
// the loop needs no host round trip.  Graphs are built once per handle and
// loop kind and reused (every parameter lives in device memory).
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/spg.h"
#include "format.h"
#include "kernels.h"

using namespace spg;

// Default cap on the rows of one workload (spg_build_opts.max_rows = 0).
static constexpr int64_t kDefaultUnitSlots = 2048;   // claim unit cost (measured)
static constexpr int64_t kBatchChunk = 8192;         // positions per chunk of the per-graph sums
// Auto tile width: the largest power of two of columns whose x slice fits
// this fraction of the L2 (16M columns on GB300: R-MAT 26 3.61 ms per
// PageRank iteration vs 3.68 ms with the 8M columns of a 40 % fraction).
static constexpr double kTileL2Fraction = 0.6;
static constexpr int64_t kDefaultMaxRows = 32;

static thread_local std::string g_err;

static spg_status fail(spg_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

static spg_status cuda_fail(cudaError_t e, const char *where)
{
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return SPG_ERR_CUDA;
}

#define CK(call)                                                       \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);            \
    } while (0)

namespace {

struct LoopGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels_per_iter = 0;
    // host-loop mode: the iteration body, launched directly (valid during one call)
    std::function<void(cudaStream_t, unsigned long long, int)> body;
};

// Device buffer that grows on demand.  A reallocation bumps *epoch, which
// invalidates every cached loop graph (they capture buffer addresses).
template <class T> struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    uint64_t *epoch = nullptr;
    cudaError_t ensure(size_t count)
    {
        if (count <= n && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        if (epoch) ++*epoch;
        cudaError_t e = cudaMalloc((void **)&p, std::max<size_t>(1, count) * sizeof(T));
        if (e == cudaSuccess) n = count;
        return e;
    }
    void release() { if (p) cudaFree(p); p = nullptr; n = 0; }
};

}  // namespace

struct spg_format_t {
    spg_kind kind = SPG_KIND_MATRIX;
    int device = 0;
    bool host_only = false;
    int64_t n_graph = 0;       // nodes of the graph (HITS: layout is 2n)
    int64_t nnz_in = 0;        // non-zeros of the input CSR
    Layout fwd;
    std::unique_ptr<Layout> bwd;
    // baselines: M in original order
    int64_t *d_rp = nullptr;
    int32_t *d_col = nullptr;
    float *d_val = nullptr;
    uint8_t *d_dangling = nullptr;
    // HITS: per permuted position, 1 if in the hub half
    uint8_t *d_row_half = nullptr;
    // row partition (Section 3.2): this handle's rank, the rank count and the
    // owner rank of every permuted position
    int32_t part_id = -1, nparts = 0;
    int8_t *d_owner = nullptr;
    DevBuf<double2> red_ranks;       // spg_pagerank_ranks: all ranks' reduction slots
    DevBuf<IterState *> rank_states; // spg_pagerank_ranks: the ranks' states
    // BATCH: graph offsets and per-graph state
    int ngraph = 0;
    std::vector<int64_t> goff;
    int64_t *d_goff = nullptr, *d_gdstart = nullptr;
    int32_t *d_gid = nullptr, *d_giters = nullptr;
    float *d_gbase = nullptr;
    double *d_gl1 = nullptr, *d_gdelta = nullptr;
    int nchunk = 0;                  // fixed position chunks of the per-graph sums
    int64_t *d_cstart = nullptr;
    int32_t *d_cgraph = nullptr, *d_gchunk = nullptr;
    double2 *d_cpart = nullptr;
    // WEIGHTED: A on the device and the current transition weights
    int64_t *d_arp = nullptr;
    int32_t *d_acol = nullptr;
    float *d_P = nullptr;
    int32_t *d_heavy = nullptr;      // nodes of many out-edges (block-per-node edge kernels)
    int nheavy = 0;
    // workspace
    DevBuf<float> x, y, stage_in, stage_out;
    DevBuf<double2> red;
    DevBuf<double> redk, delta_k, l1_k;
    DevBuf<double> colsum;       // first-stage partials of the k-column sums
    DevBuf<float> partial_k;
    DevBuf<int32_t> seeds;
    DevBuf<float> X, Y;
    DevBuf<float> aux, stage_r;
    DevBuf<float> z0, z1;        // pattern-only PageRank: gathered iterates
    DevBuf<double> init_part;    // block partials of the start vector's dangling mass
    IterState *d_state = nullptr;
    // launch views of the parts: plain (8-warp blocks) and staged (x slice in smem)
    struct Views {
        std::vector<PartView> v;
        int32_t nblk = 0;
        bool built = false;
    };
    struct LayoutRT {
        Views vplain, vstaged;
        DevBuf<uint32_t> sched;  // staged-kernel counters, 2 per part (zero between launches)
    } rt_fwd, rt_bwd;
    int64_t stage_cols = kStagedMaxCols;
    int32_t pf_ahead = 0;        // L2 bulk-prefetch distance of the slot stream (bytes, 0 = off)
    int kernel = 4;              // 1: staged x slice, 2: plain, 3: TMA ring, 4 (and 0): persistent plain
    int persist_blocks = 5;      // kernel 4: resident 8-warp blocks per SM
    uint32_t *d_status = nullptr;   // set by kernels whose bounded waits ran out
    // pinned host copies the loop's final state and the status word are read
    // back into without a synchronisation of their own
    IterState *hs_pinned = nullptr;
    uint32_t *status_pinned = nullptr;
    int loop_mode = 0;           // 0: CUDA-graph WHILE loop, 1: host loop
    bool separate_check = false; // convergence check in its own kernel (not fused)
    int num_sms = 152;
    std::map<std::string, LoopGraph> graphs;
    LoopGraph host_loop;         // loop_mode 1
    uint64_t epoch = 0;          // workspace generation the cached graphs were built for
    uint64_t graphs_epoch = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    spg_format_t()
    {
        for (DevBuf<float> *b : {&x, &y, &partial_k, &X, &Y, &z0, &z1}) b->epoch = &epoch;
        red.epoch = &epoch;
        redk.epoch = &epoch;
        delta_k.epoch = &epoch;
        l1_k.epoch = &epoch;
        colsum.epoch = &epoch;
        seeds.epoch = &epoch;
    }

    void drop_graphs()
    {
        for (auto &kv : graphs) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        }
        graphs.clear();
    }

    ~spg_format_t()
    {
        if (host_only) return;
        fwd.free_device();
        if (bwd) bwd->free_device();
        cudaFree(d_rp); cudaFree(d_col); cudaFree(d_val); cudaFree(d_dangling);
        cudaFree(d_row_half); cudaFree(d_arp); cudaFree(d_acol); cudaFree(d_P); cudaFree(d_owner);
        cudaFree(d_heavy);
        red_ranks.release(); rank_states.release();
        cudaFree(d_goff); cudaFree(d_gdstart); cudaFree(d_gid); cudaFree(d_giters);
        cudaFree(d_status);
        if (hs_pinned) cudaFreeHost(hs_pinned);
        if (status_pinned) cudaFreeHost(status_pinned);
        cudaFree(d_gbase); cudaFree(d_gl1); cudaFree(d_gdelta);
        cudaFree(d_cstart); cudaFree(d_cgraph); cudaFree(d_gchunk); cudaFree(d_cpart);
        x.release(); y.release(); stage_in.release(); stage_out.release(); red.release();
        rt_fwd.sched.release();
        rt_bwd.sched.release();
        redk.release(); delta_k.release(); l1_k.release(); partial_k.release(); seeds.release();
        X.release(); Y.release(); aux.release(); stage_r.release(); init_part.release();
        z0.release(); z1.release(); colsum.release();
        cudaFree(d_state);
        for (auto &kv : graphs) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        }
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};

// ------------------------------------------------------------------ util --

static bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int64_t pow2_floor(int64_t v)
{
    int64_t p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

// Resolved tile width: explicit, none (< 0), or auto from the L2 size.
static int64_t resolve_tile_width(const spg_build_opts &o, int64_t l2_bytes)
{
    if (o.tile_width > 0) return o.tile_width;
    if (o.tile_width < 0) return 0;
    int64_t cols = (int64_t)(kTileL2Fraction * (double)l2_bytes) / 4;
    return pow2_floor(std::max<int64_t>(cols, 1024));
}

static spg_status check_csr(const spg_csr *c, std::vector<int64_t> &rp, std::vector<int32_t> &col,
                            std::vector<float> &val, const int64_t *&prp, const int32_t *&pcol,
                            const float *&pval)
{
    if (!c || c->n_rows < 1 || c->n_rows != c->n_cols || c->nnz < 0)
        return fail(SPG_ERR_INVALID, "CSR must be square with n >= 1 and nnz >= 0");
    if (c->n_rows >= kMaxN) return fail(SPG_ERR_INVALID, "n must be < 2^28");
    if (!c->row_ptr || (c->nnz > 0 && !c->col)) return fail(SPG_ERR_INVALID, "null CSR array");
    const int64_t n = c->n_rows, nnz = c->nnz;
    prp = c->row_ptr; pcol = c->col; pval = c->val;
    if (c->on_device) {
        rp.resize((size_t)n + 1);
        CK(cudaMemcpy(rp.data(), c->row_ptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
        col.resize((size_t)nnz);
        if (nnz) CK(cudaMemcpy(col.data(), c->col, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (c->val) {
            val.resize((size_t)nnz);
            if (nnz) CK(cudaMemcpy(val.data(), c->val, nnz * sizeof(float), cudaMemcpyDeviceToHost));
            pval = val.data();
        }
        prp = rp.data(); pcol = col.data();
    }
    if (prp[0] != 0 || prp[n] != nnz) return fail(SPG_ERR_INVALID, "row_ptr[0] != 0 or row_ptr[n] != nnz");
    std::atomic<bool> bad{false};
    parallel_for(n, 1 << 16, [&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi && !bad; ++i)
            if (prp[i + 1] < prp[i]) bad = true;
    });
    if (bad) return fail(SPG_ERR_INVALID, "row_ptr is not non-decreasing");
    parallel_for(nnz, 1 << 18, [&](int64_t lo, int64_t hi) {
        for (int64_t k = lo; k < hi && !bad; ++k)
            if (pcol[k] < 0 || pcol[k] >= n) bad = true;
    });
    if (bad) return fail(SPG_ERR_INVALID, "column index out of range");
    return SPG_OK;
}

// CSR (by rows) -> CSC of the same matrix: colptr, rowidx, val, entry ids.
static void csr_to_csc(int64_t n, const int64_t *rp, const int32_t *col, const float *val,
                       std::vector<int64_t> &cp, std::vector<int32_t> &ri, std::vector<float> &cv,
                       std::vector<int64_t> &eid)
{
    const int64_t nnz = rp[n];
    cp.assign((size_t)n + 1, 0);
    for (int64_t k = 0; k < nnz; ++k) cp[(size_t)col[k] + 1]++;
    for (int64_t j = 0; j < n; ++j) cp[(size_t)j + 1] += cp[(size_t)j];
    std::vector<int64_t> fill(cp.begin(), cp.end() - 1);
    ri.resize((size_t)nnz); cv.resize((size_t)nnz); eid.resize((size_t)nnz);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            int64_t s = fill[(size_t)col[k]]++;
            ri[(size_t)s] = (int32_t)i;
            cv[(size_t)s] = val ? val[k] : 1.0f;
            eid[(size_t)s] = k;
        }
}

template <class T> static cudaError_t upload(T **d, const T *h, size_t count)
{
    cudaError_t e = cudaMalloc((void **)d, std::max<size_t>(1, count) * sizeof(T));
    if (e != cudaSuccess) return e;
    if (count) e = cudaMemcpy(*d, h, count * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

static int64_t query_max_warps()
{
    int dev = 0, sms = 0, blocks = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 9728;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    blocks = part_blocks_per_sm();
    if (blocks <= 0) {
        int per = 0;
        cudaDeviceGetAttribute(&per, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
        blocks = per / kBlock;
    }
    return (int64_t)sms * blocks * kWarpsPerBlock;
}

// ----------------------------------------------------------------- build --

// Columns of the shared-memory x slice (option 1): x_stage_cols, 0 = the
// default, < 0 = none.
static int64_t resolve_stage_cols(const spg_build_opts &o)
{
    return o.x_stage_cols < 0 ? 0
         : (o.x_stage_cols > 0 ? std::min<int64_t>(o.x_stage_cols, kStagedMaxCols) : kStagedDefaultCols);
}

// Upload the forward layout and set up the launch-time state of a handle.
static spg_status device_setup(spg_handle h, const spg_build_opts &o, cudaStream_t s)
{
    cudaError_t e = upload_layout(h->fwd, o.keep_plan != 0, s);
    if (e == cudaErrorMemoryAllocation) return fail(SPG_ERR_OOM, "device memory for the format");
    if (e != cudaSuccess) return cuda_fail(e, "upload");
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    h->stage_cols = resolve_stage_cols(o);
    h->pf_ahead = o.slab_prefetch > 0 ? (int32_t)std::min<int64_t>(o.slab_prefetch, 1 << 20) : 0;
    h->pf_ahead = (h->pf_ahead + 255) / 256 * 256;
    h->loop_mode = o.loop_mode == 1 ? 1 : 0;
    h->separate_check = o.separate_check != 0;
    h->kernel = (o.kernel >= 0 && o.kernel <= 4) ? o.kernel : 0;
    if (o.x_stage_cols < 0 && h->kernel == 1) h->kernel = 2;   // no shared-memory staging at all
    // the default: one persistent 32-warp block per SM with the part's
    // densest x columns in shared memory (option 1); without a slice, the
    // persistent 8-warp blocks (option 4)
    if (h->kernel == 0) h->kernel = o.x_stage_cols < 0 ? 4 : 1;
    {   // option 4's blocks per SM (also option 1's choice for parts whose
        // slice would serve few entries)
        const int b = persist_blocks_per_sm();
        h->persist_blocks = b > 0 ? b : 1;
    }
    CK(cudaMalloc((void **)&h->d_status, sizeof(uint32_t)));
    CK(cudaMemset(h->d_status, 0, sizeof(uint32_t)));
    CK(cudaMallocHost((void **)&h->hs_pinned, sizeof(IterState)));
    CK(cudaMallocHost((void **)&h->status_pinned, sizeof(uint32_t)));
    *h->status_pinned = 0u;
    CK(h->rt_fwd.sched.ensure(2 * h->fwd.parts.size() + 1));
    CK(cudaMemset(h->rt_fwd.sched.p, 0, (2 * h->fwd.parts.size() + 1) * sizeof(uint32_t)));
    CK(cudaMalloc((void **)&h->d_state, sizeof(IterState)));
    CK(cudaEventCreate(&h->ev0));
    CK(cudaEventCreate(&h->ev1));
    return SPG_OK;
}

extern "C" spg_status spg_build_format(const spg_csr *csr, spg_kind kind,
                                       const spg_build_opts *opts_in, void *stream,
                                       spg_handle *out)
{
    try {
        if (!out) return fail(SPG_ERR_INVALID, "out is NULL");
        *out = nullptr;
        spg_build_opts o;
        std::memset(&o, 0, sizeof o);
        o.heavy_row = -1;
        o.layout_rule = 1;
        if (opts_in) o = *opts_in;
        if (kind < SPG_KIND_MATRIX || kind > SPG_KIND_WEIGHTED) return fail(SPG_ERR_INVALID, "bad kind");
        std::vector<int64_t> hrp;
        std::vector<int32_t> hcol;
        std::vector<float> hval;
        const int64_t *rp;
        const int32_t *col;
        const float *val;
        spg_status st = check_csr(csr, hrp, hcol, hval, rp, col, val);
        if (st != SPG_OK) return st;
        if (kind == SPG_KIND_MATRIX && !val) return fail(SPG_ERR_INVALID, "MATRIX kind needs values");
        if (kind == SPG_KIND_WEIGHTED && !val) return fail(SPG_ERR_INVALID, "WEIGHTED kind needs logits");
        const int64_t n = csr->n_rows, nnz = csr->nnz;
        if (kind == SPG_KIND_HITS && 2 * n >= kMaxN) return fail(SPG_ERR_INVALID, "2n must be < 2^28");

        std::unique_ptr<spg_format_t> h(new spg_format_t());
        h->kind = kind;
        h->host_only = o.device < 0;
        h->n_graph = n;
        h->nnz_in = nnz;
        cudaStream_t s = (cudaStream_t)stream;
        int64_t l2 = 126LL << 20;
        if (!h->host_only) {
            CK(cudaGetDevice(&h->device));
            int l2i = 0;
            cudaDeviceGetAttribute(&l2i, cudaDevAttrL2CacheSize, h->device);
            if (l2i > 0) l2 = l2i;
        }
        BuildParams prm;
        prm.tile_width = resolve_tile_width(o, l2);
        prm.wl = o.wl;
        prm.heavy = o.heavy_row;
        prm.layout_rule = (o.layout_rule >= 0 && o.layout_rule <= kAutoRule) ? o.layout_rule : 1;
        prm.max_warps = o.max_warps > 0 ? o.max_warps : (h->host_only ? 9728 : query_max_warps());
        prm.max_rows = o.max_rows < 0 ? 0 : (o.max_rows > 0 ? o.max_rows : kDefaultMaxRows);
        if (o.split_cost > 0) prm.split_cost = o.split_cost;
        prm.keep_plan = o.keep_plan != 0;
        prm.track_edges = kind == SPG_KIND_WEIGHTED;
        prm.stage_cols = resolve_stage_cols(o);
        if (o.pattern_only && kind != SPG_KIND_PAGERANK)
            return fail(SPG_ERR_INVALID, "pattern_only needs a PAGERANK handle");
        prm.pattern_only = o.pattern_only != 0;
        prm.unit_slots = o.unit_slots > 0 ? o.unit_slots : kDefaultUnitSlots;
        if (o.claim_order < 0 || o.claim_order > 1) return fail(SPG_ERR_INVALID, "claim_order must be 0 or 1");
        prm.claim_order = o.claim_order;
        prm.build_coo = o.tile_coo != 0;
        std::vector<uint8_t> rkeep;
        if (o.row_part) {
            if (kind != SPG_KIND_PAGERANK) return fail(SPG_ERR_INVALID, "row_part needs a PAGERANK handle");
            if (o.nparts < 1 || o.nparts > 64 || o.part_id < 0 || o.part_id >= o.nparts)
                return fail(SPG_ERR_INVALID, "row_part needs 1 <= nparts <= 64 and 0 <= part_id < nparts");
            if (o.keep_csr) return fail(SPG_ERR_INVALID, "keep_csr holds the whole matrix: not with row_part");
            rkeep.resize((size_t)n);
            for (int64_t v = 0; v < n; ++v) {
                const int32_t q = o.row_part[v];
                if (q < 0 || q >= o.nparts) return fail(SPG_ERR_INVALID, "row_part entry out of range");
                rkeep[(size_t)v] = q == o.part_id ? 1 : 0;
            }
        }
        if (o.tune_table_path) {
            std::string err;
            if (!perf_table_load(o.tune_table_path, perf_table(), err)) return fail(SPG_ERR_INVALID, err);
        }

        // column source of the matrix to format
        ColumnSource src;
        std::vector<int64_t> cp, eid;
        std::vector<int32_t> ri;
        std::vector<float> cv;
        std::vector<uint8_t> rclass;
        std::vector<float> mval;   // PAGERANK values per entry of A
        if (kind == SPG_KIND_MATRIX) {
            csr_to_csc(n, rp, col, val, cp, ri, cv, eid);
            src.n = n; src.colptr = cp.data(); src.rowidx = ri.data(); src.val = cv.data();
            src.eid = eid.data();
        } else if (kind == SPG_KIND_PAGERANK || kind == SPG_KIND_WEIGHTED) {
            // column u of M = row u of A; value fl32(1/outdeg(u)) (Eq. 6), or the
            // softmax of u's logits (WEIGHTED)
            mval.resize((size_t)nnz);
            parallel_for(n, 1 << 14, [&](int64_t lo, int64_t hi) {
                for (int64_t u = lo; u < hi; ++u) {
                    const int64_t b = rp[u], e = rp[u + 1];
                    if (b == e) continue;
                    if (kind == SPG_KIND_PAGERANK) {
                        const float w = (float)(1.0 / (double)(e - b));
                        for (int64_t k = b; k < e; ++k) mval[(size_t)k] = w;
                    } else {
                        double m = -INFINITY, sum = 0.0;
                        for (int64_t k = b; k < e; ++k) m = std::max(m, (double)val[k]);
                        for (int64_t k = b; k < e; ++k) sum += std::exp((double)val[k] - m);
                        for (int64_t k = b; k < e; ++k)
                            mval[(size_t)k] = (float)(std::exp((double)val[k] - m) / sum);
                    }
                }
            });
            src.n = n; src.colptr = rp; src.rowidx = col; src.val = mval.data(); src.eid = nullptr;
            if (!rkeep.empty()) src.row_keep = rkeep.data();
        } else {  // HITS: B = [[0, A^T], [A, 0]] of Eq. 8
            // column v < n: rows n+u for edges u->v (A's CSC); column n+u: rows v (A's CSR row u)
            std::vector<int64_t> acp, aeid;
            std::vector<int32_t> ari;
            std::vector<float> acv;
            csr_to_csc(n, rp, col, nullptr, acp, ari, acv, aeid);
            cp.assign((size_t)(2 * n + 1), 0);
            for (int64_t j = 0; j < n; ++j) cp[(size_t)j + 1] = cp[(size_t)j] + (acp[(size_t)j + 1] - acp[(size_t)j]);
            for (int64_t u = 0; u < n; ++u) cp[(size_t)(n + u + 1)] = cp[(size_t)(n + u)] + (rp[u + 1] - rp[u]);
            ri.resize((size_t)(2 * nnz));
            cv.assign((size_t)(2 * nnz), 1.0f);
            for (int64_t j = 0; j < n; ++j)
                for (int64_t k = acp[(size_t)j], q = cp[(size_t)j]; k < acp[(size_t)j + 1]; ++k, ++q)
                    ri[(size_t)q] = (int32_t)(n + ari[(size_t)k]);
            for (int64_t u = 0; u < n; ++u)
                for (int64_t k = rp[u], q = cp[(size_t)(n + u)]; k < rp[u + 1]; ++k, ++q)
                    ri[(size_t)q] = col[k];
            rclass.assign((size_t)(2 * n), 0);
            for (int64_t i = n; i < 2 * n; ++i) rclass[(size_t)i] = 1;
            src.n = 2 * n; src.colptr = cp.data(); src.rowidx = ri.data(); src.val = cv.data();
            src.row_class = rclass.data();
        }
        std::string err;
        if (!build_layout(src, prm, h->fwd, err)) return fail(SPG_ERR_INVALID, err);
        if (o.row_part) {
            h->part_id = o.part_id;
            h->nparts = o.nparts;
        }

        if (!h->host_only) {
            st = device_setup(h.get(), o, s);
            if (st != SPG_OK) return st;
            const int64_t N = h->fwd.n;
            if (o.row_part) {
                std::vector<int8_t> owner((size_t)N);
                for (int64_t k = 0; k < N; ++k) owner[(size_t)k] = (int8_t)o.row_part[h->fwd.inv[(size_t)k]];
                CK(upload(&h->d_owner, owner.data(), owner.size()));
            }
            if (kind == SPG_KIND_HITS) {
                std::vector<uint8_t> half((size_t)N);
                for (int64_t k = 0; k < N; ++k) half[(size_t)k] = h->fwd.inv[(size_t)k] >= n ? 1 : 0;
                CK(upload(&h->d_row_half, half.data(), half.size()));
            }
            if (o.keep_csr && (kind == SPG_KIND_PAGERANK || kind == SPG_KIND_MATRIX)) {
                // M in original order by rows: transpose of the column source
                std::vector<int64_t> mrp, meid;
                std::vector<int32_t> mcol;
                std::vector<float> mv;
                csr_to_csc(n, src.colptr, src.rowidx, src.val, mrp, mcol, mv, meid);
                CK(upload(&h->d_rp, mrp.data(), mrp.size()));
                CK(upload(&h->d_col, mcol.data(), mcol.size()));
                CK(upload(&h->d_val, mv.data(), mv.size()));
                std::vector<uint8_t> dang((size_t)n);
                for (int64_t u = 0; u < n; ++u) dang[(size_t)u] = (src.colptr[u + 1] == src.colptr[u]) ? 1 : 0;
                CK(upload(&h->d_dangling, dang.data(), dang.size()));
            }
            if (kind == SPG_KIND_WEIGHTED) {
                CK(upload(&h->d_arp, rp, (size_t)n + 1));
                CK(upload(&h->d_acol, col, (size_t)nnz));
                std::vector<int32_t> heavy;
                for (int64_t v = 0; v < n; ++v)
                    if (rp[v + 1] - rp[v] > edge_heavy_degree()) heavy.push_back((int32_t)v);
                h->nheavy = (int)heavy.size();
                CK(upload(&h->d_heavy, heavy.data(), heavy.size()));
                CK(upload(&h->d_P, mval.data(), (size_t)nnz));
                if (o.build_transpose) {
                    // M^T: rows u (sources), entries (v, P_e) -> column source of M^T is
                    // M's CSR by rows, i.e. the CSC of A's pattern with values P
                    std::vector<int64_t> tcp, teid;
                    std::vector<int32_t> tri;
                    std::vector<float> tcv;
                    csr_to_csc(n, rp, col, mval.data(), tcp, tri, tcv, teid);
                    ColumnSource ts;
                    ts.n = n; ts.colptr = tcp.data(); ts.rowidx = tri.data(); ts.val = tcv.data();
                    ts.eid = teid.data();
                    // rows of M^T with no entries are the dangling nodes: they also
                    // receive c * lambda_s in the adjoint (class bit)
                    std::vector<uint8_t> dcls((size_t)n);
                    for (int64_t u = 0; u < n; ++u) dcls[(size_t)u] = rp[u + 1] == rp[u] ? 1 : 0;
                    ts.row_class = dcls.data();
                    h->bwd.reset(new Layout());
                    prm.build_coo = false;
                    if (!build_layout(ts, prm, *h->bwd, err)) return fail(SPG_ERR_INVALID, err);
                    cudaError_t e = upload_layout(*h->bwd, o.keep_plan != 0, s);
                    if (e != cudaSuccess) return cuda_fail(e, "upload transpose");
                    CK(h->rt_bwd.sched.ensure(2 * h->bwd->parts.size() + 1));
                    CK(cudaMemset(h->rt_bwd.sched.p, 0, (2 * h->bwd->parts.size() + 1) * sizeof(uint32_t)));
                }
            }
        }
        *out = h.release();
        return SPG_OK;
    } catch (const std::bad_alloc &) {
        return fail(SPG_ERR_OOM, "host memory");
    } catch (const std::exception &ex) {
        return fail(SPG_ERR_INVALID, ex.what());
    }
}

extern "C" spg_status spg_destroy(spg_handle h)
{
    delete h;
    return SPG_OK;
}

extern "C" spg_status spg_format_info(spg_handle h, spg_format_info_t *info)
{
    if (!h || !info) return fail(SPG_ERR_INVALID, "null argument");
    const Layout &L = h->fwd;
    std::memset(info, 0, sizeof *info);
    info->n = L.n;
    info->nnz = L.nnz;
    info->ntile = L.ntile;
    info->tile_width = L.tile_width;
    int64_t nw = 0;
    double pm = 0;
    for (const PartHost &p : L.parts) { nw += p.nwl_total; pm += p.predicted_s; }
    info->nworkloads = nw;
    info->padded_slots = L.padded_slots;
    info->split_rows = L.nsplit;
    info->split_chunks = L.nchunk_slots;
    info->zero_rows = (int64_t)L.zero_rows.size();
    info->device_bytes = L.device_bytes + (h->bwd ? h->bwd->device_bytes : 0);
    info->max_warps = L.max_warps;
    info->predicted_ms = pm * 1e3;
    info->dangling_start = L.dangling_start;
    return SPG_OK;
}

extern "C" spg_status spg_tile_info(spg_handle h, int64_t part, spg_tile_info_t *info)
{
    if (!h || !info || part < 0 || part >= (int64_t)h->fwd.parts.size())
        return fail(SPG_ERR_INVALID, "bad part");
    const PartHost &p = h->fwd.parts[(size_t)part];
    info->col_begin = p.c0;
    info->col_end = p.c1;
    info->heavy = p.heavy;
    info->wl = p.wl;
    info->nvirt = p.nvirt;
    info->nwl = p.nwl;
    info->nnz = p.nnz;
    info->predicted_ms = p.predicted_s * 1e3;
    info->layout_rule = p.rule;
    info->slice_share = p.slice_share;
    info->nunits = p.nunits;
    return SPG_OK;
}

extern "C" spg_status spg_format_perm(spg_handle h, int32_t *pi, int32_t *inv)
{
    if (!h) return fail(SPG_ERR_INVALID, "null handle");
    if (pi) std::memcpy(pi, h->fwd.perm.data(), h->fwd.perm.size() * sizeof(int32_t));
    if (inv) std::memcpy(inv, h->fwd.inv.data(), h->fwd.inv.size() * sizeof(int32_t));
    return SPG_OK;
}

extern "C" spg_status spg_format_export_plan(spg_handle h, int64_t part, int64_t *rank_row,
                                             int64_t *rank_chunk, int64_t *rank_len,
                                             int64_t *wl_first, int64_t *wl_h, int64_t *wl_w,
                                             int64_t *wl_major)
{
    if (!h || part < 0 || part >= (int64_t)h->fwd.parts.size()) return fail(SPG_ERR_INVALID, "bad part");
    const PartHost &p = h->fwd.parts[(size_t)part];
    if ((int64_t)p.rank_len.size() != p.nvirt) return fail(SPG_ERR_INVALID, "plan not kept (keep_plan)");
    for (int64_t i = 0; i < p.nvirt; ++i) {
        if (rank_row) rank_row[i] = p.rank_row[(size_t)i];
        if (rank_chunk) rank_chunk[i] = p.rank_chunk[(size_t)i];
        if (rank_len) rank_len[i] = p.rank_len[(size_t)i];
    }
    for (int64_t j = 0; j < p.nwl; ++j) {
        if (wl_first) wl_first[j] = p.wl_first[(size_t)j];
        if (wl_h) wl_h[j] = p.wl_h[(size_t)j];
        if (wl_w) wl_w[j] = p.wl_w[(size_t)j];
        if (wl_major) wl_major[j] = p.wl_major[(size_t)j];
    }
    return SPG_OK;
}

extern "C" spg_status spg_format_zero_rows(spg_handle h, int64_t *rows)
{
    if (!h || !rows) return fail(SPG_ERR_INVALID, "null argument");
    std::memcpy(rows, h->fwd.zero_rows.data(), h->fwd.zero_rows.size() * sizeof(int64_t));
    return SPG_OK;
}

extern "C" spg_status spg_format_export_entries(spg_handle h, int64_t *orows, int32_t *ocols,
                                                float *ovals)
{
    if (!h) return fail(SPG_ERR_INVALID, "null handle");
    const Layout &L = h->fwd;
    std::vector<Workload> wl = L.wl;
    std::vector<uint32_t> rows = L.rows;
    std::vector<uint2> slab = L.slab;
    if (L.pattern && !L.slab4.empty()) {
        slab.resize(L.slab4.size());
        for (size_t i = 0; i < slab.size(); ++i) {
            slab[i].x = L.slab4[i];
            float v = (int32_t)L.slab4[i] >= 0 ? L.inv_deg[L.slab4[i]] : 0.f;
            std::memcpy(&slab[i].y, &v, 4);
        }
    }
    if (wl.empty() && L.on_device) {
        int64_t nwl = 0;
        for (const PartHost &p : L.parts) nwl += p.nwl_total;
        int64_t nrows = 0;
        for (const PartHost &p : L.parts) nrows += p.nvirt;
        nrows += (int64_t)L.zero_rows.size();
        wl.resize((size_t)nwl);
        rows.resize((size_t)nrows);
        slab.resize((size_t)L.padded_slots);
        CK(cudaMemcpy(wl.data(), L.d_wl, nwl * sizeof(Workload), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(rows.data(), L.d_rows, nrows * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        if (L.padded_slots && !L.pattern)
            CK(cudaMemcpy(slab.data(), L.d_slab, L.padded_slots * sizeof(uint2), cudaMemcpyDeviceToHost));
        if (L.padded_slots && L.pattern) {
            std::vector<uint32_t> s4((size_t)L.padded_slots);
            CK(cudaMemcpy(s4.data(), L.d_slab4, L.padded_slots * sizeof(uint32_t), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < s4.size(); ++i) {
                slab[i].x = s4[i];
                float v = (int32_t)s4[i] >= 0 ? L.inv_deg[s4[i]] : 0.f;
                std::memcpy(&slab[i].y, &v, 4);
            }
        }
    }
    int64_t k = 0;
    for (const Workload &d : wl) {
        const int64_t hp = d.major == 0 ? d.h : (d.h + 31) / 32 * 32;
        for (int64_t i = 0; i < d.h; ++i) {
            uint32_t rid = rows[(size_t)d.rows + i];
            uint32_t r = (rid & kRowSplit) ? (L.split[(size_t)L.slot_owner[rid & 0x7fffffffu]].row & kRowIdMask)
                                           : (rid & kRowIdMask);
            for (int64_t e = 0; e < d.w; ++e) {
                int64_t slot = d.major == 0 ? d.slab + i * d.w + e
                                            : d.slab + (i / 32) * 32 * d.w + e * 32 + (i % 32);
                uint2 v = slab[(size_t)slot];
                if ((int32_t)v.x < 0) continue;
                if (k >= L.nnz) return fail(SPG_ERR_INVALID, "more stored entries than nnz");
                if (orows) orows[k] = L.inv[r];
                if (ocols) ocols[k] = L.inv[v.x];
                if (ovals) std::memcpy(&ovals[k], &v.y, 4);
                ++k;
            }
        }
        (void)hp;
    }
    if (k != L.nnz) return fail(SPG_ERR_INVALID, "stored entries != nnz");
    return SPG_OK;
}

// ---------------------------------------------------------------- drivers --

// Launch views of the forward layout.  Staged: parts at least 1024 columns
// wide get the persistent kernel with min(stage_cols, width) columns of x in
// shared memory, one block per SM; the rest (and every part when staging is
// off) get 8-warp blocks, one warp per workload.  Block reduction slots are
// laid out part after part; split rows reduce after all blocks.
// Launch view of part p of layout L (everything but the reduction base).
// `staged` selects the handle's persistent kernel option; `sched` is the
// part's pair of work counters (nullptr when the kernel takes none).
static PartView part_view(spg_handle h, const Layout &L, size_t p, bool staged, uint32_t *sched)
{
    const PartHost &ph = L.parts[p];
    PartView pv;
    std::memset(&pv, 0, sizeof pv);
    pv.wl = L.d_wl + ph.wl_off;
    pv.rows = L.d_rows;
    pv.slab = L.d_slab;
    pv.slab4 = L.d_slab4;
    pv.sched = sched;
    pv.nwl = (int32_t)ph.nwl_total;
    pv.c0 = (int32_t)ph.c0;
    pv.pf_ahead = h->pf_ahead;
    pv.status = h->d_status;
    const int64_t width = ph.c1 - ph.c0;
    // option 1 stages the slice only where it serves a useful share of the
    // part's gathers; elsewhere (a sparse remainder of low-degree columns,
    // a banded or stencil matrix) the slice-free persistent kernel runs
    const bool slice_pays = ph.slice_share >= kSliceMinShare;
    if (staged && (h->kernel == 4 || (h->kernel == 1 && !slice_pays)) && ph.nwl_total > 0) {
        // persistent 8-warp blocks, several per SM, no x slice
        pv.persist = 1;
        pv.xs_cols = 0;
        pv.nblocks = (int32_t)std::min<int64_t>((int64_t)h->num_sms * h->persist_blocks,
                                                (ph.nwl_total + kWarpsPerBlock - 1) / kWarpsPerBlock);
    } else if (staged && h->kernel == 3 && !L.pattern && ph.nwl_total > 0) {
        // TMA-pipelined persistent kernel (x slice when the part is wide enough)
        pv.tma = 1;
        pv.xs_cols = width >= 1024 ? (int32_t)std::min<int64_t>(kTmaMaxCols, width) : 0;
        pv.nblocks = (int32_t)std::min<int64_t>(h->num_sms, (ph.nwl_total + 31) / 32);
    } else if (staged && width >= 1024 && ph.nwl_total > 0) {
        pv.xs_cols = (int32_t)std::min<int64_t>(h->stage_cols, width);
        pv.nblocks = (int32_t)std::min<int64_t>(h->num_sms, (ph.nwl_total + 31) / 32);
    } else {
        pv.xs_cols = 0;
        pv.nblocks = (int32_t)((ph.nwl_total + kWarpsPerBlock - 1) / kWarpsPerBlock);
    }
    pv.units = L.d_units + ph.unit_off;
    pv.nunits = (int32_t)ph.nunits;
    return pv;
}

// Whether the handle's persistent kernel option applies (it needs work
// counters; option 2 is the plain one-warp-per-workload kernel).
static bool staged_option(spg_handle h, bool want, bool have_sched)
{
    return want && (h->stage_cols > 0 || h->kernel >= 3) && h->kernel != 2 && have_sched;
}

// Launch views of the forward layout.  Staged: the handle's persistent
// kernel option (default: persistent 8-warp blocks; option 1: parts at least
// 1024 columns wide get one block per SM with min(stage_cols, width) columns
// of x in shared memory); the rest (and every part when staging is off) get
// 8-warp blocks, one warp per workload.  Block reduction slots are laid out
// part after part; split rows reduce after all blocks.
static spg_format_t::Views &get_views_L(spg_handle h, const Layout &L,
                                        spg_format_t::LayoutRT &rt, bool staged)
{
    staged = staged_option(h, staged, rt.sched.p != nullptr);
    spg_format_t::Views &V = staged ? rt.vstaged : rt.vplain;
    if (V.built) return V;
    int32_t base = 0;
    V.v.clear();
    for (size_t p = 0; p < L.parts.size(); ++p) {
        PartView pv = part_view(h, L, p, staged, rt.sched.p ? rt.sched.p + 2 * p : nullptr);
        pv.red_base = base;
        base += pv.nblocks;
        V.v.push_back(pv);
    }
    V.nblk = base;
    V.built = true;
    return V;
}

static spg_format_t::Views &get_views(spg_handle h, bool staged)
{
    return get_views_L(h, h->fwd, h->rt_fwd, staged);
}

static SplitView split_of_L(const Layout &L, const spg_format_t::Views &V)
{
    SplitView sv = L.split_view();
    sv.red_split_base = V.nblk;
    return sv;
}

static SplitView split_of(spg_handle h, const spg_format_t::Views &V) { return split_of_L(h->fwd, V); }

static int nred_of_L(const Layout &L, const spg_format_t::Views &V) { return V.nblk + (int)L.nsplit; }
static int nred_of(spg_handle h, const spg_format_t::Views &V) { return nred_of_L(h->fwd, V); }
static spg_status ensure_vectors(spg_handle h, int64_t N)
{
    CK(h->x.ensure((size_t)N));
    CK(h->y.ensure((size_t)N));
    const int nr = std::max(nred_of(h, get_views(h, true)), nred_of(h, get_views(h, false)));
    CK(h->red.ensure((size_t)std::max(1, nr)));
    return SPG_OK;
}

// Device alias of mapped (pinned) host memory -- kernels read and write it
// straight over the host link -- or nullptr (device or pageable memory).
static void *mapped_host(const void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Input vector on the device: the caller's pointer or a staged copy.
static spg_status device_in(spg_handle h, const float *p, int64_t count, const float **out,
                            cudaStream_t s)
{
    if (!p || is_device_ptr(p)) { *out = p; return SPG_OK; }
    CK(h->stage_in.ensure((size_t)count));
    CK(cudaMemcpyAsync(h->stage_in.p, p, count * sizeof(float), cudaMemcpyHostToDevice, s));
    *out = h->stage_in.p;
    return SPG_OK;
}

// A caller's vector of n floats (original order; device, mapped host or
// pageable host memory) into position order: dst[pi(j)] = src[j], times
// d[pi(j)] when d is given.  Device memory is gathered by position; mapped
// host memory is read once, in order, over the host link (no staging
// copy); pageable memory is staged, then gathered.
static spg_status permute_in(spg_handle h, const Layout &L, const float *src, int64_t n,
                             const float *d, float *dst, cudaStream_t s)
{
    if (const float *a = is_device_ptr(src) ? nullptr : (const float *)mapped_host(src)) {
        launch_permute_in(n, L.d_perm, a, d, dst, s);
        return SPG_OK;
    }
    const float *sd;
    spg_status st = device_in(h, src, n, &sd, s);
    if (st != SPG_OK) return st;
    if (d) launch_gather_scaled(n, L.d_inv, sd, d, dst, s);
    else launch_gather(n, L.d_inv, sd, dst, s);
    return SPG_OK;
}

// Where an output kernel writes a caller's vector of n floats: its device
// memory, the device alias of its mapped host memory (written in order
// over the host link, no staging copy), or the staging buffer for pageable
// memory (*staged set: copy it out after the kernel; keep_old: the kernel
// reads the old values too, copy them in first).
static spg_status out_target(spg_handle h, float *p, int64_t n, bool keep_old, float **od, bool *staged,
                             cudaStream_t s)
{
    *staged = false;
    if (is_device_ptr(p)) { *od = p; return SPG_OK; }
    if (float *a = (float *)mapped_host(p)) { *od = a; return SPG_OK; }
    CK(h->stage_out.ensure((size_t)n));
    *od = h->stage_out.p;
    *staged = true;
    if (keep_old) CK(cudaMemcpyAsync(*od, p, n * sizeof(float), cudaMemcpyHostToDevice, s));
    return SPG_OK;
}


static void launch_parts(spg_handle h, int mode, const float *x, float *y, const IterState *st,
                         double2 *red, cudaStream_t s)
{
    if (h->fwd.pattern) mode = mode == EPI_RAW ? EPI_RAW_PAT : (mode == EPI_PAGERANK ? EPI_PR_PAT : mode);
    const spg_format_t::Views &V = get_views(h, true);
    const SplitView sv = split_of(h, V);
    for (const PartView &pv : V.v) launch_part(mode, pv, sv, x, y, st, red, s);
}

// One power iteration: the parts' kernels, then the convergence check --
// fused into the last part's kernel (its last block) when that kernel
// supports it, else the one-block check kernel.  check_mode is the form of
// the check (PageRank form for PageRank, RWR and the adjoint; HITS form).
static void launch_iteration(spg_handle h, const Layout &L, spg_format_t::LayoutRT &rt, int mode,
                             int check_mode, int nred, unsigned long long cond, int uc, cudaStream_t cs)
{
    const spg_format_t::Views &V = get_views_L(h, L, rt, true);
    const SplitView sv = split_of_L(L, V);
    if (L.pattern) mode = mode == EPI_RAW ? EPI_RAW_PAT : (mode == EPI_PAGERANK ? EPI_PR_PAT : mode);
    int last = -1;
    for (size_t p = 0; p < V.v.size(); ++p)
        if (V.v[p].nblocks > 0) last = (int)p;
    bool fused = false;
    for (size_t p = 0; p < V.v.size(); ++p) {
        FuseCheck fc;
        if ((int)p == last && !h->separate_check && nred > 0) {
            fc.cond = cond;
            fc.use_cond = uc;
            fc.nred = nred;
            fc.st = h->d_state;
            fc.done = rt.sched.p + 2 * L.parts.size();
        }
        const bool f = launch_part(mode, V.v[p], sv, nullptr, nullptr, h->d_state, h->red.p, cs, fc);
        if ((int)p == last) fused = f;
    }
    if (!fused) launch_check(check_mode, h->d_state, h->red.p, nred, cond, uc, cs);
}

extern "C" spg_status spg_spmv_permuted(spg_handle h, const float *xp, float *yp, void *stream)
{
    if (!h || h->host_only) return fail(SPG_ERR_INVALID, "no device format");
    if (!xp || !yp || xp == yp) return fail(SPG_ERR_INVALID, "x and y must be distinct device vectors");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->fwd.pattern) {           // slots hold no values: fold them into x first
        CK(h->x.ensure((size_t)h->fwd.n));
        launch_scale(h->fwd.n, xp, h->fwd.d_inv_deg, h->x.p, s);
        xp = h->x.p;
    }
    launch_parts(h, EPI_RAW, xp, yp, nullptr, nullptr, s);
    CK(cudaGetLastError());
    return SPG_OK;
}

extern "C" spg_status spg_spmv_tile_coo(spg_handle h, const float *xp, float *yp, void *stream)
{
    if (!h || h->host_only) return fail(SPG_ERR_INVALID, "no device format");
    if (!xp || !yp || xp == yp) return fail(SPG_ERR_INVALID, "x and y must be distinct device vectors");
    const Layout &L = h->fwd;
    if (L.coo_off.size() < 2 || !L.d_coo_row) return fail(SPG_ERR_INVALID, "build the handle with tile_coo");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(yp, 0, (size_t)L.n * sizeof(float), s));
    for (size_t p = 0; p + 1 < L.coo_off.size(); ++p)
        launch_tile_coo(L.d_coo_row, L.d_coo_col, L.d_coo_val, L.coo_off[p], L.coo_off[p + 1], xp, yp,
                        h->num_sms, s);
    CK(cudaGetLastError());
    return SPG_OK;
}

extern "C" spg_status spg_spmv(spg_handle h, const float *x, float *y, float alpha, float beta,
                               void *stream)
{
    if (!h || h->host_only) return fail(SPG_ERR_INVALID, "no device format");
    if (!x || !y) return fail(SPG_ERR_INVALID, "null vector");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->fwd.n;
    spg_status st = ensure_vectors(h, N);
    if (st != SPG_OK) return st;
    if ((st = permute_in(h, h->fwd, x, N, h->fwd.pattern ? h->fwd.d_inv_deg : nullptr, h->x.p, s)) != SPG_OK)
        return st;
    float *yd;
    bool staged;
    if ((st = out_target(h, y, N, beta != 0.f, &yd, &staged, s)) != SPG_OK) return st;
    launch_parts(h, EPI_RAW, h->x.p, h->y.p, nullptr, nullptr, s);
    launch_unpermute_axpby(N, h->fwd.d_perm, h->y.p, yd, alpha, beta, s);
    CK(cudaGetLastError());
    if (staged) CK(cudaMemcpyAsync(y, yd, N * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (!is_device_ptr(y)) CK(cudaStreamSynchronize(s));
    return SPG_OK;
}

extern "C" spg_status spg_spmm(spg_handle h, const float *X, int64_t ldx, float *Y, int64_t ldy,
                               int k, float alpha, float beta, void *stream)
{
    if (!h || h->host_only) return fail(SPG_ERR_INVALID, "no device format");
    if (!X || !Y || k < 1 || k > 1024 || ldx < k || ldy < k) return fail(SPG_ERR_INVALID, "bad SpMM arguments");
    if (!is_device_ptr(X) || !is_device_ptr(Y)) return fail(SPG_ERR_INVALID, "spmm takes device pointers");
    if (h->fwd.pattern) return fail(SPG_ERR_UNSUPPORTED, "spmm needs stored values (build without pattern_only)");
    cudaStream_t s = (cudaStream_t)stream;
    const Layout &L = h->fwd;
    const int64_t N = L.n;
    CK(h->X.ensure((size_t)(N * k)));
    CK(h->Y.ensure((size_t)(N * k)));
    CK(h->partial_k.ensure((size_t)std::max<int64_t>(1, L.nchunk_slots) * k));
    launch_gather_rows(N, k, L.d_inv, X, ldx, h->X.p, s);
    const spg_format_t::Views &V = get_views(h, false);
    SplitView sv = split_of(h, V);
    sv.partial = h->partial_k.p;
    for (const PartView &pv : V.v)
        launch_part_spmm(EPI_RAW, pv, sv, h->X.p, h->Y.p, k, nullptr, nullptr, nullptr, nullptr, s);
    launch_scatter_rows(N, k, L.d_inv, h->Y.p, Y, ldy, alpha, beta, s);
    CK(cudaGetLastError());
    return SPG_OK;
}

// Build (once) a graph whose body is `body(stream, cond)` inside a WHILE
// node; the body's check kernel clears the condition when done.
template <class Body>
static spg_status get_loop_graph(spg_handle h, const std::string &key, Body body, LoopGraph **out)
{
    if (h->loop_mode == 1) {             // host loop: no graph, the body is launched per iteration
        h->host_loop = LoopGraph();
        h->host_loop.body = body;
        *out = &h->host_loop;
        return SPG_OK;
    }
    if (h->graphs_epoch != h->epoch) {   // a workspace buffer moved: recapture
        h->drop_graphs();
        h->graphs_epoch = h->epoch;
    }
    auto it = h->graphs.find(key);
    if (it != h->graphs.end()) { *out = &it->second; return SPG_OK; }
    LoopGraph g;
    CK(cudaGraphCreate(&g.graph, 0));
    cudaGraphConditionalHandle ch;
    CK(cudaGraphConditionalHandleCreate(&ch, g.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = ch;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &np));
    cudaGraph_t bodyg = np.conditional.phGraph_out[0];
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const int64_t before = launch_count();
    cudaError_t e = cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        body(cs, (unsigned long long)ch, 1);
        cudaGraph_t captured = bodyg;
        e = cudaStreamEndCapture(cs, &captured);
    }
    g.kernels_per_iter = (int)(launch_count() - before);
    count_launches(-(launch_count() - before));
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) { cudaGraphDestroy(g.graph); return cuda_fail(e, "capture loop body"); }
    e = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g.graph); return cuda_fail(e, "instantiate loop graph"); }
    auto res = h->graphs.emplace(key, g);
    *out = &res.first->second;
    return SPG_OK;
}

static IterState make_state(spg_handle h, double c, double tol, int max_iter, int64_t N,
                            float *b0, float *b1)
{
    IterState st;
    std::memset(&st, 0, sizeof st);
    st.c = c;
    st.tol = tol;
    st.delta = 0.0;
    st.l1 = INFINITY;
    st.scale[0] = st.scale[1] = 1.0;
    st.inv_n = 1.0 / (double)N;
    st.iter = 0;
    st.max_iter = max_iter;
    st.parity = 0;
    st.done = 0;
    st.seed = -1;
    st.hits_norm = 2;
    st.n = N;
    st.dangling_start = h->fwd.dangling_start;
    st.buf[0] = b0;
    st.buf[1] = b1;
    return st;
}

// Run the loop graph `g` (max_iter > 0) and read back the state.
// Read and clear the kernels' status word (after the stream has synchronised).
static spg_status take_status(spg_handle h)
{
    if (!h->d_status) return SPG_OK;
    uint32_t st = 0;
    CK(cudaMemcpy(&st, h->d_status, sizeof st, cudaMemcpyDeviceToHost));
    if (st == 0) return SPG_OK;
    CK(cudaMemset(h->d_status, 0, sizeof st));
    return fail(SPG_ERR_TIMEOUT, "a bounded wait on a TMA copy ran out in the SpMV kernel");
}

// Upload the iteration state through the handle's pinned copy (an
// asynchronous copy from pageable memory would stage synchronously).  The
// pinned copy is next written by the loop's read-back, later in stream order.
static spg_status upload_state(spg_handle h, const IterState &hs, cudaStream_t s)
{
    *h->hs_pinned = hs;
    CK(cudaMemcpyAsync(h->d_state, h->hs_pinned, sizeof(IterState), cudaMemcpyHostToDevice, s));
    return SPG_OK;
}

// Enqueue the loop `g` (max_iter > 0) and the read-back of the final state
// and the status word into pinned host memory; no synchronisation, so the
// caller can queue its output passes behind it and synchronise once.
static spg_status launch_loop(spg_handle h, LoopGraph *g, int max_iter, cudaStream_t s)
{
    if (max_iter > 0) {
        CK(cudaEventRecord(h->ev0, s));
        if (g->exec) {
            CK(cudaGraphLaunch(g->exec, s));
        } else {
            // host loop (the paper's structure): poll the done flag every 16 iterations
            for (int it = 0; it < max_iter; ++it) {
                g->body(s, 0ull, 0);
                if ((it + 1) % 16 == 0 && it + 1 < max_iter) {
                    int32_t done = 0;
                    CK(cudaMemcpyAsync(&done, &h->d_state->done, sizeof done, cudaMemcpyDeviceToHost, s));
                    CK(cudaStreamSynchronize(s));
                    if (done) break;
                }
            }
        }
        CK(cudaEventRecord(h->ev1, s));
    }
    CK(cudaMemcpyAsync(h->hs_pinned, h->d_state, sizeof(IterState), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->status_pinned, h->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    return SPG_OK;
}

// After the stream has synchronised: the final state, the status word, the
// launch count and the info record of a launch_loop.
static spg_status finish_loop(spg_handle h, LoopGraph *g, int max_iter, IterState *hs,
                              spg_iter_info *info)
{
    *hs = *h->hs_pinned;
    if (*h->status_pinned) {
        *h->status_pinned = 0u;
        CK(cudaMemset(h->d_status, 0, sizeof(uint32_t)));
        return fail(SPG_ERR_TIMEOUT, "a bounded wait on a TMA copy ran out in the SpMV kernel");
    }
    count_launches((int64_t)hs->iter * g->kernels_per_iter);
    if (info) {
        info->iters = hs->iter;
        info->last_l1 = hs->l1;
        info->dangling = hs->delta;
        float ms = 0.f;
        if (max_iter > 0) cudaEventElapsedTime(&ms, h->ev0, h->ev1);
        info->ms = ms;
    }
    return SPG_OK;
}

static spg_status run_loop(spg_handle h, LoopGraph *g, int max_iter, IterState *hs,
                           spg_iter_info *info, cudaStream_t s)
{
    spg_status st = launch_loop(h, g, max_iter, s);
    if (st != SPG_OK) return st;
    CK(cudaStreamSynchronize(s));
    return finish_loop(h, g, max_iter, hs, info);
}

extern "C" spg_status spg_pagerank(spg_handle h, float damping, double tol, int max_iter,
                                   const float *p0, float *p_out, spg_iter_info *info,
                                   void *stream)
{
    if (!h || h->host_only) return fail(SPG_ERR_INVALID, "no device format");
    if (h->kind != SPG_KIND_PAGERANK) return fail(SPG_ERR_UNSUPPORTED, "pagerank needs a PAGERANK handle");
    if (!p_out || !(damping >= 0.f && damping < 1.f) || max_iter < 0)
        return fail(SPG_ERR_INVALID, "bad pagerank arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->fwd.n;
    spg_status st = ensure_vectors(h, N);
    if (st != SPG_OK) return st;
    const bool pat = h->fwd.pattern;
    if (pat) { CK(h->z0.ensure((size_t)N)); CK(h->z1.ensure((size_t)N)); }
    IterState hs = make_state(h, damping, tol, max_iter, N, h->x.p, h->y.p);
    if (pat) {
        hs.zbuf[0] = h->z0.p;
        hs.zbuf[1] = h->z1.p;
        hs.inv_deg = h->fwd.d_inv_deg;
    }
    if ((st = upload_state(h, hs, s)) != SPG_OK) return st;
    if (p0) {
        if ((st = permute_in(h, h->fwd, p0, N, nullptr, h->x.p, s)) != SPG_OK) return st;
    } else {
        launch_fill(N, (float)(1.0 / (double)N), h->x.p, s);
    }
    if (pat) launch_scale(N, h->x.p, h->fwd.d_inv_deg, h->z0.p, s);
    CK(h->init_part.ensure((size_t)init_delta_scratch()));
    launch_init_delta(h->d_state, h->init_part.p, s);
    LoopGraph *g;
    const int nred = nred_of(h, get_views(h, true));
    st = get_loop_graph(h, pat ? "pagerank_pattern" : "pagerank", [&](cudaStream_t cs, unsigned long long cond, int uc) {
        launch_iteration(h, h->fwd, h->rt_fwd, EPI_PAGERANK, EPI_PAGERANK, nred, cond, uc, cs);
    }, &g);
    if (st != SPG_OK) return st;
    CK(cudaGetLastError());
    if ((st = launch_loop(h, g, max_iter, s)) != SPG_OK) return st;
    float *od;
    bool staged;
    if ((st = out_target(h, p_out, N, false, &od, &staged, s)) != SPG_OK) return st;
    launch_unpermute_state(N, h->fwd.d_perm, h->d_state, od, nullptr, 0, s);
    if (staged) CK(cudaMemcpyAsync(p_out, od, N * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if ((st = finish_loop(h, g, max_iter, &hs, info)) != SPG_OK) return st;
    return (tol > 0 && !(hs.l1 < tol)) ? SPG_NOT_CONVERGED : SPG_OK;
}

extern "C" spg_status spg_hits(spg_handle h, int norm, double tol, int max_iter, float *auth,
                               float *hub, spg_iter_info *info, void *stream)
{
    if (!h || h->host_only) return fail(SPG_ERR_INVALID, "no device format");
    if (h->kind != SPG_KIND_HITS) return fail(SPG_ERR_UNSUPPORTED, "hits needs a HITS handle");
    if (!auth || !hub || (norm != 1 && norm != 2) || max_iter < 0 || tol > 0)
        return fail(SPG_ERR_INVALID, "bad hits arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->fwd.n, n = h->n_graph;
    spg_status st = ensure_vectors(h, N);
    if (st != SPG_OK) return st;
    IterState hs = make_state(h, 1.0, 0.0, max_iter, N, h->x.p, h->y.p);
    hs.hits_norm = norm;
    CK(cudaMemcpyAsync(h->d_state, &hs, sizeof hs, cudaMemcpyHostToDevice, s));
    launch_fill(N, (float)(1.0 / (double)n), h->x.p, s);
    LoopGraph *g;
    const int nred = nred_of(h, get_views(h, true));
    st = get_loop_graph(h, "hits", [&](cudaStream_t cs, unsigned long long cond, int uc) {
        launch_iteration(h, h->fwd, h->rt_fwd, EPI_HITS, EPI_HITS, nred, cond, uc, cs);
    }, &g);
    if (st != SPG_OK) return st;
    CK(cudaGetLastError());
    if ((st = run_loop(h, g, max_iter, &hs, info, s)) != SPG_OK) return st;
    // normalised iterate into [auth; hub] (original order)
    CK(h->stage_out.ensure((size_t)N));
    launch_unpermute_state(N, h->fwd.d_perm, h->d_state, h->stage_out.p, h->d_row_half, 1, s);
    const cudaMemcpyKind ka = is_device_ptr(auth) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const cudaMemcpyKind kh = is_device_ptr(hub) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(auth, h->stage_out.p, n * sizeof(float), ka, s));
    CK(cudaMemcpyAsync(hub, h->stage_out.p + n, n * sizeof(float), kh, s));
    CK(cudaStreamSynchronize(s));
    return SPG_OK;
}

extern "C" spg_status spg_rwr(spg_handle h, float restart, const int32_t *seeds, int k,
                              double tol, int max_iter, float *R, spg_iter_info *info,
                              void *stream)
{
    if (!h || h->host_only) return fail(SPG_ERR_INVALID, "no device format");
    if (h->kind != SPG_KIND_PAGERANK && !(h->kind == SPG_KIND_WEIGHTED && k == 1))
        return fail(SPG_ERR_UNSUPPORTED, "rwr needs a PAGERANK handle (or WEIGHTED with k = 1)");
    if (h->fwd.pattern) return fail(SPG_ERR_UNSUPPORTED, "rwr needs stored values (build without pattern_only)");
    if (!seeds || !R || k < 1 || k > 64 || !(restart > 0.f && restart <= 1.f) || max_iter < 0)
        return fail(SPG_ERR_INVALID, "bad rwr arguments (1 <= k <= 64)");
    cudaStream_t s = (cudaStream_t)stream;
    const Layout &L = h->fwd;
    const int64_t N = L.n;
    std::vector<int32_t> ps((size_t)k);
    for (int j = 0; j < k; ++j) {
        if (seeds[j] < 0 || seeds[j] >= N) return fail(SPG_ERR_INVALID, "seed out of range");
        ps[(size_t)j] = L.perm[(size_t)seeds[j]];
    }
    const double c = 1.0 - (double)restart;
    IterState hs;
    spg_status st;
    LoopGraph *g;
    const int nred = nred_of(h, get_views(h, true));
    if (k == 1) {
        if ((st = ensure_vectors(h, N)) != SPG_OK) return st;
        hs = make_state(h, c, tol, max_iter, N, h->x.p, h->y.p);
        hs.seed = ps[0];
        CK(cudaMemcpyAsync(h->d_state, &hs, sizeof hs, cudaMemcpyHostToDevice, s));
        CK(h->seeds.ensure(1));
        CK(cudaMemcpyAsync(h->seeds.p, ps.data(), sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(h->x.p, 0, N * sizeof(float), s));
        launch_set_one(h->x.p, h->seeds.p, 1, s);
        CK(h->init_part.ensure((size_t)init_delta_scratch()));
        launch_init_delta(h->d_state, h->init_part.p, s);
        st = get_loop_graph(h, "rwr1", [&](cudaStream_t cs, unsigned long long cond, int uc) {
            launch_iteration(h, h->fwd, h->rt_fwd, EPI_RWR, EPI_RWR, nred, cond, uc, cs);
        }, &g);
        if (st != SPG_OK) return st;
        CK(cudaGetLastError());
        if ((st = run_loop(h, g, max_iter, &hs, info, s)) != SPG_OK) return st;
        float *od;
        bool staged;
        if ((st = out_target(h, R, N, false, &od, &staged, s)) != SPG_OK) return st;
        launch_unpermute_state(N, L.d_perm, h->d_state, od, nullptr, 0, s);
        if (staged) CK(cudaMemcpyAsync(R, od, N * sizeof(float), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return (tol > 0 && !(hs.l1 < tol)) ? SPG_NOT_CONVERGED : SPG_OK;
    }
    // k restart vectors as one SpMM per iteration
    CK(h->X.ensure((size_t)(N * k)));
    CK(h->Y.ensure((size_t)(N * k)));
    CK(h->partial_k.ensure((size_t)std::max<int64_t>(1, L.nchunk_slots) * k));
    const spg_format_t::Views &VK = get_views(h, false);
    const int nredk = nred_of(h, VK);
    CK(h->redk.ensure((size_t)std::max(1, nredk) * 2 * k));
    CK(h->delta_k.ensure((size_t)k));
    CK(h->l1_k.ensure((size_t)k));
    CK(h->seeds.ensure((size_t)k));
    hs = make_state(h, c, tol, max_iter, N, h->X.p, h->Y.p);
    CK(cudaMemcpyAsync(h->d_state, &hs, sizeof hs, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->seeds.p, ps.data(), k * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    launch_onehot_rows(N, k, h->seeds.p, h->X.p, s);
    CK(h->colsum.ensure((size_t)colsum_scratch()));
    launch_init_delta_k(hs.dangling_start, hs.n, h->X.p, k, h->delta_k.p, h->colsum.p, s);
    SplitView sv = split_of(h, VK);
    sv.partial = h->partial_k.p;
    const std::string key = "rwrk" + std::to_string(k);
    st = get_loop_graph(h, key, [&](cudaStream_t cs, unsigned long long cond, int uc) {
        for (const PartView &pv : VK.v)
            launch_part_spmm(EPI_RWR, pv, sv, nullptr, nullptr, k, h->d_state, h->seeds.p,
                             h->delta_k.p, h->redk.p, cs);
        launch_check_k(h->d_state, h->redk.p, nredk, k, h->delta_k.p, h->l1_k.p, h->colsum.p, cond,
                       uc, cs);
    }, &g);
    if (st != SPG_OK) return st;
    CK(cudaGetLastError());
    if ((st = run_loop(h, g, max_iter, &hs, info, s)) != SPG_OK) return st;
    float *cur = hs.buf[hs.parity];
    float *od;
    bool staged;
    if ((st = out_target(h, R, N * k, false, &od, &staged, s)) != SPG_OK) return st;
    launch_unpermute_rows(N, k, L.d_perm, cur, od, k, 1.f, 0.f, s);
    if (staged) CK(cudaMemcpyAsync(R, od, N * k * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return (tol > 0 && !(hs.l1 < tol)) ? SPG_NOT_CONVERGED : SPG_OK;
}

// ---------------------------------------------------- row partition --

extern "C" spg_status spg_partition_rows(int64_t n, const int64_t *row_len, int P, int32_t *part)
{
    if (n < 0 || (n > 0 && (!row_len || !part)) || P < 1 || P > 64)
        return fail(SPG_ERR_INVALID, "partition_rows needs n >= 0, row_len, part and 1 <= P <= 64");
    // rows by decreasing length, ties ascending id (counting sort)
    int64_t maxlen = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (row_len[v] < 0) return fail(SPG_ERR_INVALID, "negative row length");
        maxlen = std::max(maxlen, row_len[v]);
    }
    std::vector<int64_t> start((size_t)maxlen + 2, 0);
    for (int64_t v = 0; v < n; ++v) start[(size_t)row_len[v]]++;
    int64_t run = 0;
    for (int64_t l = maxlen; l >= 0; --l) { const int64_t c = start[(size_t)l]; start[(size_t)l] = run; run += c; }
    // the k-th row of the order goes to round k / P, position k % P; odd
    // rounds deal from the last part back to the first
    for (int64_t v = 0; v < n; ++v) {
        const int64_t k = start[(size_t)row_len[v]]++;
        const int64_t round = k / P, pos = k % P;
        part[v] = (int32_t)((round & 1) ? P - 1 - pos : pos);
    }
    return SPG_OK;
}

extern "C" spg_status spg_pagerank_ranks(const spg_handle *ranks, int P, float damping, double tol,
                                         int max_iter, const float *p0, float *p_out,
                                         spg_iter_info *info, void *stream)
{
    if (!ranks || P < 1 || P > 8) return fail(SPG_ERR_INVALID, "pagerank_ranks needs 1 <= P <= 8 handles");
    if (!p_out || !(damping >= 0.f && damping < 1.f) || max_iter < 0)
        return fail(SPG_ERR_INVALID, "bad pagerank arguments");
    spg_handle h0 = ranks[0];
    for (int r = 0; r < P; ++r) {
        spg_handle h = ranks[r];
        if (!h || h->host_only || h->kind != SPG_KIND_PAGERANK)
            return fail(SPG_ERR_INVALID, "every rank needs a device PAGERANK handle");
        if (h->nparts != P || h->part_id != r || !h->d_owner)
            return fail(SPG_ERR_INVALID, "rank r must be built with row_part, nparts = P, part_id = r");
        if (h->fwd.n != h0->fwd.n || h->fwd.perm != h0->fwd.perm || h->fwd.pattern != h0->fwd.pattern)
            return fail(SPG_ERR_INVALID, "ranks must come from one graph (same order and storage)");
        if (h->device != h0->device) return fail(SPG_ERR_INVALID, "ranks must share one device");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h0->fwd.n;
    const bool pat = h0->fwd.pattern;
    // per rank: its own iterates, state and range of block partials
    std::vector<int> off((size_t)P + 1, 0);
    for (int r = 0; r < P; ++r) {
        spg_handle h = ranks[r];
        spg_status st = ensure_vectors(h, N);
        if (st != SPG_OK) return st;
        if (pat) { CK(h->z0.ensure((size_t)N)); CK(h->z1.ensure((size_t)N)); }
        off[(size_t)r + 1] = off[(size_t)r] + nred_of(h, get_views(h, true));
    }
    CK(h0->red_ranks.ensure((size_t)std::max(1, off[(size_t)P])));
    CK(h0->rank_states.ensure((size_t)P));
    std::vector<IterState *> sp((size_t)P);
    IterState hs{};
    for (int r = 0; r < P; ++r) {
        spg_handle h = ranks[r];
        IterState st = make_state(h, damping, tol, max_iter, N, h->x.p, h->y.p);
        if (pat) { st.zbuf[0] = h->z0.p; st.zbuf[1] = h->z1.p; st.inv_deg = h->fwd.d_inv_deg; }
        CK(cudaMemcpyAsync(h->d_state, &st, sizeof st, cudaMemcpyHostToDevice, s));
        sp[(size_t)r] = h->d_state;
        if (r == 0) hs = st;
    }
    CK(cudaMemcpyAsync(h0->rank_states.p, sp.data(), P * sizeof(IterState *), cudaMemcpyHostToDevice, s));
    const float *pd = nullptr;
    if (p0) {
        spg_status st = device_in(h0, p0, N, &pd, s);
        if (st != SPG_OK) return st;
    }
    for (int r = 0; r < P; ++r) {
        spg_handle h = ranks[r];
        if (pd) launch_gather(N, h->fwd.d_inv, pd, h->x.p, s);
        else launch_fill(N, (float)(1.0 / (double)N), h->x.p, s);
        if (pat) launch_scale(N, h->x.p, h->fwd.d_inv_deg, h->z0.p, s);
        CK(h->init_part.ensure((size_t)init_delta_scratch()));
        launch_init_delta(h->d_state, h->init_part.p, s);
    }
    const int nred = off[(size_t)P];
    LoopGraph lg;   // host-driven iterations: the body is launched once per iteration
    lg.body = [&](cudaStream_t cs, unsigned long long, int) {
        for (int r = 0; r < P; ++r)
            launch_parts(ranks[r], EPI_PAGERANK, nullptr, nullptr, ranks[r]->d_state,
                         h0->red_ranks.p + off[(size_t)r], cs);
        launch_allgather_rows(N, h0->d_owner, h0->rank_states.p, P, pat, cs);
        launch_check_ranks(h0->rank_states.p, P, h0->red_ranks.p, nred, cs);
    };
    CK(cudaGetLastError());
    spg_status st = run_loop(h0, &lg, max_iter, &hs, info, s);
    if (st != SPG_OK) return st;
    float *od;
    bool staged;
    if ((st = out_target(h0, p_out, N, false, &od, &staged, s)) != SPG_OK) return st;
    launch_unpermute_state(N, h0->fwd.d_perm, h0->d_state, od, nullptr, 0, s);
    if (staged) CK(cudaMemcpyAsync(p_out, od, N * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return (tol > 0 && !(hs.l1 < tol)) ? SPG_NOT_CONVERGED : SPG_OK;
}

// ----------------------------------------- one rank's step, row slices --

extern "C" spg_status spg_pagerank_rank_step(spg_handle h, float damping, double delta,
                                             const float *x_perm, float *y_perm, double *partial,
                                             void *stream)
{
    if (!h || h->host_only || h->kind != SPG_KIND_PAGERANK)
        return fail(SPG_ERR_INVALID, "rank step needs a device PAGERANK handle");
    if (h->fwd.pattern) return fail(SPG_ERR_UNSUPPORTED, "rank step needs stored values (no pattern_only)");
    if (!x_perm || !y_perm || x_perm == y_perm || !partial || !is_device_ptr(x_perm) || !is_device_ptr(y_perm))
        return fail(SPG_ERR_INVALID, "x' and y' must be distinct device vectors; partial a host array");
    if (!(damping >= 0.f && damping < 1.f) || !(delta >= 0.0))
        return fail(SPG_ERR_INVALID, "bad damping or dangling mass");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->fwd.n;
    spg_status st = ensure_vectors(h, N);
    if (st != SPG_OK) return st;
    // the rank's kernels on a state whose current iterate is the caller's x'
    // and whose next one is the caller's y'; the separate check kernel then
    // sums this rank's block partials in a fixed order
    IterState hs = make_state(h, damping, 0.0, 1, N, const_cast<float *>(x_perm), y_perm);
    hs.delta = delta;
    CK(cudaMemcpyAsync(h->d_state, &hs, sizeof hs, cudaMemcpyHostToDevice, s));
    const spg_format_t::Views &V = get_views(h, true);
    const int nred = nred_of(h, V);
    launch_parts(h, EPI_PAGERANK, nullptr, nullptr, h->d_state, h->red.p, s);
    launch_check(EPI_PAGERANK, h->d_state, h->red.p, nred, 0, 0, s);
    CK(cudaMemcpyAsync(h->hs_pinned, h->d_state, sizeof(IterState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    partial[0] = h->hs_pinned->l1;
    partial[1] = h->hs_pinned->delta;
    return take_status(h);
}

extern "C" spg_status spg_pack_slice(int64_t count, const int32_t *idx, const float *full, float *slice,
                                     void *stream)
{
    if (count < 0) return fail(SPG_ERR_INVALID, "negative count");
    if (count == 0) return SPG_OK;
    if (!idx || !full || !slice || !is_device_ptr(idx) || !is_device_ptr(full) || !is_device_ptr(slice))
        return fail(SPG_ERR_INVALID, "pack_slice takes device pointers");
    launch_gather(count, idx, full, slice, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return SPG_OK;
}

extern "C" spg_status spg_unpack_slice(int64_t count, const int32_t *idx, const float *slice, float *full,
                                       void *stream)
{
    if (count < 0) return fail(SPG_ERR_INVALID, "negative count");
    if (count == 0) return SPG_OK;
    if (!idx || !full || !slice || !is_device_ptr(idx) || !is_device_ptr(full) || !is_device_ptr(slice))
        return fail(SPG_ERR_INVALID, "unpack_slice takes device pointers");
    launch_scatter_axpby(count, idx, slice, full, 1.f, 0.f, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return SPG_OK;
}

// ------------------------------------------------------------ baselines --

extern "C" spg_status spg_baseline_spmv(spg_handle h, spg_baseline which, const float *x, float *y,
                                        float alpha, float beta, void *stream)
{
    if (!h || !h->d_rp) return fail(SPG_ERR_INVALID, "baselines need keep_csr");
    if (!x || !y || !is_device_ptr(x) || !is_device_ptr(y)) return fail(SPG_ERR_INVALID, "device vectors");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = h->n_graph;
    CK(h->y.ensure((size_t)n));
    if (which == SPG_BASELINE_CSR_SCALAR)
        launch_csr_scalar(EPI_RAW, n, h->d_rp, h->d_col, h->d_val, h->d_dangling, x, h->y.p, nullptr, nullptr, nullptr, s);
    else
        launch_csr_vector(EPI_RAW, n, h->d_rp, h->d_col, h->d_val, h->d_dangling, x, h->y.p, nullptr, nullptr, nullptr, s);
    launch_scatter_axpby(n, nullptr, h->y.p, y, alpha, beta, s);
    CK(cudaGetLastError());
    return SPG_OK;
}

extern "C" spg_status spg_baseline_pagerank(spg_handle h, spg_baseline which, float damping,
                                            double tol, int max_iter, float *p_out,
                                            spg_iter_info *info, void *stream)
{
    if (!h || !h->d_rp || h->kind != SPG_KIND_PAGERANK) return fail(SPG_ERR_INVALID, "baselines need a PAGERANK handle with keep_csr");
    if (!p_out || max_iter < 0) return fail(SPG_ERR_INVALID, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = h->n_graph;
    spg_status st = ensure_vectors(h, n);
    if (st != SPG_OK) return st;
    const int nb = which == SPG_BASELINE_CSR_SCALAR ? csr_scalar_blocks(n) : csr_vector_blocks(n);
    CK(h->red.ensure((size_t)nb));
    IterState hs = make_state(h, damping, tol, max_iter, n, h->x.p, h->y.p);
    CK(cudaMemcpyAsync(h->d_state, &hs, sizeof hs, cudaMemcpyHostToDevice, s));
    launch_fill(n, (float)(1.0 / (double)n), h->x.p, s);
    CK(h->init_part.ensure((size_t)init_delta_scratch()));
    launch_init_delta_flags(h->d_state, h->d_dangling, h->init_part.p, s);
    LoopGraph *g;
    const std::string key = which == SPG_BASELINE_CSR_SCALAR ? "pr_csr_scalar" : "pr_csr_vector";
    st = get_loop_graph(h, key, [&](cudaStream_t cs, unsigned long long cond, int uc) {
        if (which == SPG_BASELINE_CSR_SCALAR)
            launch_csr_scalar(EPI_PAGERANK, n, h->d_rp, h->d_col, h->d_val, h->d_dangling, nullptr, nullptr, h->d_state, h->red.p, nullptr, cs);
        else
            launch_csr_vector(EPI_PAGERANK, n, h->d_rp, h->d_col, h->d_val, h->d_dangling, nullptr, nullptr, h->d_state, h->red.p, nullptr, cs);
        launch_check(EPI_PAGERANK, h->d_state, h->red.p, nb, cond, uc, cs);
    }, &g);
    if (st != SPG_OK) return st;
    CK(cudaGetLastError());
    if ((st = run_loop(h, g, max_iter, &hs, info, s)) != SPG_OK) return st;
    float *cur = hs.buf[hs.parity];
    const cudaMemcpyKind kd = is_device_ptr(p_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(p_out, cur, n * sizeof(float), kd, s));
    CK(cudaStreamSynchronize(s));
    return (tol > 0 && !(hs.l1 < tol)) ? SPG_NOT_CONVERGED : SPG_OK;
}

extern "C" spg_status spg_time_parts(spg_handle h, int mode, int reps, float *ms_out, void *stream)
{
    if (!h || h->host_only || !ms_out || reps < 1 || (mode != 0 && mode != 1))
        return fail(SPG_ERR_INVALID, "bad arguments");
    if (mode == 1 && (h->kind != SPG_KIND_PAGERANK || !h->x.p)) return fail(SPG_ERR_INVALID, "run spg_pagerank first");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->fwd.n;
    spg_status st = ensure_vectors(h, N);
    if (st != SPG_OK) return st;
    if (mode == 0) CK(cudaMemsetAsync(h->x.p, 0, N * sizeof(float), s));
    const spg_format_t::Views &V = get_views(h, true);
    const SplitView sv = split_of(h, V);
    const std::vector<PartView> &pvs = V.v;
    for (size_t p = 0; p < pvs.size(); ++p) {
        CK(cudaEventRecord(h->ev0, s));
        for (int r = 0; r < reps; ++r) {
            const bool pat = h->fwd.pattern;
            if (mode == 0) launch_part(pat ? EPI_RAW_PAT : EPI_RAW, pvs[p], sv, h->x.p, h->y.p, nullptr, nullptr, s);
            else launch_part(pat ? EPI_PR_PAT : EPI_PAGERANK, pvs[p], sv, nullptr, nullptr, h->d_state, h->red.p, s);
        }
        CK(cudaEventRecord(h->ev1, s));
        CK(cudaEventSynchronize(h->ev1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        ms_out[p] = ms / (float)reps;
    }
    CK(cudaGetLastError());
    return take_status(h);
}

// ------------------------------------------------- allocation-free SpMV --
//
// spg_spmv_permuted_noalloc runs the same tiled-composite SpMV launches as
// spg_spmv_permuted, but every piece of scratch those kernels need -- the
// partial sums and arrival counters of rows cut into chunks, and the work
// counters of the persistent kernels -- comes from the fixed array below
// instead of from device memory the handle allocated.  The
// array is part of the library image: every GPU that loads the library
// holds it (kNoAllocBytes) until the process exits.

static constexpr int64_t kNoAllocMaxParts = 128;        // tiles + sparse part
static constexpr int64_t kNoAllocMaxSplitRows = 65536;  // rows cut into chunks
static constexpr int64_t kNoAllocMaxChunks = 262144;    // chunks of those rows
static constexpr int64_t kNoAllocSchedWords = 2 * kNoAllocMaxParts;
static constexpr size_t kNoAllocBytes =
    (size_t)(kNoAllocSchedWords + kNoAllocMaxSplitRows + kNoAllocMaxChunks) * 4;  // 1.25 MiB + 1 KiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host code cannot use g_noalloc_scratch as a device address: its device
// address is looked up once per device, with that device current.
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[256];

static spg_status noalloc_scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= 256) return fail(SPG_ERR_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_noalloc_addr[dev]);
    return SPG_OK;
}

extern "C" spg_status spg_spmv_permuted_noalloc(spg_handle h, const float *x_perm, float *y_perm,
                                                void *stream)
{
    if (!h || h->host_only) return fail(SPG_ERR_INVALID, "no device format");
    if (!x_perm || !y_perm || x_perm == y_perm)
        return fail(SPG_ERR_INVALID, "x and y must be distinct device vectors");
    const Layout &L = h->fwd;
    if (L.pattern) return fail(SPG_ERR_UNSUPPORTED, "pattern_only handles: use spg_spmv_permuted");
    if ((int64_t)L.parts.size() > kNoAllocMaxParts || L.nsplit > kNoAllocMaxSplitRows ||
        L.nchunk_slots > kNoAllocMaxChunks)
        return fail(SPG_ERR_INVALID,
                    "format too large for the fixed no-alloc scratch (at most 128 parts, 65536 "
                    "split rows, 262144 split chunks; this format has " +
                    std::to_string(L.parts.size()) + " parts, " + std::to_string(L.nsplit) +
                    " split rows, " + std::to_string(L.nchunk_slots) +
                    " chunks): use spg_spmv_permuted");
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != h->device) return fail(SPG_ERR_INVALID, "the handle's device must be current");
    unsigned char *base = nullptr;
    spg_status st = noalloc_scratch_address(cur, &base);
    if (st != SPG_OK) return st;
    uint32_t *sched = reinterpret_cast<uint32_t *>(base);
    uint32_t *counter = sched + kNoAllocSchedWords;
    float *partial = reinterpret_cast<float *>(counter + kNoAllocMaxSplitRows);
    cudaStream_t s = (cudaStream_t)stream;
    // the work counters and arrival counters must start at zero; the array
    // keeps whatever the previous call left in it
    CK(cudaMemsetAsync(sched, 0, (size_t)(2 * L.parts.size()) * sizeof(uint32_t), s));
    if (L.nsplit > 0) CK(cudaMemsetAsync(counter, 0, (size_t)L.nsplit * sizeof(uint32_t), s));
    SplitView sv = L.split_view();
    sv.partial = partial;
    sv.counter = counter;
    // the handle's own kernel option, with this call's counters in the array
    const bool staged = staged_option(h, true, true);
    for (size_t p = 0; p < L.parts.size(); ++p) {
        const PartView pv = part_view(h, L, p, staged, sched + 2 * p);
        launch_part(EPI_RAW, pv, sv, x_perm, y_perm, nullptr, nullptr, s);
    }
    CK(cudaGetLastError());
    return SPG_OK;
}

// --------------------------------------------------- not yet available --

extern "C" spg_status spg_set_edge_logits(spg_handle h, const float *theta, void *stream)
{
    if (!h || h->host_only || h->kind != SPG_KIND_WEIGHTED) return fail(SPG_ERR_UNSUPPORTED, "needs a WEIGHTED handle");
    if (!theta) return fail(SPG_ERR_INVALID, "null theta");
    cudaStream_t s = (cudaStream_t)stream;
    const float *td = theta;
    if (!is_device_ptr(theta)) {
        CK(h->stage_in.ensure((size_t)h->nnz_in));
        CK(cudaMemcpyAsync(h->stage_in.p, theta, h->nnz_in * sizeof(float), cudaMemcpyHostToDevice, s));
        td = h->stage_in.p;
    }
    Layout *b = h->bwd.get();
    launch_edge_softmax(h->n_graph, h->d_arp, td, h->fwd.d_edge_slot, h->fwd.d_slab,
                        b ? b->d_edge_slot : nullptr, b ? b->d_slab : nullptr, h->d_P, h->d_heavy,
                        h->nheavy, s);
    CK(cudaGetLastError());
    return SPG_OK;
}

extern "C" spg_status spg_rwr_weighted(spg_handle h, float restart, int32_t seed, double tol,
                                       int max_iter, float *r, spg_iter_info *info, void *stream)
{
    if (!h || h->kind != SPG_KIND_WEIGHTED) return fail(SPG_ERR_UNSUPPORTED, "needs a WEIGHTED handle");
    return spg_rwr(h, restart, &seed, 1, tol, max_iter, r, info, stream);
}

extern "C" spg_status spg_rwr_adjoint(spg_handle h, float restart, int32_t seed, const float *r,
                                      const float *g, double tol, int max_iter, float *lambda,
                                      float *dtheta, spg_iter_info *info, void *stream)
{
    if (!h || h->host_only || h->kind != SPG_KIND_WEIGHTED) return fail(SPG_ERR_UNSUPPORTED, "needs a WEIGHTED handle");
    if (!h->bwd) return fail(SPG_ERR_UNSUPPORTED, "adjoint needs build_transpose");
    const int64_t n = h->n_graph;
    if (!r || !g || seed < 0 || seed >= n || !(restart > 0.f && restart <= 1.f) || max_iter < 0)
        return fail(SPG_ERR_INVALID, "bad adjoint arguments");
    cudaStream_t s = (cudaStream_t)stream;
    Layout &Lb = *h->bwd;
    spg_status st = ensure_vectors(h, n);
    if (st != SPG_OK) return st;
    spg_format_t::Views &Vb = get_views_L(h, Lb, h->rt_bwd, true);
    const int nred = nred_of_L(Lb, Vb);
    CK(h->red.ensure((size_t)std::max(1, nred)));
    CK(h->aux.ensure((size_t)n));
    // g into the transposed layout's order; lambda(0) = g
    if ((st = permute_in(h, Lb, g, n, nullptr, h->aux.p, s)) != SPG_OK) return st;
    CK(cudaMemcpyAsync(h->x.p, h->aux.p, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    const double c = 1.0 - (double)restart;
    IterState hs = make_state(h, c, tol, max_iter, n, h->x.p, h->y.p);
    hs.seed = Lb.perm[(size_t)seed];
    hs.aux = h->aux.p;
    CK(cudaMemcpyAsync(h->d_state, &hs, sizeof hs, cudaMemcpyHostToDevice, s));
    LoopGraph *lg;
    st = get_loop_graph(h, "adjoint", [&](cudaStream_t cs, unsigned long long cond, int uc) {
        launch_iteration(h, Lb, h->rt_bwd, EPI_ADJ, EPI_PAGERANK, nred, cond, uc, cs);
    }, &lg);
    if (st != SPG_OK) return st;
    CK(cudaGetLastError());
    if ((st = run_loop(h, lg, max_iter, &hs, info, s)) != SPG_OK) return st;
    // lambda back to original order
    const bool lam_host = lambda && !is_device_ptr(lambda);
    CK(h->stage_out.ensure((size_t)n));
    float *lam_d = (lambda && !lam_host) ? lambda : h->stage_out.p;
    launch_unpermute_state(n, Lb.d_perm, h->d_state, lam_d, nullptr, 0, s);
    if (lam_host) CK(cudaMemcpyAsync(lambda, lam_d, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (dtheta) {
        const float *rd = r;
        if (!is_device_ptr(r)) {
            CK(h->stage_r.ensure((size_t)n));
            CK(cudaMemcpyAsync(h->stage_r.p, r, n * sizeof(float), cudaMemcpyHostToDevice, s));
            rd = h->stage_r.p;
        }
        const bool dt_host = !is_device_ptr(dtheta);
        float *dt_d = dtheta;
        if (dt_host) { CK(h->stage_in.ensure((size_t)std::max(n, h->nnz_in))); dt_d = h->stage_in.p; }
        launch_edge_grad(n, h->d_arp, h->d_acol, h->d_P, lam_d, rd, (float)c, dt_d, h->d_heavy,
                         h->nheavy, s);
        if (dt_host) CK(cudaMemcpyAsync(dtheta, dt_d, h->nnz_in * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return (tol > 0 && !(hs.l1 < tol)) ? SPG_NOT_CONVERGED : SPG_OK;
}

extern "C" spg_status spg_build_batch(const spg_csr *graphs, int count,
                                      const spg_build_opts *opts_in, void *stream, spg_handle *out)
{
    try {
        if (!out || !graphs || count < 1) return fail(SPG_ERR_INVALID, "bad batch arguments");
        *out = nullptr;
        spg_build_opts o;
        std::memset(&o, 0, sizeof o);
        o.heavy_row = -1;
        o.layout_rule = 1;
        if (opts_in) o = *opts_in;
        cudaStream_t s = (cudaStream_t)stream;
        std::unique_ptr<spg_format_t> h(new spg_format_t());
        h->kind = SPG_KIND_BATCH;
        h->host_only = o.device < 0;
        h->ngraph = count;
        h->goff.assign((size_t)count + 1, 0);
        std::vector<std::vector<int64_t>> hrp((size_t)count);
        std::vector<std::vector<int32_t>> hcol((size_t)count);
        std::vector<std::vector<float>> hval((size_t)count);
        std::vector<const int64_t *> rps((size_t)count);
        std::vector<const int32_t *> cols((size_t)count);
        int64_t nnz = 0;
        for (int g = 0; g < count; ++g) {
            const float *v;
            spg_status st = check_csr(&graphs[g], hrp[(size_t)g], hcol[(size_t)g], hval[(size_t)g],
                                      rps[(size_t)g], cols[(size_t)g], v);
            if (st != SPG_OK) return fail(st, "graph " + std::to_string(g) + ": " + g_err);
            h->goff[(size_t)g + 1] = h->goff[(size_t)g] + graphs[g].n_rows;
            nnz += graphs[g].nnz;
        }
        const int64_t N = h->goff[(size_t)count];
        if (N >= kMaxN) return fail(SPG_ERR_INVALID, "total nodes must be < 2^28");
        h->n_graph = N;
        h->nnz_in = nnz;
        // union column source of M: column off_g + u is row u of A_g, values 1/outdeg
        std::vector<int64_t> cp((size_t)N + 1, 0);
        std::vector<int32_t> ri((size_t)nnz);
        std::vector<float> cv((size_t)nnz);
        int64_t q = 0;
        for (int g = 0; g < count; ++g) {
            const int64_t off = h->goff[(size_t)g], ng = graphs[g].n_rows;
            const int64_t *rp = rps[(size_t)g];
            const int32_t *col = cols[(size_t)g];
            for (int64_t u = 0; u < ng; ++u) {
                const int64_t deg = rp[u + 1] - rp[u];
                const float w = deg > 0 ? (float)(1.0 / (double)deg) : 0.f;
                for (int64_t k = rp[u]; k < rp[u + 1]; ++k) {
                    ri[(size_t)q] = (int32_t)(off + col[k]);
                    cv[(size_t)q] = w;
                    ++q;
                }
                cp[(size_t)(off + u) + 1] = q;
            }
        }
        ColumnSource src;
        src.n = N; src.colptr = cp.data(); src.rowidx = ri.data(); src.val = cv.data();
        if (!h->host_only) CK(cudaGetDevice(&h->device));
        BuildParams prm;
        prm.tile_width = 0;
        prm.wl = o.wl;
        prm.heavy = o.heavy_row;
        prm.layout_rule = (o.layout_rule >= 0 && o.layout_rule <= kAutoRule) ? o.layout_rule : 1;
        prm.max_warps = o.max_warps > 0 ? o.max_warps : (h->host_only ? 9728 : query_max_warps());
        prm.max_rows = o.max_rows < 0 ? 0 : (o.max_rows > 0 ? o.max_rows : kDefaultMaxRows);
        prm.unit_slots = o.unit_slots > 0 ? o.unit_slots : kDefaultUnitSlots;
        if (o.claim_order < 0 || o.claim_order > 1) return fail(SPG_ERR_INVALID, "claim_order must be 0 or 1");
        prm.claim_order = o.claim_order;
        if (o.split_cost > 0) prm.split_cost = o.split_cost;
        prm.keep_plan = o.keep_plan != 0;
        prm.stage_cols = resolve_stage_cols(o);
        prm.seg_off = h->goff.data();
        prm.nseg = count;
        prm.segment_order = prm.claim_order == 0;   // longest first within each graph, graph by graph
        std::string err;
        if (!build_layout(src, prm, h->fwd, err)) return fail(SPG_ERR_INVALID, err);
        if (!h->host_only) {
            spg_status st = device_setup(h.get(), o, s);
            if (st != SPG_OK) return st;
            std::vector<int32_t> gid((size_t)N);
            for (int g = 0; g < count; ++g)
                for (int64_t v = h->goff[(size_t)g]; v < h->goff[(size_t)g + 1]; ++v) gid[(size_t)v] = g;
            CK(upload(&h->d_gid, gid.data(), gid.size()));
            CK(upload(&h->d_goff, h->goff.data(), h->goff.size()));
            CK(upload(&h->d_gdstart, h->fwd.seg_dstart.data(), h->fwd.seg_dstart.size()));
            CK(cudaMalloc((void **)&h->d_giters, count * sizeof(int32_t)));
            CK(cudaMalloc((void **)&h->d_gbase, count * sizeof(float)));
            CK(cudaMalloc((void **)&h->d_gl1, count * sizeof(double)));
            CK(cudaMalloc((void **)&h->d_gdelta, count * sizeof(double)));
            // per-graph sums in fixed chunks of at most kBatchChunk positions
            std::vector<int64_t> cstart;
            std::vector<int32_t> cgraph, gchunk((size_t)count + 1);
            for (int g = 0; g < count; ++g) {
                gchunk[(size_t)g] = (int32_t)cgraph.size();
                for (int64_t v = h->goff[(size_t)g]; v < h->goff[(size_t)g + 1]; v += kBatchChunk) {
                    cstart.push_back(v);
                    cgraph.push_back(g);
                }
            }
            gchunk[(size_t)count] = (int32_t)cgraph.size();
            cstart.push_back(N);
            h->nchunk = (int)cgraph.size();
            CK(upload(&h->d_cstart, cstart.data(), cstart.size()));
            CK(upload(&h->d_cgraph, cgraph.data(), cgraph.size()));
            CK(upload(&h->d_gchunk, gchunk.data(), gchunk.size()));
            CK(cudaMalloc((void **)&h->d_cpart, std::max(1, h->nchunk) * sizeof(double2)));
        }
        *out = h.release();
        return SPG_OK;
    } catch (const std::bad_alloc &) {
        return fail(SPG_ERR_OOM, "host memory");
    } catch (const std::exception &ex) {
        return fail(SPG_ERR_INVALID, ex.what());
    }
}

extern "C" spg_status spg_batch_offsets(spg_handle h, int64_t *offsets)
{
    if (!h || h->kind != SPG_KIND_BATCH || !offsets) return fail(SPG_ERR_INVALID, "needs a batch handle");
    std::memcpy(offsets, h->goff.data(), h->goff.size() * sizeof(int64_t));
    return SPG_OK;
}

extern "C" spg_status spg_batch_pagerank(spg_handle h, float damping, double tol, int max_iter,
                                         float *p_out, spg_iter_info *info, void *stream)
{
    if (!h || h->host_only || h->kind != SPG_KIND_BATCH) return fail(SPG_ERR_UNSUPPORTED, "needs a batch handle");
    if (!p_out || !(damping >= 0.f && damping < 1.f) || max_iter < 0)
        return fail(SPG_ERR_INVALID, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->fwd.n;
    const int G = h->ngraph;
    spg_status st = ensure_vectors(h, N);
    if (st != SPG_OK) return st;
    const double c = damping;
    IterState hs = make_state(h, c, tol, max_iter, N, h->x.p, h->y.p);
    hs.gid = h->d_gid;
    hs.gbase = h->d_gbase;
    hs.gl1 = h->d_gl1;
    hs.gdelta = h->d_gdelta;
    hs.giters = h->d_giters;
    hs.goff = h->d_goff;
    hs.gdstart = h->d_gdstart;
    hs.ngraph = G;
    hs.nchunk = h->nchunk;
    hs.cstart = h->d_cstart;
    hs.cgraph = h->d_cgraph;
    hs.gchunk = h->d_gchunk;
    hs.cpart = h->d_cpart;
    CK(cudaMemcpyAsync(h->d_state, &hs, sizeof hs, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(h->d_giters, 0, G * sizeof(int32_t), s));
    // p(0) = 1/n_g: its dangling mass is (#dangling_g)/n_g
    std::vector<float> base((size_t)G);
    for (int g = 0; g < G; ++g) {
        const double ng = (double)(h->goff[(size_t)g + 1] - h->goff[(size_t)g]);
        const double nd = (double)(h->goff[(size_t)g + 1] - h->fwd.seg_dstart[(size_t)g]);
        base[(size_t)g] = (float)((c * (nd / ng) + (1.0 - c)) / ng);
    }
    CK(cudaMemcpyAsync(h->d_gbase, base.data(), G * sizeof(float), cudaMemcpyHostToDevice, s));
    launch_batch_init(N, h->d_state, h->x.p, s);
    LoopGraph *lg;
    st = get_loop_graph(h, "batch", [&](cudaStream_t cs, unsigned long long cond, int uc) {
        launch_parts(h, EPI_BATCH, nullptr, nullptr, h->d_state, h->red.p, cs);
        launch_batch_reduce(h->d_state, h->nchunk, cs);
        launch_batch_check(h->d_state, G, cond, uc, cs);
    }, &lg);
    if (st != SPG_OK) return st;
    CK(cudaGetLastError());
    if ((st = run_loop(h, lg, max_iter, &hs, nullptr, s)) != SPG_OK) return st;
    float *od;
    bool staged;
    if ((st = out_target(h, p_out, N, false, &od, &staged, s)) != SPG_OK) return st;
    launch_unpermute_state(N, h->fwd.d_perm, h->d_state, od, nullptr, 0, s);
    if (staged) CK(cudaMemcpyAsync(p_out, od, N * sizeof(float), cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> it((size_t)G);
    std::vector<double> l1((size_t)G), dg((size_t)G);
    CK(cudaMemcpyAsync(it.data(), h->d_giters, G * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(l1.data(), h->d_gl1, G * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(dg.data(), h->d_gdelta, G * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool all = true;
    for (int g = 0; g < G; ++g) {
        if (it[(size_t)g] == 0) all = false;
        if (info) {
            info[g].iters = it[(size_t)g] ? it[(size_t)g] : hs.iter;
            info[g].last_l1 = l1[(size_t)g];
            info[g].dangling = dg[(size_t)g];
            info[g].ms = 0.f;
        }
    }
    return (tol > 0 && !all) ? SPG_NOT_CONVERGED : SPG_OK;
}

// ------------------------------------------------------------------ misc --

extern "C" spg_status spg_load_table(const char *path)
{
    if (!path) { perf_table_default(perf_table()); return SPG_OK; }
    std::string err;
    PerfTable t;
    if (!perf_table_load(path, t, err)) return fail(SPG_ERR_INVALID, err);
    perf_table() = t;
    return SPG_OK;
}

extern "C" int64_t spg_launch_count(void) { return launch_count(); }

extern "C" const char *spg_status_string(spg_status s)
{
    switch (s) {
    case SPG_OK: return "ok";
    case SPG_NOT_CONVERGED: return "not converged";
    case SPG_ERR_INVALID: return "invalid argument";
    case SPG_ERR_OOM: return "out of memory";
    case SPG_ERR_CUDA: return "CUDA error";
    case SPG_ERR_TIMEOUT: return "device wait timed out";
    case SPG_ERR_UNSUPPORTED: return "unsupported for this handle";
    }
    return "unknown status";
}

extern "C" const char *spg_last_error(void) { return g_err.c_str(); }
extern "C" const char *spg_version(void) { return "spg 0.1 (sm_103a)"; }
