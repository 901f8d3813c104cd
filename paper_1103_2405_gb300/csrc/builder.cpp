// builder.cpp -- host construction of the tiled composite layout.
//
// Steps, in the order of the paper (Yang, Parthasarathy, Sadayappan):
//   1. column lengths and the symmetric order by decreasing length, ties by
//      ascending id, by counting sort (Section 3.1 Solution 2; "Sorting
//      Cost" paragraph);
//   2. the permuted matrix as rows with ascending columns;
//   3. Algorithm 1: dense tiles of tile_width columns while the first column
//      of the next tile is longer than 1 and fewer than n / tile_width tiles;
//      the rest is the sparse part, itself one composite tile (Solution 3);
//   4. per part: in-tile row lengths, rows ranked by decreasing length,
//      rows above the heavy threshold cut into chunks (GB300 addition),
//      workload size by Algorithm 2 over the Algorithm 3 model, packing into
//      rectangles of w = first row's length and h = floor(WL / w) rows, row-
//      or column-major with w (or h) padded to a multiple of 32 (Solution 3).
// Host C++ with std::thread; nothing here runs on the GPU.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <limits>
#include <mutex>
#include <sstream>

#include "format.h"

namespace spg {

int hw_threads()
{
    static int n = [] {
        unsigned h = std::thread::hardware_concurrency();
        if (h == 0) h = 1;
        return (int)std::min(h, 64u);
    }();
    return n;
}

// ------------------------------------------------------- performance table --

PerfTable &perf_table()
{
    static PerfTable t = [] { PerfTable x; perf_table_default(x); return x; }();
    return t;
}

// Built-in table used until a measured one is loaded: a warp's slot rate
// grows with the rectangle it owns (more independent loads in flight), a
// row-major warp pays a 5-step shuffle reduction per row (~16 slots' worth),
// and everything saturates at a nominal 800e9 slots/s.
void perf_table_default(PerfTable &t)
{
    for (int major = 0; major < 2; ++major)
        for (int lw = 0; lw < kTableLog; ++lw)
            for (int lh = 0; lh < kTableLog; ++lh) {
                double w = std::ldexp(1.0, lw), h = std::ldexp(1.0, lh);
                double size = w * h;
                double eff = size / (size + 2048.0);
                if (major == 0) eff *= w / (w + 16.0);
                t.perf[major][lw][lh] = 800e9 * eff;
            }
    t.loaded = false;
}

static int ilog2_floor(int64_t v)
{
    int l = 0;
    while (v > 1) { v >>= 1; ++l; }
    return l;
}

double perf_lookup(const PerfTable &t, int major, int64_t wpad, int64_t hpad)
{
    int lw = std::min(ilog2_floor(wpad), kTableLog - 1);
    int lh = std::min(ilog2_floor(hpad), kTableLog - 1);
    return t.perf[major][lw][lh];
}

bool perf_table_load(const char *path, PerfTable &t, std::string &err)
{
    std::ifstream f(path);
    if (!f) { err = std::string("cannot open table ") + path; return false; }
    bool have[2][kTableLog][kTableLog] = {};
    double val[2][kTableLog][kTableLog] = {};
    std::string line;
    int nhave = 0;
    while (std::getline(f, line)) {
        auto hash = line.find('#');
        if (hash != std::string::npos) line.resize(hash);
        std::istringstream is(line);
        int mj, lw, lh;
        double p;
        if (!(is >> mj >> lw >> lh >> p)) continue;
        if (mj < 0 || mj > 1 || lw < 0 || lw >= kTableLog || lh < 0 || lh >= kTableLog ||
            !(p > 0)) {
            err = "bad table line: " + line;
            return false;
        }
        if (!have[mj][lw][lh]) ++nhave;
        have[mj][lw][lh] = true;
        val[mj][lw][lh] = p;
    }
    if (nhave == 0) { err = "empty table"; return false; }
    // missing buckets take the nearest measured one (L1 distance in (lw, lh),
    // same major first, first in scan order on ties)
    for (int mj = 0; mj < 2; ++mj)
        for (int lw = 0; lw < kTableLog; ++lw)
            for (int lh = 0; lh < kTableLog; ++lh) {
                if (have[mj][lw][lh]) { t.perf[mj][lw][lh] = val[mj][lw][lh]; continue; }
                int best = std::numeric_limits<int>::max();
                double bv = 0;
                for (int pass = 0; pass < 2 && best == std::numeric_limits<int>::max(); ++pass) {
                    int m2 = pass == 0 ? mj : 1 - mj;
                    for (int a = 0; a < kTableLog; ++a)
                        for (int b = 0; b < kTableLog; ++b)
                            if (have[m2][a][b]) {
                                int d = std::abs(a - lw) + std::abs(b - lh);
                                if (d < best) { best = d; bv = val[m2][a][b]; }
                            }
                }
                t.perf[mj][lw][lh] = bv;
            }
    t.loaded = true;
    return true;
}

// ------------------------------------------------------------------ model --

static inline int64_t ru32(int64_t v) { return (v + 31) / 32 * 32; }

static inline int pick_major(int rule, int64_t w, int64_t h)
{
    if (rule == 0) return w >= h ? 0 : 1;                 // the paper's rule
    if (rule == 2) return 0;                              // every workload CSR-vector
    if (rule == 3) return 1;                              // every workload ELL
    return h * ru32(w) < ru32(h) * w ? 0 : 1;             // fewer padded slots; tie: column-major
}

// Rows of a workload starting at a row of length w: floor(WL / w), at least
// one, at most max_rows (GB300: a warp walks its 32-row blocks in sequence,
// so a tall workload of one-entry rows is a long serial chain) and at most
// the rows left.
static inline int64_t wl_height(int64_t WL, int64_t w, int64_t left, int64_t max_rows)
{
    int64_t h = WL / w;
    if (h < 1) h = 1;
    if (max_rows > 0 && h > max_rows) h = max_rows;
    if (h > left) h = left;
    return h;
}

double latency_rounds(const Workload &d)
{
    if (d.w == 0) return 1.0 + 2.0 * (double)((d.h + 127) / 128);
    if (d.major == 1) {
        const int64_t hp = ru32(d.h);
        int64_t r = 0;
        for (int64_t b = 0; b < hp; b += 64)
            r += b + 32 < hp ? 2 * ((d.w + 3) / 4) : 2 * (d.w / 8) + (d.w % 8 ? 2 : 0);
        return 2.0 + (double)std::max<int64_t>(r, 2);
    }
    const int64_t nst = d.w / 32;
    const int64_t per = (nst >= 4 ? nst / 4 + 1 : 0) + (nst % 4 ? 2 : 0);
    return 2.0 + (double)d.h * (double)per;
}

// Claim cost of a workload: padded slots + 4 per row (a row-free workload:
// 4 per row).
static inline int64_t claim_cost(const Workload &d)
{
    const int64_t slots = d.w == 0 ? 0 : d.major == 0 ? (int64_t)d.h * d.w : ru32(d.h) * d.w;
    return slots + 4 * (int64_t)d.h;
}

// Claim order and claim units of every part.  The persistent kernels'
// warps take work in array order, so a long workload that comes late in the
// array keeps one warp busy after the others have run out of work (R-MAT
// scale 22 in ranking order with 32 x 32 workloads stored row-major: claimed
// at 105 us of a 190 us launch, each ran about 80 us).  Longest first
// (stable, by latency_rounds) ends the launch with the short ones.  Claim
// units are then runs of consecutive workloads whose cost reaches
// unit_slots, so that one atomic on the work counter covers several small
// workloads while a large one stays alone.
//
// Block-diagonal unions (BuildParams::segment_order): the workloads are then
// stored segment by segment -- the segment (graph) of a workload's first row,
// stable, so the longest-first order holds within a segment, row-free
// workloads last -- and claim units end at segment boundaries.  The per-
// segment degree order keeps every segment's rows and columns at its own
// positions, so the warps running at any moment work on a few graphs and
// share their x and y lines in L1 and L2 (512 Chung-Lu graphs, PageRank
// iteration with the persistent 8-warp kernel: 0.625 ms against 0.677 ms in
// the longest-first order over all graphs).
static void order_and_group(Layout &L, const BuildParams &prm)
{
    if (prm.claim_order == 0 && !L.wl.empty()) {
        for (const PartHost &ph : L.parts) {
            auto b = L.wl.begin() + ph.wl_off;
            std::vector<std::pair<double, Workload>> key((size_t)ph.nwl_total);
            for (int64_t j = 0; j < ph.nwl_total; ++j) key[(size_t)j] = {latency_rounds(b[j]), b[j]};
            std::stable_sort(key.begin(), key.end(),
                             [](const std::pair<double, Workload> &a, const std::pair<double, Workload> &c) {
                                 return a.first > c.first;
                             });
            for (int64_t j = 0; j < ph.nwl_total; ++j) b[j] = key[(size_t)j].second;
        }
    }
    const bool grouped = prm.segment_order && prm.nseg > 0 && L.parts.size() == 1 && !L.wl.empty();
    std::vector<int32_t> wgroup;   // segment of each workload of part 0 (nseg: row-free)
    if (grouped) {
        const int64_t *so = prm.seg_off;
        const int32_t G = (int32_t)prm.nseg;
        const PartHost &ph = L.parts[0];
        auto b = L.wl.begin() + ph.wl_off;
        std::vector<std::pair<int32_t, Workload>> key((size_t)ph.nwl_total);
        for (int64_t j = 0; j < ph.nwl_total; ++j) {
            int32_t g = G;
            if (b[j].w > 0) {
                uint32_t e = L.rows[(size_t)b[j].rows];
                if (e & kRowSplit) e = L.split[(size_t)L.slot_owner[(size_t)(e & ~kRowSplit)]].row;
                const int64_t r = (int64_t)(e & kRowIdMask);
                g = (int32_t)(std::upper_bound(so, so + G + 1, r) - so) - 1;
            }
            key[(size_t)j] = {g, b[j]};
        }
        std::stable_sort(key.begin(), key.end(),
                         [](const std::pair<int32_t, Workload> &a, const std::pair<int32_t, Workload> &c) {
                             return a.first < c.first;
                         });
        wgroup.resize((size_t)ph.nwl_total);
        for (int64_t j = 0; j < ph.nwl_total; ++j) {
            b[j] = key[(size_t)j].second;
            wgroup[(size_t)j] = key[(size_t)j].first;
        }
    }
    L.units.clear();
    for (PartHost &ph : L.parts) {
        ph.unit_off = (int64_t)L.units.size();
        int64_t acc = 0;
        for (int64_t j = 0; j < ph.nwl_total; ++j) {
            if (grouped && j > 0 && wgroup[(size_t)j] != wgroup[(size_t)j - 1]) acc = 0;
            if (acc == 0) L.units.push_back((int32_t)j);
            acc += L.wl.empty() ? 1 : claim_cost(L.wl[(size_t)(ph.wl_off + j)]);
            if (prm.unit_slots <= 1 || acc >= prm.unit_slots) acc = 0;
        }
        ph.nunits = (int64_t)L.units.size() - ph.unit_off;
        L.units.push_back((int32_t)ph.nwl_total);
    }
}

// Algorithm 3: walk the ranked rows workload by workload; every max_warps
// warps form one "iteration" (Eq. 1) whose time is its padded size over the
// mean table performance of its warps (Eqs. 3-5); the total is the sum
// (Eq. 2).
double model_time(const int32_t *vlen, int64_t nv, int64_t WL, int64_t max_warps, int rule,
                  int64_t max_rows, const PerfTable &t)
{
    if (nv <= 0) return 0.0;
    double total = 0.0, P = 0.0, S = 0.0;
    int64_t cnt = 0, j = 0;
    for (int64_t i = 0; i < nv; ++j) {
        int64_t w = vlen[i], h = wl_height(WL, w, nv - i, max_rows);
        int major = pick_major(rule, w, h);
        int64_t wp = major == 0 ? ru32(w) : w, hp = major == 0 ? h : ru32(h);
        if (j > 0 && j % max_warps == 0) {
            total += S / (P / (double)cnt);
            P = S = 0.0;
            cnt = 0;
        }
        P += perf_lookup(t, major, wp, hp);
        S += (double)(wp * hp);
        ++cnt;
        i += h;
    }
    if (cnt) total += S / (P / (double)cnt);
    return total;
}

// Algorithm 2: WL from the longest row upward in steps of it while
// WL <= nnz / max_warps; the first minimum wins; an empty range gives the
// longest row.
int64_t alg2_search(const int32_t *vlen, int64_t nv, int64_t nnz, int64_t max_warps, int rule,
                    int64_t max_rows, const PerfTable &t, double *best)
{
    if (nv <= 0) { if (best) *best = 0.0; return 0; }
    int64_t low = vlen[0], opt = 0;
    double opt_t = std::numeric_limits<double>::infinity();
    for (int64_t WL = low; WL * max_warps <= nnz; WL += low) {
        double tt = model_time(vlen, nv, WL, max_warps, rule, max_rows, t);
        if (tt < opt_t) { opt_t = tt; opt = WL; }
    }
    if (opt == 0) {
        opt = low;
        opt_t = model_time(vlen, nv, low, max_warps, rule, max_rows, t);
    }
    if (best) *best = opt_t;
    return opt;
}

// Rank the rows of one part: virtual rows (chunks of rows longer than H)
// by decreasing length, ties by ascending row id then chunk (counting sort,
// so rows are visited once in ascending order).
static void rank_rows(const std::vector<int32_t> &len, int64_t H, std::vector<int32_t> &rrow,
                      std::vector<int32_t> &rchunk, std::vector<int32_t> &rlen)
{
    const int64_t n = (int64_t)len.size();
    int64_t maxv = 0, nv = 0;
    for (int64_t r = 0; r < n; ++r) {
        int64_t L = len[r];
        if (L <= 0) continue;
        if (H > 0 && L > H) { nv += (L + H - 1) / H; maxv = std::max<int64_t>(maxv, H); }
        else { nv += 1; maxv = std::max<int64_t>(maxv, L); }
    }
    std::vector<int64_t> pos((size_t)maxv + 2, 0);
    auto vcount = [&](int64_t L, int64_t ch, int64_t nch) {
        return ch < nch - 1 ? H : L - H * (nch - 1);
    };
    for (int64_t r = 0; r < n; ++r) {
        int64_t L = len[r];
        if (L <= 0) continue;
        if (H > 0 && L > H) {
            int64_t nch = (L + H - 1) / H;
            for (int64_t ch = 0; ch < nch; ++ch) pos[(size_t)vcount(L, ch, nch)]++;
        } else {
            pos[(size_t)L]++;
        }
    }
    // descending lengths: bucket maxv first
    int64_t run = 0;
    for (int64_t l = maxv; l >= 1; --l) { int64_t c = pos[(size_t)l]; pos[(size_t)l] = run; run += c; }
    rrow.assign((size_t)nv, 0);
    rchunk.assign((size_t)nv, 0);
    rlen.assign((size_t)nv, 0);
    for (int64_t r = 0; r < n; ++r) {
        int64_t L = len[r];
        if (L <= 0) continue;
        int64_t nch = (H > 0 && L > H) ? (L + H - 1) / H : 1;
        for (int64_t ch = 0; ch < nch; ++ch) {
            int64_t vl = nch > 1 ? vcount(L, ch, nch) : L;
            int64_t k = pos[(size_t)vl]++;
            rrow[(size_t)k] = (int32_t)r;
            rchunk[(size_t)k] = (int32_t)ch;
            rlen[(size_t)k] = (int32_t)vl;
        }
    }
}

// Split threshold of one part (GB300 addition): candidates
// H_k = round_up32(ceil(base / 2^k)), base = round_up32(max(32,
// ceil(nnz / max_warps))), k = 0..3; each priced by Algorithm 3 at its
// Algorithm 2 workload size plus split_cost per chunk of a split row.
static int64_t tune_heavy(const std::vector<int32_t> &len, int64_t nnz, const BuildParams &prm,
                          const PerfTable &t)
{
    if (nnz == 0) return 32;
    int64_t base = (nnz + prm.max_warps - 1) / prm.max_warps;
    base = ru32(std::max<int64_t>(base, 32));
    int64_t bestH = base, prevH = -1;
    double best = std::numeric_limits<double>::infinity();
    std::vector<int32_t> rr, rc, rl;
    for (int k = 0; k < 4; ++k) {
        int64_t div = (int64_t)1 << k;
        int64_t H = std::max<int64_t>(32, ru32((base + div - 1) / div));
        if (H == prevH) continue;
        prevH = H;
        rank_rows(len, H, rr, rc, rl);
        double tm = 0.0;
        int64_t WL = alg2_search(rl.data(), (int64_t)rl.size(), nnz, prm.max_warps,
                                 prm.layout_rule, prm.max_rows, t, &tm);
        double chunks = 0.0;
        for (int32_t L : len)
            if (L > H) chunks += (double)((L + H - 1) / H);
        double cost = model_time(rl.data(), (int64_t)rl.size(), WL, prm.max_warps,
                                 prm.layout_rule, prm.max_rows, t) + prm.split_cost * chunks;
        if (cost < best) { best = cost; bestH = H; }
    }
    return bestH;
}

// Modelled cost of one part's plan under prm.layout_rule: the split
// threshold (tuned or given), Algorithm 2's workload size (or the given
// one), Algorithm 3's time plus split_cost per chunk of a split row -- the
// quantity the automatic storage rule minimises.
static double plan_cost(const std::vector<int32_t> &len, int64_t nnz, const BuildParams &prm,
                        const PerfTable &t, int64_t *H_out)
{
    const int64_t H = prm.heavy < 0 ? tune_heavy(len, nnz, prm, t) : prm.heavy;
    *H_out = H;
    if (nnz == 0) return 0.0;
    std::vector<int32_t> rr, rc, rl;
    rank_rows(len, H, rr, rc, rl);
    const int64_t nv = (int64_t)rl.size();
    double tm = 0.0;
    const int64_t WL = prm.wl > 0 ? prm.wl
                                  : alg2_search(rl.data(), nv, nnz, prm.max_warps, prm.layout_rule,
                                                prm.max_rows, t, &tm);
    if (prm.wl > 0) tm = model_time(rl.data(), nv, WL, prm.max_warps, prm.layout_rule, prm.max_rows, t);
    double chunks = 0.0;
    if (H > 0)
        for (int32_t L : len)
            if (L > H) chunks += (double)((L + H - 1) / H);
    return tm + prm.split_cost * chunks;
}

// ---------------------------------------------------------------- builder --

bool build_layout(const ColumnSource &src, const BuildParams &prm, Layout &L, std::string &err)
{
    const int64_t N = src.n;
    const int64_t nnz_src = src.colptr[N];
    const PerfTable &table = perf_table();
    L = Layout();
    L.n = N;
    L.max_warps = prm.max_warps;
    // rows this layout holds (all, or one rank's share of a row partition)
    auto kept = [&](int64_t orig_row) { return !src.row_keep || src.row_keep[orig_row] != 0; };

    // 1. column lengths; order by decreasing length, ties ascending id
    std::vector<int64_t> collen((size_t)N);
    int64_t maxlen = 0;
    for (int64_t j = 0; j < N; ++j) {
        collen[(size_t)j] = src.colptr[j + 1] - src.colptr[j];
        maxlen = std::max(maxlen, collen[(size_t)j]);
    }
    // (per segment when the matrix is a block-diagonal union of graphs)
    {
        const int64_t nseg = prm.nseg > 0 ? prm.nseg : 1;
        std::vector<int64_t> start((size_t)maxlen + 2);
        L.perm.assign((size_t)N, 0);
        L.inv.assign((size_t)N, 0);
        for (int64_t g = 0; g < nseg; ++g) {
            const int64_t a = prm.nseg > 0 ? prm.seg_off[g] : 0;
            const int64_t b = prm.nseg > 0 ? prm.seg_off[g + 1] : N;
            std::fill(start.begin(), start.end(), 0);
            for (int64_t j = a; j < b; ++j) start[(size_t)collen[(size_t)j]]++;
            int64_t run = a, nz = start[0];
            for (int64_t l = maxlen; l >= 0; --l) { int64_t c = start[(size_t)l]; start[(size_t)l] = run; run += c; }
            for (int64_t j = a; j < b; ++j) {
                int64_t p = start[(size_t)collen[(size_t)j]]++;
                L.perm[(size_t)j] = (int32_t)p;
                L.inv[(size_t)p] = (int32_t)j;
            }
            L.seg_dstart.push_back(b - nz);
        }
    }
    // zero-length columns sort last: dangling tail of the order
    {
        int64_t nz = 0;
        for (int64_t j = 0; j < N; ++j) nz += collen[(size_t)j] == 0;
        L.dangling_start = N - nz;
    }

    // 2. permuted matrix by rows, columns ascending
    std::vector<int64_t> rp((size_t)N + 1, 0);
    {
        std::vector<std::atomic<int64_t>> cnt((size_t)N);
        parallel_for(N, 1 << 16, [&](int64_t lo, int64_t hi) {
            for (int64_t r = lo; r < hi; ++r) cnt[(size_t)r].store(0, std::memory_order_relaxed);
        });
        parallel_for(nnz_src, 1 << 18, [&](int64_t lo, int64_t hi) {
            for (int64_t k = lo; k < hi; ++k)
                if (kept(src.rowidx[k]))
                    cnt[(size_t)L.perm[(size_t)src.rowidx[k]]].fetch_add(1, std::memory_order_relaxed);
        });
        for (int64_t r = 0; r < N; ++r) rp[(size_t)r + 1] = rp[(size_t)r] + cnt[(size_t)r].load();
    }
    const int64_t nnz = rp[(size_t)N];
    L.nnz = nnz;
    std::vector<int32_t> mcol((size_t)nnz);
    std::vector<float> mval((size_t)nnz);
    std::vector<int64_t> meid;
    if (prm.track_edges) meid.resize((size_t)nnz);
    {
        std::vector<std::atomic<int64_t>> fill((size_t)N);
        parallel_for(N, 1 << 16, [&](int64_t lo, int64_t hi) {
            for (int64_t r = lo; r < hi; ++r) fill[(size_t)r].store(rp[(size_t)r], std::memory_order_relaxed);
        });
        parallel_for(N, 1 << 12, [&](int64_t lo, int64_t hi) {
            for (int64_t j = lo; j < hi; ++j) {
                int32_t c = L.perm[(size_t)j];
                for (int64_t k = src.colptr[j]; k < src.colptr[j + 1]; ++k) {
                    if (!kept(src.rowidx[k])) continue;
                    int64_t r = L.perm[(size_t)src.rowidx[k]];
                    int64_t s = fill[(size_t)r].fetch_add(1, std::memory_order_relaxed);
                    mcol[(size_t)s] = c;
                    mval[(size_t)s] = src.val[k];
                    if (prm.track_edges) meid[(size_t)s] = src.eid ? src.eid[k] : k;
                }
            }
        });
        // sort each row by column (values and edge ids follow)
        parallel_dynamic(N, 4096, [&](int64_t lo, int64_t hi) {
            std::vector<int64_t> idx;
            std::vector<int32_t> tc;
            std::vector<float> tv;
            std::vector<int64_t> te;
            for (int64_t r = lo; r < hi; ++r) {
                int64_t b = rp[(size_t)r], e = rp[(size_t)r + 1], len = e - b;
                if (len < 2) continue;
                bool sorted = true;
                for (int64_t k = b + 1; k < e && sorted; ++k) sorted = mcol[(size_t)k - 1] < mcol[(size_t)k];
                if (sorted) continue;
                idx.resize((size_t)len);
                for (int64_t k = 0; k < len; ++k) idx[(size_t)k] = b + k;
                std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t c2) {
                    return mcol[(size_t)a] < mcol[(size_t)c2];
                });
                tc.resize((size_t)len); tv.resize((size_t)len);
                for (int64_t k = 0; k < len; ++k) { tc[(size_t)k] = mcol[(size_t)idx[(size_t)k]]; tv[(size_t)k] = mval[(size_t)idx[(size_t)k]]; }
                if (prm.track_edges) {
                    te.resize((size_t)len);
                    for (int64_t k = 0; k < len; ++k) te[(size_t)k] = meid[(size_t)idx[(size_t)k]];
                    std::copy(te.begin(), te.end(), meid.begin() + b);
                }
                std::copy(tc.begin(), tc.end(), mcol.begin() + b);
                std::copy(tv.begin(), tv.end(), mval.begin() + b);
            }
        });
    }

    // 3. Algorithm 1
    int64_t ntile = 0;
    const int64_t TW = prm.tile_width;
    if (TW > 0) {
        while (ntile < N / TW) {
            int64_t start = ntile * TW;
            if (collen[(size_t)L.inv[(size_t)start]] <= 1) break;
            ++ntile;
        }
    }
    if (ntile + 1 > 127) { err = "too many tiles (> 126)"; return false; }
    L.tile_width = TW > 0 ? TW : 0;
    L.ntile = ntile;
    const int64_t P = ntile + 1;
    std::vector<int64_t> bound((size_t)P + 1);
    for (int64_t p = 0; p < P; ++p) bound[(size_t)p] = p * (TW > 0 ? TW : 0);
    bound[(size_t)P] = N;
    if (ntile == 0) bound[0] = 0;

    // per-row start of each part (ascending columns => binary search)
    std::vector<int64_t> pstart;
    auto part_start = [&](int64_t p, int64_t r) -> int64_t {
        if (p == 0) return rp[(size_t)r];
        if (p == P) return rp[(size_t)r + 1];
        return pstart[(size_t)((p - 1) * N + r)];
    };
    if (P > 1) {
        pstart.resize((size_t)((P - 1) * N));
        parallel_for(N, 1 << 14, [&](int64_t lo, int64_t hi) {
            for (int64_t r = lo; r < hi; ++r) {
                const int32_t *b = mcol.data() + rp[(size_t)r], *e = mcol.data() + rp[(size_t)r + 1];
                for (int64_t p = 1; p < P; ++p)
                    pstart[(size_t)((p - 1) * N + r)] =
                        (std::lower_bound(b, e, (int32_t)bound[(size_t)p]) - mcol.data());
            }
        });
    }
    std::vector<int8_t> first_part((size_t)N, -1), last_part((size_t)N, -1);
    parallel_for(N, 1 << 14, [&](int64_t lo, int64_t hi) {
        for (int64_t r = lo; r < hi; ++r)
            for (int64_t p = 0; p < P; ++p)
                if (part_start(p + 1, r) > part_start(p, r)) {
                    if (first_part[(size_t)r] < 0) first_part[(size_t)r] = (int8_t)p;
                    last_part[(size_t)r] = (int8_t)p;
                }
    });

    // 4. per part: lengths, threshold, ranking, WL, workloads
    L.parts.resize((size_t)P);
    std::vector<std::vector<int32_t>> rank_row(P), rank_chunk(P), rank_len(P);
    std::vector<std::vector<int64_t>> wfirst(P);
    std::vector<std::vector<int32_t>> wh(P), ww(P), wm(P);
    std::vector<int32_t> len((size_t)N);
    for (int64_t p = 0; p < P; ++p) {
        PartHost &ph = L.parts[(size_t)p];
        ph.c0 = bound[(size_t)p];
        ph.c1 = bound[(size_t)p + 1];
        int64_t pn = 0;
        for (int64_t r = 0; r < N; ++r) {
            int64_t l = part_start(p + 1, r) - part_start(p, r);
            len[(size_t)r] = (int32_t)l;
            pn += l;
        }
        ph.nnz = pn;
        {
            int64_t all = 0, head = 0;
            for (int64_t c = ph.c0; c < ph.c1; ++c) {
                const int64_t l = collen[(size_t)L.inv[(size_t)c]];
                all += l;
                if (c < ph.c0 + prm.stage_cols) head += l;
            }
            ph.slice_share = all > 0 ? (double)head / (double)all : 0.0;
        }
        // storage rule of the part: the given one, or (kAutoRule) the rule
        // of rules 0-3 whose plan -- its own split threshold and workload
        // size -- the Algorithm 3 model prices lowest (Section 5: CSR-vector
        // and ELL are special cases of the composite format); ties keep the
        // first in the order 1, 0, 2, 3
        int rule = prm.layout_rule;
        int64_t H = -1;
        if (rule == kAutoRule) {
            // the four plans priced side by side (one thread each)
            const int order[4] = {1, 0, 2, 3};
            double cost[4];
            int64_t hs[4];
            std::vector<std::thread> th;
            for (int k = 0; k < 4; ++k)
                th.emplace_back([&, k] {
                    BuildParams q = prm;
                    q.layout_rule = order[k];
                    cost[k] = plan_cost(len, pn, q, table, &hs[k]);
                });
            for (auto &x : th) x.join();
            int kb = 0;
            for (int k = 1; k < 4; ++k)
                if (cost[k] < cost[kb]) kb = k;
            rule = order[kb];
            H = hs[kb];
        }
        ph.rule = rule;
        BuildParams pr = prm;
        pr.layout_rule = rule;
        if (H < 0) H = prm.heavy < 0 ? tune_heavy(len, pn, pr, table) : prm.heavy;
        ph.heavy = H;
        rank_rows(len, H, rank_row[p], rank_chunk[p], rank_len[p]);
        const int64_t nv = (int64_t)rank_len[p].size();
        ph.nvirt = nv;
        double tm = 0.0;
        int64_t WL = prm.wl > 0 ? prm.wl
                                : alg2_search(rank_len[p].data(), nv, pn, prm.max_warps,
                                              rule, prm.max_rows, table, &tm);
        if (prm.wl > 0)
            tm = model_time(rank_len[p].data(), nv, WL, prm.max_warps, rule,
                            prm.max_rows, table);
        ph.wl = nv > 0 ? WL : 0;
        ph.predicted_s = tm;
        for (int64_t i = 0; i < nv;) {
            int64_t w = rank_len[p][(size_t)i], h = wl_height(WL, w, nv - i, prm.max_rows);
            wfirst[p].push_back(i);
            wh[p].push_back((int32_t)h);
            ww[p].push_back((int32_t)w);
            wm[p].push_back(pick_major(rule, w, h));
            i += h;
        }
        ph.nwl = (int64_t)wfirst[p].size();
    }
    for (int64_t r = 0; r < N; ++r)
        if (first_part[(size_t)r] < 0 && kept(L.inv[(size_t)r])) L.zero_rows.push_back(r);

    // TILE-COO: the same degree order and column tiles, each part's entries
    // as a plain (row, column, value) list in row order
    if (prm.build_coo) {
        L.coo_off.assign((size_t)P + 1, 0);
        for (int64_t p = 0; p < P; ++p) L.coo_off[(size_t)p + 1] = L.coo_off[(size_t)p] + L.parts[(size_t)p].nnz;
        const int64_t tot = L.coo_off[(size_t)P];
        L.coo_row.resize((size_t)tot);
        L.coo_col.resize((size_t)tot);
        L.coo_val.resize((size_t)tot);
        std::vector<int64_t> pos((size_t)N + 1);
        for (int64_t p = 0; p < P; ++p) {
            pos[0] = L.coo_off[(size_t)p];
            for (int64_t r = 0; r < N; ++r) pos[(size_t)r + 1] = pos[(size_t)r] + part_start(p + 1, r) - part_start(p, r);
            parallel_for(N, 1 << 14, [&](int64_t lo, int64_t hi) {
                for (int64_t r = lo; r < hi; ++r) {
                    const int64_t b = part_start(p, r), e = part_start(p + 1, r);
                    for (int64_t k = b; k < e; ++k) {
                        const int64_t q = pos[(size_t)r] + (k - b);
                        L.coo_row[(size_t)q] = (int32_t)r;
                        L.coo_col[(size_t)q] = mcol[(size_t)k];
                        L.coo_val[(size_t)q] = mval[(size_t)k];
                    }
                }
            });
        }
    }

    // 5. packing: offsets.  The rows without entries (the epilogue alone)
    // go with part 0, the first and largest launch: there they are claimed
    // last, as filler while its long workloads finish, instead of forming a
    // launch of their own when the sparse part holds no entries (R-MAT
    // scale 24: 9.4M such rows, 74 us of a 0.84 ms iteration as a separate
    // launch).
    const int64_t zpart = 0;
    int64_t nwl_all = 0, nrows_all = 0, nslab = 0, nblocks_all = 0;
    std::vector<int64_t> slab_off_p((size_t)P), rows_off_p((size_t)P);
    for (int64_t p = 0; p < P; ++p) {
        PartHost &ph = L.parts[(size_t)p];
        int64_t nz = (p == zpart) ? ((int64_t)L.zero_rows.size() + kZeroRowsPerWorkload - 1) /
                                        kZeroRowsPerWorkload
                                  : 0;
        ph.nwl_total = ph.nwl + nz;
        ph.wl_off = nwl_all;
        nwl_all += ph.nwl_total;
        rows_off_p[(size_t)p] = nrows_all;
        nrows_all += ph.nvirt + (p == zpart ? (int64_t)L.zero_rows.size() : 0);
        slab_off_p[(size_t)p] = nslab;
        for (int64_t j = 0; j < ph.nwl; ++j) {
            int64_t w = ww[p][(size_t)j], h = wh[p][(size_t)j];
            nslab += wm[p][(size_t)j] == 0 ? h * ru32(w) : ru32(h) * w;
        }
        ph.nblocks = (int32_t)((ph.nwl_total + kWarpsPerBlock - 1) / kWarpsPerBlock);
        ph.red_base = (int32_t)nblocks_all;
        nblocks_all += ph.nblocks;
    }
    if (nwl_all > INT32_MAX || nrows_all > INT32_MAX) { err = "layout too large"; return false; }
    L.padded_slots = nslab;
    L.wl.resize((size_t)nwl_all);
    L.rows.resize((size_t)nrows_all);
    L.pattern = prm.pattern_only;
    if (L.pattern) {
        L.slab4.resize((size_t)nslab);
        L.inv_deg.assign((size_t)N, 0.f);
        for (int64_t j = 0; j < N; ++j)
            if (src.colptr[j + 1] > src.colptr[j]) L.inv_deg[(size_t)L.perm[(size_t)j]] = src.val[src.colptr[j]];
    } else {
        L.slab.resize((size_t)nslab);
    }
    if (prm.track_edges) L.edge_slot.assign((size_t)nnz_src, -1);

    // split rows (ascending row id per part) and their chunk slots
    std::vector<std::vector<int32_t>> split_first(P);   // per part: row -> first slot (-1)
    for (int64_t p = 0; p < P; ++p) {
        int64_t H = L.parts[(size_t)p].heavy;
        if (H <= 0) continue;
        bool any = false;
        for (int64_t r = 0; r < N && !any; ++r)
            any = part_start(p + 1, r) - part_start(p, r) > H;
        if (!any) continue;
        split_first[p].assign((size_t)N, -1);
        for (int64_t r = 0; r < N; ++r) {
            int64_t l = part_start(p + 1, r) - part_start(p, r);
            if (l <= H) continue;
            int32_t nch = (int32_t)((l + H - 1) / H);
            uint32_t flags = (uint32_t)r;
            if (first_part[(size_t)r] < p) flags |= kRowNotFirst;
            if (last_part[(size_t)r] > p) flags |= kRowNotLast;
            if (src.row_class && src.row_class[L.inv[(size_t)r]]) flags |= kRowClass;
            SplitRow s;
            s.row = flags;
            s.first_slot = (int32_t)L.nchunk_slots;
            s.nchunks = nch;
            s.red_slot = (int32_t)L.split.size();
            split_first[p][(size_t)r] = s.first_slot;
            for (int32_t c = 0; c < nch; ++c) L.slot_owner.push_back((int32_t)L.split.size());
            L.split.push_back(s);
            L.nchunk_slots += nch;
        }
    }
    L.nsplit = (int64_t)L.split.size();
    L.nred = nblocks_all + L.nsplit;   // with the plain 8-warp launch

    // workload descriptors + row entries + slab
    for (int64_t p = 0; p < P; ++p) {
        PartHost &ph = L.parts[(size_t)p];
        const int64_t H = ph.heavy;
        int64_t slab_pos = slab_off_p[(size_t)p], row_pos = rows_off_p[(size_t)p];
        std::vector<int64_t> wl_slab((size_t)ph.nwl);
        for (int64_t j = 0; j < ph.nwl; ++j) {
            int64_t w = ww[p][(size_t)j], h = wh[p][(size_t)j];
            int mj = wm[p][(size_t)j];
            Workload d;
            d.slab = slab_pos;
            d.rows = (int32_t)(row_pos + wfirst[p][(size_t)j]);
            d.w = (int32_t)(mj == 0 ? ru32(w) : w);
            d.h = (int32_t)h;
            d.major = mj;
            L.wl[(size_t)(ph.wl_off + j)] = d;
            wl_slab[(size_t)j] = slab_pos;
            slab_pos += mj == 0 ? h * ru32(w) : ru32(h) * w;
        }
        const bool has_split = !split_first[p].empty();
        // row entries
        parallel_for(ph.nvirt, 1 << 16, [&](int64_t lo, int64_t hi) {
            for (int64_t k = lo; k < hi; ++k) {
                int64_t r = rank_row[p][(size_t)k];
                uint32_t e;
                if (has_split && split_first[p][(size_t)r] >= 0) {
                    e = kRowSplit | (uint32_t)(split_first[p][(size_t)r] + rank_chunk[p][(size_t)k]);
                } else {
                    e = (uint32_t)r;
                    if (first_part[(size_t)r] < p) e |= kRowNotFirst;
                    if (last_part[(size_t)r] > p) e |= kRowNotLast;
                    if (src.row_class && src.row_class[L.inv[(size_t)r]]) e |= kRowClass;
                }
                L.rows[(size_t)(row_pos + k)] = e;
            }
        });
        // slab
        parallel_dynamic(ph.nwl, 64, [&](int64_t lo, int64_t hi) {
            for (int64_t j = lo; j < hi; ++j) {
                const Workload &d = L.wl[(size_t)(ph.wl_off + j)];
                const int64_t first = wfirst[p][(size_t)j];
                const int64_t hp = d.major == 0 ? d.h : ru32(d.h);
                for (int64_t i = 0; i < hp; ++i) {
                    int64_t len_i = 0, base = 0;
                    if (i < d.h) {
                        int64_t k = first + i;
                        int64_t r = rank_row[p][(size_t)k];
                        len_i = rank_len[p][(size_t)k];
                        base = part_start(p, r) + (H > 0 ? (int64_t)rank_chunk[p][(size_t)k] * H : 0);
                    }
                    for (int64_t e = 0; e < d.w; ++e) {
                        int64_t slot = d.major == 0 ? d.slab + i * d.w + e
                                                    : d.slab + (i / 32) * 32 * d.w + e * 32 + (i % 32);
                        uint2 v;
                        if (e < len_i) {
                            int64_t src_k = base + e;
                            v.x = (uint32_t)mcol[(size_t)src_k];
                            float fv = mval[(size_t)src_k];
                            std::memcpy(&v.y, &fv, 4);
                            if (prm.track_edges) L.edge_slot[(size_t)meid[(size_t)src_k]] = slot;
                        } else {
                            v.x = 0xffffffffu;
                            v.y = 0u;
                        }
                        if (L.pattern) L.slab4[(size_t)slot] = v.x;
                        else L.slab[(size_t)slot] = v;
                    }
                }
            }
        });
        // zero-row workloads (part 0): w = 0, rows written by the epilogue
        if (p == zpart) {
            int64_t zr = (int64_t)L.zero_rows.size();
            for (int64_t z = 0, j = ph.nwl; z < zr; z += kZeroRowsPerWorkload, ++j) {
                Workload d;
                d.slab = slab_pos;
                d.rows = (int32_t)(row_pos + ph.nvirt + z);
                d.w = 0;
                d.h = (int32_t)std::min<int64_t>(kZeroRowsPerWorkload, zr - z);
                d.major = 1;
                L.wl[(size_t)(ph.wl_off + j)] = d;
            }
            for (int64_t z = 0; z < zr; ++z) {
                int64_t r = L.zero_rows[(size_t)z];
                uint32_t e = (uint32_t)r;
                if (src.row_class && src.row_class[L.inv[(size_t)r]]) e |= kRowClass;
                L.rows[(size_t)(row_pos + ph.nvirt + z)] = e;
            }
        }
        if (prm.keep_plan) {
            ph.rank_row = std::move(rank_row[p]);
            ph.rank_chunk = std::move(rank_chunk[p]);
            ph.rank_len = std::move(rank_len[p]);
            ph.wl_first = std::move(wfirst[p]);
            ph.wl_h = std::move(wh[p]);
            ph.wl_w = std::move(ww[p]);
            ph.wl_major = std::move(wm[p]);
        }
        rank_row[p].clear(); rank_row[p].shrink_to_fit();
        rank_chunk[p].clear(); rank_chunk[p].shrink_to_fit();
        rank_len[p].clear(); rank_len[p].shrink_to_fit();
    }
    order_and_group(L, prm);
    return true;
}

// ----------------------------------------------------------------- upload --

template <class T> static cudaError_t up(T **dst, const std::vector<T> &v, int64_t &bytes,
                                          cudaStream_t s)
{
    size_t b = std::max<size_t>(1, v.size()) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)dst, b);
    if (e != cudaSuccess) return e;
    bytes += (int64_t)b;
    if (!v.empty()) e = cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    return e;
}

cudaError_t upload_layout(Layout &L, bool keep_host, cudaStream_t s)
{
    cudaError_t e;
    L.device_bytes = 0;
#define SPG_UP(d, v) if ((e = up(&L.d, L.v, L.device_bytes, s)) != cudaSuccess) return e
    SPG_UP(d_perm, perm);
    SPG_UP(d_inv, inv);
    SPG_UP(d_wl, wl);
    SPG_UP(d_units, units);
    SPG_UP(d_rows, rows);
    if (L.pattern) { SPG_UP(d_slab4, slab4); SPG_UP(d_inv_deg, inv_deg); }
    else SPG_UP(d_slab, slab);
    SPG_UP(d_split, split);
    SPG_UP(d_slot_owner, slot_owner);
    if (!L.edge_slot.empty()) SPG_UP(d_edge_slot, edge_slot);
    if (!L.coo_off.empty()) {
        SPG_UP(d_coo_row, coo_row);
        SPG_UP(d_coo_col, coo_col);
        SPG_UP(d_coo_val, coo_val);
    }
#undef SPG_UP
    size_t pb = std::max<int64_t>(1, L.nchunk_slots) * sizeof(float);
    if ((e = cudaMalloc((void **)&L.d_partial, pb)) != cudaSuccess) return e;
    size_t cb = std::max<int64_t>(1, L.nsplit) * sizeof(uint32_t);
    if ((e = cudaMalloc((void **)&L.d_counter, cb)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(L.d_counter, 0, cb, s)) != cudaSuccess) return e;
    L.device_bytes += (int64_t)(pb + cb);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    L.on_device = true;
    if (!keep_host) {
        std::vector<Workload>().swap(L.wl);
        std::vector<int32_t>().swap(L.units);
        std::vector<uint32_t>().swap(L.rows);
        std::vector<uint2>().swap(L.slab);
        std::vector<uint32_t>().swap(L.slab4);
        std::vector<int32_t>().swap(L.coo_row);
        std::vector<int32_t>().swap(L.coo_col);
        std::vector<float>().swap(L.coo_val);
    }
    return cudaSuccess;
}

void Layout::free_device()
{
    cudaFree(d_perm); cudaFree(d_inv); cudaFree(d_wl); cudaFree(d_units); cudaFree(d_rows); cudaFree(d_slab);
    cudaFree(d_split); cudaFree(d_slot_owner); cudaFree(d_partial); cudaFree(d_counter);
    cudaFree(d_edge_slot); cudaFree(d_slab4); cudaFree(d_inv_deg);
    cudaFree(d_coo_row); cudaFree(d_coo_col); cudaFree(d_coo_val);
    d_coo_row = d_coo_col = nullptr; d_coo_val = nullptr;
    d_slab4 = nullptr; d_inv_deg = nullptr;
    d_perm = d_inv = nullptr; d_wl = nullptr; d_units = nullptr; d_rows = nullptr; d_slab = nullptr;
    d_split = nullptr; d_slot_owner = nullptr; d_partial = nullptr; d_counter = nullptr;
    d_edge_slot = nullptr;
    on_device = false;
}

std::vector<PartView> Layout::part_views() const
{
    std::vector<PartView> v;
    for (const PartHost &ph : parts) {
        PartView pv;
        pv.wl = d_wl + ph.wl_off;
        pv.rows = d_rows;
        pv.slab = d_slab;
        pv.slab4 = d_slab4;
        pv.nwl = (int32_t)ph.nwl_total;
        pv.nblocks = ph.nblocks;
        pv.red_base = ph.red_base;
        pv.c0 = (int32_t)ph.c0;
        pv.xs_cols = 0;
        pv.sched = nullptr;
        pv.pf_ahead = 0;
        pv.status = nullptr;
        pv.tma = 0;
        pv.persist = 0;
        pv.units = d_units + ph.unit_off;
        pv.nunits = (int32_t)ph.nunits;
        v.push_back(pv);
    }
    return v;
}

SplitView Layout::split_view() const
{
    SplitView s;
    s.rows = d_split;
    s.slot_owner = d_slot_owner;
    s.partial = d_partial;
    s.counter = d_counter;
    s.red_split_base = 0;
    s.pad_ = 0;
    return s;
}

}  // namespace spg
