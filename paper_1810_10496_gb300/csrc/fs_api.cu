// C-ABI of the feature-similarity library (declared in include/fs.h).
//
// Host side of the method of Sec. 4: validates arguments, owns the device
// copy of the reference set (feature vectors and Table-1-style phase
// orders), plans each search call into work items and candidate buffers,
// and enqueues the kernels on the caller's stream. No call allocates device
// memory except fs_build_db; search calls use the caller's workspace.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fs_internal.cuh"

using namespace fsk;

struct fs_db {
    int dev = 0;
    int num_sms = 0;
    int64_t l2_bytes = 0;
    int64_t n = 0;
    int32_t f = 0, fu = 0, fl = 0;
    fs_precision prec = FS_FP32;
    int32_t n_seg = 1;
    std::vector<int64_t> seg_off;   // host copy
    std::vector<float> r_max;       // per segment: largest row residual
    float* raw = nullptr;
    float* unit = nullptr;
    double* b64 = nullptr;
    void* lowp = nullptr;
    float* scale = nullptr;
    float* resid = nullptr;
    int64_t* seq_off = nullptr;
    int16_t* seq_ids = nullptr;
    int64_t seq_total = 0;
    int64_t* seg_off_dev = nullptr;
    float* r_max_dev = nullptr;
    uint32_t* status = nullptr;
    unsigned long long* stats = nullptr;
    int64_t n_pad = 0;              // rows of the code array (tensor-core scans)
    CUtensorMap map_x;              // TMA map of the codes (tensor-core scans)
    CUtensorMap map_x_half;         // the same with half-tile boxes (pairs of CTAs)
    fs_tuning tune = {0, 0, 0, 0};  // scan planning parameters (0 = default)
    int metric = FS_COSINE;         // fs_metric of the searches
    double* mu = nullptr;           // [n_seg][f] standardisation statistics
    double* sg = nullptr;
    float* row_term = nullptr;      // [n] Euclidean 1/2 |z|^2
    float* row_mag = nullptr;       // [n] |z| or sum |z_i|
    float* mag_max_dev = nullptr;   // [n_seg]
    std::vector<float> mag_max;     // host copy
    uint64_t wait_ns = 0;           // limit of the scan's bounded waits (0: 2 s)
    int withhold_load = 0;          // test aid (fs_db_set_wait_test)
};

namespace {

thread_local std::string g_err;

fs_status fail(fs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define FS_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(FS_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

void free_db(fs_db* db) {
    if (!db) return;
    void* ptrs[] = {db->raw,      db->unit,      db->b64,       db->lowp,     db->scale,
                    db->resid,    db->seq_off,   db->seq_ids,   db->seg_off_dev,
                    db->r_max_dev, db->status,   db->stats,     db->mu,       db->sg,
                    db->row_term, db->row_mag,   db->mag_max_dev};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete db;
}

fs_status alloc(void** p, size_t bytes, const char* what) {
    if (bytes == 0) bytes = 256;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? FS_ENOMEM : FS_ECUDA,
                    "cudaMalloc of %zu bytes for %s failed: %s", bytes, what,
                    cudaGetErrorString(e));
    }
    return FS_OK;
}

int lowp_width(int f, fs_precision prec) {
    if (prec == FS_BF16) return (int)round_up(f, 64);
    if (prec == FS_FP8_E4M3) return (int)round_up(f, 128);
    return 0;
}

// ---------------------------------------------------------------------------
// stage timing: CUDA events recorded on the call's stream around each stage

struct Profiler {
    std::mutex mu;
    bool on = false;
    struct Rec {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> pending;
    double ms[FS_NUM_STAGES] = {};
    uint64_t calls[FS_NUM_STAGES] = {};
    std::atomic<uint64_t> launches{0};

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
};

Profiler& prof() {
    static Profiler p;
    return p;
}

// Records the start of a stage when timing is on; finish() records its end.
struct StageTimer {
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    StageTimer(int s, cudaStream_t cs) : stage(s), st(cs) {
        Profiler& p = prof();
        std::lock_guard<std::mutex> g(p.mu);
        if (!p.on) return;
        a = p.get();
        b = p.get();
        if (a && b) cudaEventRecord(a, st);
    }
    void finish(int nlaunch) {
        Profiler& p = prof();
        p.launches += (uint64_t)nlaunch;
        if (!a || !b) return;
        cudaEventRecord(b, st);
        std::lock_guard<std::mutex> g(p.mu);
        p.pending.push_back({stage, a, b});
        a = b = nullptr;
    }
};

// ---------------------------------------------------------------------------
// error bounds of the approximate scores (see select.cu for their use)

struct Bounds {
    double scan, rq, rerank;
    double rx;   // FP8 (per-row bounds): U, the bound on a unit vector's norm
};

Bounds score_bounds(const fs_db* db, double r_xmax) {
    const double u = std::ldexp(1.0, -24);
    const int m = (int)ceil_div(db->fu, 32);
    auto gamma = [u](double n) { return n * u / (1.0 - n * u); };
    // |computed 1/||x|| * ||x|| - 1| <= eta: FMA sums of m_norm squares per
    // lane (a 32-stride element per lane, or four consecutive elements per
    // 128-element block with 128-bit loads), a 5-level butterfly, a square
    // root and a reciprocal
    const int m_norm = std::max(m, 4 * (int)ceil_div(db->f, 128));
    const double eta = ((m_norm + 5) * 0.5 + 2.0) * u * 1.01;
    // |u_q . u_x - s| for the FP32 unit vectors (each element also rounded)
    const double th = 2.0 * u + u * u;
    const double e_norm = (2.0 * eta + eta * eta) * (1.0 + th) + th;
    const double U = (1.0 + eta) * (1.0 + u);   // bound on ||u||
    Bounds b;
    // the rerank's warp-wide dot products sum per lane the same elements as
    // the norms with 128-bit loads (m_norm terms), then a 5-level butterfly
    b.rerank = gamma(m_norm + 5) * U * U + e_norm;
    b.rx = 0.0;
    if (db->prec == FS_FP32) {
        b.scan = (gamma(db->fu) * U * U + e_norm) * 1.25 + 1e-12;
        b.rq = 0.0;
    } else if (db->prec == FS_FP8_E4M3) {
        // FP8 with per-row bounds: for codes with residual norms r_q and r_x,
        // |c_q.c_x - u_q.u_x| <= r_x (U + r_q) + U r_q (Cauchy-Schwarz, as
        // below, with each row's own r_x). The row term is applied per row;
        // here: the accumulation (8 K u sum|p|), the two scale products of
        // the epilogue, the FP32 unit vectors, and 1e-6 for the FP32 rounding
        // of the bounds themselves (values below 1.2, so far above it).
        const double cmax = U * 1.1;
        b.scan = 8.0 * db->fl * u * cmax * cmax + 6.0 * u * cmax * cmax + e_norm * 1.25 + 1e-6;
        b.rq = U * 1.001;
        b.rx = U;
    } else {
        // low-precision codes c with ||u - c|| = r: |c_q.c_x - u_q.u_x| <=
        // r_q (U + r_x) + U r_x by Cauchy-Schwarz. The residual norms are
        // computed from the exact rounding errors with a sum of squares and a
        // square root (relative error below 1e-6), so a 0.1 % margin covers
        // them. The accumulation of the exact products in FP32 is allowed
        // 8 K u sum|p|, twice the bound of an adder that truncates, for
        // tensor-core accumulation of undocumented internal width; FP8 adds
        // the two scale multiplications of the epilogue.
        const double cmax = U * (db->prec == FS_BF16 ? 1.004 : 1.1);
        b.scan = U * r_xmax * 1.001 + 8.0 * db->fl * u * cmax * cmax + e_norm * 1.25 +
                 (db->prec == FS_FP8_E4M3 ? 6.0 * u * cmax * cmax : 0.0) + 1e-12;
        b.rq = (U + r_xmax) * 1.001;
    }
    b.rerank = b.rerank * 1.25 + 1e-12;
    return b;
}

// ---------------------------------------------------------------------------
// planning of one search call

struct Plan {
    std::vector<SegPlan> seg;       // scan-item order: largest work first
    std::vector<int32_t> q_order;   // indices into seg sorted by first query
    int64_t total_items = 0;
    int64_t total_cand = 0;
    int k_max = 0;
    int tile_rows = 0;
    int slots = 0;                  // resident scan blocks, or pairs of blocks
    bool pair = false;              // tensor-core scan on pairs of SMs
    int list_t = kListT;
    int64_t total_band = 0;         // FP8: band-buffer entries
};

struct Layout {
    size_t plan, q_order, q_a64, q_ss, q_unit, q_lowp, q_scale, q_resid, cand, band, band_cnt,
        class_thr, counters, fb_list, fb2_list, cand_fb, fb_score, fb_index, shared_thr, q_plan,
        total;
};

bool tensor_scan(const fs_db* db) { return db->prec != FS_FP32; }

int scan_slots(const fs_db* db) {
    return tensor_scan(db) ? db->num_sms : db->num_sms * scan_fp32_ctas_per_sm();
}

// sizing != 0: plan the largest workspace any k could need (list size 16)
fs_status make_plan(const fs_db* db, int32_t nq, const int32_t* q_seg_off, const int32_t* k,
                    Plan& pl, int sizing = 0) {
    const int n_seg = db->n_seg;
    if (q_seg_off) {
        if (q_seg_off[0] != 0 || q_seg_off[n_seg] != nq)
            return fail(FS_EINVAL, "q_seg_off must start at 0 and end at nq=%d", nq);
        for (int s = 0; s < n_seg; ++s)
            if (q_seg_off[s + 1] < q_seg_off[s])
                return fail(FS_EINVAL, "q_seg_off must be non-decreasing (segment %d)", s);
    } else if (n_seg != 1) {
        return fail(FS_EINVAL, "the database has %d segments: q_seg_off is required", n_seg);
    }
    pl.tile_rows = tensor_scan(db) ? kTcTileRows : kFp32TileRows;
    const int lists = tensor_scan(db) ? kTcLists : kFp32Lists;
    pl.slots = std::max(1, scan_slots(db));
    if (tensor_scan(db) && db->tune.scan_pairs > 0) {
        const int kblocks = (int)(db->fl * (db->prec == FS_BF16 ? 2 : 1) / 128);
        const int pairs = scan_tc_pair_slots(db->prec == FS_FP8_E4M3, kblocks);
        if (pairs > 0) {
            pl.pair = true;
            pl.slots = pairs;
        }
    }
    pl.seg.resize(n_seg);
    pl.k_max = 0;
    int64_t work = 0;  // (query tile, row tile) pairs
    for (int s = 0; s < n_seg; ++s) {
        const int ks = k ? k[s] : 0;
        if (!k || ks < 1 || ks > FS_MAX_K)
            return fail(FS_EINVAL, "k[%d]=%d is outside 1..%d", s, ks, FS_MAX_K);
        pl.k_max = std::max(pl.k_max, ks);
        SegPlan& p = pl.seg[s];
        std::memset(&p, 0, sizeof(p));
        p.row0 = db->seg_off[s];
        p.seg = s;
        p.nrows = db->seg_off[s + 1] - db->seg_off[s];
        p.q0 = q_seg_off ? q_seg_off[s] : 0;
        p.nq = q_seg_off ? q_seg_off[s + 1] - q_seg_off[s] : nq;
        p.k = ks;
        p.qtiles = (int)ceil_div(p.nq, kQTile);
        p.units = pl.pair ? (int)ceil_div(p.qtiles, 2) : p.qtiles;
        p.lists = lists;
        work += (int64_t)p.units * ceil_div(p.nrows, pl.tile_rows);
    }
    // the tensor-core scan keeps 8-entry lists when every k fits (fewer
    // inserts), or 4-entry ones when tuned so and every k <= 4
    pl.list_t = kListT;
    if (tensor_scan(db) && !sizing) {
        const int want = db->tune.list_len ? db->tune.list_len : kListTSmall;
        if (want == kListTTiny && pl.k_max <= kListTTiny)
            pl.list_t = kListTTiny;
        else if (want <= kListTSmall && pl.k_max <= kListTSmall)
            pl.list_t = kListTSmall;
    }
    // Row chunking. (1) Items of about work / (4 slots) tiles keep every block
    // busy. (2) Blocks that run at the same time scan about slots / qtiles + 1
    // chunks of a segment; those chunks should fit in half of L2 so the query
    // tiles of a chunk read its rows from L2, not HBM. (3) Among chunk counts
    // meeting (1) and (2), take the one that fills the last round of items
    // best (blocks take items in number order, one at a time). The 4 and the
    // half are the defaults of the tuning parameters items_per_block and
    // l2_share_pct.
    const int items_per_block = db->tune.items_per_block ? db->tune.items_per_block : 4;
    const int l2_pct = db->tune.l2_share_pct ? db->tune.l2_share_pct : 50;
    const int64_t desired = (int64_t)pl.slots * items_per_block;
    const int64_t tiles_per_item = std::max<int64_t>(1, ceil_div(work, desired));
    const int64_t row_bytes = tensor_scan(db) ? (int64_t)db->fl * (db->prec == FS_BF16 ? 2 : 1)
                                              : (int64_t)db->fu * 4;
    const int64_t l2_bytes = std::max<int64_t>(db->l2_bytes, 32 << 20);
    std::vector<int64_t> seg_work(n_seg, 0);
    for (int s = 0; s < n_seg; ++s) {
        SegPlan& p = pl.seg[s];
        const int64_t row_tiles = ceil_div(p.nrows, pl.tile_rows);
        int64_t chunk_tiles = std::max<int64_t>(1, std::min(row_tiles, tiles_per_item));
        const double live = (double)pl.slots / std::max(1, p.units) + 1.0;
        const double l2_share = (double)l2_bytes * l2_pct / 100.0;
        if (l2_pct > 0 && n_seg == 1 && p.units >= 2 && row_tiles > 1 &&
            live * chunk_tiles * pl.tile_rows * row_bytes > (double)l2_bytes) {
            // the chunks in flight overflow L2: cap them at a share of it
            const int64_t cap = std::max<int64_t>(
                1, (int64_t)(l2_share / (live * row_bytes * pl.tile_rows)));
            int64_t c_lo = ceil_div(row_tiles, std::min(chunk_tiles, cap));
            double best = -1.0;
            int64_t best_c = c_lo;
            for (int64_t c = c_lo; c <= std::min(row_tiles, c_lo + 64); ++c) {
                const int64_t items = c * p.units;
                const double fill = (double)items / (double)(ceil_div(items, pl.slots) * pl.slots);
                if (fill > best + 1e-3) {
                    best = fill;
                    best_c = c;
                }
                if (fill > 0.985) break;
            }
            chunk_tiles = ceil_div(row_tiles, best_c);
        }
        p.chunk_rows = (int32_t)(chunk_tiles * pl.tile_rows);
        p.chunks = p.nrows > 0 ? (int32_t)ceil_div(p.nrows, p.chunk_rows) : 0;
        p.list_t = pl.list_t;
        if (db->prec == FS_FP8_E4M3) {
            // band capacity per query: the rows within the FP8 error of the k-th
            // best (measured: a few hundred per million rows; the buffer allows
            // one in 64) plus the rows each of the query's lists (two per row
            // chunk) may accept before its running bound forms (measured up to
            // about 50 in a list's first tile; many lists of one tile each, all
            // in the first wave, are the worst case); never more rows than the
            // segment has, so a segment of up to 8,192 rows cannot overflow
            const int64_t want = std::min<int64_t>(
                65536, std::max<int64_t>(8192, round_up(128 * (int64_t)p.chunks +
                                                        ceil_div(p.nrows, 64), 256)));
            p.band_cap = (int32_t)std::min<int64_t>(want, std::max<int64_t>(round_up(p.nrows, 32), 32));
        }
        if (is_std_metric(db->metric)) {
            // the per-query bound is computed with the query (E = q_resid)
            p.bound_scan = 0.0f;
            p.bound_rq = 1.0f;
            p.bound_rerank = 0.0f;
            p.mag_max = db->mag_max[s];
        } else {
            const Bounds b = score_bounds(db, db->r_max[s]);
            p.bound_scan = (float)b.scan;
            p.bound_rq = (float)b.rq;
            p.bound_rerank = (float)b.rerank;
            p.bound_rx = (float)b.rx;
        }
        if (p.nq > 0 && p.nrows > 0) seg_work[s] = (int64_t)p.units * row_tiles;
    }
    // number the scan items largest segment first: blocks take items in
    // number order, so the long ones start first and the short ones fill in
    std::vector<int32_t> order(n_seg);
    for (int s = 0; s < n_seg; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return seg_work[a] > seg_work[b]; });
    std::vector<SegPlan> sorted(n_seg);
    std::vector<int32_t> pos_of(n_seg);
    int64_t item = 0, cand = 0, band = 0;
    const bool fp8 = db->prec == FS_FP8_E4M3 && !is_std_metric(db->metric);
    for (int i = 0; i < n_seg; ++i) {
        SegPlan p = pl.seg[order[i]];
        p.item0 = item;
        p.cand0 = cand;
        p.band0 = band;
        if (p.nq > 0 && p.nrows > 0) {
            item += (int64_t)p.units * p.chunks;
            // the FP8 scan keeps a band per query instead of candidate lists
            if (fp8)
                band += (int64_t)p.nq * p.band_cap;
            else
                cand += (int64_t)p.nq * p.chunks * p.lists * pl.list_t;
        }
        sorted[i] = p;
        pos_of[order[i]] = i;
    }
    pl.seg.swap(sorted);
    // the segments in their original (first-query) order
    pl.q_order.resize(n_seg);
    for (int s = 0; s < n_seg; ++s) pl.q_order[s] = pos_of[s];
    pl.total_items = item;
    pl.total_cand = cand;
    pl.total_band = band;
    return FS_OK;
}

Layout make_layout(const fs_db* db, int32_t nq, const Plan& pl) {
    Layout L;
    size_t off = 0;
    auto take = [&off](size_t bytes) {
        size_t at = off;
        off += round_up((int64_t)std::max<size_t>(bytes, 1), 256);
        return at;
    };
    const size_t lw = db->prec == FS_BF16 ? 2 : 1;
    L.plan = take(sizeof(SegPlan) * pl.seg.size());
    L.q_order = take(sizeof(int32_t) * pl.seg.size());
    L.q_a64 = take(sizeof(double) * nq);
    L.q_ss = take(sizeof(float) * nq);
    L.q_unit = take(sizeof(float) * (size_t)nq * db->fu);
    L.q_lowp = take(lw * (size_t)round_up(nq, kTcQueryRows) * db->fl);
    L.q_scale = take(sizeof(float) * nq);
    L.q_resid = take(sizeof(float) * nq);
    L.cand = take(sizeof(uint64_t) * (size_t)pl.total_cand);
    L.band = take(sizeof(uint64_t) * (size_t)pl.total_band);
    L.band_cnt = take(sizeof(int32_t) * (db->prec == FS_FP8_E4M3 ? nq : 0));
    L.class_thr = take(sizeof(uint32_t) * (db->prec == FS_FP8_E4M3 ? (size_t)nq * FS_MAX_K : 0));
    L.counters = take(8 * sizeof(int32_t));
    L.fb_list = take(sizeof(int32_t) * nq);
    L.fb2_list = take(sizeof(int32_t) * nq);
    L.cand_fb = take(sizeof(uint64_t) * (size_t)nq * kFbChunks * kListT);
    L.fb_score = take(sizeof(double) * (size_t)nq * kFbChunks * FS_MAX_K);
    L.fb_index = take(sizeof(int32_t) * (size_t)nq * kFbChunks * FS_MAX_K);
    L.shared_thr = take(sizeof(uint32_t) * nq);
    L.q_plan = take(sizeof(int32_t) * nq);
    L.total = off;
    return L;
}

DbView db_view(const fs_db* db) {
    DbView v;
    v.raw = db->raw;
    v.unit = db->unit;
    v.b64 = db->b64;
    v.lowp = db->lowp;
    v.scale = db->scale;
    v.resid = db->resid;
    v.seq_off = db->seq_off;
    v.seq_ids = db->seq_ids;
    v.status = db->status;
    v.stats = db->stats;
    v.n = db->n;
    v.f = db->f;
    v.fu = db->fu;
    v.fl = db->fl;
    v.prec = (int32_t)db->prec;
    v.metric = db->metric;
    v.mu = db->mu;
    v.sg = db->sg;
    v.row_term = db->row_term;
    v.row_mag = db->row_mag;
    return v;
}

fs_status check_device(const fs_db* db) {
    int cur = -1;
    FS_CUDA(cudaGetDevice(&cur));
    if (cur != db->dev)
        return fail(FS_EINVAL, "current device %d is not the database's device %d", cur, db->dev);
    return FS_OK;
}

fs_status search(const fs_db* db, const float* q, int32_t nq, const int32_t* q_seg_off,
                 const int32_t* k, const int32_t* exclude, void* workspace, size_t ws_bytes,
                 int32_t* idx, float* dist, int16_t* seq_out, int32_t* seq_len, int32_t l_max,
                 int32_t* dup_of, bool gather, void* stream) {
    if (!db) return fail(FS_EINVAL, "db is NULL");
    if (nq < 0) return fail(FS_EINVAL, "nq=%d is negative", nq);
    if (nq > 0 && (!q || !idx || !dist))
        return fail(FS_EINVAL, "q, idx and dist must be non-NULL when nq > 0");
    if (gather && nq > 0 && (!seq_out || !seq_len))
        return fail(FS_EINVAL, "seq_out and seq_len must be non-NULL when nq > 0");
    if (gather && l_max < 1) return fail(FS_EINVAL, "l_max=%d must be >= 1", l_max);
    Plan pl;
    fs_status st = make_plan(db, nq, q_seg_off, k, pl);
    if (st != FS_OK) return st;
    const Layout L = make_layout(db, nq, pl);
    if (nq == 0) return FS_OK;
    if (!workspace) return fail(FS_EINVAL, "workspace is NULL");
    if (((uintptr_t)workspace & 255) != 0) return fail(FS_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < L.total)
        return fail(FS_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed", ws_bytes,
                    L.total);
    st = check_device(db);
    if (st != FS_OK) return st;

    cudaStream_t cs = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    CallView c;
    std::memset(&c, 0, sizeof(c));
    c.plan = (const SegPlan*)(ws + L.plan);
    c.q_order = (const int32_t*)(ws + L.q_order);
    c.q_raw = q;
    c.q_a64 = (double*)(ws + L.q_a64);
    c.q_ss = (float*)(ws + L.q_ss);
    c.q_unit = (float*)(ws + L.q_unit);
    c.q_lowp = ws + L.q_lowp;
    c.q_scale = (float*)(ws + L.q_scale);
    c.q_resid = (float*)(ws + L.q_resid);
    c.cand = (uint64_t*)(ws + L.cand);
    c.band = (uint64_t*)(ws + L.band);
    c.band_cnt = (int32_t*)(ws + L.band_cnt);
    c.class_thr = (uint32_t*)(ws + L.class_thr);
    c.fb_count = (int32_t*)(ws + L.counters);
    c.work_counter = c.fb_count + 1;
    c.fb2_count = c.fb_count + 2;
    c.aborted = c.fb_count + 3;
    c.sel_counter = c.fb_count + 4;
    c.wait_ns = db->wait_ns;
    c.withhold_load = db->withhold_load;
    c.fb_list = (int32_t*)(ws + L.fb_list);
    c.fb2_list = (int32_t*)(ws + L.fb2_list);
    c.cand_fb = (uint64_t*)(ws + L.cand_fb);
    c.fb_score = (double*)(ws + L.fb_score);
    c.fb_index = (int32_t*)(ws + L.fb_index);
    c.shared_thr = (uint32_t*)(ws + L.shared_thr);
    c.q_plan = (int32_t*)(ws + L.q_plan);
    c.exclude = exclude;
    c.out_idx = idx;
    c.out_dist = dist;
    c.nq = nq;
    c.n_seg = db->n_seg;
    c.k_max = pl.k_max;
    c.total_items = pl.total_items;
    const DbView v = db_view(db);

    {
        StageTimer t(FS_STAGE_PREPARE, cs);
        FS_CUDA(launch_write_plan(pl.seg.data(), pl.q_order.data(), db->n_seg,
                                  (SegPlan*)(ws + L.plan), (int32_t*)(ws + L.q_order), c.fb_count,
                                  c.work_counter, cs));
        FS_CUDA(launch_query_plan(c, (int32_t*)(ws + L.q_plan), cs));
        if (is_std_metric(db->metric))
            FS_CUDA(launch_std_queries(v, c, cs));
        else
            FS_CUDA(launch_prepare_rows(q, nq, db->f, c.q_unit, db->fu, c.q_ss, c.q_lowp,
                                        db->fl, c.q_scale, c.q_resid, db->prec, db->status, cs));
        // 0 sorts below every order-mapped score
        FS_CUDA(cudaMemsetAsync(c.shared_thr, 0, sizeof(uint32_t) * nq, cs));
        if (db->prec == FS_FP8_E4M3) {
            FS_CUDA(cudaMemsetAsync(c.band_cnt, 0, sizeof(int32_t) * nq, cs));
            FS_CUDA(cudaMemsetAsync(c.class_thr, 0, sizeof(uint32_t) * nq * FS_MAX_K, cs));
        }
        t.finish((int)ceil_div(db->n_seg, 256) + 2);
    }
    if (pl.total_items > 0) {
        StageTimer t(FS_STAGE_SCAN, cs);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(pl.total_items, pl.slots)) *
                         (pl.pair ? 2 : 1);
        if (tensor_scan(db)) {
            CUtensorMap map_q;
            const int eb = db->prec == FS_BF16 ? 2 : 1;
            FS_CUDA(make_code_map(&map_q, c.q_lowp, round_up(nq, kTcQueryRows), db->fl, eb,
                                  kTcQueryRows));
            FS_CUDA(launch_scan_tc(v, c, map_q, pl.pair ? db->map_x_half : db->map_x, grid,
                                   pl.list_t, pl.pair, cs));
        } else {
            FS_CUDA(launch_scan_fp32(v, c, grid, cs));
        }
        t.finish(1);
    }
    {
        StageTimer t(FS_STAGE_SELECT, cs);
        FS_CUDA(launch_select(v, c, db->num_sms, cs));
        t.finish(1);
    }
    {
        StageTimer t(FS_STAGE_FALLBACK, cs);
        FS_CUDA(launch_fallback(v, c, db->num_sms, cs));
        t.finish(4);
    }
    if (gather) {
        StageTimer t(FS_STAGE_GATHER, cs);
        FS_CUDA(launch_gather(v, c, seq_out, seq_len, l_max, dup_of, cs));
        t.finish(1);
    }
    return FS_OK;
}

}  // namespace

namespace fsk {
fs_status search_scratch_bytes(const fs_db* db, int32_t nq, const int32_t* q_seg_off,
                               const int32_t* k, size_t* bytes) {
    if (!db || !bytes) return fail(FS_EINVAL, "db and bytes must be non-NULL");
    if (nq < 0) return fail(FS_EINVAL, "nq=%d is negative", nq);
    Plan pl;
    fs_status st = make_plan(db, nq, q_seg_off, k, pl);
    if (st != FS_OK) return st;
    *bytes = make_layout(db, nq, pl).total;
    return FS_OK;
}

fs_status set_error(fs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}
}  // namespace fsk

extern "C" {

const char* fs_last_error(void) { return g_err.c_str(); }

fs_status fs_normalize(const float* x, int64_t n, int32_t f, int64_t ld, float* x_unit,
                       float* inv_norm, void* stream) {
    if (n < 0) return fail(FS_EINVAL, "n=%lld is negative", (long long)n);
    if (f < 1 || f > FS_MAX_F) return fail(FS_EINVAL, "f=%d is outside 1..%d", f, FS_MAX_F);
    if (ld < f) return fail(FS_EINVAL, "ld=%lld is smaller than f=%d", (long long)ld, f);
    if (n > 0 && (!x || !x_unit)) return fail(FS_EINVAL, "x and x_unit must be non-NULL");
    FS_CUDA(launch_normalize_public(x, n, f, ld, x_unit, inv_norm, (cudaStream_t)stream));
    return FS_OK;
}

fs_status fs_build_db(const float* x, int64_t n, int32_t f, const int64_t* seq_off,
                      const int16_t* seq_ids, const int64_t* seg_off, int32_t n_seg,
                      fs_precision prec, void* stream, fs_db** out) {
    if (!out) return fail(FS_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 0 || n > (int64_t)INT32_MAX)
        return fail(FS_EINVAL, "n=%lld is outside 0..2^31-1", (long long)n);
    if (prec != FS_FP32 && prec != FS_BF16 && prec != FS_FP8_E4M3)
        return fail(FS_EINVAL, "unknown precision %d", (int)prec);
    const int fmax = prec == FS_FP32 ? FS_MAX_F : FS_MAX_F_TC;
    if (f < 1 || f > fmax) return fail(FS_EINVAL, "f=%d is outside 1..%d for this precision", f, fmax);
    if (n > 0 && (!x || !seq_off)) return fail(FS_EINVAL, "x and seq_off must be non-NULL");
    if (!seq_off) return fail(FS_EINVAL, "seq_off must be non-NULL");
    std::vector<int64_t> segs;
    if (seg_off) {
        if (n_seg < 1 || n_seg > FS_MAX_SEGMENTS)
            return fail(FS_EINVAL, "n_seg=%d is outside 1..%d", n_seg, FS_MAX_SEGMENTS);
        segs.assign(seg_off, seg_off + n_seg + 1);
        if (segs[0] != 0 || segs[n_seg] != n)
            return fail(FS_EINVAL, "seg_off must start at 0 and end at n=%lld", (long long)n);
        for (int s = 0; s < n_seg; ++s)
            if (segs[s + 1] < segs[s])
                return fail(FS_EINVAL, "seg_off must be non-decreasing (segment %d)", s);
    } else {
        if (n_seg != 1 && n_seg != 0)
            return fail(FS_EINVAL, "n_seg=%d given without seg_off", n_seg);
        n_seg = 1;
        segs = {0, n};
    }

    fs_db* db = new fs_db();
    cudaStream_t cs = (cudaStream_t)stream;
    fs_status st = FS_OK;
#define FS_TRY(expr)                   \
    do {                               \
        st = (expr);                   \
        if (st != FS_OK) {             \
            free_db(db);               \
            return st;                 \
        }                              \
    } while (0)
#define FS_TRY_CUDA(call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            free_db(db);                                                                    \
            return fail(FS_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));          \
        }                                                                                   \
    } while (0)

    FS_TRY_CUDA(cudaGetDevice(&db->dev));
    FS_TRY_CUDA(cudaDeviceGetAttribute(&db->num_sms, cudaDevAttrMultiProcessorCount, db->dev));
    {
        int l2 = 0;
        FS_TRY_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, db->dev));
        db->l2_bytes = l2;
    }
    db->n = n;
    db->f = f;
    db->fu = (int)round_up(f, 32);
    db->fl = lowp_width(f, prec);
    db->prec = prec;
    db->n_seg = n_seg;
    db->seg_off = segs;

    FS_TRY(alloc((void**)&db->status, sizeof(uint32_t), "status"));
    FS_TRY(alloc((void**)&db->stats, sizeof(unsigned long long) * kNumStats, "stats"));
    FS_TRY_CUDA(cudaMemsetAsync(db->status, 0, sizeof(uint32_t), cs));
    FS_TRY_CUDA(cudaMemsetAsync(db->stats, 0, sizeof(unsigned long long) * kNumStats, cs));

    // the phase orders: read the total length, then copy and check the CSR
    int64_t total = 0;
    if (n > 0) FS_TRY_CUDA(cudaMemcpyAsync(&total, seq_off + n, sizeof(int64_t),
                                           cudaMemcpyDeviceToHost, cs));
    FS_TRY_CUDA(cudaStreamSynchronize(cs));
    if (total < 0 || (total > 0 && !seq_ids)) {
        free_db(db);
        return fail(FS_EINVAL, "seq_off[n]=%lld needs non-NULL seq_ids", (long long)total);
    }
    db->seq_total = total;
    FS_TRY(alloc((void**)&db->seq_off, sizeof(int64_t) * (n + 1), "seq_off"));
    FS_TRY(alloc((void**)&db->seq_ids, sizeof(int16_t) * std::max<int64_t>(total, 1), "seq_ids"));
    if (n > 0) {
        FS_TRY_CUDA(cudaMemcpyAsync(db->seq_off, seq_off, sizeof(int64_t) * (n + 1),
                                    cudaMemcpyDeviceToDevice, cs));
    } else {
        FS_TRY_CUDA(cudaMemsetAsync(db->seq_off, 0, sizeof(int64_t), cs));
    }
    if (total > 0)
        FS_TRY_CUDA(cudaMemcpyAsync(db->seq_ids, seq_ids, sizeof(int16_t) * total,
                                    cudaMemcpyDeviceToDevice, cs));
    if (n > 0) FS_TRY_CUDA(launch_check_sequences(db->seq_off, db->seq_ids, n, total, db->status, cs));

    // the feature vectors
    FS_TRY(alloc((void**)&db->raw, sizeof(float) * n * f, "raw features"));
    FS_TRY(alloc((void**)&db->unit, sizeof(float) * n * db->fu, "unit vectors"));
    FS_TRY(alloc((void**)&db->b64, sizeof(double) * n, "binary64 norms"));
    FS_TRY(alloc((void**)&db->resid, sizeof(float) * n, "residuals"));
    if (prec != FS_FP32) {
        // whole 256-row tiles, so every TMA box lies inside the array; the
        // padding rows stay zero
        const int eb = prec == FS_BF16 ? 2 : 1;
        db->n_pad = round_up(std::max<int64_t>(n, 1), kTcTileRows);
        FS_TRY(alloc(&db->lowp, eb * (size_t)db->n_pad * db->fl, "codes"));
        FS_TRY_CUDA(cudaMemsetAsync(db->lowp, 0, eb * (size_t)db->n_pad * db->fl, cs));
        FS_TRY_CUDA(make_code_map(&db->map_x, db->lowp, db->n_pad, db->fl, eb, kTcTileRows));
        FS_TRY_CUDA(
            make_code_map(&db->map_x_half, db->lowp, db->n_pad, db->fl, eb, kTcTileRows / 2));
    }
    if (prec == FS_FP8_E4M3) FS_TRY(alloc((void**)&db->scale, sizeof(float) * n, "scales"));
    if (n > 0) {
        FS_TRY_CUDA(cudaMemcpyAsync(db->raw, x, sizeof(float) * n * f, cudaMemcpyDeviceToDevice, cs));
        FS_TRY_CUDA(cudaMemsetAsync(db->resid, 0, sizeof(float) * n, cs));
    }
    FS_TRY_CUDA(launch_prepare_rows(db->raw, n, f, db->unit, db->fu, nullptr, db->lowp, db->fl,
                                    db->scale, db->resid, prec, db->status, cs));
    FS_TRY_CUDA(launch_norm64_rows(db->raw, n, f, db->b64, cs));

    // per-segment largest residual (bounds of the low-precision scans)
    FS_TRY(alloc((void**)&db->seg_off_dev, sizeof(int64_t) * (n_seg + 1), "segments"));
    FS_TRY(alloc((void**)&db->r_max_dev, sizeof(float) * n_seg, "segment residuals"));
    FS_TRY_CUDA(cudaMemcpyAsync(db->seg_off_dev, segs.data(), sizeof(int64_t) * (n_seg + 1),
                                cudaMemcpyHostToDevice, cs));
    FS_TRY_CUDA(launch_segment_max(db->resid, db->seg_off_dev, n_seg, db->r_max_dev, cs));
    db->r_max.assign(n_seg, 0.0f);
    FS_TRY_CUDA(cudaMemcpyAsync(db->r_max.data(), db->r_max_dev, sizeof(float) * n_seg,
                                cudaMemcpyDeviceToHost, cs));
    uint32_t status = 0;
    FS_TRY_CUDA(cudaMemcpyAsync(&status, db->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, cs));
    FS_TRY_CUDA(cudaStreamSynchronize(cs));
    if (status & kStBadFeature) {
        free_db(db);
        return fail(FS_EINVAL, "a feature is non-finite or outside [2^-40, 2^50] in magnitude");
    }
    if (status & kStBadSequence) {
        free_db(db);
        return fail(FS_EINVAL, "seq_off is not a valid CSR offset array or a pass ID is negative");
    }
#undef FS_TRY
#undef FS_TRY_CUDA
    *out = db;
    return FS_OK;
}

fs_status fs_db_set_metric(fs_db* db, fs_metric metric, void* stream) {
    if (!db) return fail(FS_EINVAL, "db is NULL");
    if (metric != FS_COSINE && metric != FS_EUCLIDEAN && metric != FS_MANHATTAN)
        return fail(FS_EINVAL, "metric %d is not a fs_metric", (int)metric);
    fs_status st = check_device(db);
    if (st != FS_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    if (metric == FS_COSINE) {
        if (db->metric != FS_COSINE)   // the unit vectors again
            FS_CUDA(launch_prepare_rows(db->raw, db->n, db->f, db->unit, db->fu, nullptr,
                                        db->lowp, db->fl, db->scale, db->resid, db->prec,
                                        db->status, cs));
        FS_CUDA(cudaStreamSynchronize(cs));
        db->metric = FS_COSINE;
        return FS_OK;
    }
    if (db->prec != FS_FP32)
        return fail(FS_EUNSUPPORTED, "the standardised metrics need an FS_FP32 database");
    const size_t stats = (size_t)db->n_seg * db->f;
    if (!db->mu) {
        st = alloc((void**)&db->mu, sizeof(double) * stats, "feature means");
        if (st == FS_OK) st = alloc((void**)&db->sg, sizeof(double) * stats, "feature deviations");
        if (st == FS_OK) st = alloc((void**)&db->row_term, sizeof(float) * db->n, "row terms");
        if (st == FS_OK) st = alloc((void**)&db->row_mag, sizeof(float) * db->n, "row magnitudes");
        if (st == FS_OK)
            st = alloc((void**)&db->mag_max_dev, sizeof(float) * db->n_seg, "segment magnitudes");
        if (st != FS_OK) return st;
    }
    FS_CUDA(launch_seg_stats(db->raw, db->seg_off_dev, db->n_seg, db->f, db->mu, db->sg, cs));
    FS_CUDA(launch_std_rows(db->raw, db->n, db->f, db->fu, db->seg_off_dev, db->n_seg, db->mu,
                            db->sg, (int)metric, db->unit, db->row_term, db->row_mag, cs));
    FS_CUDA(launch_segment_max(db->row_mag, db->seg_off_dev, db->n_seg, db->mag_max_dev, cs));
    db->mag_max.assign(db->n_seg, 0.0f);
    FS_CUDA(cudaMemcpyAsync(db->mag_max.data(), db->mag_max_dev, sizeof(float) * db->n_seg,
                            cudaMemcpyDeviceToHost, cs));
    FS_CUDA(cudaStreamSynchronize(cs));
    db->metric = metric;
    return FS_OK;
}

fs_status fs_db_set_tuning(fs_db* db, const fs_tuning* t) {
    if (!db) return fail(FS_EINVAL, "db is NULL");
    if (!t) {
        db->tune = fs_tuning{0, 0, 0, 0};
        return FS_OK;
    }
    if (t->items_per_block < 0 || t->items_per_block > 64)
        return fail(FS_EINVAL, "items_per_block=%d is outside 0..64", t->items_per_block);
    if (t->list_len != 0 && t->list_len != kListTTiny && t->list_len != kListTSmall &&
        t->list_len != kListT)
        return fail(FS_EINVAL, "list_len=%d is not 0, %d, %d or %d", t->list_len, kListTTiny,
                    kListTSmall, kListT);
    if (t->l2_share_pct < -1 || t->l2_share_pct > 100)
        return fail(FS_EINVAL, "l2_share_pct=%d is outside -1..100", t->l2_share_pct);
    if (t->scan_pairs < -1 || t->scan_pairs > 1)
        return fail(FS_EINVAL, "scan_pairs=%d is outside -1..1", t->scan_pairs);
    db->tune = *t;
    return FS_OK;
}

fs_status fs_db_set_wait_test(fs_db* db, int32_t withhold_first_load, uint32_t wait_limit_us) {
    if (!db) return fail(FS_EINVAL, "db is NULL");
    if (wait_limit_us > 2000000u)
        return fail(FS_EINVAL, "wait_limit_us=%u is above 2,000,000", wait_limit_us);
    db->withhold_load = withhold_first_load != 0;
    db->wait_ns = (uint64_t)wait_limit_us * 1000ull;
    return FS_OK;
}

fs_status fs_db_get_tuning(const fs_db* db, fs_tuning* out) {
    if (!db || !out) return fail(FS_EINVAL, "db and out must be non-NULL");
    *out = db->tune;
    return FS_OK;
}

fs_status fs_workspace_size(const fs_db* db, int32_t nq, const int32_t* q_seg_off, size_t* bytes) {
    if (!db || !bytes) return fail(FS_EINVAL, "db and bytes must be non-NULL");
    if (nq < 0) return fail(FS_EINVAL, "nq=%d is negative", nq);
    std::vector<int32_t> kk(db->n_seg, 1);
    Plan pl;
    fs_status st = make_plan(db, nq, q_seg_off, kk.data(), pl, 1);
    if (st != FS_OK) return st;
    *bytes = make_layout(db, nq, pl).total;
    return FS_OK;
}

fs_status fs_knn(const fs_db* db, const float* q, int32_t nq, const int32_t* q_seg_off,
                 const int32_t* k, const int32_t* exclude, void* workspace, size_t workspace_bytes,
                 int32_t* idx, float* dist, void* stream) {
    return search(db, q, nq, q_seg_off, k, exclude, workspace, workspace_bytes, idx, dist, nullptr,
                  nullptr, 0, nullptr, false, stream);
}

fs_status fs_recommend(const fs_db* db, const float* q, int32_t nq, const int32_t* q_seg_off,
                       const int32_t* k, const int32_t* exclude, void* workspace,
                       size_t workspace_bytes, int32_t* idx, float* dist, int16_t* seq_out,
                       int32_t* seq_len, int32_t l_max, int32_t* dup_of, void* stream) {
    return search(db, q, nq, q_seg_off, k, exclude, workspace, workspace_bytes, idx, dist, seq_out,
                  seq_len, l_max, dup_of, true, stream);
}

fs_status fs_db_destroy(fs_db* db) {
    if (!db) return fail(FS_EINVAL, "db is NULL");
    cudaDeviceSynchronize();
    free_db(db);
    return FS_OK;
}

fs_status fs_db_check(fs_db* db, void* stream) {
    if (!db) return fail(FS_EINVAL, "db is NULL");
    cudaStream_t cs = (cudaStream_t)stream;
    uint32_t status = 0;
    FS_CUDA(cudaStreamSynchronize(cs));
    FS_CUDA(cudaMemcpy(&status, db->status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    FS_CUDA(cudaMemset(db->status, 0, sizeof(uint32_t)));
    if (status & kStTimeout) return fail(FS_ETIMEOUT, "a bounded device-side wait gave up");
    if (status & kStBadFeature)
        return fail(FS_EINVAL, "a query feature was non-finite or out of range (treated as zero)");
    if (status & kStOverflow) return fail(FS_ENOMEM, "an internal candidate list overflowed");
    if (status & kStBadSequence) return fail(FS_EINVAL, "malformed phase-order CSR");
    return FS_OK;
}

fs_status fs_profile_enable(int32_t on) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.on = on != 0;
    return FS_OK;
}

fs_status fs_profile_read(int32_t reset, fs_profile* out) {
    if (!out) return fail(FS_EINVAL, "out is NULL");
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    for (const auto& r : p.pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(r.b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            p.ms[r.stage] += ms;
            p.calls[r.stage] += 1;
        }
        p.pool.push_back(r.a);
        p.pool.push_back(r.b);
    }
    p.pending.clear();
    for (int i = 0; i < FS_NUM_STAGES; ++i) {
        out->ms[i] = p.ms[i];
        out->calls[i] = p.calls[i];
    }
    out->launches = p.launches.load();
    if (reset) {
        for (int i = 0; i < FS_NUM_STAGES; ++i) {
            p.ms[i] = 0.0;
            p.calls[i] = 0;
        }
        p.launches = 0;
    }
    return FS_OK;
}

fs_status fs_db_stats(fs_db* db, void* stream, int32_t reset, fs_stats* out) {
    if (!db || !out) return fail(FS_EINVAL, "db and out must be non-NULL");
    unsigned long long v[kNumStats];
    FS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    FS_CUDA(cudaMemcpy(v, db->stats, sizeof(v), cudaMemcpyDeviceToHost));
    if (reset) FS_CUDA(cudaMemset(db->stats, 0, sizeof(v)));
    out->queries = v[kStatQueries];
    out->certified = v[kStatCertified];
    out->fallback = v[kStatFallback];
    out->fp64_evals = v[kStatFp64];
    out->near_ties = v[kStatNearTies];
    out->rerank_evals = v[kStatRerank];
    out->band_rows = v[kStatBand];
    return FS_OK;
}

}  // extern "C"
