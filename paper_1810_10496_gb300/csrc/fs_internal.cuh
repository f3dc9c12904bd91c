// Internal definitions shared by the kernels and the C-ABI layer.
//
// Ordering keys. Every candidate list orders (score, index) pairs by score
// descending and index ascending (the tie rule of the result contract). A
// pair is packed into one 64-bit key whose unsigned order is that order:
// the high word is the float score mapped to an order-preserving unsigned
// integer, the low word is (2^32 - 1 - index). Key 0 marks an empty slot
// (it decodes to index -1 and sorts below every real score).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fs.h"

namespace fsk {

constexpr int kWarp = 32;
constexpr int kListT = 16;        // largest candidate list (>= FS_MAX_K)
constexpr int kListTSmall = 8;    // list size when every k <= 8
constexpr int kListTTiny = 4;     // list size when every k <= 4 (a tuning choice)
constexpr int kWindow = 64;       // candidates the rerank takes per query
constexpr int kQTile = 128;       // queries per scan work item
constexpr int kFbChunks = 32;     // row chunks per query in the exact fallback
// Devices whose kernel attributes are cached (cudaFuncSetAttribute acts on
// the current device's context only, so every cache of it is per device;
// a device beyond this count sets its attributes on every launch).
constexpr int kMaxDevices = 64;

// device status bits (fs_db::status)
constexpr uint32_t kStBadFeature = 1u;     // non-finite / out-of-range value
constexpr uint32_t kStTimeout = 2u;        // a bounded wait gave up
constexpr uint32_t kStOverflow = 4u;       // an internal list overflowed
constexpr uint32_t kStBadSequence = 8u;    // malformed phase-order CSR

// statistics slots (fs_db::stats), same order as fs_stats
enum { kStatQueries = 0, kStatCertified, kStatFallback, kStatFp64, kStatNearTies,
       kStatRerank, kStatBand, kNumStats };

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) {
    return (a + b - 1) / b;
}
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) {
    return ceil_div(a, b) * b;
}

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t ord_f32(float s) {
    uint32_t u = __float_as_uint(s + 0.0f);  // -0 becomes +0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_f32(uint32_t o) {
    uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    return __uint_as_float(u);
}
__device__ __forceinline__ uint64_t make_key(float s, uint32_t idx) {
    return ((uint64_t)ord_f32(s) << 32) | (uint64_t)(0xffffffffu - idx);
}
__device__ __forceinline__ float key_score(uint64_t key) {
    return unord_f32((uint32_t)(key >> 32));
}
__device__ __forceinline__ int32_t key_index(uint64_t key) {
    return (int32_t)(0xffffffffu - (uint32_t)key);
}

// One thread's candidate list, held in registers: its LT best scores in
// descending order with their segment-local rows (-inf while filling; every
// index is a compile-time constant, so the arrays never leave the register
// file). A candidate is inserted by one compare-exchange pass over 32-bit
// scores; the lowest kept score is always the last. A score equal to the
// lowest kept one is not inserted: rows arrive in increasing order, so the
// earlier, lower row stays. The 64-bit keys of the merge are formed on output.
template <int LT>
struct RegList {
    float s[LT];
    uint32_t r[LT];
    float thr_s;       // lowest kept score once the list is full; -inf before
    int cnt;           // entries stored so far (at most LT)

    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int e = 0; e < LT; ++e) {
            s[e] = -INFINITY;
            r[e] = 0;
        }
        thr_s = -INFINITY;
        cnt = 0;
    }

    // Score of the kk-th best entry held (1 <= kk <= cnt): the least of the
    // first kk, taken as a minimum so that no index is computed at run time.
    __device__ __forceinline__ float kth_score(int kk) const {
        float t = INFINITY;
#pragma unroll
        for (int e = 0; e < LT; ++e)
            if (e < kk) t = fminf(t, s[e]);
        return t;
    }

    // The merge key of entry e (0 for an empty entry).
    __device__ __forceinline__ uint64_t key(int e) const {
        return cnt > e ? make_key(s[e], r[e]) : 0ull;
    }

    // Offers (score, row): kept if the list is filling or it beats the lowest.
    __device__ __forceinline__ void offer(float v, int64_t row, int64_t row_end, int64_t row0,
                                          int excl) {
        const int32_t li = (int32_t)(row - row0);
        if (row >= row_end || li == excl) return;
        if (!(v > thr_s)) return;
        float x = v;
        uint32_t xi = (uint32_t)li;
#pragma unroll
        for (int e = 0; e < LT; ++e) {
            const float a = s[e];
            const uint32_t ai = r[e];
            const bool up = x > a;
            s[e] = up ? x : a;
            r[e] = up ? xi : ai;
            x = up ? a : x;
            xi = up ? ai : xi;
        }
        cnt += cnt < LT ? 1 : 0;
        if (cnt == LT) thr_s = s[LT - 1];
    }
};
#endif

// Per-segment facts of one search call, computed on the host and written to
// the workspace by a small kernel (so a call can be captured in a graph).
struct SegPlan {
    int64_t row0;        // first database row of the segment
    int64_t nrows;       // rows in the segment
    int64_t item0;       // first scan work item of the segment
    int64_t cand0;       // first candidate-list entry of the segment
    int32_t q0;          // first query of the segment
    int32_t nq;          // queries of the segment
    int32_t k;           // neighbours requested
    int32_t qtiles;      // ceil(nq / kQTile)
    int32_t chunks;      // row chunks the scan splits the segment into
    int32_t chunk_rows;  // rows per chunk (a multiple of the scan tile)
    int32_t lists;       // candidate lists per (query, chunk)
    int32_t list_t;      // entries per candidate list (8 or 16)
    float bound_scan;    // |approximate score - exact cosine| <= bound_scan
    float bound_rq;      //   + bound_rq * (query residual norm), per query
    float bound_rerank;  // same bound for the FP32 rescoring of the window
    int32_t units;       // scan units per row chunk: query tiles, or pairs of them
    int32_t seg;         // index of the segment in the database
    float mag_max;       // standardised metrics: the segment's largest row magnitude
                         // (Euclidean |z|, Manhattan sum |z_i|), for the score bound
    int64_t band0;       // FP8: first band-buffer entry of the segment
    int32_t band_cap;    // FP8: band-buffer entries per query
    float bound_rx;      // FP8: per-row bound E = a + (bound_rx + r_q) * 1.001 * r_x,
                         //   a = bound_scan + bound_rq * r_q (r: residual norms)
};
static_assert(sizeof(SegPlan) == 104, "SegPlan layout");

// Read-only device view of a database and of one call's workspace.
struct DbView {
    const float* raw;        // [n][f] features as given (binary64 scoring)
    const float* unit;       // [n][fu] FP32 unit vectors, zero padded
    const double* b64;       // [n] sum of squares, binary64, sequential
    const void* lowp;        // [n][fl] BF16 or FP8 unit-vector codes
    const float* scale;      // [n] FP8 per-vector scale (NULL for BF16)
    const float* resid;      // [n] ||unit - dequantised||_2
    const int64_t* seq_off;  // [n+1]
    const int16_t* seq_ids;
    uint32_t* status;        // device status word
    unsigned long long* stats;
    int64_t n;
    int32_t f, fu, fl;
    int32_t prec;
    int32_t metric;          // fs_metric; for the standardised metrics `unit` holds the
                             // standardised rows z (FP32), zero padded
    const double* mu;        // [n_seg][f] per-segment feature means (standardised metrics)
    const double* sg;        // [n_seg][f] per-segment population deviations
    const float* row_term;   // [n] Euclidean: 1/2 |z_x|^2 (FP32 of the binary64 value)
    const float* row_mag;    // [n] |z_x| (Euclidean) or sum |z_x,i| (Manhattan), rounded up
};

struct CallView {
    const SegPlan* plan;      // [n_seg], in scan-item order (largest work first)
    const int32_t* q_order;   // [n_seg] plan indices sorted by first query
    const int32_t* q_plan;    // [nq] plan index of each query's segment
    const float* q_raw;       // [nq][f] caller's queries
    double* q_a64;            // [nq] binary64 sum of squares (queries sent to the fallback)
    float* q_ss;              // [nq] FP32 sum of squares (0 exactly for a zero query)
    float* q_unit;            // [nq][fu]
    void* q_lowp;             // [nq][fl]
    float* q_scale;           // [nq]
    float* q_resid;           // [nq]
    uint64_t* cand;           // candidate lists (BF16 / FP32 scans)
    uint64_t* band;           // FP8 scan: per query, the keys of every row whose score's
                              // upper bound reached the running k-th best lower bound
    int32_t* band_cnt;        // [nq] rows appended to each query's band (may exceed the
                              // capacity: then the query goes to the exact fallback)
    int32_t* fb_count;        // queries sent to the FP32 rescan (fb_count[1] is the
                              // scan scheduler, fb_count[2] is fb2_count, fb_count[3]
                              // is `aborted`, fb_count[4] the selection's counter)
    int32_t* fb_list;         // [nq]
    int32_t* fb2_count;       // queries sent on to the binary64 scan
    int32_t* fb2_list;        // [nq]
    uint64_t* cand_fb;        // [nq][kFbChunks][kListT] lists of the FP32 rescan
    double* fb_score;         // [nq][kFbChunks][FS_MAX_K]
    int32_t* fb_index;        // [nq][kFbChunks][FS_MAX_K]
    int32_t* work_counter;    // dynamic scan scheduler
    int32_t* sel_counter;     // the selection's next query (persistent warps)
    int32_t* aborted;         // nonzero once a bounded wait of this call's scan gave up:
                              // its candidate lists are incomplete, so the selection
                              // writes padding instead of reading them
    uint64_t wait_ns;         // limit of every bounded wait of the scan (0: kWaitLimitNs)
    int32_t withhold_load;    // test aid: every scan block skips its first row-tile load
    uint32_t* shared_thr;     // [nq] per query: a score below which no row can be
                              // among the k nearest (order-mapped bits)
    uint32_t* class_thr;      // FP8: [nq][FS_MAX_K] per query and row class (k classes, a
                              // fixed hash of the local row):
                              // the best lower bound of a band row of the class
    const int32_t* exclude;   // [nq] or NULL
    int32_t* out_idx;         // [nq][k_max]
    float* out_dist;          // [nq][k_max]
    int32_t nq;
    int32_t n_seg;
    int32_t k_max;
    int64_t total_items;
};

// ---------------------------------------------------------------------------
// launchers (host functions defined in the kernel translation units)

// normalize.cu
cudaError_t launch_normalize_public(const float* x, int64_t n, int f, int64_t ld,
                                    float* x_unit, float* inv_norm, cudaStream_t st);
cudaError_t launch_prepare_rows(const float* x, int64_t n, int f, float* unit, int fu,
                                float* ss_out, void* lowp, int fl, float* scale,
                                float* resid, int prec, uint32_t* status, cudaStream_t st);
cudaError_t launch_norm64_rows(const float* x, int64_t n, int f, double* b64, cudaStream_t st);
cudaError_t launch_check_sequences(const int64_t* off, const int16_t* ids, int64_t n,
                                   int64_t total, uint32_t* status, cudaStream_t st);
cudaError_t launch_segment_max(const float* v, const int64_t* seg_off_dev, int n_seg,
                               float* out, cudaStream_t st);

// select.cu
cudaError_t launch_write_plan(const SegPlan* host_plan, const int32_t* host_q_order, int n_seg,
                              SegPlan* dev_plan, int32_t* dev_q_order, int32_t* fb_count,
                              int32_t* work_counter, cudaStream_t st);
cudaError_t launch_query_plan(const CallView& call, int32_t* q_plan, cudaStream_t st);
cudaError_t launch_select(const DbView& db, const CallView& call, int num_sms, cudaStream_t st);
cudaError_t launch_fallback(const DbView& db, const CallView& call, int num_sms,
                            cudaStream_t st);
cudaError_t launch_gather(const DbView& db, const CallView& call, int16_t* seq_out,
                          int32_t* seq_len, int l_max, int32_t* dup_of, cudaStream_t st);

// fs_api.cu: records the message fs_last_error() returns on this thread
fs_status set_error(fs_status st, const char* fmt, ...);
// fs_api.cu: the workspace bytes one search call with exactly these
// arguments uses (fs_workspace_size sizes for any k, so it can be larger)
fs_status search_scratch_bytes(const fs_db* db, int32_t nq, const int32_t* q_seg_off,
                               const int32_t* k, size_t* bytes);

// scan_fp32.cu
constexpr int kFp32TileRows = 128;
constexpr int kFp32Lists = 2;
cudaError_t launch_scan_fp32(const DbView& db, const CallView& call, int grid,
                             cudaStream_t st);
int scan_fp32_ctas_per_sm();

// metric.cu (standardised Euclidean and Manhattan distances)
cudaError_t launch_seg_stats(const float* raw, const int64_t* seg_off_dev, int n_seg, int f,
                             double* mu, double* sg, cudaStream_t st);
cudaError_t launch_std_rows(const float* raw, int64_t n, int f, int fu, const int64_t* seg_off,
                            int n_seg, const double* mu, const double* sg, int metric,
                            float* z, float* row_term, float* row_mag, cudaStream_t st);
cudaError_t launch_std_queries(const DbView& db, const CallView& call, cudaStream_t st);
__host__ __device__ constexpr bool is_std_metric(int metric) { return metric != FS_COSINE; }

// scan_tc.cu (tcgen05 scan of BF16 / FP8 codes)
constexpr int kTcTileRows = 256;
constexpr int kTcQueryRows = 128;
constexpr int kTcLists = 2;        // candidate lists per (query, chunk): tile halves
size_t scan_tc_smem_bytes(int kblocks, int stages, bool pair);
int scan_tc_stages(int kblocks, bool fp8, bool pair);
int scan_tc_pair_slots(bool fp8, int kblocks);
cudaError_t make_code_map(CUtensorMap* map, const void* ptr, int64_t rows, int cols,
                          int elem_bytes, int box_rows);
// pair: clusters of two CTAs (cta_group::2); grid is then even and map_x's
// box is half a tile (kTcTileRows / 2 rows)
cudaError_t launch_scan_tc(const DbView& db, const CallView& call, const CUtensorMap& map_q,
                           const CUtensorMap& map_x, int grid, int list_t, bool pair,
                           cudaStream_t st);

}  // namespace fsk
