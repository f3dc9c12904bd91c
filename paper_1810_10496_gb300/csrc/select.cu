// Selection: from the scan's candidate lists to the exact k nearest rows, and
// the gather of their phase orders.
//
// Sec. 4 keeps the K reference kernels most similar to the new kernel and
// suggests their phase orders (Table 1). The scans only approximate the
// cosine (FP32 rounding, or BF16/FP8 codes), so this layer turns their
// candidates into the exact binary64 ranking of the result contract:
//
//  1. Per query, merge the lists of every row chunk and find the k-th best
//     approximate score t_k.
//  2. Certify: every approximate score is within E of the true cosine. A
//     list that filled up dropped rows scoring at most its lowest kept score
//     tau; if tau + 2E < t_k for every full list, no dropped row can be among
//     the k nearest. (The tensor-core scan also drops rows scoring below a
//     shared bound, the k-th best score seen minus 2E: such a row is provably
//     not among the k nearest, so it needs no certificate.) Otherwise the
//     query goes to the exact fallback scan.
//  3. Window: only candidates with approximate score >= t_k - 2E can be in
//     the top k (at most 64 are taken; more also sends the query to the
//     fallback).
//  4. Rescore the window in FP32 from the unit vectors, with a warp-wide
//     summation whose error bound E_r is small, and compute the distance as
//     1/2 |u_q - u_x|^2, which has no cancellation near 0.
//  5. Sort the window by rescored value. Neighbours closer than 2 E_r may be
//     out of order; runs of such near ties that reach into the first k
//     places are scored with the binary64 formula (sequential sums, no fused
//     multiply-add) and reordered by (score desc, index asc). Everything
//     else is already in its exact place, because its rescored gaps exceed
//     the error of both neighbours.
#include <algorithm>
#include <mutex>

#include "fs_internal.cuh"

namespace fsk {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPlanPerLaunch = 256;

struct PlanChunk {
    SegPlan p[kPlanPerLaunch];
    int32_t q_order[kPlanPerLaunch];
};

__global__ void k_write_plan(PlanChunk chunk, int n, SegPlan* dst, int32_t* dst_q_order,
                             int32_t* fb_count, int32_t* work_counter) {
    int i = threadIdx.x;
    if (i < n) {
        dst[i] = chunk.p[i];
        dst_q_order[i] = chunk.q_order[i];
    }
    if (i == 0 && fb_count) {
        fb_count[0] = 0;    // queries for the FP32 rescan
        fb_count[2] = 0;    // queries for the binary64 scan
        fb_count[3] = 0;    // the scan has not given up
        fb_count[4] = 0;    // the selection's next query
        *work_counter = 0;
    }
}

// q_plan[q] = the plan entry of the segment that owns query q: block b
// writes entry b's queries (segments partition the queries in order).
__global__ void k_query_plan(const SegPlan* __restrict__ plan, int32_t* __restrict__ q_plan) {
    const int b = blockIdx.x;
    const int q0 = plan[b].q0, nq = plan[b].nq;
    for (int i = threadIdx.x; i < nq; i += blockDim.x) q_plan[q0 + i] = b;
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t w = __shfl_xor_sync(kFull, v, o);
        v = w > v ? w : v;
    }
    return v;
}
__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t w = __shfl_xor_sync(kFull, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// (s1, i1) ranks before (s2, i2): score descending, index ascending
__device__ __forceinline__ bool better(double s1, int i1, double s2, int i2) {
    return s1 > s2 || (s1 == s2 && i1 < i2);
}

// Warp-wide best (score, index) pair; invalid entries carry index -1 and
// score -inf and lose to every valid one.
__device__ __forceinline__ void warp_best(double& s, int& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double s2 = __shfl_xor_sync(kFull, s, o);
        int i2 = __shfl_xor_sync(kFull, i, o);
        bool take = (i < 0) ? (i2 >= 0) : (i2 >= 0 && better(s2, i2, s, i));
        if (take) { s = s2; i = i2; }
    }
}

// binary64 cosine of the result contract: sums in order, no fused multiply-add
__device__ double exact_cosine(const float* __restrict__ q, const float* __restrict__ x, int f,
                               double a, double b) {
    double d = 0.0;
    for (int i = 0; i < f; ++i) d = __dadd_rn(d, __dmul_rn((double)q[i], (double)x[i]));
    if (a == 0.0 || b == 0.0) return 0.0;
    double s = __ddiv_rn(d, __dsqrt_rn(__dmul_rn(a, b)));
    return s + 0.0;  // -0 becomes +0
}

// Standardised metrics: the binary64 distance of the oracle, z = (v - mu) /
// sigma (0 where sigma = 0) for both vectors, then the sequential sum of
// squares (Euclidean, then the square root) or of magnitudes (Manhattan),
// every operation rounded to nearest, no fused multiply-add.
__device__ double exact_std_distance(const DbView& db, const SegPlan& p,
                                     const float* __restrict__ q, const float* __restrict__ x) {
    const double* m = db.mu + (int64_t)p.seg * db.f;
    const double* s = db.sg + (int64_t)p.seg * db.f;
    double acc = 0.0;
    for (int i = 0; i < db.f; ++i) {
        const double zq = s[i] > 0.0 ? __ddiv_rn(__dsub_rn((double)q[i], m[i]), s[i]) : 0.0;
        const double zx = s[i] > 0.0 ? __ddiv_rn(__dsub_rn((double)x[i], m[i]), s[i]) : 0.0;
        const double t = __dsub_rn(zq, zx);
        acc = db.metric == FS_EUCLIDEAN ? __dadd_rn(acc, __dmul_rn(t, t)) : __dadd_rn(acc, fabs(t));
    }
    return db.metric == FS_EUCLIDEAN ? __dsqrt_rn(acc) : acc;
}

__device__ __forceinline__ void write_padding(const CallView& call, int q, int from) {
    for (int c = from + (threadIdx.x & 31); c < call.k_max; c += 32) {
        call.out_idx[(int64_t)q * call.k_max + c] = -1;
        call.out_dist[(int64_t)q * call.k_max + c] = INFINITY;
    }
}

constexpr int kSelWarps = 8;
constexpr int kRescoreRows = 4;   // window rows the FP32 rescoring reads at once
constexpr int kBandRows = 4;      // band rows the FP32 rescoring reads at once
// FP32 distances below this are replaced by the binary64 one (near
// duplicates; above it the FP32 value is within 3e-6 relative)
constexpr float kExactDist = 4e-3f;

struct SelShared {
    int32_t widx[kSelWarps][kWindow];     // window rows (segment-local), scan order
    float wsc[kSelWarps][kWindow];        // their FP32 rescored cosines
    float wdist[kSelWarps][kWindow];      // their FP32 distances
    int32_t sidx[kSelWarps][kWindow];     // window sorted by (rescored desc, row asc)
    float ssc[kSelWarps][kWindow];
    float sdist[kSelWarps][kWindow];
    double s64[kSelWarps][kWindow];       // binary64 cosines of near-tie members
    uint8_t tie[kSelWarps][kWindow];      // member of a near-tie cluster
    int16_t cl_begin[kSelWarps][FS_MAX_K], cl_end[kSelWarps][FS_MAX_K];
    unsigned long long stats[kNumStats];
};

// binary64 A = sum q_i^2 and D = sum q_i x_i, sequential in i without fused
// multiply-add, then s = D / sqrt(A B) (0 for a zero vector)
__device__ double exact_cosine_ab(const float* __restrict__ q, const float* __restrict__ x, int f,
                                  double b) {
    double a = 0.0, d = 0.0;
    for (int i = 0; i < f; ++i) {
        const double qi = (double)q[i];
        a = __dadd_rn(a, __dmul_rn(qi, qi));
        d = __dadd_rn(d, __dmul_rn(qi, (double)x[i]));
    }
    if (a == 0.0 || b == 0.0) return 0.0;
    return __ddiv_rn(d, __dsqrt_rn(__dmul_rn(a, b))) + 0.0;  // -0 becomes +0
}

__device__ double exact_norm2(const float* __restrict__ q, int f) {
    double a = 0.0;
    for (int i = 0; i < f; ++i) {
        const double qi = (double)q[i];
        a = __dadd_rn(a, __dmul_rn(qi, qi));
    }
    return a;
}

// FP32 rescoring of R rows (row < 0: none) against the query's unit vector:
// the cosine u_q . u_x as a warp-wide sum (each lane sums, with FMA, the four
// consecutive features of its 128-bit load in every 128-feature block: at
// most max(fu / 32, 4 ceil(fu / 128)) terms; then a butterfly; every lane
// ends with the same bits), and with DIST also 1/2 |u_q - u_x|^2 the same way.
// The error of the cosine is within the plan's bound_rerank.
template <bool DIST, int R>
__device__ __forceinline__ void rescore_rows(const DbView& db, const float* __restrict__ qu,
                                             const int64_t (&row)[R], float (&dot)[R],
                                             float (&dd)[R], int lane) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
        dot[j] = 0.0f;
        dd[j] = 0.0f;
        if (row[j] >= 0) {
            const float* xu = db.unit + row[j] * (int64_t)db.fu;
            for (int i = 4 * lane; i < db.fu; i += 128) {
                const float4 a = *reinterpret_cast<const float4*>(qu + i);
                const float4 b = __ldg(reinterpret_cast<const float4*>(xu + i));
                dot[j] = fmaf(a.x, b.x, dot[j]);
                dot[j] = fmaf(a.y, b.y, dot[j]);
                dot[j] = fmaf(a.z, b.z, dot[j]);
                dot[j] = fmaf(a.w, b.w, dot[j]);
                if (DIST) {
                    float t = a.x - b.x;
                    dd[j] = fmaf(t, t, dd[j]);
                    t = a.y - b.y;
                    dd[j] = fmaf(t, t, dd[j]);
                    t = a.z - b.z;
                    dd[j] = fmaf(t, t, dd[j]);
                    t = a.w - b.w;
                    dd[j] = fmaf(t, t, dd[j]);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dot[j] += __shfl_xor_sync(kFull, dot[j], o);
            if (DIST) dd[j] += __shfl_xor_sync(kFull, dd[j], o);
        }
    }
}

__device__ int finish_window(const DbView& db, const CallView& call, SelShared& sh, int wid,
                             int lane, int q, const SegPlan& p, int nw, unsigned long long* stats);

// Answers query q from its candidate lists: cand holds nl lists of lt keys
// (each sorted, descending, empty entries last),
// every approximate score within E of the exact cosine. Returns the number of
// places written, or -1 when the lists do not certify the answer (nothing is
// written then). Whole warp.
__device__ int answer_from_lists(const DbView& db, const CallView& call, SelShared& sh, int wid,
                                 int lane, int q, const SegPlan& p, const uint64_t* cand, int nl,
                                 int lt, double E, unsigned long long* stats) {
    const int k = p.k;
    const int64_t out0 = (int64_t)q * call.k_max;
    const int64_t ne = (int64_t)nl * lt;

    // Every list is sorted: its keys in descending order, empty entries (0)
    // last. So the k best keys overall are among the first k of each list, a
    // full list's lowest key is its last, and the entries of a list that can
    // reach the top k form a prefix of it.
    const int kk = k < lt ? k : lt;

    // 1. k-th best approximate key (rounds after the first read L1)
    uint64_t prev = ~0ull, kth = 0;
    int ntop = 0;
    for (int r = 0; r < k; ++r) {
        uint64_t best = 0;
        for (int l = lane; l < nl; l += 32) {
            const uint64_t* L = cand + (int64_t)l * lt;
            for (int e = 0; e < kk; ++e) {
                const uint64_t v = L[e];
                if (v < prev && v > best) best = v;
            }
        }
        best = warp_max_u64(best);
        if (best == 0) break;
        prev = best;
        kth = best;
        ++ntop;
    }

    // 2. certification against the lowest kept key of every full list
    uint64_t tau = 0;
    for (int l = lane; l < nl; l += 32) {
        const uint64_t v = cand[(int64_t)l * lt + lt - 1];   // 0 unless the list is full
        tau = v > tau ? v : tau;
    }
    tau = warp_max_u64(tau);
    const double tk = ntop ? (double)key_score(kth) : -INFINITY;
    bool certified = (tau == 0) || ((double)key_score(tau) + 2.0 * E < tk);

    // 3. window of candidates that can still reach the top k: a lane per list,
    //    entry by entry until no list has one left
    int nw = 0;
    if (certified && ntop > 0) {
        // a float v satisfies v >= lo exactly when v >= lo rounded up to
        // float: the test runs in FP32 (binary64 instructions are scarce)
        const float lo = __double2float_ru(tk - 2.0 * E);
        for (int l0 = 0; l0 < nl; l0 += 32) {
            const int l = l0 + lane;
            const uint64_t* L = cand + (int64_t)l * lt;
            for (int e = 0; e < lt; ++e) {
                const uint64_t v = l < nl ? L[e] : 0;
                const bool in = v != 0 && key_score(v) >= lo;
                const unsigned m = __ballot_sync(kFull, in);
                if (m == 0) break;
                const int pos = nw + __popc(m & ((1u << lane) - 1));
                if (in && pos < kWindow) sh.widx[wid][pos] = key_index(v);
                nw += __popc(m);
            }
        }
        if (nw > kWindow) certified = false;
    }
    __syncwarp();
    if (!certified) return -1;

    if (is_std_metric(db.metric)) {
        // standardised metrics: every window row scored with the binary64
        // formula (a lane each), ranked by (distance, row); the certificate
        // holds in real arithmetic with the margin of E's 1 % inflation, far
        // above binary64 rounding
        const float* qr = call.q_raw + (int64_t)q * db.f;
        for (int w = lane; w < nw; w += 32) {
            const int64_t row = p.row0 + sh.widx[wid][w];
            sh.s64[wid][w] = -exact_std_distance(db, p, qr, db.raw + row * (int64_t)db.f);
        }
        __syncwarp();
        for (int w = lane; w < nw; w += 32) {
            const double sw = sh.s64[wid][w];
            const int rw = sh.widx[wid][w];
            int rank = 0;
            for (int v = 0; v < nw; ++v) {
                const double sv = sh.s64[wid][v];
                rank += (sv > sw) || (sv == sw && sh.widx[wid][v] < rw);
            }
            if (rank < k) {
                call.out_idx[out0 + rank] = rw;
                call.out_dist[out0 + rank] = (float)(-sw);
            }
        }
        if (lane == 0) atomicAdd(&stats[kStatFp64], (unsigned long long)nw);
        __syncwarp();
        return nw < k ? nw : k;
    }

    return finish_window(db, call, sh, wid, lane, q, p, nw, stats);
}

// Steps 4-8 for a certified window of nw <= kWindow candidates in sh.widx:
// every row that can be among the k nearest is in it. Returns the number of
// places written. Whole warp.
__device__ int finish_window(const DbView& db, const CallView& call, SelShared& sh, int wid,
                             int lane, int q, const SegPlan& p, int nw, unsigned long long* stats) {
    const int k = p.k;
    const int64_t out0 = (int64_t)q * call.k_max;
    // 4. FP32 rescoring of the window: the cosine of the unit vectors and
    //    the distance 1/2 |u_q - u_x|^2 (no cancellation near 0)
    //    (kRescoreRows window rows per pass, so their loads overlap)
    const float* qu = call.q_unit + (int64_t)q * db.fu;
    for (int w0 = 0; w0 < nw; w0 += kRescoreRows) {
        float dot[kRescoreRows], dd[kRescoreRows];
        int64_t row[kRescoreRows];
#pragma unroll
        for (int j = 0; j < kRescoreRows; ++j)
            row[j] = w0 + j < nw ? p.row0 + sh.widx[wid][w0 + j] : -1;
        rescore_rows<true, kRescoreRows>(db, qu, row, dot, dd, lane);
#pragma unroll
        for (int j = 0; j < kRescoreRows; ++j) {
            if (lane == 0 && row[j] >= 0) {
                sh.wsc[wid][w0 + j] = dot[j];
                // a zero row has cosine 0 by convention: d = 1
                sh.wdist[wid][w0 + j] = db.b64[row[j]] == 0.0 ? 1.0f : 0.5f * dd[j];
            }
        }
    }
    __syncwarp();
    // 5. sort the window by (rescored desc, row asc)
    for (int w = lane; w < nw; w += 32) {
        const float sw = sh.wsc[wid][w];
        const int rw = sh.widx[wid][w];
        int rank = 0;
        for (int v = 0; v < nw; ++v) {
            const float sv = sh.wsc[wid][v];
            rank += (sv > sw) || (sv == sw && sh.widx[wid][v] < rw);
        }
        sh.sidx[wid][rank] = rw;
        sh.ssc[wid][rank] = sw;
        sh.sdist[wid][rank] = sh.wdist[wid][w];
        sh.tie[wid][rank] = 0;
    }
    __syncwarp();
    // 6. near-tie clusters reaching into the first k places: runs whose
    //    neighbouring rescored values differ by at most 2 E_r
    int ncl = 0, nfp = 0;
    // close[j]: window place j is within 2 E_r of place j - 1 (every lane
    // tests one place, so the binary64 gaps cost one instruction per 32)
    uint64_t close = 0;
    {
        const double er2 = 2.0 * (double)p.bound_rerank;
        for (int j0 = 0; j0 < nw; j0 += 32) {
            const int j = j0 + lane;
            const bool c = j > 0 && j < nw &&
                           (double)sh.ssc[wid][j - 1] - (double)sh.ssc[wid][j] <= er2;
            close |= (uint64_t)__ballot_sync(kFull, c) << j0;
        }
    }
    if (lane == 0) {
        int pos = 0;
        const int lim = min(k, nw);
        while (pos < lim) {
            int end = pos + 1;
            while (end < nw && ((close >> end) & 1)) ++end;
            if (end - pos >= 2) {
                sh.cl_begin[wid][ncl] = (int16_t)pos;
                sh.cl_end[wid][ncl] = (int16_t)end;
                ++ncl;
                for (int m = pos; m < end; ++m) sh.tie[wid][m] = 1;
                nfp += end - pos;
            }
            pos = end;
        }
    }
    ncl = __shfl_sync(kFull, ncl, 0);
    nfp = __shfl_sync(kFull, nfp, 0);
    __syncwarp();
    // 7. binary64 scores of the cluster members, one lane each
    if (ncl > 0) {
        const float* qr = call.q_raw + (int64_t)q * db.f;
        for (int m = lane; m < nw; m += 32) {
            if (sh.tie[wid][m]) {
                const int64_t row = p.row0 + sh.sidx[wid][m];
                sh.s64[wid][m] = exact_cosine_ab(qr, db.raw + row * db.f, db.f, db.b64[row]);
            }
        }
        __syncwarp();
        // order each cluster by (binary64 desc, row asc)
        if (lane == 0) {
            for (int c = 0; c < ncl; ++c) {
                const int b = sh.cl_begin[wid][c], e = sh.cl_end[wid][c];
                for (int i = b + 1; i < e; ++i) {
                    const double si = sh.s64[wid][i];
                    const int ri = sh.sidx[wid][i];
                    int j = i;
                    while (j > b && better(si, ri, sh.s64[wid][j - 1], sh.sidx[wid][j - 1])) {
                        sh.s64[wid][j] = sh.s64[wid][j - 1];
                        sh.sidx[wid][j] = sh.sidx[wid][j - 1];
                        --j;
                    }
                    sh.s64[wid][j] = si;
                    sh.sidx[wid][j] = ri;
                }
            }
        }
        __syncwarp();
    }
    // 8. the first k places. A place outside a near-tie cluster reports the
    //    FP32 distance 1/2 |u_q - u_x|^2 unless that is below kExactDist: the
    //    rounding of the unit vectors' elements (2^-24 relative each) moves it
    //    by up to about 2^-23 sqrt(2d), more than 1e-5 d once d is below about
    //    3e-4, so near duplicates take the binary64 cosine (d = 1 - s).
    const int nout = min(nw, k);
    int nexact = 0;
    for (int c = lane; c < nout; c += 32) {
        call.out_idx[out0 + c] = sh.sidx[wid][c];
        float d = sh.sdist[wid][c];
        if (sh.tie[wid][c]) {
            d = (float)(1.0 - sh.s64[wid][c]);
        } else if (d < kExactDist) {
            const int64_t row = p.row0 + sh.sidx[wid][c];
            const float* qr = call.q_raw + (int64_t)q * db.f;
            d = (float)(1.0 - exact_cosine_ab(qr, db.raw + row * db.f, db.f, db.b64[row]));
            ++nexact;
        }
        call.out_dist[out0 + c] = d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nexact += __shfl_xor_sync(kFull, nexact, o);
    if (lane == 0) {
        atomicAdd(&stats[kStatRerank], (unsigned long long)nw);
        atomicAdd(&stats[kStatFp64], (unsigned long long)(nfp + nexact));
        atomicAdd(&stats[kStatNearTies], (unsigned long long)ncl);
    }
    return nout;
}

// A band entry holds a row: a key other than 0 (0 marks a slot a scan thread
// reserved and did not fill) whose row lies in the segment.
__device__ __forceinline__ bool band_entry(uint64_t key, const SegPlan& p) {
    return key != 0 && (uint32_t)key_index(key) < (uint32_t)p.nrows;
}

// Answers query q from its FP8 band: the keys (approximate score s, row) of
// every row whose upper bound s + E_x reached the scan's running k-th best
// lower bound, E_x = a + b r_x the row's own bound (r_x its residual norm; a
// and b per query, from the plan), with empty slots among them. Returns the places
// written, or -1 when the band does not certify the answer (it overflowed its
// buffer, or more than kWindow rows lie within the FP32 rescoring's error of
// the k-th). Whole warp.
//
//  A. L = the k-th best lower bound s - E_x over the band: k rows have cosine
//     at least L, so no row with s + E_x < L is among the k nearest. The band
//     holds every row with s + E_x >= L (the scan's running bound was never
//     above L), the k nearest among them.
//  B. Every band row with s + E_x >= L is rescored in FP32 (error E_r); the
//     others are cleared.
//  C. t = the k-th best FP32 score; the rows within 2 E_r of it form the
//     window of steps 4-8, which contains the k nearest.
__device__ int answer_from_band(const DbView& db, const CallView& call, SelShared& sh, int wid,
                                int lane, int q, const SegPlan& p, unsigned long long* stats) {
    const int k = p.k;
    const int n = call.band_cnt[q];
    if (lane == 0) atomicAdd(&stats[kStatBand], (unsigned long long)n);
    if (n > p.band_cap) return -1;   // the band overflowed its buffer
    uint64_t* band = call.band + p.band0 + (int64_t)(q - p.q0) * p.band_cap;
    const double rq = (double)call.q_resid[q];
    const double a = (double)p.bound_scan + (double)p.bound_rq * rq;
    const double b = ((double)p.bound_rx + rq) * 1.001;

    // A. k-th best lower bound: each lane keeps its k best (as order-mapped
    //    keys with the entry's index, so equal values stay distinct), then k
    //    rounds of the warp's largest key below the previous one
    //    (four entries per lane at a time, so their dependent loads, the key
    //    and then its row's residual, are in flight together)
    RegList<FS_MAX_K> lo;
    lo.reset();
    for (int e0 = 0; e0 < n; e0 += 4 * 32) {
        uint64_t key[4];
        float rx[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = e0 + 32 * j + lane;
            key[j] = e < n ? band[e] : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            rx[j] = band_entry(key[j], p) ? db.resid[p.row0 + key_index(key[j])] : 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = e0 + 32 * j + lane;
            if (band_entry(key[j], p)) {
                const double l = (double)key_score(key[j]) - a - b * (double)rx[j];
                lo.offer((float)l == (float)l ? __double2float_rd(l) : -INFINITY, e, n, 0, -1);
            }
        }
    }
    // (fewer than k entries: no bound, every entry is rescored)
    double L = -INFINITY;
    if (n >= k) {
        uint64_t prev = ~0ull, kth = 0;
        for (int r = 0; r < k; ++r) {
            uint64_t best = 0;
#pragma unroll
            for (int e = 0; e < FS_MAX_K; ++e) {
                const uint64_t v = lo.key(e);
                if (v < prev && v > best) best = v;
            }
            best = warp_max_u64(best);
            prev = best;
            kth = best;
        }
        if (kth != 0) L = (double)key_score(kth);
    }

    // B. rescoring of every band row whose upper bound reaches L (kBandRows
    //    at a time, warp-wide); its key's score becomes the FP32 cosine, the
    //    other keys are cleared. Every lane keeps the same k best scores.
    const float* qu = call.q_unit + (int64_t)q * db.fu;
    RegList<FS_MAX_K> top;
    top.reset();
    int nres = 0;
    uint64_t keys4[4];
    float rx4[4];
    for (int e0 = 0; e0 < n; e0 += 32) {
        const int e = e0 + lane;
        const int j4 = (e0 >> 5) & 3;
        if (j4 == 0) {
            // the keys and residuals of this and the next three rounds, loaded together
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int ej = e0 + 32 * j + lane;
                keys4[j] = ej < n ? band[ej] : 0;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                rx4[j] = band_entry(keys4[j], p) ? db.resid[p.row0 + key_index(keys4[j])] : 0.0f;
        }
        // round j4's key without a run-time register index
        uint64_t key = keys4[0];
        float rxe = rx4[0];
#pragma unroll
        for (int j = 1; j < 4; ++j)
            if (j == j4) {
                key = keys4[j];
                rxe = rx4[j];
            }
        bool in = false;
        if (e < n) {
            if (band_entry(key, p)) {
                const double u = (double)key_score(key) + a + b * (double)rxe;
                in = u >= L;
            }
            if (!in) band[e] = 0;
        }
        unsigned m = __ballot_sync(kFull, in);
        nres += __popc(m);
        while (m != 0) {
            int64_t row[kBandRows];
            int slot[kBandRows];
#pragma unroll
            for (int j = 0; j < kBandRows; ++j) {
                slot[j] = m != 0 ? __ffs(m) - 1 : -1;
                if (m != 0) m &= m - 1;
                const uint64_t kj = __shfl_sync(kFull, key, slot[j] < 0 ? 0 : slot[j]);
                row[j] = slot[j] < 0 ? -1 : p.row0 + key_index(kj);
            }
            float dot[kBandRows], dd[kBandRows];
            rescore_rows<false, kBandRows>(db, qu, row, dot, dd, lane);
#pragma unroll
            for (int j = 0; j < kBandRows; ++j) {
                if (slot[j] < 0) continue;
                const uint32_t li = (uint32_t)(row[j] - p.row0);
                top.offer(dot[j], li, ~0u, 0, -1);
                if (lane == slot[j]) band[e] = make_key(dot[j], li);
            }
        }
    }
    __syncwarp();
    if (nres == 0) return 0;

    // C. the window: rescored rows within 2 E_r of the k-th best
    const int kk = k < top.cnt ? k : top.cnt;
    const float tk = top.kth_score(kk);
    const float wlo = __double2float_ru((double)tk - 2.0 * (double)p.bound_rerank);
    int nw = 0;
    for (int e0 = 0; e0 < n; e0 += 4 * 32) {
        uint64_t kc[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = e0 + 32 * j + lane;
            kc[j] = e < n ? band[e] : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t key = kc[j];
            const bool in = key != 0 && key_score(key) >= wlo;
            const unsigned m = __ballot_sync(kFull, in);
            const int pos = nw + __popc(m & ((1u << lane) - 1));
            if (in && pos < kWindow) sh.widx[wid][pos] = key_index(key);
            nw += __popc(m);
        }
    }
    __syncwarp();
    if (lane == 0) atomicAdd(&stats[kStatRerank], (unsigned long long)nres);
    if (nw > kWindow) return -1;
    return finish_window(db, call, sh, wid, lane, q, p, nw, stats);
}

// Answers query q (whole warp): padding when the scan gave up, the lowest
// indices for a zero query, else from the candidate lists or (BAND) the FP8
// band; a query they do not certify goes to the fallbacks.
template <bool BAND>
__device__ __forceinline__ void select_query(const DbView& db, const CallView& call,
                                             SelShared& sh, int wid, int lane, int q) {
    if (*call.aborted) {
        // a bounded wait of the scan gave up (FS_ETIMEOUT in the status word):
        // its candidate lists are incomplete, so no answer is given
        write_padding(call, q, 0);
    } else {
        const SegPlan p = call.plan[call.q_plan[q]];
        const int k = p.k;
        const int64_t out0 = (int64_t)q * call.k_max;
        const int excl = call.exclude ? call.exclude[q] : -1;
        const int nrows = (int)p.nrows;
        int nout = 0;

        if (nrows == 0) {
            nout = 0;
        } else if (db.metric == FS_COSINE && call.q_ss[q] == 0.0f) {
            // zero query: every cosine is 0, so the lowest indices win (d = 1)
            int c = 0;
            for (int r = 0; r < nrows && c < k; ++r) {
                if (r == excl) continue;
                if (lane == 0) {
                    call.out_idx[out0 + c] = r;
                    call.out_dist[out0 + c] = 1.0f;
                }
                ++c;
            }
            nout = c;
        } else {
            if (BAND) {
                nout = answer_from_band(db, call, sh, wid, lane, q, p, sh.stats);
            } else {
                const int nl = p.chunks * p.lists;
                const uint64_t* cand = call.cand + p.cand0 + (int64_t)(q - p.q0) * nl * p.list_t;
                const double E = (double)p.bound_scan + (double)p.bound_rq * (double)call.q_resid[q];
                nout = answer_from_lists(db, call, sh, wid, lane, q, p, cand, nl, p.list_t, E,
                                         sh.stats);
            }
            if (nout < 0 && lane == 0) {
                if (is_std_metric(db.metric)) {
                    // the binary64 scan answers it directly
                    const int slot = atomicAdd(call.fb2_count, 1);
                    call.fb2_list[slot] = q;
                } else {
                    // the FP32 rescan of the fallback answers it
                    const int slot = atomicAdd(call.fb_count, 1);
                    call.fb_list[slot] = q;
                    call.q_a64[q] = exact_norm2(call.q_raw + (int64_t)q * db.f, db.f);
                }
            }
        }
        if (nout >= 0) {
            write_padding(call, q, nout);
            if (lane == 0) {
                atomicAdd(&sh.stats[kStatQueries], 1ull);
                atomicAdd(&sh.stats[kStatCertified], 1ull);
            }
        }
    }
}

// BAND: the FP8 scan's bands (two resident blocks per SM: the band pass
// keeps two 16-entry lists per lane), answered by persistent warps that each
// take the next query from the call's counter: a band holds tens to
// thousands of rows, and with a query per warp the block's quick warps would
// wait at its final barrier for the slowest (measured: 21.8 -> 16.8 ms on
// 8,192 queries of 16.7 M rows). Else the candidate lists, a warp per query
// (at most 48 registers: five blocks per SM, fewer waves on large batches;
// their work is even, and the counter measured slightly slower there).
template <bool BAND>
__global__ void __launch_bounds__(kSelWarps * 32, BAND ? 2 : 5)
k_select(DbView db, CallView call) {
    __shared__ SelShared sh;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x < kNumStats) sh.stats[threadIdx.x] = 0;
    __syncthreads();
    if (BAND) {
        // the counter runs three times over the queries: the first pass takes
        // the bands of at least a quarter of their capacity, the second those
        // of at least a sixteenth, the third the rest, so the largest bands
        // start first and do not extend the launch's tail (every query is
        // answered once)
        for (;;) {
            __syncwarp();   // the previous query's reads of sh are done
            int i = 0;
            if (lane == 0) i = atomicAdd(call.sel_counter, 1);
            i = __shfl_sync(kFull, i, 0);
            if (i >= 3 * call.nq) break;
            const int pass = i / call.nq, q = i - pass * call.nq;
            const int n = call.band_cnt[q];
            const int cap = call.plan[call.q_plan[q]].band_cap;
            const int cls = n >= cap / 4 ? 0 : n >= cap / 16 ? 1 : 2;
            if (cls != pass) continue;
            select_query<true>(db, call, sh, wid, lane, q);
        }
    } else {
        const int q = blockIdx.x * kSelWarps + wid;
        if (q < call.nq) select_query<false>(db, call, sh, wid, lane, q);
    }
    __syncthreads();
    if (threadIdx.x < kNumStats && sh.stats[threadIdx.x])
        atomicAdd(&db.stats[threadIdx.x], sh.stats[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// first fallback: an FP32 rescan of each uncertified query's database. A warp
// scores one row at a time with the warp-wide sum of the rerank (error bound
// E_r, far tighter than a low-precision scan's), keeping the 16 best rows in
// registers (every lane holds the same list); a block merges its warps into
// one list per row chunk, and the same certification and selection then run
// with E = E_r. A query these lists do not certify (more than 16 rows of one
// chunk within 2 E_r of the k-th best, e.g. many duplicates) goes on to the
// binary64 scan.

constexpr int kFbThreads = 256;
constexpr int kFbWarps = kFbThreads / 32;
constexpr int kFbRows = 4;     // rows a warp scores per pass
constexpr int kGatherPerWarp = 4;   // (query, slot) pairs a warp gathers

__global__ void __launch_bounds__(kFbThreads)
k_fb_scan32(DbView db, CallView call) {
    __shared__ uint64_t wl[kFbWarps][kListT];
    const int nfb = *call.fb_count;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t it = blockIdx.x; it < (int64_t)nfb * kFbChunks; it += gridDim.x) {
        const int slot = (int)(it / kFbChunks), chunk = (int)(it % kFbChunks);
        const int q = call.fb_list[slot];
        const SegPlan p = call.plan[call.q_plan[q]];
        const int excl = call.exclude ? call.exclude[q] : -1;
        const int64_t per = ceil_div(p.nrows, kFbChunks);
        const int64_t lo = p.row0 + chunk * per, hi = p.row0 + min(p.nrows, (int64_t)(chunk + 1) * per);
        const float* qu = call.q_unit + (int64_t)q * db.fu;
        RegList<kListT> lst;
        lst.reset();
        // kFbRows rows per pass, so their loads are in flight together
        for (int64_t row0 = lo + (int64_t)wid * kFbRows; row0 < hi; row0 += kFbWarps * kFbRows) {
            float dot[kFbRows];
#pragma unroll
            for (int r = 0; r < kFbRows; ++r) {
                dot[r] = 0.0f;
                if (row0 + r < hi) {
                    const float* xu = db.unit + (row0 + r) * (int64_t)db.fu;
                    for (int i = lane; i < db.fu; i += 32) dot[r] = fmaf(qu[i], xu[i], dot[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < kFbRows; ++r) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) dot[r] += __shfl_xor_sync(kFull, dot[r], o);
                // the same value (lane 0's sum) in every lane
                dot[r] = __shfl_sync(kFull, dot[r], 0);
            }
#pragma unroll
            for (int r = 0; r < kFbRows; ++r)
                if (row0 + r < hi && (lst.cnt < kListT || dot[r] >= lst.thr_s))
                    lst.offer(dot[r], row0 + r, hi, p.row0, excl);
        }
        if (lane == 0) {
#pragma unroll
            for (int e = 0; e < kListT; ++e) wl[wid][e] = lst.key(e);
        }
        __syncthreads();
        if (wid == 0) {
            // the block's 16 best of the warps' 8 x 16 (rows are distinct)
            uint64_t mine[kFbWarps * kListT / 32];
#pragma unroll
            for (int j = 0; j < kFbWarps * kListT / 32; ++j)
                mine[j] = (&wl[0][0])[lane + 32 * j];
            uint64_t prev = ~0ull;
            uint64_t* dst = call.cand_fb + ((int64_t)slot * kFbChunks + chunk) * kListT;
            for (int e = 0; e < kListT; ++e) {
                uint64_t best = 0;
#pragma unroll
                for (int j = 0; j < kFbWarps * kListT / 32; ++j)
                    if (mine[j] < prev && mine[j] > best) best = mine[j];
                best = warp_max_u64(best);
                if (lane == 0) dst[e] = best;
                prev = best;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSelWarps * 32)
k_fb_select(DbView db, CallView call) {
    __shared__ SelShared sh;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x < kNumStats) sh.stats[threadIdx.x] = 0;
    __syncthreads();
    const int nfb = *call.fb_count;
    for (int slot = blockIdx.x * kSelWarps + wid; slot < nfb; slot += gridDim.x * kSelWarps) {
        const int q = call.fb_list[slot];
        const SegPlan p = call.plan[call.q_plan[q]];
        const uint64_t* cand = call.cand_fb + (int64_t)slot * kFbChunks * kListT;
        const int nout = answer_from_lists(db, call, sh, wid, lane, q, p, cand, kFbChunks, kListT,
                                           (double)p.bound_rerank, sh.stats);
        if (nout >= 0) {
            write_padding(call, q, nout);
            if (lane == 0) {
                atomicAdd(&sh.stats[kStatQueries], 1ull);
                atomicAdd(&sh.stats[kStatFallback], 1ull);
            }
        } else if (lane == 0) {
            const int s2 = atomicAdd(call.fb2_count, 1);
            call.fb2_list[s2] = q;
        }
    }
    __syncthreads();
    if (threadIdx.x < kNumStats && sh.stats[threadIdx.x])
        atomicAdd(&db.stats[threadIdx.x], sh.stats[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// last fallback: binary64 scores of every row for the queries even the FP32
// rescan could not certify, split into kFbChunks row chunks per query

static_assert(kFbChunks <= 32, "one lane per fallback chunk in the merge");

__global__ void __launch_bounds__(kFbThreads)
k_fallback_scan(DbView db, CallView call) {
    __shared__ double ws[kFbThreads / 32][FS_MAX_K];
    __shared__ int wi[kFbThreads / 32][FS_MAX_K];
    const int nfb = *call.fb2_count;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t it = blockIdx.x; it < (int64_t)nfb * kFbChunks; it += gridDim.x) {
        const int slot = (int)(it / kFbChunks), chunk = (int)(it % kFbChunks);
        const int q = call.fb2_list[slot];
        const SegPlan p = call.plan[call.q_plan[q]];
        const int k = p.k;
        const int excl = call.exclude ? call.exclude[q] : -1;
        const double a64 = call.q_a64[q];
        const int64_t per = ceil_div(p.nrows, kFbChunks);
        const int64_t lo = chunk * per, hi = min(p.nrows, lo + per);
        const float* qr = call.q_raw + (int64_t)q * db.f;

        // per-thread best k, kept sorted
        double ts[FS_MAX_K];
        int ti[FS_MAX_K];
        for (int c = 0; c < FS_MAX_K; ++c) { ts[c] = -INFINITY; ti[c] = -1; }
        for (int64_t r = lo + threadIdx.x; r < hi; r += kFbThreads) {
            if ((int)r == excl) continue;
            const int64_t row = p.row0 + r;
            const double s = is_std_metric(db.metric)
                                 ? -exact_std_distance(db, p, qr, db.raw + row * db.f)
                                 : exact_cosine(qr, db.raw + row * db.f, db.f, a64, db.b64[row]);
            if (ti[k - 1] >= 0 && !better(s, (int)r, ts[k - 1], ti[k - 1])) continue;
            int pos = k - 1;
            while (pos > 0 && (ti[pos - 1] < 0 || better(s, (int)r, ts[pos - 1], ti[pos - 1]))) {
                ts[pos] = ts[pos - 1];
                ti[pos] = ti[pos - 1];
                --pos;
            }
            ts[pos] = s;
            ti[pos] = (int)r;
        }
        // warp merge: k rounds of warp-wide best over the lanes' list heads
        int head = 0;
        for (int c = 0; c < k; ++c) {
            double s = head < k ? ts[head] : -INFINITY;
            int i = head < k ? ti[head] : -1;
            double bsv = s;
            int biv = i;
            warp_best(bsv, biv);
            if (biv >= 0 && biv == i) ++head;
            if (lane == 0) { ws[wid][c] = bsv; wi[wid][c] = biv; }
        }
        __syncthreads();
        // block merge by warp 0 over the 8 warps' lists
        if (wid == 0) {
            int h = 0;  // lane < 8 owns warp lane's list
            for (int c = 0; c < k; ++c) {
                double s = (lane < kFbThreads / 32 && h < k) ? ws[lane][h] : -INFINITY;
                int i = (lane < kFbThreads / 32 && h < k) ? wi[lane][h] : -1;
                double bsv = s;
                int biv = i;
                warp_best(bsv, biv);
                if (biv >= 0 && biv == i) ++h;
                if (lane == 0) {
                    call.fb_score[((int64_t)slot * kFbChunks + chunk) * FS_MAX_K + c] = bsv;
                    call.fb_index[((int64_t)slot * kFbChunks + chunk) * FS_MAX_K + c] = biv;
                }
            }
        }
        __syncthreads();
    }
}

__global__ void k_fallback_merge(DbView db, CallView call) {
    __shared__ unsigned long long st[2];
    if (threadIdx.x < 2) st[threadIdx.x] = 0;
    __syncthreads();
    const int nfb = *call.fb2_count;
    const int lane = threadIdx.x & 31;
    // a fixed grid strides over the queries (usually none: the grid then
    // returns at once)
    for (int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); slot < nfb;
         slot += gridDim.x * (blockDim.x >> 5)) {
        const int q = call.fb2_list[slot];
        const SegPlan p = call.plan[call.q_plan[q]];
        const int k = p.k;
        const int64_t out0 = (int64_t)q * call.k_max;
        // lane c < kFbChunks owns chunk c's sorted list
        int h = 0;
        int nout = 0;
        for (int c = 0; c < k; ++c) {
            double s = -INFINITY;
            int i = -1;
            if (lane < kFbChunks && h < k) {
                s = call.fb_score[((int64_t)slot * kFbChunks + lane) * FS_MAX_K + h];
                i = call.fb_index[((int64_t)slot * kFbChunks + lane) * FS_MAX_K + h];
            }
            double bsv = s;
            int biv = i;
            warp_best(bsv, biv);
            if (biv >= 0 && biv == i) ++h;
            if (biv < 0) break;
            if (lane == 0) {
                call.out_idx[out0 + c] = biv;
                call.out_dist[out0 + c] = is_std_metric(db.metric) ? (float)(-bsv)
                                                                   : (float)(1.0 - bsv);
            }
            ++nout;
        }
        write_padding(call, q, nout);
        if (lane == 0) {
            atomicAdd(&st[0], 1ull);
            atomicAdd(&st[1], (unsigned long long)p.nrows);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && st[0]) {
        atomicAdd(&db.stats[kStatQueries], st[0]);
        atomicAdd(&db.stats[kStatFallback], st[0]);
        atomicAdd(&db.stats[kStatFp64], st[1]);
    }
}

// ---------------------------------------------------------------------------
// gather of the neighbours' phase orders: one warp per (query, slot)

// Eight lanes per (query, slot), four per warp, so four independent chains
// of loads (result row, order offsets, pass IDs) are in flight per warp.
__global__ void k_gather(DbView db, CallView call, int16_t* __restrict__ seq_out,
                         int32_t* __restrict__ seq_len, int l_max, int32_t* __restrict__ dup_of) {
    const int lane = threadIdx.x & 31, sub = lane & 7, grp = lane >> 3;
    const unsigned gmask = 0xffu << (grp * 8);
    const int64_t w =
        ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kGatherPerWarp + grp;
    if (w >= (int64_t)call.nq * call.k_max) return;   // whole groups leave together
    const int q = (int)(w / call.k_max), c = (int)(w % call.k_max);
    const SegPlan p = call.plan[call.q_plan[q]];
    const int r = call.out_idx[w];
    int16_t* dst = seq_out + w * l_max;
    int64_t lo = 0, len = 0;
    if (r >= 0) {
        lo = db.seq_off[p.row0 + r];
        len = db.seq_off[p.row0 + r + 1] - lo;
    }
    const int64_t m = len < l_max ? len : l_max;
    for (int i = sub; i < l_max; i += 8) dst[i] = i < m ? db.seq_ids[lo + i] : (int16_t)-1;
    if (sub == 0) seq_len[w] = (int32_t)len;
    if (dup_of) {
        int first = -1;
        if (r >= 0) {
            for (int c2 = 0; c2 < c && first < 0; ++c2) {
                const int r2 = call.out_idx[(int64_t)q * call.k_max + c2];
                if (r2 < 0) continue;
                const int64_t lo2 = db.seq_off[p.row0 + r2];
                const int64_t len2 = db.seq_off[p.row0 + r2 + 1] - lo2;
                if (len2 != len) continue;
                bool same = true;
                for (int64_t i = sub; i < len; i += 8)
                    same &= db.seq_ids[lo + i] == db.seq_ids[lo2 + i];
                if (__all_sync(gmask, same)) first = c2;
            }
        }
        if (sub == 0) dup_of[w] = first;
    }
}

}  // namespace

cudaError_t launch_write_plan(const SegPlan* host_plan, const int32_t* host_q_order, int n_seg,
                              SegPlan* dev_plan, int32_t* dev_q_order, int32_t* fb_count,
                              int32_t* work_counter, cudaStream_t st) {
    for (int base = 0; base < n_seg; base += kPlanPerLaunch) {
        PlanChunk chunk;
        const int n = (n_seg - base) < kPlanPerLaunch ? (n_seg - base) : kPlanPerLaunch;
        for (int i = 0; i < n; ++i) {
            chunk.p[i] = host_plan[base + i];
            chunk.q_order[i] = host_q_order[base + i];
        }
        k_write_plan<<<1, kPlanPerLaunch, 0, st>>>(chunk, n, dev_plan + base, dev_q_order + base,
                                                   base == 0 ? fb_count : nullptr, work_counter);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_query_plan(const CallView& call, int32_t* q_plan, cudaStream_t st) {
    if (call.nq == 0 || call.n_seg == 0) return cudaSuccess;
    k_query_plan<<<(unsigned)call.n_seg, 256, 0, st>>>(call.plan, q_plan);
    return cudaGetLastError();
}

// Resident blocks per SM of the band selection on the current device (kept
// per device: occupancy belongs to the device's context).
static int select_blocks_per_sm() {
    static std::mutex mu;
    static int cached[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    std::lock_guard<std::mutex> g(mu);
    if (dev >= 0 && dev < kMaxDevices && cached[dev] > 0) return cached[dev];
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_select<true>, kSelWarps * 32, 0) !=
            cudaSuccess ||
        nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    if (dev >= 0 && dev < kMaxDevices) cached[dev] = nb;
    return nb;
}

cudaError_t launch_select(const DbView& db, const CallView& call, int num_sms, cudaStream_t st) {
    if (call.nq == 0) return cudaSuccess;
    const unsigned per_query = (unsigned)ceil_div(call.nq, kSelWarps);
    if (db.prec == FS_FP8_E4M3 && db.metric == FS_COSINE) {
        // one resident wave of persistent blocks, or fewer when the queries need fewer
        const int64_t resident = (int64_t)std::max(1, num_sms) * select_blocks_per_sm();
        const unsigned grid = (unsigned)std::min<int64_t>(per_query, resident);
        k_select<true><<<grid, kSelWarps * 32, 0, st>>>(db, call);
    } else {
        k_select<false><<<per_query, kSelWarps * 32, 0, st>>>(db, call);
    }
    return cudaGetLastError();
}

cudaError_t launch_fallback(const DbView& db, const CallView& call, int num_sms, cudaStream_t st) {
    if (call.nq == 0) return cudaSuccess;
    k_fb_scan32<<<num_sms * 4, kFbThreads, 0, st>>>(db, call);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
    k_fb_select<<<num_sms, kSelWarps * 32, 0, st>>>(db, call);
    e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
    k_fallback_scan<<<num_sms * 2, kFbThreads, 0, st>>>(db, call);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_fallback_merge<<<num_sms, 256, 0, st>>>(db, call);
    return cudaGetLastError();
}

cudaError_t launch_gather(const DbView& db, const CallView& call, int16_t* seq_out, int32_t* seq_len,
                          int l_max, int32_t* dup_of, cudaStream_t st) {
    const int64_t items = (int64_t)call.nq * call.k_max;
    if (items == 0) return cudaSuccess;
    const int64_t warps = ceil_div(items, kGatherPerWarp);
    k_gather<<<(unsigned)ceil_div(warps, 8), 256, 0, st>>>(db, call, seq_out, seq_len, l_max,
                                                            dup_of);
    return cudaGetLastError();
}

}  // namespace fsk
