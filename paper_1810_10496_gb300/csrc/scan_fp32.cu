// FP32 SIMT scan: cosine scores of unit vectors with fused candidate lists.
//
// Sec. 4 selects, for a new kernel, the K reference kernels with the most
// similar feature vectors under the cosine of Sec. 4.2. With unit vectors the
// cosine is a dot product, so a block of queries against a block of database
// rows is a small matrix product. This kernel is the plain FP32 path: a
// register-tiled product (each thread owns 8 x 8 scores, accumulated with
// FMA over the features in order) followed by a filter that keeps, per query
// and per half of each row chunk, the 16 best (score, index) pairs seen.
//
// Work is split into items (segment, tile of 128 queries, chunk of rows);
// persistent blocks take items from an atomic counter. Items of one row chunk
// are numbered consecutively over the query tiles, so blocks that run at the
// same time read the same rows and share them through L2.
#include <mutex>

#include "fs_internal.cuh"

namespace fsk {

namespace {

constexpr int BQ = kQTile;          // queries per item
constexpr int BN = kFp32TileRows;   // rows per tile
constexpr int BK = 8;               // features per pipeline step
constexpr int THREADS = 256;
constexpr int T = kListT;
constexpr int SP = BN + 1;          // score-tile row pitch (odd: conflict free)

struct Smem {
    float as[2][BK][BQ];
    float bs[2][BK][BN];
    float s[BQ][SP];
    uint64_t lists[T][THREADS];
};

__device__ __forceinline__ int find_plan(const SegPlan* plan, int n_seg, int64_t item) {
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (plan[mid].item0 <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// METRIC: FS_COSINE and FS_EUCLIDEAN accumulate dot products (Euclidean then
// subtracts the row term 1/2 |z_x|^2), FS_MANHATTAN accumulates |a - b| and
// scores its negation; larger is nearer in every case.
template <int METRIC>
__global__ void __launch_bounds__(THREADS)
k_scan_fp32(DbView db, CallView call) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    __shared__ int64_t s_item;
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    const int fu = db.fu;

    // list ownership in the filter: query lq, half hf of each tile's columns
    const int lq = tid & (BQ - 1);
    const int hf = tid >> 7;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(call.work_counter, 1);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= call.total_items) break;
        const int pi = find_plan(call.plan, call.n_seg, item);
        const SegPlan p = call.plan[pi];
        const int64_t local = item - p.item0;
        const int chunk = (int)(local / p.qtiles);
        const int qtile = (int)(local % p.qtiles);
        const int qbase = p.q0 + qtile * BQ;          // first query (global)
        const int nq_tile = min(BQ, p.nq - qtile * BQ);
        const int64_t row_begin = p.row0 + (int64_t)chunk * p.chunk_rows;
        const int64_t row_end = min(p.row0 + p.nrows, row_begin + p.chunk_rows);

        // per-thread candidate list state
        int cnt = 0, min_slot = 0;
        uint64_t thr_key = 0;
        float thr_s = -INFINITY;
#pragma unroll
        for (int e = 0; e < T; ++e) sm.lists[e][tid] = 0;
        const int excl = (call.exclude && lq < nq_tile) ? call.exclude[qbase + lq] : -1;
        // the pruning bound shared by every block scanning this query (as in
        // the tensor-core scan): the k-th best score any list holds minus 2E;
        // rows below it cannot be among the k nearest
        // (a zero cosine query, q_ss = 0, ties with every row and is answered
        // by the selection from row indices alone: it offers nothing)
        const bool qv = lq < nq_tile && call.q_ss[qbase + lq] != 0.0f;
        uint32_t* shared_p = call.shared_thr + qbase + (qv ? lq : 0);
        const float e2 =
            qv ? 2.0f * (p.bound_scan + p.bound_rq * call.q_resid[qbase + lq]) * 1.0001f : 0.0f;
        float published = -INFINITY;

        // global-load mapping: one float4 of A and one of B per thread and step
        const int ld_row = tid >> 1, ld_col = (tid & 1) * 4;
        const float* qrow = call.q_unit + (int64_t)(qbase + ld_row) * fu + ld_col;
        const bool q_ok = ld_row < nq_tile;

        for (int64_t tr = row_begin; tr < row_end; tr += BN) {
            const int64_t brow = tr + ld_row;
            const bool b_ok = brow < row_end;
            const float* xrow = db.unit + brow * fu + ld_col;

            float acc[8][8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

            float4 ra = q_ok ? *reinterpret_cast<const float4*>(qrow) : make_float4(0, 0, 0, 0);
            float4 rb = b_ok ? __ldg(reinterpret_cast<const float4*>(xrow)) : make_float4(0, 0, 0, 0);
            int buf = 0;
            for (int k0 = 0; k0 < fu; k0 += BK) {
                sm.as[buf][ld_col + 0][ld_row] = ra.x;
                sm.as[buf][ld_col + 1][ld_row] = ra.y;
                sm.as[buf][ld_col + 2][ld_row] = ra.z;
                sm.as[buf][ld_col + 3][ld_row] = ra.w;
                sm.bs[buf][ld_col + 0][ld_row] = rb.x;
                sm.bs[buf][ld_col + 1][ld_row] = rb.y;
                sm.bs[buf][ld_col + 2][ld_row] = rb.z;
                sm.bs[buf][ld_col + 3][ld_row] = rb.w;
                __syncthreads();
                if (k0 + BK < fu) {
                    ra = q_ok ? *reinterpret_cast<const float4*>(qrow + k0 + BK) : make_float4(0, 0, 0, 0);
                    rb = b_ok ? __ldg(reinterpret_cast<const float4*>(xrow + k0 + BK))
                              : make_float4(0, 0, 0, 0);
                }
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    float a[8], b[8];
                    float4 t0 = *reinterpret_cast<const float4*>(&sm.as[buf][kk][ty * 4]);
                    float4 t1 = *reinterpret_cast<const float4*>(&sm.as[buf][kk][64 + ty * 4]);
                    float4 u0 = *reinterpret_cast<const float4*>(&sm.bs[buf][kk][tx * 4]);
                    float4 u1 = *reinterpret_cast<const float4*>(&sm.bs[buf][kk][64 + tx * 4]);
                    a[0] = t0.x; a[1] = t0.y; a[2] = t0.z; a[3] = t0.w;
                    a[4] = t1.x; a[5] = t1.y; a[6] = t1.z; a[7] = t1.w;
                    b[0] = u0.x; b[1] = u0.y; b[2] = u0.z; b[3] = u0.w;
                    b[4] = u1.x; b[5] = u1.y; b[6] = u1.z; b[7] = u1.w;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            if (METRIC == FS_MANHATTAN)
                                acc[i][j] += fabsf(a[i] - b[j]);
                            else
                                acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
                        }
                }
                buf ^= 1;
            }
            __syncthreads();  // every thread is done with the previous score tile
            // standardised metrics: the rows' terms and magnitudes (a row above
            // a query's magnitude cap is provably not among its k nearest and
            // scores -inf, since its FP32 score is outside the query's bound)
            float rt[8], mg[8], cap[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int rj = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
                const bool in = METRIC != FS_COSINE && tr + rj < row_end;
                rt[j] = (METRIC == FS_EUCLIDEAN && in) ? db.row_term[tr + rj] : 0.0f;
                mg[j] = in ? db.row_mag[tr + rj] : 0.0f;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int qi = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
                cap[i] = (METRIC != FS_COSINE && qi < nq_tile) ? call.q_scale[qbase + qi] : INFINITY;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int qi = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int rj = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
                    float sc = METRIC == FS_MANHATTAN ? -acc[i][j]
                               : (METRIC == FS_EUCLIDEAN ? acc[i][j] - rt[j] : acc[i][j]);
                    if (METRIC != FS_COSINE && mg[j] > cap[i]) sc = -INFINITY;
                    sm.s[qi][rj] = sc;
                }
            }
            __syncthreads();

            // filter: keep this thread's 16 best of its 64 columns
            const float* srow = &sm.s[lq][hf * 64];
            const int64_t col_row0 = tr + hf * 64;
            // (the initial bound, 0, maps to NaN: fmaxf then keeps thr_s)
            const float shared_s = qv ? unord_f32(__ldcg(shared_p)) : INFINITY;
            bool changed = false;
            for (int j = 0; j < 64; ++j) {
                const float sc = srow[j];
                if (sc >= fmaxf(thr_s, shared_s)) {
                    const int64_t row = col_row0 + j;
                    const int32_t li = (int32_t)(row - p.row0);
                    if (row < row_end && li != excl) {
                        const uint64_t key = make_key(sc, (uint32_t)li);
                        bool recompute = false;
                        if (cnt < T) {
                            sm.lists[cnt][tid] = key;
                            ++cnt;
                            recompute = (cnt == T);
                        } else if (key > thr_key) {
                            sm.lists[min_slot][tid] = key;
                            recompute = true;
                        }
                        if (recompute) {
                            uint64_t mn = ~0ull;
#pragma unroll
                            for (int e = 0; e < T; ++e) {
                                uint64_t v = sm.lists[e][tid];
                                if (v < mn) { mn = v; min_slot = e; }
                            }
                            thr_key = mn;
                            thr_s = key_score(mn);
                        }
                        changed = true;
                    }
                }
            }
            if (qv && changed && cnt >= p.k) {
                // the list's k-th best (keys are distinct), then the bound,
                // rounded down: it may only err low
                uint64_t prev = ~0ull, best = 0;
                for (int r = 0; r < p.k; ++r) {
                    best = 0;
#pragma unroll
                    for (int e = 0; e < T; ++e) {
                        const uint64_t v = sm.lists[e][tid];
                        if (v < prev && v > best) best = v;
                    }
                    prev = best;
                }
                const float kth = key_score(best);
                const float bound = (kth - e2) - fabsf(kth) * 0x1p-20f;
                if (bound > published) {
                    atomicMax(shared_p, ord_f32(bound));
                    published = bound;
                }
            }
        }

        // publish this item's lists, sorted in descending order (empty entries,
        // 0, last) as the selection expects: an odd-even transposition sort
        if (lq < nq_tile) {
            const int64_t qlocal = (int64_t)qtile * BQ + lq;
            uint64_t* dst = call.cand + p.cand0 +
                            ((qlocal * p.chunks + chunk) * p.lists + hf) * (int64_t)T;
            // (this kernel always keeps lists of kListT = T entries)
            uint64_t v[T];
#pragma unroll
            for (int e = 0; e < T; ++e) v[e] = sm.lists[e][tid];
#pragma unroll
            for (int r = 0; r < T; ++r) {
#pragma unroll
                for (int e = r & 1; e + 1 < T; e += 2) {
                    const uint64_t a = v[e], b = v[e + 1];
                    v[e] = a > b ? a : b;
                    v[e + 1] = a > b ? b : a;
                }
            }
#pragma unroll
            for (int e = 0; e < T; ++e) dst[e] = v[e];
        }
        __syncthreads();  // s_item and the lists are reused by the next item
    }
}

}  // namespace

// Sets the kernels' dynamic shared-memory limit on the current device and
// returns the resident blocks per SM. Both belong to the current device's
// context, so they are kept per device.
int scan_fp32_ctas_per_sm() {
    static std::mutex mu;
    static int cached[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    std::lock_guard<std::mutex> g(mu);
    if (dev >= 0 && dev < kMaxDevices && cached[dev] > 0) return cached[dev];
    cudaFuncSetAttribute(k_scan_fp32<FS_COSINE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(Smem));
    cudaFuncSetAttribute(k_scan_fp32<FS_EUCLIDEAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(Smem));
    cudaFuncSetAttribute(k_scan_fp32<FS_MANHATTAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(Smem));
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scan_fp32<FS_COSINE>, THREADS,
                                                      sizeof(Smem)) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    if (dev >= 0 && dev < kMaxDevices) cached[dev] = nb;
    return nb;
}

cudaError_t launch_scan_fp32(const DbView& db, const CallView& call, int grid, cudaStream_t st) {
    if (call.total_items == 0) return cudaSuccess;
    scan_fp32_ctas_per_sm();  // sets the shared-memory attribute once
    if (db.metric == FS_EUCLIDEAN)
        k_scan_fp32<FS_EUCLIDEAN><<<grid, THREADS, sizeof(Smem), st>>>(db, call);
    else if (db.metric == FS_MANHATTAN)
        k_scan_fp32<FS_MANHATTAN><<<grid, THREADS, sizeof(Smem), st>>>(db, call);
    else
        k_scan_fp32<FS_COSINE><<<grid, THREADS, sizeof(Smem), st>>>(db, call);
    return cudaGetLastError();
}

}  // namespace fsk
