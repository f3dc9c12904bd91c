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
constexpr int BK = 16;              // features per pipeline step
constexpr int THREADS = 256;
constexpr int T = kListT;
// Row pitch of the operand and score tiles: 4 floats of padding make the
// transposing operand stores, the float4 score stores and the filter's
// float4 score reads free of bank conflicts (and keep rows 16-byte aligned).
constexpr int P = 132;

struct Operands {
    float as[2][BK][P];   // queries, feature-major (double-buffered)
    float bs[2][BK][P];   // database rows, feature-major
};
struct Smem {
    union {
        Operands op;              // during the products
        float s[BQ][P];           // the tile's scores, while the filter reads them
    };
    uint64_t lists[T][THREADS];
    float thr[THREADS];           // each list's current threshold (for the skip vote)
};

// Two floats in one 64-bit register pair (lo: the first) and the two-lane
// FMA d = a * b + d on such pairs, each lane rounded to nearest.
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
    return ((uint64_t)__float_as_uint(hi) << 32) | (uint64_t)__float_as_uint(lo);
}
__device__ __forceinline__ void fma2(uint64_t& d, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

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
//
// Per tile: the 128 x 128 products in registers (each thread 8 queries x 8
// rows, features in order, FMA), then a block-wide vote: only when some score
// reaches its list's threshold is the score tile written to shared memory
// (over the idle operand buffers) for the list owners (thread = query x half
// of the tile's rows) to filter.
template <int METRIC>
__global__ void __launch_bounds__(THREADS, 2)
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
        // the vote's threshold of this list (read by other threads after the
        // next barrier): a list of an absent or zero query never takes a row
        sm.thr[tid] = qv ? -INFINITY : INFINITY;
        uint32_t* shared_p = call.shared_thr + qbase + (qv ? lq : 0);
        const float e2 =
            qv ? 2.0f * (p.bound_scan + p.bound_rq * call.q_resid[qbase + lq]) * 1.0001f : 0.0f;
        float published = -INFINITY;

        // global-load mapping: per step, two float4 of queries and two of rows
        // (rows ld_row and ld_row + 64, features ld_col .. ld_col + 3)
        const int ld_row = tid >> 2, ld_col = (tid & 3) * 4;
        const float* qrow0 = call.q_unit + (int64_t)(qbase + ld_row) * fu + ld_col;
        const float* qrow1 = qrow0 + (int64_t)64 * fu;
        const bool q_ok0 = ld_row < nq_tile, q_ok1 = ld_row + 64 < nq_tile;

        for (int64_t tr = row_begin; tr < row_end; tr += BN) {
            const bool b_ok0 = tr + ld_row < row_end, b_ok1 = tr + ld_row + 64 < row_end;
            const float* xrow0 = db.unit + (tr + ld_row) * fu + ld_col;
            const float* xrow1 = xrow0 + (int64_t)64 * fu;
            const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);

            float acc[8][8];
            // dot-product metrics: the accumulators in packed pairs (queries 2p,
            // 2p + 1 of the thread's 8, for one of its rows; pairing queries, whose
            // values arrive as adjacent pairs in each float4, measured faster than
            // pairing rows), advanced with the two-lane FMA (each lane an ordinary
            // rounded fused multiply-add, so every score is the same sequence of
            // FMAs as with scalar instructions, in half the issues)
            uint64_t acc2[4][8];   // [query pair][row]
#pragma unroll
            for (int i = 0; i < 8; ++i) {
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
#pragma unroll
                for (int j = 0; j < 8; ++j) acc2[i][j] = 0ull;
            }

            float4 ra0 = q_ok0 ? *reinterpret_cast<const float4*>(qrow0) : z4;
            float4 ra1 = q_ok1 ? *reinterpret_cast<const float4*>(qrow1) : z4;
            float4 rb0 = b_ok0 ? __ldg(reinterpret_cast<const float4*>(xrow0)) : z4;
            float4 rb1 = b_ok1 ? __ldg(reinterpret_cast<const float4*>(xrow1)) : z4;
            int buf = 0;
            for (int k0 = 0; k0 < fu; k0 += BK) {
                // fu is a multiple of 32, so every step is whole; features ld_col..+3
                // of rows ld_row and ld_row + 64, stored feature-major
                float (*as)[P] = sm.op.as[buf];
                float (*bs)[P] = sm.op.bs[buf];
                as[ld_col + 0][ld_row] = ra0.x;
                as[ld_col + 1][ld_row] = ra0.y;
                as[ld_col + 2][ld_row] = ra0.z;
                as[ld_col + 3][ld_row] = ra0.w;
                as[ld_col + 0][ld_row + 64] = ra1.x;
                as[ld_col + 1][ld_row + 64] = ra1.y;
                as[ld_col + 2][ld_row + 64] = ra1.z;
                as[ld_col + 3][ld_row + 64] = ra1.w;
                bs[ld_col + 0][ld_row] = rb0.x;
                bs[ld_col + 1][ld_row] = rb0.y;
                bs[ld_col + 2][ld_row] = rb0.z;
                bs[ld_col + 3][ld_row] = rb0.w;
                bs[ld_col + 0][ld_row + 64] = rb1.x;
                bs[ld_col + 1][ld_row + 64] = rb1.y;
                bs[ld_col + 2][ld_row + 64] = rb1.z;
                bs[ld_col + 3][ld_row + 64] = rb1.w;
                __syncthreads();
                if (k0 + BK < fu) {
                    ra0 = q_ok0 ? *reinterpret_cast<const float4*>(qrow0 + k0 + BK) : z4;
                    ra1 = q_ok1 ? *reinterpret_cast<const float4*>(qrow1 + k0 + BK) : z4;
                    rb0 = b_ok0 ? __ldg(reinterpret_cast<const float4*>(xrow0 + k0 + BK)) : z4;
                    rb1 = b_ok1 ? __ldg(reinterpret_cast<const float4*>(xrow1 + k0 + BK)) : z4;
                }
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    const float4 u0 = *reinterpret_cast<const float4*>(&bs[kk][tx * 4]);
                    const float4 u1 = *reinterpret_cast<const float4*>(&bs[kk][64 + tx * 4]);
                    const float b[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                    if (METRIC == FS_MANHATTAN) {
                        const float4 t0 = *reinterpret_cast<const float4*>(&as[kk][ty * 4]);
                        const float4 t1 = *reinterpret_cast<const float4*>(&as[kk][64 + ty * 4]);
                        const float a[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
                        for (int i = 0; i < 8; ++i)
#pragma unroll
                            for (int j = 0; j < 8; ++j) acc[i][j] += fabsf(a[i] - b[j]);
                    } else {
                        // the query pairs as two 64-bit halves of each 128-bit load (a
                        // float4 split into scalars measured slower: the compiler then
                        // issued extra narrower shared loads)
                        const ulonglong2 A0 = *reinterpret_cast<const ulonglong2*>(&as[kk][ty * 4]);
                        const ulonglong2 A1 = *reinterpret_cast<const ulonglong2*>(&as[kk][64 + ty * 4]);
                        const uint64_t ap[4] = {A0.x, A0.y, A1.x, A1.y};
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const uint64_t bp = pack2(b[j], b[j]);
#pragma unroll
                            for (int i = 0; i < 4; ++i) fma2(acc2[i][j], ap[i], bp);
                        }
                    }
                }
                buf ^= 1;
            }
            if (METRIC != FS_MANHATTAN) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const uint64_t v = acc2[i][j];
                        acc[2 * i][j] = __uint_as_float((uint32_t)v);
                        acc[2 * i + 1][j] = __uint_as_float((uint32_t)(v >> 32));
                    }
            }
            // the scores of this thread's 8 queries x 8 rows (standardised
            // metrics: minus the row term; a row above a query's magnitude cap
            // is provably not among its k nearest and scores -inf, since its
            // FP32 score is outside the query's bound)
            if (METRIC != FS_COSINE) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int rj = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
                    const bool in = tr + rj < row_end;
                    const float rt = (METRIC == FS_EUCLIDEAN && in) ? db.row_term[tr + rj] : 0.0f;
                    const float mg = in ? db.row_mag[tr + rj] : 0.0f;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int qi = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
                        const float cap = qi < nq_tile ? call.q_scale[qbase + qi] : INFINITY;
                        float sc = METRIC == FS_MANHATTAN ? -acc[i][j] : acc[i][j] - rt;
                        if (mg > cap) sc = -INFINITY;
                        acc[i][j] = sc;
                    }
                }
            }
            // does any score reach its list's threshold? (each list's owner wrote
            // it after the previous tile; the shared bound only raises it)
            bool any = false;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int qi = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
                const float t0 = sm.thr[qi], t1 = sm.thr[qi + BQ];
#pragma unroll
                for (int j = 0; j < 4; ++j) any |= acc[i][j] >= t0;
#pragma unroll
                for (int j = 4; j < 8; ++j) any |= acc[i][j] >= t1;
            }
            // every thread is done with the operand buffers (the score tile
            // overlays them) and the vote is in
            if (!__syncthreads_or(any)) continue;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int qi = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
                *reinterpret_cast<float4*>(&sm.s[qi][tx * 4]) =
                    make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                *reinterpret_cast<float4*>(&sm.s[qi][64 + tx * 4]) =
                    make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
            }
            __syncthreads();

            // filter: keep this thread's 16 best of its 64 columns
            const float* srow = &sm.s[lq][hf * 64];
            const int64_t col_row0 = tr + hf * 64;
            // (the initial bound, 0, maps to NaN: fmaxf then keeps thr_s)
            const float shared_s = qv ? unord_f32(__ldcg(shared_p)) : INFINITY;
            bool changed = false;
            for (int j4 = 0; j4 < 64; j4 += 4) {
                const float4 s4 = *reinterpret_cast<const float4*>(srow + j4);
                const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const float sc = sv[jj];
                    if (sc >= fmaxf(thr_s, shared_s)) {
                        const int64_t row = col_row0 + j4 + jj;
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
            // this list's threshold for the next tile's vote (a list of a query
            // outside the tile never takes a row)
            // (both parts only rise, so the next filter's threshold is at least
            // this: the vote never skips a tile the filter would take rows from)
            sm.thr[tid] = fmaxf(thr_s, shared_s);
            __syncthreads();   // the score tile is free for the next tile's operands
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
