// Tensor-core scan (tcgen05) of BF16 or FP8 E4M3 unit vectors, with fused
// per-query candidate lists.
//
// Sec. 4 picks the K reference kernels whose feature vectors are closest to
// the new kernel's under the cosine of Sec. 4.2. Once the database rows and
// the queries are unit vectors the scores of a block of queries against a
// block of rows form a matrix product, which this kernel computes on the
// 5th-generation tensor cores and filters without ever writing it out:
//
//   * A = 128 queries (K-major, resident in shared memory for a work item),
//     B = 256 database rows per tile (K-major, streamed by TMA through a ring
//     of 128-byte-swizzled K blocks of 32 KB, as deep as shared memory
//     allows), D = 128 x 256 FP32 scores in tensor memory, two accumulators
//     (all 512 columns) so the epilogue of one tile overlaps the MMAs of the
//     next.
//   * Warp 0 issues the TMA loads, warp 1 (one thread) issues tcgen05.mma,
//     warps 2-9 are the epilogue, two per TMEM lane quarter: a thread owns
//     one query of the tile (its TMEM lane) and one half of each tile's 256
//     columns, reads its 128 scores with tcgen05.ld and keeps its 8 or 16
//     best (score, row) pairs in registers, tested against a running
//     threshold with one max per 64 scores in the common case. Blocks share
//     per query the k-th best score seen so far minus twice the error bound,
//     below which no row can reach the top k; lanes with candidates insert
//     them together.
//   * FP8 scores are acc * s_row * s_query (per-vector scales, Sec. 4.2's
//     cosine of the dequantised vectors); BF16 scores are acc itself.
//
// Work items (query tile, row chunk) are claimed one at a time from a global
// counter by the TMA thread, which passes each to the MMA thread and the
// epilogue warps through a small queue in shared memory, so blocks that
// drew short items take more of them (items differ in size when databases
// do). Pairs of CTAs take a fixed round-robin order instead, which both CTAs
// of a pair know without talking. Items of one chunk are numbered
// consecutively so concurrently running blocks share its rows in L2. Every wait is bounded; a wait that gives up marks the launch
// failed (status word), and all roles then leave their loops, wait for their
// own outstanding copies and MMAs (bounded), free TMEM and return.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "fs_internal.cuh"
#include "tc_ptx.cuh"

namespace fsk {

namespace {

using namespace tc;

constexpr int kEpiWarps = 8;                // two per TMEM lane quarter
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = 64 + kEpiThreads;  // + TMA warp + MMA warp
constexpr int BM = 128;                     // queries per tile (MMA M)
constexpr int BN = kTcTileRows;             // database rows per tile (MMA N)
constexpr int kMaxStages = 16;              // ring slots (as many as shared memory holds)
constexpr uint32_t kStageBytes = BN * 128;  // one 128-byte K block of BN rows
constexpr uint32_t kABlockBytes = BM * 128; // one 128-byte K block of BM queries
constexpr int kMaxKBlocks = 4;              // 256 BF16 or 512 FP8 features
constexpr int kAccs = 512 / BN;              // accumulators in tensor memory
constexpr uint32_t kTmemCols = kAccs * BN;
constexpr int kItemQ = 4;                   // claimed items handed on, at most
constexpr int kBandGrab = 16;               // FP8 band slots a thread reserves at once
static_assert(kBandGrab >= 8, "a reservation holds a whole group of 8 rows");

struct Bars {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t tmem_full[kAccs];
    uint64_t tmem_empty[kAccs];
    uint64_t a_full;
    uint64_t a_empty;
    uint64_t drain;
    uint64_t item_full[kItemQ]; // a claimed item (or the end, -1) is in item_q
    uint64_t item_empty[kItemQ];// the MMA thread and every epilogue warp have read it
};

// The TMA thread claims the n-th item of this CTA and hands it on (-1: no
// items left). False when a wait gave up.
__device__ __forceinline__ bool claim_item(Bars& bars, volatile int32_t* item_q,
                                           const CallView& call, uint32_t n,
                                           volatile int* abort_flag, uint64_t wlim, int64_t& item) {
    const uint32_t slot = n % kItemQ, ph = (n / kItemQ) & 1;
    if (!mbar_wait(smem_u32(&bars.item_empty[slot]), ph ^ 1, abort_flag, wlim)) return false;
    int32_t v = atomicAdd(call.work_counter, 1);
    if ((int64_t)v >= call.total_items) v = -1;
    item_q[slot] = v;
    mbar_arrive(smem_u32(&bars.item_full[slot]));
    item = v;
    return true;
}

// Another role reads the n-th item; the caller then arrives on
// item_empty[n % kItemQ] (once per thread or warp counted there).
__device__ __forceinline__ bool take_item(Bars& bars, const volatile int32_t* item_q, uint32_t n,
                                          volatile int* abort_flag, uint64_t wlim, int64_t& item) {
    const uint32_t slot = n % kItemQ, ph = (n / kItemQ) & 1;
    if (!mbar_wait(smem_u32(&bars.item_full[slot]), ph, abort_flag, wlim)) return false;
    item = item_q[slot];
    return true;
}

__device__ __forceinline__ int find_plan(const SegPlan* plan, int n_seg, int64_t item) {
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (plan[mid].item0 <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct Item {
    SegPlan p;
    int chunk, qtile, qbase, nq_tile, ntiles;
    int64_t row_begin, row_end;
};

// An item is (unit, row chunk), units numbered fastest. A unit is one query
// tile, or with pairs of CTAs two query tiles, this CTA's being 2u + rank (a
// pair's second tile may lie past the segment's queries: then every query of
// it is invalid and only the other tile's results are kept).
__device__ __forceinline__ Item decode(const CallView& call, int64_t item, uint32_t rank, bool pair) {
    Item it;
    it.p = call.plan[find_plan(call.plan, call.n_seg, item)];
    const int64_t local = item - it.p.item0;
    it.chunk = (int)(local / it.p.units);
    const int u = (int)(local % it.p.units);
    it.qtile = pair ? 2 * u + (int)rank : u;
    it.qbase = it.p.q0 + it.qtile * BM;
    it.nq_tile = min(BM, it.p.nq - it.qtile * BM);
    it.row_begin = it.p.row0 + (int64_t)it.chunk * it.p.chunk_rows;
    it.row_end = min(it.p.row0 + it.p.nrows, it.row_begin + it.p.chunk_rows);
    it.ntiles = (int)ceil_div(it.row_end - it.row_begin, BN);
    return it;
}

// A bounded wait that ignores the abort flag (used to drain on the way out).
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity, uint64_t wlim) {
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > wlim) break;
}

// A spin of about `ns` nanoseconds (the pair path's grace period for its own
// copies on the way out, see below).
__device__ __forceinline__ void spin_ns(uint64_t ns) {
    const uint64_t t0 = globaltimer();
    while (globaltimer() - t0 < ns) {
    }
}

// PAIR: a cluster of two CTAs shares every tile (cta_group::2). Each CTA
// loads its own 128 queries and its own half (128 rows) of each tile's rows
// into its own shared memory, and both CTAs' copies signal the barriers of
// the even CTA ("leader"), which expects the bytes of both; the leader issues
// M = 256 MMAs over both, and each CTA's tensor memory receives its queries'
// 128 x 256 scores. The leader's commits reach the barriers of both CTAs (a
// CTA refills a ring slot once its own copy of the commit arrives); the odd
// CTA's epilogue frees an accumulator with an arrival on the leader's
// barrier.
template <bool FP8, int LT, bool PAIR>
__global__ void __launch_bounds__(kThreads, 1)
k_scan_tc(DbView db, CallView call, const __grid_constant__ CUtensorMap map_q,
          const __grid_constant__ CUtensorMap map_x, int kblocks, int stages) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ Bars bars;
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    __shared__ int32_t item_q[kItemQ];
    // FP8: per epilogue warp, the row scales and residual norms of its half of
    // the current tile, and per group of 8 rows the largest residual (each
    // warp stages its own copy: no barrier across warps)
    __shared__ __align__(16) float wsx[kEpiWarps][BN / 2];
    __shared__ __align__(16) float wrx[kEpiWarps][BN / 2];
    __shared__ float wgrx[kEpiWarps][BN / 16];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t a_smem = base;
    const uint32_t b_smem = a_smem + kblocks * kABlockBytes;
    constexpr int kElemsPerKBlock = FP8 ? 128 : 64;
    constexpr uint32_t kBStage = PAIR ? kStageBytes / 2 : kStageBytes;   // bytes this CTA loads
    constexpr uint32_t kM = PAIR ? 2 * BM : BM;
    const uint32_t idesc = FP8 ? instr_desc(0, kM, BN) : instr_desc(1, kM, BN);
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const bool leader = rank == 0;
    const int64_t unit0 = PAIR ? blockIdx.x / 2 : blockIdx.x;
    const int64_t nunits = PAIR ? gridDim.x / 2 : gridDim.x;
    constexpr uint16_t kPairMask = 0x3;
    const uint64_t wlim = call.wait_ns ? call.wait_ns : kWaitLimitNs;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&bars.full[s]), 1);
            mbar_init(smem_u32(&bars.empty[s]), 1);
        }
        for (int a = 0; a < kAccs; ++a) {
            mbar_init(smem_u32(&bars.tmem_full[a]), 1);
            mbar_init(smem_u32(&bars.tmem_empty[a]), (PAIR ? 2 : 1) * kEpiWarps);
        }
        mbar_init(smem_u32(&bars.a_full), 1);
        mbar_init(smem_u32(&bars.a_empty), 1);
        mbar_init(smem_u32(&bars.drain), 1);
        for (int i = 0; i < kItemQ; ++i) {
            mbar_init(smem_u32(&bars.item_full[i]), 1);
            mbar_init(smem_u32(&bars.item_empty[i]), 1 + kEpiWarps);
        }
        fence_barrier_init();
    }
    if (warp == 0) {
        if (PAIR)
            tmem_alloc_pair(smem_u32(&tmem_holder), kTmemCols);
        else
            tmem_alloc(smem_u32(&tmem_holder), kTmemCols);
    }
    tc_fence_before();
    __syncthreads();
    // the peer's barriers are initialised before any arrival can reach them
    if (PAIR) cluster_sync();
    tc_fence_after();
    const uint32_t tmem_base = tmem_holder;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            prefetch_tensormap(&map_q);
            prefetch_tensormap(&map_x);
            // pairs: the leader's query-tile and ring barriers (cluster addresses)
            const uint32_t lead_a_full = PAIR ? mapa_shared(smem_u32(&bars.a_full), 0) : 0u;
            const uint32_t lead_full0 = PAIR ? mapa_shared(smem_u32(&bars.full[0]), 0) : 0u;
            (void)lead_a_full;
            (void)lead_full0;
            uint32_t it = 0, ic = 0, a_loads = 0;
            // ring slot and phase of iteration `it`, advanced by a compare rather
            // than it % stages and it / stages: this thread (and the MMA thread)
            // paces the whole pipeline, and the two integer divisions by the run-time
            // ring depth per slot kept the scan at 0.77 of the measured BF16 peak
            // (0.95 without them, on 2,097,152 rows x 256 features)
            uint32_t s_next = 0, ph_next = 0;
            bool ok = true;
            for (uint32_t n = 0; ok; ++n, ++ic) {
                int64_t item = unit0 + (int64_t)n * nunits;
                if (PAIR) {
                    if (item >= call.total_items) break;
                } else {
                    ok = claim_item(bars, item_q, call, n, &abort_flag, wlim, item);
                    if (!ok || item < 0) break;
                }
                const Item w = decode(call, item, rank, PAIR);
                ok = mbar_wait(smem_u32(&bars.a_empty), (ic & 1) ^ 1, &abort_flag, wlim);
                if (!ok) break;
                if (PAIR) {
                    // the leader's barrier counts the query tiles of both CTAs
                    if (leader)
                        mbar_arrive_expect_tx(smem_u32(&bars.a_full), 2 * kblocks * kABlockBytes);
                    for (int kb = 0; kb < kblocks; ++kb)
                        tma_load_2d_pair(a_smem + kb * kABlockBytes, &map_q, lead_a_full,
                                         kb * kElemsPerKBlock, w.qbase);
                } else {
                    mbar_arrive_expect_tx(smem_u32(&bars.a_full), kblocks * kABlockBytes);
                    for (int kb = 0; kb < kblocks; ++kb)
                        tma_load_2d(a_smem + kb * kABlockBytes, &map_q, smem_u32(&bars.a_full),
                                    kb * kElemsPerKBlock, w.qbase);
                }
                ++a_loads;
                for (int t = 0; ok && t < w.ntiles; ++t) {
                    // this CTA's rows of the tile: all 256, or its half of them
                    const int32_t row =
                        (int32_t)(w.row_begin + (int64_t)t * BN + (PAIR ? rank * (BN / 2) : 0));
                    for (int kb = 0; kb < kblocks; ++kb, ++it) {
                        const uint32_t s = s_next, ph = ph_next;
                        if (++s_next == (uint32_t)stages) {
                            s_next = 0;
                            ph_next ^= 1;
                        }
                        ok = mbar_wait(smem_u32(&bars.empty[s]), ph ^ 1, &abort_flag, wlim);
                        if (!ok) break;
                        // test aid: the first ring slot is never filled, so the MMA
                        // issuer's wait for it runs out (nothing is left in flight)
                        if (call.withhold_load && it == 0) continue;
                        if (PAIR) {
                            if (leader) mbar_arrive_expect_tx(smem_u32(&bars.full[s]), 2 * kBStage);
                            tma_load_2d_pair(b_smem + s * kBStage, &map_x,
                                             lead_full0 + s * (uint32_t)sizeof(uint64_t),
                                             kb * kElemsPerKBlock, row);
                        } else {
                            mbar_arrive_expect_tx(smem_u32(&bars.full[s]), kBStage);
                            tma_load_2d(b_smem + s * kBStage, &map_x, smem_u32(&bars.full[s]),
                                        kb * kElemsPerKBlock, row);
                        }
                    }
                }
            }
            if (!ok && PAIR) {
                // A pair's copies signal the leader's barriers, which the odd CTA
                // cannot wait on: both CTAs leave their copies in flight a grace
                // period to land (a tile copy takes microseconds; the wait that
                // gave up took far longer).
                spin_ns(200000);
            } else if (!ok) {
                // let the copies already issued land before the block exits (the
                // withheld slot, if any, has nothing to wait for)
                for (uint32_t j = (it >= (uint32_t)stages ? it - stages : 0); j < it; ++j)
                    if (!(call.withhold_load && j == 0))
                        drain_wait(smem_u32(&bars.full[j % stages]), (j / stages) & 1, wlim);
                if (a_loads > 0) drain_wait(smem_u32(&bars.a_full), (a_loads - 1) & 1, wlim);
            }
        }
    } else if (warp == 1 && (!PAIR || leader)) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t tcount = 0, ic = 0;
            uint32_t s_next = 0, ph_next = 0;   // ring slot and phase of the next K block
            bool ok = true;
            // Shared-memory descriptors built once and advanced by addition: the
            // start-address field is the byte address / 16 in the low 14 bits, and
            // every operand lies below 256 KB, so an added offset / 16 never carries
            // into the other fields (fewer instructions between MMAs on the one
            // thread that issues them all)
            const uint64_t ad_base = sw128_kmajor_desc(a_smem);
            const uint64_t bd_base = sw128_kmajor_desc(b_smem);
            auto commit = [&](uint64_t& bar) {
                if (PAIR)
                    mma_commit_pair(smem_u32(&bar), kPairMask);
                else
                    mma_commit(smem_u32(&bar));
            };
            for (uint32_t n = 0; ok; ++n, ++ic) {
                int64_t item = unit0 + (int64_t)n * nunits;
                if (PAIR) {
                    if (item >= call.total_items) break;
                } else {
                    ok = take_item(bars, item_q, n, &abort_flag, wlim, item);
                    if (!ok) break;
                    mbar_arrive(smem_u32(&bars.item_empty[n % kItemQ]));
                    if (item < 0) break;
                }
                const Item w = decode(call, item, rank, PAIR);
                ok = mbar_wait(smem_u32(&bars.a_full), ic & 1, &abort_flag, wlim);
                if (!ok) break;
                tc_fence_after();
                for (int t = 0; ok && t < w.ntiles; ++t, ++tcount) {
                    const uint32_t acc = tcount % kAccs, aph = (tcount / kAccs) & 1;
                    ok = mbar_wait(smem_u32(&bars.tmem_empty[acc]), aph ^ 1, &abort_flag, wlim);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t d = tmem_base + acc * BN;
                    for (int kb = 0; kb < kblocks; ++kb) {
                        const uint32_t s = s_next, ph = ph_next;
                        if (++s_next == (uint32_t)stages) {
                            s_next = 0;
                            ph_next ^= 1;
                        }
                        ok = mbar_wait(smem_u32(&bars.full[s]), ph, &abort_flag, wlim);
                        if (!ok) break;
                        tc_fence_after();
                        const uint64_t adk = ad_base + (uint64_t)((kb * kABlockBytes) >> 4);
                        const uint64_t bds = bd_base + (uint64_t)((s * kBStage) >> 4);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t ad = adk + 2 * ks;
                            const uint64_t bd = bds + 2 * ks;
                            if (PAIR) {
                                if (FP8)
                                    mma_f8_pair(d, ad, bd, idesc, (kb | ks) != 0);
                                else
                                    mma_f16_pair(d, ad, bd, idesc, (kb | ks) != 0);
                            } else {
                                if (FP8)
                                    mma_f8(d, ad, bd, idesc, (kb | ks) != 0);
                                else
                                    mma_f16(d, ad, bd, idesc, (kb | ks) != 0);
                            }
                        }
                        commit(bars.empty[s]);
                    }
                    if (ok) commit(bars.tmem_full[acc]);
                }
                if (ok) commit(bars.a_empty);
            }
            // every MMA this thread issued has finished before TMEM is freed
            commit(bars.drain);
            drain_wait(smem_u32(&bars.drain), 0, wlim);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ odd CTA of a pair
        // the leader's last commit: every MMA writing this CTA's TMEM is done
        if (lane == 0) drain_wait(smem_u32(&bars.drain), 0, wlim);
    } else {
        // ------------------------------------------------ epilogue
        const int quarter = warp & 3;              // TMEM lanes this warp may read
        const int lq = quarter * 32 + lane;        // query row of the tile
        const int half = (warp - 2) >> 2;          // which half of each tile's columns
        const int ew = warp - 2;                   // epilogue warp 0..7
        constexpr int kHalfCols = BN / 2;
        uint32_t tcount = 0;
        bool ok = true;
        // the barrier that frees an accumulator: the leader's
        const uint32_t r_tmem_empty0 =
            PAIR ? mapa_shared(smem_u32(&bars.tmem_empty[0]), 0) : smem_u32(&bars.tmem_empty[0]);
        for (uint32_t n = 0; ok; ++n) {
            int64_t item = unit0 + (int64_t)n * nunits;
            if (PAIR) {
                if (item >= call.total_items) break;
            } else {
                ok = take_item(bars, item_q, n, &abort_flag, wlim, item);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bars.item_empty[n % kItemQ]));
                if (item < 0) break;
            }
            const Item w = decode(call, item, rank, PAIR);
            // A zero query scores 0 against every row, so every row would tie at
            // its list threshold and be offered; the selection answers it from
            // row indices alone (the lowest ones, d = 1), so it is not scanned.
            const bool qvalid = lq < w.nq_tile && call.q_ss[w.qbase + lq] != 0.0f;
            const int excl = (call.exclude && qvalid) ? call.exclude[w.qbase + lq] : -1;
            const float sq = FP8 ? (qvalid ? call.q_scale[w.qbase + lq] : 0.0f) : 1.0f;
            const float rq = qvalid ? call.q_resid[w.qbase + lq] : 0.0f;
            // BF16: the list of the LT best (score, row) pairs. FP8: the LT best
            // per-group lower bounds g = s - b r_x of the rows seen (rows unused).
            RegList<LT> st;
            st.reset();

            float published = -INFINITY;
            // Pruning bound shared by every block scanning this query. BF16: the
            // k-th best approximate score any block has seen, minus twice the
            // score error bound E; a row scoring below it is at least 2E under k
            // rows' scores, so its cosine is below theirs: it cannot be among the
            // k nearest, and dropping it never affects certification. FP8: the
            // k-th best lower bound s - E_x any block has seen (E_x the row's own
            // bound); a row whose upper bound s + E_x is below it cannot be among
            // the k nearest. Read one tile ahead so the L2 round trip overlaps
            // the current tile.
            const float e2 = qvalid ? 2.0f * (w.p.bound_scan + w.p.bound_rq * rq) * 1.0001f : 0.0f;
            // FP8 per-row bound E_x = fa + fb r_x, each coefficient a little above
            // the selection's binary64 one (a = bound_scan + bound_rq r_q,
            // b = 1.001 (bound_rx + r_q)), so FP32 rounding here never drops a row
            // the selection's test would keep
            const float fa = (w.p.bound_scan + w.p.bound_rq * rq) * 1.0001f;
            const float fb = (w.p.bound_rx + rq) * 1.0011f;
            // FP8: the shared bound is the least of k class slots (the rows are
            // split into k classes by a fixed hash of the local row): each slot
            // holds the best lower bound of a band row of its class, so k distinct
            // band rows reach the least of them (0 = a class without one yet: no
            // bound)
            const uint32_t* shared_p =
                FP8 ? call.class_thr + (int64_t)(w.qbase + lq) * FS_MAX_K : call.shared_thr + w.qbase + lq;
            auto read_shared = [&]() -> uint32_t {
                if (!FP8) return __ldcg(shared_p);
                uint32_t mn = 0xffffffffu;
                for (int c = 0; c < w.p.k; ++c) mn = min(mn, __ldcg(shared_p + c));
                return mn;
            };
            uint32_t shared_next = qvalid ? read_shared() : 0xffffffffu;
            // FP8: per class, the best lower bound g of this list's band rows,
            // and which classes improved since the last publication
            float cbest[LT];
#pragma unroll
            for (int c = 0; c < LT; ++c) cbest[c] = -INFINITY;
            uint32_t cdirty = 0;
            // FP8: this query's band (rows whose upper bound reaches the running
            // k-th best lower bound). The thread appends into slots it reserves
            // kBandGrab at a time from the query's counter, so the returning
            // atomic is paid once per reservation rather than once per group;
            // a reservation's unused slots are written as empty keys (0)
            uint64_t* band = nullptr;
            int32_t* band_cnt = nullptr;
            int res_at = 0, res_end = 0;   // this thread's reserved slots
            if (FP8 && qvalid) {
                band = call.band + w.p.band0 + ((int64_t)w.qtile * BM + lq) * w.p.band_cap;
                band_cnt = call.band_cnt + w.qbase + lq;
            }
            for (int t = 0; t < w.ntiles; ++t, ++tcount) {
                const uint32_t acc = tcount % kAccs, aph = (tcount / kAccs) & 1;
                const int64_t tile_row0 = w.row_begin + (int64_t)t * BN;
                const float shared_s = qvalid ? unord_f32(shared_next) : INFINITY;
                if (qvalid && t + 1 < w.ntiles) shared_next = read_shared();
                // FP8: the scales and residual norms of this warp's half of the
                // tile, loaded before the wait for the accumulator (lane l: the
                // half's columns l, l + 32, l + 64, l + 96; rows past the data: 0)
                constexpr int kStage32 = kHalfCols / 32;   // 32-column slices of the half
                float pre_s[kStage32], pre_r[kStage32];
                if (FP8) {
#pragma unroll
                    for (int i = 0; i < kStage32; ++i) {
                        const int64_t r = tile_row0 + half * kHalfCols + 32 * i + lane;
                        const bool in = r < w.row_end;
                        pre_s[i] = in ? db.scale[r] : 0.0f;
                        pre_r[i] = in ? db.resid[r] : 0.0f;
                    }
                }
                ok = mbar_wait(smem_u32(&bars.tmem_full[acc]), aph, &abort_flag, wlim);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc_fence_after();
                if (FP8) {
                    // staged for this warp alone (its previous tile is done: every
                    // lane passed the __syncwarp at its end)
#pragma unroll
                    for (int i = 0; i < kStage32; ++i) {
                        wsx[ew][32 * i + lane] = pre_s[i];
                        wrx[ew][32 * i + lane] = pre_r[i];
                        float rmax = pre_r[i];
#pragma unroll
                        for (int o = 1; o < 8; o <<= 1)
                            rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
                        if ((lane & 7) == 0) wgrx[ew][4 * i + (lane >> 3)] = rmax;
                    }
                    __syncwarp();
                }
                const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * BN;
                bool offered = false;   // the list may have changed in this tile
                // FP8 threshold on h = s + fb r_x (the upper bound minus fa)
                const float shared_h = shared_s - fa;
                // The thread's columns in chunks of 32, software-pipelined
                // through two register buffers: the next chunk's TMEM load is in
                // flight while this chunk is filtered, and the accumulator is freed
                // as soon as the last chunk has landed, before it is filtered.
                constexpr int kCW = 32, kCG = kCW / 8;
                constexpr int kChunks = kHalfCols / kCW;
                static_assert(kHalfCols % (2 * kCW) == 0, "an even number of chunks per half tile");
                auto release = [&]() {
                    // every TMEM load of this tile has landed (tcgen05.wait::ld)
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        const uint32_t bar = r_tmem_empty0 + acc * (uint32_t)sizeof(uint64_t);
                        if (PAIR && !leader)
                            mbar_arrive_cluster(bar);
                        else
                            mbar_arrive(bar);
                    }
                };
                auto filter = [&](const uint32_t (&rbuf)[kCW], const int c0) {
                        // FP8: v = acc * s_row (the codes are unit elements divided by
                        // their row's scale, so the row scale belongs to each score before
                        // any maximum); BF16: v = acc
                        float v[kCW];
    #pragma unroll
                        for (int j = 0; j < kCW; ++j) v[j] = __uint_as_float(rbuf[j]);
                        if (FP8) {
                            // two scores per instruction (mul.rn.f32x2: each lane an
                            // ordinary rounded multiply, the same bits as a scalar one)
                            const ulonglong2* s2 =
                                reinterpret_cast<const ulonglong2*>(&wsx[ew][c0 - half * kHalfCols]);
    #pragma unroll
                            for (int j = 0; j < kCW / 4; ++j) {
                                const ulonglong2 sc = s2[j];
                                uint64_t p0 = ((uint64_t)rbuf[4 * j + 1] << 32) | rbuf[4 * j];
                                uint64_t p1 = ((uint64_t)rbuf[4 * j + 3] << 32) | rbuf[4 * j + 2];
                                asm("mul.rn.f32x2 %0, %0, %1;" : "+l"(p0) : "l"(sc.x));
                                asm("mul.rn.f32x2 %0, %0, %1;" : "+l"(p1) : "l"(sc.y));
                                v[4 * j] = __uint_as_float((uint32_t)p0);
                                v[4 * j + 1] = __uint_as_float((uint32_t)(p0 >> 32));
                                v[4 * j + 2] = __uint_as_float((uint32_t)p1);
                                v[4 * j + 3] = __uint_as_float((uint32_t)(p1 >> 32));
                            }
                        }
                        float gm[kCG];
    #pragma unroll
                        for (int g = 0; g < kCG; ++g) {
                            const float a = fmax3(v[8 * g], v[8 * g + 1], v[8 * g + 2]);
                            const float b = fmax3(v[8 * g + 3], v[8 * g + 4], v[8 * g + 5]);
                            const float mx = fmax3(a, b, fmaxf(v[8 * g + 6], v[8 * g + 7]));
                            if (FP8) {
                                // an upper bound on h over the group: its largest scaled
                                // score times the query scale (a non-negative factor), plus
                                // fb times the group's largest residual; each step rounds
                                // monotonically, so no h of the group exceeds it
                                const int gi = ((c0 - half * kHalfCols) >> 3) + g;
                                gm[g] = fmaf(fb, wgrx[ew][gi], mx * sq);
                            } else {
                                gm[g] = mx;
                            }
                        }
                        static_assert(kCG == 4, "four groups of 8 per chunk");
                        const float m = fmaxf(fmax3(gm[0], gm[1], gm[2]), gm[3]);
                        if (FP8) {
                            // the threshold on h: the larger of two lower bounds on the
                            // k-th best lower bound, each reached by k distinct band rows:
                            // the k-th best of this list (below) and the shared class slots
                            float thr = fmaxf(st.cnt >= w.p.k ? st.kth_score(w.p.k) - 2.0f * fa : -INFINITY,
                                              shared_h);
                            if (__any_sync(0xffffffffu, m >= thr)) {
                                // Group by group (a loop kept rolled: the group's 8 scores
                                // are rotated to the front of v, so the body is compiled
                                // once and stays in the instruction cache):
                                // 1: the group's best lower bound g = s - fb r_x joins the
                                //    list of the LT best (the best of k groups are k
                                //    distinct rows; a group whose bound on h is under thr
                                //    holds no g the list keeps), and the threshold tightens;
                                // 2: the rows whose h = s + fb r_x reaches it are appended
                                //    to the band (the rows behind the list's k best among
                                //    them: their h is at least their g), and their g raise
                                //    their classes' bests.
    #pragma unroll 1
                                for (int g = 0; g < kCG; ++g) {
                                    if (__any_sync(0xffffffffu, gm[0] >= thr)) {
                                        const int lcg = c0 + 8 * g - half * kHalfCols;   // in the half
                                        const int64_t row0g = tile_row0 + c0 + 8 * g;
                                        if (gm[0] >= thr) {
                                            float gbest = -INFINITY;
    #pragma unroll
                                            for (int i = 0; i < 8; ++i) {
                                                const int64_t row = row0g + i;
                                                if (row < w.row_end && (int)(row - w.p.row0) != excl)
                                                    gbest = fmaxf(gbest, fmaf(-fb, wrx[ew][lcg + i], v[i] * sq));
                                            }
                                            st.offer(gbest, 0, 1, 0, -1);
                                            thr = fmaxf(st.cnt >= w.p.k ? st.kth_score(w.p.k) - 2.0f * fa
                                                                        : -INFINITY,
                                                        shared_h);
                                        }
                                        uint32_t bits = 0;
    #pragma unroll
                                        for (int i = 0; i < 8; ++i) {
                                            const float h = fmaf(fb, wrx[ew][lcg + i], v[i] * sq);
                                            const int64_t row = row0g + i;
                                            const bool in = h >= thr && row < w.row_end &&
                                                            (int)(row - w.p.row0) != excl;
                                            bits |= (in ? 1u : 0u) << i;
                                        }
                                        if (bits != 0) {
                                            const int need = __popc(bits);
                                            if (res_end - res_at < need) {
                                                for (int e = res_at; e < res_end && e < w.p.band_cap; ++e)
                                                    band[e] = 0;
                                                res_at = atomicAdd(band_cnt, kBandGrab);
                                                res_end = res_at + kBandGrab;
                                            }
                                            int at = res_at;
                                            res_at += need;
                                            for (uint32_t b = bits; b != 0; b &= b - 1, ++at) {
                                                const int i = __ffs(b) - 1;
                                                // v[i] without a run-time register index
                                                float vi = v[0];
    #pragma unroll
                                                for (int i2 = 1; i2 < 8; ++i2)
                                                    if (i2 == i) vi = v[i2];
                                                const float sc = vi * sq;
                                                const uint32_t li = (uint32_t)(row0g + i - w.p.row0);
                                                if (at < w.p.band_cap) band[at] = make_key(sc, li);
                                                // the best lower bound of its class: a fixed
                                                // map of rows onto k classes (a multiplicative
                                                // hash scaled to [0, k), where li % k would
                                                // divide once per appended row)
                                                const int cls =
                                                    (int)__umulhi(li * 0x9E3779B9u, (uint32_t)w.p.k);
                                                const float gl = fmaf(-fb, wrx[ew][lcg + i], sc);
    #pragma unroll
                                                for (int c = 0; c < LT; ++c)
                                                    if (c == cls && gl > cbest[c]) {
                                                        cbest[c] = gl;
                                                        cdirty |= 1u << c;
                                                    }
                                            }
                                        }
                                    }
                                    // the next group to the front
    #pragma unroll
                                    for (int j = 0; j < kCW - 8; ++j) v[j] = v[j + 8];
    #pragma unroll
                                    for (int j = 0; j < kCG - 1; ++j) gm[j] = gm[j + 1];
                                }
                            }
                        } else {
                            float thr = fmaxf(st.thr_s, shared_s);
                            if (__any_sync(0xffffffffu, m >= thr)) {
                                // group by group, with the threshold as it stands (a list
                                // that is filling tightens after every group): each lane
                                // collects its passing columns of the group, then every
                                // lane takes its next candidate in the same round
    #pragma unroll
                                for (int g = 0; g < kCG; ++g) {
                                    if (__any_sync(0xffffffffu, gm[g] >= thr)) {
                                        uint32_t bits = 0;
    #pragma unroll
                                        for (int i = 0; i < 8; ++i)
                                            bits |= (v[8 * g + i] >= thr ? 1u : 0u) << i;
                                        while (__any_sync(0xffffffffu, bits != 0)) {
                                            if (bits != 0) {
                                                const int i = __ffs(bits) - 1;
                                                bits &= bits - 1;
                                                const float a0 = (i & 1) ? v[8 * g + 1] : v[8 * g];
                                                const float a1 = (i & 1) ? v[8 * g + 3] : v[8 * g + 2];
                                                const float a2 = (i & 1) ? v[8 * g + 5] : v[8 * g + 4];
                                                const float a3 = (i & 1) ? v[8 * g + 7] : v[8 * g + 6];
                                                const float b0 = (i & 2) ? a1 : a0;
                                                const float b1 = (i & 2) ? a3 : a2;
                                                const float sc = (i & 4) ? b1 : b0;
                                                if (sc >= thr) {
                                                    st.offer(sc, tile_row0 + c0 + 8 * g + i, w.row_end,
                                                             w.p.row0, excl);
                                                    thr = fmaxf(st.thr_s, shared_s);
                                                    offered = true;
                                                }
                                            }
                                        }
                                    }
                                }
                            }
                        }
                    __syncwarp();
                };
                if (FP8) {
                    // one buffer (the FP8 filter's own state needs the registers)
#pragma unroll 1
                    for (int cc = 0; cc < kChunks; ++cc) {
                        uint32_t ra[kCW];
                        tmem_ld_32x32b_x32(taddr + half * kHalfCols + cc * kCW, ra);
                        tmem_ld_wait();
                        if (cc == kChunks - 1) release();
                        filter(ra, half * kHalfCols + cc * kCW);
                    }
                } else {
                    uint32_t ra[kCW], rb[kCW];
                    tmem_ld_32x32b_x32(taddr + half * kHalfCols, ra);
                    tmem_ld_wait();
#pragma unroll 1
                    for (int cc = 0; cc < kChunks; cc += 2) {
                        const int c0 = half * kHalfCols + cc * kCW;
                        tmem_ld_32x32b_x32(taddr + c0 + kCW, rb);
                        filter(ra, c0);
                        tmem_ld_wait();
                        if (cc + 2 < kChunks)
                            tmem_ld_32x32b_x32(taddr + c0 + 2 * kCW, ra);
                        else
                            release();
                        filter(rb, c0 + kCW);
                        if (cc + 2 < kChunks) tmem_ld_wait();
                    }
                }
                if (FP8) {
                    // the class slots that improved: g - fa, rounded down (the bound
                    // may only err low)
                    if (qvalid && cdirty != 0) {
#pragma unroll
                        for (int c = 0; c < LT; ++c)
                            if ((cdirty >> c) & 1u)
                                atomicMax(call.class_thr + (int64_t)(w.qbase + lq) * FS_MAX_K + c,
                                          ord_f32((cbest[c] - fa) - fabsf(cbest[c]) * 0x1p-20f));
                    }
                    cdirty = 0;
                } else if (qvalid && offered && st.cnt >= w.p.k) {
                    const float kth = st.kth_score(w.p.k);
                    // rounded down: the bound may only err low
                    const float bound = (kth - e2) - fabsf(kth) * 0x1p-20f;
                    if (bound > published) {
                        atomicMax(call.shared_thr + w.qbase + lq, ord_f32(bound));
                        published = bound;
                    }
                }
            }
            if (FP8 && qvalid) {
                // the unused slots of the last reservation
                for (int e = res_at; e < res_end && e < w.p.band_cap; ++e) band[e] = 0;
            }
            if (!FP8 && ok && qvalid) {
                const int64_t qlocal = (int64_t)w.qtile * BM + lq;
                uint64_t* dst = call.cand + w.p.cand0 +
                                ((qlocal * w.p.chunks + w.chunk) * 2 + half) * (int64_t)LT;
#pragma unroll
                for (int e = 0; e < LT; ++e) dst[e] = st.key(e);
            }
        }
    }

    if (abort_flag && threadIdx.x == 0) {
        atomicOr(db.status, kStTimeout);
        atomicOr(call.aborted, 1);
    }
    tc_fence_before();
    __syncthreads();
    // no arrival or MMA of one CTA of a pair may reach the other after it exits
    if (PAIR) cluster_sync();
    if (warp == 0) {
        tc_fence_after();
        if (PAIR)
            tmem_dealloc_pair(tmem_base, kTmemCols);
        else
            tmem_dealloc(tmem_base, kTmemCols);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

}  // namespace

// Dynamic shared memory of a launch: the alignment slack, the query tile
// (kblocks K blocks) and `stages` ring slots (half a tile's rows per slot
// with pairs of CTAs).
size_t scan_tc_smem_bytes(int kblocks, int stages, bool pair) {
    return 1024 + (size_t)kblocks * kABlockBytes +
           (size_t)stages * (pair ? kStageBytes / 2 : kStageBytes);
}

// As many ring slots as fit next to the query tile and the static shared
// memory (barriers, FP8 scale staging), between 2 and kMaxStages.
int scan_tc_stages(int kblocks, bool fp8, bool pair) {
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 232448;
    const size_t static_bytes =
        sizeof(Bars) + 64 + (fp8 ? (2 * kEpiWarps * (BN / 2) + kEpiWarps * (BN / 16)) * sizeof(float) : 0);
    const long avail = (long)optin - (long)static_bytes - 1024 - (long)kblocks * kABlockBytes;
    int st = (int)(avail / (long)(pair ? kStageBytes / 2 : kStageBytes));
    return st < 2 ? 2 : (st > kMaxStages ? kMaxStages : st);
}

// 2-D tensor map of a row-major [rows][cols] array of 1- or 2-byte codes,
// boxes of (128 bytes) x box_rows, 128-byte swizzle.
cudaError_t make_code_map(CUtensorMap* map, const void* ptr, int64_t rows, int cols, int elem_bytes,
                          int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * elem_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(map, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                     2, const_cast<void*>(ptr), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Raises the kernel's dynamic shared-memory limit to `smem` on the current
// device. The attribute belongs to that device's context, so the largest
// size set so far is remembered per device.
template <bool FP8, int LT, bool PAIR>
cudaError_t set_smem(size_t smem) {
    static std::mutex mu;
    static size_t attr_bytes[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    size_t* have = (dev >= 0 && dev < kMaxDevices) ? &attr_bytes[dev] : nullptr;
    if (have && smem <= *have) return cudaSuccess;
    e = cudaFuncSetAttribute(k_scan_tc<FP8, LT, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e == cudaSuccess && have) *have = smem;
    return e;
}

template <bool FP8, int LT, bool PAIR>
cudaError_t launch_variant(const DbView& db, const CallView& call, const CUtensorMap& map_q,
                           const CUtensorMap& map_x, int grid, int kblocks, cudaStream_t st) {
    const int stages = scan_tc_stages(kblocks, FP8, PAIR);
    const size_t smem = scan_tc_smem_bytes(kblocks, stages, PAIR);
    cudaError_t e = set_smem<FP8, LT, PAIR>(smem);
    if (e != cudaSuccess) return e;
    if (!PAIR) {
        k_scan_tc<FP8, LT, false><<<grid, kThreads, smem, st>>>(db, call, map_q, map_x, kblocks,
                                                                 stages);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_scan_tc<FP8, LT, PAIR>, db, call, map_q, map_x, kblocks,
                              stages);
}

template <bool PAIR>
cudaError_t launch_lists(bool fp8, int list_t, const DbView& db, const CallView& call,
                         const CUtensorMap& map_q, const CUtensorMap& map_x, int grid, int kblocks,
                         cudaStream_t st) {
    if (list_t == kListTTiny)
        return fp8 ? launch_variant<true, kListTTiny, PAIR>(db, call, map_q, map_x, grid, kblocks, st)
                   : launch_variant<false, kListTTiny, PAIR>(db, call, map_q, map_x, grid, kblocks, st);
    if (list_t == kListTSmall)
        return fp8 ? launch_variant<true, kListTSmall, PAIR>(db, call, map_q, map_x, grid, kblocks, st)
                   : launch_variant<false, kListTSmall, PAIR>(db, call, map_q, map_x, grid, kblocks, st);
    if (list_t == kListT)
        return fp8 ? launch_variant<true, kListT, PAIR>(db, call, map_q, map_x, grid, kblocks, st)
                   : launch_variant<false, kListT, PAIR>(db, call, map_q, map_x, grid, kblocks, st);
    return cudaErrorInvalidValue;
}

// Pairs of CTAs that can be resident at once (a cluster occupies two SMs of
// one GPU processing cluster; not every SM need find a partner), 0 on error.
int scan_tc_pair_slots(bool fp8, int kblocks) {
    static std::mutex mu;
    static int cached[kMaxDevices][2][kMaxKBlocks + 1] = {};   // per device
    if (kblocks < 1 || kblocks > kMaxKBlocks) return 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
    std::lock_guard<std::mutex> g(mu);
    int& c = cached[dev][fp8 ? 1 : 0][kblocks];
    if (c > 0) return c;
    const int stages = scan_tc_stages(kblocks, fp8, true);
    const size_t smem = scan_tc_smem_bytes(kblocks, stages, true);
    cudaError_t e = fp8 ? set_smem<true, kListTSmall, true>(smem) : set_smem<false, kListTSmall, true>(smem);
    if (e != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    e = fp8 ? cudaOccupancyMaxActiveClusters(&n, k_scan_tc<true, kListTSmall, true>, &cfg)
            : cudaOccupancyMaxActiveClusters(&n, k_scan_tc<false, kListTSmall, true>, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    c = n;
    return c;
}

cudaError_t launch_scan_tc(const DbView& db, const CallView& call, const CUtensorMap& map_q,
                           const CUtensorMap& map_x, int grid, int list_t, bool pair,
                           cudaStream_t st) {
    if (call.total_items == 0) return cudaSuccess;
    const bool fp8 = db.prec == FS_FP8_E4M3;
    const int kblocks = (int)(db.fl * (fp8 ? 1 : 2) / 128);
    if (kblocks < 1 || kblocks > kMaxKBlocks) return cudaErrorInvalidValue;
    if (pair && (grid & 1)) return cudaErrorInvalidValue;
    return pair ? launch_lists<true>(fp8, list_t, db, call, map_q, map_x, grid, kblocks, st)
                : launch_lists<false>(fp8, list_t, db, call, map_q, map_x, grid, kblocks, st);
}

}  // namespace fsk
