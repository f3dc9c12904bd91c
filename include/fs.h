/*
 * fs.h - feature-similarity phase-order suggestion on one GB300 (sm_103a).
 *
 * The operation (Nobre, Reis and Cardoso, "Improving OpenCL Performance by
 * Specializing Compiler Phase Selection and Ordering", Sec. 4 and 4.2):
 * given the code-feature vector of a new kernel, compute its cosine distance
 * to every kernel of a reference database, select the K most similar
 * (k-nearest neighbours) and return the best phase orders that were found
 * for those neighbours (Table 1). Sec. 4.2 also fixes the protocol in which
 * the query's own entry is left out of the database (leave-one-out).
 *
 * Result contract, identical for every precision:
 *   s(q, x) = D / sqrt(A * B) with D = sum q_i x_i, A = sum q_i^2,
 *   B = sum x_i^2, each summed in binary64 for i = 0..F-1 in order with
 *   every product rounded before it is added; s = 0 when A or B is 0.
 *   Neighbours are ranked by s descending, the lower database index first on
 *   equal s; the reported distance is d = 1 - s rounded to float.
 * The lower-precision scans (BF16, FP8 E4M3) only pick candidates; a
 * certified rerank returns exactly the binary64 ranking above.
 *
 * Conventions for every call:
 *   - Pointers documented as "device" are CUDA device pointers owned by the
 *     caller; "host" pointers are read during the call only.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Calls that
 *     launch work are asynchronous with respect to the host.
 *   - Arguments are checked on the host before anything is launched; a bad
 *     argument returns FS_EINVAL and launches nothing. No C++ exception
 *     crosses this interface.
 *   - Errors found on the device (a non-finite or out-of-range feature, an
 *     overflowing internal list, a bounded wait that gave up) are recorded in
 *     a status word of the database and returned by fs_db_check().
 *   - fs_last_error() gives a message for the last failing call of the
 *     calling thread.
 *   - Database indices are local to their segment (0-based). When k exceeds
 *     the rows available, the extra slots get index -1, distance +inf,
 *     length 0 and an order of -1 values.
 */
#ifndef FS_H
#define FS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FS_OK = 0,
    FS_EINVAL = 1,        /* bad argument (nothing launched) */
    FS_ENOMEM = 2,        /* device allocation failed or workspace too small */
    FS_ECUDA = 3,         /* a CUDA runtime call failed */
    FS_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    FS_EUNSUPPORTED = 5   /* valid but outside what this build supports */
} fs_status;

/* Arithmetic of the database scan. The result contract does not change. */
typedef enum {
    FS_FP32 = 0,          /* FP32 SIMT scan of unit vectors */
    FS_BF16 = 1,          /* tcgen05 kind::f16 scan of BF16 unit vectors */
    FS_FP8_E4M3 = 2       /* tcgen05 kind::f8f6f4 scan, per-vector scales */
} fs_precision;

typedef struct fs_db fs_db;   /* opaque; owns its device arrays */

#define FS_MAX_K 16           /* largest k (the paper sweeps K = 1..14) */
#define FS_MAX_F 1024         /* largest feature count, FP32 scan */
#define FS_MAX_F_TC 256       /* largest feature count, BF16/FP8 scans */
#define FS_MAX_SEGMENTS 65535 /* largest number of independent databases */

/* Counters the library keeps per database (since build or the last reset). */
typedef struct {
    uint64_t queries;           /* queries answered */
    uint64_t certified;         /* answered from the scan's candidate lists */
    uint64_t fallback;          /* re-answered by the exact binary64 scan */
    uint64_t fp64_evals;        /* (query, row) pairs scored in binary64 */
    uint64_t near_ties;         /* binary64 evaluations beyond k (near ties) */
    uint64_t rerank_evals;      /* (query, row) pairs rescored in FP32 */
    uint64_t band_rows;         /* FP8: band slots the scan filled or reserved (rows kept, plus
                                   the unused slots of each scan thread's last reservation) */
} fs_stats;

/*
 * fs_normalize - unit vectors for the cosine (Sec. 4.2).
 *   x        device, float[n][ld], row-major; row r is x[r*ld .. r*ld+f-1]
 *   n        rows (>= 0);  f  features (1..FS_MAX_F);  ld >= f
 *   x_unit   device, float[n][f], dense: x_unit[r] = x[r] / ||x[r]||_2
 *            (all zeros when x[r] is all zeros)
 *   inv_norm device, float[n] or NULL: 1/||x[r]||_2 (0 for a zero row)
 * Norms are summed in FP32. A row holding a non-finite value comes out as
 * NaN in x_unit and inv_norm, so the caller can detect it.
 */
fs_status fs_normalize(const float *x, int64_t n, int32_t f, int64_t ld,
                       float *x_unit, float *inv_norm, void *stream);

/*
 * fs_build_db - copy a reference set of feature vectors and phase orders
 * to the device and prepare it for search (Sec. 4, Table 1).
 *   x        device, float[n][f] dense: one feature vector per explored
 *            kernel. Each value must be finite and either 0 or of magnitude
 *            in [2^-40, 2^50] (else FS_EINVAL).
 *   seq_off  device, int64[n+1]: row r's phase order is
 *            seq_ids[seq_off[r] .. seq_off[r+1]); seq_off[0] = 0,
 *            non-decreasing. Empty orders (equal offsets) are legal.
 *   seq_ids  device, int16[seq_off[n]]: pass IDs, each >= 0.
 *   seg_off  host, int64[n_seg+1] or NULL: independent databases; segment s
 *            holds rows seg_off[s] .. seg_off[s+1]-1 (seg_off[0] = 0,
 *            seg_off[n_seg] = n, non-decreasing). NULL means one segment.
 *   n_seg    number of segments (1 when seg_off is NULL).
 *   prec     scan arithmetic (FS_BF16 / FS_FP8_E4M3 need f <= FS_MAX_F_TC).
 *   out      receives the database handle (NULL on failure).
 * The call synchronises `stream` once (to validate the inputs and read the
 * size of seq_ids). The database is read-only afterwards and may be searched
 * from several streams at once.
 */
fs_status fs_build_db(const float *x, int64_t n, int32_t f,
                      const int64_t *seq_off, const int16_t *seq_ids,
                      const int64_t *seg_off, int32_t n_seg,
                      fs_precision prec, void *stream, fs_db **out);

/*
 * fs_workspace_size - bytes of device workspace fs_knn/fs_recommend need.
 *   nq, q_seg_off  as in fs_knn;  bytes  host, receives the size.
 */
fs_status fs_workspace_size(const fs_db *db, int32_t nq,
                            const int32_t *q_seg_off, size_t *bytes);

/*
 * fs_knn - the k most similar database rows of each query (Sec. 4, 4.2).
 *   q          device, float[nq][f] dense query feature vectors
 *   nq         queries (>= 0)
 *   q_seg_off  host, int32[n_seg+1] or NULL: queries q_seg_off[s] ..
 *              q_seg_off[s+1]-1 search segment s (NULL: one segment, all).
 *   k          host, int32[n_seg]: neighbours per segment, 1..FS_MAX_K.
 *   exclude    device, int32[nq] or NULL: a segment-local row each query
 *              must skip (-1 = none); this is the paper's leave-one-out.
 *   workspace  device, >= fs_workspace_size() bytes, 256-byte aligned; owned
 *              by the caller, reusable once the stream has passed this call.
 *   idx        device, int32[nq][k_max], k_max = max over segments of k
 *   dist       device, float[nq][k_max]: d = 1 - s of each neighbour
 * Slots at or beyond a segment's k are written as padding (-1, +inf).
 */
fs_status fs_knn(const fs_db *db, const float *q, int32_t nq,
                 const int32_t *q_seg_off, const int32_t *k,
                 const int32_t *exclude, void *workspace,
                 size_t workspace_bytes, int32_t *idx, float *dist,
                 void *stream);

/*
 * fs_recommend - fs_knn, then the neighbours' phase orders (Sec. 4: the
 * suggested sequences, in rank order, duplicates kept).
 *   seq_out  device, int16[nq][k_max][l_max]: each order's first l_max pass
 *            IDs, padded with -1
 *   seq_len  device, int32[nq][k_max]: each order's full length
 *   l_max    >= 1
 *   dup_of   device, int32[nq][k_max] or NULL: for each slot, the first
 *            earlier slot of the same query with an identical order, else -1
 *            (the paper compiles each distinct sequence once, Sec. 4.2)
 * Other arguments as in fs_knn.
 */
fs_status fs_recommend(const fs_db *db, const float *q, int32_t nq,
                       const int32_t *q_seg_off, const int32_t *k,
                       const int32_t *exclude, void *workspace,
                       size_t workspace_bytes, int32_t *idx, float *dist,
                       int16_t *seq_out, int32_t *seq_len, int32_t l_max,
                       int32_t *dup_of, void *stream);

/*
 * fs_knn_noalloc - fs_knn for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a deployment aid. Some callers may
 * not call cudaMalloc at all: plug-ins hosted by a framework that owns every
 * byte of device memory, serving loops that fixed their memory at start-up
 * and must not add to it, and latency-bound paths where an allocation's
 * implicit device synchronisation is not acceptable. This entry point takes
 * the same inputs and outputs as fs_knn but no workspace: its scratch is a
 * fixed array of FS_NOALLOC_SCRATCH_BYTES in the library's own device memory,
 * present on every GPU the library is loaded on until the process exits.
 *   - It never allocates or frees device memory.
 *   - A call whose scratch need for its own nq, q_seg_off and k (at most
 *     what fs_workspace_size reports for the same nq and q_seg_off) exceeds
 *     FS_NOALLOC_SCRATCH_BYTES returns FS_ENOMEM and launches nothing.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before any
 *     stream capture. cudaDeviceReset unloads the library's device code, so
 *     the address looked up before it is no longer valid: do not call this
 *     entry point on a device after resetting it in the same process.
 *   - All calls on a device share the one array, which keeps what the last
 *     call left there; each call resets the counters it relies on and writes
 *     every other byte before reading it. Calls whose work overlaps on the
 *     GPU (other streams, other host threads) race on the array: serialise
 *     them.
 */
#define FS_NOALLOC_SCRATCH_BYTES (32u << 20)
fs_status fs_knn_noalloc(const fs_db *db, const float *q, int32_t nq,
                         const int32_t *q_seg_off, const int32_t *k,
                         const int32_t *exclude, int32_t *idx, float *dist,
                         void *stream);

/* Frees the database's device memory (after synchronising its last use). */
fs_status fs_db_destroy(fs_db *db);

/*
 * fs_db_check - synchronises `stream`, then returns and clears the device
 * status word of `db` (FS_OK if no device-side error was recorded).
 */
fs_status fs_db_check(fs_db *db, void *stream);

/* fs_db_stats - synchronises `stream` and copies the counters; reset != 0
 * zeroes them afterwards. */
fs_status fs_db_stats(fs_db *db, void *stream, int32_t reset, fs_stats *out);

/*
 * fs_db_set_metric - the similarity measure of later searches on db.
 *   FS_COSINE (the default): Sec. 4.2's cosine distance, d = 1 - s.
 *   FS_EUCLIDEAN, FS_MANHATTAN: Sec. 4.2 leaves other metrics to future
 *   work; these are the distances between feature vectors standardised per
 *   feature, z = (v - mu) / sigma, with the mean and population deviation
 *   of the segment's rows (binary64, sums in row order; a feature constant
 *   over the segment contributes nothing). d is the Euclidean or Manhattan
 *   distance of the z vectors (binary64 for the reported rows); ranking is
 *   d ascending, equal d to the lower index. Queries are standardised with
 *   the statistics of their segment.
 * Needs an FS_FP32 database (FS_EUNSUPPORTED otherwise: the tensor-core
 * scans hold unit-vector codes). Computes the statistics and the
 * standardised rows on `stream` and synchronises it. Not while searches on
 * db are being issued from another thread.
 */
typedef enum { FS_COSINE = 0, FS_EUCLIDEAN = 1, FS_MANHATTAN = 2 } fs_metric;

fs_status fs_db_set_metric(fs_db *db, fs_metric metric, void *stream);

/*
 * Scan planning parameters of one database. The paper has no counterpart:
 * these only change how the scan's work is split across blocks and how
 * long its internal candidate lists are, never a result (the selection is
 * exact whatever they are). A field left 0 takes the built-in default.
 *   items_per_block  scan work items (query tile x row chunk) per resident
 *                    block, 1..64 (blocks claim items one at a time); more
 *                    items leave finer pieces for the end of the scan, fewer
 *                    keep longer row chunks per item, so fewer candidate
 *                    lists start empty (default 4).
 *   list_len         entries per candidate list of the tensor-core scans:
 *                    4, 8 or 16. 4 takes effect only when every k of a call
 *                    is <= 4, 8 only when every k is <= 8; otherwise the
 *                    next longer list is kept (default: 8 when every k <= 8,
 *                    else 16). Shorter lists mean fewer inserts, but a list
 *                    that holds fewer rows than lie within the score error
 *                    of the k-th best sends its query to the exact fallback.
 *                    The FP32 scan always keeps 16.
 *   l2_share_pct     percent of the L2 cache that the row chunks scanned at
 *                    the same time may fill before they are split further
 *                    (single-segment databases), 1..100 (default 50);
 *                    -1 turns the cap off.
 *   scan_pairs       1: the tensor-core scans run on clusters of two SMs
 *                    (cta_group::2 MMAs of 256 queries x 256 rows, each SM
 *                    loading half of the rows); -1 or 0 (default): one SM per
 *                    tile. Ignored by the FP32 scan.
 * fs_workspace_size reflects the tuning set at the time of the call: size
 * the workspace after fs_db_set_tuning. Neither call may run while calls on
 * the same database are being issued from another thread. t == NULL restores
 * the defaults. FS_EINVAL for a field outside its range (nothing changes).
 */
typedef struct {
    int32_t items_per_block;
    int32_t list_len;
    int32_t l2_share_pct;
    int32_t scan_pairs;
} fs_tuning;

fs_status fs_db_set_tuning(fs_db *db, const fs_tuning *t);
fs_status fs_db_get_tuning(const fs_db *db, fs_tuning *out);

/*
 * fs_db_set_wait_test - a test aid for the failure reporting; the paper has
 * no counterpart. Every wait of the tensor-core scans (BF16, FP8) is bounded:
 * a wait that runs out makes the scan's blocks stop, release what they hold
 * and record FS_ETIMEOUT, which the next fs_db_check returns; the queries of
 * that call then get padding (-1, +inf), never a partial answer.
 *   withhold_first_load  nonzero: in later searches on db, every scan block
 *                        skips the copy of its first database tile, so the
 *                        wait for it runs out (no copy or tensor-core
 *                        operation is left in flight; nothing faults).
 *                        0: normal searches.
 *   wait_limit_us        limit of every bounded wait of the scan, in
 *                        microseconds (1..2,000,000); 0 restores the default
 *                        of 2 s.
 * FS_EINVAL for a limit above 2 s. Not while searches on db are being issued
 * from another thread.
 */
fs_status fs_db_set_wait_test(fs_db *db, int32_t withhold_first_load,
                              uint32_t wait_limit_us);

/*
 * Stage timing (tracing). While enabled, every fs_knn / fs_recommend call
 * records a CUDA event before and after each of its stages, on the call's
 * stream. fs_profile_read waits for those events and returns, per stage, the
 * summed milliseconds and the number of calls timed since the last reset.
 * `launches` counts every kernel this library enqueued (whether or not
 * timing is on) since the last reset. Safe to call from several threads.
 */
typedef enum {
    FS_STAGE_PREPARE = 0,   /* plan upload, query normalisation / codes */
    FS_STAGE_SCAN,          /* the database scan with its candidate lists */
    FS_STAGE_SELECT,        /* merge, certification, rerank, binary64 */
    FS_STAGE_FALLBACK,      /* exact scan of uncertified queries */
    FS_STAGE_GATHER,        /* phase-order gather */
    FS_NUM_STAGES
} fs_stage;

typedef struct {
    double ms[FS_NUM_STAGES];
    uint64_t calls[FS_NUM_STAGES];
    uint64_t launches;
} fs_profile;

fs_status fs_profile_enable(int32_t on);
fs_status fs_profile_read(int32_t reset, fs_profile *out);

/* Message for the last failing call on this thread ("" if none). */
const char *fs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FS_H */
