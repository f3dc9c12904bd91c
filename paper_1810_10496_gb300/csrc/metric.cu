// Standardised Euclidean and Manhattan distances (Sec. 4.2 leaves metrics
// other than the cosine distance to future work; these are the library's
// readings of the two it names for that).
//
// Per segment and feature, the mean and the population deviation of the
// rows, in binary64 with sums in row order (no fused multiply-add), exactly
// as the oracle computes them. Rows and queries are standardised to
// z = (v - mu) / sigma (0 for a feature with sigma = 0) and stored in FP32 for
// the FP32 scan, which scores
//   Euclidean:  z_q . z_x - |z_x|^2 / 2   (larger is nearer: |z_q - z_x|^2 is
//               |z_q|^2 minus twice this)
//   Manhattan:  -sum_i |z_q,i - z_x,i|
// Each query carries a rigorous bound E on its FP32 scores (written where the
// cosine path keeps the code residual), so the same certified candidate
// lists apply; the rows that reach the answer are then scored with the
// binary64 formulas of the oracle.
#include "fs_internal.cuh"

namespace fsk {

namespace {

constexpr double kU = 5.9604644775390625e-08;   // 2^-24, FP32 unit roundoff

// one thread per (segment, feature); consecutive features in a warp read
// consecutive addresses of each row
__global__ void k_seg_stats(const float* __restrict__ raw, const int64_t* __restrict__ seg_off,
                            int n_seg, int f, double* __restrict__ mu, double* __restrict__ sg) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_seg * f) return;
    const int s = (int)(t / f), j = (int)(t % f);
    const int64_t lo = seg_off[s], hi = seg_off[s + 1];
    double m = 0.0, v = 0.0;
    if (hi > lo) {
        const double n = (double)(hi - lo);
        double acc = 0.0;
        for (int64_t r = lo; r < hi; ++r) acc = __dadd_rn(acc, (double)raw[r * f + j]);
        m = __ddiv_rn(acc, n);
        acc = 0.0;
        for (int64_t r = lo; r < hi; ++r) {
            const double d = __dsub_rn((double)raw[r * f + j], m);
            acc = __dadd_rn(acc, __dmul_rn(d, d));
        }
        v = __dsqrt_rn(__ddiv_rn(acc, n));
    }
    mu[t] = m;
    sg[t] = v;
}

__device__ __forceinline__ double zscore(float v, double m, double s) {
    return s > 0.0 ? __ddiv_rn(__dsub_rn((double)v, m), s) : 0.0;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// one warp per row: z in FP32, the Euclidean row term, the row's magnitude
__global__ void k_std_rows(const float* __restrict__ raw, int64_t n, int f, int fu,
                           const int64_t* __restrict__ seg_off, int n_seg,
                           const double* __restrict__ mu, const double* __restrict__ sg,
                           int metric, float* __restrict__ z, float* __restrict__ row_term,
                           float* __restrict__ row_mag) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= row) lo = mid; else hi = mid - 1;
    }
    const double* m = mu + (int64_t)lo * f;
    const double* s = sg + (int64_t)lo * f;
    double sq = 0.0, sq32 = 0.0, l1 = 0.0;
    for (int i = lane; i < fu; i += 32) {
        const double zi = i < f ? zscore(raw[row * f + i], m[i], s[i]) : 0.0;
        const float z32 = (float)zi;
        z[row * fu + i] = z32;
        sq += zi * zi;
        sq32 += (double)z32 * (double)z32;
        l1 += fabs((double)z32);
    }
    sq = warp_sum_d(sq);
    sq32 = warp_sum_d(sq32);
    l1 = warp_sum_d(l1);
    if (lane == 0) {
        row_term[row] = metric == FS_EUCLIDEAN ? (float)(0.5 * sq) : 0.0f;
        // magnitudes rounded up (they only enter error bounds)
        const double mag = metric == FS_EUCLIDEAN ? sqrt(sq32) : l1;
        row_mag[row] = (float)(mag * (1.0 + 1e-6));
    }
}

// Per call: one warp per query. z in FP32 (q_unit), a nonzero q_ss (the zero
// vector convention is the cosine's alone), the query's magnitude cap R in
// q_scale and its score bound E in q_resid (the plan's bound_scan = 0,
// bound_rq = 1 make E = q_resid):
//   Euclidean: E = 1.01 (g Q R + 3u (R^2/2 + Q R)),  Manhattan:
//   E = 1.01 (g + 2u)(Q1 + R1), with g = gamma_(fu+2), Q / Q1 the query's
//   |z| / sum |z_i| and R / R1 the smaller of the segment's largest row
//   magnitude and the query's magnitude plus D (below). These
//   cover the FP32 accumulation of the scan (sequential, fu terms), the
//   rounding of z to FP32 on both sides, the rounding of the row term and of
//   the final subtraction.
__global__ void k_std_queries(DbView db, CallView call) {
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= call.nq) return;
    const SegPlan p = call.plan[call.q_plan[q]];
    const double* m = db.mu + (int64_t)p.seg * db.f;
    const double* s = db.sg + (int64_t)p.seg * db.f;
    const float* v = call.q_raw + (int64_t)q * db.f;
    float* zq = call.q_unit + (int64_t)q * db.fu;
    double sq32 = 0.0, l1 = 0.0;
    bool ok = true;
    for (int i = lane; i < db.fu; i += 32) {
        float z32 = 0.0f;
        if (i < db.f) {
            const float vi = v[i];
            ok &= isfinite(vi);
            z32 = isfinite(vi) ? (float)zscore(vi, m[i], s[i]) : 0.0f;
        }
        zq[i] = z32;
        sq32 += (double)z32 * (double)z32;
        l1 += fabs((double)z32);
    }
    sq32 = warp_sum_d(sq32);
    l1 = warp_sum_d(l1);
    ok = __all_sync(0xffffffffu, ok);
    // An upper bound D on the distance to the k-th nearest row: the largest
    // distance to k rows of the segment (any k; here the first ones the query
    // may select). A row farther than D from the query cannot be among its k
    // nearest, and by the triangle inequality every row within D has
    // magnitude at most |z_q| + D (Manhattan: the L1 forms), so the score
    // bound need only cover rows up to that magnitude; rows beyond it are
    // out whatever their FP32 score.
    double dmax = -1.0;
    {
        const int excl = (call.exclude && ok) ? call.exclude[q] : -1;
        int taken = 0;
        dmax = 0.0;
        for (int64_t r = 0; r < p.nrows && taken < p.k; ++r) {
            if ((int)r == excl) continue;
            const float* x = db.raw + (p.row0 + r) * (int64_t)db.f;
            double acc = 0.0;
            for (int i = lane; i < db.f; i += 32) {
                const double t = zscore(v[i], m[i], s[i]) - zscore(x[i], m[i], s[i]);
                acc += db.metric == FS_EUCLIDEAN ? t * t : fabs(t);
            }
            acc = warp_sum_d(acc);
            const double d = db.metric == FS_EUCLIDEAN ? sqrt(acc) : acc;
            dmax = fmax(dmax, d);
            ++taken;
        }
        if (taken < p.k) dmax = -1.0;   // fewer rows than k: no bound from them
    }
    if (lane == 0) {
        if (!ok) atomicOr(db.status, kStBadFeature);
        const double n = (double)(db.fu + 2);
        const double g = n * kU / (1.0 - n * kU);
        const double qmag = db.metric == FS_EUCLIDEAN ? sqrt(sq32) : l1;
        double R = (double)p.mag_max;
        // slack 1e-5 > the 1e-6 rounding up of the row magnitudes plus the FP32
        // rounding of z on both sides, so every row within D stays under the cap
        if (dmax >= 0.0) R = fmin(R, (qmag + dmax) * (1.0 + 1e-5) + 1e-30);
        double e;
        if (db.metric == FS_EUCLIDEAN) {
            const double Q = sqrt(sq32) * (1.0 + 1e-6);
            e = 1.01 * (g * Q * R + 3.0 * kU * (0.5 * R * R + Q * R));
        } else {
            e = 1.01 * (g + 2.0 * kU) * (l1 * (1.0 + 1e-6) + R);
        }
        call.q_resid[q] = (float)(e * (1.0 + 1e-6)) + 1e-30f;
        // the magnitude cap for the scan (rows above it score -inf: provably
        // out, and their FP32 scores are not covered by E)
        call.q_scale[q] = (float)R;
        call.q_ss[q] = 1.0f;
    }
}

}  // namespace

cudaError_t launch_seg_stats(const float* raw, const int64_t* seg_off_dev, int n_seg, int f,
                             double* mu, double* sg, cudaStream_t st) {
    const int64_t t = (int64_t)n_seg * f;
    if (t == 0) return cudaSuccess;
    k_seg_stats<<<(unsigned)ceil_div(t, 128), 128, 0, st>>>(raw, seg_off_dev, n_seg, f, mu, sg);
    return cudaGetLastError();
}

cudaError_t launch_std_rows(const float* raw, int64_t n, int f, int fu, const int64_t* seg_off,
                            int n_seg, const double* mu, const double* sg, int metric,
                            float* z, float* row_term, float* row_mag, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_std_rows<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(raw, n, f, fu, seg_off, n_seg, mu, sg,
                                                         metric, z, row_term, row_mag);
    return cudaGetLastError();
}

cudaError_t launch_std_queries(const DbView& db, const CallView& call, cudaStream_t st) {
    if (call.nq == 0) return cudaSuccess;
    k_std_queries<<<(unsigned)ceil_div(call.nq, 8), 256, 0, st>>>(db, call);
    return cudaGetLastError();
}

}  // namespace fsk
