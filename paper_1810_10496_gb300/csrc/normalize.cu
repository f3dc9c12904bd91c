// Row preparation: unit vectors, binary64 squared norms, BF16/FP8 codes.
//
// The cosine of Sec. 4.2 is the dot product of the two unit vectors, so the
// database is stored once as x / ||x||_2 and every scan becomes a plain
// contraction. One warp handles one row: lanes read the row with coalesced
// loads, each lane sums the squares of its elements with FMA, the warp adds
// the 32 partial sums in a butterfly and lane 0's total is broadcast so that
// every element of the row is scaled by the same reciprocal norm.
//
// Per row the kernel also writes (when asked):
//   - the FP32 sum of squares (exactly 0 only for an all-zero row);
//   - the BF16 code of each unit element (round to nearest even), or the
//     FP8 E4M3 code of u_i / s with s = max_i |u_i| / 448 (per-vector scale);
//   - the residual norm r = ||u - dequantised(u)||_2, which bounds how far a
//     low-precision score can be from the FP32 one.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "fs_internal.cuh"

namespace fsk {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum_bcast(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return __shfl_sync(kFull, v, 0);
}
__device__ __forceinline__ float warp_max_bcast(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return __shfl_sync(kFull, v, 0);
}

__device__ __forceinline__ bool feature_ok(float v) {
    float a = fabsf(v);
    return v == 0.0f || (a >= 0x1p-40f && a <= 0x1p50f);  // also rejects NaN/inf
}

__global__ void k_normalize_public(const float* __restrict__ x, int64_t n, int f, int64_t ld,
                                   float* __restrict__ xu, float* __restrict__ inv_out) {
    int lane = threadIdx.x & 31;
    int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    const float* xr = x + row * ld;
    float ss = 0.0f;
    bool finite = true;
    for (int i = lane; i < f; i += 32) {
        float v = xr[i];
        finite &= isfinite(v);
        ss = fmaf(v, v, ss);
    }
    ss = warp_sum_bcast(ss);
    finite = __all_sync(kFull, finite);
    float inv = ss > 0.0f ? 1.0f / sqrtf(ss) : 0.0f;
    if (!finite) inv = __int_as_float(0x7fc00000);
    float* ur = xu + row * (int64_t)f;
    for (int i = lane; i < f; i += 32) ur[i] = finite ? xr[i] * inv : inv;
    if (inv_out && lane == 0) inv_out[row] = inv;
}

// The same with 128-bit loads and stores: lane l handles elements 4l..4l+3
// of every 128-element block of the row. Needs 16-byte aligned rows (x, ld
// and f multiples of 4 floats), checked on the host.
__global__ void k_normalize_public_v4(const float* __restrict__ x, int64_t n, int f, int64_t ld,
                                      float* __restrict__ xu, float* __restrict__ inv_out) {
    int lane = threadIdx.x & 31;
    int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    const float4* xr = reinterpret_cast<const float4*>(x + row * ld);
    const int f4 = f >> 2;
    float ss = 0.0f;
    bool finite = true;
    for (int i = lane; i < f4; i += 32) {
        const float4 v = __ldg(xr + i);
        finite &= isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w);
        ss = fmaf(v.x, v.x, ss);
        ss = fmaf(v.y, v.y, ss);
        ss = fmaf(v.z, v.z, ss);
        ss = fmaf(v.w, v.w, ss);
    }
    ss = warp_sum_bcast(ss);
    finite = __all_sync(kFull, finite);
    float inv = ss > 0.0f ? 1.0f / sqrtf(ss) : 0.0f;
    if (!finite) inv = __int_as_float(0x7fc00000);
    float4* ur = reinterpret_cast<float4*>(xu + row * (int64_t)f);
    for (int i = lane; i < f4; i += 32) {
        const float4 v = __ldg(xr + i);
        ur[i] = finite ? make_float4(v.x * inv, v.y * inv, v.z * inv, v.w * inv)
                       : make_float4(inv, inv, inv, inv);
    }
    if (inv_out && lane == 0) inv_out[row] = inv;
}

// The per-row outputs after the norm is known; shared by the scalar and the
// 128-bit variants of k_prepare_rows.
struct RowOut {
    float* unit;
    int fu;
    float* ss_out;
    void* lowp;
    int fl;
    float* scale;
    float* resid;
    int prec;
    uint32_t* status;
};

// prec: FS_FP32 (no codes), FS_BF16, FS_FP8_E4M3
__global__ void k_prepare_rows(const float* __restrict__ x, int64_t n, int f, RowOut o) {
    int lane = threadIdx.x & 31;
    int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    const float* xr = x + row * (int64_t)f;
    float ss = 0.0f, amax = 0.0f;
    bool ok = true;
    for (int i = lane; i < f; i += 32) {
        float v = xr[i];
        ok &= feature_ok(v);
        ss = fmaf(v, v, ss);
        amax = fmaxf(amax, fabsf(v));
    }
    ok = __all_sync(kFull, ok);
    ss = warp_sum_bcast(ss);
    amax = warp_max_bcast(amax);
    if (!ok) {
        if (lane == 0) atomicOr(o.status, kStBadFeature);
        ss = 0.0f;  // the row is treated as all zeros
        amax = 0.0f;
    }
    float inv = ss > 0.0f ? 1.0f / sqrtf(ss) : 0.0f;

    // FP32 unit vector, zero padded to fu
    float* ur = o.unit + row * (int64_t)o.fu;
    for (int i = lane; i < o.fu; i += 32) ur[i] = (ok && i < f) ? xr[i] * inv : 0.0f;

    if (o.ss_out && lane == 0) o.ss_out[row] = ss;

    if (o.prec == FS_BF16) {
        __nv_bfloat16* lr = reinterpret_cast<__nv_bfloat16*>(o.lowp) + row * (int64_t)o.fl;
        float rs = 0.0f;
        for (int i = lane; i < o.fl; i += 32) {
            float u = (ok && i < f) ? xr[i] * inv : 0.0f;
            __nv_bfloat16 c = __float2bfloat16_rn(u);
            float e = u - __bfloat162float(c);  // exact: the rounding error of u
            rs = fmaf(e, e, rs);
            lr[i] = c;
        }
        rs = warp_sum_bcast(rs);
        if (lane == 0) o.resid[row] = sqrtf(rs);
    } else if (o.prec == FS_FP8_E4M3) {
        __nv_fp8_storage_t* lr = reinterpret_cast<__nv_fp8_storage_t*>(o.lowp) + row * (int64_t)o.fl;
        float umax = amax * inv;  // rounding is monotonic: this is max |u_i|
        float s = umax > 0.0f ? umax / 448.0f : 0.0f;
        float rs = 0.0f;
        for (int i = lane; i < o.fl; i += 32) {
            float u = (ok && i < f) ? xr[i] * inv : 0.0f;
            __nv_fp8_storage_t c = 0;
            float e = u;
            if (s > 0.0f) {
                c = __nv_cvt_float_to_fp8(u / s, __NV_SATFINITE, __NV_E4M3);
                __half_raw hr = __nv_cvt_fp8_to_halfraw(c, __NV_E4M3);
                float dq = __half2float(__half(hr));
                // binary64 keeps s*dq exact (8 + 24 significant bits)
                e = (float)((double)u - (double)s * (double)dq);
            }
            rs = fmaf(e, e, rs);
            lr[i] = c;
        }
        rs = warp_sum_bcast(rs);
        if (lane == 0) {
            o.resid[row] = sqrtf(rs);
            o.scale[row] = s;
        }
    }
}

// FP8 code of one unit element and its exact rounding error (binary64 keeps
// s * dq exact: 8 + 24 significant bits)
__device__ __forceinline__ uint32_t fp8_code(float u, float s, float& e) {
    e = u;
    if (s <= 0.0f) return 0u;
    const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(u / s, __NV_SATFINITE, __NV_E4M3);
    const __half_raw hr = __nv_cvt_fp8_to_halfraw(c, __NV_E4M3);
    e = (float)((double)u - (double)s * (double)__half2float(__half(hr)));
    return (uint32_t)c;
}

// k_prepare_rows with 128-bit loads: lane l reads elements 4l..4l+3 of every
// 128-element block of the row and writes the unit vector (float4), BF16
// codes (8 bytes) or FP8 codes (4 bytes) of the same four elements. Needs
// x 16-byte aligned and f a multiple of 4 (checked on the host); fu and fl
// are multiples of 32 and 64, so every output row is aligned too.
__global__ void k_prepare_rows_v4(const float* __restrict__ x, int64_t n, int f, RowOut o) {
    int lane = threadIdx.x & 31;
    int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    const float4* xr = reinterpret_cast<const float4*>(x + row * (int64_t)f);
    const int f4 = f >> 2;
    float ss = 0.0f, amax = 0.0f;
    bool ok = true;
    for (int i = lane; i < f4; i += 32) {
        const float4 v = __ldg(xr + i);
        ok &= feature_ok(v.x) && feature_ok(v.y) && feature_ok(v.z) && feature_ok(v.w);
        ss = fmaf(v.x, v.x, ss);
        ss = fmaf(v.y, v.y, ss);
        ss = fmaf(v.z, v.z, ss);
        ss = fmaf(v.w, v.w, ss);
        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    ok = __all_sync(kFull, ok);
    ss = warp_sum_bcast(ss);
    amax = warp_max_bcast(amax);
    if (!ok) {
        if (lane == 0) atomicOr(o.status, kStBadFeature);
        ss = 0.0f;  // the row is treated as all zeros
        amax = 0.0f;
    }
    const float inv = ss > 0.0f ? 1.0f / sqrtf(ss) : 0.0f;
    if (o.ss_out && lane == 0) o.ss_out[row] = ss;

    // the unit elements 4i..4i+3 (zero past f, or for a rejected row)
    auto unit4 = [&](int i) {
        if (!ok || i >= f4) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float4 v = __ldg(xr + i);
        return make_float4(v.x * inv, v.y * inv, v.z * inv, v.w * inv);
    };
    float4* ur = reinterpret_cast<float4*>(o.unit + row * (int64_t)o.fu);
    for (int i = lane; i < (o.fu >> 2); i += 32) ur[i] = unit4(i);

    if (o.prec == FS_BF16) {
        uint2* lr = reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(o.lowp) +
                                             row * (int64_t)o.fl);
        float rs = 0.0f;
        for (int i = lane; i < (o.fl >> 2); i += 32) {
            const float4 u = unit4(i);
            const __nv_bfloat162 c0 = __floats2bfloat162_rn(u.x, u.y);
            const __nv_bfloat162 c1 = __floats2bfloat162_rn(u.z, u.w);
            // exact: the rounding errors of the four elements
            const float e0 = u.x - __low2float(c0), e1 = u.y - __high2float(c0);
            const float e2 = u.z - __low2float(c1), e3 = u.w - __high2float(c1);
            rs = fmaf(e0, e0, rs);
            rs = fmaf(e1, e1, rs);
            rs = fmaf(e2, e2, rs);
            rs = fmaf(e3, e3, rs);
            uint2 w;
            w.x = *reinterpret_cast<const uint32_t*>(&c0);
            w.y = *reinterpret_cast<const uint32_t*>(&c1);
            lr[i] = w;
        }
        rs = warp_sum_bcast(rs);
        if (lane == 0) o.resid[row] = sqrtf(rs);
    } else if (o.prec == FS_FP8_E4M3) {
        uint32_t* lr = reinterpret_cast<uint32_t*>(reinterpret_cast<__nv_fp8_storage_t*>(o.lowp) +
                                                   row * (int64_t)o.fl);
        const float umax = amax * inv;  // rounding is monotonic: this is max |u_i|
        const float s = umax > 0.0f ? umax / 448.0f : 0.0f;
        float rs = 0.0f;
        for (int i = lane; i < (o.fl >> 2); i += 32) {
            const float4 u = unit4(i);
            float e0, e1, e2, e3;
            const uint32_t c = fp8_code(u.x, s, e0) | (fp8_code(u.y, s, e1) << 8) |
                               (fp8_code(u.z, s, e2) << 16) | (fp8_code(u.w, s, e3) << 24);
            rs = fmaf(e0, e0, rs);
            rs = fmaf(e1, e1, rs);
            rs = fmaf(e2, e2, rs);
            rs = fmaf(e3, e3, rs);
            lr[i] = c;
        }
        rs = warp_sum_bcast(rs);
        if (lane == 0) {
            o.resid[row] = sqrtf(rs);
            o.scale[row] = s;
        }
    }
}

// B = sum x_i^2 in binary64, summed sequentially for i = 0..F-1 without fused
// multiply-add (the exact formula of the result contract). One thread per
// row, so every lane of the narrow binary64 pipe does useful work; the rows
// are staged through shared memory 32 features at a time with coalesced
// loads. Rows flagged invalid by k_prepare_rows are not special here: their
// build fails as a whole.
constexpr int kNormRows = 256;
__global__ void __launch_bounds__(kNormRows)
k_norm64_rows(const float* __restrict__ x, int64_t n, int f, double* __restrict__ b64) {
    __shared__ float tile[kNormRows][33];
    const int64_t row0 = (int64_t)blockIdx.x * kNormRows;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double b = 0.0;
    for (int f0 = 0; f0 < f; f0 += 32) {
        // warp w loads rows w, w+8, ... (32 consecutive features each)
        for (int r = w; r < kNormRows; r += kNormRows / 32) {
            const int64_t row = row0 + r;
            tile[r][lane] = (row < n && f0 + lane < f) ? x[row * f + f0 + lane] : 0.0f;
        }
        __syncthreads();
        const int m = min(32, f - f0);
        for (int i = 0; i < m; ++i) {
            const double v = (double)tile[threadIdx.x][i];
            b = __dadd_rn(b, __dmul_rn(v, v));
        }
        __syncthreads();
    }
    const int64_t row = row0 + threadIdx.x;
    if (row < n) b64[row] = b;
}

__global__ void k_check_sequences(const int64_t* __restrict__ off, const int16_t* __restrict__ ids,
                                  int64_t n, int64_t total, uint32_t* status) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t r = t; r < n; r += stride) bad |= off[r + 1] < off[r];
    if (t == 0) bad |= (off[0] != 0) || (off[n] != total);
    for (int64_t i = t; i < total; i += stride) bad |= ids[i] < 0;
    if (bad) atomicOr(status, kStBadSequence);
}

// blockIdx.y = segment; non-negative floats order like their bit patterns
__global__ void k_segment_max(const float* __restrict__ v, const int64_t* __restrict__ seg_off,
                              float* __restrict__ out) {
    int s = blockIdx.y;
    int64_t lo = seg_off[s], hi = seg_off[s + 1];
    float m = 0.0f;
    for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, v[i]);
    m = warp_max_bcast(m);
    if ((threadIdx.x & 31) == 0 && m > 0.0f)
        atomicMax(reinterpret_cast<int*>(out + s), __float_as_int(m));
}

}  // namespace

cudaError_t launch_normalize_public(const float* x, int64_t n, int f, int64_t ld, float* x_unit,
                                    float* inv_norm, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int warps = 8;
    const bool v4 = ((uintptr_t)x & 15) == 0 && ((uintptr_t)x_unit & 15) == 0 && ld % 4 == 0 &&
                    f % 4 == 0;
    if (v4)
        k_normalize_public_v4<<<(unsigned)ceil_div(n, warps), warps * 32, 0, st>>>(
            x, n, f, ld, x_unit, inv_norm);
    else
        k_normalize_public<<<(unsigned)ceil_div(n, warps), warps * 32, 0, st>>>(x, n, f, ld,
                                                                                x_unit, inv_norm);
    return cudaGetLastError();
}

cudaError_t launch_prepare_rows(const float* x, int64_t n, int f, float* unit, int fu,
                                float* ss_out, void* lowp, int fl, float* scale, float* resid,
                                int prec, uint32_t* status, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int warps = 8;
    const RowOut o{unit, fu, ss_out, lowp, fl, scale, resid, prec, status};
    // unit rows (fu floats), BF16 rows (fl x 2 bytes) and FP8 rows (fl bytes)
    // start on 16-byte boundaries when their arrays do
    const bool v4 = ((uintptr_t)x & 15) == 0 && f % 4 == 0 && ((uintptr_t)unit & 15) == 0 &&
                    ((uintptr_t)lowp & 15) == 0;
    if (v4)
        k_prepare_rows_v4<<<(unsigned)ceil_div(n, warps), warps * 32, 0, st>>>(x, n, f, o);
    else
        k_prepare_rows<<<(unsigned)ceil_div(n, warps), warps * 32, 0, st>>>(x, n, f, o);
    return cudaGetLastError();
}

cudaError_t launch_norm64_rows(const float* x, int64_t n, int f, double* b64, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_norm64_rows<<<(unsigned)ceil_div(n, kNormRows), kNormRows, 0, st>>>(x, n, f, b64);
    return cudaGetLastError();
}

cudaError_t launch_check_sequences(const int64_t* off, const int16_t* ids, int64_t n, int64_t total,
                                   uint32_t* status, cudaStream_t st) {
    k_check_sequences<<<256, 256, 0, st>>>(off, ids, n, total, status);
    return cudaGetLastError();
}

cudaError_t launch_segment_max(const float* v, const int64_t* seg_off_dev, int n_seg, float* out,
                               cudaStream_t st) {
    if (n_seg == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * n_seg, st);
    if (e != cudaSuccess) return e;
    dim3 grid(n_seg == 1 ? 512 : 8, n_seg);
    k_segment_max<<<grid, 256, 0, st>>>(v, seg_off_dev, out);
    return cudaGetLastError();
}

}  // namespace fsk
