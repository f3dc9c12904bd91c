// fs_knn_noalloc: fs_knn with its scratch in a fixed array of this library's
// own device memory, for callers that cannot allocate (see include/fs.h).
//
// The array is a file-scope __device__ variable, so the CUDA runtime creates
// it on every device the library's module is loaded on. In host code its name
// only stands for a host-side shadow, never a device address: the device
// address is looked up with cudaGetSymbolAddress, once per device, with that
// device current, and handed to the kernels as an ordinary pointer.
#include <mutex>
#include <vector>

#include "fs_internal.cuh"

namespace {

constexpr size_t kScratchBytes = FS_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
std::vector<void*> g_addr;   // device address of g_scratch, per device ordinal

// The device address of the scratch array on the current device.
fs_status scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fsk::set_error(FS_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> g(g_mu);
    if ((int)g_addr.size() <= dev) g_addr.resize(dev + 1, nullptr);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fsk::set_error(FS_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                                  cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return FS_OK;
}

}  // namespace

extern "C" fs_status fs_knn_noalloc(const fs_db* db, const float* q, int32_t nq,
                                    const int32_t* q_seg_off, const int32_t* k,
                                    const int32_t* exclude, int32_t* idx, float* dist,
                                    void* stream) {
    if (!db) return fsk::set_error(FS_EINVAL, "db is NULL");
    // the scratch this call's own layout takes (its k and list length)
    size_t need = 0;
    fs_status st = fsk::search_scratch_bytes(db, nq, q_seg_off, k, &need);
    if (st != FS_OK) return st;
    if (need > kScratchBytes)
        return fsk::set_error(FS_ENOMEM,
                              "fs_knn_noalloc: %d queries need %zu bytes of scratch, more than the "
                              "%zu bytes of its static array; use fs_knn with a workspace",
                              nq, need, kScratchBytes);
    void* scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != FS_OK) return st;
    // fs_knn resets its counters at the start of the call and writes every
    // other scratch byte before reading it, so nothing else needs clearing.
    return fs_knn(db, q, nq, q_seg_off, k, exclude, scratch, kScratchBytes, idx, dist, stream);
}
