// Status strings, per-thread error text and launch-shape helpers for libboys.
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "boys_internal.h"

namespace boys {

static thread_local char g_last_error[512] = "";

boys_status fail(boys_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

boys_status check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return BOYS_OK;
    return fail(BOYS_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int sm_count() {
    static std::mutex mu;
    static std::unordered_map<int, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    cache[dev] = n;
    return n;
}

int blocks_per_sm(const void* kernel, int block, size_t smem) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(kernel);
    if (it != cache.end()) return it->second;
    int nb = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, smem) != cudaSuccess || nb < 1)
        nb = 1;
    cache[kernel] = nb;
    return nb;
}

int64_t grid_for(const void* kernel, int block, int64_t work, int64_t per_block, int waves, size_t smem) {
    int64_t need = (work + per_block - 1) / per_block;
    int64_t cap = (int64_t)sm_count() * blocks_per_sm(kernel, block, smem) * waves;
    if (need < 1) need = 1;
    return need < cap ? need : cap;
}

}  // namespace boys

BOYS_API const char* boys_status_string(int status) {
    switch (status) {
        case BOYS_OK: return "BOYS_OK";
        case BOYS_ERR_INVALID_ARG: return "BOYS_ERR_INVALID_ARG";
        case BOYS_ERR_KMAX: return "BOYS_ERR_KMAX";
        case BOYS_ERR_ALIGNMENT: return "BOYS_ERR_ALIGNMENT";
        case BOYS_ERR_CUDA: return "BOYS_ERR_CUDA";
        default: return "BOYS_ERR_UNKNOWN";
    }
}

BOYS_API const char* boys_last_error(void) { return boys::g_last_error; }

BOYS_API int boys_version(void) { return 100; }

BOYS_API int boys_kmax_limit(void) { return 32; }
