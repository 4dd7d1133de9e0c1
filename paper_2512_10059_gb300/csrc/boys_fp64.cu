// FP64 stored mode (boys_eval) and fused consumer (boys_eval_fused).
//
// Stored mode: one thread per argument (grid-stride loop, grid capped at a few
// waves of resident blocks); KMAX is a template parameter so every loop is
// unrolled.  A lane keeps only the first half of its orders: from the middle
// step on every step completes two order-major rows for the whole warp, which
// are written as full 256-byte segments (fp64::eval_store), and the register
// count stays low enough for the occupancy that hides the integer-pipe
// latency of the recurrence.
#include <array>
#include <utility>

#include "boys_fp64.cuh"
#include "boys_internal.h"

// Minimum resident blocks per SM of the stored-mode kernel, which caps its
// registers: swept on GB300 with the FP64-step table of boys_fp64.cuh
// (N = 2^26, 8, 9, 10, 12 and 14 blocks at kmax 2, 4, 6, 8, 12, 16, 20, 24,
// 28): up to kmax = 20 the 32-register cap of full occupancy is fastest
// despite its spills to L1 (kmax 4: 1.86 ms against 1.91 with 8 and 1.90
// with 12; kmax 12: 2.54 against 2.59 and 2.58; kmax 20: 3.33 against 3.39),
// from kmax 24 on 8 blocks (64 registers) win (kmax 24: 3.79 against 4.22
// with 14; kmax 32: 4.68 against 4.68 with 9 and 4.78 with 7).
// BOYS_STORED_MIN_BLOCKS forces one value.
constexpr int stored_min_blocks(int kmax) {
#ifdef BOYS_STORED_MIN_BLOCKS
    return BOYS_STORED_MIN_BLOCKS + 0 * kmax;
#else
    return kmax <= 20 ? 16 : 8;
#endif
}
// FP64 recurrence steps and minimum resident blocks of the fused kernel.  Its
// Horner sum adds KMAX FMAs per argument to the FP64 pipe, so half of stored
// mode's FP64 steps run in FP64 (swept on GB300 at kmax 32, N = 2^26: 5 steps
// 6.82 ms, 7 6.68, 8 6.67, 9 6.69, 11 6.84, 13 7.19; 6 and 10 blocks per SM
// were slower than 8; the smaller kmax follow the stored-mode table).
// BOYS_FUSED_FP64_STEPS forces one value.
constexpr int fused_fp64_steps(int kmax) {
#ifdef BOYS_FUSED_FP64_STEPS
    return BOYS_FUSED_FP64_STEPS + 0 * kmax;
#else
    return boys::fp64::fp64_steps_for(kmax) / 2;
#endif
}
#ifndef BOYS_FUSED_MIN_BLOCKS
#define BOYS_FUSED_MIN_BLOCKS 8
#endif

namespace boys {
namespace {

constexpr int kBlock = 128;

template <int KMAX, bool FULL_ROWS>
__global__ void __launch_bounds__(kBlock, stored_min_blocks(KMAX)) k_eval_f64(const double* __restrict__ x, int64_t n,
                                                     double* __restrict__ out, int64_t ld) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        fp64::eval_store<KMAX, FULL_ROWS>(__ldcs(x + i), out + i, ld);
}

// out[i] = sum_k (-2 rho_i)^k F_k(x_i), by Horner in a = -2 rho from F_KMAX down.
template <int KMAX>
__global__ void __launch_bounds__(kBlock, BOYS_FUSED_MIN_BLOCKS) k_fused_f64(const double* __restrict__ x,
                                                      const double* __restrict__ rho, int64_t n,
                                                      double* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double F[KMAX + 1];
        fp64::eval_point<KMAX, fused_fp64_steps(KMAX)>(__ldcs(x + i), F);
        const double a = -2.0 * __ldcs(rho + i);
        double s = F[KMAX];
#pragma unroll
        for (int k = KMAX - 1; k >= 0; --k) s = fma(s, a, F[k]);
        __stcs(out + i, s);
    }
}

template <bool FULL_ROWS, int... K>
constexpr auto eval_table(std::integer_sequence<int, K...>) {
    using Fn = void (*)(const double*, int64_t, double*, int64_t);
    return std::array<Fn, sizeof...(K)>{&k_eval_f64<K, FULL_ROWS>...};
}

template <int... K>
constexpr auto fused_table(std::integer_sequence<int, K...>) {
    using Fn = void (*)(const double*, const double*, int64_t, double*);
    return std::array<Fn, sizeof...(K)>{&k_fused_f64<K>...};
}

}  // namespace
}  // namespace boys


namespace boys {
// Checks and launches stored mode; full_rows selects the store pattern of
// fp64::eval_store (true for output in host memory).
static boys_status eval_launch(const char* name, const double* x, int64_t n, int kmax, double* out, int64_t ld,
                               void* stream, bool full_rows) {
    if (kmax < 0 || kmax > 32) return fail(BOYS_ERR_KMAX, "%s: kmax=%d outside [0, 32]", name, kmax);
    if (n < 0) return fail(BOYS_ERR_INVALID_ARG, "%s: n=%lld < 0", name, (long long)n);
    if (ld < n) return fail(BOYS_ERR_INVALID_ARG, "%s: ld=%lld < n=%lld", name, (long long)ld, (long long)n);
    if (n == 0) return BOYS_OK;
    if (!x || !out) return fail(BOYS_ERR_INVALID_ARG, "%s: NULL pointer", name);
    if (ld > INT64_MAX / (kmax + 1)) return fail(BOYS_ERR_INVALID_ARG, "%s: (kmax+1)*ld overflows", name);
    if (!aligned(x, 8) || !aligned(out, 8)) return fail(BOYS_ERR_ALIGNMENT, "%s: x/out not 8-byte aligned", name);
    // one argument per thread, each order stored as soon as its row is complete
    static constexpr auto tdev = eval_table<false>(std::make_integer_sequence<int, 33>{});
    static constexpr auto thost = eval_table<true>(std::make_integer_sequence<int, 33>{});
    const auto fn = full_rows ? thost[kmax] : tdev[kmax];
    const int64_t grid = grid_for((const void*)fn, kBlock, n, (int64_t)kBlock);
    fn<<<(unsigned)grid, kBlock, 0, (cudaStream_t)stream>>>(x, n, out, ld);
    return check_cuda(cudaGetLastError(), "boys_eval launch");
}
}  // namespace boys

BOYS_API boys_status boys_eval(const double* x, int64_t n, int kmax, double* out, int64_t ld,
                               void* stream) {
    return boys::eval_launch("boys_eval", x, n, kmax, out, ld, stream, false);
}

BOYS_API boys_status boys_eval_fused(const double* x, const double* rho, int64_t n, int kmax,
                                     double* out, void* stream) {
    using namespace boys;
    if (kmax < 0 || kmax > 32) return fail(BOYS_ERR_KMAX, "boys_eval_fused: kmax=%d outside [0, 32]", kmax);
    if (n < 0) return fail(BOYS_ERR_INVALID_ARG, "boys_eval_fused: n=%lld < 0", (long long)n);
    if (n == 0) return BOYS_OK;
    if (!x || !rho || !out) return fail(BOYS_ERR_INVALID_ARG, "boys_eval_fused: NULL pointer");
    if (!aligned(x, 8) || !aligned(rho, 8) || !aligned(out, 8))
        return fail(BOYS_ERR_ALIGNMENT, "boys_eval_fused: pointers not 8-byte aligned");
    static constexpr auto t = fused_table(std::make_integer_sequence<int, 33>{});
    const auto fn = t[kmax];
    const int64_t grid = grid_for((const void*)fn, kBlock, n, kBlock);
    fn<<<(unsigned)grid, kBlock, 0, (cudaStream_t)stream>>>(x, rho, n, out);
    return check_cuda(cudaGetLastError(), "boys_eval_fused launch");
}

// Host buffers (pinned, or pageable where the GPU can address pageable memory):
// the evaluation kernel itself reads x and writes F over the host link.
namespace boys {
static boys_status host_view(const void* p, void** dev, const char* what) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) return check_cuda(e, "boys_eval_host: cudaPointerGetAttributes");
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *dev = a.devicePointer;
        return BOYS_OK;
    }
    if (a.type == cudaMemoryTypeUnregistered) {
        int device = 0, pageable = 0;
        cudaGetDevice(&device);
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device);
        if (pageable) {
            *dev = const_cast<void*>(p);
            return BOYS_OK;
        }
    }
    return fail(BOYS_ERR_INVALID_ARG,
                "boys_eval_host: %s is not host memory the GPU can address (pin it with cudaHostAlloc/cudaHostRegister)",
                what);
}
}  // namespace boys

BOYS_API boys_status boys_eval_host(const double* x, int64_t n, int kmax, double* out, int64_t ld, void* stream) {
    using namespace boys;
    if (kmax < 0 || kmax > 32) return fail(BOYS_ERR_KMAX, "boys_eval_host: kmax=%d outside [0, 32]", kmax);
    if (n < 0) return fail(BOYS_ERR_INVALID_ARG, "boys_eval_host: n=%lld < 0", (long long)n);
    if (ld < n) return fail(BOYS_ERR_INVALID_ARG, "boys_eval_host: ld=%lld < n=%lld", (long long)ld, (long long)n);
    if (n == 0) return BOYS_OK;
    if (!x || !out) return fail(BOYS_ERR_INVALID_ARG, "boys_eval_host: NULL pointer");
    void *xd = nullptr, *od = nullptr;
    boys_status st = host_view(x, &xd, "x");
    if (st != BOYS_OK) return st;
    st = host_view(out, &od, "out");
    if (st != BOYS_OK) return st;
    // full rows: partial writes over the host link are not merged
    return eval_launch("boys_eval_host", (const double*)xd, n, kmax, (double*)od, ld, stream, true);
}
