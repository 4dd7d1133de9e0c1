// Backward of F_0..F_kmax with respect to x (boys_grad).
//
// Differentiating the definition (Eq. 3) under the integral sign gives
// dF_k/dx = -F_{k+1}, so for upstream gradients g_k:
//     dL/dx_i = -sum_{k=0}^{kmax} g[k*ldg + i] * F_{k+1}(x_i).
// The kernel re-evaluates F_0..F_{kmax+1} with the forward method at order
// kmax+1 (nothing but x is saved by the forward), so kmax <= 31.
#include <array>
#include <utility>

#include "boys_fp64.cuh"
#include "boys_internal.h"

namespace boys {
namespace {

constexpr int kBlock = 128;

// FP64 recurrence steps and minimum resident blocks of the gradient kernel
// (its own g_k F_{k+1} sum is FP64 work already): swept on GB300 at kmax 16,
// N = 2^24: 4 FP64 steps and 8 blocks per SM (64 registers), 1.00 ms, against
// 1.03 with 2, 1.02 with 6, 1.09 with 8 and, with an earlier step, 1.23 with
// the register count left free.
#ifndef BOYS_GRAD_FP64_STEPS
#define BOYS_GRAD_FP64_STEPS 4
#endif
#ifndef BOYS_GRAD_MIN_BLOCKS
#define BOYS_GRAD_MIN_BLOCKS 8
#endif

template <int KMAX>
__global__ void __launch_bounds__(kBlock, BOYS_GRAD_MIN_BLOCKS) k_grad_f64(const double* __restrict__ x, int64_t n,
                                                     const double* __restrict__ g, int64_t ldg,
                                                     double* __restrict__ dx) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double F[KMAX + 2];
        fp64::eval_point<KMAX + 1, BOYS_GRAD_FP64_STEPS>(__ldcs(x + i), F);
        double s = 0.0;
#pragma unroll
        for (int k = 0; k <= KMAX; ++k) s = fma(__ldcs(g + k * ldg + i), F[k + 1], s);
        __stcs(dx + i, -s);
    }
}

template <int... K>
constexpr auto grad_table(std::integer_sequence<int, K...>) {
    using Fn = void (*)(const double*, int64_t, const double*, int64_t, double*);
    return std::array<Fn, sizeof...(K)>{&k_grad_f64<K>...};
}

}  // namespace
}  // namespace boys

BOYS_API boys_status boys_grad(const double* x, int64_t n, int kmax, const double* g, int64_t ldg,
                               double* dx, void* stream) {
    using namespace boys;
    if (kmax < 0 || kmax > 31) return fail(BOYS_ERR_KMAX, "boys_grad: kmax=%d outside [0, 31]", kmax);
    if (n < 0) return fail(BOYS_ERR_INVALID_ARG, "boys_grad: n=%lld < 0", (long long)n);
    if (ldg < n) return fail(BOYS_ERR_INVALID_ARG, "boys_grad: ldg=%lld < n=%lld", (long long)ldg, (long long)n);
    if (n == 0) return BOYS_OK;
    if (!x || !g || !dx) return fail(BOYS_ERR_INVALID_ARG, "boys_grad: NULL pointer");
    if (ldg > INT64_MAX / (kmax + 1)) return fail(BOYS_ERR_INVALID_ARG, "boys_grad: (kmax+1)*ldg overflows");
    if (!aligned(x, 8) || !aligned(g, 8) || !aligned(dx, 8))
        return fail(BOYS_ERR_ALIGNMENT, "boys_grad: pointers not 8-byte aligned");
    static constexpr auto t = grad_table(std::make_integer_sequence<int, 32>{});
    const auto fn = t[kmax];
    const int64_t grid = grid_for((const void*)fn, kBlock, n, kBlock);
    fn<<<(unsigned)grid, kBlock, 0, (cudaStream_t)stream>>>(x, n, g, ldg, dx);
    return check_cuda(cudaGetLastError(), "boys_grad launch");
}
