// The paper's benchmark workload (Section III, Algorithm 2):
//     z_i = sum_{l=0}^{k} c_l sum_{j=0}^{n-1} F_l(x_i + x_j) y_j,
// with the three-region Algorithm 1 for every F_l (Algorithm 2 as printed has
// no region C although x_i + x_j reaches 60; the three-region method is used).
//
// One thread per i; the (x_j, y_j) are staged through shared memory in tiles
// of kBlock.  For each pair the thread evaluates F_0..F_k(x_i + x_j), forms
// w = sum_l c_l F_l as the values are produced (A lanes produce them
// downward, B/C lanes upward; the weights follow) and accumulates
// z_i += y_j w in FP64.  When x is sorted, the 32 consecutive i of a warp give
// nearly equal arguments, so almost every warp lies in one region and runs
// only that region's anchor and special functions (setup_warp); the result is
// correct for any order.  The recurrence runs entirely in the integer format:
// this kernel's own FP64 work (the w and z sums) already loads the FP64 pipe.
#include <array>
#include <utility>

#include "boys_fp64.cuh"
#include "boys_internal.h"

namespace boys {
namespace {

#ifndef BOYS_PAIRWISE_BLOCK
#define BOYS_PAIRWISE_BLOCK 128
#endif
constexpr int kBlock = BOYS_PAIRWISE_BLOCK;

template <int K>
__global__ void __launch_bounds__(kBlock) k_pairwise(const double* __restrict__ x, const double* __restrict__ y,
                                                     int64_t n, const double* __restrict__ c,
                                                     double* __restrict__ z) {
    __shared__ double sx[kBlock], sy[kBlock];
    double cw[K + 1];
#pragma unroll
    for (int l = 0; l <= K; ++l) cw[l] = __ldg(c + l);
    const int t = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * kBlock + t;
    const double xi = i < n ? __ldg(x + i) : 0.0;
    double zi = 0.0;
    for (int64_t j0 = 0; j0 < n; j0 += kBlock) {
        __syncthreads();
        if (j0 + t < n) {
            sx[t] = __ldg(x + j0 + t);
            sy[t] = __ldg(y + j0 + t);
        }
        __syncthreads();
        const int jn = (int)min((int64_t)kBlock, n - j0);
        for (int jj = 0; jj < jn; ++jj) {
            const fp64::Setup S = fp64::setup_warp<K, true>(xi + sx[jj]);
            double yd = S.y0d;
            xf::Xf yv = S.y0;
            double w = 0.0;
#pragma unroll
            for (int p = 0; p <= K; ++p) {
                const double v = fp64::next_value<K, 0>(S, p, yd, yv);
                w = fma(S.inA ? cw[K - p] : cw[p], v, w);
            }
            zi = fma(sy[jj], w, zi);
        }
    }
    if (i < n) z[i] = zi;
}

template <int... K>
constexpr auto pairwise_table(std::integer_sequence<int, K...>) {
    using Fn = void (*)(const double*, const double*, int64_t, const double*, double*);
    return std::array<Fn, sizeof...(K)>{&k_pairwise<K>...};
}

}  // namespace
}  // namespace boys

BOYS_API boys_status boys_pairwise(const double* x, const double* y, int64_t n, const double* c, int k, double* z,
                                   void* stream) {
    using namespace boys;
    if (k < 0 || k > 32) return fail(BOYS_ERR_KMAX, "boys_pairwise: k=%d outside [0, 32]", k);
    if (n < 0) return fail(BOYS_ERR_INVALID_ARG, "boys_pairwise: n=%lld < 0", (long long)n);
    if (n == 0) return BOYS_OK;
    if (!x || !y || !c || !z) return fail(BOYS_ERR_INVALID_ARG, "boys_pairwise: NULL pointer");
    if (!aligned(x, 8) || !aligned(y, 8) || !aligned(c, 8) || !aligned(z, 8))
        return fail(BOYS_ERR_ALIGNMENT, "boys_pairwise: pointers not 8-byte aligned");
    if (n > ((int64_t)1 << 40)) return fail(BOYS_ERR_INVALID_ARG, "boys_pairwise: n=%lld too large", (long long)n);
    static constexpr auto t = pairwise_table(std::make_integer_sequence<int, 33>{});
    const int64_t grid = (n + kBlock - 1) / kBlock;
    if (grid > 0x7fffffff) return fail(BOYS_ERR_INVALID_ARG, "boys_pairwise: grid too large");
    t[k]<<<(unsigned)grid, kBlock, 0, (cudaStream_t)stream>>>(x, y, n, c, z);
    return check_cuda(cudaGetLastError(), "boys_pairwise launch");
}
