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
// only that region's anchor and special functions; the result is correct for
// any order.  In region C (about half the pairs of the paper's workload) the
// values F_l = F_0 (2l-1)!! / (2X)^l need no recurrence: the warp evaluates
// w = F_0 sum_l c_l (2l-1)!! u^l, u = 1/(2X), by Horner in the signed integer
// format, which takes the w sum off the FP64 pipe.  The recurrence runs entirely in the integer format:
// this kernel's own FP64 work (the w and z sums) already loads the FP64 pipe.
#include <array>
#include <utility>

#include "boys_fp64.cuh"
#include "boys_internal.h"

namespace boys {
namespace {

// In region-A and region-B warps, the first BOYS_PAIRWISE_INT_TERMS values of
// the recurrence enter w through an integer-format accumulator (xf::fma_i on
// the recurrence's own values) and the rest through FP64 FMAs, balancing the
// two pipes: at k = 12, 8 integer terms were fastest (N = 2^19: 13.38 s with
// none, 12.82 s with 4, 12.63 s with 8, 12.72 s with 10, 13.40 s with all 13).
#ifndef BOYS_PAIRWISE_INT_TERMS
#define BOYS_PAIRWISE_INT_TERMS 8
#endif
#ifndef BOYS_PAIRWISE_BLOCK
#define BOYS_PAIRWISE_BLOCK 128
#endif
constexpr int kBlock = BOYS_PAIRWISE_BLOCK;

// w = sum_l c_l F_l for a warp whose lanes all lie in region R (A or B):
// value number p of the recurrence is F_{K-p} in A and F_p in B.
template <int R, int K>
__device__ __forceinline__ double w_region(const fp64::Setup& S, const double (&cw)[K + 1],
                                           const long long* s_cm, const int* s_ce) {
    constexpr int kInt = BOYS_PAIRWISE_INT_TERMS < K + 1 ? BOYS_PAIRWISE_INT_TERMS : K + 1;
    double yd = S.y0d;
    xf::Xf yv = S.y0;
    double w = 0.0;
    xf::XfI wi{0, xf::kXfZeroExp};
#pragma unroll
    for (int p = 0; p <= K; ++p) {
        const int l = R == fp64::kRegionA ? K - p : p;
        const double v = fp64::next_value<K, 0>(S, p, yd, yv);
        if (p < kInt)
            wi = xf::fma_i(xf::XfI{s_cm[l], s_ce[l]}, p == 0 ? xf::from_double(S.y0d) : yv, wi);
        else
            w = fma(cw[l], v, w);
    }
    return kInt > 0 ? w + xf::to_double(wi) : w;
}

template <int K>
__global__ void __launch_bounds__(kBlock) k_pairwise(const double* __restrict__ x, const double* __restrict__ y,
                                                     int64_t n, const double* __restrict__ c,
                                                     double* __restrict__ z) {
    __shared__ double sx[kBlock], sy[kBlock];
    __shared__ long long s_dm[K + 1], s_cm[K + 1];
    __shared__ int s_de[K + 1], s_ce[K + 1];
    double cw[K + 1];
#pragma unroll
    for (int l = 0; l <= K; ++l) cw[l] = __ldg(c + l);
    const int t = threadIdx.x;
    if (t <= K) {  // d_l = c_l (2l-1)!! for region C, in the integer format
        double f = 1.0;
        for (int m = 0; m < t; ++m) f *= (double)(2 * m + 1);
        const xf::XfI d = xf::from_double_signed(__ldg(c + t) * f);
        s_dm[t] = d.m;
        s_de[t] = d.e;
        const xf::XfI cc = xf::from_double_signed(__ldg(c + t));
        s_cm[t] = cc.m;
        s_ce[t] = cc.e;
    }
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
            const double X = xi + sx[jj];
            const int r = fp64::region_of(X);
            double w;
            if (__all_sync(0xffffffffu, r == fp64::kRegionC)) {
                // Region C: F_l = F_0 (2l-1)!! u^l with u = 1/(2X), so
                // w = F_0 sum_l d_l u^l, by Horner in the integer format.
                const fp64::Setup S = fp64::setup_mode<fp64::kRegionC, K, true>(X);
                xf::XfI h{s_dm[K], s_de[K]};
#pragma unroll
                for (int l = K - 1; l >= 0; --l) h = xf::fma_i(h, S.R, xf::XfI{s_dm[l], s_de[l]});
                w = S.y0d * xf::to_double(h);
            } else if (__all_sync(0xffffffffu, r == fp64::kRegionA)) {
                w = w_region<fp64::kRegionA, K>(fp64::setup_mode<fp64::kRegionA, K, true>(X), cw, s_cm, s_ce);
            } else if (__all_sync(0xffffffffu, r == fp64::kRegionB)) {
                w = w_region<fp64::kRegionB, K>(fp64::setup_mode<fp64::kRegionB, K, true>(X), cw, s_cm, s_ce);
            } else {
                const fp64::Setup S = fp64::setup<K, true>(X);
                double yd = S.y0d;
                xf::Xf yv = S.y0;
                w = 0.0;
#pragma unroll
                for (int p = 0; p <= K; ++p) {
                    const double v = fp64::next_value<K, 0>(S, p, yd, yv);
                    w = fma(S.inA ? cw[K - p] : cw[p], v, w);
                }
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
