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
// w = F_0 sum_l e_l t^l, e_l = c_l (2l-1)!! / 32^l, t = 32 / (2X) <= 0.552,
// as a fixed-point Horner sum on the integer pipes (its partial sums are
// bounded by sum_l |e_l|, so a binary point chosen per block from the weights
// holds them to ~2^-60 sum_l |c_l|).  In region-A and region-B warps w is
// summed by FP64 FMAs.  The recurrence runs entirely in the integer format:
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

// v 2^-f as a double (v a signed fixed-point integer), by integer assembly.
__device__ __forceinline__ double fixed_to_double(long long v, int f) {
    if (v == 0) return 0.0;
    const xf::Xf a = xf::from_fixed(v, f);
    const double m = xf::to_double(a);
    return v < 0 ? -m : m;
}

// Binary point f of a fixed-point sum bounded by M: M 2^f < 2^61 (f = 0 for M = 0).
__device__ __forceinline__ int fixed_point_for(double M) { return M > 0.0 ? 60 - ilogb(M) : 0; }

// w = sum_l c_l F_l for a warp whose lanes all lie in region R (A or B):
// value number p of the recurrence is F_{K-p} in A and F_p in B.  With the
// region-C sums on the integer pipes the FP64 pipe has room for all of w here:
// routing the first 2, 4 or 6 terms through a fixed-point accumulator on the
// integer pipes instead took 582 ms against 553 ms (k = 12, N = 2^17).
template <int R, int K>
__device__ __forceinline__ double w_region(const fp64::Setup& S, const double (&cw)[K + 1]) {
    double yd = S.y0d;
    xf::Xf yv = S.y0;
    double w = 0.0;
#pragma unroll
    for (int p = 0; p <= K; ++p) {
        const int l = R == fp64::kRegionA ? K - p : p;
        w = fma(cw[l], fp64::next_value<K, 0>(S, p, yd, yv), w);
    }
    return w;
}

// Minimum resident blocks per SM (caps the registers): at the paper's N = 2^19,
// x sorted, 8 blocks (64 registers) 6.98 s, 7 blocks 7.01, 9 7.06, 10 7.02,
// the uncapped 76 registers 7.07.
#ifndef BOYS_PAIRWISE_MIN_BLOCKS
#define BOYS_PAIRWISE_MIN_BLOCKS 8
#endif

template <int K>
__global__ void __launch_bounds__(kBlock, BOYS_PAIRWISE_MIN_BLOCKS) k_pairwise(const double* __restrict__ x, const double* __restrict__ y,
                                                     int64_t n, const double* __restrict__ c,
                                                     double* __restrict__ z) {
    __shared__ double sx[kBlock], sy[kBlock];
    __shared__ long long s_efx[K + 1];
    __shared__ int s_fe;
    double cw[K + 1];
#pragma unroll
    for (int l = 0; l <= K; ++l) cw[l] = __ldg(c + l);
    const int t = threadIdx.x;
    if (t == 0) {
        // Fixed-point coefficients of the region-C sum, once per block:
        // e_l = c_l (2l-1)!! / 32^l, the coefficients of w / F_0 as a
        // polynomial in t = 32 u = 16 / X (t <= 0.552 on region C), whose
        // partial Horner sums are bounded by sum |e_l|; the binary point keeps
        // that bound below 2^61.
        double e[K + 1], se = 0.0, f = 1.0;
        for (int l = 0; l <= K; ++l) {
            e[l] = ldexp(cw[l] * f, -5 * l);
            f *= (double)(2 * l + 1);
            se += fabs(e[l]);
        }
        const int fe = fixed_point_for(se);
        for (int l = 0; l <= K; ++l) s_efx[l] = __double2ll_rn(ldexp(e[l], fe));
        s_fe = fe;
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
                // w = F_0 sum_l e_l t^l with t = 32 u, by a fixed-point Horner
                // sum on the integer pipes (t in Q64, from the set-up's 1/(2X)).
                const fp64::Setup S = fp64::setup_mode<fp64::kRegionC, K, true>(X);
                const unsigned long long T = S.R.m >> min(max(-(S.R.e + 6), 0), 63);
                const unsigned long long Th = T >> 1;
                long long h = s_efx[K];
#pragma unroll
                for (int l = K - 1; l >= 0; --l) h = xf::mulhi_s(h, T, Th) + s_efx[l];
                w = S.y0d * fixed_to_double(h, s_fe);
            } else if (__all_sync(0xffffffffu, r == fp64::kRegionA)) {
                w = w_region<fp64::kRegionA, K>(fp64::setup_mode<fp64::kRegionA, K, true>(X), cw);
            } else if (__all_sync(0xffffffffu, r == fp64::kRegionB)) {
                w = w_region<fp64::kRegionB, K>(fp64::setup_mode<fp64::kRegionB, K, true>(X), cw);
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
