// FP64 stored mode (boys_eval) and fused consumer (boys_eval_fused).
//
// Stored mode: one thread per argument (grid-stride loop, grid capped at 64
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
// with 14; kmax 32: 4.68 against 4.68 with 9 and 4.78 with 7).  Re-checked
// with the 64-wave grid (8, 10, 12, 16 blocks): within 1% of the best at
// every kmax.  BOYS_STORED_MIN_BLOCKS forces one value.
constexpr int stored_min_blocks(int kmax) {
#ifdef BOYS_STORED_MIN_BLOCKS
    return BOYS_STORED_MIN_BLOCKS + 0 * kmax;
#else
    return kmax <= 20 ? 16 : 8;
#endif
}
// FP64 recurrence steps and minimum resident blocks of the fused kernel.  Its
// Horner sums add KMAX + 1 FMAs per argument to the FP64 pipe, so half of
// stored mode's FP64 steps run in FP64.  Swept on GB300 at kmax 32, N = 2^26
// (ms per launch): 8 blocks per SM with 6, 8, 10, 12 steps 6.65, 6.65, 6.79,
// 7.19; 8 steps with 4, 5, 6, 7, 10, 12 blocks 6.50, 6.58, 6.50, 6.65, 6.78,
// 6.75; 6 blocks with 6, 7, 9, 10 steps 6.56, 6.50, 6.57, 6.75.  The smaller
// kmax follow the stored-mode table.  BOYS_FUSED_FP64_STEPS forces one value.
constexpr int fused_fp64_steps(int kmax) {
#ifdef BOYS_FUSED_FP64_STEPS
    return BOYS_FUSED_FP64_STEPS + 0 * kmax;
#else
    return boys::fp64::fp64_steps_for(kmax) / 2;
#endif
}
#ifndef BOYS_FUSED_MIN_BLOCKS
#define BOYS_FUSED_MIN_BLOCKS 6
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

// |a|^E for a compile-time E >= 1, in the 64-bit-significand format (integer
// pipes), by binary powering: about 2^-58 relative for E <= 17.
template <int E>
__device__ __forceinline__ xf::Xf xf_pow(xf::Xf b) {
    xf::Xf r = b;
    bool have = false;
#pragma unroll
    for (int bit = 0; (E >> bit) != 0; ++bit) {
        if ((E >> bit) & 1) {
            r = have ? xf::mul(r, b) : b;
            have = true;
        }
        if ((E >> (bit + 1)) != 0) b = xf::mul(b, b);
    }
    return r;
}

// out[i] = sum_k a^k F_k(x_i), a = -2 rho_i, as two Horner sums in a that
// follow the order in which the step loop completes the orders.  Step p
// yields value p of the recurrence, F_{KMAX-p} on an A lane and F_p on a B or
// C lane; as in stored mode, a lane holds its values p < KMAX/2, and each
// later step p completes the pair F_q, F_p (q = KMAX - p) on every lane.
//   low  = sum_{k <= KH} a^k F_k, KH = KMAX/2: the F_q arrive with q
//          descending, so the Horner sum runs as they come;
//   high = sum_{j < NH} a^j F_{KH+1+j}: the F_p arrive ascending, so each
//          lane parks them in its own shared-memory column and sums them
//          afterwards;
//   out  = low + a^(KH+1) high, the power on the integer pipes.
// The lane never keeps all kmax+1 values, so nothing spills; the FP64 work is
// the KMAX FMAs of a single Horner sum plus one.
template <int KMAX>
__global__ void __launch_bounds__(kBlock, BOYS_FUSED_MIN_BLOCKS) k_fused_f64(const double* __restrict__ x,
                                                      const double* __restrict__ rho, int64_t n,
                                                      double* __restrict__ out) {
    constexpr int KH = KMAX / 2;
    constexpr int NH = KMAX - KH;
    constexpr int NF = fused_fp64_steps(KMAX);
    __shared__ double s_high[NH > 0 ? NH : 1][kBlock];
    double* const park = &s_high[0][threadIdx.x];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const fp64::Setup S = fp64::setup<KMAX, fp64::int_exp_for(KMAX, NF)>(__ldcs(x + i));
        const double a = -2.0 * __ldcs(rho + i);
        double hold[KH + 1];
        double yd = S.y0d, low = 0.0;
        xf::Xf y = S.y0;
#pragma unroll
        for (int p = 0; p <= KMAX; ++p) {
            const double v = fp64::next_value<KMAX, NF>(S, p, yd, y);
            if (2 * p < KMAX) {
                hold[p] = v;
            } else if (2 * p == KMAX) {
                low = v;                                    // F_KH on every lane
            } else {
                const int q = KMAX - p;
                const double fq = S.inA ? v : hold[q];
                low = (q == KH) ? fq : fma(low, a, fq);     // q == KH: the first low term (odd KMAX)
                park[(p - KH - 1) * kBlock] = S.inA ? hold[q] : v;  // F_p
            }
        }
        double r = low;
        if (NH > 0) {
            double high = park[(NH - 1) * kBlock];
#pragma unroll
            for (int j = NH - 2; j >= 0; --j) high = fma(high, a, park[j * kBlock]);
            // a^(KH+1) from |a| on the integer pipes, with the sign of a^(KH+1);
            // 0 for a zero or subnormal a (the format's zero must not be
            // powered: its exponent would overflow)
            const long long ab = __double_as_longlong(a);
            const xf::Xf P = xf_pow<KH + 1>(xf::from_double(__longlong_as_double(ab & 0x7FFFFFFFFFFFFFFFLL)));
            double w = P.e > 1023 ? __longlong_as_double(0x7FF0000000000000LL) : xf::to_double(P);
            if ((ab & 0x7FF0000000000000LL) == 0) w = 0.0;
            if (ab < 0 && ((KH + 1) & 1)) w = -w;
            r = fma(w, high, low);
        }
        __stcs(out + i, r);
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
