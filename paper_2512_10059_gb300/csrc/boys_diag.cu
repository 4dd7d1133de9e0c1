// Diagnostic entry point: evaluates the elementary functions of boys_math.cuh
// (FP64) and boys_xf.cuh (integer pipes) elementwise, so that tests can
// measure them against CUDA's own functions and an extended-precision
// reference.
#include "boys_internal.h"
#include "boys_math.cuh"
#include "boys_xf.cuh"

namespace boys {
namespace {

__global__ void k_diag_math(int fn, const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                            double* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double v = a[i];
        double r;
        switch (fn) {
            case 0: r = dmath::exp_neg(v); break;
            case 1: r = dmath::rcp(v); break;
            case 2: r = dmath::div(b[i], v); break;
            case 3: r = dmath::rsqrt(v); break;
            default: {  // integer pipes: e^{-v} (4) or v^{-1/2} (5), the 64-bit significand rounded to nearest
                const xf::Xf e = fn == 4 ? xf::exp_neg(v) : xf::rsqrt(xf::from_double(v));
                const double hi = (double)(e.m >> 11), lo = (double)(e.m & 0x7FF);
                r = ldexp(hi + lo * 0x1p-11, e.e - 52);
                break;
            }
        }
        out[i] = r;
    }
}

}  // namespace
}  // namespace boys

BOYS_API boys_status boys_diag_math(int fn, const double* a, const double* b, int64_t n, double* out, void* stream) {
    using namespace boys;
    if (fn < 0 || fn > 5) return fail(BOYS_ERR_INVALID_ARG, "boys_diag_math: fn=%d outside [0, 5]", fn);
    if (n < 0) return fail(BOYS_ERR_INVALID_ARG, "boys_diag_math: n < 0");
    if (n == 0) return BOYS_OK;
    if (!a || !out || (fn == 2 && !b)) return fail(BOYS_ERR_INVALID_ARG, "boys_diag_math: NULL pointer");
    const int64_t grid = grid_for((const void*)k_diag_math, 256, n, 256);
    k_diag_math<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(fn, a, b, n, out);
    return check_cuda(cudaGetLastError(), "boys_diag_math launch");
}
