// Double-precision elementary functions for the FP64 path, written for GB300's
// FP64 budget (one DFMA costs the issue time of ~60 FFMAs, so every FP64
// instruction saved is throughput).  Each is a published method, tested
// against CUDA's own results in tests/test_math_fp64.py:
//   * reciprocal / division: Newton–Raphson from the hardware seed
//     (rcp.approx.ftz.f64, ~2^-20 relative), with the corrected quotient
//     y + r (p - q y) of Markstein (IBM J. Res. Dev. 34(1), 1990);
//   * inverse square root: Newton–Raphson y += y (1 - x y^2) / 2 from
//     rsqrt.approx.ftz.f64 (~2^-20);
//   * e^{-x}: Tang's table-driven method (ACM TOMS 15(2), 1989) with 64
//     subintervals: x = n ln2/64 + r, |r| <= ln2/128, Cody–Waite reduction,
//     e^{-x} = 2^{-floor(n/64)} * 2^{-(n mod 64)/64} * e^{-r}, with
//     e^{-r} - 1 from its Taylor polynomial of degree 5 (remainder
//     < r^6/720 < 3.6e-17) added to the table value with one fused rounding.
#pragma once

#include "boys_exp_table.h"

namespace boys {
namespace dmath {

static __device__ double g_exp2_neg_j64[64] = BOYS_EXP2_NEG_J64_INIT;

__device__ __forceinline__ double rcp_seed(double q) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(q));
    return r;
}

__device__ __forceinline__ double rsqrt_seed(double x) {
    double r;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return r;
}

// 1/q for normal q: two Newton steps from the ~2^-20 seed (2^-40, then
// rounding-limited); 4 FP64 instructions.
__device__ __forceinline__ double rcp(double q) {
    double r = rcp_seed(q);
    double e = fma(-q, r, 1.0);
    r = fma(r, e, r);
    e = fma(-q, r, 1.0);
    return fma(r, e, r);
}

// p/q for normal q: one Newton step (2^-40) and the corrected quotient;
// 5 FP64 instructions, within an ulp.
__device__ __forceinline__ double div(double p, double q) {
    double r = rcp_seed(q);
    const double e = fma(-q, r, 1.0);
    r = fma(r, e, r);
    const double y = p * r;
    const double t = fma(-q, y, p);
    return fma(r, t, y);
}

// x^{-1/2} for normal x: two Newton steps in the form
// y += y * (1/2 - (x/2) y^2); 7 FP64 instructions.
__device__ __forceinline__ double rsqrt(double x) {
    const double hx = 0.5 * x;
    double y = rsqrt_seed(x);
    double e = fma(-hx * y, y, 0.5);
    y = fma(y, e, y);
    e = fma(-hx * y, y, 0.5);
    return fma(y, e, y);
}

// e^{-x} for 0 <= x <= 700 (callers pass 0 for arguments that do not need it).
__device__ __forceinline__ double exp_neg(double x) {
    const double kInvLn2Over64 = 0x1.71547652b82fep+6;   // 64 / ln 2
    const double kShift = 0x1.8p52;                      // 1.5 * 2^52: round to integer
    const double kLn2Over64Hi = 0x1.62e42fefa0000p-7;    // ln2/64, 37 leading bits (n*hi exact)
    const double kLn2Over64Lo = 0x1.cf79abc9e3b3ap-46;   // ln2/64 - hi
    const double t = fma(x, kInvLn2Over64, kShift);
    const int n = __double2loint(t);                     // round(64 x / ln 2)
    const double nd = t - kShift;
    double r = fma(-nd, kLn2Over64Hi, x);
    r = fma(-nd, kLn2Over64Lo, r);
    // q = e^{-r} - 1 = r (-1 + r (1/2 + r (-1/6 + r (1/24 - r/120)))), then
    // T (1 + q) = fma(T, q, T) with a single rounding
    double p = fma(-1.0 / 120.0, r, 1.0 / 24.0);
    p = fma(p, r, -1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r, -1.0);
    const double q = r * p;
    const double tj = __ldg(&g_exp2_neg_j64[n & 63]);
    const double v = fma(tj, q, tj);
    // times 2^{-floor(n/64)}: v is in [0.5, 1.01] and the result stays normal
    return __hiloint2double(__double2hiint(v) - ((n >> 6) << 20), __double2loint(v));
}

}  // namespace dmath
}  // namespace boys
