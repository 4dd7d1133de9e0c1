// A floating-point format with a 64-bit integer significand, evaluated on the
// integer pipes: value = m * 2^(e - 63) with 2^63 <= m < 2^64 (or m == 0 for
// zero, whose exponent is kXfZeroExp so that it never dominates an addition).
//
// Why: on GB300 one FP64 instruction costs the issue time of ~60 FP32/INT
// ones, and the Boys recurrences are 2 FP64 instructions per order.  Carried
// out in this format they run on the integer pipes with 2^-62 relative
// rounding per operation (finer than FP64's 2^-53) and the full exponent
// range, so the FP64 accuracy of the method (5e-14 absolute, Appendix B's
// round-off analysis) is kept; results go back to IEEE doubles by integer
// assembly of their bit patterns (truncation, < 1 ulp).  Products keep the
// high 64 bits of the 128-bit significand product; sums align to the larger
// exponent with 2 bits of headroom and renormalise with a leading-zero count
// (the product feeding an addition skips its own renormalisation, and the
// addend e^{-x} is shifted and signed once per argument).
#pragma once

#include <cstdint>

#include "boys_xf_consts.h"

namespace boys {
namespace xf {

struct Xf {
    unsigned long long m;
    int e;
};

constexpr int kXfZeroExp = -(1 << 28);

static __constant__ unsigned long long c_odd_m[64] = BOYS_XF_ODD_M_INIT;
static __constant__ int c_odd_e[64] = BOYS_XF_ODD_E_INIT;
static __constant__ unsigned long long c_rodd_m[64] = BOYS_XF_RECIP_ODD_M_INIT;
static __constant__ int c_rodd_e[64] = BOYS_XF_RECIP_ODD_E_INIT;

__device__ __forceinline__ Xf zero() { return Xf{0ULL, kXfZeroExp}; }

// Non-negative finite double -> Xf (subnormals and zero -> zero).
__device__ __forceinline__ Xf from_double(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int be = (int)((b >> 52) & 0x7FF);
    Xf r;
    r.m = ((b & 0xFFFFFFFFFFFFFULL) | 0x10000000000000ULL) << 11;
    r.e = be - 1023;
    return be == 0 ? zero() : r;
}

// Bit pattern of a normalised Xf as a double, truncating the significand to
// 53 bits; meaningful for -1022 <= e <= 1023.
__device__ __forceinline__ unsigned long long double_bits(Xf v) {
    return ((unsigned long long)(long long)(v.e + 1022) << 52) + (v.m >> 11);  // the hidden bit adds the last 1
}

// Xf -> double; values below the normal range flush to zero.  Every zero of
// this format (from zero(), or a product or sum with a zero operand) carries
// an exponent within a few thousand of kXfZeroExp, so the exponent test alone
// also catches m == 0.
__device__ __forceinline__ double to_double(Xf v) {
    return v.e < -1022 ? 0.0 : __longlong_as_double((long long)double_bits(v));
}

__device__ __forceinline__ Xf mul(Xf a, Xf b) {
    const unsigned long long hi = __umul64hi(a.m, b.m);  // in [2^62, 2^64) for normalised inputs
    const int top = (int)(hi >> 63);
    Xf r;
    r.m = top ? hi : (hi << 1);
    r.e = a.e + b.e + top;
    return r;
}

// Product without renormalisation: the high half of the significand product
// with the exponent that keeps value = m * 2^(e - 63) exact (m then has up to
// three leading zero bits).  For operands of an addition, which renormalises.
__device__ __forceinline__ Xf mul_raw(Xf a, Xf b) {
    Xf r;
    r.m = __umul64hi(a.m, b.m);
    r.e = a.e + b.e + 1;
    return r;
}

// A signed addend prepared once: value = m * 2^(e - 61), |m| < 2^62.
struct XfS {
    long long m;
    int e;
};

__device__ __forceinline__ XfS prepare_addend(Xf s, bool negate) {
    const long long v = (long long)(s.m >> 2);
    return XfS{negate ? -v : v, s.e};
}

// t + s for t >= 0 (normalised or not) and a prepared signed addend s whose
// exact sum with t is >= 0; a result at or below zero gives zero.
__device__ __forceinline__ Xf add_prepared(Xf t, XfS s) {
    const int E = max(t.e, s.e);
    const long long tm = (long long)(t.m >> min(E - t.e + 2, 63));
    const long long sm = s.m >> min(E - s.e, 63);  // arithmetic shift keeps the sign
    const long long u = tm + sm;                   // |tm|, |sm| < 2^62: no overflow
    const int lz = __clzll(u);
    Xf r;
    r.m = (unsigned long long)u << lz;
    r.e = E + 2 - lz;
    return u > 0 ? r : zero();
}

__device__ __forceinline__ Xf odd(int j) { return Xf{c_odd_m[j], c_odd_e[j]}; }        // 2j+1
__device__ __forceinline__ Xf recip_odd(int l) { return Xf{c_rodd_m[l], c_rodd_e[l]}; }  // 1/(2l+1)

__device__ __forceinline__ Xf select(bool p, Xf a, Xf b) { return p ? a : b; }

}  // namespace xf
}  // namespace boys
