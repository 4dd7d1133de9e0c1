// A floating-point format with a 64-bit integer significand, evaluated on the
// integer pipes: value = m * 2^(e - 63) with 2^63 <= m < 2^64 (or m == 0 for
// zero, whose exponent is kXfZeroExp so that it never dominates an addition).
//
// Why: on GB300 one FP64 instruction costs the issue time of ~60 FP32/INT
// ones, and the Boys recurrences are 2 FP64 instructions per order.  Carried
// out in this format they run on the integer pipes with about 2^-59 relative
// rounding per operation (finer than FP64's 2^-53) and the full exponent
// range, so the FP64 accuracy of the method (5e-14 absolute, Appendix B's
// round-off analysis) is kept; results go back to IEEE doubles by integer
// assembly of their bit patterns (truncation, < 1 ulp).
//
// The operations are built for the recurrence steps y' = (a y + s) c and cost
// few instructions each:
//  * products keep the high 64 bits of the 128-bit significand product from
//    three 32 x 32-bit partial products (mulhi3: at most 2 units of 2^-64
//    below the exact high half);
//  * a sum aligns both terms to the larger exponent, one bit below the top,
//    and is left unnormalised: the recurrences never cancel more than two
//    leading bits (the upward step (2j+1) F_j - e^{-x} keeps at least 0.36
//    of (2j+1) F_j on region B, and the downward step adds two positive
//    terms), so a sum keeps its leading bit within its top four bits;
//  * the product that follows a sum renormalises by a 32-bit leading-zero
//    count of its high word, so a recurrence step renormalises once; the
//    product feeding a sum skips renormalisation, and the addend e^{-x} is
//    shifted and signed once per argument.
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

// High 64 bits of the 128-bit product a b from three 32 x 32-bit partial
// products: the low x low product and the low halves of the two cross
// products are dropped, so the result is at most 2 below the exact high half
// (never above it).  For a, b >= 2^63 it lies in [2^62, 2^64).
__device__ __forceinline__ unsigned long long mulhi3(unsigned long long a, unsigned long long b) {
    const unsigned a0 = (unsigned)a, a1 = (unsigned)(a >> 32);
    const unsigned b0 = (unsigned)b, b1 = (unsigned)(b >> 32);
    return (unsigned long long)a1 * b1 + __umulhi(a1, b0) + __umulhi(a0, b1);
}

__device__ __forceinline__ Xf mul(Xf a, Xf b) {
    const unsigned long long hi = mulhi3(a.m, b.m);
    const int top = (int)(hi >> 63);
    Xf r;
    r.m = hi << (1 - top);
    r.e = a.e + b.e + top;
    return r;
}

// floor(v t / 2^64) within 3 units, for |v| < 2^63 and t < 2^64, with
// t_half = t >> 1: the biased operand v + 2^63 is unsigned and
// (v + 2^63) t / 2^64 = v t / 2^64 + t / 2.
__device__ __forceinline__ long long mulhi_s(long long v, unsigned long long t, unsigned long long t_half) {
    return (long long)(mulhi3((unsigned long long)v ^ 0x8000000000000000ULL, t) - t_half);
}

// |v| 2^-f as a normalised Xf (v != 0).
__device__ __forceinline__ Xf from_fixed(long long v, int f) {
    const unsigned long long a = v < 0 ? 0ULL - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)a);
    return Xf{a << (lz & 63), 63 - lz - f};
}

// Product without renormalisation: value = m * 2^(e - 63) with m in
// [2^62, 2^64) (one possible leading zero).  For operands of an addition,
// which renormalises.
__device__ __forceinline__ Xf mul_raw(Xf a, Xf b) {
    Xf r;
    r.m = mulhi3(a.m, b.m);
    r.e = a.e + b.e + 1;
    return r;
}

// A signed addend prepared once: value = m * 2^(e - 62), |m| < 2^63.
struct XfS {
    long long m;
    int e;
};

__device__ __forceinline__ XfS prepare_addend(Xf s, bool negate) {
    const long long v = (long long)(s.m >> 1);
    return XfS{negate ? -v : v, s.e};
}

// Logical and arithmetic right shifts by n >= 0 with PTX semantics: shift
// counts of 64 and more give 0 (or the sign), so no clamp is needed.
__device__ __forceinline__ unsigned long long shr_u64(unsigned long long a, int n) {
    unsigned long long r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(a), "r"(n));
    return r;
}
__device__ __forceinline__ long long shr_s64(long long a, int n) {
    long long r;
    asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(a), "r"(n));
    return r;
}

// t + s for a raw product t (m in [2^62, 2^64), or zero) and a prepared
// signed addend s, where either both terms are >= 0 or the exact sum is at
// least a quarter of t (the recurrences' cases).  Both terms are aligned to
// 2^(E - 62), E the larger exponent (t one bit below the top, so two positive
// terms cannot carry out), and added modulo 2^64.  The result is left
// unnormalised for mul_norm: m = u with its leading bit in bits 59..63
// (u >= t/4 >= 2^59 after the alignment), e = E + 1.  A zero sum stays zero
// (m = 0, exponent near kXfZeroExp).
__device__ __forceinline__ Xf add_raw(Xf t, XfS s) {
    const int E = max(t.e, s.e);
    const unsigned long long ta = shr_u64(t.m, E - t.e + 1);
    const long long sa = shr_s64(s.m, E - s.e);  // arithmetic shift keeps the sign
    return Xf{ta + (unsigned long long)sa, E + 1};
}

// a b for an operand a with at most four leading zeros (a sum from add_raw)
// and a normalised b, renormalised by a 32-bit leading-zero count of the high
// word (the product's leading bit lies in bits 57..63; zero stays zero).
// With the leading zeros of a the product keeps about 59 significant bits.
__device__ __forceinline__ Xf mul_norm(Xf a, Xf b) {
    const unsigned long long hi = mulhi3(a.m, b.m);
    const int lz = __clz((int)(hi >> 32));
    Xf r;
    r.m = hi << lz;
    r.e = a.e + b.e + 1 - lz;
    return r;
}

// z^{-1/2} for normalised z > 0 (exponent within +-2^30), relative error
// below 2^-59.  Seed: rsqrt.approx.ftz.f32 of the top 23 bits of z's
// significand with the exponent's parity (z = s 2^(2h), s in [1, 4)), so the
// seed y has |1 - z y^2| < 2^-21 (any |d| < 2^-19 keeps the fixed-point
// ranges below); then one third-order Newton step
//   y' = y (1 + d/2 + 3 d^2/8),  d = 1 - z y^2,
// whose truncation error is 5 d^3/16 < 2^-64.  d is formed in Q62 fixed
// point (z y^2 is within 2^-19 of 1), d^2 from its top 31 bits.
__device__ __forceinline__ Xf rsqrt(Xf z) {
    const int h = z.e >> 1;  // floor(e / 2)
    const float s = __int_as_float(((127 + (z.e & 1)) << 23) | (int)((z.m >> 40) & 0x7FFFFF));
    float sf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(sf) : "f"(s));
    const int sb = __float_as_int(sf);
    const Xf y{(unsigned long long)((sb & 0x7FFFFF) | 0x800000) << 40, ((sb >> 23) & 0xFF) - 127 - h};
    const Xf w = mul(mul(y, y), z);                                   // 1 - d, exponent 0 or -1
    const unsigned long long W = w.m >> min(max(1 - w.e, 0), 63);     // in Q62
    const long long D = (long long)(1ULL << 62) - (long long)W;       // d in Q62, |D| < 2^43
    const int Ds = (int)(D >> 12);
    const unsigned long long D2 = (unsigned long long)((long long)Ds * Ds);  // d^2 in Q38
    const long long C = (D >> 1) + (long long)((3 * D2) >> 41);       // d/2 + 3 d^2/8 in Q62
    const unsigned long long Cm = (unsigned long long)(C < 0 ? -C : C);
    const unsigned long long corr = mulhi3(y.m, Cm << 21) >> 20;      // (y.m / 2) |C| / 2^62
    const unsigned long long hm = y.m >> 1;
    const unsigned long long u = C < 0 ? hm - corr : hm + corr;       // leading bit 61..63
    const int lz = __clz((int)(u >> 32));
    return Xf{u << lz, y.e + 1 - lz};
}

// sqrt(pi)/2, the factor of the asymptotic F_0 of region C.
__device__ __forceinline__ Xf sqrt_pi_over_2() { return Xf{BOYS_XF_SQRTPI_2_M, -1}; }

// (a b) / 2^62 for signed Q62 operands whose product stays below 2^125.
__device__ __forceinline__ long long mul_q62(long long a, long long b) {
    const long long hi = __mul64hi(a, b);
    const unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
    return (long long)(((unsigned long long)hi << 2) | (lo >> 62));
}

// 2^(-j/256) = m * 2^(e-63) with e = 0 for j = 0 and -1 otherwise.
static __device__ unsigned long long g_exp2_neg_j256[256] = BOYS_XF_EXP2_NEG_J256_M_INIT;

// e^{-x} for 0 <= x < 32 in this format, on the integer pipes: Tang's
// table-driven method (ACM TOMS 15(2), 1989) in fixed point.
//   n = round(256 x / ln 2) from x in Q57, r = x - n ln2/256 in Q62 with
//   ln2/256 to 2^-89, so |r| <= ln2/512 + 2^-56, exact to 2^-62;
//   q = e^{-r} - 1 = -r + r^2 (1/2 + r (-1/6 + r (1/24 - r/120))) in Q62:
//   the inner terms, weighted by r^3 and r^4 (< 2.5e-9), take 32-bit
//   operands (their 2^-30 truncation costs < 2^-63), r p1 (weight r^2 <
//   1.9e-6) is formed from two ~31-bit parts (< 2^-61), the rest at full
//   width; the omitted r^6/720 < 1e-20;
//   e^{-x} = 2^{-floor(n/256)} * T_{n mod 256} * (1 + q).
// Relative error below 2^-59.5 (before the conversion to double), checked
// against an exact emulation and a binary128 reference.
__device__ __forceinline__ Xf exp_neg(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int be = (int)((b >> 52) & 0x7FF);
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFULL) | 0x10000000000000ULL;
    const int sh = be - 1018;  // x = mant 2^(be - 1075), x 2^57 = mant 2^sh
    unsigned long long X = sh >= 0 ? (mant << min(sh, 9)) : (mant >> min(-sh, 63));
    if (be == 0) X = 0;
    const unsigned long long t = __umul64hi(X, BOYS_XF_EXP_INVLN2_Q54);  // 256 x / ln2 in Q47
    const long long n = (long long)((t + (1ULL << 46)) >> 47);
    // r in Q62, exact to 2^-62: x 2^62 and n (ln2/256) 2^62 can exceed 64 bits
    // but their difference cannot, so both are formed modulo 2^64
    const int s62 = be - 1013;  // x 2^62 = mant 2^s62
    unsigned long long xq = s62 >= 0 ? (mant << min(s62, 14)) : (mant >> min(-s62, 63));
    if (be == 0) xq = 0;
    const long long r =
        (long long)(xq - (unsigned long long)n * (BOYS_XF_EXP_LN2_HI << 5) -
                    (((unsigned long long)n * BOYS_XF_EXP_LN2_LO + (1ULL << 26)) >> 27));
    const long long rh = r >> 32;                        // Q30
    const long long p0 = (long long)BOYS_XF_EXP_24TH_Q62 - rh * (long long)BOYS_XF_EXP_120TH_Q32;
    const long long p1 = rh * (p0 >> 32) * 4 - (long long)BOYS_XF_EXP_SIXTH_Q62;
    // r p1 from ~31-bit parts (Q41 x Q33, product < 2^62), error < 2^-41.9
    const long long p2 = (long long)BOYS_XF_EXP_HALF_Q62 + (((r >> 21) * (p1 >> 29)) >> 12);
    const long long q = mul_q62(mul_q62(r, r), p2) - r;  // |q| < 0.0014
    const int j = (int)(n & 255);
    const unsigned long long P = __umul64hi(__ldg(&g_exp2_neg_j256[j]), (unsigned long long)((1LL << 62) + q));
    const int lz = __clzll((long long)P);                // 1..3
    Xf res;
    res.m = P << lz;
    res.e = (j ? -1 : 0) + 2 - lz - (int)(n >> 8);
    return res;
}

__device__ __forceinline__ Xf odd(int j) { return Xf{c_odd_m[j], c_odd_e[j]}; }        // 2j+1
__device__ __forceinline__ Xf recip_odd(int l) { return Xf{c_rodd_m[l], c_rodd_e[l]}; }  // 1/(2l+1)

__device__ __forceinline__ Xf select(bool p, Xf a, Xf b) { return p ? a : b; }

}  // namespace xf
}  // namespace boys
