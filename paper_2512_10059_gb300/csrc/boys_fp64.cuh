// FP64 evaluation of F_0..F_KMAX at one argument: the paper's Algorithm 1
// (Section II.E) with the Appendix D coefficients, written so that every lane
// of a warp executes the same instruction stream whatever region its x is in.
//
//   A = [0, x_0):   F_KMAX = r_{A,KMAX}(x) = P(x)/Q(x), then downward
//                   F_l = (2x F_{l+1} + e^{-x}) / (2l+1)      (Eq. downwardsrecursion)
//   B = [x_0, x_1): F_0 = r_B(x), then upward
//                   F_{l+1} = ((2l+1) F_l - e^{-x}) / (2x)    (Eq. upwardsrecursion)
//   C = [x_1, inf): F_0 = sqrt(pi)/2 x^{-1/2}, then F_{l+1} = (2l+1)/(2x) F_l
//                   (Eq. asymptoticapproximation; the same step as B with e^{-x} := 0)
//
// Region membership is half-open (Eq. regions): x == x_0 is in B, x == x_1 in C.
// Branch-free form: both rationals are evaluated by one Horner loop whose
// coefficient is selected per lane (the shorter polynomial is padded with
// leading zeros, which leaves its value bit-identical), and one step loop
//     y_{j+1} = (a_j * y_j + s) * c_j
// covers all three regions with per-lane operands:
//     A:  a_j = 2x,      s = +e^{-x},  c_j = 1/(2l+1), l = KMAX-1-j  (y_j = F_{KMAX-j})
//     B:  a_j = 2j+1,    s = -e^{-x},  c_j = 1/(2x)                  (y_j = F_j)
//     C:  a_j = 2j+1,    s = 0,        c_j = 1/(2x)
// Division by 2l+1 is a multiplication by the rounded constant 1/(2l+1); the
// paper's zeroth-order error analysis (Appendix B) is indifferent to it.
#pragma once

#include <cstdint>

#include "boys_coeffs_fp64.h"

namespace boys {
namespace fp64 {

constexpr int kRaN[33] = BOYS_RA_N_INIT;
constexpr int kRaM[33] = BOYS_RA_M_INIT;
constexpr double kX0 = BOYS_FP64_X0;
constexpr double kX1 = BOYS_FP64_X1;
constexpr double kSqrtPiOver2 = 0.88622692545275801364908374167057259139877473;

static __constant__ double c_ra_p[33][BOYS_RA_PLEN] = BOYS_RA_P_INIT;
static __constant__ double c_ra_q[33][BOYS_RA_QLEN] = BOYS_RA_Q_INIT;
// r_B padded with zeros to the r_A row lengths
static __constant__ double c_rb_p[BOYS_RA_PLEN] = BOYS_RB_P_INIT;
static __constant__ double c_rb_q[BOYS_RA_QLEN] = BOYS_RB_Q_INIT;

constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <int K>
struct Degrees {
    static constexpr int NP = cmax(kRaN[K], BOYS_RB_N);  // common numerator degree
    static constexpr int NQ = cmax(kRaM[K], BOYS_RB_M);  // common denominator degree
    static_assert(NP < BOYS_RA_PLEN && NQ < BOYS_RA_QLEN, "padding too short");
};

__device__ __forceinline__ double quiet_nan() { return __longlong_as_double(0x7ff8000000000000LL); }

// F_0..F_KMAX (KMAX <= 32) at x; results in F[0..KMAX].
template <int KMAX>
__device__ __forceinline__ void eval_point(double x, double (&F)[KMAX + 1]) {
    static_assert(KMAX >= 0 && KMAX <= 32, "tables cover orders 0..32");
    constexpr int NP = Degrees<KMAX>::NP;
    constexpr int NQ = Degrees<KMAX>::NQ;

    x = (x >= 0.0) ? x : quiet_nan();  // x < 0 and NaN -> NaN everywhere
    const bool inA = x < kX0;
    const bool inC = x >= kX1;

    // Anchor: r_{A,KMAX} in A, r_B in B (Horner, monic denominators).
    double p = inA ? c_ra_p[KMAX][NP] : c_rb_p[NP];
#pragma unroll
    for (int i = NP - 1; i >= 0; --i) p = fma(p, x, inA ? c_ra_p[KMAX][i] : c_rb_p[i]);
    double q = inA ? c_ra_q[KMAX][NQ] : c_rb_q[NQ];
#pragma unroll
    for (int i = NQ - 1; i >= 0; --i) q = fma(q, x, inA ? c_ra_q[KMAX][i] : c_rb_q[i]);
    const double rat = p / q;

    const double asym0 = kSqrtPiOver2 * rsqrt(x);  // region C anchor
    const double e = inC ? 0.0 : exp(-x);
    const double two_x = x + x;
    const double inv2x = 1.0 / two_x;

    double y[KMAX + 1];
    y[0] = inC ? asym0 : rat;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        const int l = KMAX - 1 - j;
        const double a = inA ? two_x : (double)(2 * j + 1);
        const double c = inA ? (1.0 / (double)(2 * l + 1)) : inv2x;
        const double s = inA ? e : -e;
        y[j + 1] = fma(a, y[j], s) * c;
    }
#pragma unroll
    for (int k = 0; k <= KMAX; ++k) F[k] = inA ? y[KMAX - k] : y[k];
}

}  // namespace fp64
}  // namespace boys
