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
// The anchors p/q, F_0 in C and 1/(2x) come from one inverse square root in
// the 64-bit-significand format; it, e^{-x}, most recurrence steps and, at
// small kmax, the denominator q run on the integer pipes (boys_xf.cuh), and
// region tests compare bit patterns there too: the FP64 pipe evaluates the
// Horner sums and whatever recurrence steps the balance gives it.
#pragma once

#include <cstdint>

#include "boys_coeffs_fixed.h"
#include "boys_coeffs_fp64.h"
#include "boys_math.cuh"
#include "boys_xf.cuh"

namespace boys {
namespace fp64 {

// Recurrence steps that run in FP64; the rest use the 64-bit-significand
// integer format (boys_xf.cuh), and e^{-x} always runs on the integer pipes
// (xf::exp_neg).  The set-up's FP64 work (at most the denominator's Horner
// sum) is the same at every kmax while the integer pipes take one step per
// order, so the balance depends on kmax only (the kernels are branch-free, so
// not on the argument mix).  Swept on GB300 (stored mode, N = 2^26, every kmax
// x 0..22 FP64 steps, median of 3, with the kernel's register caps and grid):
// with the denominator in FP64 (kmax <= 5 and 7) at most 2 steps; with both
// Horner sums on the integer pipes every step up to kmax = 8, then about
// kmax / 2 + 1 up to kmax = 20 and fewer above, 15 at kmax = 32 (4.55 ms,
// against 6.26 with none, 4.82 with 12, 4.59 with 17 and 5.04 with 20).
// Defining BOYS_FP64_STEPS forces one value for every kmax.
constexpr int kFp64Steps[33] = {0, 0, 0, 0, 2, 0, 6, 2, 8, 8, 8, 9, 9, 9, 10, 10, 11,
                                11, 11, 12, 12, 11, 12, 12, 13, 14, 14, 14, 14, 14, 15, 16, 15};
// The anchor's numerator p runs as a fixed-point Horner sum on the integer
// pipes for kmax up to BOYS_FIXED_P_MAXK (-1: never), the denominator q in
// FP64.  A fixed binary point serves the numerators (degree <= 8) to about
// 1e-17 of the anchor, but not the denominators of degree 12 and 13; q in a
// floating integer format (about 30 instructions a step) was slower than the
// FP64 Horner sum at every kmax (kmax 4: 2.71 ms against 2.07; kmax 32: 6.71
// against 5.30).
#ifndef BOYS_FIXED_P_MAXK
#define BOYS_FIXED_P_MAXK 32
#endif
#ifndef BOYS_FIXED_Q_MAXK
#define BOYS_FIXED_Q_MAXK 32
#endif
// Denominators in fixed point from kmax = 6 on, except the degree-13
// denominator of k = 7: there it adds at most 4.1e-16 to the anchor (the
// degree-12 and -13 denominators, k = 3, 5, 7, would add up to 2.4e-15), and
// it pays once the FP64 pipe carries recurrence steps (kmax 8: 2.17 ms against
// 2.33; kmax 32: 4.86 against 5.06).  Below kmax 6 the FP64 Horner sum costs
// no time (kmax 0: 1.10 ms against 1.16 in fixed point) and is kept.
constexpr bool fixed_q_for(int kmax) {
    return kmax >= 6 && kmax != 7 && kmax <= BOYS_FIXED_Q_MAXK;
}

constexpr int fp64_steps_for(int kmax) {
#ifdef BOYS_FP64_STEPS
    return BOYS_FP64_STEPS + 0 * kmax;
#else
    return kFp64Steps[kmax];
#endif
}

// The integer-pipe e^{-x} is the default everywhere; BOYS_INT_EXP_ALWAYS=0
// selects the FP64 one (boys_math.cuh) for comparison.
#ifndef BOYS_INT_EXP_ALWAYS
#define BOYS_INT_EXP_ALWAYS 1
#endif
constexpr bool int_exp_for(int kmax, int nsteps_fp64) {
    return BOYS_INT_EXP_ALWAYS + 0 * (kmax + nsteps_fp64);
}

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
// the same in 64-bit fixed point (value = V 2^-f, t = x/16 in A, x/32 in B)
static __constant__ long long c_ra_p_fx[33][BOYS_RA_PLEN] = BOYS_RA_P_FX_INIT;
static __constant__ long long c_rb_p_fx[BOYS_RA_PLEN] = BOYS_RB_P_FX_INIT;
static __constant__ long long c_ra_q_fx[33][BOYS_RA_QLEN] = BOYS_RA_Q_FX_INIT;
static __constant__ long long c_rb_q_fx[BOYS_RA_QLEN] = BOYS_RB_Q_FX_INIT;
constexpr int kRaPFxf[33] = BOYS_RA_P_FXF_INIT;
constexpr int kRaQFxf[33] = BOYS_RA_Q_FXF_INIT;

constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <int K>
struct Degrees {
    static constexpr int NP = cmax(kRaN[K], BOYS_RB_N);  // common numerator degree
    static constexpr int NQ = cmax(kRaM[K], BOYS_RB_M);  // common denominator degree
    static_assert(NP < BOYS_RA_PLEN && NQ < BOYS_RA_QLEN, "padding too short");
};

__device__ __forceinline__ double quiet_nan() { return __longlong_as_double(0x7ff8000000000000LL); }

// Bit patterns of the region boundaries: for non-negative doubles (and +inf)
// the IEEE order equals the integer order of the bit patterns, so the region
// tests run on the integer pipes instead of the scarce FP64 pipe.
constexpr long long kBitsX0 = BOYS_FP64_X0_BITS;
constexpr long long kBitsX1 = BOYS_FP64_X1_BITS;
constexpr long long kBitsInf = 0x7FF0000000000000LL;
constexpr long long kBits1e300 = 0x7E37E43C8800759CLL;  // 1e300

// Everything Algorithm 1 needs before the recurrence, for one argument.
struct Setup {
    bool valid, inA;
    double y0d, two_x, sd, inv2x;   // FP64 anchor, 2x, s = +-e^{-x} (0 in C), 1/(2x)
    xf::Xf y0, X2, Ev, R;           // the same in the 64-bit-significand format
    xf::XfS Es;                     // s = +e^{-x} (A) or -e^{-x} (B), 0 (C), ready to add
};

enum Region { kRegionA = 0, kRegionB = 1, kRegionC = 2, kRegionNone = 3 };

// Set-up for one argument.  MODE = kRegionNone takes any x (branch-free:
// every lane evaluates the arithmetic of all three regions and selects);
// MODE = kRegionA/B/C is for x known to be valid and in that region, where
// the other regions' work folds away at compile time.
//
// Branch-free, one inverse square root serves all three anchors: r = z^{-1/2}
// with z = q^2 in A, (2x q)^2 in B and x in C, so that
//   A: p/q = |p| r,  B: p/q = 2x |p| r,  1/(2x) = |q| r,
//   C: F_0 = (sqrt(pi)/2) r,  1/(2x) = r (r/2)
// (p and q have one common sign on each region's interval, since p/q
// approximates a positive F_k, and |q| lies in [2e7, 7e16] for every table
// row).  All of it runs in the 64-bit-significand format on the integer pipes
// (xf::rsqrt, xf::mul), about 2^-58 relative in all, against 3 ulp for the
// same chain in FP64, which took 14 FP64 instructions per argument.  A single
// region (MODE) keeps only its own products.
template <int MODE, int KMAX, bool INT_EXP = false>
__device__ __forceinline__ Setup setup_mode(double x) {
    static_assert(KMAX >= 0 && KMAX <= 32, "tables cover orders 0..32");
    constexpr int NP = Degrees<KMAX>::NP;
    constexpr int NQ = Degrees<KMAX>::NQ;

    long long xb = __double_as_longlong(x);
    if (xb == (long long)0x8000000000000000ULL) xb = 0;  // -0.0 -> +0.0
    bool valid = true, inA = MODE == kRegionA, inC = MODE == kRegionC;
    if (MODE == kRegionNone) {
        valid = xb >= 0 && xb <= kBitsInf;                // x < 0 and NaN -> NaN everywhere
        inA = valid && xb < kBitsX0;
        inC = !valid || xb >= kBitsX1;
    }
    x = valid ? __longlong_as_double(xb) : quiet_nan();

    // Anchor: r_{A,KMAX} in A, r_B in B (Horner, monic denominators).  The
    // numerator p: fixed-point Horner on the integer pipes in t = x/16 (A) or
    // x/32 (B), t in Q64 (t < 1 on both regions; other lanes get a clamped
    // t whose result is not used), or FP64 Horner.
    constexpr bool kFixedP = KMAX <= BOYS_FIXED_P_MAXK;
    constexpr bool kFixedQ = fixed_q_for(KMAX);
    double p = 0.0, q = 0.0;
    xf::Xf Pfx = xf::zero(), Qfx = xf::zero();
    if (kFixedP || kFixedQ) {
        const unsigned long long xbu = (unsigned long long)xb;
        const int be = (int)((xbu >> 52) & 0x7FF);
        const unsigned long long mant = (xbu & 0xFFFFFFFFFFFFFULL) | 0x10000000000000ULL;
        const int sh = be - (inA ? 1075 - 64 + BOYS_FX_SHIFT_A : 1075 - 64 + BOYS_FX_SHIFT_B);  // t 2^64 = mant 2^sh
        unsigned long long T = sh >= 0 ? (mant << min(sh, 11)) : (mant >> min(-sh, 63));
        if (be == 0) T = 0;
        const unsigned long long Th = T >> 1;
        if (kFixedP) {
            long long v = inA ? c_ra_p_fx[KMAX][NP] : c_rb_p_fx[NP];
#pragma unroll
            for (int i = NP - 1; i >= 0; --i) v = xf::mulhi_s(v, T, Th) + (inA ? c_ra_p_fx[KMAX][i] : c_rb_p_fx[i]);
            constexpr int kFa = kRaPFxf[KMAX];
            Pfx = xf::from_fixed(v, inA ? kFa : BOYS_RB_P_FXF);
        }
        if (kFixedQ) {
            long long v = inA ? c_ra_q_fx[KMAX][NQ] : c_rb_q_fx[NQ];
#pragma unroll
            for (int i = NQ - 1; i >= 0; --i) v = xf::mulhi_s(v, T, Th) + (inA ? c_ra_q_fx[KMAX][i] : c_rb_q_fx[i]);
            constexpr int kFa = kRaQFxf[KMAX];
            Qfx = xf::from_fixed(v, inA ? kFa : BOYS_RB_Q_FXF);
        }
    }
    if (!kFixedP) {
        p = inA ? c_ra_p[KMAX][NP] : c_rb_p[NP];
#pragma unroll
        for (int i = NP - 1; i >= 0; --i) p = fma(p, x, inA ? c_ra_p[KMAX][i] : c_rb_p[i]);
    }
    if (!kFixedQ) {
        q = inA ? c_ra_q[KMAX][NQ] : c_rb_q[NQ];
#pragma unroll
        for (int i = NQ - 1; i >= 0; --i) q = fma(q, x, inA ? c_ra_q[KMAX][i] : c_rb_q[i]);
    }

    // Arguments beyond 1e300 are clamped there in C (F_0 < 1e-150 and F_k = 0
    // for k > 0 either way); +inf gives exactly 0.
    const bool huge = xb > kBits1e300 && xb <= kBitsInf;
    const xf::Xf X = xf::from_double(huge ? 1e300 : x);
    const xf::Xf X2{X.m, X.e + 1};  // 2x, exact
    // The anchors from one inverse square root in the 64-bit-significand
    // format (integer pipes): r = z^{-1/2} with z = q^2 (A), (2x q)^2 (B), x (C).
    // p/q > 0 on both regions, so magnitudes suffice (from_double drops signs).
    const xf::Xf P = kFixedP ? Pfx : xf::from_double(p);
    const xf::Xf Q = kFixedQ ? Qfx : xf::from_double(q);
    xf::Xf y0, R;
    if (MODE == kRegionNone) {
        const xf::Xf tq = inA ? Q : xf::mul(X2, Q);
        const xf::Xf r = xf::rsqrt(inC ? X : xf::mul(tq, tq));
        y0 = xf::mul(inA ? P : (inC ? xf::sqrt_pi_over_2() : xf::mul(X2, P)), r);
        R = xf::mul(inC ? xf::Xf{r.m, r.e - 1} : Q, r);
    } else if (MODE == kRegionA) {
        y0 = xf::mul(P, xf::rsqrt(xf::mul(Q, Q)));
        R = xf::zero();
    } else if (MODE == kRegionB) {
        const xf::Xf tq = xf::mul(X2, Q);
        const xf::Xf r = xf::rsqrt(xf::mul(tq, tq));
        y0 = xf::mul(xf::mul(X2, P), r);
        R = xf::mul(Q, r);
    } else {
        const xf::Xf r = xf::rsqrt(X);
        y0 = xf::mul(xf::sqrt_pi_over_2(), r);
        R = xf::mul(xf::Xf{r.m, r.e - 1}, r);
    }
    // +inf gives exactly 0; an invalid argument starts the integer-format
    // recurrence from zero (its values flush to NaN in out_value) and the
    // FP64 one from NaN, which every FP64 step propagates.
    if (xb == kBitsInf || !valid) y0 = xf::zero();
    // e^{-x}: on the integer pipes, straight into the recurrence's format, when
    // no step runs in FP64 (the FP64 copy is then only assembled if used)
    double e;
    xf::Xf E;
    if (INT_EXP) {
        E = xf::exp_neg(inC ? 0.0 : x);
        e = xf::to_double(E);
    } else {
        e = dmath::exp_neg(inC ? 0.0 : x);
        E = xf::from_double(e);
    }

    Setup S;
    S.valid = valid;
    S.inA = inA;
    S.y0 = y0;
    S.y0d = valid ? xf::to_double(y0) : quiet_nan();
    S.X2 = X2;
    S.two_x = xf::to_double(X2);
    S.sd = inC ? 0.0 : (inA ? e : -e);
    S.R = R;
    S.inv2x = xf::to_double(R);
    S.Ev = inC ? xf::zero() : E;                     // zero in region C
    S.Es = xf::prepare_addend(S.Ev, !inA);
    return S;
}

template <int KMAX, bool INT_EXP = false>
__device__ __forceinline__ Setup setup(double x) {
    return setup_mode<kRegionNone, KMAX, INT_EXP>(x);
}

__device__ __forceinline__ int region_of(double x) {
    long long xb = __double_as_longlong(x);
    if (xb == (long long)0x8000000000000000ULL) xb = 0;
    if (!(xb >= 0 && xb <= kBitsInf)) return kRegionNone;  // x < 0 or NaN
    return xb < kBitsX0 ? kRegionA : (xb < kBitsX1 ? kRegionB : kRegionC);
}

// One step y_{j+1} = (a_j y_j + s) c_j of the unified recurrence, in the
// 64-bit-significand format of boys_xf.cuh on the integer pipes:
//   A: a_j = 2x, s = +e^{-x}, c_j = 1/(2l+1), l = KMAX-1-j  (y_j = F_{KMAX-j})
//   B: a_j = 2j+1, s = -e^{-x}, c_j = 1/(2x)                (y_j = F_j)
//   C: a_j = 2j+1, s = 0,        c_j = 1/(2x)
template <int KMAX>
__device__ __forceinline__ xf::Xf step(const Setup& S, int j, xf::Xf y) {
    const int l = KMAX - 1 - j;
    const xf::Xf a = xf::select(S.inA, S.X2, xf::odd(j));
    const xf::Xf c = xf::select(S.inA, xf::recip_odd(l), S.R);
    return xf::mul_norm(xf::add_raw(xf::mul_raw(a, y), S.Es), c);
}

// One select per output: NaN for an invalid argument, 0 below the normal
// range (see xf::to_double), the value otherwise.
__device__ __forceinline__ double out_value(const Setup& S, xf::Xf y) {
    const double flush = S.valid ? 0.0 : quiet_nan();
    return (y.e < -1022 || !S.valid) ? flush : __longlong_as_double((long long)xf::double_bits(y));
}

// The same step in FP64 (y_{j+1} = fma(a_j, y_j, s) * c_j).
template <int KMAX>
__device__ __forceinline__ double step_fp64(const Setup& S, int j, double y) {
    const int l = KMAX - 1 - j;
    const double a = S.inA ? S.two_x : (double)(2 * j + 1);
    const double c = S.inA ? (1.0 / (double)(2 * l + 1)) : S.inv2x;
    return fma(a, y, S.sd) * c;
}

// Value number p of the recurrence (p = 0: the anchor; FP64 for p <= NF64,
// the integer format after), advancing yd / y in place.  FP64 values need no
// select: an invalid argument's yd is NaN from the anchor on.
template <int KMAX, int NSTEPS_FP64 = fp64_steps_for(KMAX)>
__device__ __forceinline__ double next_value(const Setup& S, int p, double& yd, xf::Xf& y) {
    constexpr int NF64 = NSTEPS_FP64 < KMAX ? NSTEPS_FP64 : KMAX;
    if (p <= NF64) {
        if (p > 0) yd = step_fp64<KMAX>(S, p - 1, yd);
        return yd;
    }
    if (p - 1 == NF64 && p > 1) y = S.valid ? xf::from_double(yd) : xf::zero();
    y = step<KMAX>(S, p - 1, y);
    return out_value(S, y);
}

// F_0..F_KMAX (KMAX <= 32) at x; results in F[0..KMAX].  NSTEPS_FP64 lets a
// caller whose own work already loads the FP64 pipe move more steps to the
// integer format; stored and ragged modes use the default and agree bitwise.
template <int KMAX, int NSTEPS_FP64 = fp64_steps_for(KMAX), bool INT_EXP = int_exp_for(KMAX, NSTEPS_FP64)>
__device__ __forceinline__ void eval_point(double x, double (&F)[KMAX + 1]) {
    const Setup S = setup<KMAX, INT_EXP>(x);
    double yd = S.y0d;
    xf::Xf y = S.y0;
    double v[KMAX + 1];
#pragma unroll
    for (int p = 0; p <= KMAX; ++p) v[p] = next_value<KMAX, NSTEPS_FP64>(S, p, yd, y);
#pragma unroll
    for (int k = 0; k <= KMAX; ++k) F[k] = S.inA ? v[KMAX - k] : v[k];
}

// Same values, stored by the whole warp: F_k(x) to col[k * ld].  Value number
// p of the recurrence (p = 0 is the anchor) is F_{KMAX-p} on an A lane and
// F_p on a B or C lane, so row k is complete once both p = k and p = KMAX-k
// have been produced.  A lane therefore keeps its values p < KMAX/2 (at most
// 17 doubles); from p >= KMAX/2 on, step p completes rows p and KMAX-p for
// every lane of the warp and the two stores of that step cover both rows
// completely between them, so L2 holds whole lines when they go to DRAM (a
// value stored as soon as it is produced would leave rows partly written for
// many steps, and L2 would evict partly written sectors that DRAM then
// read-modify-writes).
//
// FULL_ROWS selects the store pattern.  false (device memory): each of the
// step's two stores picks its row per lane, so each writes two half rows that
// L2 merges before DRAM (cheaper on the ALU).  true (host memory over the
// host link, where partial writes are not merged and would double the link
// traffic): each store picks its value per lane and writes one full row.
template <int KMAX, bool FULL_ROWS = false>
__device__ __forceinline__ void eval_store(double x, double* __restrict__ col, int64_t ld) {
    constexpr int H = KMAX / 2 + 1;
    const Setup S = setup<KMAX, int_exp_for(KMAX, fp64_steps_for(KMAX))>(x);
    double hold[H];
    // Value p belongs to row KMAX - p on an A lane and to row p otherwise:
    // row colp + p sld on every lane, and the held value's row colp + q sld
    // (q = KMAX - p), with a lane's base and row stride chosen once.
    double* const colp = S.inA ? col + (int64_t)KMAX * ld : col;
    const int64_t sld = S.inA ? -ld : ld;
    double yd = S.y0d;
    xf::Xf y = S.y0;
#pragma unroll
    for (int p = 0; p <= KMAX; ++p) {
        const double v = next_value<KMAX>(S, p, yd, y);
        if (2 * p < KMAX) {
            hold[p] = v;
        } else if (2 * p == KMAX) {
            __stcs(colp + p * sld, v);
        } else {
            // rows p and q = KMAX - p: this step's value is F_q on an A lane and
            // F_p otherwise; the held one is the other.  Picking the row per
            // lane (an address IMAD on the FMA pipe) instead of the value (two
            // SELs per double on the ALU) makes each store write two half rows,
            // which L2 merges before DRAM (kmax 32: 5.32 -> 5.24 ms; the lane's
            // base and stride instead of a row select per store: 4.68 -> 4.65).
            const int q = KMAX - p;
            if (FULL_ROWS) {
                __stcs(col + p * ld, S.inA ? hold[q] : v);
                __stcs(col + q * ld, S.inA ? v : hold[q]);
            } else {
                __stcs(colp + p * sld, v);
                __stcs(colp + q * sld, hold[q]);
            }
        }
    }
}

}  // namespace fp64
}  // namespace boys
