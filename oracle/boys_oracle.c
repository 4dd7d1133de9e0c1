/*
 * Boys-function oracle — TEST INFRASTRUCTURE, not part of the product.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg may build, load or call this file.  It shares no code,
 * header, table or constant with the CUDA library: it does not implement
 * the paper's method (rational minimax + recurrences), it evaluates the
 * function the method approximates, to far more digits than the method's
 * 5e-14 absolute tolerance.
 *
 * Definition (paper, Section 1, Eq. 3):
 *     F_k(x) = \int_0^1 t^{2k} e^{-x t^2} dt,   x in [0, inf), k in N_0.
 *
 * Arithmetic is IEEE binary128 throughout: __float128 + libquadmath on
 * x86-64, `long double` (which is binary128 on AArch64 Linux) + libm on
 * AArch64.  Results are returned as an unevaluated double-double
 * (hi + lo, hi = rounded value) so callers keep ~106 bits.
 *
 * Two evaluation routes:
 *  (1) x < X_SWITCH: the all-positive series used by the paper for its
 *      reference values (Section II "Reference values of Boys functions"):
 *          F_k(x) = (e^{-x}/2) * sum_{l>=0} x^l / prod_{j=0}^{l} (k+j+1/2).
 *      Every order k is summed independently (no recurrence).  The sum is
 *      truncated adaptively with a rigorous geometric tail bound: the ratio
 *      of consecutive terms q_l = x/(k+l+3/2) decreases in l, so once
 *      q_l < 1 the remainder after term t_l is at most t_l*q_l/(1-q_l).
 *      (The paper's fixed L=150 and its bound, Eq. errobound, are not
 *      used: the last step of its derivation in Appendix A bounds F_n from
 *      below by the asymptotic form, which is an upper bound of F_n, so the
 *      printed bound is not valid for small x.)
 *  (2) x >= X_SWITCH: the closed form of F_0 (the k=0 case of Eq. 3,
 *      substituting u = t*sqrt(x)):
 *          F_0(x) = (1/2) sqrt(pi/x) erf(sqrt(x)),
 *      then the upward recurrence (Section II, Eq. upwardsrecursion)
 *          F_{k+1}(x) = ((2k+1) F_k(x) - e^{-x}) / (2x),
 *      an exact identity (integration by parts of Eq. 3).  Its round-off
 *      amplification factor prod_{n<l} (n+1/2)/x is <= 1 for every
 *      l <= 34 once x >= 12.3 (Appendix B, derivation of x_0), so in
 *      binary128 it loses nothing at x >= 30.
 *
 * Domain conventions (the paper defines x >= 0 only): x < 0 or NaN -> NaN
 * for every order; x = +inf -> 0 for every order; -0.0 is treated as 0.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>
#include <float.h>

#if defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 qreal;
#define QEXP expq
#define QERF erfq
#define QSQRT sqrtq
#define QFABS fabsq
#define QL(c) c##Q
#elif defined(__aarch64__)
typedef long double qreal;
_Static_assert(LDBL_MANT_DIG == 113, "oracle needs binary128 long double on AArch64");
#define QEXP expl
#define QERF erfl
#define QSQRT sqrtl
#define QFABS fabsl
#define QL(c) c##L
#else
#error "oracle needs a binary128 type (__float128 on x86-64 or long double on AArch64)"
#endif

#define ORACLE_KMAX 40          /* highest order any oracle entry point accepts */
#define X_SWITCH QL(30.0)       /* series below, erf + upward recurrence at and above */
#define SERIES_REL_TOL QL(1e-40)
#define SERIES_MAX_TERMS 200000

#ifdef _OPENMP
#include <omp.h>
static int oracle_threads(int requested) { return requested > 0 ? requested : omp_get_max_threads(); }
#else
static int oracle_threads(int requested) { (void)requested; return 1; }
#endif

static const qreal Q_PI = QL(3.14159265358979323846264338327950288419716939937510582);

static inline void q_split(qreal v, double* hi, double* lo) {
    double h = (double)v;
    *hi = h;
    *lo = (double)(v - (qreal)h);
}

/* Route (1): one order k, series in the paper's notation (t_l, partial sum S). */
static qreal series_fk(qreal x, int k) {
    qreal kh = (qreal)k + QL(0.5);
    qreal t = QL(1.0) / kh;                 /* t_0 = x^0 / (k + 1/2) */
    qreal s = t;
    for (int l = 0; l < SERIES_MAX_TERMS; ++l) {
        qreal q = x / (kh + (qreal)(l + 1)); /* t_{l+1} / t_l = x / (k + l + 3/2) */
        if (q < QL(1.0) && t * q / (QL(1.0) - q) <= SERIES_REL_TOL * s) break;
        t *= q;
        s += t;
    }
    return QL(0.5) * QEXP(-x) * s;
}

/* Route (2): all orders 0..kmax from the F_0 closed form + upward identity. */
static void erf_upward(qreal x, int kmax, qreal* f) {
    qreal rx = QSQRT(x);
    qreal emx = QEXP(-x);
    f[0] = QL(0.5) * QSQRT(Q_PI / x) * QERF(rx);
    for (int k = 0; k < kmax; ++k)
        f[k + 1] = ((qreal)(2 * k + 1) * f[k] - emx) / (QL(2.0) * x);
}

/* branch: 0 = automatic, 1 = force series, 2 = force erf + upward (x > 0). */
static int boys_q(double xd, int kmax, int branch, qreal* f) {
    if (kmax < 0 || kmax > ORACLE_KMAX) return -1;
    if (isnan(xd) || xd < 0.0) {
        for (int k = 0; k <= kmax; ++k) f[k] = (qreal)NAN;
        return 0;
    }
    if (isinf(xd)) {
        for (int k = 0; k <= kmax; ++k) f[k] = QL(0.0);
        return 0;
    }
    qreal x = (qreal)xd;
    if (x == QL(0.0)) x = QL(0.0);          /* -0.0 -> +0.0 */
    int use_series = (branch == 1) || (branch == 0 && x < X_SWITCH) || x == QL(0.0);
    if (use_series) {
        for (int k = 0; k <= kmax; ++k) f[k] = series_fk(x, k);
    } else {
        erf_upward(x, kmax, f);
    }
    return 0;
}

/* ---------------------------------------------------------------- exports */

int oracle_kmax_limit(void) { return ORACLE_KMAX; }
int oracle_max_threads(void) { return oracle_threads(0); }
int oracle_mantissa_bits(void) {
#if defined(__x86_64__) || defined(__i386__)
    return FLT128_MANT_DIG;
#else
    return LDBL_MANT_DIG;
#endif
}

/* F_0..F_kmax at one x via the given branch; hi/lo have kmax+1 entries. */
int oracle_boys_branch(double x, int kmax, int branch, double* hi, double* lo) {
    qreal f[ORACLE_KMAX + 1];
    int rc = boys_q(x, kmax, branch, f);
    if (rc) return rc;
    for (int k = 0; k <= kmax; ++k) q_split(f[k], &hi[k], &lo[k]);
    return 0;
}

/*
 * Batch: hi/lo are [kmax+1][ld] (order-major), element (k, i) at k*ld + i.
 * nthreads <= 0 lets OpenMP decide.
 */
int oracle_boys_batch(const double* x, int64_t n, int kmax, double* hi, double* lo,
                      int64_t ld, int nthreads) {
    if (kmax < 0 || kmax > ORACLE_KMAX || n < 0 || ld < n) return -1;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 64) num_threads(oracle_threads(nthreads)) reduction(| : err)
    for (int64_t i = 0; i < n; ++i) {
        qreal f[ORACLE_KMAX + 1];
        if (boys_q(x[i], kmax, 0, f)) { err |= 1; continue; }
        for (int k = 0; k <= kmax; ++k) q_split(f[k], &hi[(int64_t)k * ld + i], &lo[(int64_t)k * ld + i]);
    }
    return err ? -1 : 0;
}

/*
 * Fused consumer: S_i = sum_{k=0}^{kmax} (-2 rho_i)^k F_k(x_i), all in binary128
 * (the McMurchie-Davidson-style scaling named for the fused mode).
 */
int oracle_fused_batch(const double* x, const double* rho, int64_t n, int kmax,
                       double* s_hi, double* s_lo, int nthreads) {
    if (kmax < 0 || kmax > ORACLE_KMAX || n < 0) return -1;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 64) num_threads(oracle_threads(nthreads)) reduction(| : err)
    for (int64_t i = 0; i < n; ++i) {
        qreal f[ORACLE_KMAX + 1];
        if (boys_q(x[i], kmax, 0, f)) { err |= 1; continue; }
        qreal a = QL(-2.0) * (qreal)rho[i], p = QL(1.0), s = QL(0.0);
        for (int k = 0; k <= kmax; ++k) { s += p * f[k]; p *= a; }
        q_split(s, &s_hi[i], &s_lo[i]);
    }
    return err ? -1 : 0;
}

/*
 * Gradient: dL/dx_i = -sum_{k=0}^{kmax} g[k*ldg + i] * F_{k+1}(x_i), using
 * dF_k/dx = -F_{k+1} (differentiate Eq. 3 under the integral sign).
 */
int oracle_grad_batch(const double* x, int64_t n, int kmax, const double* g, int64_t ldg,
                      double* d_hi, double* d_lo, int nthreads) {
    if (kmax < 0 || kmax + 1 > ORACLE_KMAX || n < 0 || ldg < n) return -1;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 64) num_threads(oracle_threads(nthreads)) reduction(| : err)
    for (int64_t i = 0; i < n; ++i) {
        qreal f[ORACLE_KMAX + 1];
        if (boys_q(x[i], kmax + 1, 0, f)) { err |= 1; continue; }
        qreal s = QL(0.0);
        for (int k = 0; k <= kmax; ++k) s += (qreal)g[(int64_t)k * ldg + i] * f[k + 1];
        q_split(-s, &d_hi[i], &d_lo[i]);
    }
    return err ? -1 : 0;
}

/*
 * Pairwise benchmark of the paper (Section III, Algorithm 2, Eq. benchmarkequation):
 *   z_i = sum_{l=0}^{k} c_l sum_{j=0}^{n-1} F_l(x_i + x_j) y_j,
 * every F_l and every sum in binary128.  O(n^2 k): small n only.
 */
int oracle_pairwise(const double* x, const double* y, int64_t n, const double* c, int k,
                    double* z_hi, double* z_lo, int nthreads) {
    if (k < 0 || k > ORACLE_KMAX || n < 0) return -1;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(oracle_threads(nthreads)) reduction(| : err)
    for (int64_t i = 0; i < n; ++i) {
        qreal f[ORACLE_KMAX + 1];
        qreal z = QL(0.0);
        for (int64_t j = 0; j < n; ++j) {
            if (boys_q(x[i] + x[j], k, 0, f)) { err |= 1; break; }
            qreal w = QL(0.0);
            for (int l = 0; l <= k; ++l) w += (qreal)c[l] * f[l];
            z += w * (qreal)y[j];
        }
        q_split(z, &z_hi[i], &z_lo[i]);
    }
    return err ? -1 : 0;
}

/* The same for selected rows only: z[r] = z_{rows[r]}, r < nrows (n may be large). */
int oracle_pairwise_rows(const double* x, const double* y, int64_t n, const double* c, int k,
                         const int64_t* rows, int64_t nrows, double* z_hi, double* z_lo, int nthreads) {
    if (k < 0 || k > ORACLE_KMAX || n < 0 || nrows < 0) return -1;
    int err = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        if (i < 0 || i >= n) return -1;
        qreal z = QL(0.0);
#pragma omp parallel for schedule(dynamic, 256) num_threads(oracle_threads(nthreads)) reduction(+ : z) reduction(| : err)
        for (int64_t j = 0; j < n; ++j) {
            qreal f[ORACLE_KMAX + 1];
            if (boys_q(x[i] + x[j], k, 0, f)) { err |= 1; continue; }
            qreal w = QL(0.0);
            for (int l = 0; l <= k; ++l) w += (qreal)c[l] * f[l];
            z += w * (qreal)y[j];
        }
        q_split(z, &z_hi[r], &z_lo[r]);
    }
    return err ? -1 : 0;
}
