"""Pins for the binary128 oracle: facts fixed by the paper and by mathematics,
not by the oracle's own formulas.

Each ``pin_*`` takes an ``oracle.OracleLib`` and raises ``AssertionError``
when the oracle disagrees with the fact it is pinned to.  ``test_oracle_pins``
runs them on the real oracle; ``test_oracle_mutants`` compiles copies of the
oracle with one planted mistake each and checks that some pin fails.

Independent routes used here:
  * F_k(0) = 1/(2k+1)                    (Eq. 3 at x = 0)
  * F_0(x) = 1/2 sqrt(pi/x) erf(sqrt x)  (Eq. 3, k = 0, via scipy / mpmath)
  * F_k(x) = gamma(k+1/2, x) / (2 x^{k+1/2})  (mpmath lower incomplete gamma)
  * (2k+1) F_k - 2x F_{k+1} = e^{-x}     (Eqs. upwardsrecursion / downwardsrecursion)
  * dF_k/dx = -F_{k+1}                    (Eq. 3 differentiated)
  * bounds e^{-x}/(2k+1) <= F_k <= min(1/(2k+1), Gamma(k+1/2)/(2 x^{k+1/2}))
  * composite Gauss-Legendre quadrature of Eq. 3 and of the fused / gradient
    integrands (numpy Legendre nodes)
  * the paper's printed x_1 solving Eq. x1 (golden fixture)
"""
import json
import math
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _exact(hi, lo):
    return Fraction(float(hi)) + Fraction(float(lo))


def _gl_panels(f, a=0.0, b=1.0, panels=128, order=40):
    """Composite Gauss-Legendre quadrature of a vectorised f on [a, b]."""
    t, w = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(a, b, panels + 1)
    total = 0.0
    for lo_e, hi_e in zip(edges[:-1], edges[1:]):
        half = 0.5 * (hi_e - lo_e)
        mid = 0.5 * (hi_e + lo_e)
        total += half * np.dot(w, f(mid + half * t))
    return total


def pin_at_zero(o):
    hi, lo = o.boys([0.0, -0.0], 40)
    for k in range(41):
        for j in range(2):
            v = _exact(hi[k, j], lo[k, j])
            assert abs(v - Fraction(1, 2 * k + 1)) <= Fraction(1, 10**32), (k, j, float(v))


def pin_f0_closed_form(o):
    from scipy.special import erf
    xs = np.concatenate([np.logspace(-8, math.log10(2e3), 60), [11.9, 28.99, 30.0, 30.5]])
    hi, lo = o.boys(xs, 0)
    ref = 0.5 * np.sqrt(np.pi / xs) * erf(np.sqrt(xs))
    rel = np.abs((hi[0] - ref) + lo[0]) / ref
    assert rel.max() < 4e-16, (xs[rel.argmax()], rel.max())


def pin_f0_closed_form_mp(o, mpmath):
    mpmath.mp.dps = 45
    xs = [1e-8, 1e-3, 0.37, 1.0, 5.5, 11.9, 20.0, 29.9, 30.0, 41.0, 200.0]
    hi, lo = o.boys(xs, 0)
    for j, x in enumerate(xs):
        X = mpmath.mpf(x)
        ref = mpmath.sqrt(mpmath.pi / X) * mpmath.erf(mpmath.sqrt(X)) / 2
        got = mpmath.mpf(hi[0, j]) + mpmath.mpf(lo[0, j])
        assert abs(got - ref) <= mpmath.mpf("1e-30") * ref, (x, float(got - ref))


def pin_gammainc_mp(o, mpmath):
    mpmath.mp.dps = 45
    xs = [1e-6, 0.5, 3.0, 11.899848152108484, 17.0, 28.98933773882074, 30.0, 33.0, 60.0, 500.0]
    ks = [0, 1, 2, 7, 16, 31, 32, 33, 40]
    hi, lo = o.boys(xs, 40)
    for j, x in enumerate(xs):
        X = mpmath.mpf(x)
        for k in ks:
            s = mpmath.mpf(k) + mpmath.mpf(1) / 2
            ref = mpmath.gammainc(s, 0, X) / (2 * X**s)
            got = mpmath.mpf(hi[k, j]) + mpmath.mpf(lo[k, j])
            assert abs(got - ref) <= mpmath.mpf("1e-29") * ref + mpmath.mpf("1e-300"), \
                (x, k, float((got - ref) / ref))


def pin_recurrence_identity(o, mpmath=None):
    xs = [1e-7, 0.01, 0.9, 4.0, 11.9, 12.5, 25.0, 29.99]
    hi, lo = o.boys(xs, 33)
    for j, x in enumerate(xs):
        X = Fraction(x)
        if mpmath is not None:
            mpmath.mp.dps = 45
            e = Fraction(str(mpmath.exp(-mpmath.mpf(x))))
            tol = Fraction(1, 10**30)
        else:
            e = Fraction(math.exp(-x))
            tol = Fraction(1, 10**15)
        for k in range(33):
            fk, fk1 = _exact(hi[k, j], lo[k, j]), _exact(hi[k + 1, j], lo[k + 1, j])
            res = (2 * k + 1) * fk - 2 * X * fk1 - e
            # the two products cancel down to e^{-x}: scale by the larger term
            assert abs(res) <= tol * ((2 * k + 1) * fk + e), (x, k, float(res))


def pin_branch_overlap(o):
    for x in np.linspace(12.3, 60.0, 24):
        a = o.boys_branch(x, 34, 1)
        b = o.boys_branch(x, 34, 2)
        for k in range(35):
            va, vb = _exact(a[0][k], a[1][k]), _exact(b[0][k], b[1][k])
            assert abs(va - vb) <= Fraction(1, 10**27) * va, (x, k, float((va - vb) / va))


def pin_derivative(o):
    """4th-order central difference of F_k (exact rational arithmetic on the
    oracle's double-double values) against -F_{k+1}.  x and h = 2^-10 are
    dyadic, so every abscissa x +- h, x +- 2h is an exact double."""
    h = 2.0 ** -10
    for x in [0.0625, 0.75, 6.0, 11.875, 19.0, 29.0, 30.5, 45.0]:
        pts = [x - 2 * h, x - h, x + h, x + 2 * h, x]
        hi, lo = o.boys(pts, 34)
        for k in range(34):
            f = [_exact(hi[k, j], lo[k, j]) for j in range(4)]
            d = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * Fraction(h))
            ref = -_exact(hi[k + 1, 4], lo[k + 1, 4])
            # truncation h^4/30 |F_k^(5)| = h^4/30 F_{k+5} <= 3e-14
            assert abs(d - ref) <= Fraction(1, 10**13), (x, k, float(d), float(ref))


def pin_bounds_monotone(o):
    xs = np.concatenate([[0.0], np.logspace(-10, 4, 300)])
    hi, lo = o.boys(xs, 40)
    assert np.all(np.diff(hi, axis=1) <= 0), "F_k must be non-increasing in x"
    assert np.all(hi[1:, 1:] < hi[:-1, 1:]), "F_{k+1} < F_k for x > 0"
    k = np.arange(41)[:, None]
    lower = np.exp(-xs)[None, :] / (2 * k + 1)
    upper = 1.0 / (2 * k + 1) * np.ones_like(xs)[None, :]
    with np.errstate(divide="ignore", over="ignore"):
        lg = np.array([math.lgamma(kk + 0.5) for kk in range(41)])[:, None]
        asym = np.exp(lg - (k + 0.5) * np.log(np.where(xs > 0, xs, 1.0))[None, :]) / 2
    upper = np.where(xs[None, :] > 0, np.minimum(upper, asym), upper)
    # the bounds are formed in double (exp / lgamma of arguments up to ~1e4):
    # a few 1e-14 relative slack; a real violation (a dropped factor) is O(1)
    slack = 1e-13
    assert np.all(hi >= lower * (1 - slack)), "F_k >= e^{-x}/(2k+1)"
    assert np.all(hi <= upper * (1 + slack)), "F_k <= min(1/(2k+1), Gamma(k+1/2)/(2x^{k+1/2}))"


def pin_quadrature(o):
    for x in [0.1, 1.0, 5.0, 11.9, 25.0, 40.0, 100.0, 1000.0]:
        hi, lo = o.boys([x], 33)
        for k in [0, 1, 3, 12, 20, 32, 33]:
            q = _gl_panels(lambda t: t ** (2 * k) * np.exp(-x * t * t))
            v = hi[k, 0] + lo[k, 0]
            assert abs(q - v) <= 1e-13 * v, (x, k, q, v)


def pin_fused_quadrature(o):
    """sum_{k<=K} a^k F_k(x) = int_0^1 (1 - (a t^2)^{K+1}) / (1 - a t^2) e^{-x t^2} dt
    for a = -2 rho < 0 (geometric series under the integral of Eq. 3)."""
    xs = np.array([0.3, 4.0, 12.0, 29.0, 35.0])
    for K in [0, 3, 8, 16]:
        for rho in [0.1, 0.35, 0.7]:
            hi, lo = o.fused(xs, np.full(xs.size, rho), K)
            a = -2.0 * rho
            for j, x in enumerate(xs):
                q = _gl_panels(lambda t: (1 - (a * t * t) ** (K + 1)) / (1 - a * t * t)
                               * np.exp(-x * t * t))
                v = hi[j] + lo[j]
                assert abs(q - v) <= 1e-13 * max(abs(v), 1e-3), (x, K, rho, q, v)


def pin_grad_quadrature(o):
    """-sum_k g_k F_{k+1}(x) = int_0^1 -sum_k g_k t^{2k+2} e^{-x t^2} dt."""
    rng = np.random.default_rng(7)
    xs = np.array([0.2, 3.0, 12.5, 31.0])
    for K in [0, 5, 16]:
        g = rng.standard_normal((K + 1, xs.size))
        hi, lo = o.grad(xs, g, K)
        for j, x in enumerate(xs):
            gj = g[:, j]
            q = _gl_panels(lambda t: -sum(gj[k] * t ** (2 * k + 2) for k in range(K + 1))
                           * np.exp(-x * t * t))
            v = hi[j] + lo[j]
            assert abs(q - v) <= 1e-13 * np.abs(gj).sum(), (x, K, q, v)


def pin_pairwise_reduces_to_boys(o):
    """Algorithm 2 with one-hot c and y is a single Boys value:
    c = e_l, y = e_m  =>  z_i = F_l(x_i + x_m); and z is linear in c and y."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 30, 9)
    k = 5
    for l, m in [(0, 0), (3, 4), (5, 8)]:
        c = np.zeros(k + 1)
        c[l] = 1.0
        y = np.zeros(9)
        y[m] = 1.0
        zh, zl = o.pairwise(x, y, c)
        fh, fl = o.boys(x + x[m], k)
        assert np.all(np.abs((zh - fh[l]) + (zl - fl[l])) <= 1e-30 * np.abs(fh[l]) + 1e-300), (l, m)
    yy = rng.standard_normal(9)
    cc = rng.standard_normal(k + 1)
    full = o.pairwise(x, yy, cc)
    part = o.pairwise_rows(x, yy, cc, [2, 7])
    assert np.array_equal(full[0][[2, 7]], part[0])
    c1, c2 = rng.standard_normal(k + 1), rng.standard_normal(k + 1)
    y = rng.standard_normal(9)
    a = o.pairwise(x, y, c1)[0] + o.pairwise(x, y, c2)[0]
    b = o.pairwise(x, y, c1 + c2)[0]
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(b))


def pin_x1_golden(o):
    """Appendix D prints x_1 = 28.989337738820740 as the root of Eq. x1 for
    k_max = 32, eps_tol = 5e-14: Gamma(32.5, x1) / (2 x1^32.5) = eps_tol, i.e.
    Gamma(32.5)/(2 x1^32.5) - F_32(x1) = 5e-14 (Section II.C)."""
    with open(os.path.join(GOLDEN, "x1_root_kmax32.json")) as fh:
        gold = json.load(fh)
    x1 = float(gold["x1"])
    k = int(gold["kmax"])
    eps = float(gold["eps_tol"])
    hi, lo = o.boys([x1], k)
    fk = hi[k, 0] + lo[k, 0]
    asym = math.exp(math.lgamma(k + 0.5) - (k + 0.5) * math.log(x1)) / 2
    err = asym - fk
    assert abs(err - eps) <= float(gold["rel_tol"]) * eps, (err, eps)


CPU_PINS = [pin_at_zero, pin_f0_closed_form, pin_recurrence_identity, pin_branch_overlap,
            pin_derivative, pin_bounds_monotone, pin_quadrature, pin_fused_quadrature,
            pin_grad_quadrature, pin_x1_golden, pin_pairwise_reduces_to_boys]
MP_PINS = [pin_f0_closed_form_mp, pin_gammainc_mp]
