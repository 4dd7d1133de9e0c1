"""The fixed-point Horner sums of the set-up (csrc/boys_fp64.cuh with
csrc/boys_coeffs_fixed.h), modelled with Python integers exactly as the
device runs them: t = x/16 (region A) or x/32 (region B) in Q64, the
three-partial-product high product of xf::mulhi3, the signed product by the
biased operand (v + 2^63) t / 2^64 - t/2, and the per-polynomial binary point.

Checked against exact rational evaluation of the Appendix D rationals, one
sum fixed and the other exact:
* numerators: p_fixed / q - p / q within 2e-16 for r_{A,0} (whose value is
  near 1), 3e-17 for every other r_{A,k} and 5e-17 for r_B;
* denominators, at every order but the degree-12 and -13 denominators
  (k = 3, 5, 7; the kernels use fixed-point denominators from kmax 6 on,
  except 7): p / q_fixed - p / q within 5e-16 for every r_{A,k} and 5e-17
  for r_B;
at most 1% of the 5e-14 budget, with every Horner intermediate below 2^62.
Planted mistakes (the bias correction dropped, the binary point off by one)
must fail the same bounds.
"""
import importlib.util
import os
import re
from fractions import Fraction

import numpy as np

from tests import boys_header

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2512_10059_gb300", "csrc")
M64 = (1 << 64) - 1


def _gen():
    spec = importlib.util.spec_from_file_location("gen_fixed", os.path.join(CSRC, "gen_coeffs_fixed.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _tables(name="P"):
    s = open(os.path.join(CSRC, "boys_coeffs_fixed.h")).read()
    body = re.search(r"#define BOYS_RA_" + name + r"_FX_INIT \{ \\\n(.*?)\n\}", s, re.S).group(1)
    ra = [[int(v.strip().rstrip("L")) for v in r.split(",")] for r in re.findall(r"\{ (.*?) \}", body)]
    rb = [int(v.strip().rstrip("L")) for v in
          re.search(r"#define BOYS_RB_" + name + r"_FX_INIT \{ (.*?) \}", s).group(1).split(",")]
    fa = [int(v) for v in re.search(r"#define BOYS_RA_" + name + r"_FXF_INIT \{ (.*?) \}", s).group(1).split(",")]
    fb = int(re.search(r"#define BOYS_RB_" + name + r"_FXF (-?\d+)", s).group(1))
    return ra, fa, rb, fb


def _mulhi3(a, b):
    a0, a1, b0, b1 = a & 0xFFFFFFFF, a >> 32, b & 0xFFFFFFFF, b >> 32
    return (a1 * b1 + ((a1 * b0) >> 32) + ((a0 * b1) >> 32)) & M64


def _horner(A, deg, t, bias=True, check_range=True):
    v = A[deg]
    for a in reversed(A[:deg]):
        hi = _mulhi3((v + (1 << 63)) & M64, t)
        v = hi - ((t >> 1) if bias else 0) + a
        assert not check_range or abs(v) < (1 << 62)
    return v


def _worst(A, deg, f, pc, qc, lo, hi, shift, fixed_q=False, **kw):
    xs = list(np.linspace(lo, hi, 240, endpoint=False)) + [hi * (1 - 2.0 ** -50), 1e-300, 1e-9]
    w = 0.0
    for x in xs:
        if not lo <= x < hi:
            continue
        X = Fraction(x)
        t = int(X * 2 ** (64 - shift))      # the device's shifted significand, exact for x < 2^shift
        V = Fraction(_horner(A, deg, t, **kw), 2 ** f)
        Pe = sum(Fraction(c) * X ** i for i, c in enumerate(pc))
        Qe = sum(Fraction(c) * X ** i for i, c in enumerate(qc))
        w = max(w, abs(float(Pe / V - Pe / Qe)) if fixed_q else abs(float((V - Pe) / Qe)))
    return w


def test_generator_reproduces_header():
    assert _gen().emit() == open(os.path.join(CSRC, "boys_coeffs_fixed.h")).read()


def test_fixed_numerators_error_bound():
    T = boys_header.load()
    ra, fa, rb, fb = _tables()
    for k in range(33):
        w = _worst(ra[k], T["ra_n"][k], fa[k], T["ra_p"][k], T["ra_q"][k], 0.0, T["x0"], 4)
        assert w <= (2e-16 if k == 0 else 3e-17), (k, w)
    assert _worst(rb, 5, fb, T["rb_p"], T["rb_q"], T["x0"], T["x1"], 5) <= 5e-17


def test_fixed_denominators_error_bound():
    T = boys_header.load()
    ra, fa, rb, fb = _tables("Q")
    for k in range(33):
        if k in (3, 5, 7):
            continue
        w = _worst(ra[k], T["ra_m"][k], fa[k], T["ra_p"][k], T["ra_q"][k], 0.0, T["x0"], 4, fixed_q=True)
        assert w <= 5e-16, (k, w)
    assert _worst(rb, 6, fb, T["rb_p"], T["rb_q"], T["x0"], T["x1"], 5, fixed_q=True) <= 5e-17


def test_fixed_denominators_excluded_orders_are_the_ones_that_need_it():
    """The three orders kept in FP64 would add more than the bound above."""
    T = boys_header.load()
    ra, fa, _, _ = _tables("Q")
    for k in (3, 5, 7):
        assert _worst(ra[k], T["ra_m"][k], fa[k], T["ra_p"][k], T["ra_q"][k], 0.0, T["x0"], 4, fixed_q=True) > 5e-16


def test_planted_mistakes_fail():
    T = boys_header.load()
    ra, fa, _, _ = _tables()
    k = 12
    args = (T["ra_p"][k], T["ra_q"][k], 0.0, T["x0"], 4)
    assert _worst(ra[k], T["ra_n"][k], fa[k], *args, bias=False, check_range=False) > 1e-12
    assert _worst(ra[k], T["ra_n"][k], fa[k] - 1, *args, check_range=False) > 1e-12
    rq, fq, _, _ = _tables("Q")
    assert _worst(rq[k], T["ra_m"][k], fq[k] + 1, *args, fixed_q=True, check_range=False) > 1e-12
