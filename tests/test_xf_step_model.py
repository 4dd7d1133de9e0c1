"""The integer-format recurrence step of csrc/boys_fp64.cuh (step:
mul_norm(add_raw(mul_raw(a, y), s), c) on the operands of region A, B or C),
modelled operation by operation with Python integers (the three-partial-product
high product, 64-bit wrap-around, PTX's saturating shifts, the 32-bit
leading-zero count) and run through all 32 steps of kmax = 32 on every region
(Eq. downwardsrecursion in A, Eq. upwardsrecursion in B, the asymptotic
recurrence in C), from anchors (the exact F_kmax or F_0 of the binary128
oracle), e^{-x} and 1/(2x) rounded to the format.  The values are checked
against the same recurrence in exact rational arithmetic on the same rounded
operands, so only the format's own rounding is measured, and the format's
structural claims are checked on every step: the unnormalised sum keeps its
leading bit in bits 59..63 (at most four leading zeros, so a 32-bit
leading-zero count of the high word normalises the product that follows),
and that product's leading bit lies in bits 57..63.  Planted mistakes in the
exponent bookkeeping and the alignment fail it.
"""
import re
from decimal import Decimal, getcontext
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

import oracle

M64 = (1 << 64) - 1
ZERO_EXP = -(1 << 28)
KMAX = 32
X0 = 11.899848152108484
X1 = 28.989337738820740
CONSTS = Path(__file__).resolve().parents[1] / "paper_2512_10059_gb300" / "csrc" / "boys_xf_consts.h"


def _xf(v: Fraction):
    """Positive rational -> (m, e), value m 2^(e-63), m rounded to nearest."""
    e = v.numerator.bit_length() - v.denominator.bit_length()
    if Fraction(2) ** e > v:
        e -= 1
    m = round(v * Fraction(2) ** (63 - e))
    if m >> 64:
        m >>= 1
        e += 1
    return m, e


def _val(x):
    m, e = x
    return Fraction(m) * Fraction(2) ** (e - 63)


def _mulhi3(a, b):
    a0, a1, b0, b1 = a & 0xFFFFFFFF, a >> 32, b & 0xFFFFFFFF, b >> 32
    return (a1 * b1 + ((a1 * b0) >> 32) + ((a0 * b1) >> 32)) & M64


def _clz32(v):
    return 32 - v.bit_length()


class Model:
    def __init__(self, mistake=None):
        self.mistake = mistake
        self.max_sum_lz = 0
        self.min_prod_bit = 63

    def mul_raw(self, a, b):
        return _mulhi3(a[0], b[0]), a[1] + b[1] + 1

    def add_raw(self, t, s):
        E = max(t[1], s[1])
        sh_t = E - t[1] + (0 if self.mistake == "no_headroom" else 1)
        ta = t[0] >> sh_t if sh_t < 64 else 0
        sh_s = E - s[1]
        sa = s[0] >> sh_s if sh_s < 64 else (-1 if s[0] < 0 else 0)  # arithmetic shift
        u = (ta + sa) & M64
        if u:
            self.max_sum_lz = max(self.max_sum_lz, 63 - (u.bit_length() - 1))
        return u, E + (0 if self.mistake == "sum_exponent" else 1)

    def mul_norm(self, a, b):
        hi = _mulhi3(a[0], b[0])
        if hi:
            self.min_prod_bit = min(self.min_prod_bit, hi.bit_length() - 1)
        lz = _clz32(hi >> 32)
        return (hi << lz) & M64, a[1] + b[1] + (0 if self.mistake == "product_exponent" else 1) - lz


def _consts(name):
    s = CONSTS.read_text()
    body = re.search(r"#define " + name + r" \{(.*?)\}", s, re.S).group(1)
    return [int(v.strip().rstrip("ULL").rstrip("LL"), 0) for v in body.replace("\\", " ").split(",") if v.strip()]


def test_odd_and_reciprocal_tables_are_their_definitions():
    """boys_xf_consts.h holds 2j+1 exactly and 1/(2l+1) rounded to nearest."""
    om, oe = _consts("BOYS_XF_ODD_M_INIT"), _consts("BOYS_XF_ODD_E_INIT")
    rm, re_ = _consts("BOYS_XF_RECIP_ODD_M_INIT"), _consts("BOYS_XF_RECIP_ODD_E_INIT")
    for j in range(len(om)):
        assert (om[j], oe[j]) == _xf(Fraction(2 * j + 1))
        assert (rm[j], re_[j]) == _xf(Fraction(1, 2 * j + 1))


def _run(x: float, model: Model):
    """All kmax+1 values of one argument through the modelled step, and the
    same recurrence in exact rational arithmetic on the same rounded operands
    (anchor, e^{-x}, 1/(2x), 2x, 2j+1, 1/(2l+1)).  Returns both in order
    k = 0..kmax, and F_0 (the largest value) for scale."""
    getcontext().prec = 60
    hi, lo = oracle.boys(np.array([x]), KMAX)
    exact = [Fraction(float(hi[k, 0])) + Fraction(float(lo[k, 0])) for k in range(KMAX + 1)]
    xf = Fraction(x)
    inA, inC = x < X0, x >= X1
    X2 = _xf(2 * xf)
    R = _xf(1 / (2 * xf))
    E = _xf(Fraction((-Decimal(x)).exp()))
    if inC:
        Es, s_exact = (0, ZERO_EXP), Fraction(0)
    else:
        v = E[0] >> 1
        Es, s_exact = (v if inA else -v, E[1]), (_val(E) if inA else -_val(E))
    y = _xf(exact[KMAX] if inA else exact[0])
    yr = _val(y)
    vals, ref = [y], [yr]
    for j in range(KMAX):
        l = KMAX - 1 - j
        a = X2 if inA else _xf(Fraction(2 * j + 1))
        c = _xf(Fraction(1, 2 * l + 1)) if inA else R
        y = model.mul_norm(model.add_raw(model.mul_raw(a, y), Es), c)
        yr = (_val(a) * yr + s_exact) * _val(c)
        vals.append(y)
        ref.append(yr)
    order = (lambda z: list(reversed(z))) if inA else (lambda z: z)
    return [_val(v) for v in order(vals)], order(ref), exact[0]


XS = [1e-9, 0.3, 2.5, 7.0, 11.8, X0, 14.0, 20.0, 28.9, X1, 40.0, 300.0, 1e5]


def _worst(model):
    worst = 0.0
    for x in XS:
        F, ref, f0 = _run(x, model)
        worst = max(worst, max(abs(float((F[k] - ref[k]) / f0)) for k in range(KMAX + 1)))
    return worst


def test_step_model_rounding_and_structure():
    """Against the same recurrence in exact arithmetic: the format's rounding
    over 32 steps stays below 2^-55 of F_0 (FP64 rounds each operation at
    2^-53), every sum keeps its leading bit in bits 59..63 and every product
    in bits 57..63."""
    model = Model()
    worst = _worst(model)
    assert model.max_sum_lz <= 4, model.max_sum_lz
    assert model.min_prod_bit >= 57, model.min_prod_bit
    assert worst < 2.0 ** -55, worst


@pytest.mark.parametrize("mistake", ["sum_exponent", "product_exponent", "no_headroom"])
def test_planted_mistakes_fail(mistake):
    model = Model(mistake)
    worst = _worst(model)
    assert worst > 2.0 ** -55 or model.max_sum_lz > 4 or model.min_prod_bit < 57, \
        f"planted mistake {mistake} went unnoticed"
