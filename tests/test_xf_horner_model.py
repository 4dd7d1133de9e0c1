"""The signed integer-significand Horner step (xf::fma_i in csrc/boys_xf.cuh)
that evaluates the anchor's denominator at small kmax, modelled operation by
operation with Python integers and checked against exact rational arithmetic
on every Appendix D denominator and numerator over its region.  Also pins the
integer-format coefficient tables of boys_coeffs_fp64.h as exact copies of the
double tables."""
import math
import random
import re
from fractions import Fraction
from pathlib import Path

HEADER = Path(__file__).resolve().parents[1] / "paper_2512_10059_gb300" / "csrc" / "boys_coeffs_fp64.h"
ZERO_E = -(1 << 28)
X0, X1 = 11.899848152108484, 28.98933773882074


def _arr(h, name):
    m = re.search(r"#define " + name + r"\s+(\{.*?\})\s*\n(?=#|\s*$|//)", h.replace("\\\n", " "), re.S)
    return eval(m.group(1).replace("{", "[").replace("}", "]").replace("LL", ""))


def _from_double(x):                     # xf::from_double for x >= 0
    if x == 0.0:
        return 0, ZERO_E
    fr, ex = math.frexp(x)
    return int(fr * (1 << 64)), ex - 1


def _fma_i(t, u, c):
    (tm, te), (um, ue), (cm, ce) = t, u, c
    p = (tm * (um >> 1)) >> 64          # __mul64hi of the signed product
    ep = te + ue + 2
    e = max(ep, ce)
    s = (p >> min(e - ep, 63)) + (cm >> min(e - ce, 63))
    assert abs(s) < (1 << 63)
    if s == 0:
        return 0, ZERO_E
    lz = 64 - abs(s).bit_length()
    return (s << (lz - 2), e - (lz - 2)) if lz >= 2 else (s >> 1, e + 1)


def _value(t):
    return Fraction(0) if t[0] == 0 else Fraction(t[0]) * Fraction(2) ** (t[1] - 61)


def test_integer_tables_are_exact_copies():
    h = HEADER.read_text()
    for dname, mname, ename in (("BOYS_RA_P_INIT", "BOYS_RA_P_XM_INIT", "BOYS_RA_P_XE_INIT"),
                                ("BOYS_RA_Q_INIT", "BOYS_RA_Q_XM_INIT", "BOYS_RA_Q_XE_INIT")):
        D, M, E = _arr(h, dname), _arr(h, mname), _arr(h, ename)
        for drow, mrow, erow in zip(D, M, E):
            for d, m, e in zip(drow, mrow, erow):
                assert m == 0 and e == ZERO_E if d == 0.0 else (1 << 61) <= abs(m) < (1 << 62)
                assert _value((m, e)) == Fraction(d)
    for dname, mname, ename in (("BOYS_RB_P_INIT", "BOYS_RB_P_XM_INIT", "BOYS_RB_P_XE_INIT"),
                                ("BOYS_RB_Q_INIT", "BOYS_RB_Q_XM_INIT", "BOYS_RB_Q_XE_INIT")):
        D, M, E = _arr(h, dname), _arr(h, mname), _arr(h, ename)
        for d, m, e in zip(D, M, E):
            assert _value((m, e)) == Fraction(d)


def test_signed_horner_model_error():
    h = HEADER.read_text()
    rng = random.Random(5)
    cases = []
    for name in ("BOYS_RA_P", "BOYS_RA_Q"):
        D, M, E = _arr(h, name + "_INIT"), _arr(h, name + "_XM_INIT"), _arr(h, name + "_XE_INIT")
        for k in range(33):
            cases += [(D[k], M[k], E[k], [0.0, X0 * (1 - 1e-16)] + [rng.uniform(0, X0) for _ in range(12)])]
    for name in ("BOYS_RB_P", "BOYS_RB_Q"):
        D, M, E = _arr(h, name + "_INIT"), _arr(h, name + "_XM_INIT"), _arr(h, name + "_XE_INIT")
        cases += [(D, M, E, [X0, X1] + [rng.uniform(X0, X1) for _ in range(100)])]
    worst = 0.0
    for D, M, E, xs in cases:
        n = max(i for i, v in enumerate(D) if v != 0.0)
        for x in xs:
            u = _from_double(x)
            t = (M[n], E[n])
            for i in range(n - 1, -1, -1):
                t = _fma_i(t, u, (M[i], E[i]))
            fx = Fraction(x)
            exact = scale = Fraction(0)
            for i in range(n, -1, -1):
                exact = exact * fx + Fraction(D[i])
                scale = scale * fx + abs(Fraction(D[i]))
            worst = max(worst, float(abs(_value(t) - exact) / scale))
    # FP64 Horner's own bound is about n 2^-53; this format is several bits finer
    assert worst < 2.0 ** -56, math.log2(worst)
