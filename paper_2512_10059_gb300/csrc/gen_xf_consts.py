"""Generate ``boys_xf_consts.h``: the odd integers 2j+1 and their reciprocals
1/(2l+1), j, l = 0..63, in the library's 64-bit-mantissa format
(value = m * 2^(e - 63), 2^63 <= m < 2^64), with exact integer arithmetic
(reciprocals rounded to nearest).

Usage:  python gen_xf_consts.py > boys_xf_consts.h
"""


def odd(v):
    e = v.bit_length() - 1
    return v << (63 - e), e


def recip(v):
    # 1/v = m * 2^(e-63) with e = -ceil(log2 v) for v > 1 (e = 0 for v = 1)
    e = 0 if v == 1 else -(v - 1).bit_length()
    num = 1 << (63 - e)
    m = (2 * num + v) // (2 * v)
    assert (1 << 63) <= m < (1 << 64), v
    return m, e


print("// Odd integers 2j+1 and reciprocals 1/(2l+1) as (m, e), value = m * 2^(e-63);")
print("// generated by gen_xf_consts.py; do not edit.")
print("#pragma once")
for name, fn in (("ODD", odd), ("RECIP_ODD", recip)):
    ms, es = zip(*(fn(2 * j + 1) for j in range(64)))
    print(f"#define BOYS_XF_{name}_M_INIT {{ " + ", ".join(f"0x{m:016X}ULL" for m in ms) + " }")
    print(f"#define BOYS_XF_{name}_E_INIT {{ " + ", ".join(str(e) for e in es) + " }")

# e^{-x} on the integer pipes (Tang's method in fixed point, 256 subintervals):
# T_j = 2^(-j/256) as (m, e); 256/ln2 in Q54; ln2/256 in Q89 split into the
# high bits (>> 32) and the low 32 bits; 1/2, 1/6, 1/24 in Q62 and 1/120 in Q32;
# and sqrt(pi)/2 (pi to 63 digits) in Q64.
from decimal import Decimal, getcontext, ROUND_HALF_EVEN

getcontext().prec = 60
LN2 = Decimal(2).ln()


def q(v, bits):
    return int((v * (Decimal(2) ** bits)).to_integral_value(rounding=ROUND_HALF_EVEN))


tm, te = [], []
for j in range(256):
    v = (-(Decimal(j) * LN2) / 256).exp()
    if j == 0:
        tm.append(1 << 63)
        te.append(0)
    else:
        m = q(v, 64)
        assert (1 << 63) <= m < (1 << 64), j
        tm.append(m)
        te.append(-1)
l89 = q(LN2 / 256, 89)
consts = {
    "BOYS_XF_EXP_INVLN2_Q54": q(256 / LN2, 54),
    "BOYS_XF_EXP_LN2_HI": l89 >> 32,
    "BOYS_XF_EXP_LN2_LO": l89 & 0xFFFFFFFF,
    "BOYS_XF_EXP_HALF_Q62": q(Decimal(1) / 2, 62),
    "BOYS_XF_EXP_SIXTH_Q62": q(Decimal(1) / 6, 62),
    "BOYS_XF_EXP_24TH_Q62": q(Decimal(1) / 24, 62),
    "BOYS_XF_EXP_120TH_Q32": q(Decimal(1) / 120, 32),
}
# sqrt(pi)/2 = m * 2^(-1-63), the asymptotic F_0 factor of region C
PI = Decimal("3.14159265358979323846264338327950288419716939937510582097494459")
consts["BOYS_XF_SQRTPI_2_M"] = q(PI.sqrt() / 2, 64)
assert (1 << 63) <= consts["BOYS_XF_SQRTPI_2_M"] < (1 << 64)
assert consts["BOYS_XF_EXP_INVLN2_Q54"] < (1 << 63)
print("// Tang's e^{-x} in fixed point: T_j = 2^(-j/256) = m * 2^(e-63), and the")
print("// reduction and polynomial constants (see xf::exp_neg).")
print("#define BOYS_XF_EXP2_NEG_J256_M_INIT { " + ", ".join(f"0x{m:016X}ULL" for m in tm) + " }")
for k, v in consts.items():
    print(f"#define {k} 0x{v:016X}ULL")
