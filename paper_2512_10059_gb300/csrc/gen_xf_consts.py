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
