"""Generate ``boys_coeffs_fixed.h``: the numerators and denominators of the
Appendix D rationals (the exact doubles of ``boys_coeffs_fp64.h``) as 64-bit
fixed-point polynomials, for Horner evaluation on the integer pipes.

On region A (x < x_0 < 16) the variable is t = x / 16, on region B
(x < x_1 < 32) t = x / 32, so t lies in [0, 1) and the coefficients of a
polynomial sum_i c_i x^i as a polynomial in t are a_i = c_i 16^i (or 32^i),
exactly.  Every Horner intermediate v_i = sum_{j >= i} a_j t^(j-i) is bounded
by M = sum_j |a_j|, so with f = 61 - ceil(log2 M) the integers
A_i = round(a_i 2^f) and every intermediate stay below 2^61 in magnitude; the
polynomial is V 2^-f for the final integer V, with f emitted per polynomial.

A fixed binary point cannot follow the partial sums of the high-degree
denominators (degree 12 and 13 for k = 3, 5, 7) down at small x; the kernels
keep those three in FP64 (their tables are emitted all the same).

Usage:  python gen_coeffs_fixed.py > boys_coeffs_fixed.h
"""
import os
import re
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
SHIFT_A, SHIFT_B = 4, 5  # t = x / 2^SHIFT


def tables():
    s = open(os.path.join(HERE, "boys_coeffs_fp64.h")).read()

    def vec(name):
        return [float(v) for v in re.search(r"#define " + name + r" \{ (.*?) \}\n", s).group(1).split(",")]

    def mat(name, deg):
        rows = re.findall(r"\{ (.*?) \}", re.search(r"#define " + name + r" \{ \\\n(.*?)\n\}", s, re.S).group(1))
        return [[float(v) for v in r.split(",")][:deg[k] + 1] for k, r in enumerate(rows)], len(rows[0].split(","))

    n = [int(v) for v in vec("BOYS_RA_N_INIT")]
    m = [int(v) for v in vec("BOYS_RA_M_INIT")]
    ra_p, plen = mat("BOYS_RA_P_INIT", n)
    ra_q, qlen = mat("BOYS_RA_Q_INIT", m)
    return vec("BOYS_RB_P_INIT"), vec("BOYS_RB_Q_INIT"), ra_p, ra_q, plen, qlen


def fixed(coeffs, shift):
    a = [Fraction(c) * (1 << (shift * i)) for i, c in enumerate(coeffs)]
    M = sum(abs(v) for v in a)
    f = 61 - (int(M) if M.denominator == 1 else int(M) + 1).bit_length()
    while M * (1 << f) > (1 << 61):
        f -= 1
    A = [round(v * (Fraction(2) ** f)) for v in a]
    assert all(abs(v) < (1 << 61) for v in A)
    return A, f


def emit():
    rb_p, rb_q, ra_p, ra_q, plen, qlen = tables()
    out = ["// Numerators and denominators of the Appendix D rationals as 64-bit",
           "// fixed-point polynomials in t = x / 16 (r_{A,k}) or t = x / 32 (r_B):",
           "// value = V * 2^-f for the Horner integer V; generated by gen_coeffs_fixed.py",
           "// from boys_coeffs_fp64.h; do not edit.  Rows are zero-padded to the FP64",
           "// rows' lengths.",
           "#pragma once",
           f"#define BOYS_FX_SHIFT_A {SHIFT_A}",
           f"#define BOYS_FX_SHIFT_B {SHIFT_B}"]

    def row(A, length):
        return "{ " + ", ".join(f"{v}LL" for v in A + [0] * (length - len(A))) + " }"

    for name, rb, ra, length in (("P", rb_p, ra_p, plen), ("Q", rb_q, ra_q, qlen)):
        A, f = fixed(rb, SHIFT_B)
        out.append(f"#define BOYS_RB_{name}_FX_INIT {row(A, length)}")
        out.append(f"#define BOYS_RB_{name}_FXF {f}")
        fs = []
        out.append(f"#define BOYS_RA_{name}_FX_INIT {{ \\")
        for c in ra:
            A, f = fixed(c, SHIFT_A)
            fs.append(f)
            out.append(f"  {row(A, length)}, \\")
        out.append("}")
        out.append(f"#define BOYS_RA_{name}_FXF_INIT {{ " + ", ".join(str(f) for f in fs) + " }")
    return "\n".join(out) + "\n"


if __name__ == "__main__":
    print(emit(), end="")
