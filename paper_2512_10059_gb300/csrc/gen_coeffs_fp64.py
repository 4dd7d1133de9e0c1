"""Generate ``boys_coeffs_fp64.h`` from the coefficient tables of the paper.

Usage:  python gen_coeffs_fp64.py <the paper's LaTeX source> > boys_coeffs_fp64.h

The paper's Appendix D prints, for eps_tol = 5e-14 and kmax = 32:
  * the region boundaries x_0 and x_1 (Eqs. value_of_x0 / value_of_x1),
  * r_B, the rational minimax approximation of F_0 on [x_0, x_1),
  * r_{A,k}, k = 0..32, the approximations of F_k on [0, x_0),
with numerator and denominator coefficients ordered by increasing degree
downwards and 17 significant digits (enough to round correctly to double).
The denominators are monic (their last coefficient is 1).  Each literal is
converted by the C library's correctly rounded ``strtod`` semantics (Python
``float``), and re-emitted with ``repr`` (shortest round-tripping form), so
the header holds exactly the doubles the paper specifies.
"""
import re
import struct
import sys

CAPTION = re.compile(r"\\caption\{Rational minimax coefficients for \$F_\{?(\d+)\}?\$ on \$\[(.*?)\\rangle\$\}")
NUM = r"[-+]?\d\.\d+E[-+]\d+"


def parse(text):
    lines = text.splitlines()
    x0 = x1 = None
    for ln in lines:
        m = re.match(r"\s*x_0 &= ([0-9.]+)", ln)
        if m:
            x0 = m.group(1)
        m = re.match(r"\s*x_1 &= ([0-9.]+)", ln)
        if m:
            x1 = m.group(1).rstrip(".")
    tables = []
    i = 0
    while i < len(lines):
        m = CAPTION.search(lines[i])
        if not m:
            i += 1
            continue
        k = int(m.group(1))
        region = "B" if m.group(2).startswith("x_0") else "A"
        num, den = [], []
        first = i + 1
        i += 1
        while "\\end{tabular}" not in lines[i]:
            row = lines[i].replace("\\\\", "")
            if "&" in row and re.search(NUM, row):
                left, right = row.split("&", 1)
                if re.search(NUM, left):
                    num.append(re.search(NUM, left).group(0))
                if re.search(NUM, right):
                    den.append(re.search(NUM, right).group(0))
            i += 1
        tables.append({"k": k, "region": region, "num": num, "den": den, "first_line": first})
    return x0, x1, tables


def emit(x0, x1, tables, src_name):
    rb = [t for t in tables if t["region"] == "B"]
    ra = sorted([t for t in tables if t["region"] == "A"], key=lambda t: t["k"])
    assert len(rb) == 1 and [t["k"] for t in ra] == list(range(33)), "unexpected table set"
    rb = rb[0]
    for t in [rb] + ra:
        assert float(t["den"][-1]) == 1.0, f"denominator of table k={t['k']} is not monic"
    pmax = max(len(t["num"]) for t in ra)
    qmax = max(len(t["den"]) for t in ra)
    out = []
    w = out.append
    w("// Rational minimax coefficients for the Boys functions, eps_tol = 5e-14, kmax = 32.")
    w("// Generated by gen_coeffs_fp64.py from the paper's Appendix D tables")
    w("// (\"Coefficients of minimax approximations of Boys functions\"); do not edit.")
    w("// Ordering: index i multiplies x^i.  Denominators are monic (Q[m] == 1).")
    w("#pragma once")
    w("")
    w("#define BOYS_FP64_KMAX 32")
    w(f"#define BOYS_FP64_X0 {float(x0)!r}  /* Appendix D, Eq. value_of_x0 */")
    w(f"#define BOYS_FP64_X1 {float(x1)!r}  /* Appendix D, Eq. value_of_x1 */")
    # IEEE bit patterns (for integer-pipe region tests on non-negative doubles)
    w(f"#define BOYS_FP64_X0_BITS 0x{struct.unpack('<q', struct.pack('<d', float(x0)))[0]:016X}LL")
    w(f"#define BOYS_FP64_X1_BITS 0x{struct.unpack('<q', struct.pack('<d', float(x1)))[0]:016X}LL")
    w("")
    w(f"// r_B: F_0 on [x_0, x_1), (n, m) = ({len(rb['num']) - 1}, {len(rb['den']) - 1})")
    w(f"#define BOYS_RB_N {len(rb['num']) - 1}")
    w(f"#define BOYS_RB_M {len(rb['den']) - 1}")
    w("#define BOYS_RB_P_INIT { " + ", ".join(repr(float(v)) for v in rb["num"]) + " }")
    w("#define BOYS_RB_Q_INIT { " + ", ".join(repr(float(v)) for v in rb["den"]) + " }")
    w("")
    w(f"// r_{{A,k}}: F_k on [0, x_0); rows zero-padded to {pmax} / {qmax} entries")
    w(f"#define BOYS_RA_PLEN {pmax}")
    w(f"#define BOYS_RA_QLEN {qmax}")
    w("#define BOYS_RA_N_INIT { " + ", ".join(str(len(t["num"]) - 1) for t in ra) + " }")
    w("#define BOYS_RA_M_INIT { " + ", ".join(str(len(t["den"]) - 1) for t in ra) + " }")
    w("#define BOYS_RA_P_INIT { \\")
    for t in ra:
        vals = [repr(float(v)) for v in t["num"]] + ["0.0"] * (pmax - len(t["num"]))
        w("  { " + ", ".join(vals) + " }, \\")
    w("}")
    w("#define BOYS_RA_Q_INIT { \\")
    for t in ra:
        vals = [repr(float(v)) for v in t["den"]] + ["0.0"] * (qmax - len(t["den"]))
        w("  { " + ", ".join(vals) + " }, \\")
    w("}")
    w("")
    return "\n".join(out) + "\n"


def main():
    path = sys.argv[1]
    with open(path) as fh:
        text = fh.read()
    x0, x1, tables = parse(text)
    sys.stdout.write(emit(x0, x1, tables, path))


if __name__ == "__main__":
    main()
