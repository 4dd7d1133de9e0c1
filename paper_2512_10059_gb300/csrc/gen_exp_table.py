"""Generate ``boys_exp_table.h``: T[j] = 2^(-j/64), j = 0..63, correctly rounded
doubles (the table of Tang's table-driven exponential, ACM TOMS 15(2), 1989),
computed with Python's decimal module at 50 significant digits.

Usage:  python gen_exp_table.py > boys_exp_table.h
"""
from decimal import Decimal, getcontext

getcontext().prec = 50
ln2 = Decimal(2).ln()
vals = [float((-(Decimal(j) * ln2) / 64).exp()) for j in range(64)]
print("// T[j] = 2^(-j/64), j = 0..63, correctly rounded to double; generated by gen_exp_table.py")
print("#pragma once")
print("#define BOYS_EXP2_NEG_J64_INIT { \\")
for i in range(0, 64, 4):
    print("  " + ", ".join(v.hex() for v in vals[i:i + 4]) + ", \\")
print("}")
