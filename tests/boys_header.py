"""Reads the product's generated FP64 coefficient header as plain data (tests only)."""
import os
import re

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2512_10059_gb300", "csrc", "boys_coeffs_fp64.h")


def load():
    s = open(HEADER).read()

    def vec(name):
        body = re.search(name + r" \{ (.*?) \}\n", s).group(1)
        return [float(v) for v in body.split(",")]

    def mat(name):
        body = re.search(name + r" \{ \\\n(.*?)\n\}", s, re.S).group(1)
        rows = re.findall(r"\{ (.*?) \}", body)
        return [[float(v) for v in r.split(",")] for r in rows]

    def num(name):
        return float(re.search(r"#define " + name + r" ([0-9.eE+-]+)", s).group(1))

    ra_n = [int(v) for v in vec("BOYS_RA_N_INIT")]
    ra_m = [int(v) for v in vec("BOYS_RA_M_INIT")]
    ra_p = mat("BOYS_RA_P_INIT")
    ra_q = mat("BOYS_RA_Q_INIT")
    return {
        "x0": num("BOYS_FP64_X0"), "x1": num("BOYS_FP64_X1"),
        "rb_p": vec("BOYS_RB_P_INIT"), "rb_q": vec("BOYS_RB_Q_INIT"),
        "ra_p": [ra_p[k][:ra_n[k] + 1] for k in range(33)],
        "ra_q": [ra_q[k][:ra_m[k] + 1] for k in range(33)],
        "ra_n": ra_n, "ra_m": ra_m,
    }
