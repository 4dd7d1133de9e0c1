"""The fixed-point e^{-x} of the integer-pipe recurrence (xf::exp_neg in
csrc/boys_xf.cuh), modelled operation by operation with Python integers
(64-bit wrap-around, arithmetic shifts, high halves of products) and checked
against e^{-x} to 60 significant digits.  This pins the generated table and
constants of csrc/boys_xf_consts.h and the error budget of the design
(relative error below 2^-59.5); tests/test_math_fp64.py checks the compiled
function on the GPU against a binary128 reference."""
import math
import re
import struct
from decimal import Decimal, getcontext
from pathlib import Path

import numpy as np

CONSTS = Path(__file__).resolve().parents[1] / "paper_2512_10059_gb300" / "csrc" / "boys_xf_consts.h"
M64 = (1 << 64) - 1


def _load():
    h = CONSTS.read_text()
    table = [int(v, 16) for v in
             re.search(r"BOYS_XF_EXP2_NEG_J256_M_INIT \{ (.*?) \}", h).group(1).replace("ULL", "").split(", ")]
    consts = {k: int(v, 16) for k, v in re.findall(r"#define (BOYS_XF_EXP_\w+) 0x([0-9A-F]+)ULL", h)}
    return table, consts


def _s64(v):
    v &= M64
    return v - (1 << 64) if v >> 63 else v


def _mul_q62(a, b):
    p = a * b                              # exact; the device takes the high word and two low bits
    hi = p >> 64
    lo = p & M64
    return _s64(((hi & M64) << 2) | (lo >> 62))


def _model(x, table, c):
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    be = (b >> 52) & 0x7FF
    mant = (b & ((1 << 52) - 1)) | (1 << 52)
    sh = be - 1018
    X = (mant << min(sh, 9)) if sh >= 0 else (mant >> min(-sh, 63))
    if be == 0:
        X = 0
    t = (X * c["BOYS_XF_EXP_INVLN2_Q54"]) >> 64
    n = (t + (1 << 46)) >> 47
    s62 = be - 1013
    xq = ((mant << min(s62, 14)) if s62 >= 0 else (mant >> min(-s62, 63))) & M64
    if be == 0:
        xq = 0
    r = _s64(xq - n * (c["BOYS_XF_EXP_LN2_HI"] << 5) - ((n * c["BOYS_XF_EXP_LN2_LO"] + (1 << 26)) >> 27))
    rh = r >> 32
    p0 = _s64(c["BOYS_XF_EXP_24TH_Q62"] - rh * c["BOYS_XF_EXP_120TH_Q32"])
    p1 = _s64(rh * (p0 >> 32) * 4 - c["BOYS_XF_EXP_SIXTH_Q62"])
    prod = (r >> 21) * (p1 >> 29)
    assert abs(prod) < (1 << 62)
    p2 = _s64(c["BOYS_XF_EXP_HALF_Q62"] + (prod >> 12))
    q = _s64(_mul_q62(_mul_q62(r, r), p2) - r)
    j = n & 255
    P = (table[j] * ((1 << 62) + q)) >> 64
    lz = 64 - P.bit_length()
    assert 1 <= lz <= 3
    return (P << lz) & M64, (-1 if j else 0) + 2 - lz - (n >> 8)


def test_fixed_point_exp_model_error_budget():
    getcontext().prec = 60
    table, c = _load()
    assert table[0] == 1 << 63 and all((1 << 63) <= t < (1 << 64) for t in table)
    rng = np.random.default_rng(3)
    ln2_256 = math.log(2.0) / 256
    xs = np.concatenate([rng.uniform(0, 32, 6000), np.exp(rng.uniform(-700, 0.5, 1500)),
                         np.arange(0, 11090, 7) * ln2_256, np.arange(3, 11090, 7) * ln2_256 + 1e-15,
                         [0.0, 5e-324, 2.0 ** -5, 2.0 ** -10, 11.899848152108484, 28.98933773882074,
                          np.nextafter(32.0, 0.0)]])
    worst = 0.0
    for x in xs[(xs >= 0) & (xs < 32)]:
        m, e = _model(float(x), table, c)
        got = Decimal(m) * Decimal(2) ** (e - 63)
        rel = abs(got / (-Decimal(float(x))).exp() - 1)
        worst = max(worst, float(rel))
    assert worst < 2.0 ** -59.5, math.log2(worst)
    m, e = _model(0.0, table, c)
    assert (m, e) == (1 << 63, 0)
