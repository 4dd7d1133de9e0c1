"""The integer-pipe inverse square root (xf::rsqrt in csrc/boys_xf.cuh) that
gives the set-up its anchors p/q, F_0 and 1/(2x), modelled operation by
operation with Python integers (the three-partial-product high product,
64-bit wrap-around, arithmetic shifts) and checked against z^{-1/2} to 60
significant digits.

The seed comes from the hardware's rsqrt.approx.f32, whose bits the model
cannot reproduce; the model therefore runs the Newton step from seeds
perturbed across +-2^-21 relative (the approximation's documented error is
near 2^-23, and the truncated 23-bit input adds 2^-24), which covers any seed
the hardware can return, and asserts the design's budget: relative error
below 2^-59.  tests/test_math_fp64.py checks the compiled routine on the GPU.
"""
import math
import struct
from decimal import Decimal, getcontext

import numpy as np

M64 = (1 << 64) - 1


def _s64(v):
    v &= M64
    return v - (1 << 64) if v >> 63 else v


def _mulhi3(a, b):
    a0, a1, b0, b1 = a & 0xFFFFFFFF, a >> 32, b & 0xFFFFFFFF, b >> 32
    return (a1 * b1 + ((a1 * b0) >> 32) + ((a0 * b1) >> 32)) & M64


def _mul(a, b):
    hi = _mulhi3(a[0], b[0])
    top = hi >> 63
    return ((hi << (1 - top)) & M64, a[1] + b[1] + top)


def _f32(v):
    return struct.unpack("<f", struct.pack("<f", v))[0]


def _model(z, perturb, second_order=True):
    """xf::rsqrt on z = (m, e) with the seed rsqrt(s) (1 + perturb), rounded to float."""
    m, e = z
    h = e >> 1
    s_bits = ((127 + (e & 1)) << 23) | ((m >> 40) & 0x7FFFFF)
    s = struct.unpack("<f", struct.pack("<I", s_bits))[0]
    sf = _f32(_f32(1.0 / math.sqrt(s)) * (1.0 + perturb))
    sb = struct.unpack("<I", struct.pack("<f", sf))[0]
    y = (((sb & 0x7FFFFF) | 0x800000) << 40, ((sb >> 23) & 0xFF) - 127 - h)
    w = _mul(_mul(y, y), z)
    W = w[0] >> min(max(1 - w[1], 0), 63)
    D = _s64((1 << 62) - W)
    Ds = D >> 12
    assert abs(Ds) < (1 << 31)
    D2 = Ds * Ds
    C = (D >> 1) + (((3 * D2) >> 41) if second_order else 0)
    Cm = abs(C)
    corr = _mulhi3(y[0], (Cm << 21) & M64) >> 20
    hm = y[0] >> 1
    u = (hm - corr if C < 0 else hm + corr) & M64
    hi = u >> 32
    lz = 32 - hi.bit_length()
    return (u << lz) & M64, y[1] + 1 - lz


def _xf(v):
    """A positive normal double as (m, e): value = m 2^(e-63)."""
    b = struct.unpack("<Q", struct.pack("<d", v))[0]
    return ((b & ((1 << 52) - 1)) | (1 << 52)) << 11, ((b >> 52) & 0x7FF) - 1023


def _worst(zs, perturbs, **kw):
    worst = 0.0
    for z in zs:
        for perturb in perturbs:
            m, e = _model(_xf(float(z)), perturb, **kw)
            assert (1 << 63) <= m <= M64
            got = Decimal(m) * Decimal(2) ** (e - 63)
            worst = max(worst, float(abs(got * Decimal(float(z)).sqrt() - 1)))
    return worst


def test_rsqrt_model_error_budget():
    getcontext().prec = 60
    rng = np.random.default_rng(5)
    zs = np.concatenate([np.exp(rng.uniform(-690, 690, 1500)), rng.uniform(1.0, 4.0, 800),
                         2.0 ** np.arange(-40, 40), 1.0 + 2.0 ** -23 * np.arange(0, 64),
                         np.nextafter(2.0 ** np.arange(-20, 20), 0.0), [1e300, 5e33, 4e14, 28.98933773882074]])
    worst = _worst(zs, (-2.0 ** -21, -2.0 ** -23, 0.0, 2.0 ** -23, 2.0 ** -21))
    assert worst < 2.0 ** -59, math.log2(worst)


def test_rsqrt_model_needs_the_second_order_term():
    """Without the 3 d^2/8 term a seed error of 2^-21 leaves ~2^-41: the
    budget above is not met by a plain (second-order) Newton step."""
    getcontext().prec = 60
    assert _worst([1.7, 3.1, 1e-200, 7e150], (2.0 ** -21,), second_order=False) > 2.0 ** -45
