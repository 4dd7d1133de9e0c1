"""The FP64 coefficient header against what the paper fixes (CPU only).

* degrees (n, m) of every printed table (Appendix D, Tables r_B, r_{A,0..32})
* monic denominators (Appendix D: "degree increasing downwards", last = 1)
* r_{A,k}(0) = P_0/Q_0 within eps_tol of F_k(0) = 1/(2k+1) (Eq. 3 at x = 0)
* x_0 equals Eq. x0, the kmax = 32 case of max{1, (prod_{k<kmax}(k+1/2))^(1/kmax)}
* x_1 is the printed root of Eq. x1 (same golden fixture that pins the oracle)
* a plain-double host port of Algorithm 1 using these coefficients stays within
  eps_tol of the oracle: this validates the transcription of every table.
"""
import json
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2512_10059_gb300 import workloads
from tests import boys_header

EPS = 5e-14
SLACK = 1e-27  # round-off slack at x = x_1 exactly, where Eq. x1 is tight

# (n, m) as printed: Appendix D, one table per approximant
PRINTED_DEGREES = {
    "B": (5, 6),
    0: (6, 9), 1: (6, 10), 2: (6, 10), 3: (4, 12), 4: (8, 9), 5: (4, 13), 6: (8, 9), 7: (4, 13),
    8: (8, 9), 9: (8, 9), 10: (8, 9), 11: (8, 9), 12: (8, 9), 13: (8, 9), 14: (8, 9), 15: (8, 9),
    16: (8, 9), 17: (8, 9), 18: (8, 8), 19: (8, 8), 20: (7, 9), 21: (8, 8), 22: (8, 8), 23: (8, 8),
    24: (8, 8), 25: (8, 8), 26: (7, 8), 27: (7, 8), 28: (7, 8), 29: (7, 8), 30: (7, 8), 31: (7, 8),
    32: (7, 8),
}


@pytest.fixture(scope="module")
def H():
    return boys_header.load()


def test_degrees(H):
    assert (len(H["rb_p"]) - 1, len(H["rb_q"]) - 1) == PRINTED_DEGREES["B"]
    for k in range(33):
        assert (H["ra_n"][k], H["ra_m"][k]) == PRINTED_DEGREES[k], k


def test_monic(H):
    assert H["rb_q"][-1] == 1.0
    for k in range(33):
        assert H["ra_q"][k][-1] == 1.0


def test_value_at_zero(H):
    for k in range(33):
        r0 = H["ra_p"][k][0] / H["ra_q"][k][0]
        assert abs(r0 - 1.0 / (2 * k + 1)) <= EPS, (k, r0)


def test_x0_equation(H):
    kmax = 32
    logprod = sum(math.log(k + 0.5) for k in range(kmax))
    x0 = max(1.0, math.exp(logprod / kmax))
    assert abs(x0 - H["x0"]) <= 4e-15 * x0, (x0, H["x0"])


def test_x1_golden(H):
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "x1_root_kmax32.json")))
    assert H["x1"] == float(gold["x1"])


def _horner(c, x):
    v = np.zeros_like(x) + c[-1]
    for a in reversed(c[:-1]):
        v = v * x + a
    return v


def algorithm1_host(H, x, kmax):
    """Test-only plain-double restatement of Algorithm 1 with the header's
    tables (numpy, no fused multiply-add): used to check the transcription."""
    x = np.asarray(x, dtype=np.float64)
    F = np.empty((kmax + 1, x.size))
    A = x < H["x0"]
    B = (x >= H["x0"]) & (x < H["x1"])
    C = x >= H["x1"]
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        e = np.exp(-x)
        # A: anchor r_{A,kmax}, downward
        Fa = np.empty((kmax + 1, x.size))
        Fa[kmax] = _horner(H["ra_p"][kmax], x) / _horner(H["ra_q"][kmax], x)
        for l in range(kmax - 1, -1, -1):
            Fa[l] = (2 * x * Fa[l + 1] + e) / (2 * l + 1)
        # B: anchor r_B, upward
        Fb = np.empty((kmax + 1, x.size))
        Fb[0] = _horner(H["rb_p"], x) / _horner(H["rb_q"], x)
        for l in range(kmax):
            Fb[l + 1] = ((2 * l + 1) * Fb[l] - e) / (2 * x)
        # C: asymptotic, upward
        Fc = np.empty((kmax + 1, x.size))
        Fc[0] = math.sqrt(math.pi) / 2 / np.sqrt(x)
        for l in range(kmax):
            Fc[l + 1] = (2 * l + 1) / (2 * x) * Fc[l]
    F[:, A] = Fa[:, A]
    F[:, B] = Fb[:, B]
    F[:, C] = Fc[:, C]
    return F


@pytest.mark.parametrize("kmax", [0, 1, 2, 3, 5, 8, 12, 16, 24, 31, 32])
def test_algorithm1_host_port_within_eps(H, kmax):
    x = np.concatenate([workloads.mixture_c1(6000, seed=kmax), workloads.small_parity_set()[:-1],
                        np.linspace(0, 35, 3001)])
    x = x[np.isfinite(x) & (x >= 0) & (x < 1e300)]
    F = algorithm1_host(H, x, kmax)
    hi, lo = oracle.boys(x, kmax)
    err = np.abs((F - hi) - lo)
    assert err.max() <= EPS + SLACK, (kmax, err.max(), x[np.unravel_index(err.argmax(), err.shape)[1]])


def test_boundary_bit_patterns():
    """The kernels classify arguments by comparing IEEE bit patterns."""
    import struct
    s = open(boys_header.HEADER).read()
    for name, val in (("X0", 11.899848152108484), ("X1", 28.989337738820740)):
        bits = int(re.search(rf"#define BOYS_FP64_{name}_BITS 0x([0-9A-F]+)LL", s).group(1), 16)
        assert bits == struct.unpack("<q", struct.pack("<d", val))[0]
    assert struct.unpack("<q", struct.pack("<d", 1e300))[0] == 0x7E37E43C8800759C
