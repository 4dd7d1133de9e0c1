"""The FP32-tier tables produced by the project's Remez generator (CPU only).

* x0(kmax) equals Eq. x0 for every kmax (rounded to float)
* x1(kmax) solves Eq. x1 for the 3e-7 region-C budget: the asymptotic form's
  error Gamma(k+1/2)/(2 x1^{k+1/2}) - F_kmax(x1) (oracle) is 3e-7 at x1
* monic denominators, no pole of r_A on [0, x0] or of r_B on [x0, x1]
* every fit whose levelled error is well above the FP32 rounding of its
  coefficients equioscillates (Theorem 1): at least n+m+2 alternating error
  extrema of nearly equal size on its interval
* the generator reproduces the committed header (x86-64 only: the tables
  depend on the long double format)
"""
import math
import os
import platform
import re

import numpy as np
import pytest

import oracle

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2512_10059_gb300", "csrc", "boys_coeffs_fp32.h")


def load():
    s = open(HEADER).read()

    def vec(name, cast=float):
        body = re.search(r"#define " + name + r" \{ (.*?) \}\n", s).group(1)
        return [cast(v.strip().rstrip("f")) for v in body.split(",")]

    def mat(name):
        body = re.search(r"#define " + name + r" \{ \\\n(.*?)\n\}", s, re.S).group(1)
        rows = re.findall(r"\{ (.*?) \}", body)
        return [[float(v.strip().rstrip("f")) for v in r.split(",")] for r in rows]

    T = {"x0": vec("BOYS_F32_X0_INIT"), "x1": vec("BOYS_F32_X1_INIT"),
         "an": vec("BOYS_F32_AN_INIT", int), "am": vec("BOYS_F32_AM_INIT", int),
         "bn": vec("BOYS_F32_BN_INIT", int), "bm": vec("BOYS_F32_BM_INIT", int),
         "ap": mat("BOYS_F32_AP_INIT"), "aq": mat("BOYS_F32_AQ_INIT"),
         "bp": mat("BOYS_F32_BP_INIT"), "bq": mat("BOYS_F32_BQ_INIT")}
    for key, name in (("eap", "AP"), ("eaq", "AQ"), ("ebp", "BP"), ("ebq", "BQ")):
        T[key] = mat(f"BOYS_F32_{name}_EXT")
    T["EA"], T["EB"] = {}, {}
    for m in re.finditer(r"kmax=\s*(\d+)\s+worst (\S+)\s+\|E_A\| (\S+)\s+\|E_B\| (\S+)", s):
        k = int(m.group(1))
        T["EA"][k] = float(m.group(3))
        T["EB"][k] = float(m.group(4))
    return T


@pytest.fixture(scope="module")
def T():
    return load()


def test_x0_equation(T):
    for kmax in range(33):
        lp = sum(math.log(k + 0.5) for k in range(kmax))
        x0 = 1.0 if kmax == 0 else max(1.0, math.exp(lp / kmax))
        assert abs(T["x0"][kmax] - np.float32(x0)) <= 2e-7 * x0, kmax


def test_x1_equation(T):
    for kmax in range(33):
        x1 = T["x1"][kmax]
        hi, lo = oracle.boys([x1], kmax)
        asym = math.exp(math.lgamma(kmax + 0.5) - (kmax + 0.5) * math.log(x1)) / 2
        err = asym - (hi[kmax, 0] + lo[kmax, 0])
        # float rounding of x1 moves the error by < 1e-6 relative of itself per ulp
        assert abs(err - 3e-7) <= 1e-5 * 3e-7 + 1e-12, (kmax, err)


def _poly(c, x):
    v = np.zeros_like(x) + c[-1]
    for a in reversed(c[:-1]):
        v = v * x + a
    return v


def _fit(T, kmax, region, exact=False):
    """(n, m, p, q, a, b, k, E) of one approximant; ``exact`` selects the
    unrounded coefficients instead of the FP32 ones."""
    if region == "A":
        n, m = T["an"][kmax], T["am"][kmax]
        p, q = (T["eap"][kmax], T["eaq"][kmax]) if exact else (T["ap"][kmax][:n + 1], T["aq"][kmax][:m + 1])
        a, b, k, E = 0.0, T["x0"][kmax], kmax, T["EA"][kmax]
    else:
        n, m = T["bn"][kmax], T["bm"][kmax]
        p, q = (T["ebp"][kmax], T["ebq"][kmax]) if exact else (T["bp"][kmax][:n + 1], T["bq"][kmax][:m + 1])
        a, b, k, E = T["x0"][kmax], T["x1"][kmax], 0, T["EB"][kmax]
    assert len(p) == n + 1 and len(q) == m + 1
    return n, m, p, q, a, b, k, E


def _rho(kmax, x, region):
    if region != "A":
        return np.ones_like(x)
    best = np.ones_like(x)
    prod = np.ones_like(x)
    for nn in range(kmax - 1, -1, -1):
        prod = prod * x / (nn + 0.5)
        best = np.maximum(best, prod)
    return best


@pytest.mark.parametrize("region", ["A", "B"])
def test_monic_and_pole_free(T, region):
    for kmax in range(33):
        n, m, p, q, a, b, k, E = _fit(T, kmax, region)
        assert q[-1] == 1.0
        xs = np.linspace(a, b, 20001)
        qv = _poly(q, xs)
        assert np.all(qv > 0) or np.all(qv < 0), (kmax, region)


@pytest.mark.parametrize("region", ["A", "B"])
def test_equioscillation(T, region):
    """Theorem 1 on the unrounded approximants (the FP32 rounding of the
    coefficients perturbs the error curve by about as much as E itself)."""
    checked = 0
    for kmax in range(33):
        n, m, p, q, a, b, k, E = _fit(T, kmax, region, exact=True)
        xs = np.linspace(a, b, 8001)
        hi, lo = oracle.boys(xs, k)
        e = _rho(kmax, xs, region) * ((hi[k] + lo[k]) - _poly(p, xs) / _poly(q, xs))
        # alternating extrema: split at sign changes, keep the max of each run
        runs = []
        for v in e:
            if runs and (v > 0) == (runs[-1] > 0):
                if abs(v) > abs(runs[-1]):
                    runs[-1] = v
            else:
                runs.append(v)
        big = [v for v in runs if abs(v) >= 0.98 * E]
        alternations = 1 + sum(1 for u, v in zip(big[:-1], big[1:]) if (u > 0) != (v > 0))
        assert alternations >= n + m + 2, (kmax, region, n, m, alternations, E)
        assert np.max(np.abs(e)) <= 1.01 * E, (kmax, region, np.max(np.abs(e)), E)
        checked += 1
    assert checked == 33


@pytest.mark.skipif(platform.machine() != "x86_64", reason="tables were generated with x86-64 long double")
def test_generator_reproduces_committed_header():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "gen", os.path.join(os.path.dirname(HEADER), "remez", "generate.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    text = gen.run()
    assert text == open(HEADER).read()
