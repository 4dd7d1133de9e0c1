"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case copies ``oracle/boys_oracle.c``, applies one plausible mistake
(a dropped factor, a wrong sign or index, a loose truncation, a route used
where it is unstable), compiles the copy to a temporary library and runs
the full pin battery against it: at least one pin has to fail.  Nothing is
changed in the real oracle.
"""
import os

import pytest

import oracle
from oracle import build as obuild
from tests import oracle_pins as P

SRC = obuild.SRC

MUTANTS = {
    "series_ratio_index": ("x / (kh + (qreal)(l + 1))", "x / (kh + (qreal)(l + 2))"),
    "series_missing_half": ("return QL(0.5) * QEXP(-x) * s;", "return QEXP(-x) * s;"),
    "series_first_term": ("qreal t = QL(1.0) / kh;", "qreal t = QL(1.0) / (kh + QL(1.0));"),
    "series_loose_truncation": ("#define SERIES_REL_TOL QL(1e-40)", "#define SERIES_REL_TOL QL(1e-9)"),
    "upward_exp_sign": ("* f[k] - emx) / (QL(2.0) * x)", "* f[k] + emx) / (QL(2.0) * x)"),
    "upward_order_index": ("(qreal)(2 * k + 1) * f[k] - emx", "(qreal)(2 * k + 3) * f[k] - emx"),
    "erf_route_missing_sqrt": ("QL(0.5) * QSQRT(Q_PI / x) * QERF(rx)", "QL(0.5) * (Q_PI / x) * QERF(rx)"),
    "upward_used_at_small_x": ("#define X_SWITCH QL(30.0)", "#define X_SWITCH QL(2.0)"),
    "fused_sign": ("qreal a = QL(-2.0) * (qreal)rho[i]", "qreal a = QL(2.0) * (qreal)rho[i]"),
    "grad_order_index": ("* f[k + 1];", "* f[k];"),
    "grad_sign": ("q_split(-s, &d_hi[i], &d_lo[i]);", "q_split(s, &d_hi[i], &d_lo[i]);"),
    "pairwise_argument": ("boys_q(x[i] + x[j], k, 0, f)) { err |= 1; break; }",
                          "boys_q(x[i] + x[i], k, 0, f)) { err |= 1; break; }"),
    "pairwise_sign": ("q_split(z, &z_hi[i], &z_lo[i]);", "q_split(-z, &z_hi[i], &z_lo[i]);"),
    "pairwise_rows_scale": ("q_split(z, &z_hi[r], &z_lo[r]);", "q_split(z + z, &z_hi[r], &z_lo[r]);"),
}


def _battery(o):
    failures = []
    pins = list(P.CPU_PINS)
    try:
        import mpmath
        pins += [lambda oo, f=f: f(oo, mpmath) for f in P.MP_PINS]
    except ImportError:
        pass
    for pin in pins:
        try:
            pin(o)
        except (AssertionError, ValueError, FloatingPointError, OverflowError, ZeroDivisionError) as exc:
            failures.append((getattr(pin, "__name__", "pin"), repr(exc)[:120]))
    return failures


def test_real_oracle_passes_battery():
    assert _battery(oracle.default()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    with open(SRC) as fh:
        text = fh.read()
    assert text.count(old) == 1, f"mutation site for {name} not found exactly once"
    src = os.path.join(tmp_path, "boys_oracle_mutant.c")
    with open(src, "w") as fh:
        fh.write(text.replace(old, new))
    lib = obuild.build(force=True, src=src, lib=os.path.join(tmp_path, "libmutant.so"))
    failures = _battery(oracle.OracleLib(lib))
    assert failures, f"planted mistake {name} passed every pin"
