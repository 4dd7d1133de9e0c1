"""The oracle against facts fixed by the paper and by mathematics (CPU only)."""
import pytest

import oracle
from tests import oracle_pins as P


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


def test_precision_is_binary128(orc):
    assert orc.mantissa_bits() == 113


@pytest.mark.parametrize("pin", P.CPU_PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin(orc)


@pytest.mark.parametrize("pin", P.MP_PINS, ids=lambda f: f.__name__)
def test_pin_mpmath(orc, pin):
    mpmath = pytest.importorskip("mpmath")
    pin(orc, mpmath)


def test_recurrence_identity_mpmath(orc):
    mpmath = pytest.importorskip("mpmath")
    P.pin_recurrence_identity(orc, mpmath)


def test_domain_conventions(orc):
    import math
    import numpy as np
    hi, lo = orc.boys([float("nan"), -1.0, float("inf"), -0.0], 5)
    assert np.all(np.isnan(hi[:, 0])) and np.all(np.isnan(hi[:, 1]))
    assert np.all(hi[:, 2] == 0.0)
    assert np.all(hi[:, 3] == 1.0 / (2 * np.arange(6) + 1))
    with pytest.raises(ValueError):
        orc.boys([1.0], orc.kmax_limit() + 1)
    assert not math.isnan(orc.boys([1e-300], 40)[0][40, 0])
