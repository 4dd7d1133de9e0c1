"""The order in which the fused kernel (k_fused_f64 in csrc/boys_fp64.cu) forms
sum_k a^k F_k, replayed in exact rational arithmetic for every kmax 0..32 and
both lane kinds.

The step loop yields value p of the recurrence, F_{kmax-p} on a region-A lane
(downward, Eq. downwardsrecursion) and F_p on a B or C lane (upward); a lane
holds its values p < kmax/2, and each later step p completes the pair F_q, F_p
(q = kmax - p).  The kernel sums the low half sum_{k<=kmax/2} a^k F_k by Horner
as the F_q arrive (descending q), parks the F_p (ascending p), sums them by
Horner afterwards and joins the two with a^(kmax/2+1).  The replay must equal
the definition exactly, for random rationals standing in for the F_k; planted
mistakes in the join power or the parking index fail it.
"""
from fractions import Fraction
import random

import pytest


def _fused_order(kmax, in_a, F, a, mistake=None):
    kh = kmax // 2
    nh = kmax - kh
    vals = [F[kmax - p] if in_a else F[p] for p in range(kmax + 1)]
    hold, park, low = {}, {}, Fraction(0)
    for p, v in enumerate(vals):
        if 2 * p < kmax:
            hold[p] = v
        elif 2 * p == kmax:
            low = v
        else:
            q = kmax - p
            fq = v if in_a else hold[q]
            low = fq if q == kh else low * a + fq
            slot = p - kh - 1 if mistake != "park_index" else p - kh
            park[slot] = hold[q] if in_a else v
    if nh == 0:
        return low
    high = park.get(nh - 1, Fraction(0))
    for j in range(nh - 2, -1, -1):
        high = high * a + park.get(j, Fraction(0))
    power = kh + 1 if mistake != "join_power" else kh
    return low + a ** power * high


@pytest.mark.parametrize("kmax", range(33))
def test_fused_order_equals_definition(kmax):
    rng = random.Random(kmax)
    for trial in range(4):
        F = [Fraction(rng.randint(1, 10 ** 9), rng.randint(1, 10 ** 9)) for _ in range(kmax + 1)]
        a = Fraction(rng.randint(-2000, 2000), rng.randint(1, 97))
        exact = sum(a ** k * F[k] for k in range(kmax + 1))
        for in_a in (True, False):
            assert _fused_order(kmax, in_a, F, a) == exact


@pytest.mark.parametrize("mistake", ["join_power", "park_index"])
def test_fused_order_planted_mistakes_fail(mistake):
    rng = random.Random(7)
    bad = False
    for kmax in (2, 5, 16, 32):
        F = [Fraction(rng.randint(1, 10 ** 6), rng.randint(1, 10 ** 6)) for _ in range(kmax + 1)]
        a = Fraction(-3, 2)
        exact = sum(a ** k * F[k] for k in range(kmax + 1))
        bad = bad or any(_fused_order(kmax, in_a, F, a, mistake) != exact for in_a in (True, False))
    assert bad
