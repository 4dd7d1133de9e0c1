"""The paper's benchmark workload (Section III, Algorithm 2) against the
binary128 oracle.

Tolerance: each F_l carries at most 5e-14, so |dz_i| <= 5e-14 sum_l|c_l|
sum_j|y_j|, plus the FP64 rounding of the two sums (k+1 and n terms of size
at most |c_l| |y_j|): 2^-53 (n + k + 2) sum_l|c_l| sum_j|y_j|.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2512_10059_gb300 as pb
from paper_2512_10059_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _tol(y, c, n, k):
    s = np.abs(c).sum() * np.abs(y).sum()
    return 5e-14 * s + 2.0 ** -53 * (n + k + 2) * s + 1e-27


def _run(x, y, c):
    z = pb.boys_pairwise(torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV), torch.from_numpy(c).to(DEV))
    torch.cuda.synchronize()
    return z.cpu().numpy()


@pytest.mark.parametrize("n,k,sort", [(1, 0, True), (97, 5, False), (300, 12, True), (300, 12, False),
                                      (257, 32, True), (200, 3, False)])
def test_pairwise_vs_oracle(n, k, sort):
    x, y, c = W.pairwise_alg2(n, k, seed=n + k, sort=sort)
    got = _run(x, y, c)
    hi, lo = oracle.pairwise(x, y, c)
    err = np.abs((got - hi) - lo)
    assert err.max() <= _tol(y, c, n, k), err.max()


def test_pairwise_special_arguments():
    x = np.array([0.0, 5.0, W.X0_PRINTED / 2, W.X1_PRINTED / 2, 15.0, 30.0])
    y = np.array([1.0, -2.0, 0.5, 3.0, -1.0, 0.25])
    c = np.array([1.0, -1.0, 0.5, 2.0])
    got = _run(x, y, c)
    hi, lo = oracle.pairwise(x, y, c)
    assert np.max(np.abs((got - hi) - lo)) <= _tol(y, c, 6, 3)


def test_pairwise_order_invariant():
    x, y, c = W.pairwise_alg2(1000, 12, seed=5, sort=False)
    perm = np.argsort(x)
    z1 = _run(x, y, c)
    z2 = _run(x[perm], y[perm], c)
    assert np.max(np.abs(z1[perm] - z2)) <= _tol(y, c, 1000, 12)


@pytest.mark.parametrize("log2n,nrows", [(17, 8), (19, 3)])
def test_pairwise_bench_sizes_sampled(log2n, nrows):
    """The two launches bench.py times: N = 2^17 and the paper's N = 2^19,
    sorted x on [0, 30], k = 12, seed 8; sampled rows against the oracle."""
    x, y, c = W.pairwise_alg2(1 << log2n, 12, seed=8, sort=True)
    got = _run(x, y, c)
    rows = np.random.default_rng(log2n).choice(x.size, nrows, replace=False)
    hi, lo = oracle.pairwise_rows(x, y, c, rows)
    err = np.abs((got[rows] - hi) - lo)
    assert err.max() <= _tol(y, c, x.size, 12), err.max()


@pytest.mark.parametrize("k,sort", [(12, True), (12, False), (32, True), (3, False)])
def test_pairwise_one_hot_pins_each_pair(k, sort):
    """y = e_m makes z_i = sum_l c_l F_l(x_i + x_m): every output pins one
    pair, so the bound is the per-pair one, 5e-14 sum_l|c_l| plus the rounding
    of the k+1-term sum, independent of n.  The m are chosen so that x_i + x_m
    covers regions A, B and C (and the region-C Horner form in sorted warps)."""
    n = 640
    x, _, c = W.pairwise_alg2(n, k, seed=70 + k, sort=sort)
    sc = np.abs(c).sum()
    tol = 5e-14 * sc + 2.0 ** -53 * (k + 2) * sc + 1e-27
    order = np.argsort(x)
    for m in (order[0], order[n // 3], order[2 * n // 3], order[-1]):
        y = np.zeros(n)
        y[m] = 1.0
        got = _run(x, y, c)
        hi, lo = oracle.pairwise(x, y, c)
        err = np.abs((got - hi) - lo)
        assert err.max() <= tol, (m, err.max(), tol)


@pytest.mark.parametrize("k", [0, 1, 12, 32])
def test_pairwise_region_c_closed_form(k):
    """Every x_i + x_j >= 30 lies in region C, where the kernel forms
    w = F_0 sum_l c_l (2l-1)!! u^l (u = 1/(2X)) instead of running the
    recurrence; same tolerance."""
    rng = np.random.default_rng(40 + k)
    n = 160
    x = np.sort(rng.uniform(15.0, 30.0, n))
    y = rng.standard_normal(n)
    c = rng.standard_normal(k + 1)
    got = _run(x, y, c)
    hi, lo = oracle.pairwise(x, y, c)
    assert np.max(np.abs((got - hi) - lo)) <= _tol(y, c, n, k)
