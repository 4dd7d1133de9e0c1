"""Seeded input generators: determinism, the published splitmix64 stream and
the shapes the workloads promise (CPU only)."""
import numpy as np

from paper_2512_10059_gb300 import workloads as W


def test_splitmix64_reference_vector():
    # splitmix64 seeded with 0: first outputs as published with the reference
    # implementation (Vigna, splitmix64.c): 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4
    out = W.raw64(np.uint64(0), 2)
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_splitmix64_scalar_definition():
    M = (1 << 64) - 1
    s = 0x1234567
    ref = []
    for _ in range(5):
        s = (s + 0x9E3779B97F4A7C15) & M
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        ref.append(z ^ (z >> 31))
    assert [int(v) for v in W.raw64(np.uint64(0x1234567), 5)] == ref


def test_deterministic_and_offsets():
    a = W.uniform01(W.stream_key(3, 1), 1000)
    b = W.uniform01(W.stream_key(3, 1), 500, start=500)
    assert np.array_equal(a[500:], b)
    assert np.all((a >= 0) & (a < 1))


def test_c1_mixture_shape():
    x = W.mixture_c1(65536, seed=0)
    assert x.size == 65536
    assert np.array_equal(x, W.mixture_c1(65536, seed=0))
    assert np.count_nonzero(x == 0.0) == round(0.05 * 65536)
    near = (np.abs(x - W.X0_PRINTED) <= 1.001e-12) | (np.abs(x - W.X1_PRINTED) <= 1.001e-12)
    assert np.count_nonzero(near) == round(0.05 * 65536)
    assert np.any(x == W.X0_PRINTED) and np.any(x == W.X1_PRINTED)
    rest = x[(x != 0) & ~near]
    assert rest.min() >= 1e-8 and rest.max() <= 1e3


def test_c2_mixture_fractions():
    x = W.mixture_c2(1 << 18, seed=1)
    assert x.min() >= 0 and x.max() <= 1e4
    big = np.mean(x >= 60)
    assert 0.17 < big < 0.23


def test_c3_ragged_shape():
    x, off, km = W.ragged_c3()
    assert off.size == 4097 and km.size == 4096 and off[0] == 0 and off[-1] == x.size
    lens = np.diff(off)
    assert lens.min() >= 32 and lens.max() <= 65536
    assert km.min() >= 0 and km.max() <= 16
    assert 3.6 < km.mean() < 4.6


def test_c5_grad_shape():
    x, g = W.grad_c5(n=4096)
    assert g.shape == (17, 4096)
    assert abs(g.mean()) < 0.05 and 0.95 < g.std() < 1.05
