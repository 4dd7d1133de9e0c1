"""The library's elementary functions (FP64: Tang exp, Newton reciprocal and
division, Newton rsqrt; integer pipes: Tang exp in fixed point and the
third-order Newton inverse square root) against CUDA's functions and a long
double reference (binary128 on the AArch64 GPU hosts)."""
import numpy as np
import pytest
import torch

from paper_2512_10059_gb300 import _lib

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _run(fn, a, b=None):
    L = _lib.lib()
    at = torch.from_numpy(a).to(DEV)
    bt = torch.from_numpy(b).to(DEV) if b is not None else None
    out = torch.empty_like(at)
    st = L.boys_diag_math(fn, at.data_ptr(), bt.data_ptr() if bt is not None else None, a.size, out.data_ptr(),
                          int(torch.cuda.current_stream().cuda_stream))
    _lib.check("boys_diag_math", st)
    torch.cuda.synchronize()
    return out.cpu().numpy(), at, bt


def _ulps(got, ref_ld):
    ref = ref_ld.astype(np.float64)
    spacing = np.spacing(np.abs(ref))
    return np.abs((got.astype(np.longdouble) - ref_ld) / spacing.astype(np.longdouble)).astype(np.float64)


def test_exp_neg():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.uniform(0, 30, 200000), rng.uniform(0, 700, 50000), [0.0, 1e-300, 29.0, 700.0]])
    got, at, _ = _run(0, a)
    ref = np.exp(-a.astype(np.longdouble))
    assert _ulps(got, ref).max() <= 2.0
    cuda = torch.exp(-at).cpu().numpy()
    assert np.max(np.abs(got - cuda) / np.spacing(cuda)) <= 2.0


@pytest.mark.parametrize("fn", [1, 2, 3])
def test_reciprocal_division_rsqrt(fn):
    rng = np.random.default_rng(fn)
    a = np.exp(rng.uniform(-300, 300, 300000) * np.log(2.0))
    b = rng.uniform(-1e3, 1e3, a.size) if fn == 2 else None
    got, at, bt = _run(fn, a, b)
    A = a.astype(np.longdouble)
    if fn == 1:
        ref, cuda = 1 / A, (1.0 / at).cpu().numpy()
        bound = 1.0
    elif fn == 2:
        ref, cuda = b.astype(np.longdouble) / A, (bt / at).cpu().numpy()
        bound = 1.0
    else:
        ref, cuda = 1 / np.sqrt(A), torch.rsqrt(at).cpu().numpy()
        bound = 1.5
    assert _ulps(got, ref).max() <= bound
    assert np.max(np.abs(got - cuda) / np.spacing(np.abs(cuda))) <= bound + 1.0


def test_exp_neg_integer_pipes():
    """e^{-a} in the 64-bit-significand format (Tang's method in fixed point):
    relative error below 2^-59, so the significand rounded to nearest double
    is within 0.5 + 2^-6 ulp of the exact value."""
    rng = np.random.default_rng(7)
    k = np.arange(0, 10600)
    grid = k * (np.log(2.0) / 256)                      # reduction points and their neighbours
    a = np.concatenate([rng.uniform(0, 32, 300000), np.exp(rng.uniform(np.log(1e-300), np.log(2.0), 50000)),
                        grid, np.nextafter(grid, 0.0), np.nextafter(grid, 64.0),
                        [0.0, 5e-324, 1e-310, 2.0 ** -5, np.nextafter(2.0 ** -5, 0.0), 11.899848152108484,
                         28.98933773882074, np.nextafter(32.0, 0.0)]])
    a = a[(a >= 0) & (a < 32)]
    got, at, _ = _run(4, a)
    assert got[a == 0.0][0] == 1.0
    ref = np.exp(-a.astype(np.longdouble))
    assert _ulps(got, ref).max() <= 0.52
    cuda = torch.exp(-at).cpu().numpy()
    assert np.max(np.abs(got - cuda) / np.spacing(cuda)) <= 1.0


def test_rsqrt_integer_pipes():
    """a^{-1/2} in the 64-bit-significand format (rsqrt.approx.f32 seed of the
    top 23 significand bits, one third-order Newton step): relative error
    below 2^-59, so the significand rounded to nearest double is within
    0.5 + 2^-6 ulp.  Both exponent parities, powers of two, the seed's
    mantissa boundaries and the anchors' range (q^2 up to 5e33, x up to 1e300)."""
    rng = np.random.default_rng(11)
    a = np.concatenate([np.exp(rng.uniform(-690, 690, 300000)), rng.uniform(1.0, 4.0, 100000),
                        2.0 ** np.arange(-1000, 1000), np.nextafter(2.0 ** np.arange(-60, 60), 0.0),
                        1.0 + 2.0 ** -23 * np.arange(0, 4096), [1e300, 5e33, 4e14, 28.98933773882074]])
    got, at, _ = _run(5, a)
    ref = 1 / np.sqrt(a.astype(np.longdouble))
    assert _ulps(got, ref).max() <= 0.52
    cuda = torch.rsqrt(at).cpu().numpy()
    assert np.max(np.abs(got - cuda) / np.spacing(cuda)) <= 1.0
