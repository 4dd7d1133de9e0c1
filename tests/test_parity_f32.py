"""FP32 tier through the C ABI against the binary128 oracle.

Tolerance 1e-6 absolute for every order, measured against the exact F_k at
the float input promoted exactly to double (the tier's contract: accuracy of
the function at the argument it was given).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2512_10059_gb300 as pb
from paper_2512_10059_gb300 import workloads as W
from tests.test_tables_f32 import load

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-6


def _boundary_points(T, kmax):
    pts = []
    for b in (T["x0"][kmax], T["x1"][kmax]):
        v = np.float32(b)
        for _ in range(4):
            v = np.nextafter(v, np.float32(0))
        for _ in range(9):
            pts.append(v)
            v = np.nextafter(v, np.float32(np.inf))
    return np.array(pts, dtype=np.float32)


def _check(xf, got, kmax):
    hi, lo = oracle.boys(xf.astype(np.float64), kmax)
    nan_ref = np.isnan(hi)
    assert np.array_equal(np.isnan(got), nan_ref)
    err = np.where(nan_ref, 0.0, np.abs((got.astype(np.float64) - hi) - lo))
    per_k = err.max(axis=1) if err.size else np.zeros(kmax + 1)
    assert per_k.max() <= TOL, f"kmax={kmax}: worst {per_k.max():.3e} at k={per_k.argmax()}"
    return per_k


def _eval(xf, kmax):
    out = pb.boys_eval_f32(torch.from_numpy(xf).to(DEV), kmax)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def T():
    return load()


@pytest.mark.parametrize("kmax", list(range(33)))
def test_every_kmax(T, kmax):
    xf = np.concatenate([W.mixture_c1(4000, seed=200 + kmax).astype(np.float32), _boundary_points(T, kmax),
                         np.linspace(0, 1.2 * T["x1"][kmax], 3001, dtype=np.float32),
                         np.array([0.0, 1e-30, 1e-8, 1e3, 1e4, 3e38], dtype=np.float32)])
    _check(xf, _eval(xf, kmax), kmax)


@pytest.mark.parametrize("kmax", [5, 9])
@pytest.mark.parametrize("n", [1, 3, 4, 5, 127, 129, 511, 513, 4099])
def test_sizes_tails_and_vector_path(n, kmax):
    """kmax 5 runs four arguments per thread (16-byte vectors), kmax 9 two
    (8-byte vectors); both must agree bitwise with the 8-byte and scalar paths."""
    xf = W.mixture_c2(n, seed=13).astype(np.float32)
    got = _eval(xf, kmax)
    _check(xf, got, kmax)
    base1 = torch.from_numpy(np.concatenate([[0.0], xf]).astype(np.float32)).to(DEV)
    out = torch.empty((kmax + 1, n + 1), dtype=torch.float32, device=DEV)[:, :n]
    pb.boys_eval_f32(base1[1:], kmax, out=out)    # x 4-byte aligned only: scalar path
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), got)
    base2 = torch.from_numpy(np.concatenate([[0.0, 0.0], xf]).astype(np.float32)).to(DEV)
    ld = n + 4 + (n % 2)                           # even ld, 8-byte aligned starts: 2-vector path
    out2 = torch.empty((kmax + 1, ld), dtype=torch.float32, device=DEV)[:, 2:2 + n]
    pb.boys_eval_f32(base2[2:], kmax, out=out2)
    torch.cuda.synchronize()
    assert np.array_equal(out2.cpu().numpy(), got)


def test_special_values():
    xf = np.array([np.nan, -1.0, np.inf, -0.0, 0.0], dtype=np.float32)
    got = _eval(xf, 12)
    assert np.all(np.isnan(got[:, :2]))
    assert np.all(got[:, 2] == 0.0)
    assert np.array_equal(got[:, 3], got[:, 4])


@pytest.mark.parametrize("kmax", [4, 12, 24])
def test_c4_full_size_sampled(T, kmax):
    """N = 2^26 FP32 arguments from the kmax=8 parity mixture (seed 4):
    2^15 sampled arguments plus every argument near this kmax's x0/x1."""
    n = 1 << 26
    xf = W.mixture_c1(n, seed=4).astype(np.float32)
    out = pb.boys_eval_f32(torch.from_numpy(xf).to(DEV), kmax)
    idx = np.random.default_rng(kmax).choice(n, size=1 << 15, replace=False)
    near = np.nonzero((np.abs(xf - T["x0"][kmax]) < 1e-5) | (np.abs(xf - T["x1"][kmax]) < 1e-5) | (xf == 0))[0]
    idx = np.unique(np.concatenate([idx, near[:4096]]))
    got = out[:, torch.from_numpy(idx).to(DEV)].cpu().numpy()
    per_k = _check(xf[idx], got, kmax)
    print(f"kmax={kmax} per-k max abs error vs oracle:", " ".join(f"{v:.2e}" for v in per_k))
