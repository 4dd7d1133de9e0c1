"""Backward kernel and autograd against the oracle and finite differences.

Tolerances: vs the oracle's -sum_k g_k F_{k+1} (binary128), the F_{k+1}
errors add up to at most 5e-14 * sum_k |g_k| (plus the x_1 slack and the
FMA chain's rounding); vs central differences of the forward with
h = 1e-5 * max(1, x), truncation h^2 |F'''|/6 and round-off ~1e-16/h, plus the
method's own jumps at the region seams (<= 1e-13 / (2h)), are covered by
1e-7 * max(1, sum_k |g_k|).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2512_10059_gb300 as pb
from paper_2512_10059_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _tol(g):
    return 5e-14 * np.abs(g).sum(axis=0) + 64 * 2.0 ** -53 * np.abs(g).sum(axis=0) + 1e-27


@pytest.mark.parametrize("kmax", [0, 1, 5, 16, 31])
def test_grad_vs_oracle(kmax):
    x = np.concatenate([W.mixture_c1(8000, seed=60 + kmax), W.small_parity_set()[:-1]])
    x = x[np.isfinite(x) & (x >= 0) & (x < 1e300)]
    g = W.normal(W.stream_key(6, kmax), (kmax + 1) * x.size).reshape(kmax + 1, x.size)
    dx = pb.boys_grad(torch.from_numpy(x).to(DEV), torch.from_numpy(g).to(DEV), kmax)
    torch.cuda.synchronize()
    got = dx.cpu().numpy()
    hi, lo = oracle.grad(x, g, kmax)
    err = np.abs((got - hi) - lo)
    tol = _tol(g)
    assert np.all(err <= tol), f"kmax={kmax}: worst ratio {np.max(err / tol):.3f}"


def test_grad_c5_full_size():
    """N = 2^24, kmax = 16, x log-uniform [1e-10, 1e3], g ~ N(0,1): sampled
    against the oracle and against central finite differences of the forward."""
    kmax = 16
    x, g = W.grad_c5()
    xt = torch.from_numpy(x).to(DEV)
    gt = torch.from_numpy(g).to(DEV)
    dx = pb.boys_grad(xt, gt, kmax)
    idx = np.random.default_rng(5).choice(x.size, size=1 << 14, replace=False)
    it = torch.from_numpy(idx).to(DEV)
    got = dx[it].cpu().numpy()
    hi, lo = oracle.grad(x[idx], g[:, idx], kmax)
    err = np.abs((got - hi) - lo)
    tol = _tol(g[:, idx])
    assert np.all(err <= tol), f"oracle: worst ratio {np.max(err / tol):.3f}"

    xs = xt[it]
    h = 1e-5 * torch.clamp(xs, min=1.0)
    gs = gt[:, it]

    def L(z):
        return (gs * pb.boys_eval(z.contiguous(), kmax)).sum(0)

    central = (L(xs + h) - L(xs - h)) / (2 * h)
    # below h the central stencil leaves the domain x >= 0: one-sided, same order
    one_sided = (-3 * L(xs) + 4 * L(xs + h) - L(xs + 2 * h)) / (2 * h)
    fd = torch.where(xs >= h, central, one_sided)
    diff = (fd - dx[it]).abs().cpu().numpy()
    bound = 1e-7 * np.maximum(1.0, np.abs(g[:, idx]).sum(axis=0))
    assert np.all(diff <= bound), f"FD: worst ratio {np.max(diff / bound):.3f}"


def test_autograd_function():
    x = torch.from_numpy(W.mixture_c2(3000, seed=8)).to(DEV).requires_grad_(True)
    F = pb.boys(x, 12)
    w = torch.linspace(-1, 1, 13, dtype=torch.float64, device=DEV)[:, None]
    loss = (w * F).sum()
    loss.backward()
    ref = pb.boys_grad(x.detach(), w.expand(13, 3000).contiguous(), 12)
    assert torch.equal(x.grad, ref)


def test_gradcheck_small():
    x = torch.tensor([1e-3, 0.3, 2.0, 11.0, 13.0, 25.0, 40.0], dtype=torch.float64, device=DEV,
                     requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: pb.boys(t, 6), (x,), eps=1e-6, atol=1e-7, rtol=1e-5)
