"""Ragged batches (per-segment kmax) through the C ABI: the plan-less call in
both of its launch shapes (one persistent launch, or the kmax-grouped
launches over a tile table it builds on the device) and the plans.

Each argument must be evaluated by the same code as boys_eval at its
segment's kmax: ragged and flat results are compared bitwise, across every
launch shape the autotuner can pick and across graph replays; a sample is
also checked against the oracle at the paper's 5e-14.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2512_10059_gb300 as pb
from paper_2512_10059_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _small_batch(seed=0, nseg=97):
    rng = np.random.default_rng(seed)
    lens = rng.choice([0, 1, 2, 31, 32, 33, 64, 100, 257, 1000], size=nseg)
    kmax = rng.integers(0, 33, size=nseg).astype(np.int32)
    off = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    x = W.mixture_c1(int(off[-1]), seed=seed + 50)
    return x, off, kmax


def _to(dev, *arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrs]


def _flat_reference(x, off, kmax, out, out_off):
    """Per-kmax flat boys_eval over the concatenated segments, compared bitwise
    with the ragged output blocks (on the device)."""
    xt = torch.from_numpy(x).to(DEV)
    out_off = out_off.cpu().numpy()
    lens = np.diff(off)
    for k in np.unique(kmax):
        segs = np.nonzero((kmax == k) & (lens > 0))[0]
        if segs.size == 0:
            continue
        seg_of = np.repeat(segs, lens[segs])
        j = np.arange(seg_of.size) - np.repeat(np.cumsum(lens[segs]) - lens[segs], lens[segs])
        src = off[seg_of] + j
        flat = pb.boys_eval(xt[torch.from_numpy(src).to(DEV)].contiguous(), int(k))
        pos = out_off[seg_of][None, :] + np.arange(k + 1)[:, None] * lens[seg_of][None, :] + j[None, :]
        got = out[torch.from_numpy(pos.ravel()).to(DEV)].view(k + 1, -1)
        assert torch.equal(got, flat), f"kmax={k}: ragged differs from flat boys_eval"


def test_small_ragged_matches_flat_and_oracle():
    x, off, kmax = _small_batch()
    xt, ot, kt = _to(DEV, x, off, kmax)
    out, out_off = pb.boys_eval_ragged(xt, ot, kt)
    torch.cuda.synchronize()
    _flat_reference(x, off, kmax, out, out_off)
    # oracle on every argument of the batch
    oo = out_off.cpu().numpy()
    host = out.cpu().numpy()
    for s in range(kmax.size):
        n = off[s + 1] - off[s]
        if n == 0:
            continue
        k = int(kmax[s])
        blk = host[oo[s]:oo[s] + (k + 1) * n].reshape(k + 1, n)
        hi, lo = oracle.boys(x[off[s]:off[s + 1]], k)
        assert np.max(np.abs((blk - hi) - lo)) <= 5e-14 + 1e-27, s


@pytest.mark.parametrize("cfg", ["64,1,1", "64,2,2", "128,1,1", "128,2,1", "256,1,2", "256,2,1",
                                 "128,1,0", "256,1,0", "64,1,0"])
def test_launch_shapes_bitwise_identical(cfg, monkeypatch):
    x, off, kmax = _small_batch(seed=3, nseg=300)
    xt, ot, kt = _to(DEV, x, off, kmax)
    ref, out_off = pb.boys_eval_ragged(xt, ot, kt)
    monkeypatch.setenv("BOYS_FORCE_CONFIG", cfg)
    plan = pb.RaggedPlan(xt, ot, kt, autotune=False, force_config=True)
    b, xp, w = (int(v) for v in cfg.split(","))
    assert plan.config() == {"block": b, "xpt": xp, "waves": w}
    got = plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    plan.close()


def test_graph_replay_and_workspace_reset():
    x, off, kmax = _small_batch(seed=7, nseg=200)
    xt, ot, kt = _to(DEV, x, off, kmax)
    plan = pb.RaggedPlan(xt, ot, kt, autotune=False)
    first = plan.launch().clone()
    plan.out.fill_(float("nan"))
    second = plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(first, second), "replay did not redo every tile (counter not reset)"
    plan.close()


def _workspace(nbytes):
    return torch.empty(nbytes, dtype=torch.uint8, device=DEV)


def test_planless_shapes_bitwise_identical():
    """The grouped shape (default workspace), the persistent shape (256 bytes)
    and the grouped shape whose table does not fit (528 + 16 bytes: the
    persistent fallback runs) give the same bits."""
    x, off, kmax = _small_batch(seed=11, nseg=250)
    xt, ot, kt = _to(DEV, x, off, kmax)
    grouped, out_off = pb.boys_eval_ragged(xt, ot, kt)
    persistent, _ = pb.boys_eval_ragged(xt, ot, kt, workspace=_workspace(256))
    overflow, _ = pb.boys_eval_ragged(xt, ot, kt, workspace=_workspace(528 + 16))
    torch.cuda.synchronize()
    assert torch.equal(grouped, persistent)
    assert torch.equal(grouped, overflow)
    _flat_reference(x, off, kmax, grouped, out_off)


def test_grouped_bad_kmax_is_flagged_and_skipped():
    x, off, kmax = _small_batch(seed=12, nseg=40)
    lens = np.diff(off)
    bad = int(np.flatnonzero(lens > 0)[2])
    kmax[bad] = 33
    xt, ot, kt = _to(DEV, x, off, kmax)
    ws = _workspace(pb._lib.lib().boys_ragged_workspace_size_grouped(kmax.size, x.size))
    out_off, total = pb.api.ragged_layout(ot, torch.from_numpy(np.minimum(kmax, 32)).to(DEV))
    out = torch.full((total,), float("nan"), dtype=torch.float64, device=DEV)
    pb.boys_eval_ragged(xt, ot, kt, out=out, out_off=out_off, workspace=ws)
    assert pb.ragged_status(ws) is True
    host = out.cpu().numpy()
    oo = out_off.cpu().numpy()
    assert np.isnan(host[oo[bad]:oo[bad] + 33 * lens[bad]]).all()
    good = np.ones(kmax.size, bool)
    good[bad] = False
    for s in np.flatnonzero(good & (lens > 0)):
        assert not np.isnan(host[oo[s]:oo[s] + (kmax[s] + 1) * lens[s]]).any()


def test_bad_kmax_is_flagged_not_fatal():
    x, off, kmax = _small_batch(seed=9, nseg=20)
    kmax[5] = 40
    xt, ot, kt = _to(DEV, x, off, kmax)
    ws = torch.empty(256, dtype=torch.uint8, device=DEV)
    out, out_off = pb.boys_eval_ragged(xt, ot, kt, workspace=ws)
    assert pb.ragged_status(ws) is True
    kmax[5] = 3
    out, out_off = pb.boys_eval_ragged(xt, ot, torch.from_numpy(kmax).to(DEV), workspace=ws)
    assert pb.ragged_status(ws) is False
    with pytest.raises(pb._lib.BoysError):
        pb.RaggedPlan(xt, ot, torch.from_numpy(np.where(np.arange(20) == 2, 33, kmax).astype(np.int32)).to(DEV))


def test_c3_full_batch_autotuned(tmp_path, monkeypatch):
    """4096 segments, lengths log-uniform 32..65536 (~3.5e7 arguments), kmax =
    la+lb+lc+ld: one autotuned, graph-captured persistent launch, bitwise equal
    to flat per-kmax evaluation, sampled against the oracle."""
    monkeypatch.setenv("BOYS_AUTOTUNE_CACHE", os.path.join(tmp_path, "tune.txt"))
    x, off, kmax = W.ragged_c3()
    xt, ot, kt = _to(DEV, x, off, kmax)
    plan = pb.RaggedPlan(xt, ot, kt, autotune=True)
    out = plan.launch()
    torch.cuda.synchronize()
    _flat_reference(x, off, kmax, out, plan.out_off)
    # the cache file now holds the choice; a second plan reuses it
    assert open(os.path.join(tmp_path, "tune.txt")).read().strip()
    plan2 = pb.RaggedPlan(xt, ot, kt, autotune=True)
    assert plan2.config() == plan.config()
    # the plan-less call (grouped shape, device-built table) gives the same bits
    planless, _ = pb.boys_eval_ragged(xt, ot, kt, out_off=plan.out_off, out=torch.empty_like(out))
    torch.cuda.synchronize()
    assert torch.equal(planless, out)
    rng = np.random.default_rng(3)
    segs = rng.choice(kmax.size, size=64, replace=False)
    oo = plan.out_off.cpu().numpy()
    for s in segs:
        n = int(off[s + 1] - off[s])
        k = int(kmax[s])
        j = rng.choice(n, size=min(n, 64), replace=False)
        pos = oo[s] + np.arange(k + 1)[:, None] * n + j[None, :]
        got = out[torch.from_numpy(pos.ravel()).to(DEV)].view(k + 1, -1).cpu().numpy()
        hi, lo = oracle.boys(x[off[s] + j], k)
        assert np.max(np.abs((got - hi) - lo)) <= 5e-14 + 1e-27
    plan.close()
    plan2.close()
