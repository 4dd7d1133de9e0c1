"""The ragged entry point that allocates nothing, boys_eval_ragged_noalloc.

It exists for callers that cannot give the library device memory (their
framework or application owns every allocation, or they cannot afford
cudaMalloc's synchronisation): its scratch is a static array inside the
library.  The GPU test calls it through the C ABI twice in a row (the second
call must find the shared tile counter re-zeroed) and compares each result
with the workspace-taking boys_eval_ragged at the parity tolerance used by the
other tests (5e-14 absolute); the two share the kernel, so the results are
also expected to be bitwise equal.  A batch with one segment of kmax 33 checks
that the segment is skipped and that boys_ragged_noalloc_status reports it
(an ordinary input check: the kernel skips the segment and sets a flag).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2512_10059_gb300 import _lib, api, build
from paper_2512_10059_gb300 import workloads as W

FAKE = 0x10000  # never dereferenced: the argument checks reject these calls first


def test_noalloc_argument_errors_without_gpu():
    build.build()
    L = _lib.lib()
    assert L.boys_eval_ragged_noalloc(FAKE, FAKE, FAKE, -1, FAKE, FAKE, None) == 1
    assert L.boys_eval_ragged_noalloc(None, None, None, 0, None, None, None) == 0
    assert L.boys_eval_ragged_noalloc(FAKE, None, FAKE, 4, FAKE, FAKE, None) == 1
    assert L.boys_eval_ragged_noalloc(FAKE, FAKE, FAKE + 2, 4, FAKE, FAKE, None) == 3
    assert L.boys_ragged_noalloc_status(None, None) == 1


def _batch(seed, nseg):
    rng = np.random.default_rng(seed)
    lens = rng.choice([0, 1, 7, 32, 33, 100, 513, 4000], size=nseg)
    kmax = rng.integers(0, 33, size=nseg).astype(np.int32)
    off = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    x = W.mixture_c1(int(off[-1]), seed=seed + 1)
    return x, off, kmax


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_twice():
    dev = "cuda:0"
    L = _lib.lib()
    for call, (seed, nseg) in enumerate([(31, 150), (32, 400)]):
        x, off, kmax = _batch(seed, nseg)
        xt = torch.from_numpy(x).to(dev)
        ot = torch.from_numpy(off).to(dev)
        kt = torch.from_numpy(kmax).to(dev)
        ref, out_off = api.boys_eval_ragged(xt, ot, kt)
        got = torch.full_like(ref, float("nan"))
        stream = torch.cuda.current_stream(dev)
        st = L.boys_eval_ragged_noalloc(xt.data_ptr(), ot.data_ptr(), kt.data_ptr(), nseg, got.data_ptr(),
                                        out_off.data_ptr(), int(stream.cuda_stream))
        assert st == 0, L.boys_last_error()
        torch.cuda.synchronize()
        assert not torch.isnan(got).any(), f"call {call}: some outputs were not written"
        assert torch.max(torch.abs(got - ref)).item() <= 5e-14, f"call {call}: differs from boys_eval_ragged"
        assert torch.equal(got, ref), f"call {call}: not bitwise equal to boys_eval_ragged"


@pytest.mark.gpu
def test_noalloc_reports_bad_kmax_and_clears_it():
    dev = "cuda:0"
    L = _lib.lib()
    x, off, kmax = _batch(33, 60)
    bad = int(np.flatnonzero(np.diff(off) > 0)[3])  # a non-empty segment
    kmax[bad] = 33
    xt = torch.from_numpy(x).to(dev)
    ot = torch.from_numpy(off).to(dev)
    kt = torch.from_numpy(kmax).to(dev)
    lens = np.diff(off)
    out_off = np.zeros(kmax.size, dtype=np.int64)
    np.cumsum(((np.minimum(kmax, 32) + 1) * lens)[:-1], out=out_off[1:])
    oo = torch.from_numpy(out_off).to(dev)
    got = torch.full((int(out_off[-1] + (min(kmax[-1], 32) + 1) * lens[-1]),), float("nan"),
                     dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    hs = int(stream.cuda_stream)
    assert L.boys_eval_ragged_noalloc(xt.data_ptr(), ot.data_ptr(), kt.data_ptr(), kmax.size, got.data_ptr(),
                                      oo.data_ptr(), hs) == 0, L.boys_last_error()
    flag = ctypes.c_int(-1)
    assert L.boys_ragged_noalloc_status(ctypes.byref(flag), hs) == 0
    assert flag.value == 1
    g = got.cpu().numpy()
    o0, n0 = int(out_off[bad]), int(lens[bad])
    assert np.isnan(g[o0:o0 + 33 * n0]).all(), "the skipped segment's block was written"
    for s in range(kmax.size):
        if s == bad or lens[s] == 0:
            continue
        blk = g[int(out_off[s]):int(out_off[s]) + (int(kmax[s]) + 1) * int(lens[s])]
        assert not np.isnan(blk).any(), f"segment {s} was not written"
        ref = api.boys_eval(xt[int(off[s]):int(off[s + 1])], int(kmax[s])).cpu().numpy().reshape(-1)
        assert np.array_equal(blk, ref), f"segment {s} differs from boys_eval"
    # a following valid call clears the flag
    kt.copy_(torch.from_numpy(np.minimum(kmax, 32)))
    assert L.boys_eval_ragged_noalloc(xt.data_ptr(), ot.data_ptr(), kt.data_ptr(), kmax.size, got.data_ptr(),
                                      oo.data_ptr(), hs) == 0
    assert L.boys_ragged_noalloc_status(ctypes.byref(flag), hs) == 0
    assert flag.value == 0


@pytest.mark.gpu
def test_noalloc_python_binding():
    """The binding's wrappers marshal to the same calls: bitwise the result
    of boys_eval_ragged, and the status reads the error word."""
    dev = "cuda:0"
    x, off, kmax = _batch(34, 120)
    xt = torch.from_numpy(x).to(dev)
    ot = torch.from_numpy(off).to(dev)
    kt = torch.from_numpy(kmax).to(dev)
    ref, out_off = api.boys_eval_ragged(xt, ot, kt)
    got, got_off = api.boys_eval_ragged_noalloc(xt, ot, kt)
    assert torch.equal(got_off, out_off)
    assert torch.equal(got, ref)
    assert api.ragged_noalloc_status() is False

