"""torch-facing wrappers of the libboys entry points (argument marshalling only).

Tensors must live on a CUDA device; work is enqueued on the current torch
stream of that device (or ``stream``) and is asynchronous like any torch op.
"""
import ctypes

import torch

from . import _lib


def _stream_handle(t: torch.Tensor, stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream(t.device)
    return int(s.cuda_stream)


def _require(t: torch.Tensor, name: str, dtype=torch.float64):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")


def version() -> int:
    return _lib.lib().boys_version()


def kmax_limit() -> int:
    return _lib.lib().boys_kmax_limit()


def boys_eval(x: torch.Tensor, kmax: int, out: torch.Tensor = None, stream=None) -> torch.Tensor:
    """F_0..F_kmax(x) in FP64: returns ``out`` of shape [kmax+1, n] (row stride = ld).

    ``x`` is a contiguous float64 CUDA tensor of n arguments.  ``out`` may be
    given as any [kmax+1, n] float64 view with unit column stride.
    """
    _require(x, "x")
    x = x.contiguous().view(-1)
    n = x.numel()
    if out is None:
        out = torch.empty((kmax + 1, n), dtype=torch.float64, device=x.device)
    _require(out, "out")
    if out.dim() != 2 or out.shape[0] != kmax + 1 or out.shape[1] != n or (n > 1 and out.stride(1) != 1):
        raise ValueError(f"out must be [{kmax + 1}, {n}] with unit column stride")
    ld = out.stride(0) if kmax > 0 else max(n, 1)
    st = _lib.lib().boys_eval(x.data_ptr(), n, int(kmax), out.data_ptr(), ld, _stream_handle(x, stream))
    _lib.check("boys_eval", st)
    return out


def boys_eval_host(x: torch.Tensor, kmax: int, out: torch.Tensor = None, stream=None,
                   device=None) -> torch.Tensor:
    """F_0..F_kmax for a pinned HOST tensor x, written into a pinned host
    tensor ``out`` [kmax+1, n] by the kernel over the host link (no device
    staging).  Asynchronous on the current stream of ``device`` (default
    cuda:0): synchronise before reading ``out``."""
    if x.is_cuda or x.dtype != torch.float64:
        raise TypeError("x must be a float64 CPU tensor (pinned)")
    x = x.contiguous().view(-1)
    n = x.numel()
    if out is None:
        out = torch.empty((kmax + 1, n), dtype=torch.float64, pin_memory=True)
    if out.is_cuda or out.dtype != torch.float64 or out.dim() != 2 or out.shape != (kmax + 1, n) \
            or (n > 1 and out.stride(1) != 1):
        raise ValueError(f"out must be a float64 CPU tensor [{kmax + 1}, {n}] with unit column stride")
    dev = torch.device(device) if device is not None else torch.device("cuda", 0)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    ld = out.stride(0) if kmax > 0 else max(n, 1)
    st = _lib.lib().boys_eval_host(x.data_ptr(), n, int(kmax), out.data_ptr(), ld, int(s.cuda_stream))
    _lib.check("boys_eval_host", st)
    return out


def boys_eval_f32(x: torch.Tensor, kmax: int, out: torch.Tensor = None, stream=None) -> torch.Tensor:
    """FP32 tier: F_0..F_kmax(x) at 1e-6 absolute accuracy, [kmax+1, n] float32."""
    _require(x, "x", torch.float32)
    x = x.contiguous().view(-1)
    n = x.numel()
    if out is None:
        out = torch.empty((kmax + 1, n), dtype=torch.float32, device=x.device)
    _require(out, "out", torch.float32)
    if out.dim() != 2 or out.shape[0] != kmax + 1 or out.shape[1] != n or (n > 1 and out.stride(1) != 1):
        raise ValueError(f"out must be [{kmax + 1}, {n}] with unit column stride")
    ld = out.stride(0) if kmax > 0 else max(n, 1)
    st = _lib.lib().boys_eval_f32(x.data_ptr(), n, int(kmax), out.data_ptr(), ld, _stream_handle(x, stream))
    _lib.check("boys_eval_f32", st)
    return out


def boys_eval_fused(x: torch.Tensor, rho: torch.Tensor, kmax: int, out: torch.Tensor = None,
                    stream=None) -> torch.Tensor:
    """sum_k (-2 rho_i)^k F_k(x_i) for every i, F_k kept in registers."""
    _require(x, "x")
    _require(rho, "rho")
    x = x.contiguous().view(-1)
    rho = rho.contiguous().view(-1)
    if rho.numel() != x.numel():
        raise ValueError("x and rho must have the same length")
    n = x.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=x.device)
    _require(out, "out")
    if not out.is_contiguous() or out.numel() != n:
        raise ValueError("out must be a contiguous [n] tensor")
    st = _lib.lib().boys_eval_fused(x.data_ptr(), rho.data_ptr(), n, int(kmax), out.data_ptr(),
                                    _stream_handle(x, stream))
    _lib.check("boys_eval_fused", st)
    return out


def boys_grad(x: torch.Tensor, g: torch.Tensor, kmax: int, out: torch.Tensor = None,
              stream=None) -> torch.Tensor:
    """dL/dx = -sum_k g[k] * F_{k+1}(x) for upstream gradients g [kmax+1, n]."""
    _require(x, "x")
    _require(g, "g")
    x = x.contiguous().view(-1)
    n = x.numel()
    if g.dim() != 2 or g.shape[0] != kmax + 1 or g.shape[1] != n:
        raise ValueError(f"g must be [{kmax + 1}, {n}]")
    if n > 1 and g.stride(1) != 1:
        g = g.contiguous()
    ldg = g.stride(0) if kmax > 0 else max(n, 1)
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=x.device)
    _require(out, "out")
    st = _lib.lib().boys_grad(x.data_ptr(), n, int(kmax), g.data_ptr(), ldg, out.data_ptr(),
                              _stream_handle(x, stream))
    _lib.check("boys_grad", st)
    return out


class BoysFunction(torch.autograd.Function):
    """F_0..F_kmax(x) as a differentiable op: forward is boys_eval, backward is
    boys_grad (only x is saved; F_{kmax+1} is recomputed).  kmax <= 31 when a
    gradient is needed."""

    @staticmethod
    def forward(ctx, x, kmax):
        ctx.kmax = int(kmax)
        ctx.save_for_backward(x)
        return boys_eval(x, ctx.kmax)

    @staticmethod
    def backward(ctx, grad_out):
        (x,) = ctx.saved_tensors
        dx = boys_grad(x, grad_out.contiguous(), ctx.kmax)
        return dx.view_as(x), None


def boys(x: torch.Tensor, kmax: int) -> torch.Tensor:
    """Differentiable F_0..F_kmax(x): [kmax+1, n] float64."""
    return BoysFunction.apply(x, kmax)


def boys_pairwise(x: torch.Tensor, y: torch.Tensor, c: torch.Tensor, out: torch.Tensor = None,
                  stream=None) -> torch.Tensor:
    """z_i = sum_l c_l sum_j F_l(x_i + x_j) y_j (the paper's Algorithm 2);
    k = len(c) - 1.  Sort x ascending (with y) for speed."""
    for t, name in ((x, "x"), (y, "y"), (c, "c")):
        _require(t, name)
    x = x.contiguous().view(-1)
    y = y.contiguous().view(-1)
    c = c.contiguous().view(-1)
    if y.numel() != x.numel():
        raise ValueError("x and y must have the same length")
    n = x.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=x.device)
    _require(out, "out")
    st = _lib.lib().boys_pairwise(x.data_ptr(), y.data_ptr(), n, c.data_ptr(), c.numel() - 1, out.data_ptr(),
                                  _stream_handle(x, stream))
    _lib.check("boys_pairwise", st)
    return out


# ----------------------------------------------------------------- ragged

PLAN_AUTOTUNE = 1
PLAN_FORCE_CONFIG = 2


def ragged_layout(seg_off: torch.Tensor, seg_kmax: torch.Tensor):
    """Packed output layout of a ragged batch: out_off[s] = sum_{r<s} (kmax_r+1)*len_r.
    Returns (out_off int64 [nseg], total output elements)."""
    lens = seg_off[1:] - seg_off[:-1]
    sizes = (seg_kmax.to(torch.int64) + 1) * lens
    ends = torch.cumsum(sizes, 0)
    out_off = (ends - sizes).contiguous()
    total = int(ends[-1].item()) if ends.numel() else 0
    return out_off, total


def _ragged_args(x, seg_off, seg_kmax):
    _require(x, "x")
    _require(seg_off, "seg_off", torch.int64)
    _require(seg_kmax, "seg_kmax", torch.int32)
    x = x.contiguous().view(-1)
    seg_off = seg_off.contiguous().view(-1)
    seg_kmax = seg_kmax.contiguous().view(-1)
    if seg_off.numel() != seg_kmax.numel() + 1:
        raise ValueError("seg_off must have nseg+1 entries")
    return x, seg_off, seg_kmax


def boys_eval_ragged(x, seg_off, seg_kmax, out=None, out_off=None, workspace=None, stream=None):
    """All segments of a ragged batch, without a plan.  Returns (out, out_off):
    segment s's F_k(x[seg_off[s]+j]) is at out[out_off[s] + k*len_s + j].
    Without ``workspace`` one of boys_ragged_workspace_size_grouped bytes is
    allocated, which selects the kmax-grouped launches; a 256-byte workspace
    selects the single persistent launch."""
    x, seg_off, seg_kmax = _ragged_args(x, seg_off, seg_kmax)
    nseg = seg_kmax.numel()
    if out_off is None:
        out_off, total_out = ragged_layout(seg_off, seg_kmax)
    else:
        _require(out_off, "out_off", torch.int64)
        total_out = None
    if out is None:
        if total_out is None:
            raise ValueError("give out together with out_off")
        out = torch.empty(max(total_out, 1), dtype=torch.float64, device=x.device)
    _require(out, "out")
    L = _lib.lib()
    wsb = L.boys_ragged_workspace_size_grouped(nseg, x.numel())
    if workspace is None:
        workspace = torch.empty(wsb, dtype=torch.uint8, device=x.device)
    st = L.boys_eval_ragged(x.data_ptr(), seg_off.data_ptr(), seg_kmax.data_ptr(), nseg, out.data_ptr(),
                            out_off.data_ptr(), workspace.data_ptr(), workspace.numel(),
                            _stream_handle(x, stream))
    _lib.check("boys_eval_ragged", st)
    return out, out_off


def boys_eval_ragged_noalloc(x, seg_off, seg_kmax, out=None, out_off=None, stream=None):
    """The same batch as boys_eval_ragged through boys_eval_ragged_noalloc:
    no workspace, and the library allocates nothing (its scratch is a static
    array shared by every call on the device, so calls must not overlap on
    the GPU).  ``out`` and ``out_off`` are created here only when not given.
    Returns (out, out_off)."""
    x, seg_off, seg_kmax = _ragged_args(x, seg_off, seg_kmax)
    nseg = seg_kmax.numel()
    if out_off is None:
        out_off, total_out = ragged_layout(seg_off, seg_kmax)
    else:
        _require(out_off, "out_off", torch.int64)
        total_out = None
    if out is None:
        if total_out is None:
            raise ValueError("give out together with out_off")
        out = torch.empty(max(total_out, 1), dtype=torch.float64, device=x.device)
    _require(out, "out")
    st = _lib.lib().boys_eval_ragged_noalloc(x.data_ptr(), seg_off.data_ptr(), seg_kmax.data_ptr(), nseg,
                                             out.data_ptr(), out_off.data_ptr(), _stream_handle(x, stream))
    _lib.check("boys_eval_ragged_noalloc", st)
    return out, out_off


def ragged_noalloc_status(device=None, stream=None) -> bool:
    """True if the latest boys_eval_ragged_noalloc call on the current device
    met a kmax outside [0, 32] (synchronises the stream)."""
    with torch.cuda.device(device if device is not None else torch.cuda.current_device()):
        hs = int(stream.cuda_stream) if stream is not None else int(torch.cuda.current_stream().cuda_stream)
        flag = ctypes.c_int(0)
        st = _lib.lib().boys_ragged_noalloc_status(ctypes.byref(flag), hs)
    _lib.check("boys_ragged_noalloc_status", st)
    return bool(flag.value)


def ragged_status(workspace: torch.Tensor, stream=None) -> bool:
    """True if the last ragged launch on ``workspace`` met a kmax outside [0, 32]."""
    flag = ctypes.c_int(0)
    st = _lib.lib().boys_ragged_status(workspace.data_ptr(), ctypes.byref(flag), _stream_handle(workspace, stream))
    _lib.check("boys_ragged_status", st)
    return bool(flag.value)


class RaggedPlan:
    """A ragged batch bound to its buffers, with an autotuned launch shape and a
    captured CUDA graph (workspace reset + persistent kernel, or one kernel per
    kmax group as parallel branches: ``config()["waves"] == 0``).  ``launch()``
    replays the graph on the current stream.  The tensors are kept alive by
    the plan."""

    def __init__(self, x, seg_off, seg_kmax, out=None, out_off=None, autotune=True, force_config=False):
        x, seg_off, seg_kmax = _ragged_args(x, seg_off, seg_kmax)
        if out_off is None:
            out_off, total_out = ragged_layout(seg_off, seg_kmax)
            if out is None:
                out = torch.empty(max(total_out, 1), dtype=torch.float64, device=x.device)
        _require(out, "out")
        torch.cuda.synchronize(x.device)
        self._keep = (x, seg_off, seg_kmax, out, out_off)
        self.out, self.out_off = out, out_off
        flags = (PLAN_AUTOTUNE if autotune else 0) | (PLAN_FORCE_CONFIG if force_config else 0)
        h = ctypes.c_void_p()
        st = _lib.lib().boys_ragged_plan_create(x.data_ptr(), seg_off.data_ptr(), seg_kmax.data_ptr(),
                                                seg_kmax.numel(), out.data_ptr(), out_off.data_ptr(), flags,
                                                ctypes.byref(h))
        _lib.check("boys_ragged_plan_create", st)
        self._h = h
        self.device = x.device

    def launch(self, stream=None):
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        st = _lib.lib().boys_ragged_plan_launch(self._h, int(s.cuda_stream))
        _lib.check("boys_ragged_plan_launch", st)
        return self.out

    def config(self):
        b, x, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        st = _lib.lib().boys_ragged_plan_config(self._h, ctypes.byref(b), ctypes.byref(x), ctypes.byref(w))
        _lib.check("boys_ragged_plan_config", st)
        return {"block": b.value, "xpt": x.value, "waves": w.value}

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().boys_ragged_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
