"""torch-facing wrappers of the libboys entry points (argument marshalling only).

Tensors must live on a CUDA device; work is enqueued on the current torch
stream of that device (or ``stream``) and is asynchronous like any torch op.
"""
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
