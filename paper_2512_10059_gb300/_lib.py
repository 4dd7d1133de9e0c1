"""ctypes binding of libboys.so: argument marshalling only.

The library must have been built in-tree (``paper_2512_10059_gb300.build``);
there is no fallback implementation, so a missing or unloadable library
raises immediately.
"""
import ctypes
import os

from . import build as _build

_c_double_p = ctypes.c_void_p  # device pointers travel as plain addresses
_lib = None


class BoysError(RuntimeError):
    """A libboys entry point returned a non-zero boys_status."""

    def __init__(self, fn: str, status: int, text: str):
        super().__init__(f"{fn} -> {status} ({text})")
        self.status = status


SIGNATURES = {}


def _declare(lib):
    i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    sig = {
        "boys_status_string": (ctypes.c_char_p, [i32]),
        "boys_last_error": (ctypes.c_char_p, []),
        "boys_version": (i32, []),
        "boys_kmax_limit": (i32, []),
        "boys_diag_math": (i32, [i32, vp, vp, i64, vp, vp]),
        "boys_eval": (i32, [vp, i64, i32, vp, i64, vp]),
        "boys_eval_host": (i32, [vp, i64, i32, vp, i64, vp]),
        "boys_eval_fused": (i32, [vp, vp, i64, i32, vp, vp]),
        "boys_grad": (i32, [vp, i64, i32, vp, i64, vp, vp]),
        "boys_eval_f32": (i32, [vp, i64, i32, vp, i64, vp]),
        "boys_ragged_workspace_size": (ctypes.c_size_t, []),
        "boys_ragged_workspace_size_grouped": (ctypes.c_size_t, [i32, i64]),
        "boys_eval_ragged": (i32, [vp, vp, vp, i32, vp, vp, vp, ctypes.c_size_t, vp]),
        "boys_ragged_status": (i32, [vp, ctypes.POINTER(i32), vp]),
        "boys_ragged_plan_create": (i32, [vp, vp, vp, i32, vp, vp, i32, ctypes.POINTER(vp)]),
        "boys_ragged_plan_launch": (i32, [vp, vp]),
        "boys_ragged_plan_config": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "boys_ragged_plan_destroy": (None, [vp]),
        "boys_eval_ragged_noalloc": (i32, [vp, vp, vp, i32, vp, vp, vp]),
        "boys_ragged_noalloc_status": (i32, [ctypes.POINTER(i32), vp]),
        "boys_pairwise": (i32, [vp, vp, i64, vp, i32, vp, vp]),
    }
    SIGNATURES.update(sig)
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


def lib():
    """The loaded libboys (loaded once per process)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"libboys.so is not built ({path}); run __graft_entry__.build() "
                              "or python -m paper_2512_10059_gb300.build")
        l = ctypes.CDLL(path)
        _declare(l)
        _lib = l
    return _lib


def path() -> str:
    return _build.LIB


def check(fn: str, status: int):
    if status != 0:
        l = lib()
        raise BoysError(fn, status, l.boys_last_error().decode() or l.boys_status_string(status).decode())
