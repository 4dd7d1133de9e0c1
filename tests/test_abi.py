"""libboys loads, exports every symbol include/boys.h declares, and rejects bad
arguments synchronously without touching a GPU (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_2512_10059_gb300 import _lib, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "boys.h")

FAKE = 0x10000  # never dereferenced: every call below fails its argument checks first


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(boys_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert "boys_eval" in names
    for name in names:
        assert hasattr(L, name), f"{name} declared in include/boys.h but not exported"


def test_status_strings(L):
    assert L.boys_status_string(0) == b"BOYS_OK"
    assert L.boys_status_string(2) == b"BOYS_ERR_KMAX"
    assert L.boys_status_string(99) == b"BOYS_ERR_UNKNOWN"
    assert L.boys_kmax_limit() == 32
    assert L.boys_version() >= 100


def test_eval_argument_errors(L):
    assert L.boys_eval(FAKE, 10, 33, FAKE, 10, None) == 2
    assert L.boys_eval(FAKE, 10, -1, FAKE, 10, None) == 2
    assert L.boys_eval(FAKE, -1, 4, FAKE, 10, None) == 1
    assert L.boys_eval(FAKE, 10, 4, FAKE, 9, None) == 1
    assert L.boys_eval(None, 10, 4, FAKE, 10, None) == 1
    assert L.boys_eval(FAKE, 10, 4, None, 10, None) == 1
    assert L.boys_eval(FAKE + 4, 10, 4, FAKE, 10, None) == 3
    assert b"x/out" in L.boys_last_error()
    assert L.boys_eval(FAKE, 1, 32, FAKE, (1 << 62), None) == 1  # (kmax+1)*ld overflows
    assert L.boys_eval(None, 0, 4, None, 0, None) == 0  # n == 0 is a no-op


def test_fused_argument_errors(L):
    assert L.boys_eval_fused(FAKE, FAKE, 10, 33, FAKE, None) == 2
    assert L.boys_eval_fused(FAKE, None, 10, 3, FAKE, None) == 1
    assert L.boys_eval_fused(FAKE, FAKE + 2, 10, 3, FAKE, None) == 3
    assert L.boys_eval_fused(None, None, 0, 3, None, None) == 0


def test_grad_argument_errors(L):
    assert L.boys_grad(FAKE, 10, 32, FAKE, 10, FAKE, None) == 2  # needs F_{kmax+1} <= F_32
    assert L.boys_grad(FAKE, 10, 4, FAKE, 9, FAKE, None) == 1
    assert L.boys_grad(FAKE, 10, 4, None, 10, FAKE, None) == 1
    assert L.boys_grad(None, 0, 4, None, 0, None, None) == 0


def test_ragged_argument_errors(L):
    import ctypes
    assert L.boys_ragged_workspace_size() == 256
    assert L.boys_ragged_workspace_size_grouped(-1, 0) == 0
    assert L.boys_ragged_workspace_size_grouped(0, 0) == 528
    assert L.boys_ragged_workspace_size_grouped(4096, 1 << 25) == 512 + 16 * ((1 << 25) // 128 + 4097)
    assert L.boys_eval_ragged(FAKE, FAKE, FAKE, -1, FAKE, FAKE, FAKE, 256, None) == 1
    assert L.boys_eval_ragged(None, None, None, 0, None, None, None, 0, None) == 0
    assert L.boys_eval_ragged(FAKE, None, FAKE, 3, FAKE, FAKE, FAKE, 256, None) == 1
    assert L.boys_eval_ragged(FAKE, FAKE, FAKE, 3, FAKE, FAKE, FAKE, 255, None) == 1
    assert L.boys_eval_ragged(FAKE, FAKE, FAKE, 3, FAKE, FAKE, None, 256, None) == 1
    assert L.boys_eval_ragged(FAKE, FAKE, FAKE + 2, 3, FAKE, FAKE, FAKE, 256, None) == 3
    assert L.boys_eval_ragged(FAKE, FAKE, FAKE, 3, FAKE, FAKE, FAKE + 8, 256, None) == 3
    h = ctypes.c_void_p()
    assert L.boys_ragged_plan_create(FAKE, FAKE, FAKE, 0, FAKE, FAKE, 0, ctypes.byref(h)) == 1
    assert L.boys_ragged_plan_create(FAKE, FAKE, FAKE, 3, FAKE, FAKE, 0, None) == 1
    assert L.boys_ragged_plan_launch(None, None) == 1
    L.boys_ragged_plan_destroy(None)


def test_every_declared_function_has_ctypes_signature(L):
    """Without argtypes ctypes passes Python ints as 32-bit C ints, silently
    truncating 64-bit device pointers: every entry point must be declared."""
    for name in declared_functions():
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature in _lib"
        assert getattr(L, name).argtypes is not None or _lib.SIGNATURES[name][1] == []


def test_eval_host_argument_errors(L):
    assert L.boys_eval_host(FAKE, 10, 33, FAKE, 10, None) == 2
    assert L.boys_eval_host(FAKE, 10, 4, FAKE, 9, None) == 1
    assert L.boys_eval_host(None, 10, 4, FAKE, 10, None) == 1
    assert L.boys_eval_host(None, 0, 4, None, 0, None) == 0


def test_pairwise_argument_errors(L):
    assert L.boys_pairwise(FAKE, FAKE, 10, FAKE, 33, FAKE, None) == 2
    assert L.boys_pairwise(FAKE, FAKE, -1, FAKE, 3, FAKE, None) == 1
    assert L.boys_pairwise(FAKE, None, 10, FAKE, 3, FAKE, None) == 1
    assert L.boys_pairwise(None, None, 0, None, 3, None, None) == 0
