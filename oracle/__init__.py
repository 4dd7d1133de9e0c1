"""Binary128 Boys-function oracle — TEST INFRASTRUCTURE, not the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` leg may import this package.  It
evaluates the definition F_k(x) = int_0^1 t^{2k} exp(-x t^2) dt (paper,
Eq. 3) in IEEE binary128 (see ``boys_oracle.c`` for the two routes and the
passages they follow) and shares nothing with the CUDA library.

Every value comes back as an unevaluated double-double ``(hi, lo)``:
``hi`` is the correctly rounded double, ``lo`` the remainder, so
``abs((y - hi) - lo)`` measures the error of a double ``y`` to ~1e-32
relative.
"""
import ctypes

import numpy as np

from . import build as _build

_c_double_p = ctypes.POINTER(ctypes.c_double)


def _ptr(a):
    return a.ctypes.data_as(_c_double_p)


class OracleLib:
    """ctypes view of one compiled oracle library (the real one, or a test's
    deliberately broken copy)."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        lib.oracle_boys_branch.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                           _c_double_p, _c_double_p]
        lib.oracle_boys_batch.argtypes = [_c_double_p, ctypes.c_int64, ctypes.c_int,
                                          _c_double_p, _c_double_p, ctypes.c_int64, ctypes.c_int]
        lib.oracle_fused_batch.argtypes = [_c_double_p, _c_double_p, ctypes.c_int64, ctypes.c_int,
                                           _c_double_p, _c_double_p, ctypes.c_int]
        lib.oracle_grad_batch.argtypes = [_c_double_p, ctypes.c_int64, ctypes.c_int,
                                          _c_double_p, ctypes.c_int64,
                                          _c_double_p, _c_double_p, ctypes.c_int]
        lib.oracle_pairwise_rows.argtypes = [_c_double_p, _c_double_p, ctypes.c_int64, _c_double_p, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, _c_double_p, _c_double_p,
                                             ctypes.c_int]
        lib.oracle_pairwise_rows.restype = ctypes.c_int
        lib.oracle_pairwise.argtypes = [_c_double_p, _c_double_p, ctypes.c_int64, _c_double_p, ctypes.c_int,
                                        _c_double_p, _c_double_p, ctypes.c_int]
        for name in ("oracle_boys_branch", "oracle_boys_batch", "oracle_fused_batch",
                     "oracle_grad_batch", "oracle_kmax_limit", "oracle_mantissa_bits",
                     "oracle_max_threads", "oracle_pairwise"):
            getattr(lib, name).restype = ctypes.c_int
        self._lib = lib
        self.path = path

    def kmax_limit(self) -> int:
        return self._lib.oracle_kmax_limit()

    def mantissa_bits(self) -> int:
        return self._lib.oracle_mantissa_bits()

    def max_threads(self) -> int:
        return self._lib.oracle_max_threads()

    def boys(self, x, kmax: int, nthreads: int = 0):
        """F_0..F_kmax at every x: returns (hi, lo), each float64 [kmax+1][n]."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
        n = x.size
        hi = np.empty((kmax + 1, n), dtype=np.float64)
        lo = np.empty((kmax + 1, n), dtype=np.float64)
        rc = self._lib.oracle_boys_batch(_ptr(x), n, kmax, _ptr(hi), _ptr(lo), n, nthreads)
        if rc != 0:
            raise ValueError(f"oracle_boys_batch rejected kmax={kmax}")
        return hi, lo

    def boys_branch(self, x: float, kmax: int, branch: int):
        """One x through a forced route: 1 = series, 2 = erf + upward identity."""
        hi = np.empty(kmax + 1)
        lo = np.empty(kmax + 1)
        rc = self._lib.oracle_boys_branch(float(x), kmax, branch, _ptr(hi), _ptr(lo))
        if rc != 0:
            raise ValueError(f"oracle_boys_branch rejected kmax={kmax}")
        return hi, lo

    def fused(self, x, rho, kmax: int, nthreads: int = 0):
        """S_i = sum_k (-2 rho_i)^k F_k(x_i) in binary128: returns (hi, lo) [n]."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
        rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).ravel())
        if rho.size != x.size:
            raise ValueError("x and rho differ in length")
        n = x.size
        hi = np.empty(n)
        lo = np.empty(n)
        rc = self._lib.oracle_fused_batch(_ptr(x), _ptr(rho), n, kmax, _ptr(hi), _ptr(lo), nthreads)
        if rc != 0:
            raise ValueError(f"oracle_fused_batch rejected kmax={kmax}")
        return hi, lo

    def grad(self, x, g, kmax: int, nthreads: int = 0):
        """dL/dx_i = -sum_k g[k, i] F_{k+1}(x_i) in binary128: returns (hi, lo) [n]."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
        g = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
        n = x.size
        if g.shape != (kmax + 1, n):
            raise ValueError(f"g must be [{kmax + 1}][{n}], got {g.shape}")
        hi = np.empty(n)
        lo = np.empty(n)
        rc = self._lib.oracle_grad_batch(_ptr(x), n, kmax, _ptr(g), n, _ptr(hi), _ptr(lo), nthreads)
        if rc != 0:
            raise ValueError(f"oracle_grad_batch rejected kmax={kmax}")
        return hi, lo

    def pairwise(self, x, y, c, nthreads: int = 0):
        """z_i = sum_l c_l sum_j F_l(x_i + x_j) y_j in binary128: (hi, lo) [n]."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
        y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).ravel())
        c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).ravel())
        if y.size != x.size:
            raise ValueError("x and y differ in length")
        n = x.size
        hi = np.empty(n)
        lo = np.empty(n)
        rc = self._lib.oracle_pairwise(_ptr(x), _ptr(y), n, _ptr(c), c.size - 1, _ptr(hi), _ptr(lo), nthreads)
        if rc != 0:
            raise ValueError("oracle_pairwise rejected its arguments")
        return hi, lo

    def pairwise_rows(self, x, y, c, rows, nthreads: int = 0):
        """z_i for the given rows only: (hi, lo) [len(rows)]."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
        y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).ravel())
        c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).ravel())
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64).ravel())
        hi = np.empty(rows.size)
        lo = np.empty(rows.size)
        rc = self._lib.oracle_pairwise_rows(_ptr(x), _ptr(y), x.size, _ptr(c), c.size - 1,
                                            rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), rows.size,
                                            _ptr(hi), _ptr(lo), nthreads)
        if rc != 0:
            raise ValueError("oracle_pairwise_rows rejected its arguments")
        return hi, lo


_default = None


def default() -> OracleLib:
    """The oracle built from ``boys_oracle.c`` (compiled on first use)."""
    global _default
    if _default is None:
        _default = OracleLib(_build.build())
    return _default


def boys(x, kmax, nthreads=0):
    return default().boys(x, kmax, nthreads)


def boys_branch(x, kmax, branch):
    return default().boys_branch(x, kmax, branch)


def fused(x, rho, kmax, nthreads=0):
    return default().fused(x, rho, kmax, nthreads)


def grad(x, g, kmax, nthreads=0):
    return default().grad(x, g, kmax, nthreads)


def pairwise(x, y, c, nthreads=0):
    return default().pairwise(x, y, c, nthreads)


def pairwise_rows(x, y, c, rows, nthreads=0):
    return default().pairwise_rows(x, y, c, rows, nthreads)


def kmax_limit():
    return default().kmax_limit()


def mantissa_bits():
    return default().mantissa_bits()


def max_threads():
    return default().max_threads()
