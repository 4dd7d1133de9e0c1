"""Seeded synthetic inputs for the Boys-function workloads.

This module holds only random-number generation and the shapes of the
workloads; none of the method's arithmetic.  Tests feed the same arrays to
the CUDA library and to the oracle; the bench uses them as resident inputs.

Generator: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-style: output i of a stream
with key s is mix64(s + (i + 1) * GAMMA), GAMMA = 0x9e3779b97f4a7c15, with
Stafford's variant-13 finaliser.  Doubles in [0, 1) take the top 53 bits.
Streams inside one workload get keys mix64(seed * 2^16 + stream).

Workloads (argument distributions shaped like electron-repulsion-integral
arguments; names give their sizes):

* ``mixture_c1``   90% log-uniform on [1e-8, 1e3], 5% exact zeros, 5% within
                   +-1e-12 of the region boundaries x0 and x1 (half each,
                   including the boundaries themselves and their neighbouring
                   doubles); used at N = 65536 with kmax = 8, and as the x
                   law of the ragged and FP32-tier workloads.
* ``mixture_c2``   40% log-uniform on [1e-12, 1e2], 40% uniform on [0, 60],
                   20% uniform on [60, 1e4]; N = 2^26 with kmax = 32; rho for
                   the fused consumer uniform on [0.1, 10].
* ``ragged_c3``    4096 segments, lengths log-uniform on [32, 65536],
                   kmax_s = la+lb+lc+ld with each l drawn from
                   {0: .40, 1: .30, 2: .20, 3: .08, 4: .02}; x per segment
                   from ``mixture_c1``.
* ``grad_c5``      N = 2^24 x log-uniform on [1e-10, 1e3]; upstream
                   gradients g_k ~ N(0, 1) (Box-Muller), [17][N].
* ``pairwise_alg2`` the paper's benchmark inputs (Section III): x ~ U[0, 30],
                   y, c ~ N(0, 1); N = 2^19 in the paper.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Region boundaries printed in the paper's Appendix D (x_0, x_1 for
# eps_tol = 5e-14, kmax = 32).  Used here only to place test arguments at and
# around the boundaries.
X0_PRINTED = 11.899848152108484
X1_PRINTED = 28.989337738820740


def mix64(z):
    """splitmix64 finaliser on a uint64 numpy array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    return mix64(np.array([(seed << 16) + stream], dtype=np.uint64))[0]


def raw64(key, n: int, start: int = 0):
    """Outputs start..start+n-1 of the splitmix64 stream with state ``key``."""
    with np.errstate(over="ignore"):
        ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        ctr *= GAMMA
        ctr += np.uint64(key)
    return mix64(ctr)


def uniform01(key, n: int, start: int = 0):
    """Doubles in [0, 1) from the top 53 bits."""
    return (raw64(key, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def log_uniform(u, lo: float, hi: float):
    return np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))


def _boundary_points(key, n: int):
    """n arguments within +-1e-12 of x0 and x1 (half each); the first slots of
    each half are the boundary itself and its nearest doubles."""
    out = np.empty(n)
    u = uniform01(key, n)
    half = n // 2
    for j, (b, lo, hi) in enumerate(((X0_PRINTED, 0, half), (X1_PRINTED, half, n))):
        m = hi - lo
        vals = b + (2.0 * u[lo:hi] - 1.0) * 1e-12
        exact = [b, np.nextafter(b, 0.0), np.nextafter(b, np.inf),
                 np.nextafter(np.nextafter(b, 0.0), 0.0), np.nextafter(np.nextafter(b, np.inf), np.inf)]
        for i, v in enumerate(exact[:m]):
            vals[i] = v
        out[lo:hi] = vals
    return out


def mixture_c1(n: int = 65536, seed: int = 0):
    """The kmax=8 parity mixture (see module docstring); exact category counts,
    positions shuffled by a seeded permutation."""
    n_zero = int(round(0.05 * n))
    n_bnd = int(round(0.05 * n))
    n_log = n - n_zero - n_bnd
    x = np.empty(n)
    x[:n_log] = log_uniform(uniform01(stream_key(seed, 1), n_log), 1e-8, 1e3)
    x[n_log:n_log + n_zero] = 0.0
    x[n_log + n_zero:] = _boundary_points(stream_key(seed, 2), n_bnd)
    perm = np.argsort(raw64(stream_key(seed, 3), n), kind="stable")
    return np.ascontiguousarray(x[perm])


def mixture_c2(n: int = 1 << 26, seed: int = 1, start: int = 0):
    """The kmax=32 headline mixture: per-element category from one uniform.
    Elements start..start+n-1 of the stream, so that consecutive ranges (one
    per GPU) partition one global workload."""
    c = uniform01(stream_key(seed, 1), n, start)
    u = uniform01(stream_key(seed, 2), n, start)
    x = np.where(c < 0.4, log_uniform(u, 1e-12, 1e2),
                 np.where(c < 0.8, 60.0 * u, 60.0 + (1e4 - 60.0) * u))
    return np.ascontiguousarray(x)


def rho_c2(n: int = 1 << 26, seed: int = 2):
    """rho ~ U[0.1, 10] for the fused consumer sum_k (-2 rho)^k F_k."""
    return 0.1 + 9.9 * uniform01(stream_key(seed, 1), n)


def ragged_c3(nseg: int = 4096, seed: int = 3, max_len: int = 65536, min_len: int = 32):
    """Returns (x, seg_off[int64, nseg+1], seg_kmax[int32, nseg])."""
    u = uniform01(stream_key(seed, 1), nseg)
    lens = np.floor(log_uniform(u, min_len, max_len + 1)).astype(np.int64)
    lens = np.clip(lens, min_len, max_len)
    probs = np.array([0.40, 0.30, 0.20, 0.08, 0.02])
    cdf = np.cumsum(probs)
    ls = np.searchsorted(cdf, uniform01(stream_key(seed, 2), 4 * nseg) * cdf[-1], side="right")
    ls = np.minimum(ls, 4).reshape(nseg, 4)
    seg_kmax = ls.sum(axis=1).astype(np.int32)
    seg_off = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(lens, out=seg_off[1:])
    x = mixture_c1(int(seg_off[-1]), seed=seed * 1000 + 7)
    return x, seg_off, seg_kmax


def grad_c5(n: int = 1 << 24, kmax: int = 16, seed: int = 5, gseed: int = 6):
    """Returns (x, g[kmax+1][n])."""
    x = log_uniform(uniform01(stream_key(seed, 1), n), 1e-10, 1e3)
    g = normal(stream_key(gseed, 1), (kmax + 1) * n).reshape(kmax + 1, n)
    return np.ascontiguousarray(x), np.ascontiguousarray(g)


def normal(key, n: int):
    """Standard normals by Box-Muller from pairs of uniforms."""
    m = (n + 1) // 2
    u1 = uniform01(key, m)
    u2 = uniform01(key, m, start=m)
    r = np.sqrt(-2.0 * np.log1p(-u1))
    t = 2.0 * np.pi * u2
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(t)
    z[1::2] = r * np.sin(t)
    return z[:n]


def small_parity_set(seed: int = 11):
    """Edge arguments every parity test includes: zeros, both boundaries and
    their neighbours, tiny and huge values."""
    pts = [0.0, -0.0, 5e-324, 1e-300, 1e-16, 1e-8, 0.5, 1.0, 2.0, 11.0, 12.0, 28.0, 29.0,
           30.0, 60.0, 1e3, 1e4, 1e6, 1e15, 1.7e308]
    for b in (X0_PRINTED, X1_PRINTED):
        v = b
        for _ in range(3):
            v = np.nextafter(v, 0.0)
        for _ in range(7):
            pts.append(float(v))
            v = np.nextafter(v, np.inf)
    u = uniform01(stream_key(seed, 1), 64)
    pts.extend(list(log_uniform(u, 1e-12, 1e4)))
    return np.array(pts)


def pairwise_alg2(n: int = 1 << 17, k: int = 12, seed: int = 8, sort: bool = True):
    """The paper's benchmark inputs (Section III): x uniform on [0, 30], y and
    c standard normal.  Returns (x, y, c); with ``sort`` the x are ascending
    (y drawn per sorted position, so the set of pairs is unchanged in law)."""
    x = 30.0 * uniform01(stream_key(seed, 1), n)
    if sort:
        x = np.sort(x)
    y = normal(stream_key(seed, 2), n)
    c = normal(stream_key(seed, 3), k + 1)
    return np.ascontiguousarray(x), np.ascontiguousarray(y), np.ascontiguousarray(c)
