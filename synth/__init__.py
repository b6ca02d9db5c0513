"""Seeded synthetic inputs shared by the tests, ``bench.py`` and ``smoke()``.

This module holds no arithmetic of the expression method itself: it only
draws numbers.  Both the CUDA path and the CPU oracle receive the arrays it
returns, so neither side generates its own inputs.

Generator
---------
Counter-based splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; constants as in Vigna's
public-domain ``splitmix64.c``).  Element ``i`` of stream ``s`` under seed
``seed`` is the ``(i+1)``-th output of a splitmix64 whose state starts at
``seed * GOLDEN + s * STREAM_MUL`` (mod 2^64):

    z  = seed*GOLDEN + s*STREAM_MUL + (i+1)*GOLDEN
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9
    z ^= z >> 27; z *= 0x94D049BB133111EB
    z ^= z >> 31
    u  = (z >> 11) * 2^-53            in [0, 1)
    x  = 2u - 1                       in [-1, 1)

``i`` is the column-major linear index, so a matrix is the same whatever
its storage order in memory.  Values are produced in FP64 and rounded to
the storage dtype (FP32 by round-to-nearest, BF16 by round-to-nearest-even
from FP32); the oracle then sees exactly the stored values.

The workloads are random dense matrices with entries uniform in [-1, 1]:
the paper fills its benchmark matrices with uniform random values
(Sec. III, Fig. 2's ``fill::randu``).
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
STREAM_MUL = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream ids of the named operands of the benchmark expressions.
STREAMS = {"A": 1, "B": 2, "C": 3, "D": 4, "v": 5, "x": 6, "b": 7,
           "Q": 8, "Q2": 9, "E": 10}


def _mix(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * _M1
    z = z ^ (z >> np.uint64(27))
    z = z * _M2
    z = z ^ (z >> np.uint64(31))
    return z


def raw_u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of stream ``stream`` as uint64."""
    with np.errstate(over="ignore"):
        base = (np.uint64(seed % 2**64) * GOLDEN
                + np.uint64(stream % 2**64) * STREAM_MUL)
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(base + idx * GOLDEN)


def uniform_flat(seed: int, stream: int, count: int, start: int = 0,
                 chunk: int = 1 << 23) -> np.ndarray:
    """``count`` FP64 values uniform in [-1, 1) (column-major order)."""
    out = np.empty(count, dtype=np.float64)
    scale = 2.0 ** -53
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        z = raw_u64(seed, stream, start + s, e - s)
        out[s:e] = (z >> np.uint64(11)).astype(np.float64) * scale * 2.0 - 1.0
    return out


def round_bf16(x32: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (ties to even); returns FP32
    arrays holding BF16-representable values."""
    x32 = np.ascontiguousarray(x32, dtype=np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).reshape(x32.shape)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """uint16 BF16 bit patterns of FP32 values that are BF16-representable."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    return (x.view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def matrix(seed: int, name_or_stream, rows: int, cols: int,
           dtype: str = "f64") -> np.ndarray:
    """A rows x cols matrix, Fortran (column-major) order, uniform [-1, 1).

    ``dtype`` is the storage type: "f64", "f32" or "bf16" (the latter
    returned as FP32 arrays holding BF16 values)."""
    stream = STREAMS[name_or_stream] if isinstance(name_or_stream, str) else int(name_or_stream)
    v = uniform_flat(seed, stream, rows * cols)
    return cast(v.reshape((rows, cols), order="F"), dtype)


def cast(x: np.ndarray, dtype: str) -> np.ndarray:
    if dtype == "f64":
        return np.asfortranarray(x, dtype=np.float64)
    if dtype == "f32":
        return np.asfortranarray(x.astype(np.float32))
    if dtype == "bf16":
        return np.asfortranarray(round_bf16(x.astype(np.float32)))
    raise ValueError(dtype)


def small_ints(seed: int, stream: int, rows: int, cols: int, lo: int = -4,
               hi: int = 4) -> np.ndarray:
    """Integer-valued FP64 matrix with entries in [lo, hi]; sums and products
    of such values are exact in FP64 at the sizes the tests use."""
    z = raw_u64(seed, stream, 0, rows * cols)
    span = np.uint64(hi - lo + 1)
    v = (z % span).astype(np.int64) + lo
    return np.asfortranarray(v.reshape((rows, cols), order="F").astype(np.float64))


# ---------------------------------------------------------------------------
# Structured inputs
# ---------------------------------------------------------------------------

def gaussian_flat(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Standard normal values by the Box-Muller transform of pairs of
    uniforms from the same counter stream."""
    n2 = (count + 1) // 2
    z = raw_u64(seed, stream, 2 * start, 2 * n2)
    u = ((z >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    g = np.empty(2 * n2)
    g[0::2] = r * np.cos(2.0 * math.pi * u2)
    g[1::2] = r * np.sin(2.0 * math.pi * u2)
    return g[:count]


def householder_vectors(seed: int, stream: int, n: int, r: int = 8) -> np.ndarray:
    """r unit Gaussian vectors of length n (columns), the reflectors of an
    orthogonal Q = H_1 ... H_r with H_k = I - 2 u_k u_k^T."""
    U = gaussian_flat(seed, stream, n * r).reshape((n, r), order="F")
    U /= np.linalg.norm(U, axis=0, keepdims=True)
    return np.asfortranarray(U)


def _apply_reflectors_left(U: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Q M with Q = H_1 ... H_r: apply H_r first, H_1 last."""
    for k in range(U.shape[1] - 1, -1, -1):
        u = U[:, k:k + 1]
        M = M - 2.0 * u @ (u.T @ M)
    return M


def geometric_spectrum(n: int, cond: float = 1e6) -> np.ndarray:
    """s_i = cond^(i/(n-1)), i = 0..n-1: 1 .. cond, geometric."""
    if n == 1:
        return np.ones(1)
    return cond ** (np.arange(n, dtype=np.float64) / (n - 1))


def conditioned_matrix(seed: int, n: int, cond: float = 1e6,
                       symmetric: bool = True, r: int = 8) -> np.ndarray:
    """A = Q1 diag(s) Q2^T in FP64 with s geometric from 1 to ``cond``.

    symmetric=True uses Q2 = Q1 (an SPD matrix whose 2-norm condition
    number is exactly ``cond`` up to rounding); symmetric=False draws an
    independent Q2 so that partial pivoting has rows to swap."""
    U1 = householder_vectors(seed, STREAMS["Q"], n, r)
    U2 = U1 if symmetric else householder_vectors(seed, STREAMS["Q2"], n, r)
    s = geometric_spectrum(n, cond)
    # Q1 diag(s) Q2^T = Q1 (Q2 diag(s))^T
    M = _apply_reflectors_left(U2, np.diag(s))       # Q2 diag(s)
    M = _apply_reflectors_left(U1, np.ascontiguousarray(M.T))  # Q1 (Q2 diag(s))^T
    if symmetric:
        M = 0.5 * (M + M.T)
    return np.asfortranarray(M)


def log_uniform_ints(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers drawn log-uniform in [lo, hi] (rounded, clipped)."""
    z = raw_u64(seed, stream, 0, count)
    u = (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    v = np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    return np.clip(np.rint(v), lo, hi).astype(np.int64)


def band_matrix(seed: int, stream: int, n: int, kl: int, ku: int, dtype: str = "f64",
                diag_shift: float = 0.0, zero_diag_every: int = 0) -> np.ndarray:
    """An n x n matrix whose entries on diagonals -kl .. ku are uniform
    [-1, 1) (the main diagonal shifted by ``diag_shift``) and zero elsewhere.
    With ``zero_diag_every`` = k > 0, every k-th main-diagonal entry is set
    to zero, so elimination without row exchanges would break down there."""
    v = uniform_flat(seed, stream, n * n).reshape((n, n), order="F")
    i, j = np.indices((n, n))
    a = np.where((i - j <= kl) & (j - i <= ku), v, 0.0)
    a[np.arange(n), np.arange(n)] += diag_shift
    if zero_diag_every > 0:
        z = np.arange(0, n, zero_diag_every)
        a[z, z] = 0.0
    return cast(a, dtype)
