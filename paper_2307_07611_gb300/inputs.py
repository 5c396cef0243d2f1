"""Seeded synthetic inputs shared by the tests, the bench and the oracle's callers.

This module only draws and shapes random numbers; it holds none of the inversion
arithmetic.  Every generator returns a logical matrix as a NumPy array (row-major
NumPy indexing ``a[i, j]`` = row i, column j); how the matrix is laid out in device or
host memory for a call is the caller's business.

Value laws follow the workloads of the paper's numerical section (random non-singular
triangular matrices, Section 6, Table "tab:combrit") made concrete:

* ``tri_lower(n, seed, law="uniform")``: diagonal U[1,2], strict lower U[-1,1]/sqrt(n)
  (the single FP64 n=512 case, the batched blocks and the adjoint batch);
* ``tri_lower(n, seed, law="normal")``: diagonal U[1,2], strict lower N(0,1)/sqrt(n)
  (the FP32 n=8192 case);
* ``general(n, seed)``: N(0,1)/sqrt(n) + 2I (the general n=16384 case);
* integer unit-triangular families whose inverses are small integers (Corollary
  "integer closure", Section 3).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "tri_lower",
    "general",
    "batched_sizes",
    "batched_blocks",
    "adjoint_batch",
    "ones_unit_lower",
    "bidiagonal_unit_lower",
    "level_nilpotent_unit_lower",
    "poison_upper",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def tri_lower(n: int, seed: int = 0, law: str = "uniform", dtype=np.float64,
              rng: np.random.Generator | None = None) -> np.ndarray:
    """Lower-triangular T: diag ~ U[1,2] (drawn first), strict lower ~ law/sqrt(n).

    The upper triangle is exactly zero.  The result is cast to ``dtype`` with
    round-to-nearest from the float64 draw.
    """
    g = _rng(seed) if rng is None else rng
    n = int(n)
    d = g.uniform(1.0, 2.0, n)
    if law == "uniform":
        e = g.uniform(-1.0, 1.0, (n, n))
    elif law == "normal":
        e = g.standard_normal((n, n))
    else:
        raise ValueError(f"unknown law {law!r}")
    if n > 0:
        e *= 1.0 / np.sqrt(n)
    t = np.tril(e, -1)
    t[np.arange(n), np.arange(n)] = d
    return t.astype(dtype)


def general(n: int, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """Dense A = N(0,1)/sqrt(n) + 2I, cast to ``dtype`` with round-to-nearest."""
    g = _rng(seed)
    a = g.standard_normal((n, n))
    if n > 0:
        a *= 1.0 / np.sqrt(n)
    a[np.arange(n), np.arange(n)] += 2.0
    return a.astype(dtype)


def batched_sizes(count: int, seed: int = 0, lo: int = 16, hi: int = 256) -> np.ndarray:
    """Block sizes drawn uniformly from {lo..hi} (inclusive)."""
    return _rng(seed).integers(lo, hi + 1, count)


def batched_blocks(count: int, seed: int = 0, lo: int = 16, hi: int = 256,
                   dtype=np.float32):
    """Sizes, then blocks in index order, all from one generator seeded with ``seed``.

    Each block follows the uniform law with its own sqrt(n_b) scaling.
    """
    g = _rng(seed)
    sizes = g.integers(lo, hi + 1, count)
    blocks = [tri_lower(int(nb), law="uniform", dtype=dtype, rng=g) for nb in sizes]
    return sizes, blocks


def adjoint_batch(batch: int, n: int, seed: int = 0, dtype=np.float32):
    """``batch`` lower-triangular T (uniform law) and cotangents W ~ N(0,1) of the same shape."""
    g = _rng(seed)
    ts = np.stack([tri_lower(n, law="uniform", dtype=dtype, rng=g) for _ in range(batch)])
    ws = g.standard_normal((batch, n, n)).astype(dtype)
    return ts, ws


def ones_unit_lower(n: int, dtype=np.float64) -> np.ndarray:
    """Unit lower-triangular matrix whose every lower entry is 1."""
    return np.tril(np.ones((n, n))).astype(dtype)


def bidiagonal_unit_lower(n: int, seed: int = 0, values=(-1.0, 1.0), dtype=np.float64):
    """Unit lower bidiagonal T with sub-diagonal entries drawn from ``values``.

    Returns (T, b) where b[k] = T[k+1, k].
    """
    g = _rng(seed)
    b = g.choice(np.asarray(values, dtype=np.float64), size=max(n - 1, 0))
    t = np.eye(n)
    if n > 1:
        t[np.arange(1, n), np.arange(n - 1)] = b
    return t.astype(dtype), b


def level_nilpotent_unit_lower(n: int, half: int, seed: int = 0, lo: int = -2, hi: int = 2,
                               dtype=np.float64):
    """T = I + N where N is supported only on the off-diagonal blocks of one split level.

    With split half-size ``half``, pair q covers rows/cols [2*q*half, 2*q*half + 2*half);
    N is non-zero only in rows [2*q*half + half, 2*q*half + 2*half) x
    cols [2*q*half, 2*q*half + half) (clipped to n), with integer entries in [lo, hi].
    Returns (T, N).
    """
    g = _rng(seed)
    nmat = np.zeros((n, n))
    q0 = 0
    while q0 < n:
        r0, r1 = q0 + half, min(q0 + 2 * half, n)
        c0, c1 = q0, min(q0 + half, n)
        if r0 < r1:
            nmat[r0:r1, c0:c1] = g.integers(lo, hi + 1, (r1 - r0, c1 - c0))
        q0 += 2 * half
    return (np.eye(n) + nmat).astype(dtype), nmat.astype(dtype)


def poison_upper(t: np.ndarray, value=np.nan) -> np.ndarray:
    """Copy of a lower-triangular matrix with its strict upper triangle set to ``value``."""
    p = np.array(t, copy=True)
    iu = np.triu_indices(p.shape[0], 1)
    p[iu] = value
    return p
