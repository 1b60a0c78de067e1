"""Seeded synthetic inputs for C = A^t A (random draws only, no product math).

Both the tests / benchmark and the oracle checks take their matrices from
here, so the GPU path and the oracle see the same bytes.  Every generator
uses ``numpy.random.default_rng(seed)`` and draws in a fixed order.

Recipes (the paper measures random square matrices of order 5000 and 10000,
Section 6.2; no dataset is involved):

* ``uniform``      entries i.i.d. U(-1, 1)                 (512 x 384, seed 0)
* ``normal``       entries i.i.d. N(0, 1)                  (paper scale, seed 1)
* ``scaled_cols``  N(0, 1) FP32, columns j = 0 mod 8 x 1e3 (16384 x 8192, seed 2)
* ``batch_shapes`` m log-uniform in [lo, hi], then n log-uniform, rounded to
                   nearest integers                         (512 instances, seed 3)
* ``poisson_arrivals`` exponential gaps at a given rate     (serving, seed 4)
* ``integers`` / ``small_integers`` i.i.d. integers in [-4, 4] (exact-result
                   parity; the latter as int8 for inputs past 2^31 entries)
"""
from __future__ import annotations

import numpy as np


def uniform(m: int, n: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(m, n)).astype(dtype)


def normal(m: int, n: int, seed: int = 1, dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=(m, n)).astype(dtype, copy=False)


def scaled_cols(m: int, n: int, seed: int = 2, scale: float = 1e3, every: int = 8,
                dtype=np.float32) -> np.ndarray:
    A = normal(m, n, seed, dtype=np.float64)
    A[:, ::every] *= scale
    return A.astype(dtype)


def integers(m: int, n: int, seed: int = 5, lo: int = -4, hi: int = 4, dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(m, n)).astype(dtype)


def small_integers(m: int, n: int, seed: int = 6, lo: int = -4, hi: int = 4) -> np.ndarray:
    """Integers in [lo, hi] drawn directly as int8: one byte per entry on the
    host, for inputs of billions of entries (converted on the device)."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(m, n), dtype=np.int8)


def log_uniform_ints(rng, lo: int, hi: int, count: int) -> np.ndarray:
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def batch_shapes(count: int = 512, m_range=(64, 4096), n_range=(32, 1024), seed: int = 3):
    """Shapes of the batched workload: all m first, then all n."""
    rng = np.random.default_rng(seed)
    ms = log_uniform_ints(rng, *m_range, count)
    ns = log_uniform_ints(rng, *n_range, count)
    return rng, list(zip(ms.tolist(), ns.tolist()))


def batch(count: int = 512, m_range=(64, 4096), n_range=(32, 1024), seed: int = 3, dtype=np.float32):
    """Instances of the batched workload: U(-1, 1) entries drawn in instance order."""
    rng, shapes = batch_shapes(count, m_range, n_range, seed)
    mats = [rng.uniform(-1.0, 1.0, size=s).astype(dtype) for s in shapes]
    return mats


def poisson_arrivals(rate: float, duration: float, seed: int = 4) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: exponential gaps at `rate`."""
    rng = np.random.default_rng(seed)
    n_est = int(rate * duration * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_est))
    return t[t < duration]


def serving_pool(pool: int = 256, m_range=(128, 8192), n_range=(64, 2048), seed: int = 4, dtype=np.float32):
    """Request matrices of the serving workload: a pool of N(0, 1) matrices
    with log-uniform shapes, and the generator that continues the stream."""
    rng = np.random.default_rng(seed + 1000)
    ms = log_uniform_ints(rng, *m_range, pool)
    ns = log_uniform_ints(rng, *n_range, pool)
    mats = [rng.standard_normal(size=(int(a), int(b))).astype(dtype) for a, b in zip(ms, ns)]
    return rng, mats
