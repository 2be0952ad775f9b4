"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds none of the key-switching arithmetic: it only draws random
numbers (numpy PCG64, seeded) and arranges them into the shapes of the paper's
workloads (CiFlow Table III parameter sets and the batched / serving mixes).
Primes are passed in by the caller; nothing here computes them.

Recipes:
  * key-switch input d: uniform residues per tower, [towers][N] uint64,
    already in evaluation form (a uniform element is uniform in either form);
  * secret s: ternary, uniform over {-1, 0, 1} per coefficient;
  * target secret s' for rotation keys: s(X^g) for a Galois element g;
  * target secret s' for relinearisation keys: s^2 in Z[X]/(X^N+1);
  * Galois elements: 5^r mod 2N for distinct seeded r in [1, N/2).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0xC1F10


def rng(seed: int) -> np.random.Generator:
    """The seeded generator every input comes from (numpy PCG64)."""
    return np.random.Generator(np.random.PCG64(seed))


def uniform_towers(primes, N: int, seed: int) -> np.ndarray:
    """[len(primes)][N] uint64, row t uniform in [0, primes[t])."""
    g = rng(seed)
    out = np.empty((len(primes), N), dtype=np.uint64)
    for t, q in enumerate(primes):
        out[t] = g.integers(0, int(q), size=N, dtype=np.uint64)
    return out


def ternary_secret(N: int, seed: int) -> np.ndarray:
    """A uniform ternary secret in coefficient form (int8[N])."""
    return rng(seed).integers(-1, 2, size=N, dtype=np.int64).astype(np.int8)


def galois_elements(N: int, count: int, seed: int) -> list[int]:
    """`count` distinct Galois elements 5^r mod 2N, r seeded in [1, N/2)."""
    g = rng(seed)
    rs = g.choice(np.arange(1, N // 2), size=count, replace=False)
    return [pow(5, int(r), 2 * N) for r in rs]


def galois_secret(s: np.ndarray, gal: int) -> np.ndarray:
    """Coefficients of s(X^gal) in Z[X]/(X^N+1): coefficient i moves to
    i*gal mod 2N and changes sign when that index is >= N."""
    N = len(s)
    out = np.zeros(N, dtype=np.int64)
    idx = (np.arange(N, dtype=np.int64) * gal) % (2 * N)
    sign = np.where(idx >= N, -1, 1)
    out[idx % N] = sign * s.astype(np.int64)
    return out


def square_secret(s: np.ndarray) -> np.ndarray:
    """s^2 in Z[X]/(X^N+1) (exact: |coefficients| <= N, computed with a
    float64 FFT of length 2N and rounded)."""
    N = len(s)
    f = np.fft.rfft(s.astype(np.float64), 2 * N)
    full = np.rint(np.fft.irfft(f * f, 2 * N)).astype(np.int64)
    return full[:N] - full[N:]


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process."""
    return np.cumsum(rng(seed).exponential(1.0 / rate_per_s, size=count))
