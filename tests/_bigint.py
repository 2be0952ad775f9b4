"""Big-integer helpers for pinning the oracle (Python ints, no oracle code)."""
from __future__ import annotations

from functools import reduce

import numpy as np


def prod(xs) -> int:
    return reduce(lambda a, b: a * b, (int(x) for x in xs), 1)


def crt(residues, primes) -> int:
    """Textbook CRT: the unique X in [0, prod(primes)) with X = r_i mod p_i."""
    M = prod(primes)
    X = 0
    for r, p in zip(residues, primes):
        Mi = M // p
        X += int(r) * Mi * pow(Mi, -1, p)
    return X % M


def crt_poly(towers, primes) -> list[int]:
    """Per-coefficient CRT of a [towers][N] residue matrix."""
    towers = [[int(v) for v in row] for row in towers]
    N = len(towers[0])
    return [crt([row[n] for row in towers], primes) for n in range(N)]


def centre(x: int, M: int) -> int:
    x %= M
    return x - M if x > M // 2 else x


def mulmod_arr(a, b, q: int) -> np.ndarray:
    return ((np.asarray(a).astype(object) * np.asarray(b).astype(object)) % q).astype(np.uint64)


def negacyclic_schoolbook(a, b) -> list[int]:
    """a*b in Z[X]/(X^N+1) over the integers (lists of Python ints)."""
    N = len(a)
    out = [0] * N
    for i, ai in enumerate(a):
        if ai == 0:
            continue
        for j, bj in enumerate(b):
            k = i + j
            if k < N:
                out[k] += ai * bj
            else:
                out[k - N] -= ai * bj
    return out


def brv(k: int, bits: int) -> int:
    return int(format(k, f"0{bits}b")[::-1], 2) if bits else 0
