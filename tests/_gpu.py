"""Shared helpers of the GPU parity tests (library vs oracle on the same seeded inputs)."""
from __future__ import annotations

import functools

import pytest

from oracle import oracle as orc
from paper_2311_01598_gb300 import inputs


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@functools.lru_cache(maxsize=None)
def built_lib():
    from paper_2311_01598_gb300 import build, ks
    build.build()
    return ks


def pair(logN, nq, kp, dnum, bits=54):
    """Library params and oracle context for the same parameter set; the two
    sides pick their primes independently and must agree."""
    ks = built_lib()
    P = ks.Params(logN, nq, kp, dnum, prime_bits=bits)
    C = orc.Ctx(logN, nq, kp, dnum, bits=bits)
    assert P.q == C.q and P.p == C.p, "prime rule differs between library and oracle"
    assert P.alpha == C.alpha and P.ndig == C.ndig
    return P, C


def secret_pair(N, seed, kind="rot"):
    s = inputs.ternary_secret(N, seed)
    if kind == "relin":
        sp = inputs.square_secret(s)
    else:
        g = inputs.galois_elements(N, 1, seed + 1)[0]
        sp = inputs.galois_secret(s, g)
    return s, sp
