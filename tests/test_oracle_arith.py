"""Pins for the oracle's primes, roots of unity and NTT (no GPU).

None of these checks reuse the oracle's own formulas: primality comes from
sympy, roots are checked by their defining equations, and the transform is
pinned by the convolution theorem against an independent schoolbook product
in Python integers plus the evaluation points it must use.
"""
import numpy as np
import pytest
import sympy

from oracle import oracle as orc
from tests._bigint import brv, negacyclic_schoolbook


@pytest.mark.parametrize("logN,bits,count", [(4, 50, 4), (12, 50, 4), (16, 54, 32), (17, 54, 48)])
def test_prime_rule(logN, bits, count):
    """The count largest primes q < 2^bits with q = 1 mod 2N, descending,
    none skipped (checked against sympy over the whole progression)."""
    ps = orc.gen_primes(logN, bits, count)
    step = 2 << logN
    assert len(ps) == count
    assert all(p < 2**bits for p in ps)
    assert all(p % step == 1 for p in ps)
    assert all(sympy.isprime(p) for p in ps)
    assert all(a > b for a, b in zip(ps, ps[1:]))
    # completeness: every member of 1 + k*2N in [ps[-1], 2^bits) that is prime is listed
    top = (2**bits - 2) // step
    bottom = (ps[-1] - 1) // step
    listed = set(ps)
    for k in range(bottom, top + 1):
        c = 1 + k * step
        assert sympy.isprime(c) == (c in listed), c


def test_is_prime_matches_sympy():
    rng = np.random.default_rng(1)
    cases = [0, 1, 2, 3, 4, 561, 1105, 2047, 3215031751, 341550071728321,
             3825123056546413051, 2**61 - 1, 2**62 - 57, (2**31 - 1) * (2**31 + 11)]
    cases += [int(x) | 1 for x in rng.integers(1, 2**62, size=300, dtype=np.int64)]
    for n in cases:
        assert orc.is_prime(n) == sympy.isprime(n), n


@pytest.mark.parametrize("logN,bits", [(3, 30), (12, 50), (16, 54), (17, 54)])
def test_psi_rule(logN, bits):
    """psi = x^((q-1)/2N) for the smallest x >= 2 with psi^N = -1."""
    N = 1 << logN
    for q in orc.gen_primes(logN, bits, 3):
        psi = orc.find_psi(q, logN)
        assert pow(psi, N, q) == q - 1
        assert pow(psi, 2 * N, q) == 1
        x = 2
        while pow(pow(x, (q - 1) // (2 * N), q), N, q) != q - 1:
            x += 1
        assert psi == pow(x, (q - 1) // (2 * N), q)


def _prime_psi(logN, bits=50):
    q = orc.gen_primes(logN, bits, 1)[0]
    return q, orc.find_psi(q, logN)


@pytest.mark.parametrize("logN", [2, 3, 4, 5])
def test_ntt_evaluation_points(logN):
    """NTT(X) lists the 2N-th primitive roots psi^(2*brv(k)+1): the slot
    convention.  NTT(1) is all ones.  The points are N distinct roots of
    X^N + 1."""
    N = 1 << logN
    q, psi = _prime_psi(logN)
    x = np.zeros(N, dtype=np.uint64)
    x[1] = 1
    pts = [int(v) for v in orc.ntt_naive(x, logN, q, psi)]
    assert pts == [pow(psi, 2 * brv(k, logN) + 1, q) for k in range(N)]
    assert len(set(pts)) == N
    assert all(pow(p, N, q) == q - 1 for p in pts)
    one = np.zeros(N, dtype=np.uint64)
    one[0] = 1
    assert all(int(v) == 1 for v in orc.ntt_naive(one, logN, q, psi))


@pytest.mark.parametrize("logN", [3, 4, 5, 6])
def test_ntt_convolution_theorem(logN):
    """NTT(a) * NTT(b) = NTT(a*b mod X^N+1) with the product taken by an
    independent schoolbook in Python integers; with NTT(X) fixed above this
    determines the transform (a ring map fixed on the generator X)."""
    N = 1 << logN
    q, psi = _prime_psi(logN)
    rng = np.random.default_rng(logN)
    for _ in range(3):
        a = rng.integers(0, q, size=N, dtype=np.uint64)
        b = rng.integers(0, q, size=N, dtype=np.uint64)
        ab = [v % q for v in negacyclic_schoolbook([int(v) for v in a], [int(v) for v in b])]
        lhs = [(int(u) * int(v)) % q for u, v in zip(orc.ntt_naive(a, logN, q, psi), orc.ntt_naive(b, logN, q, psi))]
        rhs = [int(v) for v in orc.ntt_naive(np.array(ab, dtype=np.uint64), logN, q, psi)]
        assert lhs == rhs
        # linearity
        s = (a.astype(object) + b.astype(object)) % q
        lin = [(int(u) + int(v)) % q for u, v in zip(orc.ntt_naive(a, logN, q, psi), orc.ntt_naive(b, logN, q, psi))]
        assert lin == [int(v) for v in orc.ntt_naive(np.array(s, dtype=np.uint64), logN, q, psi)]


@pytest.mark.parametrize("logN", [1, 2, 5, 8, 10])
def test_fast_ntt_equals_naive(logN):
    N = 1 << logN
    q, psi = _prime_psi(logN, 54 if logN > 5 else 50)
    a = np.random.default_rng(logN + 100).integers(0, q, size=N, dtype=np.uint64)
    A = orc.ntt(a, logN, q, psi)
    assert np.array_equal(A, orc.ntt_naive(a, logN, q, psi))
    assert np.array_equal(orc.intt(A, logN, q, psi), a)
    assert np.array_equal(orc.intt_naive(A, logN, q, psi), a)


@pytest.mark.parametrize("logN", [12, 16, 17])
def test_fast_ntt_roundtrip_large(logN):
    q, psi = _prime_psi(logN, 54)
    a = np.random.default_rng(logN).integers(0, q, size=1 << logN, dtype=np.uint64)
    A = orc.ntt(a, logN, q, psi)
    assert np.array_equal(orc.intt(A, logN, q, psi), a)
    assert int(A.max()) < q


def test_fast_ntt_convolution_large():
    """Convolution theorem at N=2^12 against the oracle's schoolbook, which
    is itself pinned against Python integers at small N below."""
    logN = 12
    q, psi = _prime_psi(logN, 50)
    rng = np.random.default_rng(7)
    a = rng.integers(0, q, size=1 << logN, dtype=np.uint64)
    b = rng.integers(0, q, size=1 << logN, dtype=np.uint64)
    lhs = (orc.ntt(a, logN, q, psi).astype(object) * orc.ntt(b, logN, q, psi).astype(object)) % q
    rhs = orc.ntt(orc.negacyclic_mul(a, b, logN, q), logN, q, psi)
    assert np.array_equal(lhs.astype(np.uint64), rhs)


@pytest.mark.parametrize("logN", [2, 4, 6])
def test_schoolbook_matches_python(logN):
    N = 1 << logN
    q = orc.gen_primes(logN, 50, 1)[0]
    rng = np.random.default_rng(logN)
    a = rng.integers(0, q, size=N, dtype=np.uint64)
    b = rng.integers(0, q, size=N, dtype=np.uint64)
    ref = [v % q for v in negacyclic_schoolbook([int(v) for v in a], [int(v) for v in b])]
    assert [int(v) for v in orc.negacyclic_mul(a, b, logN, q)] == ref
