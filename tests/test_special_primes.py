"""ks_special_primes (host only, no GPU): the largest primes of the form
k*2^32 + 1 below 2^bits, pinned by sympy primality over the whole
progression (every skipped k is composite), the form, the order and the
congruence 1 mod 2N for every supported ring degree."""
import pytest

from tests._gpu import built_lib

sympy = pytest.importorskip("sympy")


@pytest.mark.parametrize("bits,count", [(54, 32), (56, 48), (40, 12), (38, 4)])
def test_special_primes_are_the_largest_of_their_form(bits, count):
    ks = built_lib()
    ps = ks.special_primes(bits, count)
    assert len(ps) == count and ps == sorted(ps, reverse=True)
    assert all(p < 2 ** bits and p % (1 << 32) == 1 and sympy.isprime(p) for p in ps)
    assert all(p % (1 << 18) == 1 for p in ps)   # 1 mod 2N up to N = 2^17
    # completeness: no prime of the form between 2^bits and the last one is skipped
    k_top = (2 ** bits - 2) >> 32
    k_low = ps[-1] >> 32
    found = [(k << 32) + 1 for k in range(k_top, k_low - 1, -1) if sympy.isprime((k << 32) + 1)]
    assert found == ps


def test_special_primes_rejects_bad_arguments():
    ks = built_lib()
    for bits in (32, 57):
        with pytest.raises(RuntimeError, match="bits must be"):
            ks.special_primes(bits, 1)
    with pytest.raises(RuntimeError, match="not enough primes"):
        ks.special_primes(33, 10 ** 6)
