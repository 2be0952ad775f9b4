"""Host-side accounting of bench.py (no GPU): the algorithmic work and bytes
it divides by, counted independently here from the structure of hybrid key
switching at N = 2^16, L+1 = 24, K = 8, dnum = 3 (alpha = 8)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_work_per_key_switch():
    b = _bench()
    N, L1, K, alpha, dnum = 1 << 16, 24, 8, 8, 3
    w = b.algorithmic_work()
    # NTTs: ModUp inverse on the 24 inputs; forward on every raised limb
    # (each digit to the 24 + 8 - 8 towers outside it); ModDown inverse on
    # 2 x 8 special limbs and forward on 2 x 24
    inv, fwd = L1 + 2 * K, dnum * (L1 + K - alpha) + 2 * L1
    assert (w["inverse_butterflies"], w["forward_butterflies"]) == (inv * N // 2 * 16, fwd * N // 2 * 16)
    assert w["ntt"] == inv + fwd == 160 and w["butterflies"] == 83886080
    # base conversions: each digit's 8 sources to 24 targets, then 8 -> 24 for both polynomials
    assert w["bconv_macs"] == dnum * alpha * (L1 + K - alpha) * N + 2 * K * L1 * N == 62914560
    # key product: digits x two halves x (24 + 8) towers
    assert w["key_macs"] == dnum * 2 * (L1 + K) * N


def test_algorithmic_bytes_per_key_switch():
    b = _bench()
    limb = (1 << 16) * 8
    # input + key (3 digits x 2 halves x 32 towers) + two outputs
    assert b.ALG_BYTES_PER_KS == 24 * limb + 3 * 2 * 32 * limb + 2 * 24 * limb == 138412032
