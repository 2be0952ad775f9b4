"""GPU parity at the edges of what ks_params_create admits, element by
element against the oracle (bit-exact, integer outputs).

The kernels' correctness rests on range bounds that hold for moduli below
2^56 (lazy NTT values below a small multiple of q, 7-byte slices in the
tensor-core base conversion, 128-bit sums of products before one Montgomery
reduction).  Uniform inputs at 50-54 bits never reach those bounds, so these
cases push them: 56-bit and 30-bit primes, explicit primes just below 2^56
with special primes smaller than every Q prime, alpha = 1 with dnum = L+1 at
N = 2^16, and inputs / keys whose every word is the largest residue (or 0),
including inputs whose ModUp pre-scaled coefficients (Sec. III-B P1) and
ModDown pre-scaled special towers (Sec. III-C P1) are all q-1, so the base
conversions see their largest operands everywhere."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2311_01598_gb300 import inputs
from tests._gpu import built_lib, need_gpu, pair

pytestmark = pytest.mark.gpu


def random_evk(C, seed):
    """An evaluation key of uniform words ([ndig][2][nq+kp][N]); bit-exact
    parity needs no key relation."""
    towers = C.q + C.p
    return np.stack([np.stack([inputs.uniform_towers(towers, C.N, seed=seed + 2 * j + x) for x in range(2)])
                     for j in range(C.ndig)])


def max_evk(C):
    """Every key word the largest residue r-1 of its tower."""
    towers = np.array(C.q + C.p, dtype=np.uint64)
    one = np.ones((C.ndig, 2, len(towers), C.N), dtype=np.uint64)
    return one * (towers - np.uint64(1))[None, None, :, None]


def digit_hat(primes, nact, alpha, i):
    """prod of the other active primes of the digit holding tower i, mod q_i
    (Q_j/q_i of Sec. III-B over the active primes of digit j)."""
    j = i // alpha
    hat = 1
    for k in range(j * alpha, min((j + 1) * alpha, nact)):
        if k != i:
            hat *= primes[k]
    return hat % primes[i]


def max_y_input(C, nact):
    """Evaluation-form input whose ModUp P1 output y_i = [x_i (Q_j/q_i)^-1]_{q_i}
    is q_i - 1 in every coefficient: x_i = (q_i - 1)(Q_j/q_i) mod q_i, then
    the oracle's forward NTT."""
    out = np.empty((nact, C.N), dtype=np.uint64)
    for i in range(nact):
        qi = C.q[i]
        x = (qi - 1) * digit_hat(C.q, nact, C.alpha, i) % qi
        out[i] = orc.ntt(np.full(C.N, x, dtype=np.uint64), C.logN, qi, C.psi_q[i])
    return out


def max_w_cprime(C, nact):
    """c' over D_l (evaluation form, [2][nact+K][N]) whose ModDown P1 output
    w_k = [iNTT(c'_{p_k}) (P/p_k)^-1]_{p_k} is p_k - 1 everywhere; Q towers
    all q_i - 1."""
    K = C.kp
    out = np.empty((2, nact + K, C.N), dtype=np.uint64)
    for x in range(2):
        for i in range(nact):
            out[x, i] = C.q[i] - 1
        for k in range(K):
            pk = C.p[k]
            hat = 1
            for m in range(K):
                if m != k:
                    hat *= C.p[m]
            v = (pk - 1) * (hat % pk) % pk
            out[x, nact + k] = orc.ntt(np.full(C.N, v, dtype=np.uint64), C.logN, pk, C.psi_p[k])
    return out


def check_all_paths(ks, P, C, key, nact, d, w0, w1, engines=(True,), what=""):
    """MP, DC and OC single switches and the batched split, whole-basis and
    per-tower cluster schedules, under each base-conversion engine (the
    tower kernel's base conversions are always on the CUDA cores), all equal
    to (w0, w1)."""
    dd = ks.to_device(d)
    for tensor in engines:
        P.set_bconv_tensor(tensor)
        for df in ("MP", "DC", "OC"):
            o0, o1 = ks.empty((nact, C.N)), ks.empty((nact, C.N))
            P.switch(key, nact, dd, o0, o1, df)
            assert np.array_equal(ks.to_host(o0), w0), (what, nact, df, tensor, "out0")
            assert np.array_equal(ks.to_host(o1), w1), (what, nact, df, tensor, "out1")
        for variant in (1, 2, 3):
            jobs = [(key, nact, dd, ks.empty((nact, C.N)), ks.empty((nact, C.N))) for _ in range(2)]
            P.switch_batch_sched(jobs, ks.Schedule(2, variant, 64, 0))
            for (_, _, _, o0, o1) in jobs:
                assert np.array_equal(ks.to_host(o0), w0), (what, nact, variant, tensor, "batch out0")
                assert np.array_equal(ks.to_host(o1), w1), (what, nact, variant, tensor, "batch out1")
    P.set_bconv_tensor(True)
    assert P.device_status(clear=True) == 0


EDGE_SETS = [
    # id, logN, nq, kp, dnum, bits, levels
    ("56bit_N2^16_24+8_d3", 16, 24, 8, 3, 56, [24, 9]),
    ("56bit_N2^17_36+12_d3", 17, 36, 12, 3, 56, [36, 20]),
    ("30bit_N2^16_24+8_d3", 16, 24, 8, 3, 30, [24, 10]),
    ("30bit_N2^12_6+2_d3", 12, 6, 2, 3, 30, [6, 2]),
    ("alpha1_N2^16_24+8_d24", 16, 24, 8, 24, 54, [24, 13]),
]


@pytest.mark.parametrize("case", EDGE_SETS, ids=[c[0] for c in EDGE_SETS])
def test_edge_parameter_sets(case):
    """Prime sizes at both ends of 30..56 bits, and alpha = 1 with one digit
    per tower at N = 2^16: every dataflow and the batched schedules, both
    base-conversion engines where the shape has two."""
    need_gpu()
    ks = built_lib()
    _, logN, nq, kp, dnum, bits, levels = case
    P, C = pair(logN, nq, kp, dnum, bits)
    evk = random_evk(C, seed=700 + logN + bits)
    key = P.upload_key(evk)
    for nact in levels:
        d = inputs.uniform_towers(C.q[:nact], C.N, seed=710 + nact)
        w0, w1 = C.keyswitch(nact, d, evk)
        check_all_paths(ks, P, C, key, nact, d, w0, w1, engines=(True, False), what=case[0])


def test_explicit_primes_near_2_56():
    """Explicit prime lists (h_q/h_p): Q the largest primes = 1 mod 2N below
    2^56 in ascending order, P primes of 44 bits (every special prime smaller
    than every Q prime)."""
    need_gpu()
    ks = built_lib()
    logN, nq, kp, dnum = 13, 10, 4, 3
    q = sorted(orc.gen_primes(logN, 56, nq))
    p = orc.gen_primes(logN, 44, kp)
    assert max(q) < 2 ** 56 and max(p) < min(q)
    P = ks.Params(logN, nq, kp, dnum, q=q, p=p)
    C = orc.Ctx(logN, nq, kp, dnum, q=q, p=p)
    assert P.q == C.q == q and P.p == C.p == p
    evk = random_evk(C, seed=720)
    key = P.upload_key(evk)
    for nact in (10, 4):
        d = inputs.uniform_towers(C.q[:nact], C.N, seed=721 + nact)
        w0, w1 = C.keyswitch(nact, d, evk)
        check_all_paths(ks, P, C, key, nact, d, w0, w1, engines=(True, False), what="explicit")


@pytest.mark.parametrize("kind", ["zero", "all_q_minus_1", "max_y"])
@pytest.mark.parametrize("key_kind", ["uniform", "all_r_minus_1"])
def test_extreme_inputs_56bit(kind, key_kind):
    """N = 2^16, 24+8 primes of 56 bits, dnum 3: inputs of all 0, all q-1,
    or with every ModUp pre-scaled coefficient q-1; keys uniform or with
    every word r-1; MP, DC, OC and the batched schedules, both engines."""
    need_gpu()
    ks = built_lib()
    P, C = pair(16, 24, 8, 3, 56)
    evk = random_evk(C, seed=730) if key_kind == "uniform" else max_evk(C)
    key = P.upload_key(evk)
    for nact in (24, 17):
        if kind == "zero":
            d = np.zeros((nact, C.N), dtype=np.uint64)
        elif kind == "all_q_minus_1":
            d = np.ones((nact, C.N), dtype=np.uint64) * (np.array(C.q[:nact], dtype=np.uint64) - 1)[:, None]
        else:
            d = max_y_input(C, nact)
        w0, w1 = C.keyswitch(nact, d, evk)
        if kind == "zero":
            assert not w0.any() and not w1.any()
        check_all_paths(ks, P, C, key, nact, d, w0, w1, engines=(True, False), what=(kind, key_kind))


# (logN, nq, kp, dnum, levels, bits): one K block of the tensor-core base
# conversion (8 sources) with byte slices of the constants (56-bit moduli) and
# with 9-bit slices (54-bit moduli: partial sums up to 8*7*255*511), and two K
# blocks at their limit (18 sources: partial sums up to 7*18*255^2, just below
# the 2^23 of the accumulator's fixed read-out)
EXTREME_SHAPES = [(16, 24, 8, 3, (24, 9), 56), (16, 24, 8, 3, (24, 9), 54), (13, 36, 18, 2, (36, 19), 56)]
EXTREME_IDS = ["8src", "8src_9bit", "18src"]


@pytest.mark.parametrize("shape", EXTREME_SHAPES, ids=EXTREME_IDS)
@pytest.mark.parametrize("kind", ["all_q_minus_1", "max_y"])
def test_modup_extreme_56bit(kind, shape):
    """ModUp P1-P3 stage (Sec. III-B) with the largest inputs, 56-bit primes
    (and 54-bit ones for the 9-bit constant slices)."""
    need_gpu()
    ks = built_lib()
    logN, nq, kp, dnum, levels, bits = shape
    P, C = pair(logN, nq, kp, dnum, bits)
    for nact in levels:
        if kind == "all_q_minus_1":
            d = np.ones((nact, C.N), dtype=np.uint64) * (np.array(C.q[:nact], dtype=np.uint64) - 1)[:, None]
        else:
            d = max_y_input(C, nact)
        want = C.modup(nact, d)
        for tensor in (True, False):
            P.set_bconv_tensor(tensor)
            ext = ks.empty(want.shape)
            P.modup(nact, ks.to_device(d), ext)
            assert np.array_equal(ks.to_host(ext), want), (kind, nact, tensor)
    P.set_bconv_tensor(True)


@pytest.mark.parametrize("shape", EXTREME_SHAPES, ids=EXTREME_IDS)
@pytest.mark.parametrize("kind", ["all_r_minus_1", "max_w"])
def test_moddown_extreme_56bit(kind, shape):
    """ModDown P1-P4 stage (Sec. III-C) with c' of all r-1, or with every
    pre-scaled special-tower coefficient p_k - 1, 56-bit primes (and 54-bit
    ones for the 9-bit constant slices)."""
    need_gpu()
    ks = built_lib()
    logN, nq, kp, dnum, levels, bits = shape
    P, C = pair(logN, nq, kp, dnum, bits)
    for nact in levels:
        if kind == "all_r_minus_1":
            towers = np.array(C.towers(nact), dtype=np.uint64)
            cp = np.ones((2, nact + C.kp, C.N), dtype=np.uint64) * (towers - 1)[None, :, None]
        else:
            cp = max_w_cprime(C, nact)
        for x in range(2):
            want = C.moddown(nact, cp[x])
            for tensor in (True, False):
                P.set_bconv_tensor(tensor)
                out = ks.empty(want.shape)
                P.moddown(nact, ks.to_device(cp[x]), out)
                assert np.array_equal(ks.to_host(out), want), (kind, nact, x, tensor)
    P.set_bconv_tensor(True)


@pytest.mark.parametrize("logN,nq,kp,dnum,levels", [(12, 6, 2, 3, [6, 2]), (16, 24, 8, 3, [24, 11]),
                                                     (17, 20, 6, 2, [20, 7])])
def test_special_form_primes(logN, nq, kp, dnum, levels):
    """Explicit primes of the form k*2^32 + 1 (ks_special_primes): the
    two-pass NTT kernels take the cheaper butterfly product; forward and
    inverse NTTs and every key-switch path equal the oracle's on the same
    primes, both base-conversion engines."""
    need_gpu()
    ks = built_lib()
    allp = ks.special_primes(54, nq + kp)
    p, q = allp[:kp], allp[kp:]
    P = ks.Params(logN, nq, kp, dnum, q=q, p=p)
    C = orc.Ctx(logN, nq, kp, dnum, q=q, p=p)
    assert P.q == C.q == q and P.p == C.p == p
    towers = C.q + C.p
    psis = C.psi_q + C.psi_p
    a = inputs.uniform_towers(towers[:6], C.N, seed=900 + logN)
    t = ks.to_device(a)
    P.ntt(0, t, inverse=False)
    got = ks.to_host(t)
    for i in range(6):
        assert np.array_equal(got[i], orc.ntt(a[i], logN, towers[i], psis[i])), i
    P.ntt(0, t, inverse=True)
    assert np.array_equal(ks.to_host(t), a)
    evk = random_evk(C, seed=910)
    key = P.upload_key(evk)
    for nact in levels:
        d = inputs.uniform_towers(C.q[:nact], C.N, seed=920 + nact)
        w0, w1 = C.keyswitch(nact, d, evk)
        check_all_paths(ks, P, C, key, nact, d, w0, w1, engines=(True, False), what="special-form")
