"""Pins for the oracle's base conversion, ModDown, key generation and whole
key switch (no GPU).  Everything is checked against big-integer identities,
published generator outputs, Table III of the paper, or the decryption
invariant of key switching -- never by re-running the oracle's formula.
"""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2311_01598_gb300 import inputs
from tests._bigint import centre, crt, negacyclic_schoolbook, prod

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ BConv
@pytest.mark.parametrize("a,b", [(1, 3), (2, 3), (3, 4), (8, 5)])
def test_bconv_crt_identity(a, b):
    """Fast base conversion (CiFlow Sec. III-B, ModUp P2) of x over a source
    basis S gives, on every target prime, X + u*S with X the exact CRT value
    and ONE integer u in [0, a) per coefficient; with a = 1, u = 0."""
    logN = 4
    N = 1 << logN
    primes = orc.gen_primes(logN, 54, a + b)
    src, dst = primes[:a], primes[a:]
    x = inputs.uniform_towers(src, N, seed=a * 10 + b)
    out = orc.bconv(src, x, dst, logN)
    S = prod(src)
    for n in range(N):
        X = crt([x[i, n] for i in range(a)], src)
        got = [int(out[t, n]) for t in range(b)]
        us = [u for u in range(a) if [(X + u * S) % r for r in dst] == got]
        assert len(us) == 1, "target residues are not X + u*S for one u in [0, a)"
        if a == 1:
            assert us == [0]


# ------------------------------------------------------------------ ModDown
def test_moddown_divides_by_P():
    """ModDown (Sec. III-C): for c' = C in [0, PQ) given per tower in
    evaluation form, the output equals floor(C/P) - u (mod Q) per
    coefficient, with one u in [0, K)."""
    logN, nq, kp = 4, 3, 2
    ctx = orc.Ctx(logN, nq, kp, dnum=3, bits=54)
    N = ctx.N
    Q, P = prod(ctx.q), prod(ctx.p)
    rng = np.random.default_rng(3)
    C = [int(rng.integers(0, 2**62)) * int(rng.integers(0, 2**62)) * int(rng.integers(0, 2**62)) % (P * Q)
         for _ in range(N)]
    primes = ctx.q + ctx.p
    psis = ctx.psi_q + ctx.psi_p
    cp = np.array([[c % m for c in C] for m in primes], dtype=np.uint64)
    cp_eval = np.stack([orc.ntt(cp[t], logN, primes[t], psis[t]) for t in range(len(primes))])
    out = ctx.moddown(nq, cp_eval)
    out_coef = np.stack([orc.intt(out[i], logN, ctx.q[i], ctx.psi_q[i]) for i in range(nq)])
    for n in range(N):
        got = crt([out_coef[i, n] for i in range(nq)], ctx.q)
        u = (C[n] // P - got) % Q
        assert 0 <= u < kp, (n, u)


# ------------------------------------------------------------------ keygen
def _golden_splitmix():
    rows = {}
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t) for t in line.split()]
            rows[v[0]] = v[1:]
    return rows


def test_splitmix64_published_vectors():
    for seed, want in _golden_splitmix().items():
        got = [int(v) for v in orc.splitmix64(seed, len(want))]
        assert got == want


def test_gaussian_sampler_moments():
    e = orc.sample_gauss(12345, 200000)
    assert np.abs(e).max() <= 19
    assert abs(e.mean()) < 0.05
    assert abs(e.std() - 3.2) < 0.05


@pytest.mark.parametrize("logN,nq,kp,dnum", [(4, 3, 1, 3), (5, 5, 2, 2), (6, 4, 2, 1)])
def test_keygen_relation(logN, nq, kp, dnum):
    """b_j + a_j*s = e_j + [P*g_j]*s' on every tower, with e_j one small
    integer polynomial (|e| <= 19) common to all towers and g_j the CRT
    idempotent of digit j (1 on its own Q towers, 0 elsewhere)."""
    ctx = orc.Ctx(logN, nq, kp, dnum, bits=54)
    N = ctx.N
    s = inputs.ternary_secret(N, seed=logN)
    sp = inputs.galois_secret(s, 5)
    evk = ctx.keygen(s, sp, seed=99)
    assert evk.shape == (ctx.ndig, 2, nq + kp, N)
    primes = ctx.q + ctx.p
    P = prod(ctx.p)
    s_int = [int(v) for v in s]
    sp_int = [int(v) for v in sp]
    for j in range(ctx.ndig):
        e_ref = None
        for t, r in enumerate(primes):
            psi = (ctx.psi_q + ctx.psi_p)[t]
            b = orc.intt(evk[j, 0, t], logN, r, psi)
            a = orc.intt(evk[j, 1, t], logN, r, psi)
            a_s = negacyclic_schoolbook([int(v) for v in a], s_int)
            in_digit = t < nq and t // ctx.alpha == j
            g = P % r if in_digit else 0
            g_sp = [g * v for v in sp_int]
            e = [centre(int(bv) + asv - gv, r) for bv, asv, gv in zip(b, a_s, g_sp)]
            assert max(abs(v) for v in e) <= 19
            if e_ref is None:
                e_ref = e
            assert e == e_ref


def test_table3_evk_sizes():
    """evk = ndig x 2 x (k_l + k_p) towers x N words of 8 bytes reproduces
    every evk size and alpha of CiFlow Table III (MB read as MiB)."""
    with open(os.path.join(GOLDEN, "table3_params.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for name, logN, kl, kp, dnum, alpha, mb in rows:
        logN, kl, kp, dnum, alpha, mb = map(int, (logN, kl, kp, dnum, alpha, mb))
        ctx = orc.Ctx(logN, kl, kp, dnum, bits=54)
        assert ctx.alpha == alpha, name
        assert ctx.evk_bytes() == mb * 2**20, name
    small = orc.Ctx(4, 5, 2, 2, bits=54)
    evk = small.keygen(inputs.ternary_secret(16, 1), np.zeros(16, dtype=np.int64), 1)
    assert evk.nbytes == small.evk_bytes()


# ------------------------------------------------------------------ whole KS
def _decrypt_noise(ctx, nact, d, out0, out1, s, sp):
    """e = out0 + out1*s - d*s' (mod Q_l), centred, as Python integers."""
    logN, N = ctx.logN, ctx.N
    towers = []
    for i in range(nact):
        q, psi = ctx.q[i], ctx.psi_q[i]
        sh = orc.ntt(np.array([v % q for v in s.astype(object)], dtype=np.uint64), logN, q, psi)
        sph = orc.ntt(np.array([int(v) % q for v in sp], dtype=np.uint64), logN, q, psi)
        eh = (out0[i].astype(object) + out1[i].astype(object) * sh.astype(object)
              - d[i].astype(object) * sph.astype(object)) % q
        towers.append(orc.intt(np.array(eh, dtype=np.uint64), logN, q, psi))
    Ql = prod(ctx.q[:nact])
    return [centre(crt([towers[i][n] for i in range(nact)], ctx.q[:nact]), Ql) for n in range(N)]


def _noise_bound(ctx, nact):
    """|e| <= sum_j N*alpha_j*Q_j*B_e / P + 1 + K*(N+1): D_j < alpha_j*Q_j
    per coefficient, |e_j| <= B_e = 19, and ModDown's fast base conversion
    adds u*P with u < K to each polynomial (times s for the second)."""
    P = prod(ctx.p)
    tot = 0
    for j in range(ctx.active_digits(nact)):
        lo, hi = j * ctx.alpha, min((j + 1) * ctx.alpha, nact)
        tot += ctx.N * (hi - lo) * prod(ctx.q[lo:hi]) * 19
    return tot // P + 1 + ctx.kp * (ctx.N + 1)


@pytest.mark.parametrize("logN,nq,kp,dnum,bits,nact", [
    (4, 3, 1, 3, 50, 3),      # brute-force size, config-1 shape
    (4, 3, 1, 3, 50, 2),      # lower level
    (5, 6, 2, 2, 54, 6),
    (5, 6, 2, 2, 54, 5),      # ragged last digit
    (5, 6, 2, 1, 54, 6),      # dnum = 1: one digit, no reduce
    (6, 7, 3, 3, 54, 7),      # alpha = 3, last digit of one tower
    (6, 7, 3, 3, 54, 1),      # single tower
    (12, 3, 1, 3, 50, 3),     # config 1: N=2^12, 3+1 primes, dnum=3
])
def test_keyswitch_decrypts(logN, nq, kp, dnum, bits, nact):
    """Decryption invariant of hybrid key switching: out0 + out1*s equals
    d*s' up to a noise polynomial within the stated bound (a wrong sign,
    index, constant or dropped term leaves noise of the size of Q)."""
    ctx = orc.Ctx(logN, nq, kp, dnum, bits=bits)
    N = ctx.N
    s = inputs.ternary_secret(N, seed=11)
    sp = inputs.square_secret(s)
    evk = ctx.keygen(s, sp, seed=5)
    d = inputs.uniform_towers(ctx.q[:nact], N, seed=17)
    out0, out1 = ctx.keyswitch(nact, d, evk)
    assert out0.shape == (nact, N)
    for i in range(nact):
        assert int(out0[i].max()) < ctx.q[i] and int(out1[i].max()) < ctx.q[i]
    e = _decrypt_noise(ctx, nact, d, out0, out1, s, sp)
    bound = _noise_bound(ctx, nact)
    assert max(abs(v) for v in e) <= bound
    assert bound < prod(ctx.q[:nact]) // 1024


def test_keyswitch_with_rotation_key():
    ctx = orc.Ctx(5, 4, 2, 2, bits=54)
    s = inputs.ternary_secret(ctx.N, seed=2)
    g = inputs.galois_elements(ctx.N, 1, seed=3)[0]
    sp = inputs.galois_secret(s, g)
    evk = ctx.keygen(s, sp, seed=7)
    d = inputs.uniform_towers(ctx.q, ctx.N, seed=8)
    out0, out1 = ctx.keyswitch(4, d, evk)
    e = _decrypt_noise(ctx, 4, d, out0, out1, s, sp)
    assert max(abs(v) for v in e) <= _noise_bound(ctx, 4)


def test_modup_bypass_and_digit_shape():
    """ModUp (Sec. III-B P3): the digit's own towers are the input towers;
    the raised digit is one integer polynomial D_j = X_j + u*Q_j over all
    of D_l (checked by CRT in coefficient form)."""
    ctx = orc.Ctx(4, 5, 2, 2, bits=54)
    nact = 5
    d = inputs.uniform_towers(ctx.q, ctx.N, seed=4)
    D = ctx.modup(nact, d)
    assert D.shape == (2, nact + 2, ctx.N)
    prim = ctx.towers(nact)
    psis = ctx.psi_q[:nact] + ctx.psi_p
    for j in range(2):
        lo, hi = j * ctx.alpha, min((j + 1) * ctx.alpha, nact)
        assert np.array_equal(D[j, lo:hi], d[lo:hi])
        coef = [orc.intt(D[j, t], ctx.logN, prim[t], psis[t]) for t in range(len(prim))]
        xq = [orc.intt(d[i], ctx.logN, ctx.q[i], ctx.psi_q[i]) for i in range(lo, hi)]
        Qj = prod(ctx.q[lo:hi])
        for n in range(ctx.N):
            X = crt([x[n] for x in xq], ctx.q[lo:hi])
            V = crt([c[n] for c in coef], prim)
            assert (V - X) % Qj == 0 and 0 <= (V - X) // Qj < hi - lo


def test_apply_key_pointwise():
    ctx = orc.Ctx(3, 3, 1, 3, bits=50)
    nact = 3
    rng = np.random.default_rng(0)
    prim = ctx.towers(nact)
    D = np.stack([inputs.uniform_towers(prim, ctx.N, seed=j) for j in range(3)])
    evk = np.stack([np.stack([inputs.uniform_towers(ctx.q + ctx.p, ctx.N, seed=10 + 2 * j + x)
                              for x in range(2)]) for j in range(3)])
    cb, ca = ctx.apply_key(nact, D, evk)
    for t, r in enumerate(prim):
        want_b = sum(D[j, t].astype(object) * evk[j, 0, t].astype(object) for j in range(3)) % r
        want_a = sum(D[j, t].astype(object) * evk[j, 1, t].astype(object) for j in range(3)) % r
        assert list(cb[t]) == list(want_b) and list(ca[t]) == list(want_a)
    del rng


# ------------------------------------------------------------------ rotations, hoisting
def _coeff_automorph(a, g, q):
    """a(X) -> a(X^g) mod (X^N + 1, q) on coefficients, written from the
    definition: X^i goes to X^(i*g mod 2N), and X^N = -1."""
    N = len(a)
    out = [0] * N
    for i, v in enumerate(a):
        k = (i * g) % (2 * N)
        if k < N:
            out[k] = (out[k] + int(v)) % q
        else:
            out[k - N] = (out[k - N] - int(v)) % q
    return np.array(out, dtype=np.uint64)


@pytest.mark.parametrize("logN", [3, 6, 10])
def test_automorph_eval_is_the_galois_map(logN):
    """In the evaluation domain X -> X^g is a slot permutation equal to
    NTT(a(X^g)) computed from the coefficients (NTT itself pinned against
    its O(N^2) definition); it composes as phi_g phi_h = phi_gh and phi_1 = id."""
    N = 1 << logN
    q = orc.gen_primes(logN, 54, 1)[0]
    psi = orc.find_psi(q, logN)
    x = inputs.uniform_towers([q], N, seed=logN)[0]
    a = orc.intt(x, logN, q, psi)
    for g in [1, 3, 5, 2 * N - 1, pow(5, 7, 2 * N)]:
        want = orc.ntt(_coeff_automorph(a, g, q), logN, q, psi)
        got = orc.automorph_eval(x, logN, g)
        assert np.array_equal(got, want), g
        assert sorted(got.tolist()) == sorted(x.tolist())
    g, h = 5, pow(5, 3, 2 * N)
    assert np.array_equal(orc.automorph_eval(orc.automorph_eval(x, logN, h), logN, g),
                          orc.automorph_eval(x, logN, g * h % (2 * N)))


def test_hoisted_identity_is_the_key_switch():
    """With g = 1 the hoisted path is the plain key switch, bit for bit."""
    ctx = orc.Ctx(5, 6, 2, 2, bits=54)
    s = inputs.ternary_secret(ctx.N, seed=21)
    evk = ctx.keygen(s, inputs.galois_secret(s, 5), seed=22)
    for nact in (6, 5, 3):
        d = inputs.uniform_towers(ctx.q[:nact], ctx.N, seed=23 + nact)
        w0, w1 = ctx.keyswitch(nact, d, evk)
        h0, h1 = ctx.keyswitch_hoisted(nact, d, [evk], [1])
        assert np.array_equal(h0[0], w0) and np.array_equal(h1[0], w1)


@pytest.mark.parametrize("logN,nq,kp,dnum,nact", [(5, 6, 2, 2, 6), (6, 7, 3, 3, 5), (6, 4, 2, 1, 4)])
def test_hoisted_rotations_decrypt(logN, nq, kp, dnum, nact):
    """Each hoisted rotation decrypts: out0 + out1*s = phi_g(d)*s(X^g) up to
    the key-switching noise bound (the automorphism permutes the raised
    digits' coefficients up to sign, so the bound is unchanged), with
    phi_g(d) computed from the coefficient definition."""
    ctx = orc.Ctx(logN, nq, kp, dnum, bits=54)
    N = ctx.N
    s = inputs.ternary_secret(N, seed=31)
    gals = inputs.galois_elements(N, 3, seed=32)
    evks = [ctx.keygen(s, inputs.galois_secret(s, g), seed=33 + i) for i, g in enumerate(gals)]
    d = inputs.uniform_towers(ctx.q[:nact], N, seed=34)
    out0, out1 = ctx.keyswitch_hoisted(nact, d, evks, gals)
    bound = _noise_bound(ctx, nact)
    for r, g in enumerate(gals):
        dg = np.stack([orc.ntt(_coeff_automorph(orc.intt(d[i], logN, ctx.q[i], ctx.psi_q[i]), g, ctx.q[i]),
                               logN, ctx.q[i], ctx.psi_q[i]) for i in range(nact)])
        e = _decrypt_noise(ctx, nact, dg, out0[r], out1[r], s, inputs.galois_secret(s, g))
        assert max(abs(v) for v in e) <= bound, r


# ------------------------------------------------------------------ compressed keys
def test_key_a_word_is_the_splitmix_stream_at_its_counter():
    """The compressed key's a-words read SplitMix64 at a computed counter:
    word (j, t, n) is the first draw, masked to bitlen(r), below r among
    stream outputs ((j*nfull + t)*N + n)*64 + m of seed^2 -- checked against
    the sequential generator, itself pinned to published outputs."""
    ctx = orc.Ctx(4, 3, 2, 2, bits=54)
    N, nfull, seed = ctx.N, 5, 0x5EED
    primes = ctx.q + ctx.p
    for (j, t, n) in [(0, 0, 0), (0, 4, 15), (1, 2, 7), (1, 4, 3)]:
        base = ((j * nfull + t) * N + n) * 64
        stream = orc.splitmix64(seed ^ 2, base + 64)[base:]
        mask = (1 << primes[t].bit_length()) - 1
        want = next(int(v) & mask for v in stream if (int(v) & mask) < primes[t])
        assert ctx.key_a_word(seed, j, t, n) == want


@pytest.mark.parametrize("logN,nq,kp,dnum", [(4, 3, 1, 3), (5, 5, 2, 2)])
def test_compressed_keygen_relation_and_uniformity(logN, nq, kp, dnum):
    """A compressed key satisfies the key relation b_j + a_j*s = e_j +
    [P g_j] s' with one small e_j per digit, and its a-words are uniform
    residues (mean within 5 sigma of r/2 on every tower)."""
    ctx = orc.Ctx(logN, nq, kp, dnum, bits=54)
    N = ctx.N
    s = inputs.ternary_secret(N, seed=logN + 40)
    sp = inputs.galois_secret(s, 5)
    evk = ctx.keygen_compressed(s, sp, seed=77)
    primes = ctx.q + ctx.p
    P = prod(ctx.p)
    s_int, sp_int = [int(v) for v in s], [int(v) for v in sp]
    for j in range(ctx.ndig):
        e_ref = None
        for t, r in enumerate(primes):
            assert ctx.key_a_word(77, j, t, 3) == int(evk[j, 1, t, 3])
            psi = (ctx.psi_q + ctx.psi_p)[t]
            b = orc.intt(evk[j, 0, t], logN, r, psi)
            a = orc.intt(evk[j, 1, t], logN, r, psi)
            a_s = negacyclic_schoolbook([int(v) for v in a], s_int)
            g = P % r if (t < nq and t // ctx.alpha == j) else 0
            e = [centre(int(bv) + asv - g * spv, r) for bv, asv, spv in zip(b, a_s, sp_int)]
            assert max(abs(v) for v in e) <= 19
            e_ref = e if e_ref is None else e_ref
            assert e == e_ref
    words = evk[:, 1].astype(np.float64) / np.array(primes, dtype=np.float64)[None, :, None]
    sd = (1 / 12) ** 0.5 / (ctx.ndig * N) ** 0.5
    assert np.all(np.abs(words.mean(axis=(0, 2)) - 0.5) < 5 * sd)


def test_compressed_key_switch_decrypts():
    ctx = orc.Ctx(6, 7, 3, 3, bits=54)
    s = inputs.ternary_secret(ctx.N, seed=81)
    sp = inputs.galois_secret(s, 5)
    evk = ctx.keygen_compressed(s, sp, seed=82)
    d = inputs.uniform_towers(ctx.q, ctx.N, seed=83)
    out0, out1 = ctx.keyswitch(7, d, evk)
    e = _decrypt_noise(ctx, 7, d, out0, out1, s, sp)
    assert max(abs(v) for v in e) <= _noise_bound(ctx, 7)
