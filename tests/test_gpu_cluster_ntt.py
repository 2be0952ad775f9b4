"""GPU parity of the one-launch cluster NTT (KS_OPT_NTT_CLUSTER): the same
transforms and key switches as the two-pass NTT, bit for bit against the
oracle, on every ring degree (2^13 and 2^17 fall back to two passes)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2311_01598_gb300 import inputs
from tests._gpu import built_lib, need_gpu, pair, secret_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("logN", [10, 11, 12, 13, 14, 15, 16, 17])
def test_cluster_ntt_parity(logN, mode):
    """Forward (canonical output) and inverse (N^-1 scale) negacyclic NTT of
    Q and P towers, one cluster per limb (mode 1: CTAs of the two-pass size,
    mode 2: twice as wide)."""
    need_gpu()
    ks = built_lib()
    P, C = pair(logN, 3, 2, 3)
    P.set_ntt_cluster(mode)
    towers = C.q + C.p
    psis = C.psi_q + C.psi_p
    a = inputs.uniform_towers(towers, C.N, seed=300 + logN)
    t = ks.to_device(a)
    P.ntt(0, t, inverse=False)
    got = ks.to_host(t)
    for i in range(len(towers)):
        assert np.array_equal(got[i], orc.ntt(a[i], logN, towers[i], psis[i])), f"forward tower {i}"
    P.ntt(0, t, inverse=True)
    assert np.array_equal(ks.to_host(t), a)
    b = inputs.uniform_towers(towers[2:], C.N, seed=350 + logN)
    tb = ks.to_device(b)
    P.ntt(2, tb, inverse=True)
    gb = ks.to_host(tb)
    for i in range(3):
        assert np.array_equal(gb[i], orc.intt(b[i], logN, towers[2 + i], psis[2 + i]))


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("logN,nq,kp,dnum", [(11, 6, 2, 2), (12, 7, 3, 3), (15, 9, 4, 3), (16, 24, 8, 3)])
def test_cluster_ntt_keyswitch(logN, nq, kp, dnum, mode):
    """Key switches whose every NTT (ModUp P1 with its prescale, P3, ModDown
    P1 and P3) runs as a cluster launch: MP, DC, OC and the batched split and
    whole-basis schedules over uneven levels give the oracle's outputs."""
    need_gpu()
    ks = built_lib()
    P, C = pair(logN, nq, kp, dnum)
    P.set_ntt_cluster(mode)
    s, sp = secret_pair(C.N, seed=311)
    evk = C.keygen(s, sp, seed=312)
    key = P.upload_key(evk)
    d = inputs.uniform_towers(C.q, C.N, seed=313)
    w0, w1 = C.keyswitch(nq, d, evk)
    dd = ks.to_device(d)
    for df in ("MP", "DC", "OC"):
        o0, o1 = ks.empty((nq, C.N)), ks.empty((nq, C.N))
        P.switch(key, nq, dd, o0, o1, df)
        assert np.array_equal(ks.to_host(o0), w0) and np.array_equal(ks.to_host(o1), w1), df
    levels = [nq, max(1, nq // 2), 1, nq - 1 if nq > 1 else 1, nq]
    jobs, want = [], []
    for i, nact in enumerate(levels):
        di = inputs.uniform_towers(C.q[:nact], C.N, seed=320 + i)
        want.append(C.keyswitch(nact, di, evk))
        jobs.append((key, nact, ks.to_device(di), ks.empty((nact, C.N)), ks.empty((nact, C.N))))
    for variant in (1, 2):
        for (_, _, _, o0, o1) in jobs:
            o0.zero_()
            o1.zero_()
        P.switch_batch_sched(jobs, ks.Schedule(2, variant, 64, 0))
        for (_, _, _, o0, o1), (x0, x1) in zip(jobs, want):
            assert np.array_equal(ks.to_host(o0), x0) and np.array_equal(ks.to_host(o1), x1), variant
    P.set_ntt_cluster(0)
