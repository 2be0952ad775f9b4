"""Tower-sharded key switching (one key switch split over G ranks by tower,
CiFlow Sec. IV-C: output towers are independent), with G ranks emulated on
one device: each rank runs the library's per-rank calls on its own towers
and key shard, and the two all-gathers (the pre-scaled input y, the special
part w) are device copies.  The gathered outputs must equal the oracle's
key switch bit for bit."""
import numpy as np
import pytest

from paper_2311_01598_gb300 import dist as kd
from paper_2311_01598_gb300 import inputs
from tests._gpu import built_lib, need_gpu, pair, secret_pair

pytestmark = pytest.mark.gpu


def _run(P, key, G, nact, d_host):
    torch = need_gpu()
    ks = built_lib()
    parts = [kd.tower_partition(P.nq, P.kp, G, g) for g in range(G)]
    skeys = [P.key_shard(key, ks.Shard(*pt)) for pt in parts]
    assert sum(k.nbytes for k in skeys) == key.nbytes      # sharded, not replicated
    d_own = []
    for pt in parts:
        q0, q1 = kd.active_q(pt, nact)
        d_own.append(ks.to_device(np.ascontiguousarray(d_host[q0:q1])) if q1 > q0 else ks.empty((0, P.N)))
    outs = kd.sharded_keyswitch(P, skeys, parts, nact, d_own,
                                gather_y=lambda ys: torch.cat(ys, dim=0),
                                gather_w=lambda ws: torch.cat(ws, dim=1))
    o0 = np.concatenate([ks.to_host(o[0]) for o in outs if o[0].shape[0] > 0])
    o1 = np.concatenate([ks.to_host(o[1]) for o in outs if o[1].shape[0] > 0])
    return o0, o1


@pytest.mark.parametrize("logN,nq,kp,dnum,G,levels", [
    (13, 10, 4, 3, 2, [10, 5]),
    (13, 10, 4, 3, 3, [10, 5, 1]),      # at level 5 the last rank owns special towers only
    (12, 7, 3, 7, 4, [7, 2]),           # alpha 1; one rank's special range is empty
    (16, 24, 8, 3, 4, [24, 17]),        # the benchmark's parameter set
])
def test_tower_sharded_keyswitch_matches_oracle(logN, nq, kp, dnum, G, levels):
    need_gpu()
    ks = built_lib()
    P, C = pair(logN, nq, kp, dnum)
    s, sp = secret_pair(C.N, seed=61)
    evk = C.keygen(s, sp, seed=62)
    key = P.upload_key(evk)
    for nact in levels:
        d = inputs.uniform_towers(C.q[:nact], C.N, seed=630 + nact)
        w0, w1 = C.keyswitch(nact, d, evk)
        o0, o1 = _run(P, key, G, nact, d)
        assert np.array_equal(o0, w0) and np.array_equal(o1, w1), (G, nact)


def test_shard_key_refused_by_plain_calls_and_bad_ranges():
    need_gpu()
    ks = built_lib()
    P, C = pair(11, 4, 2, 2)
    s, sp = secret_pair(C.N, seed=71)
    key = P.upload_key(C.keygen(s, sp, seed=72))
    sk = P.key_shard(key, ks.Shard(0, 2, 0, 1))
    d = ks.to_device(inputs.uniform_towers(C.q, C.N, seed=73))
    with pytest.raises(RuntimeError, match="tower shard"):
        P.switch(sk, 4, d, ks.empty((4, C.N)), ks.empty((4, C.N)), "OC")
    with pytest.raises(RuntimeError, match="shard ranges"):
        P.key_shard(key, ks.Shard(3, 5, 0, 1))
    with pytest.raises(RuntimeError, match="tower shard"):
        P.shard_keyprod(key, 4, d, d, ks.empty((2, 3, C.N)), ks.empty((C.N * 8,)))
