"""Serving engine: continuous batching with HBM-budget admission.  Every
request's result equals the library's stand-alone key switch (itself pinned
to the oracle) whether it ran alone or in a mixed stream of two ring degrees
with admission pressure."""
import numpy as np
import pytest

from paper_2311_01598_gb300 import inputs
from tests._gpu import built_lib, need_gpu, pair

pytestmark = pytest.mark.gpu


def _setup(ks, logN, nq, kp, dnum, nkeys, seed):
    P, C = pair(logN, nq, kp, dnum)
    s = inputs.ternary_secret(C.N, seed)
    evks = [C.keygen(s, inputs.galois_secret(s, g), seed=g) for g in inputs.galois_elements(C.N, nkeys, seed + 1)]
    return P, C, evks, [P.upload_key(e) for e in evks]


def test_results_alone_equal_results_in_the_mix():
    torch = need_gpu()
    ks = built_lib()
    A = _setup(ks, 12, 8, 2, 3, 2, 1)
    B = _setup(ks, 13, 10, 3, 3, 2, 2)
    rng = np.random.default_rng(5)
    reqs, alone, bufs = [], [], []
    for i in range(24):
        P, C, evks, keys = A if rng.random() < 0.6 else B
        nact = int(rng.integers(1, P.nq + 1))
        k = int(rng.integers(0, len(keys)))
        d = ks.to_device(inputs.uniform_towers(C.q[:nact], C.N, seed=500 + i))
        o0, o1 = ks.empty((nact, C.N)), ks.empty((nact, C.N))
        w0, w1 = ks.empty((nact, C.N)), ks.empty((nact, C.N))
        P.switch(keys[k], nact, d, w0, w1, "OC")
        torch.cuda.synchronize()
        alone.append((ks.to_host(w0), ks.to_host(w1)))
        bufs.append((d, o0, o1))
        reqs.append(ks.Server.request(P, keys[k], nact, d, o0, o1))
    # tight budget: at most a few requests fit at once, forcing admission waits
    srv = ks.Server(max_inflight_jobs=6, max_batch=4, n_streams=2, hbm_budget_bytes=48 << 20)
    arrivals = np.cumsum(rng.exponential(2e-4, size=len(reqs)))
    lat = srv.run_trace(reqs, arrivals)
    st = srv.stats()
    srv.close()
    assert st["done"] == len(reqs) and st["batches"] >= 2 and st["max_batch"] <= 4
    assert np.all(lat > 0)
    for (d, o0, o1), (w0, w1) in zip(bufs, alone):
        assert np.array_equal(ks.to_host(o0), w0) and np.array_equal(ks.to_host(o1), w1)


def test_submit_wait_and_admission_limits():
    torch = need_gpu()
    ks = built_lib()
    P, C, evks, keys = _setup(ks, 14, 12, 4, 3, 1, 3)
    srv = ks.Server(max_inflight_jobs=1, max_batch=1, n_streams=1, hbm_budget_bytes=64 << 20)
    tickets, outs = [], []
    for i in range(5):
        d = ks.to_device(inputs.uniform_towers(C.q, C.N, seed=700 + i))
        o0, o1 = ks.empty((12, C.N)), ks.empty((12, C.N))
        outs.append((d, o0, o1))
        tickets.append(srv.submit(P, keys[0], 12, d, o0, o1))
    assert srv.wait(tickets[-1], 0) in (ks.KS_ETIMEOUT, ks.KS_OK)
    for t in tickets:
        assert srv.wait(t, 60000) == ks.KS_OK
    times = [srv.times(t) for t in tickets]
    # one slot: each request is admitted only after the previous finished
    for (a0, m0, d0), (a1, m1, d1) in zip(times, times[1:]):
        assert m1 >= d0 - 1e-3
    st = srv.stats()
    srv.close()
    assert st["done"] == 5 and st["max_batch"] == 1
    for d, o0, o1 in outs:
        w0, w1 = ks.empty((12, C.N)), ks.empty((12, C.N))
        P.switch(keys[0], 12, d, w0, w1, "OC")
        assert torch.equal(w0, o0) and torch.equal(w1, o1)


def test_submit_rejects_misaligned_and_overlapping_buffers():
    """Requests with buffers the kernels cannot take (not 16-byte aligned,
    or outputs overlapping the input) are refused at submission; the server
    keeps serving valid requests."""
    torch = need_gpu()
    ks = built_lib()
    P, C, evks, keys = _setup(ks, 12, 4, 2, 2, 1, 4)
    srv = ks.Server(max_inflight_jobs=4, max_batch=4, n_streams=1, hbm_budget_bytes=64 << 20)
    d = ks.to_device(inputs.uniform_towers(C.q, C.N, seed=720))
    o0, o1 = ks.empty((4, C.N)), ks.empty((4, C.N))
    flat = torch.zeros(4 * C.N + 1, dtype=torch.int64, device="cuda")
    shifted = flat[1:].view(4, C.N)
    with pytest.raises(RuntimeError, match="16-byte aligned"):
        srv.submit(P, keys[0], 4, shifted, o0, o1)
    with pytest.raises(RuntimeError, match="overlap"):
        srv.submit(P, keys[0], 4, d, d, o1)
    t = srv.submit(P, keys[0], 4, d, o0, o1)
    assert srv.wait(t, 60000) == ks.KS_OK
    srv.close()
    w0, w1 = ks.empty((4, C.N)), ks.empty((4, C.N))
    P.switch(keys[0], 4, d, w0, w1, "OC")
    assert torch.equal(w0, o0) and torch.equal(w1, o1)
