"""Autotuner and learned cost model on the GPU.

* the MLP's forward pass and gradients (library kernels, FP32) agree with
  the float64 oracle MLP (relative error <= 1e-3);
* Adam steps reduce the loss;
* ks_autotune returns the fastest candidate it timed, caches it, and KS_AUTO
  then runs that schedule with the oracle's results;
* on the committed GB300 timing dataset, the model trained by the library's
  kernels picks schedules within 5% of the exhaustive search on held-out
  workloads and beats the fixed default schedule;
* attached to a parameter set, the committed model is what KS_AUTO runs on
  a tuning-cache miss: its pick is cached and executed with the oracle's
  results, and the library's features equal the training code's.
"""
import os
import tempfile

import numpy as np
import pytest

from oracle import mlp_oracle as mo
from paper_2311_01598_gb300 import inputs
from tests._gpu import built_lib, need_gpu, pair

pytestmark = pytest.mark.gpu
DIMS = [10, 64, 64, 64, 17]


def _batch(seed, n=37):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, DIMS[0])).astype(np.float32)
    T = rng.normal(size=(n, DIMS[-1])).astype(np.float32)
    M = (rng.random((n, DIMS[-1])) > 0.25).astype(np.float32)
    return X, T, M


def test_mlp_forward_and_gradients_match_oracle():
    torch = need_gpu()
    ks = built_lib()
    mlp = ks.Mlp(DIMS, seed=11)
    p = mlp.get_params().astype(np.float64)
    X, T, M = _batch(1)
    x, t, m = (torch.from_numpy(a).cuda() for a in (X, T, M))
    y = mlp.forward(x).cpu().numpy()
    y_ref = mo.forward(p, DIMS, X)[-1]
    assert np.max(np.abs(y - y_ref)) <= 1e-4 * max(1.0, np.max(np.abs(y_ref)))
    for mask, mref in ((None, None), (m, M)):
        loss, g = mlp.gradients(x, t, mask)
        L_ref, g_ref = mo.gradients(p, DIMS, X, T, mref)
        assert abs(loss - L_ref) <= 1e-4 * max(1.0, abs(L_ref))
        assert np.linalg.norm(g - g_ref) <= 1e-3 * np.linalg.norm(g_ref)
        assert np.max(np.abs(g - g_ref)) <= 1e-3 * np.max(np.abs(g_ref))


def test_mlp_training_reduces_loss():
    torch = need_gpu()
    ks = built_lib()
    rng = np.random.default_rng(3)
    X = rng.normal(size=(256, DIMS[0])).astype(np.float32)
    W = rng.normal(size=(DIMS[0], DIMS[-1])).astype(np.float32)
    T = np.tanh(X @ W).astype(np.float32)
    x, t = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    mlp = ks.Mlp(DIMS, seed=2)
    first = mlp.train_step(x, t, 3e-3)
    for _ in range(300):
        last = mlp.train_step(x, t, 3e-3)
    assert last < 0.1 * first


def test_autotune_caches_fastest_and_auto_uses_it():
    need_gpu()
    ks = built_lib()
    P, C = pair(12, 5, 2, 2)
    s = inputs.ternary_secret(C.N, 4)
    evk = C.keygen(s, inputs.galois_secret(s, 5), seed=4)
    key = P.upload_key(evk)
    jobs, want = [], []
    for i in range(6):
        d = inputs.uniform_towers(C.q, C.N, seed=200 + i)
        want.append(C.keyswitch(5, d, evk))
        jobs.append((key, 5, ks.to_device(d), ks.empty((5, C.N)), ks.empty((5, C.N))))
    cands = P.tune_candidates()
    assert all(c.impl() == (-1, -1) for c in cands)
    best, ms = P.autotune(jobs, reps=2)
    # stage 1 picks the structure (the largest launch group among those
    # within 0.3% of the fastest), stage 2 an explicit implementation pair
    # (bounds a hair apart: the library compares in float)
    assert len(ms) == len(cands)
    loose = [c.as_tuple() for c, m in zip(cands, ms) if m <= min(ms) * 1.0031]
    tight = [c.chunk for c, m in zip(cands, ms) if m <= min(ms) * 1.0029]
    assert best.as_tuple() in loose and best.chunk >= max(tight)
    assert best.impl() in ((0, 1), (1, 1), (0, 0), (1, 0))
    cached = P.tune_cache_get(6, 5)
    assert cached is not None and cached.as_tuple() == best.as_tuple() and cached.impl() == best.impl()
    for (_, _, _, o0, o1) in jobs:   # clear, then run KS_AUTO (the cached schedule)
        o0.zero_()
        o1.zero_()
    P.switch_batch(jobs, "AUTO")
    for (_, _, _, o0, o1), (w0, w1) in zip(jobs, want):
        assert np.array_equal(ks.to_host(o0), w0) and np.array_equal(ks.to_host(o1), w1)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "cache.txt")
        P.tune_cache_save(path)
        P2 = ks.Params(12, 5, 2, 2)
        P2.tune_cache_load(path)
        got = P2.tune_cache_get(6, 5)
        assert got.as_tuple() == best.as_tuple() and got.impl() == best.impl()
        # a line of the four-field format loads with the options' implementation
        with open(path) as f:
            line = [l for l in f if "sched=" in l and not l.startswith("#")][0]
        with open(path, "w") as f:
            f.write(line.split("sched=")[0] + "sched=2,1,8,0\n")
        P3 = ks.Params(12, 5, 2, 2)
        P3.tune_cache_load(path)
        got = P3.tune_cache_get(6, 5)
        assert got.as_tuple() == (2, 1, 8, 0) and got.impl() == (-1, -1)


def test_autotune_impl_times_four_implementations():
    """Stage 2 alone: the four (ntt, bconv) pairs of a structure are timed,
    the fastest is returned, and every pair gives the oracle's outputs."""
    need_gpu()
    ks = built_lib()
    P, C = pair(12, 5, 2, 2)
    s = inputs.ternary_secret(C.N, 14)
    evk = C.keygen(s, inputs.galois_secret(s, 3), seed=14)
    key = P.upload_key(evk)
    jobs, want = [], []
    for i in range(4):
        d = inputs.uniform_towers(C.q, C.N, seed=240 + i)
        want.append(C.keyswitch(5, d, evk))
        jobs.append((key, 5, ks.to_device(d), ks.empty((5, C.N)), ks.empty((5, C.N))))
    base = ks.Schedule(2, 2, 64, 0)
    best, ms = P.autotune_impl(jobs, base, reps=2)
    pairs = [(0, 1), (1, 1), (0, 0), (1, 0)]
    assert len(ms) == 4 and best.impl() == pairs[int(np.argmin(ms))] and best.as_tuple() == base.as_tuple()
    for pr in pairs:
        for (_, _, _, o0, o1) in jobs:
            o0.zero_()
            o1.zero_()
        P.switch_batch_sched(jobs, ks.Schedule(2, 2, 64, 0, *pr))
        for (_, _, _, o0, o1), (w0, w1) in zip(jobs, want):
            assert np.array_equal(ks.to_host(o0), w0) and np.array_equal(ks.to_host(o1), w1), pr


def test_learned_schedule_on_the_execution_path():
    """A cold tuning cache plus KS_AUTO: the library runs the attached cost
    model (its forward kernel), caches the predicted schedule under the
    batch's signature and executes it; every output equals the oracle's.
    The pick equals ks_predict_schedule's and tune.choose's, and the
    library's model inputs equal the training code's features."""
    need_gpu()
    ks = built_lib()
    from paper_2311_01598_gb300 import tune
    model = tune.CostModel.load(os.path.join(tune.DATA_DIR, "cost_model_gb300.npz"))
    P, C = pair(13, 8, 3, 2)
    s = inputs.ternary_secret(C.N, 51)
    evk = C.keygen(s, inputs.galois_secret(s, 3), seed=52)
    key = P.upload_key(evk)
    jobs, want = [], []
    for i in range(5):
        d = inputs.uniform_towers(C.q, C.N, seed=530 + i)
        want.append(C.keyswitch(8, d, evk))
        jobs.append((key, 8, ks.to_device(d), ks.empty((8, C.N)), ks.empty((8, C.N))))
    assert np.allclose(P.cost_features(jobs), tune.features(13, 8, 2, 3, 5, P.alpha), rtol=0, atol=1e-6)
    assert P.tune_cache_get(5, 8) is None
    P.switch_batch(jobs, "AUTO")            # no model: the default schedule
    assert P.tune_cache_get(5, 8) is None
    P.set_cost_model(model.mlp, model.t_mean, model.t_scale)
    pick, pred = P.predict_schedule(jobs)
    assert len(pred) == len(P.tune_candidates()) + 4
    ref = tune.choose(model, P, 5, P.tune_candidates())
    assert pick.as_tuple() == ref.as_tuple() and pick.impl() == ref.impl()
    for (_, _, _, o0, o1) in jobs:
        o0.zero_()
        o1.zero_()
    P.switch_batch(jobs, "AUTO")            # cache miss: the model's pick, cached
    got = P.tune_cache_get(5, 8)
    assert got is not None and got.as_tuple() == pick.as_tuple() and got.impl() == pick.impl()
    for (_, _, _, o0, o1), (w0, w1) in zip(jobs, want):
        assert np.array_equal(ks.to_host(o0), w0) and np.array_equal(ks.to_host(o1), w1)
    # a batch at lower levels: the model's inputs use the mean level and the active digits
    low = [(key, 5, ks.to_device(inputs.uniform_towers(C.q[:5], C.N, seed=540)), ks.empty((5, C.N)),
            ks.empty((5, C.N))), (key, 3, ks.to_device(inputs.uniform_towers(C.q[:3], C.N, seed=541)),
                                  ks.empty((3, C.N)), ks.empty((3, C.N)))]
    assert np.allclose(P.cost_features(low), tune.features(13, 4, 1, 3, 2, P.alpha), rtol=0, atol=1e-6)
    P.switch_batch(low, "AUTO")
    for (_, nact, d, o0, o1) in low:
        w0, w1 = C.keyswitch(nact, ks.to_host(d), evk)
        assert np.array_equal(ks.to_host(o0), w0) and np.array_equal(ks.to_host(o1), w1)
    # the host-buffer path consults the model per chunk the same way
    torch = need_gpu()
    hjobs, hwant = [], []
    for i in range(3):
        d = inputs.uniform_towers(C.q[:6], C.N, seed=550 + i)
        hwant.append(C.keyswitch(6, d, evk))
        hjobs.append((key, 6, torch.from_numpy(d.view(np.int64)).pin_memory(),
                      torch.zeros((6, C.N), dtype=torch.int64).pin_memory(),
                      torch.zeros((6, C.N), dtype=torch.int64).pin_memory()))
    assert P.tune_cache_get(3, 6) is None
    P.switch_batch_host(hjobs, "AUTO")
    torch.cuda.synchronize()
    assert P.tune_cache_get(3, 6) is not None
    for (_, _, _, h0, h1), (w0, w1) in zip(hjobs, hwant):
        assert np.array_equal(h0.numpy().view(np.uint64), w0) and np.array_equal(h1.numpy().view(np.uint64), w1)
    P.set_cost_model(None)


def test_host_auto_takes_the_whole_calls_schedule():
    """ks_switch_batch_host with KS_AUTO: chunks whose own shape has no tuned
    entry run the schedule tuned for the whole call (here MP, told apart from
    the default schedule by its launch count), with the oracle's results."""
    torch = need_gpu()
    ks = built_lib()
    P, C = pair(12, 5, 2, 2)
    s = inputs.ternary_secret(C.N, 41)
    evk = C.keygen(s, inputs.galois_secret(s, 5), seed=6)
    key = P.upload_key(evk)
    n = 10  # two chunks of 5
    hjobs, djobs, want = [], [], []
    for i in range(n):
        d = inputs.uniform_towers(C.q, C.N, seed=700 + i)
        want.append(C.keyswitch(5, d, evk))
        hjobs.append((key, 5, torch.from_numpy(d.view(np.int64)).pin_memory(),
                      torch.zeros((5, C.N), dtype=torch.int64).pin_memory(),
                      torch.zeros((5, C.N), dtype=torch.int64).pin_memory()))
        djobs.append((key, 5, ks.to_device(d), ks.empty((5, C.N)), ks.empty((5, C.N))))
    mp = ks.Schedule(ks.MP, 1, 64, 0)
    P.tune_cache_put(n, 5, mp)
    assert P.tune_cache_get(5, 5) is None

    def launches(fn):
        torch.cuda.synchronize()
        l0 = ks.kernel_launches()
        fn()
        torch.cuda.synchronize()
        return ks.kernel_launches() - l0

    per_chunk = {name: launches(lambda sc=sc: P.switch_batch_sched(djobs[:5], sc))
                 for name, sc in (("mp", mp), ("default", P.default_schedule()))}
    assert per_chunk["mp"] != per_chunk["default"]
    assert launches(lambda: P.switch_batch_host(hjobs, "AUTO")) == 2 * per_chunk["mp"]
    assert P.tune_cache_get(5, 5) is None
    for (_, _, _, h0, h1), (w0, w1) in zip(hjobs, want):
        assert np.array_equal(h0.numpy().view(np.uint64), w0) and np.array_equal(h1.numpy().view(np.uint64), w1)


def test_cost_model_regret_on_gb300_dataset():
    """Held-out regret of the learned schedule <= 5% of the exhaustive
    autotuner's best, and less total time than the fixed default schedule."""
    need_gpu()
    ks = built_lib()
    from paper_2311_01598_gb300 import tune
    path = os.path.join(tune.DATA_DIR, "tune_gb300.jsonl")
    if not os.path.exists(path):
        pytest.skip("no committed timing dataset")
    rows = tune.load(path)
    train_rows, test_rows = tune.split(rows, 0.8, seed=0)
    model, _ = tune.train(train_rows, epochs=3000)
    P = ks.Params(12, 3, 1, 3, prime_bits=50)
    di = tune.default_candidate_index(P.tune_candidates(), P.default_schedule())
    ev = tune.evaluate(model, test_rows, di)
    assert ev["model_time_over_best"] <= 0.05, ev
    assert ev["model_time_over_best"] < ev["default_time_over_best"], ev
    assert ev["impl_time_over_best"] <= 0.05, ev
