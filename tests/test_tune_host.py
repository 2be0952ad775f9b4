"""Host-side checks of the schedule-selection pipeline (no GPU)."""
import math
import os

import numpy as np

from paper_2311_01598_gb300 import tune


def test_workload_sampler_respects_domain_and_cap():
    rng = np.random.default_rng(0)
    for _ in range(500):
        logN, nq, dnum, kp, batch = tune.sample_workload(rng)
        assert 13 <= logN <= 17 and 2 <= nq <= 48 and 1 <= dnum <= nq and 1 <= kp <= 12
        assert 1 <= batch <= 256 and (batch == 1 or batch * nq * (1 << logN) <= tune.WORDS_CAP)


def test_features_and_targets():
    rows = [{"logN": 16, "nq": 24, "dnum": 3, "kp": 8, "batch": 16, "ms": [float(i + 1) for i in range(13)],
             "best": 0, "base": 0, "impl_ms": [2.0, 3.0, 4.0, 5.0], "best_impl": 0}]
    X, T = tune.arrays(rows)
    assert X.shape == (1, len(tune.FEATURE_NAMES)) and T.shape == (1, 13 + 4)
    assert np.all(np.abs(X) < 3)
    assert math.isclose(float(T[0, 0]), math.log(1 / 16), rel_tol=1e-6)
    assert math.isclose(float(T[0, 13]), math.log(2 / 16), rel_tol=1e-6)


def test_committed_dataset_shape():
    """The committed GB300 timings: 13 structural candidates and the four
    implementation pairs per workload, over 5000 timings in all."""
    path = os.path.join(tune.DATA_DIR, "tune_gb300.jsonl")
    assert os.path.exists(path)
    rows = tune.load(path)
    n_timings = sum(len(r["ms"]) + len(r["impl_ms"]) for r in rows)
    assert n_timings >= 5000
    for r in rows:
        assert len(r["ms"]) == 13 and len(r["impl_ms"]) == 4
        assert r["best"] == int(np.argmin(r["ms"])) and r["best_impl"] == int(np.argmin(r["impl_ms"]))
        assert 0 <= r["base"] < 13


def test_impl_pairs_match_the_library_order():
    """The model's last four outputs are the implementation pairs in the
    order the library's stage 2 times them (ks.h: {(0,1), (1,1), (0,0),
    (1,0)})."""
    hdr = open(os.path.join(os.path.dirname(tune.HERE), "include", "ks.h")).read()
    assert "{(0,1), (1,1), (0,0), (1,0)}" in hdr
    assert tune.IMPL_PAIRS == ((0, 1), (1, 1), (0, 0), (1, 0))


def test_implementation_flags_follow_the_kernels_limits():
    """The last three inputs flag which implementations exist for a shape:
    the tensor-core base conversion up to 18 sources (two K blocks) for
    ModUp (the parameter set's alpha) and ModDown (K), the cluster NTT at
    ring degrees other than 2^13 and 2^17."""
    def flags(logN, nq, dnum, kp, alpha_params=None):
        return tuple(float(x) for x in tune.features(logN, nq, dnum, kp, 16, alpha_params)[-3:])
    assert flags(16, 24, 3, 8) == (1.0, 1.0, 1.0)              # alpha 8, K 8
    assert flags(17, 36, 3, 12) == (1.0, 1.0, -1.0)            # alpha 12, K 12: two K blocks; no 2^17 cluster
    assert flags(16, 36, 2, 18) == (1.0, 1.0, 1.0)             # alpha 18, K 18: the limit
    assert flags(16, 38, 2, 19) == (-1.0, -1.0, 1.0)           # alpha 19, K 19: CUDA cores only
    assert flags(13, 24, 1, 8, alpha_params=12) == (1.0, 1.0, -1.0)  # the parameter set's alpha decides
    assert flags(14, 40, 2, 20) == (-1.0, -1.0, 1.0)
