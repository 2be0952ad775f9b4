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
    rows = [{"logN": 16, "nq": 24, "dnum": 3, "kp": 8, "batch": 16, "ms": [float(i + 1) for i in range(12)],
             "best": 0}]
    X, T = tune.arrays(rows)
    assert X.shape == (1, len(tune.FEATURE_NAMES)) and T.shape == (1, 12)
    assert np.all(np.abs(X) < 3)
    assert math.isclose(float(T[0, 0]), math.log(1 / 16), rel_tol=1e-6)


def test_committed_dataset_shape():
    path = os.path.join(tune.DATA_DIR, "tune_gb300.jsonl")
    if not os.path.exists(path):
        return
    rows = tune.load(path)
    n_timings = sum(len(r["ms"]) for r in rows)
    assert n_timings >= 4000
    for r in rows:
        assert r["best"] == int(np.argmin(r["ms"]))
