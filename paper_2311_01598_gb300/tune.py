"""Schedule selection: exhaustive autotuning data and the learned cost model.

* ``collect``: sample workloads of the cost model's domain (logN 13-17, L+1
  2-48, dnum 1..L+1, K 1-12, batch 1-256, capped so one batch holds at most
  2^16*24*16 words of input; uniformly, or near the paper-sized parameter
  sets with ``--anchors``), time every structural candidate schedule of
  each and then the fastest structure under the four implementation pairs
  (NTT form x base-conversion engine) with ``ks_autotune`` (CUDA events, best
  of k), and write one JSON line per workload.
* ``train``: fit the FP32 MLP (7 inputs -> 3 x 64 ReLU -> one predicted
  log-time per structural candidate, then one per implementation pair) on
  those timings with the library's own forward, backward and Adam kernels.
* ``evaluate``: for held-out workloads, pick the structure and the
  implementation pair with the lowest predicted times and report the regret
  against the measured best (the exhaustive search), as a fraction and in
  microseconds, and against the fixed default schedule.

At run time the library itself runs the model: attached to a parameter set
(``Params.set_cost_model``), it is consulted by ``KS_AUTO`` on a
tuning-cache miss and its pick is cached and executed.  ``choose`` gives the
same pick from Python.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DATA_DIR = os.path.join(HERE, "data")
HIDDEN = (64, 64, 64)
IMPL_PAIRS = ((0, 1), (1, 1), (0, 0), (1, 0))  # (ntt, bconv) in the library's stage-2 order
FEATURE_NAMES = ("logN", "L+1", "dnum", "K", "log2 batch", "alpha", "log2 words", "tensor-core ModUp BConv",
                 "tensor-core ModDown BConv", "cluster NTT")
WORDS_CAP = (1 << 16) * 24 * 16


def features(logN, nq, dnum, kp, batch, alpha_params=None):
    """Model inputs: the workload's sizes scaled to roughly unit range by
    fixed constants, then +-1 flags of which implementations exist for the
    shape (tensor-core ModUp base conversion: at most 18 sources per digit,
    alpha_params being the parameter set's alpha, by default ceil(nq/dnum);
    tensor-core ModDown: at most 18 special towers; cluster NTT: ring degrees
    other than 2^13 and 2^17).  The library computes the same vector
    (ks_cost_features)."""
    alpha = -(-nq // dnum)
    ap = alpha if alpha_params is None else alpha_params
    words = batch * nq * (1 << logN)
    return np.array([(logN - 15) / 2.0, (nq - 25) / 14.0, (dnum - 12) / 12.0, (kp - 6.5) / 3.5,
                     (math.log2(batch) - 4) / 2.5, (alpha - 12) / 12.0, (math.log2(words) - 22) / 3.0,
                     1.0 if ap <= 18 else -1.0, 1.0 if kp <= 18 else -1.0, 1.0 if logN not in (13, 17) else -1.0],
                    dtype=np.float32)


def sample_workload(rng):
    """One workload (logN, nq, dnum, kp, batch) of the cost-model domain."""
    logN = int(rng.integers(13, 18))
    nq = int(rng.integers(2, 49))
    dnum = int(rng.integers(1, nq + 1))
    kp = int(rng.integers(1, 13))
    batch = int(round(2 ** rng.uniform(0, 8)))
    batch = max(1, min(batch, WORDS_CAP // (nq << logN)))
    return logN, nq, dnum, kp, batch


# Parameter sets of the paper's size inside the model's domain (logN, L+1,
# K, dnum): the benchmark set, ARK and DPRIVE (Table III), the serving mix's
# N = 2^17 set.
ANCHORS = ((16, 24, 8, 3), (16, 24, 6, 4), (16, 26, 7, 3), (17, 36, 12, 3))


def sample_anchor(rng):
    """One workload near a paper-sized parameter set: L+1 within 4 and K
    within 2 of an anchor, dnum within 1, batch log-uniform 1..128."""
    logN, nq0, kp0, d0 = ANCHORS[int(rng.integers(0, len(ANCHORS)))]
    nq = int(np.clip(nq0 + rng.integers(-4, 5), 2, 48))
    kp = int(np.clip(kp0 + rng.integers(-2, 3), 1, 12))
    dnum = int(np.clip(d0 + rng.integers(-1, 2), 1, nq))
    batch = int(round(2 ** rng.uniform(0, 7)))
    batch = max(1, min(batch, WORDS_CAP // (nq << logN)))
    return logN, nq, dnum, kp, batch


def collect(n_workloads, seed, out_path, reps=2, log=print, anchors=False):
    """Time every candidate schedule on n_workloads sampled workloads
    (uniform over the domain, or near the paper-sized sets with anchors)."""
    import torch

    from . import ks
    rng = np.random.default_rng(seed)
    t0 = time.time()
    with open(out_path, "w") as f:
        for w in range(n_workloads):
            logN, nq, dnum, kp, batch = (sample_anchor if anchors else sample_workload)(rng)
            P = ks.Params(logN, nq, kp, dnum)
            key = P.key_synthetic(seed * 1000 + w)
            qmin = min(P.q)
            jobs = []
            for b in range(batch):
                d = torch.randint(0, qmin, (nq, P.N), dtype=torch.int64, device="cuda")
                jobs.append((key, nq, d, ks.empty((nq, P.N)), ks.empty((nq, P.N))))
            cands = [c.as_tuple() for c in P.tune_candidates()]
            best, ms = P.autotune(jobs, reps=reps, with_impl=True)
            ms_s, ms_i = ms[:len(cands)], ms[len(cands):]
            row = {"logN": logN, "nq": nq, "dnum": dnum, "kp": kp, "batch": batch,
                   "ms": [round(m, 5) for m in ms_s], "best": int(np.argmin(ms_s)),
                   "base": cands.index(best.as_tuple()),
                   "impl_ms": [round(m, 5) for m in ms_i], "best_impl": int(np.argmin(ms_i)),
                   "sampler": "anchor" if anchors else "uniform"}
            f.write(json.dumps(row) + "\n")
            f.flush()
            del jobs, key, P
            torch.cuda.empty_cache()
            if log and (w + 1) % 25 == 0:
                log(f"collected {w + 1}/{n_workloads} workloads in {time.time() - t0:.0f} s")
    return out_path


def load(path):
    """Rows of a timing dataset (JSON lines)."""
    with open(path) as f:
        return [json.loads(l) for l in f if l.strip()]


def arrays(rows):
    """Features X and targets T: log time per key switch (ms) of every
    structural candidate, then of the autotuner's fastest structure under
    each implementation pair."""
    X = np.stack([features(r["logN"], r["nq"], r["dnum"], r["kp"], r["batch"]) for r in rows])
    T = np.array([[math.log(m / r["batch"]) for m in list(r["ms"]) + list(r["impl_ms"])] for r in rows],
                 dtype=np.float32)
    return X, T


class CostModel:
    """The trained MLP plus the target normalisation (mean, scale)."""

    def __init__(self, mlp, t_mean, t_scale):
        self.mlp, self.t_mean, self.t_scale = mlp, float(t_mean), float(t_scale)

    def predict(self, X):
        """Predicted log time per key switch of every candidate for each row of X."""
        import torch
        x = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        y = self.mlp.forward(x).cpu().numpy()
        return y * self.t_scale + self.t_mean

    def save(self, path):
        """Parameters and target normalisation as .npz."""
        np.savez(path, params=self.mlp.get_params(), dims=np.array(self.mlp.dims), t_mean=self.t_mean,
                 t_scale=self.t_scale)

    @staticmethod
    def load(path):
        """A model saved by save()."""
        from . import ks
        z = np.load(path)
        m = ks.Mlp([int(v) for v in z["dims"]])
        m.set_params(z["params"])
        return CostModel(m, float(z["t_mean"]), float(z["t_scale"]))


def train(rows, epochs=3000, lr=3e-3, seed=1, log=None):
    """Full-batch Adam on the normalised log-times; returns a CostModel."""
    import torch

    from . import ks
    X, T = arrays(rows)
    t_mean, t_scale = float(T.mean()), float(T.std() + 1e-6)
    Tn = (T - t_mean) / t_scale
    dims = [X.shape[1], *HIDDEN, T.shape[1]]
    mlp = ks.Mlp(dims, seed=seed)
    x = torch.from_numpy(X).cuda()
    t = torch.from_numpy(Tn.astype(np.float32)).cuda()
    loss = None
    for ep in range(epochs):
        step_lr = lr * (0.5 * (1 + math.cos(math.pi * ep / epochs)) * 0.9 + 0.1)
        loss = mlp.train_step(x, t, step_lr)
        if log and (ep % 500 == 0 or ep == epochs - 1):
            log(f"epoch {ep} loss {loss:.4f}")
    return CostModel(mlp, t_mean, t_scale), loss


def evaluate(model, rows, default_index):
    """Regret of the model's choices against the measured best, per workload:
    the structure (argmin of the structural outputs, timed with the
    parameter set's default implementation) and the implementation pair
    (argmin of the last four outputs, timed on the autotuner's structure),
    as fractions (0 = optimal) and in microseconds (per batch and per key
    switch); the fixed default schedule beside it."""
    X, _ = arrays(rows)
    pred = model.predict(X)
    ns = len(rows[0]["ms"])
    pick = pred[:, :ns].argmin(axis=1)
    pick_i = pred[:, ns:].argmin(axis=1)
    ms = np.array([r["ms"] for r in rows])
    mi = np.array([r["impl_ms"] for r in rows])
    batch = np.array([r["batch"] for r in rows], dtype=np.float64)
    ar = np.arange(len(rows))
    best, chosen, default = ms.min(axis=1), ms[ar, pick], ms[:, default_index]
    best_i, chosen_i = mi.min(axis=1), mi[ar, pick_i]
    return {"n": len(rows),
            "model_regret_mean": float(np.mean(chosen / best - 1)),
            "model_regret_median": float(np.median(chosen / best - 1)),
            "model_regret_p90": float(np.quantile(chosen / best - 1, 0.9)),
            "model_time_over_best": float(chosen.sum() / best.sum() - 1),
            "model_regret_us_mean": float(np.mean(chosen - best) * 1e3),
            "model_regret_us_per_ks_mean": float(np.mean((chosen - best) / batch) * 1e3),
            "model_regret_us_max": float(np.max(chosen - best) * 1e3),
            "default_regret_mean": float(np.mean(default / best - 1)),
            "default_time_over_best": float(default.sum() / best.sum() - 1),
            "default_regret_us_mean": float(np.mean(default - best) * 1e3),
            "exact_pick_rate": float(np.mean(chosen == best)),
            "impl_regret_mean": float(np.mean(chosen_i / best_i - 1)),
            "impl_time_over_best": float(chosen_i.sum() / best_i.sum() - 1),
            "impl_regret_us_mean": float(np.mean(chosen_i - best_i) * 1e3),
            "impl_exact_pick_rate": float(np.mean(chosen_i == best_i))}


def split(rows, frac=0.8, seed=0):
    """Seeded train/test split of the rows."""
    idx = np.random.default_rng(seed).permutation(len(rows))
    k = int(len(rows) * frac)
    return [rows[i] for i in idx[:k]], [rows[i] for i in idx[k:]]


def default_candidate_index(candidates, default):
    """Index of the default schedule among the candidates."""
    return [c.as_tuple() for c in candidates].index(default.as_tuple())


def choose(model, params, batch, candidates):
    """Schedule the model predicts fastest for a batch of `batch` top-level
    ciphertexts on params (no timing): the structure and the implementation
    pair with the lowest predicted times (the library's KS_AUTO makes the
    same pick with the model attached)."""
    from . import ks
    x = features(params.logN, params.nq, params.dnum, params.kp, batch, params.alpha)[None, :]
    y = model.predict(x)[0]
    ns = len(candidates)
    s = candidates[int(y[:ns].argmin())]
    ntt, bconv = IMPL_PAIRS[int(y[ns:].argmin())]
    return ks.Schedule(s.dataflow, s.oc_variant, s.chunk, s.order, ntt, bconv)


def main():
    """Command line: `collect` timings on the GPU or `train` the cost model."""
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--n", type=int, default=400)
    c.add_argument("--seed", type=int, default=7)
    c.add_argument("--reps", type=int, default=2)
    c.add_argument("--out", default=os.path.join(DATA_DIR, "tune_gb300.jsonl"))
    c.add_argument("--anchors", action="store_true", help="sample near the paper-sized parameter sets")
    t = sub.add_parser("train")
    t.add_argument("--data", default=os.path.join(DATA_DIR, "tune_gb300.jsonl"))
    t.add_argument("--epochs", type=int, default=3000)
    t.add_argument("--out", default=os.path.join(DATA_DIR, "cost_model_gb300.npz"))
    a = ap.parse_args()
    if a.cmd == "collect":
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        collect(a.n, a.seed, a.out, a.reps, anchors=a.anchors)
    else:
        from . import ks
        rows = load(a.data)
        tr, te = split(rows)
        model, loss = train(tr, a.epochs, log=print)
        P = ks.Params(12, 3, 1, 3, prime_bits=50)
        di = default_candidate_index(P.tune_candidates(), P.default_schedule())
        print(json.dumps({"train_loss": loss, "train": evaluate(model, tr, di), "test": evaluate(model, te, di)}))
        model.save(a.out)


if __name__ == "__main__":
    main()
