"""Serving benchmark: a Poisson stream of key-switch requests through the
continuous-batching server (ks_server_*), swept over arrival rates.

Mix: 70% N=2^16 (L+1 uniform in 4..24 of 24 Q primes, K=8, dnum=3) and
30% N=2^17 (L+1 uniform in 8..36 of 36 Q primes, K=12, dnum=3, 288 MiB
keys); 4 device-resident keys per ring degree; requests in device memory.
For each rate: throughput (requests/s) and latency percentiles (arrival to
completion, host clock of the server).

    python -m paper_2311_01598_gb300.serve_bench --rates 500,1000,2000,3000 --n 1500
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def build_mix(seed=0, n_bufsets=96):
    """Parameter sets, device-resident keys and reusable buffers of the serving mix."""
    import torch

    from . import inputs, ks
    p16 = ks.Params(16, 24, 8, 3)
    p17 = ks.Params(17, 36, 12, 3)
    keys16 = [p16.key_synthetic(100 + i) for i in range(4)]
    keys17 = [p17.key_synthetic(200 + i) for i in range(4)]
    bufs16 = [(torch.randint(0, min(p16.q), (24, p16.N), dtype=torch.int64, device="cuda"),
               ks.empty((24, p16.N)), ks.empty((24, p16.N))) for _ in range(n_bufsets)]
    bufs17 = [(torch.randint(0, min(p17.q), (36, p17.N), dtype=torch.int64, device="cuda"),
               ks.empty((36, p17.N)), ks.empty((36, p17.N))) for _ in range(n_bufsets // 2)]
    del inputs
    return p16, p17, keys16, keys17, bufs16, bufs17


def make_trace(mix, n, rate, seed):
    """n requests of the mix with Poisson arrival times at the given rate."""
    from . import inputs, ks
    p16, p17, keys16, keys17, bufs16, bufs17 = mix
    rng = np.random.default_rng(seed)
    reqs, kinds = [], []
    for i in range(n):
        if rng.random() < 0.7:
            nact = int(rng.integers(4, 25))
            d, o0, o1 = bufs16[i % len(bufs16)]
            reqs.append(ks.Server.request(p16, keys16[int(rng.integers(0, 4))], nact, d, o0, o1))
            kinds.append(16)
        else:
            nact = int(rng.integers(8, 37))
            d, o0, o1 = bufs17[i % len(bufs17)]
            reqs.append(ks.Server.request(p17, keys17[int(rng.integers(0, 4))], nact, d, o0, o1))
            kinds.append(17)
    arrivals = inputs.poisson_arrivals(rate, n, seed + 1)
    return reqs, arrivals - arrivals[0], np.array(kinds)


def run(rates, n, seed=0, slots=48, batch=16, lanes=3, budget_gib=24):
    """Replay one trace per offered rate through a fresh server; one result dict per rate."""
    from . import ks
    mix = build_mix(seed)
    out = []
    for r, rate in enumerate(rates):
        reqs, arr, kinds = make_trace(mix, n, rate, seed + 10 * r)
        srv = ks.Server(max_inflight_jobs=slots, max_batch=batch, n_streams=lanes,
                        hbm_budget_bytes=int(budget_gib * (1 << 30)))
        lat = srv.run_trace(reqs, arr)
        st = srv.stats()
        srv.close()
        span = float(arr[-1] + lat[-1]) if n else 0.0
        row = {"offered_rate": rate, "n": n, "throughput_rps": round(n / max(span, 1e-9), 1),
               "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
               "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3),
               "p50_ms_N16": round(float(np.percentile(lat[kinds == 16], 50)) * 1e3, 3),
               "p50_ms_N17": round(float(np.percentile(lat[kinds == 17], 50)) * 1e3, 3),
               "batches": st["batches"], "max_batch": st["max_batch"],
               "config": {"slots": slots, "max_batch": batch, "lanes": lanes, "hbm_budget_gib": budget_gib}}
        print(json.dumps(row), flush=True)
        out.append(row)
    return out


def main():
    """Command line: one JSON line per offered rate."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", default="500,1000,2000,3000,4000")
    ap.add_argument("--n", type=int, default=1500)
    ap.add_argument("--slots", type=int, default=48)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lanes", type=int, default=3)
    a = ap.parse_args()
    run([float(x) for x in a.rates.split(",")], a.n, slots=a.slots, batch=a.batch, lanes=a.lanes)


if __name__ == "__main__":
    main()
