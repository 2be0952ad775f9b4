"""Profiling driver: run a few key switches through the C ABI and exit.

Used under ncu (the launch list and single-kernel captures under profiles/):
    python -m paper_2311_01598_gb300.profile_ks --dataflow OC,MP
    python -m paper_2311_01598_gb300.profile_ks --dataflow OC --batch 16
    python -m paper_2311_01598_gb300.profile_ks --batch 4 --keys 4 --schedule 2,2,64,0
Key generation runs first (a few launches), then one key switch per
dataflow listed (or one batched call per dataflow with --batch B > 1).
"""
from __future__ import annotations

import argparse

import torch

from . import inputs, ks


def main():
    """Run the key switches to be profiled (see the module docstring)."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--dataflow", default="OC")
    ap.add_argument("--logN", type=int, default=16)
    ap.add_argument("--nq", type=int, default=24)
    ap.add_argument("--kp", type=int, default=8)
    ap.add_argument("--dnum", type=int, default=3)
    ap.add_argument("--level", type=int, default=0)
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--keys", type=int, default=1, help="distinct keys, used round-robin by the batch")
    ap.add_argument("--schedule", default=None,
                    help="'dataflow,oc_variant,chunk,order': one batched call with this schedule")
    a = ap.parse_args()
    P = ks.Params(a.logN, a.nq, a.kp, a.dnum)
    nact = a.level or a.nq
    s = inputs.ternary_secret(P.N, 1)
    keys = [P.key_synthetic(7 + k) if k else P.keygen(s, inputs.galois_secret(s, 5), 7) for k in range(a.keys)]
    jobs = []
    for i in range(a.batch):
        d = ks.to_device(inputs.uniform_towers(P.q[:nact], P.N, 3 + i))
        jobs.append((keys[i % a.keys], nact, d, ks.empty((nact, P.N)), ks.empty((nact, P.N))))
    if a.schedule:
        P.switch_batch_sched(jobs, ks.Schedule(*[int(x) for x in a.schedule.split(",")]))
    else:
        for df in a.dataflow.split(","):
            if a.batch == 1:
                P.switch(keys[0], nact, jobs[0][2], jobs[0][3], jobs[0][4], df)
            else:
                P.switch_batch(jobs, df)
    torch.cuda.synchronize()
    print("ok launches", ks.kernel_launches())


if __name__ == "__main__":
    main()
