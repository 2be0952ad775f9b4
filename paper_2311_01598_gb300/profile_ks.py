"""Profiling driver: run a few key switches through the C ABI and exit.

Used under ncu (the launch list and single-kernel captures under profiles/):
    python -m paper_2311_01598_gb300.profile_ks --dataflow OC,MP
    python -m paper_2311_01598_gb300.profile_ks --dataflow OC --batch 16
    python -m paper_2311_01598_gb300.profile_ks --batch 4 --keys 4 --schedule 2,2,64,0
    python -m paper_2311_01598_gb300.profile_ks --hoisted 4      # hoisted rotations + automorphism
    python -m paper_2311_01598_gb300.profile_ks --shard 4        # tower-sharded key switch, 4 ranks emulated
    python -m paper_2311_01598_gb300.profile_ks --mlp            # cost-model MLP forward, backward, Adam
    python -m paper_2311_01598_gb300.profile_ks --batch 4 --keys 4 --compressed --schedule 2,2,64,0
Key generation runs first (a few launches), then one key switch per
dataflow listed (or one batched call per dataflow with --batch B > 1), or
the workload one of the other options names.
"""
from __future__ import annotations

import argparse
import os

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
    ap.add_argument("--row-stage", action="store_true", help="forward row passes staged by bulk copies")
    ap.add_argument("--hoisted", type=int, default=0, help="R hoisted rotations of one ciphertext, then the automorphism")
    ap.add_argument("--shard", type=int, default=0, help="one key switch sharded by tower over G emulated ranks")
    ap.add_argument("--mlp", action="store_true", help="one training step and one forward pass of the cost model")
    ap.add_argument("--compressed", action="store_true", help="compressed keys (a halves regenerated on chip)")
    ap.add_argument("--schedule", default=None,
                    help="'dataflow,oc_variant,chunk,order': one batched call with this schedule")
    a = ap.parse_args()
    P = ks.Params(a.logN, a.nq, a.kp, a.dnum)
    if a.row_stage:
        P.set_row_stage(True)
    nact = a.level or a.nq
    s = inputs.ternary_secret(P.N, 1)
    if a.compressed:
        keys = [P.keygen_compressed(s, inputs.galois_secret(s, 5 + 2 * k), 7 + k) for k in range(a.keys)]
    else:
        keys = [P.key_synthetic(7 + k) if k else P.keygen(s, inputs.galois_secret(s, 5), 7) for k in range(a.keys)]
    jobs = []
    for i in range(a.batch):
        d = ks.to_device(inputs.uniform_towers(P.q[:nact], P.N, 3 + i))
        jobs.append((keys[i % a.keys], nact, d, ks.empty((nact, P.N)), ks.empty((nact, P.N))))
    if a.mlp:
        from . import tune
        rows = tune.load(os.path.join(tune.DATA_DIR, "tune_gb300.jsonl"))
        X, T = tune.arrays(rows)
        m = ks.Mlp([X.shape[1], *tune.HIDDEN, T.shape[1]], seed=1)
        x, t = torch.from_numpy(X).cuda(), torch.from_numpy((T - T.mean()) / T.std()).cuda()
        m.train_step(x, t, 1e-3)
        m.forward(x)
    elif a.hoisted:
        gals = inputs.galois_elements(P.N, a.hoisted, seed=5)
        rkeys = [P.key_synthetic(20 + r) for r in range(a.hoisted)]
        o0 = [ks.empty((nact, P.N)) for _ in gals]
        o1 = [ks.empty((nact, P.N)) for _ in gals]
        P.switch_hoisted(rkeys, gals, nact, jobs[0][2], o0, o1)
        P.automorph(0, gals[0], jobs[0][2], jobs[0][3], accumulate=True)
    elif a.shard:
        from . import dist
        parts = [dist.tower_partition(P.nq, P.kp, a.shard, g) for g in range(a.shard)]
        skeys = [P.key_shard(keys[0], ks.Shard(*pt)) for pt in parts]
        d = jobs[0][2]
        d_own = [d[dist.active_q(pt, nact)[0]:dist.active_q(pt, nact)[1]].contiguous() for pt in parts]
        dist.sharded_keyswitch(P, skeys, parts, nact, d_own, gather_y=lambda ys: torch.cat(ys, dim=0),
                               gather_w=lambda ws: torch.cat(ws, dim=1))
    elif a.schedule:
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
