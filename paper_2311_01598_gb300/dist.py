"""Multi-GPU plumbing for key switching.

* Data parallelism over ciphertexts: independent key switches shard across
  ranks with no collective on the data path (each rank owns its jobs, keys
  and outputs); the only collectives are the benchmark's barrier and the
  max-over-ranks of its timings.
* Tower sharding of one key switch (CiFlow Sec. IV-C: output towers are
  independent): rank g owns a contiguous range of Q towers and of special
  towers (``tower_partition``), holds their input towers and key limbs, and
  the ranks exchange twice: an all-gather of the pre-scaled input y and one
  of the special part w (``all_gather_towers``).  ``sharded_keyswitch`` runs
  the per-rank library calls with any gather function.

One process per GPU (torchrun), NCCL on GPUs, gloo on CPU (tests).
"""
from __future__ import annotations

import os


def env_rank():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank: int, world: int):
    """Contiguous block of items owned by rank (sizes differ by at most one)."""
    n = len(items)
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return items[lo:hi]


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a per-rank scalar (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    """Sum of a value over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_per_rank, seconds_per_rank, device=None) -> float:
    """Whole-job rate: units of all ranks over the slowest rank's time."""
    return sum_over_ranks(units_per_rank, device) / max_over_ranks(seconds_per_rank, device)


# ------------------------------------------------------------------ tower sharding
def tower_partition(nq: int, kp: int, world: int, rank: int):
    """(q_begin, q_end, p_begin, p_end): the rank's contiguous Q towers and
    special towers; over all ranks the ranges partition [0, nq) and [0, kp)
    (sizes differ by at most one)."""
    def rng(n):
        base, extra = divmod(n, world)
        lo = rank * base + min(rank, extra)
        return lo, lo + base + (1 if rank < extra else 0)
    q0, q1 = rng(nq)
    p0, p1 = rng(kp)
    return q0, q1, p0, p1


def active_q(part, nact: int):
    """The rank's active Q towers [q0, q1) at level nact (possibly empty)."""
    q0, q1, _, _ = part
    return min(q0, nact), min(q1, nact)


def all_gather_towers(local, counts, group=None):
    """All-gather of tower rows along dim -2: every rank contributes its
    rows local[..., :counts[rank], :] (counts may differ); the result holds
    all ranks' rows in rank order (which is tower order for
    tower_partition's ranges).  Rows are padded to the largest count for the
    collective (torch.distributed.all_gather; NCCL on GPUs, gloo on CPU)."""
    import torch
    import torch.distributed as dist
    width = max(counts)
    shape = list(local.shape)
    shape[-2] = width
    pad = torch.zeros(shape, dtype=local.dtype, device=local.device)
    pad.narrow(-2, 0, local.shape[-2]).copy_(local)
    parts = [torch.empty_like(pad) for _ in counts]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p.narrow(-2, 0, c) for p, c in zip(parts, counts)], dim=-2)


def sharded_keyswitch(P, skeys, parts, nact, d_own, gather_y, gather_w, stream=None):
    """One tower-sharded key switch through the library's per-rank calls.

    skeys/parts/d_own: per local rank, its shard key, its tower_partition
    tuple and its input towers [nq_own][N] (device).  gather_y(list of
    y_own) -> y_all [nact][N] and gather_w(list of w_own [2][np_own][N]) ->
    w_all [2][K][N] perform the two exchanges (an NCCL all-gather across
    processes, or device copies when the ranks are emulated on one device).
    Returns per rank (out0_own, out1_own)."""
    from . import ks
    N = P.N
    shards = [ks.Shard(*pt) for pt in parts]
    ys = []
    for sh, pt, d in zip(shards, parts, d_own):
        q0, q1 = active_q(pt, nact)
        y = ks.empty((q1 - q0, N))
        if q1 > q0:
            P.shard_prep(sh, nact, d, y, stream)
        ys.append(y)
    y_all = gather_y(ys)
    cps, scr = [], []
    for sh, pt, sk, d in zip(shards, parts, skeys, d_own):
        q0, q1 = active_q(pt, nact)
        nown = (q1 - q0) + (pt[3] - pt[2])
        cp = ks.empty((2, nown, N))
        s = ks.empty((max(1, P.shard_scratch_words(sh, nact)),))
        P.shard_keyprod(sk, nact, y_all, d, cp, s, stream)
        cps.append(cp)
        scr.append(s)
    w_all = gather_w([cp[:, (active_q(pt, nact)[1] - active_q(pt, nact)[0]):, :] for cp, pt in zip(cps, parts)])
    outs = []
    for sh, pt, sk, cp, s in zip(shards, parts, skeys, cps, scr):
        q0, q1 = active_q(pt, nact)
        o0, o1 = ks.empty((q1 - q0, N)), ks.empty((q1 - q0, N))
        if q1 > q0:
            P.shard_moddown(sk, nact, w_all.contiguous(), cp, o0, o1, s, stream)
        outs.append((o0, o1))
    return outs
