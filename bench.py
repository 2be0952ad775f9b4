"""Benchmark: hybrid key switching at N=2^16, L+1=24 Q primes, K=8 P primes,
dnum=3 (alpha=8), 54-bit primes -- the Output-Centric batched path, with the
plain single-ciphertext Max-Parallel path beside it.

One step = one ks_switch_batch call over B ciphertexts at the top level, each
with its own Galois key (B distinct 96 MiB keys, so no key is reused within a
step and every key switch streams its whole key).  Inputs and keys together
exceed the 126 MB L2 (B=16: 192 MiB inputs, 1.5 GiB keys), so no L2 flush is
needed between steps.

Prints ONE JSON line (rank 0).  `value` is key-switches/s over the timed
region on device-resident inputs; `e2e` is the same metric through
ks_switch_batch_host (pinned host buffers, both copies inside the timed
region); `roofline` describes the kernel with the largest share of device
time, timed live with CUDA events on its launch stream.

--impl reference times the CPU oracle (oracle/, plain C, OpenMP over towers)
on this host's cores on the same workload and prints the same line with
"impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "key-switches/s at N=2^16 L+1=24 dnum=3, OC batched vs MP plain; % HBM roofline"
UNIT = "key-switches/s"
LOGN, NQ, KP, DNUM, BITS = 16, 24, 8, 3, 54
N = 1 << LOGN
LIMB = N * 8
# algorithmic bytes of one key switch at the top level: input + key + both outputs
ALG_BYTES_PER_KS = NQ * LIMB + DNUM * 2 * (NQ + KP) * LIMB + 2 * NQ * LIMB


def peaks():
    """(HBM copy GB/s, maximum SM MHz, source): the measured peaks file, else the fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), float(m.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


# ------------------------------------------------------------------ workload model
def algorithmic_work(nact=NQ):
    """Per key switch at level nact: modular multiplications of every stage
    (butterflies count one each) and bytes per kernel class.  Used for the
    roofline of the dominant kernel."""
    nt = nact + KP
    alpha = (NQ + DNUM - 1) // DNUM
    nd = (nact + alpha - 1) // alpha
    a_last = nact - (nd - 1) * alpha
    bfly = (N // 2) * LOGN
    ntt = {
        "modup_intt": nact,
        "modup_ntt": sum(nt - min(alpha, nact - j * alpha) for j in range(nd)),
        "moddown_intt": 2 * KP,
        "moddown_ntt": 2 * nact,
    }
    n_ntt = sum(ntt.values())
    bconv_up = sum(min(alpha, nact - j * alpha) * (nt - min(alpha, nact - j * alpha)) for j in range(nd)) * N
    bconv_down = 2 * KP * nact * N
    key_mac = 2 * nd * nt * N
    n_inv = ntt["modup_intt"] + ntt["moddown_intt"]
    return {"ntt": n_ntt, "butterflies": n_ntt * bfly, "forward_butterflies": (n_ntt - n_inv) * bfly,
            "inverse_butterflies": n_inv * bfly, "bconv_macs": bconv_up + bconv_down, "key_macs": key_mac,
            "modmul": n_ntt * bfly + bconv_up + bconv_down + key_mac + nact * N, "a_last": a_last}


def class_work(nact=NQ):
    """Algorithmic work per key switch of each kernel class of the
    Output-Centric schedule (split variant): (kind, units, bytes).  kind
    "bfly"/"ibfly": units are forward/inverse NTT butterflies; "mac": base-conversion
    multiply-accumulates; "hbm": a streaming kernel judged on bytes.  Bytes
    count each limb the kernel must read or write once (1 limb = 8N bytes)."""
    alpha = (NQ + DNUM - 1) // DNUM
    nd = (nact + alpha - 1) // alpha
    al = [min(alpha, nact - j * alpha) for j in range(nd)]
    K, half = KP, N // 2
    LA = {16: 8, 17: 9}.get(LOGN, (LOGN + 1) // 2)
    LB = LOGN - LA
    q_modup = sum(nact - a for a in al)          # ModUp limbs produced for Q towers
    inv_limbs = nact + 2 * K                      # prep + ModDown P1
    fwd_limbs = nd * K + q_modup + 2 * nact       # P section + Q section (ModUp, ModDown)
    return {
        "ntt_inv_row": ("ibfly", inv_limbs * half * LB, 2 * inv_limbs * LIMB),
        "ntt_inv_col": ("ibfly", inv_limbs * half * LA, 2 * inv_limbs * LIMB),
        "ntt_fwd_col": ("bfly", fwd_limbs * half * LA, 2 * fwd_limbs * LIMB),
        "ntt_fwd_row": ("bfly", fwd_limbs * half * LB, 2 * fwd_limbs * LIMB),
        "ntt_inv_cl": ("ibfly", inv_limbs * half * LOGN, 2 * inv_limbs * LIMB),
        "ntt_fwd_cl": ("bfly", fwd_limbs * half * LOGN, 2 * fwd_limbs * LIMB),
        "bconv_up": ("mac", sum(a * (K + nact - a) for a in al) * N, (2 * nact + nd * K + q_modup) * LIMB),
        "bconv_down": ("mac", 2 * K * nact * N, (2 * K + 2 * nact) * LIMB),
        "oc_comb_p": ("hbm", 2 * nd * K * N, (3 * nd * K + 2 * K) * LIMB),
        "oc_comb_q": ("hbm", 2 * nd * nact * N, (q_modup + nact + 2 * nd * nact + 2 * nact + 2 * nact) * LIMB),
    }


def workload_config(B, dataflow, world):
    """The `config` object of the JSON line."""
    return {"workload": f"hybrid key switch N=2^16 L+1=24 K=8 dnum=3 alpha=8 54-bit primes, {B} "
                        f"ciphertexts/step each with its own Galois key, {dataflow} batched",
            "batch_per_gpu": B, "dataflow": dataflow, "parallelism": f"replicas x{world}",
            "l2": "inputs+keys per step exceed L2 (no flush)"}


def mixed_batch(P, keys, stream, timed, world, steps, seed, n_jobs=64, learned=None):
    """Key switches/s on a batch of n_jobs ciphertexts with levels uniform in
    4..24 (L+1 towers), each with one of the given keys: the schedule the
    autotuner picks, and the same schedule with jobs grouped by key."""
    import numpy as np

    from paper_2311_01598_gb300 import inputs, ks
    rng = np.random.default_rng(seed)
    levels = [int(x) for x in rng.integers(4, NQ + 1, size=n_jobs)]
    kidx = [int(x) for x in rng.integers(0, len(keys), size=n_jobs)]
    jobs = []
    for i, (lv, k) in enumerate(zip(levels, kidx)):
        d = ks.to_device(inputs.uniform_towers(P.q[:lv], N, seed=seed + 1 + i))
        jobs.append((keys[k], lv, d, ks.empty((lv, N)), ks.empty((lv, N))))
    tuned, _ = P.autotune(jobs, reps=2, stream=stream)
    t_auto = timed(lambda: P.switch_batch(jobs, "AUTO", stream), steps, 2)
    by_key = ks.Schedule(tuned.dataflow, tuned.oc_variant, tuned.chunk, 2, tuned.ntt, tuned.bconv)
    t_key = timed(lambda: P.switch_batch_sched(jobs, by_key, stream), steps, 2)
    out = {"value": round(world * n_jobs * steps / (t_auto / 1e3), 2), "unit": "key-switches/s",
           "jobs": n_jobs, "levels": "uniform 4..24 of 24", "keys": len(keys),
           "schedule": list(tuned.as_tuple() + tuned.impl()),
           "grouped_by_key": round(world * n_jobs * steps / (t_key / 1e3), 2),
           "mean_level": round(sum(levels) / n_jobs, 2)}
    if learned is not None:
        out["learned_schedule"] = learned_regret(P, jobs, tuned, t_auto / steps, stream, timed, steps)
    return out


def learned_regret(P, jobs, tuned, ms_tuned, stream, timed, steps):
    """The attached cost model's pick for a batch, timed beside the
    exhaustive autotuner's pick (ms_tuned per call): regret in microseconds
    per call and per key switch."""
    pick, _ = P.predict_schedule(jobs, stream)
    ms_pick = timed(lambda: P.switch_batch_sched(jobs, pick, stream), steps, 2) / steps
    n = len(jobs)
    return {"model_pick": list(pick.as_tuple() + pick.impl()), "autotuner_pick": list(tuned.as_tuple() + tuned.impl()),
            "model_ms": round(ms_pick, 4), "autotuner_ms": round(ms_tuned, 4),
            "regret_us_per_call": round((ms_pick - ms_tuned) * 1e3, 2),
            "regret_us_per_ks": round((ms_pick - ms_tuned) * 1e3 / n, 3),
            "regret_frac": round(ms_pick / ms_tuned - 1, 4)}


def hoisted_rotations(P, keys, gals, d, stream, timed, world, steps):
    """Rotations/s of R rotations of one ciphertext at the top level: the
    hoisted call (one ModUp shared by all) against R independent key
    switches (one batched call under KS_AUTO)."""
    from paper_2311_01598_gb300 import ks
    R = len(keys)
    o0 = [ks.empty((NQ, N)) for _ in range(R)]
    o1 = [ks.empty((NQ, N)) for _ in range(R)]
    t_h = timed(lambda: P.switch_hoisted(keys, gals, NQ, d, o0, o1, stream), steps, 2)
    jobs = [(keys[r], NQ, d, o0[r], o1[r]) for r in range(R)]
    P.autotune(jobs, reps=2, stream=stream)
    t_s = timed(lambda: P.switch_batch(jobs, "AUTO", stream), steps, 2)
    return {"value": round(world * R * steps / (t_h / 1e3), 2), "unit": "rotations/s", "rotations": R,
            "separate_key_switches": round(world * R * steps / (t_s / 1e3), 2),
            "note": "hoisted: one ModUp, per rotation a permuted key product and a ModDown"}


TABLE3 = [("BTS1", 17, 28, 28, 1), ("BTS2", 17, 40, 20, 2), ("BTS3", 17, 45, 15, 3),
          ("ARK", 16, 24, 6, 4), ("DPRIVE", 16, 26, 7, 3)]


def table3_sets(stream, timed, world, steps, seed, batch=4):
    """Key switches/s at the top level of each Table III parameter set (54-bit
    primes), a batch of `batch` ciphertexts with distinct keys per step, under
    the autotuned schedule; keys are synthetic (uniform words)."""
    import torch

    from paper_2311_01598_gb300 import inputs, ks
    out = {}
    for name, logN, nq, kp, dnum in TABLE3:
        P3 = ks.Params(logN, nq, kp, dnum, prime_bits=BITS)
        n3 = 1 << logN
        keys3 = [P3.key_synthetic(seed + i) for i in range(batch)]
        jobs3 = [(keys3[i], nq, ks.to_device(inputs.uniform_towers(P3.q, n3, seed=seed + 10 + i)),
                  ks.empty((nq, n3)), ks.empty((nq, n3))) for i in range(batch)]
        tuned3, _ = P3.autotune(jobs3, reps=2, stream=stream)
        t = timed(lambda: P3.switch_batch(jobs3, "AUTO", stream), steps, 2)
        out[name] = {"value": round(world * batch * steps / (t / 1e3), 2), "unit": "key-switches/s",
                     "logN": logN, "q_towers": nq, "p_towers": kp, "dnum": dnum, "batch": batch,
                     "schedule": list(tuned3.as_tuple() + tuned3.impl())}
        del jobs3, keys3, P3
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        """Start sampling nvidia-smi in the background."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        """Stop sampling; returns the clock summary."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power) if power else None}


# ------------------------------------------------------------------ CPU oracle
def oracle_rate(seconds: float = 10.0, min_reps: int = 2):
    """The oracle, as it stands, on this host's cores: key switches per
    second on the same parameter set (bounded sample of whole key switches)."""
    import numpy as np
    from oracle import oracle as orc
    from paper_2311_01598_gb300 import inputs
    C = orc.Ctx(LOGN, NQ, KP, DNUM, bits=BITS)
    s = inputs.ternary_secret(N, inputs.SEED_BASE + 1)
    sp = inputs.galois_secret(s, inputs.galois_elements(N, 1, inputs.SEED_BASE + 2)[0])
    evk = C.keygen(s, sp, seed=inputs.SEED_BASE + 3)
    d = inputs.uniform_towers(C.q, N, seed=inputs.SEED_BASE + 4)
    reps, t0 = 0, time.perf_counter()
    while True:
        C.keyswitch(NQ, d, evk)
        reps += 1
        el = time.perf_counter() - t0
        if reps >= min_reps and el >= seconds:
            break
    del np
    return reps / el, reps, el, orc.get_threads()


# ------------------------------------------------------------------ main
def main():
    """Parse the arguments and print one JSON line (our arm or the reference arm)."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--dataflow", default="OC", choices=["MP", "DC", "OC"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--schedule", default=None,
                    help="fix the batch schedule 'dataflow,oc_variant,chunk,order' instead of autotuning it "
                         "(used to take an ncu launch list of the schedule a plain run chose)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_2311_01598_gb300 import dist as kdist
    rank, world, local_rank = kdist.env_rank()

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2311_01598_gb300 import build as kbuild
    if rank == 0 and not os.path.exists(kbuild.LIB):
        kbuild.build()
    if dist is not None:
        dist.barrier()
    from paper_2311_01598_gb300 import inputs, ks

    P = ks.Params(LOGN, NQ, KP, DNUM, prime_bits=BITS)
    B = args.batch
    s = inputs.ternary_secret(N, inputs.SEED_BASE + 1 + rank)
    gals = inputs.galois_elements(N, B, seed=inputs.SEED_BASE + 2)
    keys = [P.keygen(s, inputs.galois_secret(s, g), seed=inputs.SEED_BASE + 100 + i) for i, g in enumerate(gals)]
    d = [ks.to_device(inputs.uniform_towers(P.q, N, seed=inputs.SEED_BASE + 1000 * (rank + 1) + i))
         for i in range(B)]
    o0 = [ks.empty((NQ, N)) for _ in range(B)]
    o1 = [ks.empty((NQ, N)) for _ in range(B)]
    jobs = [(keys[i], NQ, d[i], o0[i], o1[i]) for i in range(B)]
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        return kdist.max_over_ranks(x, dev)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1))

    # the library's autotuner picks the batch's schedule (untimed); the timed
    # steps then run KS_AUTO, which finds it in the tuning cache
    if args.schedule:
        tuned, tune_ms = ks.Schedule(*[int(x) for x in args.schedule.split(",")]), []
        P.tune_cache_put(B, NQ, tuned)
        impl_ms = []
    else:
        tuned, tune_ms = P.autotune(jobs, reps=2, stream=stream)
        # the second stage's timings of the winning structure, for the record
        _, impl_ms = P.autotune_impl(jobs, tuned, reps=2, stream=stream)
    if args.dataflow == "OC":
        step = lambda: P.switch_batch(jobs, "AUTO", stream)  # noqa: E731
    else:
        step = lambda: P.switch_batch(jobs, args.dataflow, stream)  # noqa: E731

    # ---- headline: device-resident inputs, clocks sampled during the region
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    l0 = ks.kernel_launches()
    ms = timed(step, args.steps, 0)
    launches = ks.kernel_launches() - l0
    clocks = sampler.stop()
    ms_per_step = ms / args.steps
    value = world * B * args.steps / (ms / 1e3)

    # ---- per-kernel device time of the same workload (CUDA events per launch),
    # with the batch on one stream: the headline's lanes overlap kernels, which
    # would stretch each one's event-timed duration
    P.set_batch_lanes(1)
    ks.profile_enable(True)
    ms_prof = timed(step, args.steps, 0)
    ks.profile_enable(False)
    P.set_batch_lanes(2)
    prof = ks.profile_collect()
    top = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None

    # ---- every Output-Centric variant on the same batch (schedule comparison)
    variants = {}
    for vname, v in (("fused", 0), ("split", 1), ("whole", 2), ("tower", 3)):
        sc = ks.Schedule(2, v, 64, 0)
        f = lambda sc=sc: P.switch_batch_sched(jobs, sc, stream)  # noqa: E731
        t = timed(f, max(3, args.steps // 2), 2)
        variants[vname] = round(world * B * max(3, args.steps // 2) / (t / 1e3), 2)

    # ---- mixed batch: 64 ciphertexts with levels uniform in 4..24, each keyed
    # by one of the 16 Galois keys (jobs of one key and level share key limbs)
    # ---- the learned cost model (committed, trained on GB300 autotuner
    # timings by the library's kernels) attached to the parameter set: its
    # pick for the headline batch and the mixed batch against the
    # autotuner's, and its held-out regret on the committed dataset
    from paper_2311_01598_gb300 import tune
    cm = tune.CostModel.load(os.path.join(tune.DATA_DIR, "cost_model_gb300.npz"))
    P.set_cost_model(cm.mlp, cm.t_mean, cm.t_scale)
    learned = {"bench_batch": learned_regret(P, jobs, tuned, ms_per_step, stream, timed, max(3, args.steps // 2))}
    mixed = mixed_batch(P, keys, stream, timed, world, steps=max(3, args.steps // 2), seed=inputs.SEED_BASE + 7,
                        learned=cm)
    learned["mixed_batch"] = mixed.pop("learned_schedule", None)
    rows = tune.load(os.path.join(tune.DATA_DIR, "tune_gb300.jsonl"))
    _, test_rows = tune.split(rows, 0.8, seed=0)
    di = tune.default_candidate_index(P.tune_candidates(), P.default_schedule())
    learned["held_out"] = {k: (round(v, 4) if isinstance(v, float) else v)
                           for k, v in tune.evaluate(cm, test_rows, di).items()}
    P.set_cost_model(None)

    # ---- 8 rotations of one ciphertext: hoisted (one ModUp) vs 8 separate switches
    hoisted = hoisted_rotations(P, keys[:8], gals[:8], d[0], stream, timed, world, steps=max(3, args.steps // 2))

    # ---- the same 16-ciphertext step with compressed keys (a regenerated on chip)
    ckeys = [P.keygen_compressed(s, inputs.galois_secret(s, g), seed=inputs.SEED_BASE + 100 + i)
             for i, g in enumerate(gals)]
    cjobs = [(ckeys[i], NQ, d[i], ks.empty((NQ, N)), ks.empty((NQ, N))) for i in range(B)]  # own outputs
    ctuned, _ = P.autotune(cjobs, reps=2, stream=stream)
    t_c = timed(lambda: P.switch_batch_sched(cjobs, ctuned, stream), args.steps, 2)
    compressed = {"value": round(world * B * args.steps / (t_c / 1e3), 2), "unit": UNIT,
                  "key_bytes": ckeys[0].nbytes, "full_key_bytes": keys[0].nbytes,
                  "schedule": list(ctuned.as_tuple() + ctuned.impl())}
    del cjobs, ckeys

    # ---- the same step with moduli of the special form k*2^32 + 1 (explicit
    # primes: the 32 largest below 2^54; the two-pass NTTs' cheaper product)
    sp_all = ks.special_primes(BITS, NQ + KP)
    Psp = ks.Params(LOGN, NQ, KP, DNUM, q=sp_all[KP:], p=sp_all[:KP])
    sp_keys = [Psp.keygen(s, inputs.galois_secret(s, g), seed=inputs.SEED_BASE + 100 + i) for i, g in enumerate(gals)]
    sp_jobs = [(sp_keys[i], NQ, ks.to_device(inputs.uniform_towers(Psp.q, N, seed=inputs.SEED_BASE + 5000 + i)),
                ks.empty((NQ, N)), ks.empty((NQ, N))) for i in range(B)]
    sp_tuned, _ = Psp.autotune(sp_jobs, reps=2, stream=stream)
    t_sp = timed(lambda: Psp.switch_batch(sp_jobs, "AUTO", stream), args.steps, 2)
    special = {"value": round(world * B * args.steps / (t_sp / 1e3), 2), "unit": UNIT,
               "primes": "the 32 largest primes k*2^32+1 below 2^54 (explicit lists; 8 special, 24 Q)",
               "schedule": list(sp_tuned.as_tuple() + sp_tuned.impl())}
    del sp_jobs, sp_keys, Psp

    # ---- the paper's parameter sets (Table III): 4 ciphertexts a step, own keys
    table3 = table3_sets(stream, timed, world, steps=max(3, args.steps // 2), seed=inputs.SEED_BASE + 9)

    # ---- the plain single-ciphertext paths beside it, and the Output-Centric
    # one replayed from a CUDA graph (launch gaps matter at this size)
    singles = {}
    for df in ("MP", "DC", "OC"):
        f = lambda df=df: P.switch(keys[0], NQ, d[0], o0[0], o1[0], df, stream)  # noqa: E731
        t = timed(f, args.steps, 3)
        singles[df] = world * args.steps / (t / 1e3)
    gs = torch.cuda.Stream()  # capture needs a stream of its own; warm it (scratch) first
    with torch.cuda.stream(gs):
        P.switch(keys[0], NQ, d[0], o0[0], o1[0], "OC", gs)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        P.switch(keys[0], NQ, d[0], o0[0], o1[0], "OC", gs)
    t = timed(graph.replay, args.steps, 3)  # replays on the timing stream
    singles["OC_graph"] = world * args.steps / (t / 1e3)

    # ---- end to end through the host-buffer entry point
    hin = [torch.empty((NQ, N), dtype=torch.int64, pin_memory=True) for _ in range(B)]
    for i in range(B):
        hin[i].copy_(d[i].cpu())
    h0 = [torch.empty((NQ, N), dtype=torch.int64, pin_memory=True) for _ in range(B)]
    h1 = [torch.empty((NQ, N), dtype=torch.int64, pin_memory=True) for _ in range(B)]
    hjobs = [(keys[i], NQ, hin[i], h0[i], h1[i]) for i in range(B)]
    # the same dataflow argument as the headline step (KS_AUTO for OC: the
    # host path's chunks take the schedule tuned for this batch)
    e2e_df = "AUTO" if args.dataflow == "OC" else args.dataflow
    e2e_step = lambda: P.switch_batch_host(hjobs, e2e_df, stream)  # noqa: E731
    ms_e2e = timed(e2e_step, args.steps, 3)
    torch.cuda.synchronize()
    e2e_ok = all(torch.equal(h0[i], o0[i].cpu()) and torch.equal(h1[i], o1[i].cpu()) for i in range(B))
    e2e_value = world * B * args.steps / (ms_e2e / 1e3)

    hbm_gbs, sm_max_mhz, peak_src = peaks()
    hbm_achieved = value / world * ALG_BYTES_PER_KS / 1e9

    bfly_peak, mac_peak = ks.probe_alu()
    ibfly_peak = ks.probe_inv_bfly()
    work = class_work()
    from paper_2311_01598_gb300 import launch_summary
    traffic_rec = launch_summary.recorded_traffic()  # ncu DRAM bytes per key switch, current sources only
    pipes_rec = launch_summary.recorded_pipes()      # ncu integer-pipe utilisation, current sources only

    def class_roofline(name, cnt, tot_ms):
        secs_per_ks = tot_ms / 1e3 / (args.steps * B)
        out = {"kernel": name, "launches_per_step": cnt / args.steps, "per_launch_ms": round(tot_ms / cnt, 4),
               "share_of_step": round(tot_ms / ms_prof, 4), "traffic": None}
        if name in pipes_rec:
            out["pipe"] = {k: v for k, v in pipes_rec[name].items() if k != "capture"}
            out["pipe"]["basis"] = ("ncu hardware counters of one launch (fmaheavy = the 32-bit integer multiply "
                                    "pipe): paper_2311_01598_gb300/data/ncu_pipes_gb300.json")
        if name in traffic_rec:
            out["traffic"] = int(traffic_rec[name] * B * args.steps / cnt)
            out["traffic_basis"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per key switch "
                                    "(paper_2311_01598_gb300/data/ncu_traffic_gb300.json), scaled to this launch")
        wk = work.get(name) if args.dataflow == "OC" and tuned.dataflow == 2 and tuned.oc_variant in (1, 2) else None
        if wk is None:
            out.update({"bound": "alu", "achieved": None, "peak": None, "frac": None})
            return out
        kind, units, nbytes = wk
        gbs = nbytes / secs_per_ks / 1e9
        out["algorithmic_bytes_per_launch"] = int(nbytes * B * args.steps / cnt)
        if kind == "hbm":
            out.update({"bound": "hbm", "unit": "GB/s", "achieved": round(gbs, 1), "peak": hbm_gbs,
                        "frac": round(gbs / hbm_gbs, 4), "peak_basis": f"{peak_src} copy bandwidth"})
        else:
            peak = {"bfly": bfly_peak, "ibfly": ibfly_peak}.get(kind, mac_peak)
            rate = units / secs_per_ks
            out.update({"bound": "alu", "unit": "G" + ("mac" if kind == "mac" else "butterfly") + "/s",
                        "achieved": round(rate / 1e9, 2), "peak": round(peak / 1e9, 2), "frac": round(rate / peak, 4),
                        "algorithmic_units_per_launch": int(units * B * args.steps / cnt),
                        "peak_basis": ("ks_probe_inv_bfly" if kind == "ibfly" else "ks_probe_alu")
                        + ": register-only loop of the same device code on all 152 SMs",
                        "hbm_frac_of_kernel": round(gbs / hbm_gbs, 4)})
        return out

    roofline = class_roofline(top[0], *top[1]) if top is not None else None
    per_kernel = {k: class_roofline(k, c, t) for k, (c, t) in prof.items()}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as orc
        rate, reps, el, cores = oracle_rate()
        cpu = {"value": round(rate, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{reps} whole key switches at N=2^16 L+1=24 K=8 dnum=3 ({el:.1f} s)"}
        orc.set_threads(1)  # the same oracle on one core (one whole key switch)
        rate1, reps1, el1, _ = oracle_rate(seconds=1.0, min_reps=1)
        orc.set_threads(cores)
        cpu["single_core"] = {"value": round(rate1, 4), "unit": UNIT,
                              "sample": f"{reps1} whole key switch(es), one thread ({el1:.1f} s)"}

    # step-level integer ceiling: the step's butterflies and base-conversion
    # multiply-accumulates at the probes' rates (the key products are
    # streaming work, judged by the HBM fraction)
    wk = algorithmic_work()
    alu_s_per_ks = (wk["forward_butterflies"] / bfly_peak + wk["inverse_butterflies"] / ibfly_peak
                    + wk["bconv_macs"] / mac_peak)
    alu_roofline = {"achieved": round(value / world, 2), "ceiling": round(1.0 / alu_s_per_ks, 1), "unit": UNIT,
                    "frac": round(value / world * alu_s_per_ks, 4),
                    "basis": "forward/inverse butterflies and CUDA-core-equivalent base-conversion MACs per key "
                             "switch at the ks_probe_alu / ks_probe_inv_bfly rates"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(B, args.dataflow, world),
            "mp_plain": {"value": round(singles["MP"], 2), "unit": UNIT, "note": "single ciphertext per call"},
            "single_ciphertext": {k: round(v, 2) for k, v in singles.items()},
            "oc_batched_over_mp_plain": round(value / singles["MP"], 3),
            "oc_variants": variants,
            "mixed_batch": mixed,
            "learned_schedule": learned,
            "table3_sets": table3,
            "hoisted_rotations": hoisted,
            "compressed_keys": compressed,
            "special_form_moduli": special,
            "schedule": {"tuned": list(tuned.as_tuple() + tuned.impl()),
                         "fields": "dataflow, oc_variant, chunk, order, ntt, bconv",
                         "source": "fixed by --schedule" if args.schedule else "ks_autotune",
                         "candidates_ms": [round(x, 3) for x in tune_ms],
                         "impl_ms": dict(zip(["two-pass NTT, tensor-core BConv", "cluster NTT, tensor-core BConv",
                                              "two-pass NTT, CUDA-core BConv", "cluster NTT, CUDA-core BConv"],
                                             [round(x, 3) for x in impl_ms]))},
            "hbm_roofline": {"achieved": round(hbm_achieved, 1), "peak": hbm_gbs, "unit": "GB/s",
                             "frac": round(hbm_achieved / hbm_gbs, 4), "basis": f"{peak_src} copy bandwidth",
                             "algorithmic_bytes_per_ks": ALG_BYTES_PER_KS},
            "roofline": roofline,
            "alu_roofline": alu_roofline,
            "kernels": {k: {"launches": c, "ms": round(t, 3), "frac": per_kernel[k].get("frac"),
                            "bound": per_kernel[k].get("bound")}
                        for k, (c, t) in sorted(prof.items(), key=lambda kv: -kv[1][1])},
            "alu_probe": {"butterflies_per_s": bfly_peak, "inverse_butterflies_per_s": ibfly_peak,
                          "bconv_macs_per_s": mac_peak,
                          "int_pipes_lanes_per_clk_sm": ks.probe_int_pipes()},
            "work_per_ks": algorithmic_work(),
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": B * NQ * LIMB,
                    "d2h_bytes_per_step": 2 * B * NQ * LIMB, "outputs_match_device_path": e2e_ok},
            "gpu_launches": int(launches),
            "profile_pass": {"ms_per_step": round(ms_prof / args.steps, 4), "batch_lanes": 1,
                             "note": "per-kernel times come from this pass; the headline runs 2 lanes"},
            "launch_window": {"first": int(l0), "count": int(launches),
                              "note": "library launches before / inside the timed region"},
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on this host's cores, same metric."""
    if rank != 0:
        return
    from oracle import oracle as orc
    orc.build()
    # each step: one whole key switch of the workload (bounded sample)
    import numpy as np
    from paper_2311_01598_gb300 import inputs
    C = orc.Ctx(LOGN, NQ, KP, DNUM, bits=BITS)
    s = inputs.ternary_secret(N, inputs.SEED_BASE + 1)
    sp = inputs.galois_secret(s, inputs.galois_elements(N, 1, inputs.SEED_BASE + 2)[0])
    evk = C.keygen(s, sp, seed=inputs.SEED_BASE + 3)
    d = inputs.uniform_towers(C.q, N, seed=inputs.SEED_BASE + 4)
    # W untimed warm-up steps, then K timed steps; each step is one whole key
    # switch of the workload (a bounded sample: the oracle takes ~0.5 s per
    # key switch on 16 cores, so a 16-ciphertext step would take ~8 s)
    for _ in range(args.warmup):
        C.keyswitch(NQ, d, evk)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        C.keyswitch(NQ, d, evk)
    el = time.perf_counter() - t0
    value = args.steps / el
    del np
    config = workload_config(1, args.dataflow, world)
    config["workload"] = ("hybrid key switch N=2^16 L+1=24 K=8 dnum=3 alpha=8 54-bit primes, CPU oracle: "
                          "1 ciphertext/step (a bounded sample of the 16-ciphertext GPU step)")
    config["dataflow"] = "oracle stage order (Sec. III)"
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic", "impl": "reference",
        "config": config,
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": orc.get_threads(), "kind": "oracle",
                         "sample": f"{args.warmup} untimed + {args.steps} timed steps of one whole key switch "
                                   f"each, CPU oracle (plain C, OpenMP over towers)"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
