"""Thin ctypes binding of the C ABI in include/ks.h.

Argument marshalling only: every step of key switching runs in the CUDA
library.  Device buffers are torch tensors (dtype int64 holding the uint64
bit patterns); streams are torch CUDA streams.  If the library has not been
built, ``lib()`` raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

KS_OK, KS_EINVAL, KS_ENOMEM, KS_ECUDA, KS_ETIMEOUT, KS_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
MP, DC, OC, AUTO = 0, 1, 2, 3
DATAFLOWS = {"MP": MP, "DC": DC, "OC": OC, "AUTO": AUTO}

_lock = threading.Lock()
_lib = None


class KSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ks error {code}: {msg}")
        self.code = code


class Shard(ctypes.Structure):
    """ks_shard: the full Q towers [q_begin, q_end) and special towers
    [p_begin, p_end) one rank owns in a tower-sharded key switch."""
    _fields_ = [("q_begin", ctypes.c_uint32), ("q_end", ctypes.c_uint32), ("p_begin", ctypes.c_uint32),
                ("p_end", ctypes.c_uint32)]


class Schedule(ctypes.Structure):
    """ks_schedule: dataflow (MP/DC/OC), oc_variant (0 fused rows, 1 split,
    2 whole basis, 3 one cluster kernel per output tower), chunk (jobs per batched launch group), order (0 given,
    1 by level, 2 by key), ntt (0 two launches, 1/2 cluster launch, -1 the
    parameter set's option) and bconv (0 CUDA cores, 1 tensor cores, -1 the
    option)."""
    _fields_ = [("dataflow", ctypes.c_int32), ("oc_variant", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("order", ctypes.c_int32), ("ntt", ctypes.c_int32), ("bconv", ctypes.c_int32)]

    def __init__(self, dataflow=0, oc_variant=0, chunk=1, order=0, ntt=-1, bconv=-1):
        super().__init__(dataflow, oc_variant, chunk, order, ntt, bconv)

    def as_tuple(self):
        """The structural fields (what the cost model ranks)."""
        return (self.dataflow, self.oc_variant, self.chunk, self.order)

    def impl(self):
        """The implementation fields (ntt, bconv)."""
        return (self.ntt, self.bconv)

    def __repr__(self):
        return (f"Schedule(dataflow={self.dataflow}, oc_variant={self.oc_variant}, chunk={self.chunk}, "
                f"order={self.order}, ntt={self.ntt}, bconv={self.bconv})")


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_inflight_jobs", ctypes.c_uint32), ("max_batch", ctypes.c_uint32),
                ("n_streams", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("hbm_budget_bytes", ctypes.c_uint64)]


class Request(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("key", ctypes.c_void_p), ("level_towers", ctypes.c_uint32),
                ("d_in", ctypes.c_void_p), ("d_out0", ctypes.c_void_p), ("d_out1", ctypes.c_void_p)]


class HostJob(ctypes.Structure):
    _fields_ = [("key", ctypes.c_void_p), ("level_towers", ctypes.c_uint32),
                ("h_in", ctypes.c_void_p), ("h_out0", ctypes.c_void_p), ("h_out1", ctypes.c_void_p)]


class Job(ctypes.Structure):
    _fields_ = [("key", ctypes.c_void_p), ("level_towers", ctypes.c_uint32),
                ("d_in", ctypes.c_void_p), ("d_out0", ctypes.c_void_p), ("d_out1", ctypes.c_void_p)]


def lib_path() -> str:
    """Path of the in-tree CUDA library."""
    return _build.LIB


def lib():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing at {path}: run paper_2311_01598_gb300.build.build()")
        L = ctypes.CDLL(path)
        vp, u32, u64, ci = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        pvp = ctypes.POINTER(ctypes.c_void_p)
        L.ks_last_error.restype = ctypes.c_char_p
        L.ks_params_create.argtypes = [u32, u32, u32, u32, vp, vp, u32, pvp]
        L.ks_params_destroy.argtypes = [vp]
        L.ks_params_destroy.restype = None
        L.ks_params_info.argtypes = [vp, vp, vp, ctypes.POINTER(u32), ctypes.POINTER(u32)]
        L.ks_keygen_upload.argtypes = [vp, vp, vp, u64, vp, pvp]
        L.ks_keygen_upload_compressed.argtypes = [vp, vp, vp, u64, vp, pvp]
        L.ks_key_upload_raw.argtypes = [vp, vp, vp, pvp]
        L.ks_key_destroy.argtypes = [vp]
        L.ks_key_destroy.restype = None
        L.ks_key_bytes.argtypes = [vp]
        L.ks_key_bytes.restype = ctypes.c_size_t
        L.ks_switch.argtypes = [vp, vp, u32, vp, vp, vp, ci, vp]
        L.ks_switch_batch.argtypes = [vp, u32, ctypes.POINTER(Job), ci, vp]
        L.ks_ntt.argtypes = [vp, u32, u32, vp, ci, vp]
        L.ks_modup.argtypes = [vp, u32, vp, vp, vp]
        L.ks_moddown.argtypes = [vp, u32, vp, vp, vp]
        L.ks_switch_batch_host.argtypes = [vp, u32, ctypes.POINTER(HostJob), ci, vp]
        L.ks_switch_batch_sched.argtypes = [vp, u32, ctypes.POINTER(Job), ctypes.POINTER(Schedule), vp]
        L.ks_switch_batch_sched.restype = ci
        L.ks_get_default_schedule.argtypes = [vp, ctypes.POINTER(Schedule)]
        L.ks_get_default_schedule.restype = ci
        L.ks_set_default_schedule.argtypes = [vp, ctypes.POINTER(Schedule)]
        L.ks_set_default_schedule.restype = ci
        L.ks_switch_noalloc.argtypes = [vp, vp, u32, vp, vp, vp, vp]
        L.ks_switch_noalloc.restype = ci
        L.ks_switch_noalloc_max_words.argtypes = []
        L.ks_switch_noalloc_max_words.restype = ctypes.c_size_t
        L.ks_tune_candidates.argtypes = [vp, u32, ctypes.POINTER(Schedule), ctypes.POINTER(u32)]
        L.ks_autotune.argtypes = [vp, u32, ctypes.POINTER(Job), u32, vp, u32, ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(Schedule)]
        L.ks_autotune_impl.argtypes = [vp, u32, ctypes.POINTER(Job), u32, vp, ctypes.POINTER(Schedule),
                                       ctypes.POINTER(ctypes.c_float), ctypes.POINTER(Schedule)]
        L.ks_tune_cache_put.argtypes = [vp, u32, u32, ctypes.POINTER(Schedule)]
        L.ks_tune_cache_get.argtypes = [vp, u32, u32, ctypes.POINTER(Schedule)]
        L.ks_tune_cache_save.argtypes = [vp, ctypes.c_char_p]
        L.ks_tune_cache_load.argtypes = [vp, ctypes.c_char_p]
        L.ks_key_synthetic.argtypes = [vp, u64, vp, pvp]
        L.ks_params_set_cost_model.argtypes = [vp, vp, ctypes.c_float, ctypes.c_float]
        L.ks_special_primes.argtypes = [u32, u32, ctypes.POINTER(ctypes.c_uint64)]
        L.ks_special_primes.restype = ci
        L.ks_key_shard.argtypes = [vp, ctypes.POINTER(Shard), vp, pvp]
        L.ks_key_shard.restype = ci
        L.ks_shard_scratch_words.argtypes = [vp, ctypes.POINTER(Shard), u32]
        L.ks_shard_scratch_words.restype = ctypes.c_size_t
        L.ks_shard_prep.argtypes = [vp, ctypes.POINTER(Shard), u32, vp, vp, vp]
        L.ks_shard_prep.restype = ci
        L.ks_shard_keyprod.argtypes = [vp, vp, u32, vp, vp, vp, vp, vp]
        L.ks_shard_keyprod.restype = ci
        L.ks_shard_moddown.argtypes = [vp, vp, u32, vp, vp, vp, vp, vp, vp]
        L.ks_shard_moddown.restype = ci
        L.ks_predict_schedule.argtypes = [vp, u32, ctypes.POINTER(Job), vp, ctypes.POINTER(Schedule),
                                          ctypes.POINTER(ctypes.c_float)]
        L.ks_cost_features.argtypes = [vp, u32, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_float)]
        L.ks_mlp_create.argtypes = [u32, ctypes.POINTER(u32), u64, pvp]
        L.ks_mlp_destroy.argtypes = [vp]
        L.ks_mlp_destroy.restype = None
        L.ks_mlp_num_params.argtypes = [vp]
        L.ks_mlp_num_params.restype = ctypes.c_size_t
        L.ks_mlp_get_params.argtypes = [vp, vp]
        L.ks_mlp_set_params.argtypes = [vp, vp]
        L.ks_mlp_forward.argtypes = [vp, u32, vp, vp, vp]
        L.ks_mlp_gradients.argtypes = [vp, u32, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_float), vp]
        L.ks_mlp_train_step.argtypes = [vp, u32, vp, vp, vp, ctypes.c_float, ctypes.POINTER(ctypes.c_float), vp]
        for name in ("ks_tune_candidates", "ks_autotune", "ks_autotune_impl", "ks_tune_cache_put", "ks_tune_cache_get",
                     "ks_tune_cache_save", "ks_tune_cache_load", "ks_key_synthetic", "ks_params_set_cost_model",
                     "ks_predict_schedule", "ks_cost_features", "ks_mlp_create",
                     "ks_mlp_get_params", "ks_mlp_set_params", "ks_mlp_forward", "ks_mlp_gradients",
                     "ks_mlp_train_step"):
            getattr(L, name).restype = ci
        L.ks_server_create.argtypes = [ctypes.POINTER(ServerConfig), pvp]
        L.ks_server_destroy.argtypes = [vp]
        L.ks_server_destroy.restype = None
        L.ks_server_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(u64)]
        L.ks_server_wait.argtypes = [vp, u64, u32]
        L.ks_server_times.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
        L.ks_server_stats.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.ks_server_run_trace.argtypes = [vp, u32, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), u32]
        for name in ("ks_server_create", "ks_server_submit", "ks_server_wait", "ks_server_times", "ks_server_stats",
                     "ks_server_run_trace"):
            getattr(L, name).restype = ci
        L.ks_params_set_option.argtypes = [vp, ci, ci]
        L.ks_params_set_option.restype = ci
        L.ks_device_status.argtypes = [vp, ci, ctypes.POINTER(u32)]
        L.ks_device_status.restype = ci
        L.ks_switch_hoisted.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.c_uint32, vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
        L.ks_switch_hoisted.restype = ci
        L.ks_automorph.argtypes = [vp, u32, u32, u64, vp, vp, ci, vp]
        L.ks_automorph.restype = ci
        L.ks_probe_int_pipes.argtypes = [ctypes.POINTER(ctypes.c_double), ci]
        L.ks_probe_int_pipes.restype = ci
        L.ks_probe_alu.argtypes = [ci, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.ks_probe_alu.restype = ci
        L.ks_probe_inv_bfly.argtypes = [ci, ctypes.POINTER(ctypes.c_double)]
        L.ks_probe_inv_bfly.restype = ci
        L.ks_kernel_launches.argtypes = []
        L.ks_kernel_launches.restype = ctypes.c_uint64
        L.ks_profile_enable.argtypes = [ci]
        L.ks_profile_enable.restype = None
        L.ks_profile_collect.argtypes = [u32, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(u32), ctypes.POINTER(u32)]
        for name in ("ks_params_create", "ks_params_info", "ks_keygen_upload", "ks_keygen_upload_compressed",
                     "ks_key_upload_raw", "ks_switch",
                     "ks_switch_batch", "ks_ntt", "ks_modup", "ks_moddown", "ks_switch_batch_host",
                     "ks_profile_collect"):
            getattr(L, name).restype = ci
        _lib = L
        return L


def exported_symbols() -> list[str]:
    """Names declared in include/ks.h that the library must export."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ks.h")
    with open(hdr) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(ks_[a-z_0-9]+)\s*\(", text)))


def check(rc: int) -> None:
    """Raise KSError with ks_last_error() unless rc is KS_OK."""
    if rc != KS_OK:
        raise KSError(rc, lib().ks_last_error().decode())


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return ctypes.c_void_p(t.ctypes.data)
    assert t.is_contiguous(), "tensor must be contiguous"
    return ctypes.c_void_p(t.data_ptr())


class Key:
    def __init__(self, params: "Params", handle: int):
        self.params = params
        self.handle = handle

    @property
    def nbytes(self) -> int:
        """ks_key_bytes: device memory the key occupies."""
        return int(lib().ks_key_bytes(self.handle))

    def close(self) -> None:
        """ks_key_destroy (idempotent)."""
        if self.handle:
            lib().ks_key_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Params:
    """A parameter set (N = 2^logN, nq = L+1 Q primes, kp = K P primes, dnum)."""

    def __init__(self, logN: int, nq: int, kp: int, dnum: int, prime_bits: int = 54, q=None, p=None):
        L = lib()
        h = ctypes.c_void_p()
        qa = pa = None
        if q is not None:
            qa = np.ascontiguousarray(q, dtype=np.uint64)
            pa = np.ascontiguousarray(p, dtype=np.uint64)
        check(L.ks_params_create(logN, nq, kp, dnum, _ptr(qa), _ptr(pa), prime_bits, ctypes.byref(h)))
        self.handle = h.value
        self.logN, self.N, self.nq, self.kp, self.dnum = logN, 1 << logN, nq, kp, dnum
        qo = np.zeros(nq, dtype=np.uint64)
        po = np.zeros(kp, dtype=np.uint64)
        alpha, ndig = ctypes.c_uint32(), ctypes.c_uint32()
        check(L.ks_params_info(self.handle, _ptr(qo), _ptr(po), ctypes.byref(alpha), ctypes.byref(ndig)))
        self.q = [int(x) for x in qo]
        self.p = [int(x) for x in po]
        self.alpha, self.ndig = alpha.value, ndig.value

    def close(self) -> None:
        """ks_params_destroy (idempotent)."""
        if self.handle:
            lib().ks_params_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def active_digits(self, nact: int) -> int:
        """Digits holding towers at level nact: ceil(nact / alpha)."""
        return (nact + self.alpha - 1) // self.alpha

    # -- keys ---------------------------------------------------------------
    def keygen(self, s, s_prime, seed: int, stream=None) -> Key:
        """ks_keygen_upload: a key switching s_prime to s (s ternary int8[N],
        s_prime int64[N] in coefficient form), sampled from seed."""
        s = np.ascontiguousarray(s, dtype=np.int8)
        sp = np.ascontiguousarray(s_prime, dtype=np.int64)
        h = ctypes.c_void_p()
        check(lib().ks_keygen_upload(self.handle, _ptr(s), _ptr(sp), seed & (2**64 - 1), _stream_handle(stream),
                                     ctypes.byref(h)))
        return Key(self, h.value)

    def keygen_compressed(self, s, s_prime, seed: int, stream=None) -> Key:
        """ks_keygen_upload_compressed: b_j stored, a_j regenerated by the
        kernels from the seed (half the key's device memory and traffic)."""
        s = np.ascontiguousarray(s, dtype=np.int8)
        sp = np.ascontiguousarray(s_prime, dtype=np.int64)
        h = ctypes.c_void_p()
        check(lib().ks_keygen_upload_compressed(self.handle, _ptr(s), _ptr(sp), seed & (2**64 - 1),
                                                _stream_handle(stream), ctypes.byref(h)))
        return Key(self, h.value)

    def upload_key(self, evk: np.ndarray, stream=None) -> Key:
        """ks_key_upload_raw: an evaluation key given in full,
        [ndig][2][nq+kp][N] canonical words in evaluation form."""
        evk = np.ascontiguousarray(evk, dtype=np.uint64)
        assert evk.shape == (self.ndig, 2, self.nq + self.kp, self.N)
        h = ctypes.c_void_p()
        check(lib().ks_key_upload_raw(self.handle, _ptr(evk), _stream_handle(stream), ctypes.byref(h)))
        return Key(self, h.value)

    # -- key switching --------------------------------------------------------
    def switch(self, key: Key, nact: int, d, out0, out1, dataflow=OC, stream=None) -> None:
        """ks_switch: key switch of d ([nact][N], evaluation form) into
        out0, out1 under dataflow "MP", "DC", "OC" or "AUTO"."""
        df = DATAFLOWS[dataflow] if isinstance(dataflow, str) else dataflow
        check(lib().ks_switch(self.handle, key.handle, nact, _ptr(d), _ptr(out0), _ptr(out1), df,
                              _stream_handle(stream)))

    def set_bconv_tensor(self, on: bool) -> None:
        """KS_OPT_BCONV_TENSOR: base conversions on the tensor cores (default)
        or on the CUDA cores."""
        check(lib().ks_params_set_option(self.handle, 1, 1 if on else 0))

    def set_batch_lanes(self, lanes: int) -> None:
        """KS_OPT_BATCH_LANES: library streams a large Output-Centric batch is split over."""
        check(lib().ks_params_set_option(self.handle, 2, int(lanes)))

    def set_ntt_cluster(self, on: bool) -> None:
        """KS_OPT_NTT_CLUSTER: each NTT as one thread-block-cluster launch
        (distributed shared memory between its passes) where supported."""
        check(lib().ks_params_set_option(self.handle, 3, int(on)))

    def set_row_stage(self, on: bool) -> None:
        """KS_OPT_NTT_ROW_STAGE: forward row passes staged in shared memory by
        bulk copies (persistent blocks, next block's copy in flight)."""
        check(lib().ks_params_set_option(self.handle, 4, 1 if on else 0))

    def device_status(self, clear: bool = True) -> int:
        """ks_device_status: bit 0 = a tensor-core kernel's bounded MMA wait
        gave up, bit 1 = a staged row pass's bounded copy wait gave up."""
        f = ctypes.c_uint32()
        check(lib().ks_device_status(self.handle, 1 if clear else 0, ctypes.byref(f)))
        return int(f.value)

    def switch_hoisted(self, keys, galois, nact: int, d, outs0, outs1, stream=None) -> None:
        """ks_switch_hoisted: key switches of the rotations X -> X^g (g in
        galois, keys[r] the key of rotation r) of d with one shared ModUp;
        outs0[r], outs1[r] receive rotation r."""
        R = len(keys)
        if not (len(galois) == len(outs0) == len(outs1) == R):
            raise ValueError("keys, galois and outputs must have the same length")
        ka = (ctypes.c_void_p * max(1, R))(*[k.handle for k in keys])
        ga = (ctypes.c_uint64 * max(1, R))(*[int(g) for g in galois])
        o0 = (ctypes.c_void_p * max(1, R))(*[_ptr(o).value for o in outs0])
        o1 = (ctypes.c_void_p * max(1, R))(*[_ptr(o).value for o in outs1])
        check(lib().ks_switch_hoisted(self.handle, R, ka, ga, nact, _ptr(d), o0, o1, _stream_handle(stream)))

    def automorph(self, first_tower: int, galois: int, d_in, d_out, accumulate: bool = False, stream=None) -> None:
        """ks_automorph: d_out = phi_g(d_in) (or d_out + phi_g(d_in) with
        accumulate), X -> X^g on the evaluation slots of every tower."""
        check(lib().ks_automorph(self.handle, first_tower, d_in.shape[0], int(galois), _ptr(d_in), _ptr(d_out),
                                 1 if accumulate else 0, _stream_handle(stream)))

    def switch_noalloc(self, key: Key, nact: int, d, out0, out1, stream=None) -> None:
        """ks_switch_noalloc: Output-Centric key switch using the library's
        static scratch array instead of allocated scratch."""
        check(lib().ks_switch_noalloc(self.handle, key.handle, nact, _ptr(d), _ptr(out0), _ptr(out1),
                                      _stream_handle(stream)))

    def switch_batch(self, jobs, dataflow=OC, stream=None) -> None:
        """ks_switch_batch: jobs is an iterable of (key, nact, d, out0, out1);
        "AUTO" uses the tuned schedule of the batch's signature."""
        df = DATAFLOWS[dataflow] if isinstance(dataflow, str) else dataflow
        jobs = list(jobs)
        arr = (Job * max(1, len(jobs)))()
        for i, (key, nact, d, o0, o1) in enumerate(jobs):
            arr[i] = Job(key.handle, nact, _ptr(d).value, _ptr(o0).value, _ptr(o1).value)
        check(lib().ks_switch_batch(self.handle, len(jobs), arr, df, _stream_handle(stream)))

    @staticmethod
    def _jobs(jobs):
        jobs = list(jobs)
        arr = (Job * max(1, len(jobs)))()
        for i, (key, nact, d, o0, o1) in enumerate(jobs):
            arr[i] = Job(key.handle, nact, _ptr(d).value, _ptr(o0).value, _ptr(o1).value)
        return arr, len(jobs)

    def switch_batch_sched(self, jobs, schedule: "Schedule", stream=None) -> None:
        """ks_switch_batch_sched: the batch run under an explicit schedule."""
        arr, n = self._jobs(jobs)
        check(lib().ks_switch_batch_sched(self.handle, n, arr, ctypes.byref(schedule), _stream_handle(stream)))

    def default_schedule(self) -> "Schedule":
        """ks_get_default_schedule: the schedule of single calls and non-AUTO batches."""
        sc = Schedule()
        check(lib().ks_get_default_schedule(self.handle, ctypes.byref(sc)))
        return sc

    def set_default_schedule(self, schedule: "Schedule") -> None:
        """ks_set_default_schedule."""
        check(lib().ks_set_default_schedule(self.handle, ctypes.byref(schedule)))

    # -- autotuning -----------------------------------------------------------
    def tune_candidates(self) -> list:
        """ks_tune_candidates: the structural schedules, in the cost model's order."""
        n = ctypes.c_uint32()
        check(lib().ks_tune_candidates(self.handle, 0, None, ctypes.byref(n)))
        arr = (Schedule * n.value)()
        check(lib().ks_tune_candidates(self.handle, n.value, arr, ctypes.byref(n)))
        return [arr[i] for i in range(n.value)]

    def autotune(self, jobs, reps: int = 3, stream=None, with_impl: bool = False):
        """ks_autotune: times the structural candidates (returned ms, in
        candidate order), then the fastest one under each implementation
        pair (their four ms appended when with_impl); returns (best, [ms])
        and caches best for KS_AUTO."""
        arr, n = self._jobs(jobs)
        nc = len(self.tune_candidates()) + (4 if with_impl else 0)
        ms = (ctypes.c_float * nc)()
        best = Schedule()
        check(lib().ks_autotune(self.handle, n, arr, reps, _stream_handle(stream), nc, ms, ctypes.byref(best)))
        return best, [float(x) for x in ms]

    def autotune_impl(self, jobs, base: "Schedule", reps: int = 3, stream=None):
        """Time `base` under the implementation pairs (ntt, bconv) = (0,1),
        (1,1), (0,0), (1,0); returns (best, [ms])."""
        arr, n = self._jobs(jobs)
        ms = (ctypes.c_float * 4)()
        best = Schedule()
        check(lib().ks_autotune_impl(self.handle, n, arr, reps, _stream_handle(stream), ctypes.byref(base), ms,
                                     ctypes.byref(best)))
        return best, [float(x) for x in ms]

    def tune_cache_put(self, n_jobs: int, mean_level: int, schedule: "Schedule") -> None:
        """ks_tune_cache_put: the schedule KS_AUTO uses for this batch signature."""
        check(lib().ks_tune_cache_put(self.handle, n_jobs, mean_level, ctypes.byref(schedule)))

    def tune_cache_get(self, n_jobs: int, mean_level: int):
        """ks_tune_cache_get: the cached schedule of a signature, or None."""
        sc = Schedule()
        rc = lib().ks_tune_cache_get(self.handle, n_jobs, mean_level, ctypes.byref(sc))
        return sc if rc == KS_OK else None

    def tune_cache_save(self, path: str) -> None:
        """ks_tune_cache_save: the cache as text keyed by device and parameter set."""
        check(lib().ks_tune_cache_save(self.handle, path.encode()))

    def tune_cache_load(self, path: str) -> None:
        """ks_tune_cache_load: lines for this device and parameter set are merged in."""
        check(lib().ks_tune_cache_load(self.handle, path.encode()))

    def set_cost_model(self, mlp, t_mean: float = 0.0, t_scale: float = 1.0) -> None:
        """ks_params_set_cost_model: attach a trained Mlp (None detaches);
        KS_AUTO then runs it on a tuning-cache miss.  The Mlp must outlive
        its use by this parameter set."""
        self._cost_model = mlp  # keeps the model alive while attached
        check(lib().ks_params_set_cost_model(self.handle, mlp.handle if mlp is not None else None, float(t_mean),
                                             float(t_scale)))

    def predict_schedule(self, jobs, stream=None):
        """ks_predict_schedule: (the attached model's schedule for the batch,
        its de-normalised outputs: log ms per key switch per structural
        candidate, then per implementation pair)."""
        arr, n = self._jobs(jobs)
        nout = len(self.tune_candidates()) + 4
        pred = (ctypes.c_float * nout)()
        sc = Schedule()
        check(lib().ks_predict_schedule(self.handle, n, arr, _stream_handle(stream), ctypes.byref(sc), pred))
        return sc, [float(x) for x in pred]

    def cost_features(self, jobs) -> np.ndarray:
        """ks_cost_features: the cost model's 10 inputs for a batch."""
        arr, n = self._jobs(jobs)
        x = (ctypes.c_float * 10)()
        check(lib().ks_cost_features(self.handle, n, arr, x))
        return np.array(list(x), dtype=np.float32)

    # -- tower-sharded key switching ------------------------------------------
    def key_shard(self, key: Key, shard: "Shard", stream=None) -> Key:
        """ks_key_shard: a key holding only the shard's towers (copied on the device)."""
        h = ctypes.c_void_p()
        check(lib().ks_key_shard(key.handle, ctypes.byref(shard), _stream_handle(stream), ctypes.byref(h)))
        return Key(self, h.value)

    def shard_scratch_words(self, shard: "Shard", nact: int) -> int:
        """ks_shard_scratch_words: scratch of one rank's keyprod/moddown at level nact."""
        return int(lib().ks_shard_scratch_words(self.handle, ctypes.byref(shard), nact))

    def shard_prep(self, shard: "Shard", nact: int, d_own, y_own, stream=None) -> None:
        """ks_shard_prep: ModUp P1 of the rank's input towers."""
        check(lib().ks_shard_prep(self.handle, ctypes.byref(shard), nact, _ptr(d_own), _ptr(y_own),
                                  _stream_handle(stream)))

    def shard_keyprod(self, skey: Key, nact: int, y_all, d_own, cp_own, scratch, stream=None) -> None:
        """ks_shard_keyprod: c' of the rank's towers from the gathered y;
        the special rows of cp_own then hold w_own."""
        check(lib().ks_shard_keyprod(self.handle, skey.handle, nact, _ptr(y_all), _ptr(d_own), _ptr(cp_own),
                                     _ptr(scratch), _stream_handle(stream)))

    def shard_moddown(self, skey: Key, nact: int, w_all, cp_own, out0_own, out1_own, scratch, stream=None) -> None:
        """ks_shard_moddown: the rank's output towers from the gathered w."""
        check(lib().ks_shard_moddown(self.handle, skey.handle, nact, _ptr(w_all), _ptr(cp_own), _ptr(out0_own),
                                     _ptr(out1_own), _ptr(scratch), _stream_handle(stream)))

    def key_synthetic(self, seed: int, stream=None) -> Key:
        """ks_key_synthetic: a key of pseudo-random residues (timing and tuning only)."""
        h = ctypes.c_void_p()
        check(lib().ks_key_synthetic(self.handle, seed & (2**64 - 1), _stream_handle(stream), ctypes.byref(h)))
        return Key(self, h.value)

    def switch_batch_host(self, jobs, dataflow=OC, stream=None) -> None:
        """jobs: iterable of (key, nact, h_in, h_out0, h_out1) with host
        buffers (pinned torch tensors or numpy arrays)."""
        df = DATAFLOWS[dataflow] if isinstance(dataflow, str) else dataflow
        jobs = list(jobs)
        arr = (HostJob * max(1, len(jobs)))()
        for i, (key, nact, hi, h0, h1) in enumerate(jobs):
            arr[i] = HostJob(key.handle, nact, _ptr(hi).value, _ptr(h0).value, _ptr(h1).value)
        check(lib().ks_switch_batch_host(self.handle, len(jobs), arr, df, _stream_handle(stream)))

    # -- stages ----------------------------------------------------------------
    def ntt(self, first_tower: int, data, inverse: bool = False, stream=None) -> None:
        """ks_ntt: in-place forward (canonical output) or inverse negacyclic NTT
        of data[i] in the tower first_tower + i."""
        n = data.shape[0]
        check(lib().ks_ntt(self.handle, first_tower, n, _ptr(data), 1 if inverse else 0, _stream_handle(stream)))

    def modup(self, nact: int, d, ext, stream=None) -> None:
        """ks_modup: ModUp P1-P3 of d into the raised digits ext."""
        check(lib().ks_modup(self.handle, nact, _ptr(d), _ptr(ext), _stream_handle(stream)))

    def moddown(self, nact: int, cp, out, stream=None) -> None:
        """ks_moddown: ModDown P1-P4 of cp (over D_l) into out."""
        check(lib().ks_moddown(self.handle, nact, _ptr(cp), _ptr(out), _stream_handle(stream)))


# -- serving ---------------------------------------------------------------------------
class Server:
    """Continuous-batching key-switch server (ks_server_*)."""

    def __init__(self, max_inflight_jobs=32, max_batch=16, n_streams=2, hbm_budget_bytes=8 << 30):
        cfg = ServerConfig(max_inflight_jobs, max_batch, n_streams, 0, hbm_budget_bytes)
        h = ctypes.c_void_p()
        check(lib().ks_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h.value
        self._keep = []

    def close(self):
        """ks_server_destroy: finish every request, then stop (idempotent)."""
        if self.handle:
            lib().ks_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def request(params, key, nact, d, out0, out1) -> Request:
        """A ks_request for submit or run_trace."""
        return Request(params.handle, key.handle, nact, _ptr(d).value, _ptr(out0).value, _ptr(out1).value)

    def submit(self, params, key, nact, d, out0, out1) -> int:
        """ks_server_submit: queue a key switch; returns its ticket."""
        t = ctypes.c_uint64()
        r = self.request(params, key, nact, d, out0, out1)
        check(lib().ks_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 60000) -> int:
        """ks_server_wait: KS_OK once the request is done, KS_ETIMEOUT if not yet."""
        return int(lib().ks_server_wait(self.handle, ticket, timeout_ms))

    def times(self, ticket: int):
        """ks_server_times: (arrival, admission, completion) in seconds of the server's clock."""
        a, m, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(lib().ks_server_times(self.handle, ticket, ctypes.byref(a), ctypes.byref(m), ctypes.byref(d)))
        return a.value, m.value, d.value

    def stats(self):
        """ks_server_stats: requests done, batches launched, largest batch."""
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        check(lib().ks_server_stats(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"done": a.value, "batches": b.value, "max_batch": c.value}

    def run_trace(self, reqs, arrival_s, timeout_ms: int = 600000):
        """reqs: list of Request; arrival_s: seconds from now.  Returns latencies (s)."""
        n = len(reqs)
        arr = (Request * max(1, n))(*reqs)
        at = (ctypes.c_double * max(1, n))(*[float(x) for x in arrival_s])
        lat = (ctypes.c_double * max(1, n))()
        check(lib().ks_server_run_trace(self.handle, n, arr, at, lat, timeout_ms))
        return np.array([lat[i] for i in range(n)])


# -- learned cost model --------------------------------------------------------------
class Mlp:
    """FP32 MLP trained and evaluated by the library's kernels (ks_mlp_*).
    Inputs and targets are torch float32 CUDA tensors [batch][width]."""

    def __init__(self, dims, seed: int = 1):
        arr = (ctypes.c_uint32 * len(dims))(*dims)
        h = ctypes.c_void_p()
        check(lib().ks_mlp_create(len(dims) - 1, arr, seed & (2**64 - 1), ctypes.byref(h)))
        self.handle = h.value
        self.dims = list(dims)

    def close(self):
        """ks_mlp_destroy (idempotent)."""
        if self.handle:
            lib().ks_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nparams(self) -> int:
        """ks_mlp_num_params: weights and biases of every layer."""
        return int(lib().ks_mlp_num_params(self.handle))

    def get_params(self) -> np.ndarray:
        """ks_mlp_get_params: the flat parameter vector (host copy)."""
        out = np.zeros(self.nparams, dtype=np.float32)
        check(lib().ks_mlp_get_params(self.handle, _ptr(out)))
        return out

    def set_params(self, p) -> None:
        """ks_mlp_set_params: replace the flat parameter vector."""
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparams
        check(lib().ks_mlp_set_params(self.handle, _ptr(p)))

    def forward(self, x, stream=None):
        """ks_mlp_forward: y = MLP(x) for x [batch][dims[0]] on the GPU."""
        import torch
        y = torch.empty((x.shape[0], self.dims[-1]), dtype=torch.float32, device=x.device)
        check(lib().ks_mlp_forward(self.handle, x.shape[0], _ptr(x), _ptr(y), _stream_handle(stream)))
        return y

    def gradients(self, x, t, mask=None, stream=None):
        """ks_mlp_gradients: (masked mean-square loss, flat gradient)."""
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = ctypes.c_float()
        check(lib().ks_mlp_gradients(self.handle, x.shape[0], _ptr(x), _ptr(t), _ptr(mask), _ptr(g),
                                     ctypes.byref(loss), _stream_handle(stream)))
        return float(loss.value), g

    def train_step(self, x, t, lr: float, mask=None, stream=None) -> float:
        """ks_mlp_train_step: one full-batch Adam step; returns the loss before it."""
        loss = ctypes.c_float()
        check(lib().ks_mlp_train_step(self.handle, x.shape[0], _ptr(x), _ptr(t), _ptr(mask), lr,
                                      ctypes.byref(loss), _stream_handle(stream)))
        return float(loss.value)


# -- measurement hooks ---------------------------------------------------------------
def kernel_launches() -> int:
    """ks_kernel_launches: library kernel launches so far in this process."""
    return int(lib().ks_kernel_launches())


def probe_int_pipes() -> dict:
    """ks_probe_int_pipes: lanes per SM per clock of single integer instructions."""
    out = (ctypes.c_double * 5)()
    check(lib().ks_probe_int_pipes(out, 5))
    return dict(zip(("mad.lo.u32", "mad.wide.u32", "mul.lo.u64", "mul.hi.u64", "add.u32"), [round(x, 2) for x in out]))


def probe_alu(iters: int = 4096) -> tuple[float, float]:
    """(forward butterflies/s, base-conversion MACs/s) ceilings of this GPU."""
    b, m = ctypes.c_double(), ctypes.c_double()
    check(lib().ks_probe_alu(iters, ctypes.byref(b), ctypes.byref(m)))
    return b.value, m.value


def probe_inv_bfly(iters: int = 4096) -> float:
    """Inverse butterflies/s ceiling of this GPU."""
    b = ctypes.c_double()
    check(lib().ks_probe_inv_bfly(iters, ctypes.byref(b)))
    return b.value


def profile_enable(on: bool = True) -> None:
    """ks_profile_enable: bracket every library launch with CUDA events."""
    lib().ks_profile_enable(1 if on else 0)


def profile_collect(max_names: int = 64) -> dict:
    """{kernel name: (launches, total ms)} since the last collect."""
    names = ctypes.create_string_buffer(48 * max_names)
    ms = (ctypes.c_double * max_names)()
    cnt = (ctypes.c_uint32 * max_names)()
    n = ctypes.c_uint32()
    check(lib().ks_profile_collect(max_names, names, ms, cnt, ctypes.byref(n)))
    out = {}
    for i in range(min(n.value, max_names)):
        nm = names.raw[48 * i:48 * i + 48].split(b"\0", 1)[0].decode()
        out[nm] = (int(cnt[i]), float(ms[i]))
    return out


# -- torch helpers (device memory only) ------------------------------------------
def special_primes(bits: int, count: int) -> list:
    """ks_special_primes: the count largest primes k*2^32 + 1 below 2^bits,
    descending (for explicit prime lists; the two-pass NTTs use a cheaper
    butterfly product when every prime of a parameter set has this form)."""
    out = (ctypes.c_uint64 * count)()
    check(lib().ks_special_primes(bits, count, out))
    return [int(x) for x in out]


def to_device(a: np.ndarray, device="cuda"):
    """uint64 numpy array -> int64 torch tensor on the GPU (same bits)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(device)


def to_host(t) -> np.ndarray:
    """int64 torch tensor -> uint64 numpy array (same bits)."""
    return t.cpu().numpy().view(np.uint64)


def empty(shape, device="cuda"):
    """Uninitialised int64 device tensor for library outputs."""
    import torch
    return torch.empty(shape, dtype=torch.int64, device=device)
