"""ks_switch_noalloc: the key switch for callers that cannot allocate device
memory while running (a server whose device memory is owned by its own pool
allocator, or a loop that cannot afford cudaMalloc's device-wide
synchronisation).  Its output must equal ks_switch's (and the oracle's), bit
for bit, on consecutive calls that reuse the one static scratch array; a call
on a fresh stream must leave the device's free memory unchanged; requests
larger than the array, and misaligned buffers, are refused before anything
runs.

This file is named to be collected last, so that a run stopping at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2311_01598_gb300 import inputs
from tests._gpu import built_lib, need_gpu, pair, secret_pair

pytestmark = pytest.mark.gpu


def _noalloc_c(ks, P, key, nact, d, o0, o1, stream=None):
    """The C entry point called directly through the C ABI."""
    return ks.lib().ks_switch_noalloc(P.handle, key.handle, nact, ctypes.c_void_p(d.data_ptr()),
                                      ctypes.c_void_p(o0.data_ptr()), ctypes.c_void_p(o1.data_ptr()),
                                      ks._stream_handle(stream))


def test_noalloc_matches_switch_on_consecutive_calls():
    need_gpu()
    ks = built_lib()
    P, C = pair(13, 10, 4, 3)
    s, sp = secret_pair(C.N, seed=21)
    evk = C.keygen(s, sp, seed=22)
    key = P.upload_key(evk)
    for call, nact in enumerate((10, 7)):  # two calls in a row, different level and data
        d_h = inputs.uniform_towers(C.q[:nact], C.N, seed=300 + call)
        d = ks.to_device(d_h)
        w0, w1 = ks.empty((nact, C.N)), ks.empty((nact, C.N))
        P.switch(key, nact, d, w0, w1, "OC")
        g0, g1 = ks.empty((nact, C.N)), ks.empty((nact, C.N))
        rc = _noalloc_c(ks, P, key, nact, d, g0, g1)
        assert rc == ks.KS_OK, ks.lib().ks_last_error()
        assert np.array_equal(ks.to_host(g0), ks.to_host(w0)), f"out0, call {call}"
        assert np.array_equal(ks.to_host(g1), ks.to_host(w1)), f"out1, call {call}"
        o0, o1 = C.keyswitch(nact, d_h, evk)
        assert np.array_equal(ks.to_host(g0), o0) and np.array_equal(ks.to_host(g1), o1), f"oracle, call {call}"


def test_noalloc_binding_and_free_memory_unchanged():
    """Through the Python binding (Params.switch_noalloc): after the first
    call on the device (which looks up the array's address), a call on a
    fresh params object and a fresh stream leaves cudaMemGetInfo's free
    memory unchanged, while ks_switch on another fresh stream allocates its
    scratch (so the measurement would see an allocation)."""
    torch = need_gpu()
    ks = built_lib()
    P0, _ = pair(12, 6, 2, 3)
    s, sp = secret_pair(P0.N, seed=31)
    k0 = P0.keygen(s, sp, seed=32)
    d0 = ks.to_device(inputs.uniform_towers(P0.q, P0.N, seed=33))
    P0.switch_noalloc(k0, 6, d0, ks.empty((6, P0.N)), ks.empty((6, P0.N)))  # first call on the device
    torch.cuda.synchronize()

    P, C = pair(12, 6, 2, 3)
    evk = C.keygen(s, sp, seed=34)
    key = P.upload_key(evk)
    d_h = inputs.uniform_towers(C.q, C.N, seed=35)
    d = ks.to_device(d_h)
    g0, g1 = ks.empty((6, C.N)), ks.empty((6, C.N))
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    P.switch_noalloc(key, 6, d, g0, g1, st)
    st.synchronize()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    w0, w1 = C.keyswitch(6, d_h, evk)
    assert np.array_equal(ks.to_host(g0), w0) and np.array_equal(ks.to_host(g1), w1)
    # contrast: ks_switch on a fresh stream allocates its per-stream scratch
    st2 = torch.cuda.Stream()
    o0, o1 = ks.empty((6, C.N)), ks.empty((6, C.N))
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    P.switch(key, 6, d, o0, o1, "OC", st2)
    torch.cuda.synchronize()
    free3, _ = torch.cuda.mem_get_info()
    assert free3 < free2, "ks_switch on a fresh stream was expected to allocate its scratch"
    assert np.array_equal(ks.to_host(o0), w0) and np.array_equal(ks.to_host(o1), w1)


def test_noalloc_rejects_requests_beyond_the_static_buffer():
    need_gpu()
    ks = built_lib()
    P = ks.Params(16, 24, 8, 3)   # 232 limbs = 15.2 million words at the top level
    s = inputs.ternary_secret(P.N, 1)
    key = P.keygen(s, inputs.galois_secret(s, 5), seed=2)
    d, o0, o1 = ks.empty((24, P.N)), ks.empty((24, P.N)), ks.empty((24, P.N))
    rc = _noalloc_c(ks, P, key, 24, d, o0, o1)
    assert rc == ks.KS_EINVAL
    msg = ks.lib().ks_last_error().decode()
    assert "scratch words" in msg and str(ks.lib().ks_switch_noalloc_max_words()) in msg
    assert str(232 * P.N) in msg


def test_noalloc_rejects_misaligned_buffers():
    """An input or output view 8 bytes past an aligned base is refused with
    KS_EINVAL before any launch (the same check as ks_switch), and the next
    call with aligned buffers gives the oracle's result."""
    torch = need_gpu()
    ks = built_lib()
    P, C = pair(11, 4, 2, 2)
    s, sp = secret_pair(C.N, seed=41)
    evk = C.keygen(s, sp, seed=42)
    key = P.upload_key(evk)
    d_h = inputs.uniform_towers(C.q, C.N, seed=43)
    flat = torch.zeros(4 * C.N + 1, dtype=torch.int64, device="cuda")
    flat[1:] = ks.to_device(d_h).reshape(-1)
    dd = flat[1:].view(4, C.N)
    o0, o1 = ks.empty((4, C.N)), ks.empty((4, C.N))
    assert _noalloc_c(ks, P, key, 4, dd, o0, o1) == ks.KS_EINVAL
    assert "16-byte aligned" in ks.lib().ks_last_error().decode()
    oflat = torch.zeros(4 * C.N + 1, dtype=torch.int64, device="cuda")
    assert _noalloc_c(ks, P, key, 4, ks.to_device(d_h), oflat[1:].view(4, C.N), o1) == ks.KS_EINVAL
    assert "16-byte aligned" in ks.lib().ks_last_error().decode()
    assert _noalloc_c(ks, P, key, 4, ks.to_device(d_h), o0, o1) == ks.KS_OK
    w0, w1 = C.keyswitch(4, d_h, evk)
    assert np.array_equal(ks.to_host(o0), w0) and np.array_equal(ks.to_host(o1), w1)
