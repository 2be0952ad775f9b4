"""ks_switch_noalloc: the key switch for callers that cannot allocate device
memory while running (pool-owned device memory, or loops that cannot afford
cudaMalloc's synchronisation).  Its output must equal ks_switch's, bit for
bit, on consecutive calls that reuse the one static scratch array; requests
larger than the array are refused before anything runs.

This file is named to be collected last, so that a run stopping at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2311_01598_gb300 import inputs
from tests._gpu import built_lib, need_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_matches_switch_on_consecutive_calls():
    need_gpu()
    ks = built_lib()
    P = ks.Params(13, 10, 4, 3)
    s = inputs.ternary_secret(P.N, 21)
    key = P.keygen(s, inputs.galois_secret(s, 5), seed=22)
    for call, nact in enumerate((10, 7)):  # two calls in a row, different level and data
        d = ks.to_device(inputs.uniform_towers(P.q[:nact], P.N, seed=300 + call))
        w0, w1 = ks.empty((nact, P.N)), ks.empty((nact, P.N))
        P.switch(key, nact, d, w0, w1, "OC")
        g0, g1 = ks.empty((nact, P.N)), ks.empty((nact, P.N))
        rc = ks.lib().ks_switch_noalloc(P.handle, key.handle, nact, ctypes.c_void_p(d.data_ptr()),
                                        ctypes.c_void_p(g0.data_ptr()), ctypes.c_void_p(g1.data_ptr()),
                                        ks._stream_handle(None))
        assert rc == ks.KS_OK, ks.lib().ks_last_error()
        assert np.array_equal(ks.to_host(g0), ks.to_host(w0)), f"out0, call {call}"
        assert np.array_equal(ks.to_host(g1), ks.to_host(w1)), f"out1, call {call}"


def test_noalloc_rejects_requests_beyond_the_static_buffer():
    need_gpu()
    ks = built_lib()
    P = ks.Params(16, 24, 8, 3)   # needs about 13.6 M words at the top level
    s = inputs.ternary_secret(P.N, 1)
    key = P.keygen(s, inputs.galois_secret(s, 5), seed=2)
    d, o0, o1 = ks.empty((24, P.N)), ks.empty((24, P.N)), ks.empty((24, P.N))
    rc = ks.lib().ks_switch_noalloc(P.handle, key.handle, 24, ctypes.c_void_p(d.data_ptr()),
                                    ctypes.c_void_p(o0.data_ptr()), ctypes.c_void_p(o1.data_ptr()),
                                    ks._stream_handle(None))
    assert rc == ks.KS_EINVAL
    msg = ks.lib().ks_last_error().decode()
    assert "scratch words" in msg and str(ks.lib().ks_switch_noalloc_max_words()) in msg
