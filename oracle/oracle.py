"""Python face of the plain CPU oracle (oracle/ks_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports this module, and this module imports nothing from the product
package.  Arrays are numpy uint64 in limb-major layout ``[tower][N]``.

The oracle follows the hybrid key-switching stages of CiFlow Sec. III
(ModUp P1-P5, ModDown P1-P4); see the header of ks_oracle.c for the readings
it takes where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ks_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

u64p = ctypes.POINTER(ctypes.c_uint64)
i64p = ctypes.POINTER(ctypes.c_int64)
i8p = ctypes.POINTER(ctypes.c_int8)


def build(force: bool = False) -> str:
    """Compile ks_oracle.c with gcc (plain C, OpenMP over towers)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        ci = ctypes.c_int
        lib.orc_is_prime.argtypes = [ctypes.c_uint64]
        lib.orc_is_prime.restype = ci
        lib.orc_gen_primes.argtypes = [ci, ci, ci, u64p]
        lib.orc_gen_primes.restype = ci
        lib.orc_find_psi.argtypes = [ctypes.c_uint64, ci]
        lib.orc_find_psi.restype = ctypes.c_uint64
        for name in ("orc_ntt_naive", "orc_intt_naive"):
            getattr(lib, name).argtypes = [u64p, u64p, ci, ctypes.c_uint64, ctypes.c_uint64]
            getattr(lib, name).restype = None
        for name in ("orc_ntt", "orc_intt"):
            getattr(lib, name).argtypes = [u64p, ci, ctypes.c_uint64, ctypes.c_uint64]
            getattr(lib, name).restype = None
        lib.orc_negacyclic_mul.argtypes = [u64p, u64p, u64p, ci, ctypes.c_uint64]
        lib.orc_negacyclic_mul.restype = None
        lib.orc_bconv.argtypes = [u64p, ci, u64p, u64p, ci, u64p, ci]
        lib.orc_bconv.restype = None
        lib.orc_ctx_create.argtypes = [ci, ci, ci, ci, ci, u64p, u64p]
        lib.orc_ctx_create.restype = vp
        lib.orc_ctx_destroy.argtypes = [vp]
        lib.orc_ctx_destroy.restype = None
        lib.orc_ctx_primes.argtypes = [vp, u64p, u64p, u64p, u64p]
        lib.orc_ctx_primes.restype = None
        lib.orc_ctx_alpha.argtypes = [vp]
        lib.orc_ctx_alpha.restype = ci
        lib.orc_ctx_ndig.argtypes = [vp]
        lib.orc_ctx_ndig.restype = ci
        lib.orc_active_digits.argtypes = [vp, ci]
        lib.orc_active_digits.restype = ci
        lib.orc_modup.argtypes = [vp, ci, u64p, u64p]
        lib.orc_modup.restype = None
        lib.orc_apply_key.argtypes = [vp, ci, u64p, u64p, u64p, u64p]
        lib.orc_apply_key.restype = None
        lib.orc_moddown.argtypes = [vp, ci, u64p, u64p]
        lib.orc_moddown.restype = None
        lib.orc_keyswitch.argtypes = [vp, ci, u64p, u64p, u64p, u64p]
        lib.orc_keyswitch.restype = None
        lib.orc_automorph_eval.argtypes = [u64p, u64p, ci, ctypes.c_uint64]
        lib.orc_automorph_eval.restype = None
        lib.orc_keyswitch_hoisted.argtypes = [vp, ci, u64p, ci, u64p, u64p, u64p, u64p]
        lib.orc_keyswitch_hoisted.restype = None
        lib.orc_keygen_compressed.argtypes = [vp, i8p, i64p, ctypes.c_uint64, u64p]
        lib.orc_keygen_compressed.restype = None
        lib.orc_key_a_word.argtypes = [ctypes.c_uint64, ci, ci, ctypes.c_uint64, ci, ci, ctypes.c_uint64]
        lib.orc_key_a_word.restype = ctypes.c_uint64
        lib.orc_keygen.argtypes = [vp, i8p, i64p, ctypes.c_uint64, u64p]
        lib.orc_keygen.restype = None
        lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ci, u64p]
        lib.orc_splitmix64.restype = None
        lib.orc_sample_gauss.argtypes = [ctypes.c_uint64, ci, i64p]
        lib.orc_sample_gauss.restype = None
        lib.orc_set_threads.argtypes = [ci]
        lib.orc_set_threads.restype = None
        lib.orc_get_threads.argtypes = []
        lib.orc_get_threads.restype = ci
        _lib = lib
        return lib


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def _p(a: np.ndarray):
    if a.dtype == np.uint64:
        return a.ctypes.data_as(u64p)
    if a.dtype == np.int64:
        return a.ctypes.data_as(i64p)
    if a.dtype == np.int8:
        return a.ctypes.data_as(i8p)
    raise TypeError(a.dtype)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


# ---------------------------------------------------------------- scalars
def is_prime(n: int) -> bool:
    return bool(_load().orc_is_prime(int(n)))


def gen_primes(logN: int, bits: int, count: int) -> list[int]:
    out = np.zeros(count, dtype=np.uint64)
    if _load().orc_gen_primes(logN, bits, count, _p(out)) != 0:
        raise ValueError("not enough primes")
    return [int(x) for x in out]


def find_psi(q: int, logN: int) -> int:
    return int(_load().orc_find_psi(int(q), logN))


def automorph_eval(a, logN: int, g: int) -> np.ndarray:
    """X -> X^g on an evaluation-form tower (bit-reversed slot order)."""
    a = _u64(a)
    out = np.zeros_like(a)
    _load().orc_automorph_eval(_p(a), _p(out), logN, g)
    return out


# ---------------------------------------------------------------- NTT
def ntt_naive(a, logN: int, q: int, psi: int) -> np.ndarray:
    a = _u64(a)
    out = np.zeros_like(a)
    _load().orc_ntt_naive(_p(a), _p(out), logN, q, psi)
    return out


def intt_naive(a, logN: int, q: int, psi: int) -> np.ndarray:
    a = _u64(a)
    out = np.zeros_like(a)
    _load().orc_intt_naive(_p(a), _p(out), logN, q, psi)
    return out


def ntt(a, logN: int, q: int, psi: int) -> np.ndarray:
    a = _u64(a).copy()
    _load().orc_ntt(_p(a), logN, q, psi)
    return a


def intt(a, logN: int, q: int, psi: int) -> np.ndarray:
    a = _u64(a).copy()
    _load().orc_intt(_p(a), logN, q, psi)
    return a


def negacyclic_mul(a, b, logN: int, q: int) -> np.ndarray:
    a, b = _u64(a), _u64(b)
    out = np.zeros_like(a)
    _load().orc_negacyclic_mul(_p(a), _p(b), _p(out), logN, q)
    return out


def bconv(src_primes, x, dst_primes, logN: int) -> np.ndarray:
    """Fast base conversion of coefficient-form residues x [a][N]."""
    sp = _u64(src_primes)
    dp = _u64(dst_primes)
    x = _u64(x)
    out = np.zeros((len(dp), 1 << logN), dtype=np.uint64)
    _load().orc_bconv(_p(sp), len(sp), _p(x), _p(dp), len(dp), _p(out), logN)
    return out


def splitmix64(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    _load().orc_splitmix64(seed & (2**64 - 1), n, _p(out))
    return out


def sample_gauss(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.int64)
    _load().orc_sample_gauss(seed & (2**64 - 1), n, _p(out))
    return out


# ---------------------------------------------------------------- context
class Ctx:
    """Oracle parameter set: N = 2^logN, nq = L+1 Q primes, kp = K P primes."""

    def __init__(self, logN: int, nq: int, kp: int, dnum: int, bits: int = 54,
                 q=None, p=None):
        lib = _load()
        self.logN, self.N, self.nq, self.kp, self.dnum = logN, 1 << logN, nq, kp, dnum
        if q is not None:
            qa, pa = _u64(q), _u64(p)
            h = lib.orc_ctx_create(logN, nq, kp, dnum, bits, _p(qa), _p(pa))
        else:
            h = lib.orc_ctx_create(logN, nq, kp, dnum, bits, None, None)
        if not h:
            raise ValueError("oracle context rejected the parameters")
        self._h = h
        qa = np.zeros(nq, dtype=np.uint64)
        pa = np.zeros(kp, dtype=np.uint64)
        psq = np.zeros(nq, dtype=np.uint64)
        psp = np.zeros(kp, dtype=np.uint64)
        lib.orc_ctx_primes(h, _p(qa), _p(pa), _p(psq), _p(psp))
        self.q = [int(x) for x in qa]
        self.p = [int(x) for x in pa]
        self.psi_q = [int(x) for x in psq]
        self.psi_p = [int(x) for x in psp]
        self.alpha = int(lib.orc_ctx_alpha(h))
        self.ndig = int(lib.orc_ctx_ndig(h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_ctx_destroy(h)
            self._h = None

    def active_digits(self, nact: int) -> int:
        return int(_lib.orc_active_digits(self._h, nact))

    def towers(self, nact: int) -> list[int]:
        """Primes of the level basis D_l in compact order (Q then P)."""
        return self.q[:nact] + self.p

    def modup(self, nact: int, d) -> np.ndarray:
        d = _u64(d)
        nd = self.active_digits(nact)
        out = np.zeros((nd, nact + self.kp, self.N), dtype=np.uint64)
        _lib.orc_modup(self._h, nact, _p(d), _p(out))
        return out

    def apply_key(self, nact: int, D, evk):
        D, evk = _u64(D), _u64(evk)
        cb = np.zeros((nact + self.kp, self.N), dtype=np.uint64)
        ca = np.zeros_like(cb)
        _lib.orc_apply_key(self._h, nact, _p(D), _p(evk), _p(cb), _p(ca))
        return cb, ca

    def moddown(self, nact: int, cp) -> np.ndarray:
        cp = _u64(cp)
        out = np.zeros((nact, self.N), dtype=np.uint64)
        _lib.orc_moddown(self._h, nact, _p(cp), _p(out))
        return out

    def keyswitch(self, nact: int, d, evk):
        d, evk = _u64(d), _u64(evk)
        out0 = np.zeros((nact, self.N), dtype=np.uint64)
        out1 = np.zeros_like(out0)
        _lib.orc_keyswitch(self._h, nact, _p(d), _p(evk), _p(out0), _p(out1))
        return out0, out1

    def keyswitch_hoisted(self, nact: int, d, evks, gals):
        """Key switches of the rotations X -> X^g (g in gals) of d with one
        shared ModUp; evks[r] is the key of rotation r.  Returns (out0, out1),
        each [len(gals)][nact][N]."""
        d = _u64(d)
        ev = _u64(np.stack([np.asarray(e, dtype=np.uint64) for e in evks]))
        g = _u64(np.asarray(gals, dtype=np.uint64))
        out0 = np.zeros((len(gals), nact, self.N), dtype=np.uint64)
        out1 = np.zeros_like(out0)
        _lib.orc_keyswitch_hoisted(self._h, nact, _p(d), len(gals), _p(ev), _p(g), _p(out0), _p(out1))
        return out0, out1

    def keygen(self, s, sp, seed: int) -> np.ndarray:
        s = np.ascontiguousarray(s, dtype=np.int8)
        sp = np.ascontiguousarray(sp, dtype=np.int64)
        evk = np.zeros((self.ndig, 2, self.nq + self.kp, self.N), dtype=np.uint64)
        _lib.orc_keygen(self._h, _p(s), _p(sp), seed & (2**64 - 1), _p(evk))
        return evk

    def keygen_compressed(self, s, sp, seed: int) -> np.ndarray:
        """Full evaluation key of a compressed key (a_j regenerated from the
        seed, see orc_keygen_compressed); same layout as keygen."""
        s = np.ascontiguousarray(s, dtype=np.int8)
        sp = np.ascontiguousarray(sp, dtype=np.int64)
        evk = np.zeros((self.ndig, 2, self.nq + self.kp, self.N), dtype=np.uint64)
        _lib.orc_keygen_compressed(self._h, _p(s), _p(sp), seed & (2**64 - 1), _p(evk))
        return evk

    def key_a_word(self, seed: int, j: int, t: int, n: int) -> int:
        r = (self.q + self.p)[t]
        return int(_lib.orc_key_a_word(seed & (2**64 - 1), j, t, n, self.logN, self.nq + self.kp, r))

    def evk_bytes(self) -> int:
        return self.ndig * 2 * (self.nq + self.kp) * self.N * 8
