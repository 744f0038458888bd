"""ctypes wrapper around the C oracle (qis_oracle.c) -- TEST INFRASTRUCTURE ONLY.

The oracle is the plain FP64 CPU transcription of the QI search (Algorithms 1-4 of
Ueda, Otsuka and Yunoki, arXiv 2010.00180). Only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import this module; the library never does.

Arrays: J is (n, n) float64 C-contiguous, symmetric with zero diagonal; h is (n,);
states are (count, W) uint64 with W = ceil(n / 64), bit i of the state = sigma_i.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qis_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

EMPTY_STAMP = np.uint64(0xFFFFFFFFFFFFFFFF)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fused multiply-add) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.orc_energy.restype = C.c_double
            lib.orc_energy.argtypes = [C.c_int, P, P, P]
            lib.orc_fields.restype = None
            lib.orc_fields.argtypes = [C.c_int, P, P, P, P]
            lib.orc_candidates.restype = None
            lib.orc_candidates.argtypes = [C.c_int, P, P, P, P]
            lib.orc_candidates_flips.restype = None
            lib.orc_candidates_flips.argtypes = [C.c_int, P, P, P, C.c_int, P]
            lib.orc_pair_rank.restype = C.c_int64
            lib.orc_pair_rank.argtypes = [C.c_int, C.c_int, C.c_int]
            lib.orc_qi_search.restype = C.c_int
            lib.orc_qi_search.argtypes = [C.c_int, P, P, C.c_int, C.c_int, P, P, P, P, P, P, P]
            lib.orc_qi_search_flips.restype = C.c_int
            lib.orc_qi_search_flips.argtypes = [C.c_int, P, P, C.c_int, C.c_int, C.c_int, P, P, P, P, P, P, P]
            lib.orc_qi_multi_search.restype = C.c_int
            lib.orc_qi_multi_search.argtypes = [C.c_int, P, P, C.c_int, C.c_int, C.c_int, P,
                                                P, P, P, P, P, P, P, P, P, P]
            lib.orc_qi_multi_search_flips.restype = C.c_int
            lib.orc_qi_multi_search_flips.argtypes = [C.c_int, P, P, C.c_int, C.c_int, C.c_int, C.c_int, P,
                                                      P, P, P, P, P, P, P, P, P, P]
            lib.orc_brute_force.restype = C.c_int
            lib.orc_brute_force.argtypes = [C.c_int, P, P, C.c_int, P, P]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _prep(J, h):
    J = np.ascontiguousarray(J, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    n = h.shape[0]
    assert J.shape == (n, n)
    return J, h, n


def words(n: int) -> int:
    return (n + 63) // 64


def energy(J, h, bits) -> float:
    """H0 of one packed state (Eq. (1))."""
    J, h, n = _prep(J, h)
    b = np.ascontiguousarray(bits, dtype=np.uint64).reshape(-1)
    assert b.size == words(n)
    return _load().orc_energy(n, _p(J), _p(h), _p(b))


def energies(J, h, states) -> np.ndarray:
    states = np.atleast_2d(np.asarray(states, dtype=np.uint64))
    return np.array([energy(J, h, s) for s in states])


def fields(J, h, bits) -> np.ndarray:
    J, h, n = _prep(J, h)
    b = np.ascontiguousarray(bits, dtype=np.uint64).reshape(-1)
    f = np.empty(n)
    _load().orc_fields(n, _p(J), _p(h), _p(b), _p(f))
    return f


FLIPS = {"singles+pairs": 0, "singles": 1, "exchange": 2}


def candidates(J, h, bits, flips: int = 0) -> np.ndarray:
    """E' of every single and pair flip of one state, in candidate order (n(n+1)/2 values);
    candidates outside the flip set (1: singles only, 2: exchanges only) are +inf."""
    J, h, n = _prep(J, h)
    b = np.ascontiguousarray(bits, dtype=np.uint64).reshape(-1)
    out = np.empty(n * (n + 1) // 2)
    _load().orc_candidates_flips(n, _p(J), _p(h), _p(b), int(flips), _p(out))
    return out


def pair_rank(n: int, i: int, j: int) -> int:
    return _load().orc_pair_rank(n, i, j)


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise OracleError({-1: "invalid argument", -2: "out of memory",
                           -3: "placeholder would become a parent"}.get(rc, str(rc)))


def qi_search(J, h, K: int, I: int, psi0, flips: int = 0) -> dict:
    """Algorithm 3 from one initial state; returns the K+1-slot list in energy order.
    flips: 0 single and pair flips (Eq. (H1)), 1 single flips only, 2 spin exchanges only."""
    J, h, n = _prep(J, h)
    W, K1 = words(n), K + 1
    psi0 = np.ascontiguousarray(psi0, dtype=np.uint64).reshape(-1)
    assert psi0.size == W
    bits = np.zeros((K1, W), np.uint64)
    E = np.zeros(K1)
    used = np.zeros(K1, np.uint8)
    stamp = np.zeros(K1, np.uint64)
    cnt = C.c_int(0)
    prod = C.c_int(0)
    _check(_load().orc_qi_search_flips(n, _p(J), _p(h), K, I, int(flips), _p(psi0), _p(bits), _p(E),
                                       _p(used), _p(stamp), C.byref(cnt), C.byref(prod)))
    return dict(bits=bits, E=E, used=used, stamp=stamp, count=cnt.value, productive=prod.value)


def qi_multi_search(J, h, K: int, I: int, phi, per_search: bool = False, flips: int = 0) -> dict:
    """Algorithm 4 with the L initial states ``phi`` (L, W); returns the merged list."""
    J, h, n = _prep(J, h)
    W, K1 = words(n), K + 1
    phi = np.ascontiguousarray(np.atleast_2d(phi), dtype=np.uint64)
    L = phi.shape[0]
    assert phi.shape[1] == W
    bits = np.zeros((K1, W), np.uint64)
    E = np.zeros(K1)
    used = np.zeros(K1, np.uint8)
    src = np.zeros(K1, np.uint64)
    cnt = C.c_int(0)
    if per_search:
        ab = np.zeros((L, K1, W), np.uint64)
        aE = np.zeros((L, K1))
        au = np.zeros((L, K1), np.uint8)
        ast = np.zeros((L, K1), np.uint64)
        ac = np.zeros(L, np.int32)
    else:
        ab = aE = au = ast = ac = None
    _check(_load().orc_qi_multi_search_flips(n, _p(J), _p(h), K, I, int(flips), L, _p(phi), _p(bits), _p(E),
                                             _p(used), _p(src), C.byref(cnt), _p(ab), _p(aE), _p(au), _p(ast),
                                             _p(ac)))
    out = dict(bits=bits, E=E, used=used, src=src, count=cnt.value)
    if per_search:
        out["searches"] = [dict(bits=ab[r], E=aE[r], used=au[r], stamp=ast[r], count=int(ac[r]))
                           for r in range(L)]
    return out


def brute_force(J, h, k: int):
    """The k lowest states of all 2^n (n <= 24) by (E, psi): (psi uint64 array, E array)."""
    J, h, n = _prep(J, h)
    psi = np.zeros(k, np.uint64)
    E = np.zeros(k)
    _check(_load().orc_brute_force(n, _p(J), _p(h), k, _p(psi), _p(E)))
    return psi, E
