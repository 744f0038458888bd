"""Python binding of libqis.so (the C ABI declared in include/qis.h).

Argument marshalling only: every step of the search runs in the library's CUDA kernels.
Importing this module never builds anything; ``load()`` raises if libqis.so is missing
(build it with ``paper_2010_00180_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqis.so")

QIS_FP64, QIS_SPLIT_BF16, QIS_PM1_FP8 = 0, 1, 2
PRECISIONS = {"fp64": QIS_FP64, "split_bf16": QIS_SPLIT_BF16, "pm1_fp8": QIS_PM1_FP8}
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "DEVICE_TIMEOUT", -5: "CAPACITY", -6: "STATE"}

# the entry points of include/qis.h
SYMBOLS = ["qis_create", "qis_destroy", "qis_last_error", "qis_create_instance", "qis_create_instances",
           "qis_clear_instances", "qis_topk_states_all",
           "qis_instance_info", "qis_init_states", "qis_reset", "qis_iterate", "qis_search_list",
           "qis_set_search_list", "qis_save", "qis_load", "qis_instance_n",
           "qis_get_tuning", "qis_set_tuning", "qis_autotune", "qis_evaluated_pairs", "qis_survivor_count",
           "qis_set_incremental_fields",
           "qis_topk_states", "qis_merge", "qis_energies", "qis_synchronize", "qis_kernel_launches",
           "qis_candidate_count", "qis_get_stream", "qis_profile_enable", "qis_profile_query",
           "qis_set_wait_limit",
           "qis_select_candidates_noalloc",
           "qis_mlp_create", "qis_mlp_destroy", "qis_mlp_last_error", "qis_mlp_num_params", "qis_mlp_get_params",
           "qis_mlp_set_params", "qis_mlp_features", "qis_mlp_add_example", "qis_mlp_clear_examples",
           "qis_mlp_forward", "qis_mlp_loss_grad", "qis_mlp_train", "qis_init_states_learned"]
KERNEL_CLASSES = ["pick", "fields", "bound", "scan", "merge", "search"]


class QISError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class MLPConfig(C.Structure):
    _fields_ = [("hidden", C.c_int), ("max_sites", C.c_int), ("batch", C.c_int), ("max_n", C.c_int),
                ("device", C.c_int), ("seed", C.c_uint64)]


class Tuning(C.Structure):
    _fields_ = [("scan_chunk_nc", C.c_int), ("scan_search_group", C.c_int), ("gemm_tile_searches", C.c_int),
                ("pair_scan", C.c_int)]


class Config(C.Structure):
    _fields_ = [("K", C.c_int), ("R", C.c_int), ("precision", C.c_int), ("max_n", C.c_int),
                ("max_instances", C.c_int), ("survivor_cap", C.c_int), ("device", C.c_int),
                ("seed", C.c_uint64), ("flips", C.c_int)]


FLIPS = {"single_pair": 0, "single": 1, "exchange": 2}


_lib = None


def load():
    """dlopen libqis.so (no GPU needed for loading) and declare the signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2010_00180_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    P, I, U64 = C.c_void_p, C.c_int, C.c_uint64
    sig = {
        "qis_create": (I, [C.POINTER(Config), C.POINTER(P)]),
        "qis_destroy": (None, [P]),
        "qis_last_error": (C.c_char_p, [P]),
        "qis_create_instance": (I, [P, I, P, P, C.POINTER(I)]),
        "qis_create_instances": (I, [P, I, P, P, P, P]),
        "qis_topk_states_all": (I, [P, I, P, P, P, P]),
        "qis_clear_instances": (I, [P]),
        "qis_instance_info": (I, [P, I, C.POINTER(I), C.POINTER(I), C.POINTER(I)]),
        "qis_init_states": (I, [P, I, P]),
        "qis_reset": (I, [P]),
        "qis_iterate": (I, [P, I, C.POINTER(I)]),
        "qis_search_list": (I, [P, I, I, P, P, P, P, C.POINTER(I)]),
        "qis_set_search_list": (I, [P, I, I, I, P, P, P, P, I]),
        "qis_save": (I, [P, C.c_char_p]),
        "qis_instance_n": (I, [P, I, C.POINTER(I)]),
        "qis_get_tuning": (I, [P, C.POINTER(Tuning)]),
        "qis_evaluated_pairs": (I, [P, C.POINTER(U64)]),
        "qis_survivor_count": (I, [P, C.POINTER(U64)]),
        "qis_set_tuning": (I, [P, C.POINTER(Tuning)]),
        "qis_autotune": (I, [P, I, C.POINTER(Tuning), C.POINTER(C.c_double)]),
        "qis_load": (I, [P, C.c_char_p]),
        "qis_topk_states": (I, [P, I, I, P, P, P, C.POINTER(I)]),
        "qis_merge": (I, [P]),
        "qis_energies": (I, [P, I, I, P, P]),
        "qis_synchronize": (I, [P]),
        "qis_kernel_launches": (I, [P, C.POINTER(U64)]),
        "qis_candidate_count": (I, [P, C.POINTER(U64), C.POINTER(U64)]),
        "qis_get_stream": (I, [P, C.POINTER(P)]),
        "qis_profile_enable": (I, [P, I]),
        "qis_profile_query": (I, [P, I, C.POINTER(C.c_double), C.POINTER(U64)]),
        "qis_select_candidates_noalloc": (I, [I, P, P, P, I, P, P, P, P]),
        "qis_mlp_create": (I, [C.POINTER(MLPConfig), C.POINTER(P)]),
        "qis_mlp_destroy": (None, [P]),
        "qis_mlp_last_error": (C.c_char_p, [P]),
        "qis_mlp_num_params": (I, [P, C.POINTER(I)]),
        "qis_mlp_get_params": (I, [P, P]),
        "qis_mlp_set_params": (I, [P, P]),
        "qis_mlp_features": (I, [P, I, P, P, P]),
        "qis_mlp_add_example": (I, [P, I, P, P, P]),
        "qis_mlp_clear_examples": (I, [P]),
        "qis_mlp_forward": (I, [P, I, P, P]),
        "qis_mlp_loss_grad": (I, [P, I, P, P, C.POINTER(C.c_double), P]),
        "qis_mlp_train": (I, [P, I, C.c_float, C.POINTER(C.c_double)]),
        "qis_init_states_learned": (I, [P, I, P]),
        "qis_set_incremental_fields": (I, [P, I]),
        "qis_set_wait_limit": (I, [P, U64, I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def words(n: int) -> int:
    return (n + 63) // 64


def select_candidates_noalloc(n: int, J_ptr: int, h_ptr: int, bits_ptr: int, k: int, E_ptr: int, c_ptr: int,
                              Ep_ptr: int = 0, stream: int = 0) -> None:
    """qis_select_candidates_noalloc: all pointers are device addresses owned by the caller;
    the library allocates nothing (its scratch is a static device array)."""
    lib = load()
    rc = lib.qis_select_candidates_noalloc(n, J_ptr, h_ptr, bits_ptr, k, E_ptr, c_ptr, Ep_ptr or None,
                                           stream or None)
    if rc != 0:
        raise QISError(rc, lib.qis_last_error(None).decode())


class Context:
    """One qis_ctx: instances, R searches per instance, kept lists of K+1 states."""

    def __init__(self, K: int, R: int, precision="split_bf16", max_n: int = 1024, max_instances: int = 1,
                 survivor_cap: int = 0, device: int = 0, seed: int = 0, flips="single_pair"):
        """flips: the candidate set -- "single_pair" (single and pair flips, the default),
        "single" (single flips only) or "exchange" (spin exchanges, magnetisation conserving)."""
        self.lib = load()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        fl = FLIPS[flips] if isinstance(flips, str) else int(flips)
        self.cfg = Config(K, R, prec, max_n, max_instances, survivor_cap, device, seed & 0xFFFFFFFFFFFFFFFF, fl)
        self.K, self.R = K, R
        self.h = C.c_void_p()
        rc = self.lib.qis_create(C.byref(self.cfg), C.byref(self.h))
        if rc != 0:
            raise QISError(rc, self.lib.qis_last_error(None).decode())
        self.n = {}

    # --------------------------------------------------------------- helpers
    def _check(self, rc):
        if rc != 0:
            raise QISError(rc, self.lib.qis_last_error(self.h).decode())

    def close(self):
        if self.h:
            self.lib.qis_destroy(self.h)
            self.h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------- API
    def create_instance(self, J, h) -> int:
        J = np.ascontiguousarray(J, dtype=np.float64)
        h = np.ascontiguousarray(h, dtype=np.float64)
        n = h.shape[0]
        assert J.shape == (n, n)
        iid = C.c_int(-1)
        self._check(self.lib.qis_create_instance(self.h, n, _ptr(J), _ptr(h), C.byref(iid)))
        self.n[iid.value] = n
        return iid.value

    def create_instances(self, pairs) -> list:
        """Add several instances [(J, h), ...] with one validation read-back (qis_create_instances)."""
        Js = [np.ascontiguousarray(J, dtype=np.float64) for J, _ in pairs]
        hs = [np.ascontiguousarray(h, dtype=np.float64) for _, h in pairs]
        cnt = len(Js)
        if cnt == 0:
            return []
        ns = np.array([h.shape[0] for h in hs], dtype=np.int32)
        for J, n in zip(Js, ns):
            assert J.shape == (n, n)
        Jp = (C.c_void_p * cnt)(*[J.ctypes.data for J in Js])
        hp = (C.c_void_p * cnt)(*[h.ctypes.data for h in hs])
        ids = np.zeros(cnt, dtype=np.int32)
        self._check(self.lib.qis_create_instances(self.h, cnt, _ptr(ns), Jp, hp, _ptr(ids)))
        for iid, n in zip(ids, ns):
            self.n[int(iid)] = int(n)
        return [int(i) for i in ids]

    def clear_instances(self):
        self._check(self.lib.qis_clear_instances(self.h))
        self.n = {}

    def instance_info(self, iid: int):
        q, d, r = C.c_int(), C.c_int(), C.c_int()
        self._check(self.lib.qis_instance_info(self.h, iid, C.byref(q), C.byref(d), C.byref(r)))
        return q.value, d.value, bool(r.value)

    def init_states(self, iid: int, bits=None):
        if bits is not None:
            bits = np.ascontiguousarray(bits, dtype=np.uint64)
            assert bits.shape == (self.R, words(self.n[iid]))
        self._check(self.lib.qis_init_states(self.h, iid, _ptr(bits)))

    def reset(self):
        self._check(self.lib.qis_reset(self.h))

    def iterate(self, n_iters: int, count_active: bool = False):
        na = C.c_int(-1)
        self._check(self.lib.qis_iterate(self.h, n_iters, C.byref(na) if count_active else None))
        return na.value if count_active else None

    def search_list(self, iid: int, r: int) -> dict:
        n, K1 = self.n[iid], self.K + 1
        bits = np.zeros((K1, words(n)), np.uint64)
        E = np.zeros(K1)
        used = np.zeros(K1, np.uint8)
        stamp = np.zeros(K1, np.uint64)
        cnt = C.c_int()
        self._check(self.lib.qis_search_list(self.h, iid, r, _ptr(bits), _ptr(E), _ptr(used), _ptr(stamp),
                                             C.byref(cnt)))
        c = cnt.value
        return dict(bits=bits[:c], E=E[:c], used=used[:c], stamp=stamp[:c], count=c)

    def set_search_list(self, iid: int, r: int, bits, E, used=None, stamp=None, t: int = 0):
        """Replace the kept list of search r (entries in list order), e.g. with a list computed
        by another process, before qis_merge / topk_states."""
        n = self.n[iid]
        bits = np.ascontiguousarray(bits, np.uint64).reshape(-1, words(n))
        E = np.ascontiguousarray(E, np.float64)
        cnt = bits.shape[0]
        if E.shape != (cnt,):
            raise ValueError("E must have one energy per state")
        u = None if used is None else np.ascontiguousarray(used, np.uint8)
        st = None if stamp is None else np.ascontiguousarray(stamp, np.uint64)
        self._check(self.lib.qis_set_search_list(self.h, iid, r, cnt, _ptr(bits), _ptr(E),
                                                 _ptr(u) if u is not None else None,
                                                 _ptr(st) if st is not None else None, int(t)))

    def evaluated_pairs(self) -> int:
        """Pair terms the scan evaluated one by one (the rest were decided by the row bound)."""
        v = C.c_uint64()
        self._check(self.lib.qis_evaluated_pairs(self.h, C.byref(v)))
        return v.value

    def survivor_count(self) -> int:
        """Candidates that passed the FP32 filters and were evaluated exactly by the merge."""
        v = C.c_uint64()
        self._check(self.lib.qis_survivor_count(self.h, C.byref(v)))
        return v.value

    def tuning(self) -> dict:
        t = Tuning()
        self._check(self.lib.qis_get_tuning(self.h, C.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def set_tuning(self, scan_chunk_nc: int = 8, scan_search_group: int = 0, gemm_tile_searches: int = 0,
                   pair_scan: int = 0):
        """pair_scan: 1 output-sensitive (in the fused search kernel where it can run), 3 output-sensitive
        as its own kernel in every iteration, 2 dense register tiles, 0 automatic."""
        t = Tuning(scan_chunk_nc, scan_search_group, gemm_tile_searches, pair_scan)
        self._check(self.lib.qis_set_tuning(self.h, C.byref(t)))

    def set_incremental_fields(self, on: bool):
        """Local fields by update from the generating parent's (qis_set_incremental_fields)."""
        self._check(self.lib.qis_set_incremental_fields(self.h, 1 if on else 0))

    def autotune(self, iters: int = 8) -> dict:
        """Pick the fastest launch shapes for the current instances (resets every search)."""
        t, ms = Tuning(), C.c_double()
        self._check(self.lib.qis_autotune(self.h, iters, C.byref(t), C.byref(ms)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_} | {"ms": ms.value, "iters": iters}

    def save(self, path: str):
        self._check(self.lib.qis_save(self.h, os.fsencode(path)))

    def load(self, path: str):
        """Restore a qis_save checkpoint into this (empty) context."""
        self._check(self.lib.qis_load(self.h, os.fsencode(path)))
        self.n = {}
        n = C.c_int()
        while self.lib.qis_instance_n(self.h, len(self.n), C.byref(n)) == 0:
            self.n[len(self.n)] = n.value

    def topk_states(self, iid: int, k: int) -> dict:
        n = self.n[iid]
        bits = np.zeros((max(k, 1), words(n)), np.uint64)
        E = np.zeros(max(k, 1))
        src = np.zeros(max(k, 1), np.uint64)
        cnt = C.c_int()
        self._check(self.lib.qis_topk_states(self.h, iid, k, _ptr(bits), _ptr(E), _ptr(src), C.byref(cnt)))
        c = cnt.value
        return dict(bits=bits[:c], E=E[:c], src=src[:c], count=c)

    def topk_states_all(self, k: int) -> list:
        """topk_states of every instance at once (qis_topk_states_all): one dict per instance."""
        ni = len(self.n)
        wm = words(self.cfg.max_n)
        bits = np.zeros((max(ni * k, 1), wm), np.uint64)
        E = np.zeros(max(ni * k, 1))
        src = np.zeros(max(ni * k, 1), np.uint64)
        cnt = np.zeros(max(ni, 1), np.int32)
        self._check(self.lib.qis_topk_states_all(self.h, k, _ptr(bits), _ptr(E), _ptr(src), _ptr(cnt)))
        out = []
        for i in range(ni):
            c = int(cnt[i])
            w = words(self.n[i])
            out.append(dict(bits=bits[i * k:i * k + c, :w].copy(), E=E[i * k:i * k + c].copy(),
                            src=src[i * k:i * k + c].copy(), count=c))
        return out

    def merge(self):
        self._check(self.lib.qis_merge(self.h))

    def energies(self, iid: int, bits) -> np.ndarray:
        bits = np.ascontiguousarray(np.atleast_2d(bits), dtype=np.uint64)
        E = np.zeros(bits.shape[0])
        self._check(self.lib.qis_energies(self.h, iid, bits.shape[0], _ptr(bits), _ptr(E)))
        return E

    def synchronize(self):
        self._check(self.lib.qis_synchronize(self.h))

    def kernel_launches(self) -> int:
        v = C.c_uint64()
        self._check(self.lib.qis_kernel_launches(self.h, C.byref(v)))
        return v.value

    def candidate_count(self):
        p, s = C.c_uint64(), C.c_uint64()
        self._check(self.lib.qis_candidate_count(self.h, C.byref(p), C.byref(s)))
        return p.value, s.value

    def stream_handle(self) -> int:
        v = C.c_void_p()
        self._check(self.lib.qis_get_stream(self.h, C.byref(v)))
        return v.value or 0

    def profile(self, on: bool):
        self._check(self.lib.qis_profile_enable(self.h, 1 if on else 0))

    def profile_query(self, kernel_class) -> tuple:
        k = KERNEL_CLASSES.index(kernel_class) if isinstance(kernel_class, str) else int(kernel_class)
        ms, n = C.c_double(), C.c_uint64()
        self._check(self.lib.qis_profile_query(self.h, k, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def set_wait_limit(self, limit_ns: int, probe: bool = False):
        """Bound of the kernels' device-side waits (qis_set_wait_limit); probe makes the field
        GEMM wait on a barrier nothing completes, so the timeout path runs (tests)."""
        self._check(self.lib.qis_set_wait_limit(self.h, int(limit_ns), int(probe)))

    def init_states_learned(self, iid: int, mlp: "MLP"):
        """Initial states of instance iid proposed by the network (qis_init_states_learned)."""
        self._check(self.lib.qis_init_states_learned(self.h, iid, mlp.h))


class MLP:
    """The warm-start network (qis_mlp_*): features -> 3 hidden ReLU layers -> logit of s_i = +1."""

    N_FEATURES = 8

    def __init__(self, hidden=256, max_sites=1 << 20, batch=4096, max_n=1024, device=0, seed=0):
        self.lib = load()
        self.cfg = MLPConfig(hidden, max_sites, batch, max_n, device, seed & 0xFFFFFFFFFFFFFFFF)
        self.h = C.c_void_p()
        rc = self.lib.qis_mlp_create(C.byref(self.cfg), C.byref(self.h))
        if rc != 0:
            raise QISError(rc, self.lib.qis_last_error(None).decode())
        cnt = C.c_int()
        self._check(self.lib.qis_mlp_num_params(self.h, C.byref(cnt)))
        self.n_params = cnt.value

    def _check(self, rc):
        if rc != 0:
            raise QISError(rc, self.lib.qis_mlp_last_error(self.h).decode())

    def close(self):
        if self.h:
            self.lib.qis_mlp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        self._check(self.lib.qis_mlp_get_params(self.h, _ptr(out)))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        assert flat.size == self.n_params
        self._check(self.lib.qis_mlp_set_params(self.h, _ptr(flat)))

    def features(self, J, h) -> np.ndarray:
        J = np.ascontiguousarray(J, np.float64)
        h = np.ascontiguousarray(h, np.float64)
        n = h.shape[0]
        out = np.zeros((n, self.N_FEATURES), np.float32)
        self._check(self.lib.qis_mlp_features(self.h, n, _ptr(J), _ptr(h), _ptr(out)))
        return out

    def add_example(self, J, h, bits):
        J = np.ascontiguousarray(J, np.float64)
        h = np.ascontiguousarray(h, np.float64)
        bits = np.ascontiguousarray(bits, np.uint64).reshape(-1)
        self._check(self.lib.qis_mlp_add_example(self.h, h.shape[0], _ptr(J), _ptr(h), _ptr(bits)))

    def clear_examples(self):
        self._check(self.lib.qis_mlp_clear_examples(self.h))

    def forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float32)
        z = np.zeros(X.shape[0], np.float32)
        self._check(self.lib.qis_mlp_forward(self.h, X.shape[0], _ptr(X), _ptr(z)))
        return z

    def loss_grad(self, X, y):
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        g = np.zeros(self.n_params, np.float32)
        L = C.c_double()
        self._check(self.lib.qis_mlp_loss_grad(self.h, X.shape[0], _ptr(X), _ptr(y), C.byref(L), _ptr(g)))
        return L.value, g

    def train(self, epochs: int, lr: float = 1e-3) -> float:
        L = C.c_double()
        self._check(self.lib.qis_mlp_train(self.h, epochs, lr, C.byref(L)))
        return L.value
