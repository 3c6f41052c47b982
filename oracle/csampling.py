"""ctypes binding of oracle/sampling.c (the oracle's integer sampling primitives).

Test infrastructure only: the product path never imports anything under
`oracle/`.  The shared object is built by `build()` (gcc, no GPU needed) into
`oracle/_build/liboracle_sampling.so`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sampling.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle_sampling.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile sampling.c with gcc into a shared object; returns its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        L.orc_philox_batch.argtypes = [P, P, P, ctypes.c_int64]
        L.orc_log2_batch.argtypes = [P, P, ctypes.c_int64]
        L.orc_es_key_batch.argtypes = [P, P, P, P, ctypes.c_int64]
        L.orc_sample_mode.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                      ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, P]
        L.orc_sample_mode.restype = ctypes.c_int64
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 of each row of `ctr` (n x 4 uint32) under key (2 x uint32)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctr)
    lib().orc_philox_batch(_ptr(ctr), _ptr(k), _ptr(out), ctr.shape[0])
    return out


def log2_q32(t: np.ndarray) -> np.ndarray:
    """Q.32 fixed-point log2 of integers 1 <= t < 2^33."""
    t = np.ascontiguousarray(t, dtype=np.uint64).reshape(-1)
    out = np.empty_like(t)
    lib().orc_log2_batch(_ptr(t), _ptr(out), t.shape[0])
    return out


def es_keys(v: np.ndarray, w: np.ndarray) -> list[int]:
    """Exponential keys floor(L 2^64 / w) as Python ints."""
    v = np.ascontiguousarray(v, dtype=np.uint32).reshape(-1)
    w = np.ascontiguousarray(w, dtype=np.uint64).reshape(-1)
    hi = np.empty(v.shape, np.uint64)
    lo = np.empty(v.shape, np.uint64)
    lib().orc_es_key_batch(_ptr(v), _ptr(w), _ptr(hi), _ptr(lo), v.shape[0])
    return [(int(h) << 64) | int(l) for h, l in zip(hi, lo)]


def sample_mode(w: np.ndarray, n: int, seed: int, stream_id: int, mode: int, rep: int,
                batch: int) -> np.ndarray:
    """n indices drawn without replacement with probability proportional to w."""
    w = np.ascontiguousarray(w, dtype=np.uint64).reshape(-1)
    out = np.empty(max(int(n), 1), np.int32)
    got = lib().orc_sample_mode(_ptr(w), w.shape[0], int(n), int(seed) & ((1 << 64) - 1),
                                int(stream_id) & 0xFFFFFFFF, int(mode), int(rep),
                                int(batch) & 0xFFFFFFFF, _ptr(out))
    if got < 0:
        raise ValueError("sample size exceeds the number of positive weights")
    return out[:n].copy()
