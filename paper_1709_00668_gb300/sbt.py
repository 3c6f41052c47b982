"""Python binding of libsambaten (the C ABI in include/sambaten.h).

Argument marshalling only: every step of the update runs in the library's CUDA
kernels.  The library is loaded from the package's `_build/` directory; if it
is missing the import fails loudly (there is no CPU fallback).  Build it with
`paper_1709_00668_gb300.build.build()`.

Device tensors are torch CUDA tensors passed by pointer; their work must be
ordered on the stream handed to the library (by default torch's current
stream).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsambaten.so")

SBT_MAX_RANK = 32
SBT_MAX_REPS = 64

SBT_OK = 0
SBT_E_INVALID = 1
SBT_E_SHAPE = 2
SBT_E_NOMEM = 3
SBT_E_CUDA = 4
SBT_E_NONFINITE = 5
SBT_E_RANGE = 6
SBT_E_TIMEOUT = 7
SBT_E_STATE = 8

SBT_F64 = 0
SBT_F32 = 1
SBT_BF16 = 2
SBT_PREC_F64 = 0
SBT_PREC_F32 = 1
SBT_PREC_BF16 = 2
SBT_PREC_FP8 = 3
PREC = {"f64": SBT_PREC_F64, "f32": SBT_PREC_F32, "bf16": SBT_PREC_BF16, "fp8": SBT_PREC_FP8}

SBT_FLAG_CHOL_REGULARIZED = 1
SBT_FLAG_ZERO_COLUMN = 2
SBT_FLAG_SAMPLE_LT_RANK = 4
SBT_FLAG_NO_REFINE = 8

EXPORTS = [
    "sbt_version", "sbt_last_error", "sbt_default_options", "sbt_init", "sbt_init_factors",
    "sbt_update", "sbt_factors", "sbt_fit", "sbt_recompute", "sbt_stats", "sbt_last_samples", "sbt_last_summary",
    "sbt_last_summary_factors", "sbt_destroy", "sbt_philox4x32_10", "sbt_sample", "sbt_mttkrp",
    "sbt_core_consistency",
    "sbt_profile_reset", "sbt_profile_read", "sbt_sample_noalloc",
    "sbt_device_bytes", "sbt_update_bytes", "sbt_reserve", "sbt_tile_table",
    "sbt_init_coo", "sbt_init_coo_factors", "sbt_update_coo",
    "sbt_server_default_options", "sbt_server_create", "sbt_server_open_stream", "sbt_server_submit",
    "sbt_server_wait", "sbt_server_stream_ctx", "sbt_server_close_stream", "sbt_server_stats",
    "sbt_server_stats_reset", "sbt_server_destroy",
    "sbt_nmode_init_factors", "sbt_nmode_update", "sbt_nmode_factors", "sbt_nmode_fit", "sbt_nmode_stats",
    "sbt_nmode_last_samples", "sbt_nmode_destroy",
]
SBT_NMODE_MAX = 8
SBT_SAMPLE_NOALLOC_MAX_N = 262144


class SbtTensor(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("on_device", ctypes.c_int32),
                ("I", ctypes.c_int64), ("J", ctypes.c_int64), ("K", ctypes.c_int64),
                ("data", ctypes.c_void_p)]


class SbtTensorN(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("on_device", ctypes.c_int32), ("N", ctypes.c_int32),
                ("dims", ctypes.c_int64 * SBT_NMODE_MAX), ("data", ctypes.c_void_p)]


class SbtOptions(ctypes.Structure):
    _fields_ = [("s_I", ctypes.c_int32), ("s_J", ctypes.c_int32), ("s_K", ctypes.c_int32),
                ("r", ctypes.c_int32), ("tol", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("max_iters_init", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("stream_id", ctypes.c_uint32), ("prec", ctypes.c_int32),
                ("lambda_mode", ctypes.c_int32), ("fixed_iters", ctypes.c_int32),
                ("K_capacity", ctypes.c_int64), ("max_batch", ctypes.c_int64),
                ("cuda_stream", ctypes.c_void_p), ("check_every", ctypes.c_int32),
                ("refine_sweeps", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("mode3_pass", ctypes.c_int32), ("als_groups", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("get_rank", ctypes.c_int32),
                ("get_rank_trials", ctypes.c_int32), ("get_rank_threshold", ctypes.c_double),
                ("fp64_tail", ctypes.c_int32), ("persistent_als", ctypes.c_int32)]


class SbtStats(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("r", ctypes.c_int32), ("R", ctypes.c_int32),
                ("n_I", ctypes.c_int32), ("n_J", ctypes.c_int32), ("n_K", ctypes.c_int32),
                ("flags", ctypes.c_int32),
                ("iters", ctypes.c_int32 * SBT_MAX_REPS),
                ("fit", ctypes.c_double * SBT_MAX_REPS),
                ("min_score", ctypes.c_double * SBT_MAX_REPS),
                ("perm", (ctypes.c_int32 * SBT_MAX_RANK) * SBT_MAX_REPS),
                ("rank", ctypes.c_int32 * SBT_MAX_REPS)]


class SbtProfile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("updates", ctypes.c_int64),
                ("mttkrp_launches", ctypes.c_int64), ("mttkrp_ms", ctypes.c_double),
                ("mttkrp_bytes", ctypes.c_double), ("mttkrp_passes", ctypes.c_int64),
                ("mttkrp_busy_ms", ctypes.c_double), ("mttkrp_launch_ms", ctypes.c_double)]


class SbtCoo(ctypes.Structure):
    _fields_ = [("I", ctypes.c_int64), ("J", ctypes.c_int64), ("K", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("ii", ctypes.c_void_p), ("jj", ctypes.c_void_p), ("kk", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("on_device", ctypes.c_int32)]


TILE_FIELDS = ("fp8", "R", "NP", "NC", "Kp_bucket", "nrep", "epi", "ctas_per_sm", "stages")


class SbtTileEntry(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in TILE_FIELDS]


class SbtServerOptions(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("mem_budget", ctypes.c_uint64), ("device", ctypes.c_int32),
                ("batch_als", ctypes.c_int32)]


class SbtRequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("stream", ctypes.c_int32), ("K", ctypes.c_int64),
                ("queue_ms", ctypes.c_double), ("service_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]


class SbtServingStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("in_flight", ctypes.c_int64), ("streams", ctypes.c_int64),
                ("slices", ctypes.c_int64), ("resident_bytes", ctypes.c_uint64),
                ("peak_resident_bytes", ctypes.c_uint64), ("mem_budget", ctypes.c_uint64),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("service_p50_ms", ctypes.c_double), ("service_p99_ms", ctypes.c_double),
                ("busy_fraction", ctypes.c_double), ("elapsed_s", ctypes.c_double),
                ("als_launches", ctypes.c_int64), ("als_sets", ctypes.c_int64)]


class SbtError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Load libsambaten.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsambaten.so not found at {LIB_PATH}: run "
                           "paper_1709_00668_gb300.build.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U32, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
    S = ctypes.c_int
    L.sbt_version.restype = ctypes.c_char_p
    L.sbt_last_error.restype = ctypes.c_char_p
    L.sbt_default_options.argtypes = [ctypes.POINTER(SbtOptions)]
    L.sbt_init.argtypes = [ctypes.POINTER(SbtTensor), I32, ctypes.POINTER(SbtOptions), ctypes.POINTER(P)]
    L.sbt_init_factors.argtypes = [ctypes.POINTER(SbtTensor), I32, P, P, P, P, ctypes.POINTER(SbtOptions),
                                   ctypes.POINTER(P)]
    L.sbt_update.argtypes = [P, ctypes.POINTER(SbtTensor)]
    L.sbt_factors.argtypes = [P, P, P, P, P, ctypes.POINTER(I64)]
    L.sbt_fit.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    L.sbt_recompute.argtypes = [P, I32, ctypes.c_double, ctypes.c_uint64, P, P, P, P, ctypes.POINTER(ctypes.c_double)]
    L.sbt_stats.argtypes = [P, ctypes.POINTER(SbtStats)]
    L.sbt_last_samples.argtypes = [P, I32, I32, P, I64, ctypes.POINTER(I64)]
    L.sbt_last_summary.argtypes = [P, I32, P, I64, P]
    L.sbt_last_summary_factors.argtypes = [P, I32, P, P, P, P]
    L.sbt_destroy.argtypes = [P]
    L.sbt_destroy.restype = None
    L.sbt_philox4x32_10.argtypes = [P, U32, U32, P, I64, P]
    L.sbt_sample.argtypes = [P, I64, I64, U64, U32, I32, I32, U32, P, P]
    L.sbt_mttkrp.argtypes = [I32, P, I64, I64, I64, I64, P, P, P, I32, I32, P, P]
    L.sbt_core_consistency.argtypes = [I32, P, I64, I64, I64, I64, P, P, P, P, I32,
                                       ctypes.POINTER(ctypes.c_double), P]
    L.sbt_sample_noalloc.argtypes = [P, I64, I64, U64, U32, I32, I32, U32, P, P]
    L.sbt_profile_reset.argtypes = [P, I32]
    L.sbt_profile_read.argtypes = [P, ctypes.POINTER(SbtProfile)]
    L.sbt_device_bytes.argtypes = [P, ctypes.POINTER(U64)]
    L.sbt_update_bytes.argtypes = [P, I64, ctypes.POINTER(U64)]
    L.sbt_reserve.argtypes = [P, I64, I64]
    L.sbt_tile_table.argtypes = [I32, P, I32, ctypes.POINTER(I32)]
    L.sbt_init_coo.argtypes = [ctypes.POINTER(SbtCoo), I32, ctypes.POINTER(SbtOptions), ctypes.POINTER(P)]
    L.sbt_init_coo_factors.argtypes = [ctypes.POINTER(SbtCoo), I32, P, P, P, P, ctypes.POINTER(SbtOptions),
                                       ctypes.POINTER(P)]
    L.sbt_update_coo.argtypes = [P, ctypes.POINTER(SbtCoo)]
    L.sbt_server_default_options.argtypes = [ctypes.POINTER(SbtServerOptions)]
    L.sbt_server_create.argtypes = [ctypes.POINTER(SbtServerOptions), ctypes.POINTER(P)]
    L.sbt_server_open_stream.argtypes = [P, ctypes.POINTER(SbtTensor), I32, ctypes.POINTER(SbtOptions),
                                         ctypes.POINTER(I32)]
    L.sbt_server_submit.argtypes = [P, I32, ctypes.POINTER(SbtTensor), ctypes.POINTER(U64)]
    L.sbt_server_wait.argtypes = [P, U64, I32, ctypes.POINTER(SbtRequestResult)]
    L.sbt_server_stream_ctx.argtypes = [P, I32, ctypes.POINTER(P)]
    L.sbt_server_close_stream.argtypes = [P, I32]
    L.sbt_server_stats.argtypes = [P, ctypes.POINTER(SbtServingStats)]
    L.sbt_server_stats_reset.argtypes = [P]
    L.sbt_server_destroy.argtypes = [P]
    L.sbt_server_destroy.restype = None
    L.sbt_nmode_init_factors.argtypes = [ctypes.POINTER(SbtTensorN), I32, P, P, ctypes.POINTER(SbtOptions),
                                         ctypes.POINTER(P)]
    L.sbt_nmode_update.argtypes = [P, ctypes.POINTER(SbtTensorN)]
    L.sbt_nmode_factors.argtypes = [P, P, P, ctypes.POINTER(I64)]
    L.sbt_nmode_fit.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    L.sbt_nmode_stats.argtypes = [P, ctypes.POINTER(SbtStats)]
    L.sbt_nmode_last_samples.argtypes = [P, I32, I32, P, I64, ctypes.POINTER(I64)]
    L.sbt_nmode_destroy.argtypes = [P]
    L.sbt_nmode_destroy.restype = None
    for name in EXPORTS:
        f = getattr(L, name)
        if name not in ("sbt_version", "sbt_last_error", "sbt_destroy", "sbt_nmode_destroy"):
            f.restype = S
    _lib = L
    return L


def _check(status: int, where: str):
    if status != SBT_OK:
        raise SbtError(status, where, lib().sbt_last_error().decode())


def version() -> str:
    return lib().sbt_version().decode()


def tile_table() -> list:
    """The MTTKRP tile table as a list of dicts (TILE_FIELDS)."""
    n = ctypes.c_int32()
    _check(lib().sbt_tile_table(0, None, 0, ctypes.byref(n)), "sbt_tile_table")
    arr = (SbtTileEntry * max(1, n.value))()
    _check(lib().sbt_tile_table(0, ctypes.cast(arr, ctypes.c_void_p), n.value, ctypes.byref(n)), "sbt_tile_table")
    return [{f: getattr(arr[q], f) for f in TILE_FIELDS} for q in range(n.value)]


def tile_table_merge(entries: list):
    arr = (SbtTileEntry * max(1, len(entries)))()
    for q, e in enumerate(entries):
        for f in TILE_FIELDS:
            setattr(arr[q], f, int(e[f]))
    n = ctypes.c_int32()
    _check(lib().sbt_tile_table(1, ctypes.cast(arr, ctypes.c_void_p), len(entries), ctypes.byref(n)),
           "sbt_tile_table")


def tile_table_clear():
    n = ctypes.c_int32()
    _check(lib().sbt_tile_table(2, None, 0, ctypes.byref(n)), "sbt_tile_table")


# ---------------------------------------------------------------------------
def sbt_default_options(**kw) -> SbtOptions:
    o = SbtOptions()
    _check(lib().sbt_default_options(ctypes.byref(o)), "sbt_default_options")
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = PREC[v]
        if k == "cuda_stream" and v is not None and not isinstance(v, int):
            v = int(v)
        setattr(o, k, v)
    return o


def _tensor_desc(X, keep: list) -> SbtTensor:
    """SbtTensor for a torch tensor (CUDA or CPU) or a numpy array, slice-major (K, I, J)."""
    import torch
    if isinstance(X, np.ndarray):
        X = torch.from_numpy(np.ascontiguousarray(X))
    if X.dim() != 3:
        raise ValueError("X must be (K, I, J)")
    if X.dtype == torch.float64:
        dt = SBT_F64
    elif X.dtype == torch.float32:
        dt = SBT_F32
    else:
        raise ValueError("X must be float32 or float64")
    X = X.contiguous()
    keep.append(X)
    K, I, J = X.shape
    return SbtTensor(dt, 1 if X.is_cuda else 0, I, J, K, ctypes.c_void_p(X.data_ptr()))


def _coo_desc(ii, jj, kk, val, shape, keep: list) -> SbtCoo:
    """SbtCoo for coordinate arrays (torch tensors on one device, or numpy)."""
    import torch

    def as_t(x, dt):
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(np.ascontiguousarray(x))
        return x.to(dt).contiguous()
    ii, jj, kk = (as_t(x, torch.int32) for x in (ii, jj, kk))
    val = as_t(val, torch.float32)
    n = int(val.numel())
    if not (ii.numel() == jj.numel() == kk.numel() == n):
        raise ValueError("coordinate and value arrays differ in length")
    devs = {t.device for t in (ii, jj, kk, val)}
    if len(devs) != 1:
        raise ValueError("COO arrays on different devices")
    keep.extend([ii, jj, kk, val])
    I, J, K = (int(x) for x in shape)
    ptr = (lambda t: ctypes.c_void_p(t.data_ptr()) if n else None)
    return SbtCoo(I, J, K, n, ptr(ii), ptr(jj), ptr(kk), ptr(val), 1 if val.is_cuda else 0)


def _current_stream():
    import torch
    if torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return None


class SamBaTen:
    """One tensor stream: resident store, factors and marginals on the GPU."""

    def __init__(self, X0, R: int, *, factors=None, **opts):
        if "cuda_stream" not in opts:
            opts["cuda_stream"] = _current_stream()
        self.opts = sbt_default_options(**opts)
        self.R = int(R)
        keep: list = []
        desc = _tensor_desc(X0, keep)
        self.I, self.J = int(desc.I), int(desc.J)
        h = ctypes.c_void_p()
        if factors is None:
            _check(lib().sbt_init(ctypes.byref(desc), self.R, ctypes.byref(self.opts), ctypes.byref(h)),
                   "sbt_init")
        else:
            lam, A, B, C = (np.ascontiguousarray(np.asarray(f, dtype=np.float64)) for f in factors)
            _check(lib().sbt_init_factors(ctypes.byref(desc), self.R, lam.ctypes.data, A.ctypes.data,
                                          B.ctypes.data, C.ctypes.data, ctypes.byref(self.opts),
                                          ctypes.byref(h)), "sbt_init_factors")
        self._h = h

    @classmethod
    def from_coo(cls, ii, jj, kk, val, shape, R: int, *, factors=None, **opts) -> "SamBaTen":
        """A stream whose initial tensor is given by its nonzeros (float32 values,
        unique coordinates, kk in [0, K)); CP-ALS init unless factors are given."""
        if "cuda_stream" not in opts:
            opts["cuda_stream"] = _current_stream()
        opts.setdefault("prec", "f32")
        obj = cls.__new__(cls)
        obj.opts = sbt_default_options(**opts)
        obj.R = int(R)
        keep: list = []
        desc = _coo_desc(ii, jj, kk, val, shape, keep)
        obj.I, obj.J = int(desc.I), int(desc.J)
        h = ctypes.c_void_p()
        if factors is None:
            _check(lib().sbt_init_coo(ctypes.byref(desc), obj.R, ctypes.byref(obj.opts), ctypes.byref(h)),
                   "sbt_init_coo")
        else:
            lam, A, B, C = (np.ascontiguousarray(np.asarray(f, dtype=np.float64)) for f in factors)
            _check(lib().sbt_init_coo_factors(ctypes.byref(desc), obj.R, lam.ctypes.data, A.ctypes.data,
                                              B.ctypes.data, C.ctypes.data, ctypes.byref(obj.opts),
                                              ctypes.byref(h)), "sbt_init_coo_factors")
        obj._h = h
        return obj

    def update_coo(self, ii, jj, kk, val, K_new: int):
        keep: list = []
        desc = _coo_desc(ii, jj, kk, val, (self.I, self.J, K_new), keep)
        _check(lib().sbt_update_coo(self._h, ctypes.byref(desc)), "sbt_update_coo")

    def update_coo_status(self, ii, jj, kk, val, K_new: int) -> int:
        keep: list = []
        desc = _coo_desc(ii, jj, kk, val, (self.I, self.J, K_new), keep)
        return int(lib().sbt_update_coo(self._h, ctypes.byref(desc)))

    @classmethod
    def _borrow(cls, h, R: int, I: int, J: int) -> "SamBaTen":
        """View of a context owned elsewhere (a server stream); close() does not free it."""
        obj = cls.__new__(cls)
        obj._h, obj.R, obj.I, obj.J, obj._owned = h, int(R), int(I), int(J), False
        return obj

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                lib().sbt_destroy(self._h)
            self._h = None

    def device_bytes(self) -> int:
        b = ctypes.c_uint64()
        _check(lib().sbt_device_bytes(self._h, ctypes.byref(b)), "sbt_device_bytes")
        return int(b.value)

    def update_bytes(self, K_new: int) -> int:
        b = ctypes.c_uint64()
        _check(lib().sbt_update_bytes(self._h, int(K_new), ctypes.byref(b)), "sbt_update_bytes")
        return int(b.value)

    def reserve(self, K_max: int, K_new_max: int):
        _check(lib().sbt_reserve(self._h, int(K_max), int(K_new_max)), "sbt_reserve")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, X_new):
        keep: list = []
        desc = _tensor_desc(X_new, keep)
        _check(lib().sbt_update(self._h, ctypes.byref(desc)), "sbt_update")

    def update_status(self, X_new) -> int:
        """sbt_update returning the raw status instead of raising."""
        keep: list = []
        desc = _tensor_desc(X_new, keep)
        return int(lib().sbt_update(self._h, ctypes.byref(desc)))

    @property
    def K(self) -> int:
        k = ctypes.c_int64()
        _check(lib().sbt_factors(self._h, None, None, None, None, ctypes.byref(k)), "sbt_factors")
        return int(k.value)

    def factors(self):
        K = self.K
        lam = np.empty(self.R)
        A = np.empty((self.I, self.R))
        B = np.empty((self.J, self.R))
        C = np.empty((K, self.R))
        k = ctypes.c_int64()
        _check(lib().sbt_factors(self._h, lam.ctypes.data, A.ctypes.data, B.ctypes.data, C.ctypes.data,
                                 ctypes.byref(k)), "sbt_factors")
        return lam, A, B, C

    def fit(self) -> float:
        f = ctypes.c_double()
        _check(lib().sbt_fit(self._h, ctypes.byref(f)), "sbt_fit")
        return float(f.value)

    def recompute(self, max_iters: int = 50, tol: float = 1e-6, seed: int = 0):
        """CP-ALS of the whole resident tensor from scratch (the comparator of
        Relative Fitness): (fit, lambda, A, B, C); the context is unchanged."""
        lam = np.empty(self.R)
        A = np.empty((self.I, self.R))
        B = np.empty((self.J, self.R))
        C = np.empty((self.K, self.R))
        f = ctypes.c_double()
        _check(lib().sbt_recompute(self._h, max_iters, tol, seed, lam.ctypes.data, A.ctypes.data, B.ctypes.data,
                                   C.ctypes.data, ctypes.byref(f)), "sbt_recompute")
        return float(f.value), lam, A, B, C

    def relative_fitness(self, max_iters: int = 50, tol: float = 1e-6, seed: int = 0) -> float:
        """Relative Fitness (Section 4.2): ||X - X_sbt|| / ||X - X_cp|| with X_cp
        the recomputed CP-ALS of the whole tensor; 1 = as good as recomputing."""
        f_cp = self.recompute(max_iters, tol, seed)[0]
        return (1.0 - self.fit()) / (1.0 - f_cp) if f_cp < 1.0 else float("inf")

    def stats(self) -> dict:
        st = SbtStats()
        _check(lib().sbt_stats(self._h, ctypes.byref(st)), "sbt_stats")
        r, R = st.r, st.R
        return {"K": st.K, "r": r, "R": R, "n_I": st.n_I, "n_J": st.n_J, "n_K": st.n_K,
                "flags": st.flags, "iters": list(st.iters[:r]), "fit": list(st.fit[:r]),
                "min_score": list(st.min_score[:r]),
                "perm": [list(st.perm[q][:R]) for q in range(r)], "rank": list(st.rank[:r])}

    def profile_reset(self, timing: bool = True, direct: bool = False):
        """timing: CUDA events around every MTTKRP launch; direct: the ALS
        kernels launched one by one instead of as graph chunks."""
        mode = 0 if not timing else (2 if direct else 1)
        _check(lib().sbt_profile_reset(self._h, mode), "sbt_profile_reset")

    def profile(self) -> dict:
        p = SbtProfile()
        _check(lib().sbt_profile_read(self._h, ctypes.byref(p)), "sbt_profile_read")
        return {"launches": p.launches, "updates": p.updates, "mttkrp_launches": p.mttkrp_launches,
                "mttkrp_ms": p.mttkrp_ms, "mttkrp_bytes": p.mttkrp_bytes, "mttkrp_passes": p.mttkrp_passes,
                "mttkrp_busy_ms": p.mttkrp_busy_ms, "mttkrp_launch_ms": p.mttkrp_launch_ms}

    def last_samples(self, rep: int, mode: int) -> np.ndarray:
        n = ctypes.c_int64()
        _check(lib().sbt_last_samples(self._h, rep, mode, None, 0, ctypes.byref(n)), "sbt_last_samples")
        out = np.empty(max(1, n.value), np.int32)
        _check(lib().sbt_last_samples(self._h, rep, mode, out.ctypes.data, n.value, ctypes.byref(n)),
               "sbt_last_samples")
        return out[:n.value].copy()

    def last_summary(self, rep: int) -> np.ndarray:
        dims = np.zeros(3, np.int64)
        _check(lib().sbt_last_summary(self._h, rep, None, 0, dims.ctypes.data), "sbt_last_summary")
        nI, nJ, Kp = (int(v) for v in dims)
        out = np.empty((Kp, nI, nJ))
        _check(lib().sbt_last_summary(self._h, rep, out.ctypes.data, out.size, dims.ctypes.data),
               "sbt_last_summary")
        return out

    def last_summary_factors(self, rep: int):
        """Summary factors of the last update after the shared-row normalisation."""
        dims = np.zeros(3, np.int64)
        _check(lib().sbt_last_summary(self._h, rep, None, 0, dims.ctypes.data), "sbt_last_summary")
        nI, nJ, Kp = (int(v) for v in dims)
        lam = np.empty(self.R)
        A = np.empty((nI, self.R))
        B = np.empty((nJ, self.R))
        C = np.empty((Kp, self.R))
        _check(lib().sbt_last_summary_factors(self._h, rep, lam.ctypes.data, A.ctypes.data, B.ctypes.data,
                                              C.ctypes.data), "sbt_last_summary_factors")
        return lam, A, B, C


def _tensor_n_desc(X, keep: list) -> SbtTensorN:
    """SbtTensorN for an order-N torch tensor or numpy array, time first (K, I_1, ..., I_{N-1})."""
    import torch
    if isinstance(X, np.ndarray):
        X = torch.from_numpy(np.ascontiguousarray(X))
    if not (3 <= X.dim() <= SBT_NMODE_MAX):
        raise ValueError("X must have 3..SBT_NMODE_MAX axes")
    if X.dtype == torch.float64:
        dt = SBT_F64
    elif X.dtype == torch.float32:
        dt = SBT_F32
    else:
        raise ValueError("X must be float32 or float64")
    X = X.contiguous()
    keep.append(X)
    dims = (ctypes.c_int64 * SBT_NMODE_MAX)(*([int(v) for v in X.shape] + [0] * (SBT_NMODE_MAX - X.dim())))
    return SbtTensorN(dt, 1 if X.is_cuda else 0, X.dim(), dims, ctypes.c_void_p(X.data_ptr()))


class SamBaTenN:
    """An order-N tensor stream (time first): the pre-existing decomposition
    lambda, U = [U_1, ..., U_{N-1}, C] is given; sbt_nmode_* underneath."""

    def __init__(self, X0, R: int, *, factors, **opts):
        if "cuda_stream" not in opts:
            opts["cuda_stream"] = _current_stream()
        self.opts = sbt_default_options(**opts)
        self.R = int(R)
        keep: list = []
        desc = _tensor_n_desc(X0, keep)
        self.N = int(desc.N)
        self.dims = [int(desc.dims[a]) for a in range(1, self.N)]
        lam, U = factors
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float64))
        Us = [np.ascontiguousarray(np.asarray(u, dtype=np.float64)) for u in U]
        ptrs = (ctypes.c_void_p * self.N)(*[u.ctypes.data for u in Us])
        h = ctypes.c_void_p()
        _check(lib().sbt_nmode_init_factors(ctypes.byref(desc), self.R, lam.ctypes.data, ptrs,
                                            ctypes.byref(self.opts), ctypes.byref(h)), "sbt_nmode_init_factors")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().sbt_nmode_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, X_new):
        keep: list = []
        desc = _tensor_n_desc(X_new, keep)
        _check(lib().sbt_nmode_update(self._h, ctypes.byref(desc)), "sbt_nmode_update")

    def factors(self):
        K = ctypes.c_int64()
        lib().sbt_nmode_factors(self._h, None, None, ctypes.byref(K))
        lam = np.empty(self.R)
        U = [np.empty((d, self.R)) for d in self.dims] + [np.empty((K.value, self.R))]
        ptrs = (ctypes.c_void_p * self.N)(*[u.ctypes.data for u in U])
        _check(lib().sbt_nmode_factors(self._h, lam.ctypes.data, ptrs, ctypes.byref(K)), "sbt_nmode_factors")
        return lam, U

    def fit(self) -> float:
        f = ctypes.c_double()
        _check(lib().sbt_nmode_fit(self._h, ctypes.byref(f)), "sbt_nmode_fit")
        return f.value

    def stats(self) -> dict:
        st = SbtStats()
        _check(lib().sbt_nmode_stats(self._h, ctypes.byref(st)), "sbt_nmode_stats")
        r, R = st.r, st.R
        return {"K": st.K, "r": r, "R": R, "n_I": st.n_I, "n_J": st.n_J, "n_K": st.n_K, "flags": st.flags,
                "iters": list(st.iters[:r]), "fit": list(st.fit[:r]), "min_score": list(st.min_score[:r]),
                "perm": [list(st.perm[q][:R]) for q in range(r)]}

    def last_samples(self, rep: int, mode: int) -> np.ndarray:
        n = ctypes.c_int64()
        _check(lib().sbt_nmode_last_samples(self._h, rep, mode, None, 0, ctypes.byref(n)), "sbt_nmode_last_samples")
        out = np.empty(max(1, n.value), np.int32)
        _check(lib().sbt_nmode_last_samples(self._h, rep, mode, out.ctypes.data, n.value, ctypes.byref(n)),
               "sbt_nmode_last_samples")
        return out[:n.value].copy()


# module-level names of the C ABI --------------------------------------------
def sbt_init(X0, R, **opts) -> SamBaTen:
    return SamBaTen(X0, R, **opts)


def sbt_init_factors(X0, R, lam, A, B, C, **opts) -> SamBaTen:
    return SamBaTen(X0, R, factors=(lam, A, B, C), **opts)


def sbt_update(ctx: SamBaTen, X_new):
    ctx.update(X_new)


def sbt_factors(ctx: SamBaTen):
    return ctx.factors()


def sbt_fit(ctx: SamBaTen) -> float:
    return ctx.fit()


def sbt_stats(ctx: SamBaTen) -> dict:
    return ctx.stats()


def sbt_destroy(ctx: SamBaTen):
    ctx.close()


def _stream_arg(stream):
    if stream is None:
        return _current_stream()
    return stream if isinstance(stream, int) else int(stream)


def sbt_philox4x32_10(ctr, key, stream=None):
    """Philox4x32-10 of each row of a (n, 4) int32/uint32 CUDA tensor; returns (n, 4) int32."""
    import torch
    ctr = ctr.contiguous()
    out = torch.empty_like(ctr)
    _check(lib().sbt_philox4x32_10(ctr.data_ptr(), int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF,
                                   out.data_ptr(), ctr.shape[0], _stream_arg(stream)), "sbt_philox4x32_10")
    return out


def sbt_sample(w, n, *, seed=0, stream_id=0, mode=0, rep=0, batch=0, stream=None):
    """Weighted draw of n indices (ascending) from a CUDA int64 tensor of weights."""
    import torch
    w = w.contiguous()
    out = torch.empty(max(1, int(n)), dtype=torch.int32, device=w.device)
    _check(lib().sbt_sample(w.data_ptr(), w.numel(), int(n), int(seed) & ((1 << 64) - 1),
                            int(stream_id) & 0xFFFFFFFF, int(mode), int(rep), int(batch) & 0xFFFFFFFF,
                            out.data_ptr(), _stream_arg(stream)), "sbt_sample")
    return out[:int(n)]


def sbt_sample_noalloc(w, n, *, seed=0, stream_id=0, mode=0, rep=0, batch=0, stream=None, out=None):
    """sbt_sample without any device allocation inside the call (scratch is a
    fixed array in the library, N <= SBT_SAMPLE_NOALLOC_MAX_N).  `out` may be a
    preallocated CUDA int32 tensor of at least n elements."""
    import torch
    w = w.contiguous()
    if out is None:
        out = torch.empty(max(1, int(n)), dtype=torch.int32, device=w.device)
    _check(lib().sbt_sample_noalloc(w.data_ptr(), w.numel(), int(n), int(seed) & ((1 << 64) - 1),
                                    int(stream_id) & 0xFFFFFFFF, int(mode), int(rep), int(batch) & 0xFFFFFFFF,
                                    out.data_ptr(), _stream_arg(stream)), "sbt_sample_noalloc")
    return out[:int(n)]


def sbt_mttkrp(X, A, B, C, mode, *, stream=None):
    """MTTKRP of a (K, I, ld) CUDA tensor (ld >= J, a multiple of 8; J = B.shape[0]).
    bfloat16 X takes float32 factors and returns float32 (tensor cores)."""
    import torch
    K, I, ld = X.shape
    J = B.shape[0]
    R = A.shape[1]
    dt = {torch.float64: SBT_F64, torch.float32: SBT_F32, torch.bfloat16: SBT_BF16}[X.dtype]
    n = (I, J, K)[mode]
    out = torch.empty(n, R, dtype=torch.float32 if dt == SBT_BF16 else X.dtype, device=X.device)
    A, B, C = A.contiguous(), B.contiguous(), C.contiguous()
    _check(lib().sbt_mttkrp(dt, X.data_ptr(), K, I, J, ld, A.data_ptr(), B.data_ptr(), C.data_ptr(), R,
                            int(mode), out.data_ptr(), _stream_arg(stream)), "sbt_mttkrp")
    return out


def sbt_core_consistency(X, lam, A, B, C, *, stream=None) -> float:
    """CorConDia of the CP model (lam, A, B, C) of a (K, I, ld) CUDA tensor
    (float64 or float32; J = B.shape[0]); the factors are float64 tensors on
    the same device."""
    import torch
    K, I, ldx = X.shape
    J = B.shape[0]
    R = A.shape[1]
    dt = {torch.float64: SBT_F64, torch.float32: SBT_F32}[X.dtype]
    lam, A, B, C = (t.to(device=X.device, dtype=torch.float64).contiguous() for t in (lam, A, B, C))
    cc = ctypes.c_double()
    _check(lib().sbt_core_consistency(dt, X.data_ptr(), K, I, J, ldx, lam.data_ptr(), A.data_ptr(), B.data_ptr(),
                                      C.data_ptr(), R, ctypes.byref(cc), _stream_arg(stream)),
           "sbt_core_consistency")
    return float(cc.value)


# ---------------------------------------------------------------------------
class Server:
    """Serving loop over many tensor streams (sbt_server_*).

    Batches are borrowed until their ticket is waited for: the binding keeps a
    reference to each submitted tensor until then."""

    def __init__(self, slots: int = 4, mem_budget: int = 0, device: int = -1, batch_als: int = 0):
        o = SbtServerOptions()
        _check(lib().sbt_server_default_options(ctypes.byref(o)), "sbt_server_default_options")
        o.slots, o.mem_budget, o.device = int(slots), int(mem_budget), int(device)
        o.batch_als = int(batch_als)
        h = ctypes.c_void_p()
        _check(lib().sbt_server_create(ctypes.byref(o), ctypes.byref(h)), "sbt_server_create")
        self._h = h
        self._keep = {}
        self._shape = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().sbt_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def open_stream(self, X0, R: int, **opts) -> int:
        o = sbt_default_options(**opts)
        keep: list = []
        desc = _tensor_desc(X0, keep)
        sid = ctypes.c_int32()
        _check(lib().sbt_server_open_stream(self._h, ctypes.byref(desc), int(R), ctypes.byref(o),
                                            ctypes.byref(sid)), "sbt_server_open_stream")
        self._shape[sid.value] = (int(R), int(desc.I), int(desc.J))
        return int(sid.value)

    def open_stream_status(self, X0, R: int, **opts):
        """(status, sid) without raising."""
        o = sbt_default_options(**opts)
        keep: list = []
        desc = _tensor_desc(X0, keep)
        sid = ctypes.c_int32()
        st = int(lib().sbt_server_open_stream(self._h, ctypes.byref(desc), int(R), ctypes.byref(o),
                                              ctypes.byref(sid)))
        if st == SBT_OK:
            self._shape[sid.value] = (int(R), int(desc.I), int(desc.J))
        return st, int(sid.value)

    def submit(self, sid: int, X_new) -> int:
        keep: list = []
        desc = _tensor_desc(X_new, keep)
        t = ctypes.c_uint64()
        _check(lib().sbt_server_submit(self._h, int(sid), ctypes.byref(desc), ctypes.byref(t)),
               "sbt_server_submit")
        self._keep[t.value] = keep
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        r = SbtRequestResult()
        _check(lib().sbt_server_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(r)), "sbt_server_wait")
        self._keep.pop(int(ticket), None)
        return {"status": r.status, "stream": r.stream, "K": r.K, "queue_ms": r.queue_ms,
                "service_ms": r.service_ms, "total_ms": r.total_ms}

    def stream(self, sid: int) -> SamBaTen:
        """The stream's context (factors, fit, stats) while it has no batch queued or in flight."""
        h = ctypes.c_void_p()
        _check(lib().sbt_server_stream_ctx(self._h, int(sid), ctypes.byref(h)), "sbt_server_stream_ctx")
        R, I, J = self._shape[int(sid)]
        return SamBaTen._borrow(h, R, I, J)

    def close_stream(self, sid: int):
        _check(lib().sbt_server_close_stream(self._h, int(sid)), "sbt_server_close_stream")
        self._shape.pop(int(sid), None)

    def stats(self) -> dict:
        st = SbtServingStats()
        _check(lib().sbt_server_stats(self._h, ctypes.byref(st)), "sbt_server_stats")
        return {f: getattr(st, f) for f, _ in SbtServingStats._fields_}

    def stats_reset(self):
        _check(lib().sbt_server_stats_reset(self._h), "sbt_server_stats_reset")
