"""The oracle's batch update with its repetitions in parallel processes.

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`): the benchmark's CPU
baseline and reference arm time the FP64 oracle with this, and the CPU tests
pin it against the serial `sambaten.update`.

Algorithm 1's repetitions are independent (every one anchors on the
pre-update factors, Section 3.1), so steps 3-9 of each run as one task in a
worker process (`sambaten.update_rep`, unchanged), and steps 10-13 run in the
caller (`sambaten.commit`).  The stored slices live in one shared-memory
block that the workers map read-only, so no task copies the tensor.  Workers
are started with the `spawn` method (never forked from a process that may
hold a CUDA context) and each limits its BLAS threads, so that
workers x threads = the cores used.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

from . import sambaten as O

_W: dict = {}
_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def _attach(name: str, shape, dtype: str):
    shm = shared_memory.SharedMemory(name=name)
    _W["shm"] = shm
    _W["X"] = np.ndarray(shape, dtype=np.dtype(dtype), buffer=shm.buf)


def _rep_task(args):
    K_all, K_new, factors, marg, S, batch, opts, sizes, rho = args
    A, B, C, lam = factors
    xa, xb, xc = marg
    X_all = _W["X"][:K_all]
    st = O.State(X=X_all[:K_all - K_new], A=A, B=B, C=C, lam=lam, S=S, xa=xa, xb=xb, xc=xc,
                 batch=batch, opts=opts)
    t = O.update_rep(st, X_all, sizes, K_new, rho)
    return rho, t


def _marg_task(args):
    k0, k1, S = args
    xa, xb, xc = O.marginals(_W["X"][k0:k1], S)
    return k0, xa, xb, xc


def _fit_task(args):
    k0, k1, lam, A, B, C = args
    # sambaten.full_fit's sums over slices k0..k1-1
    num = 0.0
    den = 0.0
    X = _W["X"]
    for k in range(k0, k1):
        Xk = X[k].astype(np.float64)
        Xh = (A * (lam * C[k])) @ B.T
        D = Xk - Xh
        num += float(np.sum(D * D))
        den += float(np.sum(Xk * Xk))
    return k0, num, den


class PoolOracle:
    """Holds a (K_total, I, J) store in shared memory and runs the oracle's
    updates on it with `workers` processes of `threads` BLAS threads each."""

    def __init__(self, X_store, workers: int, threads: int = 1, *, shape=None, dtype=None):
        """X_store: the (K_total, I, J) slices (copied into shared memory), or
        None with `shape` and `dtype`, the slices then written into self.X
        before the first update."""
        if X_store is not None:
            X_store = np.ascontiguousarray(X_store)
            shape, dtype = X_store.shape, X_store.dtype
        self.shape = tuple(int(x) for x in shape)
        self.dtype = np.dtype(dtype)
        nbytes = int(np.prod(self.shape)) * self.dtype.itemsize
        self.shm = shared_memory.SharedMemory(create=True, size=max(1, nbytes))
        self.X = np.ndarray(self.shape, dtype=self.dtype, buffer=self.shm.buf)
        if X_store is not None:
            self.X[...] = X_store
        self.workers = max(1, int(workers))
        self.threads = max(1, int(threads))
        saved = {v: os.environ.get(v) for v in _THREAD_VARS}
        for v in _THREAD_VARS:
            os.environ[v] = str(self.threads)
        try:
            ctx = mp.get_context("spawn")
            self.pool = ctx.Pool(self.workers, initializer=_attach,
                                 initargs=(self.shm.name, self.shape, self.dtype.str))
        finally:
            for v, old in saved.items():
                if old is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old

    @property
    def cores(self) -> int:
        return self.workers * self.threads

    def _chunks(self, K: int):
        step = max(1, -(-K // (4 * self.workers)))
        return [(k0, min(K, k0 + step)) for k0 in range(0, K, step)]

    def state(self, K: int, lam, A, B, C, opts: O.Options, *, K_shift: int | None = None,
              batch: int = 0) -> O.State:
        """State of the first K stored slices with the given decomposition.
        The marginals of Eq. 1 are recomputed from the slices, chunks of
        slices in the workers (exact integer sums, so the chunking changes
        nothing); the fixed-point shift comes from the first K_shift slices
        (the initial tensor; default all K)."""
        X0 = self.X[:K]
        S = O.marginal_shift(self.X[:K if K_shift is None else K_shift])
        xa = np.zeros(self.shape[1], np.uint64)
        xb = np.zeros(self.shape[2], np.uint64)
        xc = np.zeros(K, np.uint64)
        for k0, a, b, c in self.pool.imap_unordered(_marg_task, [(k0, k1, S) for k0, k1 in self._chunks(K)]):
            xa += a
            xb += b
            xc[k0:k0 + c.shape[0]] = c
        return O.State(X=X0, A=np.array(A, np.float64), B=np.array(B, np.float64), C=np.array(C, np.float64),
                       lam=np.array(lam, np.float64), S=S, xa=xa, xb=xb, xc=xc, batch=batch, opts=opts)

    def full_fit(self, state: O.State) -> float:
        """sambaten.full_fit of the state's model against its slices, the
        slice sums computed in the workers and added in slice order."""
        K = state.X.shape[0]
        parts = sorted(self.pool.imap_unordered(
            _fit_task, [(k0, k1, state.lam, state.A, state.B, state.C) for k0, k1 in self._chunks(K)]))
        num = 0.0
        den = 0.0
        for _, n, d in parts:
            num += n
            den += d
        return 1.0 - float(np.sqrt(num)) / float(np.sqrt(den))

    def update(self, state: O.State, K_new: int):
        """Algorithm 1 for the K_new stored slices that follow state's; the
        same steps and results as sambaten.update on those slices."""
        K_old = state.X.shape[0]
        K_all = K_old + K_new
        if K_all > self.shape[0]:
            raise ValueError("the store holds fewer slices")
        X_all = self.X[:K_all]
        if not np.all(np.isfinite(X_all[K_old:])):
            raise FloatingPointError("non-finite value in the new slices")
        sizes = O.batch_sample_sizes(state)
        args = [(K_all, K_new, (state.A, state.B, state.C, state.lam), (state.xa, state.xb, state.xc), state.S,
                 state.batch, state.opts, sizes, rho) for rho in range(state.opts.r)]
        traces = [None] * state.opts.r
        for rho, t in self.pool.imap_unordered(_rep_task, args):
            traces[rho] = t
        return O.commit(state, X_all, K_new, traces), traces

    def close(self):
        if getattr(self, "pool", None) is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None
        if getattr(self, "shm", None) is not None:
            self.X = None
            try:
                self.shm.close()
            except BufferError:
                # states returned by update() still view the slices: the
                # mapping stays until they are gone; the name is removed now
                pass
            self.shm.unlink()
            self.shm = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
