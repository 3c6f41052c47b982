"""Test scaffolding shared by the GPU parity tests (input preparation only)."""
import numpy as np
import torch

from paper_1709_00668_gb300 import synth


def planted(I, J, K, R, *, noise=0.01, seed=0, dtype=torch.float32, dist="uniform"):
    """Planted tensor as numpy (K, I, J) plus unit-column factors and lambda of the first K0 rows."""
    p = synth.planted_dense(I, J, K, R, noise=noise, seed=seed, dtype=dtype, dist=dist)
    return p.X.numpy(), p.A.numpy(), p.B.numpy(), p.C.numpy()


def unit_factors(A, B, C):
    na, nb, nc = (np.linalg.norm(u, axis=0) for u in (A, B, C))
    return na * nb * nc, A / na, B / nb, C / nc


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
