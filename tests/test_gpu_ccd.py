"""GPU CorConDia (sbt_core_consistency) against the oracle's core consistency.

The diagnostic GetRank scores candidate decompositions with (Section 3.2,
Algorithm 2); both sides compute it in float64 from the same values, so the
bar is 1e-9 relative (rounding order only)."""
import numpy as np
import pytest
import torch

from oracle import sambaten as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbt():
    from paper_1709_00668_gb300 import build, sbt as s
    build.build()
    s.lib()
    return s


def _model(I, J, K, R, seed):
    rng = np.random.default_rng(seed)
    return (rng.random(R) + 0.5, rng.random((I, R)), rng.random((J, R)), rng.random((K, R)))


def _gpu_cc(sbt, X, model, ld, dtype):
    K, I, J = X.shape
    Xp = np.zeros((K, I, ld), dtype=dtype)
    Xp[:, :, :J] = X
    dev = [torch.from_numpy(np.ascontiguousarray(t)).cuda() for t in model]
    return sbt.sbt_core_consistency(torch.from_numpy(Xp).cuda(), *dev)


@pytest.mark.parametrize("dtype,shape,ld", [(np.float64, (23, 37, 29, 5), 32), (np.float32, (30, 40, 36, 4), 40),
                                            (np.float32, (24, 26, 22, 20), 24)])
def test_core_consistency_matches_oracle(sbt, dtype, shape, ld):
    K, I, J, R = shape
    lam, A, B, C = _model(I, J, K, R, seed=K)
    X = O.reconstruct(lam, A, B, C).astype(dtype)
    Xo = X.astype(np.float64)
    rng = np.random.default_rng(1)
    # the exact model (100), a perturbed one, and an over-factored one (an extra
    # random component): all well conditioned
    models = [(lam, A, B, C),
              (lam * 1.02, A + 0.01 * rng.random(A.shape), B, C),
              (np.concatenate([lam, [0.3]]), np.hstack([A, rng.random((I, 1))]),
               np.hstack([B, rng.random((J, 1))]), np.hstack([C, rng.random((K, 1))]))]
    if R + 1 > min(I, J, K):
        models = models[:2]
    for m in models:
        ref = O.core_consistency(Xo, *m)
        got = _gpu_cc(sbt, X, m, ld, dtype)
        assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref)), (got, ref)
    assert abs(_gpu_cc(sbt, X, models[0], ld, dtype) - 100.0) < (1e-6 if dtype == np.float64 else 1e-2)


def test_core_consistency_rejects_rank_deficient_factor(sbt):
    K, I, J, R = 10, 12, 11, 3
    lam, A, B, C = _model(I, J, K, R, seed=3)
    A[:, 2] = 0.0  # a zero column: row and column 2 of A^T A stay exactly zero, so the pivot is 0
    X = O.reconstruct(lam, A, B, C)
    with pytest.raises(RuntimeError):
        _gpu_cc(sbt, X, (lam, A, B, C), 16, np.float64)
