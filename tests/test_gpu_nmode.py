"""Order-N tensors on the GPU (Section 2.2's extension) against the order-N
oracle (`oracle/nmode.py`), element by element on the same seeded inputs.

Sampled indices of every mode bit-exact; matches equal; the summary ALS's
iteration counts and fits; the appended time rows and the full-tensor fit
within the tolerance of the arithmetic (float64 1e-8 relative, float32
summaries 1e-4).  N = 3 through the order-N path, N = 4 and N = 5, with
ragged sizes that span several CTAs of the MTTKRP and both its variants.
"""
import numpy as np
import pytest
import torch

from oracle import nmode
from oracle import sambaten as O
from tests._util import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbt():
    from paper_1709_00668_gb300 import build, sbt as s
    build.build()
    s.lib()
    return s


def _case(dims, K0, Kn, R, dtype, seed):
    from paper_1709_00668_gb300 import synth
    p = synth.planted_dense_n(dims, K0 + Kn, R, noise=0.01, seed=seed, dtype=dtype)
    X = p.X.numpy()
    U = [u.numpy() for u in p.U[:-1]] + [p.U[-1].numpy()[:K0]]
    norms = [np.linalg.norm(u, axis=0) for u in U]
    lam = np.prod(norms, axis=0)
    return X, lam, [u / n for u, n in zip(U, norms)]


@pytest.mark.parametrize("dims,K0,Kn,R,prec,ftol", [
    ((40, 36), 30, 7, 3, "f64", 1e-8),
    ((18, 17, 70), 21, 5, 3, "f64", 1e-8),
    ((18, 17, 70), 21, 5, 3, "f32", 1e-4),
    ((9, 7, 6, 11), 10, 3, 2, "f64", 1e-8),
])
def test_nmode_update_matches_order_n_oracle(sbt, dims, K0, Kn, R, prec, ftol):
    dtype = torch.float64 if prec == "f64" else torch.float32
    X, lam, U = _case(dims, K0, Kn, R, dtype, seed=len(dims) * 7 + K0)
    N = len(dims) + 1
    opts = dict(s_I=2, s_J=2, s_K=2, r=3, tol=0.0, max_iters=25, fixed_iters=1, seed=0)
    ctx = sbt.SamBaTenN(torch.from_numpy(X[:K0]).cuda(), R, factors=(lam, U), prec=prec, **opts)
    ctx.update(torch.from_numpy(X[K0:K0 + Kn]).cuda())
    oo = O.Options(s_I=2, s_J=2, s_K=2, r=3, tol=0.0, max_iters=25, fixed_iters=True, seed=0, prec=prec)
    ost = nmode.init_state_from_factors(X[:K0], lam, U, oo)
    ost2, traces = nmode.update(ost, X[K0:K0 + Kn])
    st = ctx.stats()
    for rep, t in enumerate(traces):
        for m in range(N):
            assert np.array_equal(ctx.last_samples(rep, m), t["idx"][m]), (rep, m)
        assert st["perm"][rep] == list(t["match"].perm), rep
        assert st["iters"][rep] == t["als"].iters == 25
        assert abs(st["fit"][rep] - t["als"].fit) < ftol
    lam_g, Ug = ctx.factors()
    assert Ug[-1].shape == ost2.U[-1].shape
    assert rel_err(Ug[-1][K0:], ost2.U[-1][K0:]) < ftol
    for m in range(N - 1):
        assert np.array_equal(Ug[m], ost2.U[m])
    assert np.array_equal(Ug[-1][:K0], ost2.U[-1][:K0]) and np.array_equal(lam_g, ost2.lam)
    Xh = nmode.reconstruct(ost2.lam, ost2.U)
    f_o = 1.0 - np.linalg.norm((ost2.X.astype(np.float64) - Xh).ravel()) / np.linalg.norm(ost2.X.astype(np.float64).ravel())
    assert abs(ctx.fit() - f_o) < 10 * ftol
    ctx.close()


def test_nmode_stream_with_tolerance_stop(sbt):
    """Three batches at N = 4 with the tolerance stop (float64): the same
    iteration counts and samples as the oracle after every batch, and the
    marginals carried across batches (the later samples depend on them)."""
    dims, K0, R = (12, 11, 10), 16, 2
    X, lam, U = _case(dims, K0, 12, R, torch.float64, seed=3)
    opts = dict(s_I=2, s_J=2, s_K=2, r=2, tol=1e-8, max_iters=80, seed=5)
    ctx = sbt.SamBaTenN(torch.from_numpy(X[:K0]).cuda(), R, factors=(lam, U), prec="f64", **opts)
    oo = O.Options(s_I=2, s_J=2, s_K=2, r=2, tol=1e-8, max_iters=80, seed=5, prec="f64")
    ost = nmode.init_state_from_factors(X[:K0], lam, U, oo)
    for k0, k1 in ((16, 20), (20, 21), (21, 28)):
        ctx.update(torch.from_numpy(X[k0:k1]).cuda())
        ost, traces = nmode.update(ost, X[k0:k1])
        st = ctx.stats()
        assert st["iters"] == [t["als"].iters for t in traces]
        for rep, t in enumerate(traces):
            assert np.array_equal(ctx.last_samples(rep, 3), t["idx"][3])
        assert rel_err(ctx.factors()[1][-1], ost.U[-1]) < 1e-7
    ctx.close()


def test_nmode_rejects_bad_batches(sbt):
    X, lam, U = _case((10, 9, 8), 8, 2, 2, torch.float64, seed=4)
    ctx = sbt.SamBaTenN(torch.from_numpy(X[:8]).cuda(), 2, factors=(lam, U), prec="f64", r=2)
    bad = X[8:10].copy()
    bad[1, 2, 3, 4] = np.nan
    with pytest.raises(sbt.SbtError) as e:
        ctx.update(torch.from_numpy(bad).cuda())
    assert e.value.status == sbt.SBT_E_NONFINITE
    lam_g, Ug = ctx.factors()
    assert Ug[-1].shape[0] == 8  # state unchanged
    with pytest.raises(sbt.SbtError) as e:
        ctx.update(torch.from_numpy(X[8:10, :, :, :5].copy()).cuda())
    assert e.value.status == sbt.SBT_E_SHAPE
    ctx.update(torch.from_numpy(X[8:10]).cuda())
    assert ctx.factors()[1][-1].shape[0] == 10
    ctx.close()
