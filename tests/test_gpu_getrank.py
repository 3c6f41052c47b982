"""GetRank (Section 3.2, Algorithm 2) inside the GPU update, against the oracle.

The tensor is planted at rank 2 and the model has R = 4 components (the two
planted ones and two spurious ones).  Every summary's candidate
decompositions at ranks 1..4 (two trials each) are scored by core
consistency; the summaries are rank 2, so R_new = 2, the two summary
components are matched to the two planted old components (a rectangular
assignment), and the new rows of C average each component over the
repetitions that matched it (the spurious components get zero rows).

Compared: sampled indices bit-exact, R_new per repetition and the matches
equal, the summary factors and the updated model within the tolerance of
the arithmetic (float64 1e-7, float32 1e-4, bfloat16 1e-3 relative).
"""
import numpy as np
import pytest
import torch

from oracle import sambaten as O
from tests._util import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbt():
    from paper_1709_00668_gb300 import build, sbt as s
    build.build()
    s.lib()
    return s


def _data(dtype):
    from paper_1709_00668_gb300 import synth
    I, J, K0, Kn = 40, 36, 24, 6
    p = synth.planted_dense(I, J, K0 + Kn, 2, noise=0.01, seed=31, dtype=dtype)
    X = p.X.numpy()
    rng = np.random.default_rng(5)
    # the pre-existing rank-4 model: the planted components and two spurious ones
    A = np.concatenate([p.A.numpy(), rng.random((I, 2))], axis=1)
    B = np.concatenate([p.B.numpy(), rng.random((J, 2))], axis=1)
    C = np.concatenate([p.C.numpy()[:K0], rng.random((K0, 2))], axis=1)
    na, nb, nc = (np.linalg.norm(u, axis=0) for u in (A, B, C))
    lam = na * nb * nc
    lam[2:] *= 0.05
    return X, K0, Kn, (lam, A / na, B / nb, C / nc)


@pytest.mark.parametrize("prec,dtype,ftol", [("f64", torch.float64, 1e-7), ("f32", torch.float32, 1e-4),
                                             ("bf16", torch.float32, 1e-3)])
def test_get_rank_update_matches_oracle(sbt, prec, dtype, ftol):
    X, K0, Kn, fac = _data(dtype)
    R, r, iters = 4, 3, 60
    opts = dict(s_I=2, s_J=2, s_K=2, r=r, tol=0.0, max_iters=iters, fixed_iters=1, seed=0, get_rank=1,
                get_rank_trials=2, get_rank_threshold=90.0)
    ctx = sbt.SamBaTen(torch.from_numpy(X[:K0]).cuda(), R, factors=fac, prec=prec, **opts)
    ctx.update(torch.from_numpy(X[K0:K0 + Kn]).cuda())
    oo = O.Options(s_I=2, s_J=2, s_K=2, r=r, tol=0.0, max_iters=iters, fixed_iters=True, seed=0, prec=prec,
                   get_rank=True, get_rank_trials=2, get_rank_threshold=90.0)
    ost = O.init_state_from_factors(X[:K0], *fac, oo)
    ost2, traces = O.update(ost, X[K0:K0 + Kn])
    st = ctx.stats()
    assert [t.R_new for t in traces] == [2] * r  # the planted rank
    assert st["rank"] == [t.R_new for t in traces]
    for rep, t in enumerate(traces):
        for m, ref in enumerate((t.Is, t.Js, t.Ks)):
            assert np.array_equal(ctx.last_samples(rep, m), ref), (rep, m)
        Rs = t.R_new
        assert st["perm"][rep][:Rs] == list(t.match.perm), rep
        assert all(v == -1 for v in st["perm"][rep][Rs:])
        assert sorted(t.match.perm) == [0, 1]  # the planted components
        lam_s, As, Bs, Cs = ctx.last_summary_factors(rep)
        for g, o in zip((As, Bs, Cs), t.Us):
            assert rel_err(g[:, :Rs], o) < ftol, rep
            assert np.all(g[:, Rs:] == 0.0)
        assert rel_err(lam_s[:Rs], t.lam_s) < ftol
    lam, Ag, Bg, Cg = ctx.factors()
    assert Cg.shape == ost2.C.shape
    assert rel_err(Cg[K0:, :2], ost2.C[K0:, :2]) < ftol
    assert np.all(Cg[K0:, 2:] == 0.0) and np.all(ost2.C[K0:, 2:] == 0.0)  # matched by no repetition
    assert np.array_equal(Cg[:K0], ost2.C[:K0]) and rel_err(lam, ost2.lam) < 1e-15
    f_g = ctx.fit()
    f_o = O.full_fit(ost2.X, ost2.lam, ost2.A, ost2.B, ost2.C)
    assert abs(f_g - f_o) < 10 * ftol
    ctx.close()


def test_get_rank_rejects_unsupported_settings(sbt):
    X, K0, Kn, fac = _data(torch.float32)
    for kw in (dict(prec="fp8"), dict(prec="bf16", refine_sweeps=2)):
        with pytest.raises(sbt.SbtError) as e:
            c = sbt.SamBaTen(torch.from_numpy(X[:K0]).cuda(), 4, factors=fac, get_rank=1, **kw)
            c.update(torch.from_numpy(X[K0:K0 + Kn]).cuda())
        assert e.value.status == sbt.SBT_E_INVALID
