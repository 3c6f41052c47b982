"""The persistent ALS (one cooperative launch for every iteration and
repetition, grid barriers between the steps) against the launch-per-step ALS.

Both run the same device functions in the same summation orders with the
float64 R x R tail, so every result is the same bits:
  * float64 summaries (the graph path's tail is float64 already): the small
    dense workload (100 x 100 x (50 + 5), R = 5, s = 2, r = 4) to
    convergence, and with fixed iterations;
  * float32 summaries against the graph path with fp64_tail = 1;
  * GetRank (Section 3.2) on float32 summaries: candidate ALS at every rank,
    then the final ALS at each repetition's rank, both through the
    persistent launch;
and the persistent path's update agrees with the FP64 oracle like the graph
path does (float64 1e-7 relative).
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


def _data(I, J, K, R, dtype, seed=3):
    from paper_1709_00668_gb300 import synth
    p = synth.planted_dense(I, J, K, R, noise=0.01, seed=seed, dtype=dtype)
    return p.X.numpy(), p.A.numpy(), p.B.numpy(), p.C.numpy()


def _unit(A, B, C):
    na, nb, nc = (np.linalg.norm(u, axis=0) for u in (A, B, C))
    return na * nb * nc, A / na, B / nb, C / nc


def _run(sbt, X, fac, K0, Kn, R, **opts):
    r = opts["r"]
    ctx = sbt.SamBaTen(torch.from_numpy(X[:K0]).cuda(), R, factors=fac, **opts)
    ctx.update(torch.from_numpy(X[K0:K0 + Kn]).cuda())
    st = ctx.stats()
    out = {"factors": ctx.factors(), "iters": st["iters"], "fit": st["fit"], "perm": st["perm"],
           "rank": st.get("rank"), "Us": [ctx.last_summary_factors(rep) for rep in range(r)],
           "model_fit": ctx.fit()}
    ctx.close()
    return out


def _same(a, b):
    for x, y in zip(a["factors"], b["factors"]):
        assert np.array_equal(x, y)
    assert a["iters"] == b["iters"] and a["perm"] == b["perm"] and a["rank"] == b["rank"]
    assert a["fit"] == b["fit"]
    for ua, ub in zip(a["Us"], b["Us"]):
        for x, y in zip(ua, ub):
            assert np.array_equal(x, y)
    assert a["model_fit"] == b["model_fit"]


@pytest.mark.parametrize("fixed", [0, 1])
def test_f64_persistent_equals_graph_path(sbt, fixed):
    K0, Kn, R, r = 50, 5, 5, 4
    X, A, B, C = _data(100, 100, K0 + Kn, R, torch.float64)
    fac = _unit(A, B, C[:K0])
    opts = dict(s_I=2, s_J=2, s_K=2, r=r, seed=0, prec="f64", tol=1e-6 if not fixed else 0.0,
                max_iters=60 if not fixed else 12, fixed_iters=fixed)
    g = _run(sbt, X, fac, K0, Kn, R, **opts)
    p = _run(sbt, X, fac, K0, Kn, R, persistent_als=1, **opts)
    _same(g, p)
    if fixed:
        assert p["iters"] == [12] * r
    # and against the FP64 oracle (with the tolerance stop: its iteration counts)
    oo = O.Options(s_I=2, s_J=2, s_K=2, r=r, tol=opts["tol"], max_iters=opts["max_iters"],
                   fixed_iters=bool(fixed), seed=0, prec="f64")
    ost2, traces = O.update(O.init_state_from_factors(X[:K0], *fac, oo), X[K0:K0 + Kn])
    assert p["iters"] == [t.als.iters for t in traces]
    lam, Ag, Bg, Cg = p["factors"]
    assert rel_err(Cg[K0:], ost2.C[K0:]) < 1e-7


def test_f32_persistent_equals_fp64_tail(sbt):
    K0, Kn, R, r = 60, 12, 8, 6
    X, A, B, C = _data(150, 130, K0 + Kn, R, torch.float32, seed=7)
    fac = _unit(A, B, C[:K0])
    opts = dict(s_I=2, s_J=2, s_K=2, r=r, seed=0, prec="f32", tol=1e-7, max_iters=30)
    g = _run(sbt, X, fac, K0, Kn, R, fp64_tail=1, **opts)
    p = _run(sbt, X, fac, K0, Kn, R, persistent_als=1, **opts)
    _same(g, p)


def test_get_rank_persistent_equals_fp64_tail(sbt):
    K0, Kn, R, r = 24, 6, 4, 3
    X, A, B, C = _data(40, 36, K0 + Kn, 2, torch.float32, seed=31)
    rng = np.random.default_rng(5)
    A = np.concatenate([A, rng.random((40, 2))], axis=1)
    B = np.concatenate([B, rng.random((36, 2))], axis=1)
    C = np.concatenate([C[:K0], rng.random((K0, 2))], axis=1)
    fac = _unit(A, B, C)
    opts = dict(s_I=2, s_J=2, s_K=2, r=r, seed=0, prec="f32", tol=0.0, max_iters=40, fixed_iters=1,
                get_rank=1, get_rank_trials=2, get_rank_threshold=90.0)
    g = _run(sbt, X, fac, K0, Kn, R, fp64_tail=1, **opts)
    p = _run(sbt, X, fac, K0, Kn, R, persistent_als=1, **opts)
    _same(g, p)
    assert p["rank"] == [2] * r


def test_persistent_option_validated(sbt):
    X, A, B, C = _data(30, 30, 20, 3, torch.float64)
    with pytest.raises(sbt.SbtError) as e:
        sbt.SamBaTen(torch.from_numpy(X).cuda(), 3, prec="f64", persistent_als=2)
    assert e.value.status == sbt.SBT_E_INVALID
