"""The float64 and double-float R x R arithmetic on ill-conditioned normal
equations, against the FP64 oracle fed the same summary values.

Planted rank-20 factors mixed toward a shared direction (the precision-sweep
recipe) so that their Grams have a set condition number; noise 1e-3; the
summary ALS warm-started from those factors at the sampled rows, 8 fixed
iterations on both sides.  For Grams with unit diagonals the Hadamard product
V = G1 * G2 is no worse conditioned than either factor (Schur's bounds on its
eigenvalues), so cond(V) stays near cond(G).

  * cond(G) ~ 1e3 (the sweep's recipe; cond(V) ~ 6e2): both tails within the
    parity bars against FP64 (float32 summaries 1e-4, bfloat16 1e-3) and
    within half the bar of each other.
  * cond(G) ~ 1e4 (cond(V) ~ 7e3): the float32 MTTKRP's rounding (~1e-7
    relative per sum) times cond(V) bounds the summary factors near 1e-3 with
    either tail; the float64 tail keeps the new rows of C within 2e-4 of the
    FP64 oracle, at least 3x closer than the double-float tail.
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


def _data(cond):
    from paper_1709_00668_gb300 import synth
    p = synth.planted_dense(160, 150, 110, 20, noise=1e-3, seed=11, dtype=torch.float32, cond=cond)
    X = p.X.numpy()
    A, B, C = p.A.numpy(), p.B.numpy(), p.C.numpy()[:90]
    na, nb, nc = (np.linalg.norm(u, axis=0) for u in (A, B, C))
    return X, (na * nb * nc, A / na, B / nb, C / nc)


def _run(sbt, X, fac, prec, fp64, K0, Kn, R, iters):
    opts = dict(s_I=2, s_J=2, s_K=2, r=4, tol=0.0, max_iters=iters, fixed_iters=1, seed=0, warm_start=1)
    ctx = sbt.SamBaTen(torch.from_numpy(X[:K0]).cuda(), R, factors=fac, prec=prec, fp64_tail=fp64, **opts)
    ctx.update(torch.from_numpy(X[K0:K0 + Kn]).cuda())
    out = {"stats": ctx.stats(), "C": ctx.factors()[3][K0:],
           "Us": [ctx.last_summary_factors(rep) for rep in range(4)],
           "samples": [ctx.last_samples(rep, 0) for rep in range(4)]}
    ctx.close()
    return out


def _compare(sbt, cond, prec):
    X, fac = _data(cond)
    K0, Kn, R, iters = 90, 20, 20, 8
    res = {fp: _run(sbt, X, fac, prec, fp, K0, Kn, R, iters) for fp in (0, 1)}
    oo = O.Options(s_I=2, s_J=2, s_K=2, r=4, tol=0.0, max_iters=iters, fixed_iters=True, seed=0, prec=prec,
                   warm_start=True)
    ost = O.init_state_from_factors(X[:K0], *fac, oo)
    ost2, traces = O.update(ost, X[K0:K0 + Kn])
    G = [u.T @ u for u in traces[0].als.U]
    condV = np.linalg.cond(G[1] * G[2])
    for fp in (0, 1):
        st = res[fp]["stats"]
        for rep, t in enumerate(traces):
            assert np.array_equal(res[fp]["samples"][rep], t.Is)
            assert st["perm"][rep] == list(t.match.perm) == list(range(R))  # the warm start keeps the order
    gap = max(rel_err(a[q], b[q]) for a, b in zip(res[0]["Us"], res[1]["Us"]) for q in range(1, 4))
    err = {fp: max(max(rel_err(g[q], o) for q, o in zip(range(1, 4), t.Us)) for g, t in zip(res[fp]["Us"], traces))
           for fp in (0, 1)}
    err_c = {fp: rel_err(res[fp]["C"], ost2.C[K0:]) for fp in (0, 1)}
    print(f"cond(G) {cond:.0e} {prec}: cond(V) {condV:.3g}; tails apart {gap:.3g}; against FP64 (double-float / "
          f"float64 tail): summary factors {err[0]:.3g} / {err[1]:.3g}, new C rows {err_c[0]:.3g} / {err_c[1]:.3g}")
    return condV, gap, err, err_c


@pytest.mark.parametrize("prec,bar", [("f32", 1e-4), ("bf16", 1e-3)])
def test_sweep_conditioning_both_tails_within_the_bar(sbt, prec, bar):
    condV, gap, err, err_c = _compare(sbt, 1e3, prec)
    assert 2e2 < condV < 2e3
    assert gap < bar / 2
    for fp in (0, 1):
        assert err[fp] < bar and err_c[fp] < bar


def test_harder_conditioning_fp64_tail(sbt):
    condV, gap, err, err_c = _compare(sbt, 1e4, "f32")
    assert condV > 3e3
    assert max(err.values()) < 2e-3
    assert err_c[1] < 2e-4 and err_c[1] * 3 < err_c[0]
