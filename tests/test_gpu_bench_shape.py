"""Whole-update parity at the launch configuration the benchmark times.

The dense FP32 single-stream workload (1000 x 1000 store, R = 10, s = 5,
r = 8, bfloat16 summaries) gives 200 x 200 summaries with 150 slices at the
first batch and up to 340 later: two 104-row tensor-core tiles per slice, the
repetitions in the default two groups, 13-chunk cluster tails for modes 1 and
2, and the mode-3 MTTKRP formed from the mode-2 pass's products over every
slice.  These tests run that path through the C ABI and compare it with the
oracle element by element:
  * fixed iterations, oracle on the same bfloat16 values: samples and
    summaries bit-exact, matches equal, summary factors and the updated model
    within the bfloat16 bar (1e-3 relative);
  * the benchmark's own settings (tol 1e-6, at most 50 iterations) against
    the FP64 oracle: samples bit-exact and the full-tensor fit after the
    batch within 1e-3 (the metric's condition).
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


def _planted_gpu(I, J, K, R, seed=0):
    from paper_1709_00668_gb300 import synth
    p = synth.planted_dense(I, J, K, R, noise=0.01, seed=seed, dtype=torch.float32, device="cuda")
    A, B, C = p.A.cpu().numpy(), p.B.cpu().numpy(), p.C.cpu().numpy()
    return p.X, A, B, C


def _unit(A, B, C):
    na, nb, nc = (np.linalg.norm(u, axis=0) for u in (A, B, C))
    return na * nb * nc, A / na, B / nb, C / nc


def _run(sbt, Xd, K0, Kn, R, fac, s, **kw):
    opts = dict(s_I=s, s_J=s, s_K=s, r=8, seed=0, prec="bf16")
    opts.update(kw)
    ctx = sbt.SamBaTen(Xd[:K0], R, factors=fac, **opts)
    ctx.update(Xd[K0:K0 + Kn])
    return ctx


@pytest.mark.parametrize("I,s,K0", [(1000, 5, 500), (400, 2, 580)])
def test_bf16_update_at_benchmark_summary_geometry(sbt, I, s, K0):
    """200 x 200 summaries, 150 (first batch of the benchmark) and 340
    slices (its last batch at 20 steps), r = 8 in the default groups, the
    memoised mode 3; 6 fixed ALS iterations on both sides."""
    Kn, R, iters = 50, 10, 6
    Xd, A, B, C = _planted_gpu(I, I, K0 + Kn, R, seed=1)
    fac = _unit(A, B, C[:K0])
    ctx = _run(sbt, Xd, K0, Kn, R, fac, s, tol=0.0, max_iters=iters, fixed_iters=1)
    X = Xd[:K0 + Kn].cpu().numpy()
    oo = O.Options(s_I=s, s_J=s, s_K=s, r=8, tol=0.0, max_iters=iters, fixed_iters=True, seed=0, prec="bf16")
    ost = O.init_state_from_factors(X[:K0], *fac, oo)
    ost2, traces = O.update(ost, X[K0:K0 + Kn], keep_summaries=True)
    st = ctx.stats()
    assert (st["n_I"], st["n_J"], st["n_K"]) == (200, 200, K0 // s)
    for rep, t in enumerate(traces):
        for m, ref in enumerate((t.Is, t.Js, t.Ks)):
            assert np.array_equal(ctx.last_samples(rep, m), ref), (rep, m)
        if rep in (0, 5):  # two repetitions, one in each group: the summary values bit for bit
            assert np.array_equal(ctx.last_summary(rep), t.Xs), rep
        assert st["perm"][rep] == list(t.match.perm), rep
        assert st["iters"][rep] == iters
        lam_s, As, Bs, Cs = ctx.last_summary_factors(rep)
        for g, o in zip((lam_s, As, Bs, Cs), (t.lam_s, t.Us[0], t.Us[1], t.Us[2])):
            assert rel_err(g, o) < 1e-3, rep
        assert abs(st["fit"][rep] - t.als.fit) < 1e-4, rep
    lam, Ag, Bg, Cg = ctx.factors()
    assert Cg.shape == ost2.C.shape
    assert rel_err(Cg[K0:], ost2.C[K0:]) < 1e-3
    assert np.array_equal(Ag, ost2.A) and np.array_equal(Cg[:K0], ost2.C[:K0])  # no zero entries to fill
    f_g = ctx.fit()
    f_o = O.full_fit(ost2.X, ost2.lam, ost2.A, ost2.B, ost2.C)
    assert abs(f_g - f_o) < 1e-5, (f_g, f_o)
    ctx.close()


def test_benchmark_settings_fit_within_1e3_of_fp64(sbt):
    """The benchmark's first batch with its own settings (tol 1e-6, 50
    iterations): the bf16 GPU update and the FP64 oracle update from the same
    pre-update model draw the same samples, and the full-tensor fits after
    the batch agree within 1e-3."""
    from oracle.pool import PoolOracle
    import os
    I, K0, Kn, R, s = 1000, 500, 50, 10, 5
    Xd, A, B, C = _planted_gpu(I, I, K0 + Kn, R, seed=0)
    fac = _unit(A, B, C[:K0])
    ctx = _run(sbt, Xd, K0, Kn, R, fac, s, tol=1e-6, max_iters=50)
    f_g = ctx.fit()
    cores = len(os.sched_getaffinity(0))
    oo = O.Options(s_I=s, s_J=s, s_K=s, r=8, tol=1e-6, max_iters=50, seed=0, prec="f64")
    with PoolOracle(Xd[:K0 + Kn].cpu().numpy(), workers=min(8, cores), threads=max(1, cores // 8)) as po:
        st0 = po.state(K0, *fac, oo)
        st1, traces = po.update(st0, Kn)
        f_o = po.full_fit(st1)
        for rep, t in enumerate(traces):
            for m, ref in enumerate((t.Is, t.Js, t.Ks)):
                assert np.array_equal(ctx.last_samples(rep, m), ref), (rep, m)
        del st0, st1
    print(f"full-tensor fit after the batch: GPU bf16 {f_g:.7f}, FP64 oracle {f_o:.7f}")
    assert abs(f_g - f_o) <= 1e-3
    ctx.close()
