"""GPU parity of the sparse (COO) path against the FP64 oracle.

The oracle has no sparse code: a COO tensor's update is the dense method
applied to the densified tensor, so the oracle runs on the dense array.
Sampled indices match bit for bit; factors and fits within the tolerance of
float32 products added in fixed point (1e-4 relative)."""
import numpy as np
import pytest
import torch

from oracle import sambaten as O
from paper_1709_00668_gb300 import synth
from tests._util import rel_err, unit_factors

pytestmark = pytest.mark.gpu

I, J, K0, KT, R = 400, 360, 40, 60, 4


@pytest.fixture(scope="module")
def sbt():
    from paper_1709_00668_gb300 import build, sbt as s
    build.build()
    s.lib()
    return s


@pytest.fixture(scope="module")
def data():
    return synth.planted_sparse(I, J, KT, R, support=60, coords=4000, noise=0.01, seed=3)


def _opts(**kw):
    o = dict(s_I=4, s_J=4, s_K=4, r=3, tol=1e-6, max_iters=12, seed=5, fixed_iters=1, prec="f32")
    o.update(kw)
    return o


def _pair(sbt, p, perm=None, **kw):
    X = p.dense().numpy()
    fac = unit_factors(p.A.numpy(), p.B.numpy(), p.C[:K0].numpy())
    ii, jj, kk, vv = p.batch(0, K0)
    if perm is not None:
        g = torch.Generator().manual_seed(perm)
        q = torch.randperm(ii.numel(), generator=g)
        ii, jj, kk, vv = ii[q], jj[q], kk[q], vv[q]
    o = _opts(**kw)
    ctx = sbt.SamBaTen.from_coo(ii.cuda(), jj.cuda(), kk.cuda(), vv.cuda(), (I, J, K0), R, factors=fac, **o)
    oo = O.Options(s_I=o["s_I"], s_J=o["s_J"], s_K=o["s_K"], r=o["r"], tol=o["tol"], max_iters=o["max_iters"],
                   seed=o["seed"], fixed_iters=True, prec="f32")
    return ctx, O.init_state_from_factors(X[:K0], *fac, oo), X


def _batch(p, k0, k1, perm=None):
    ii, jj, kk, vv = p.batch(k0, k1)
    if perm is not None:
        g = torch.Generator().manual_seed(perm + k0)
        q = torch.randperm(ii.numel(), generator=g)
        ii, jj, kk, vv = ii[q], jj[q], kk[q], vv[q]
    return ii.cuda(), jj.cuda(), kk.cuda(), vv.cuda()


def test_coo_updates_match_oracle_on_the_dense_tensor(sbt, data):
    ctx, ost, X = _pair(sbt, data)
    for k0, k1 in ((K0, 50), (50, 51), (51, KT)):
        ost, traces = O.update(ost, X[k0:k1])
        ctx.update_coo(*_batch(data, k0, k1), k1 - k0)
        st = ctx.stats()
        for rep, t in enumerate(traces):
            assert np.array_equal(ctx.last_samples(rep, 0), t.Is)
            assert np.array_equal(ctx.last_samples(rep, 1), t.Js)
            assert np.array_equal(ctx.last_samples(rep, 2), t.Ks)
            assert st["perm"][rep] == list(t.match.perm)
            assert abs(st["fit"][rep] - t.als.fit) < 1e-5
        lam, A, B, C = ctx.factors()
        assert rel_err(C, ost.C) < 1e-4 and rel_err(A, ost.A) < 1e-4 and rel_err(B, ost.B) < 1e-4
        assert rel_err(lam, ost.lam) < 1e-4
    assert ctx.K == KT
    f = ctx.fit()
    assert abs(f - O.full_fit(ost.X, ost.lam, ost.A, ost.B, ost.C)) < 1e-6


def test_coo_results_do_not_depend_on_input_order(sbt, data):
    """Fixed-point MTTKRP sums: the same factors, bit for bit, whatever the
    order of the nonzeros in the initial tensor and in the batches."""
    outs = []
    for perm in (None, 11, 12):
        ctx, _, _ = _pair(sbt, data, perm=perm)
        for k0, k1 in ((K0, 50), (50, KT)):
            ctx.update_coo(*_batch(data, k0, k1, perm=perm), k1 - k0)
        outs.append(ctx.factors())
        ctx.close()
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b)


def test_coo_bad_batches_leave_the_state_unchanged(sbt, data):
    ctx, _, _ = _pair(sbt, data)
    before = ctx.factors()
    ii, jj, kk, vv = _batch(data, K0, 50)
    bad_v = vv.clone()
    bad_v[3] = float("nan")
    assert ctx.update_coo_status(ii, jj, kk, bad_v, 10) == sbt.SBT_E_NONFINITE
    bad_i = ii.clone()
    bad_i[5] = I
    assert ctx.update_coo_status(bad_i, jj, kk, vv, 10) == sbt.SBT_E_SHAPE
    assert ctx.K == K0
    for a, b in zip(before, ctx.factors()):
        assert np.array_equal(a, b)
    ctx.update_coo(ii, jj, kk, vv, 10)
    assert ctx.K == 50
    with pytest.raises(sbt.SbtError):
        ctx.update(torch.zeros(2, I, J, device="cuda"))


def test_coo_init_als_matches_oracle(sbt, data):
    """CP-ALS of the initial COO tensor (the identity summary) against the
    oracle's initial decomposition of the dense tensor."""
    X = data.dense().numpy()
    ii, jj, kk, vv = data.batch(0, K0)
    o = _opts(max_iters_init=15)
    ctx = sbt.SamBaTen.from_coo(ii.cuda(), jj.cuda(), kk.cuda(), vv.cuda(), (I, J, K0), R, **o)
    oo = O.Options(s_I=4, s_J=4, s_K=4, r=3, max_iters_init=15, seed=5, fixed_iters=True)
    st, _ = O.init_decomposition(X[:K0], R, oo)
    lam, A, B, C = ctx.factors()
    assert rel_err(A, st.A) < 1e-4 and rel_err(C, st.C) < 1e-4 and rel_err(lam, st.lam) < 1e-4
