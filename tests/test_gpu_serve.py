"""Serving loop and device-memory accounting on the GPU.

Many tensor streams are absorbed concurrently by one server; each stream's
factors must be bit-identical to those of the same stream absorbed alone
(every kernel reduces in a fixed order, whatever shares the GPU), and the
server must keep the device bytes of all streams within its budget."""
import numpy as np
import pytest
import torch

from tests._util import planted

pytestmark = pytest.mark.gpu

# (I, J, R, prec, seed): uneven shapes and precisions in one mix.  Every
# standalone path here is the one the parity tests check against the oracle.
STREAMS = [(60, 50, 3, "bf16", 1), (80, 40, 5, "f32", 2), (48, 64, 4, "bf16", 3), (100, 30, 2, "f32", 4)]
K0 = 20


@pytest.fixture(scope="module")
def sbt():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_00668_gb300 import build, sbt as S
    build.build()
    return S


def _opts(prec, seed):
    return dict(s_I=2, s_J=2, s_K=2, r=3, tol=1e-6, max_iters=12, max_iters_init=15, seed=seed,
                prec=prec, stream_id=seed, K_capacity=80, max_batch=8)


def _data(I, J, R, seed, batches):
    X, *_ = planted(I, J, K0 + sum(batches), R, seed=seed)
    return torch.from_numpy(X).cuda()


def _batch_sizes(seed):
    return [int(b) for b in np.random.default_rng(seed).integers(1, 9, size=4)]


def _alone(sbt, I, J, R, prec, seed):
    sizes = _batch_sizes(seed)
    X = _data(I, J, R, seed, sizes)
    ctx = sbt.SamBaTen(X[:K0], R, **_opts(prec, seed))
    k = K0
    for b in sizes:
        ctx.update(X[k:k + b])
        k += b
    out = ctx.factors()
    ctx.close()
    return out


def test_update_bytes_predicts_the_footprint(sbt):
    I, J, R = 70, 45, 3
    X = _data(I, J, R, 5, [6] * 6)
    for prec in ("bf16", "f32"):
        ctx = sbt.SamBaTen(X[:K0], R, **{**_opts(prec, 5), "K_capacity": 22, "max_batch": 0})
        k = K0
        for b in (6, 1, 6, 6, 5):  # the store doubles on the way
            want = ctx.update_bytes(b)
            ctx.update(X[k:k + b])
            k += b
            assert ctx.device_bytes() == want
        ctx.close()


def test_reserve_makes_updates_allocation_free(sbt):
    I, J, R = 64, 52, 4
    sizes = [8, 1, 5, 8, 3, 8, 2, 7]
    X = _data(I, J, R, 6, sizes)
    ctx = sbt.SamBaTen(X[:K0], R, **{**_opts("bf16", 6), "K_capacity": K0 + sum(sizes), "max_batch": 8})
    held = ctx.device_bytes()
    k = K0
    for b in sizes:
        assert ctx.update_bytes(b) == held
        ctx.update(X[k:k + b])
        k += b
        assert ctx.device_bytes() == held
    ctx.close()


def test_each_stream_same_alone_and_in_the_mix(sbt):
    alone = [_alone(sbt, *s) for s in STREAMS]
    srv = sbt.Server(slots=4, mem_budget=8 << 30)
    data, sids, sizes = [], [], []
    for (I, J, R, prec, seed) in STREAMS:
        sz = _batch_sizes(seed)
        X = _data(I, J, R, seed, sz)
        data.append(X)
        sizes.append(sz)
        sids.append(srv.open_stream(X[:K0], R, **_opts(prec, seed)))
    torch.cuda.synchronize()
    tickets = []
    offs = [K0] * len(STREAMS)
    for b in range(4):  # round robin: every stream's batches in flight together
        for q in range(len(STREAMS)):
            n = sizes[q][b]
            tickets.append((q, srv.submit(sids[q], data[q][offs[q]:offs[q] + n]), offs[q] + n))
            offs[q] += n
    for q, t, k_after in tickets:
        res = srv.wait(t, 120000)
        assert res["status"] == sbt.SBT_OK, res
        assert res["stream"] == sids[q] and res["K"] == k_after
        assert res["total_ms"] >= res["service_ms"] > 0
    st = srv.stats()
    assert st["completed"] == 4 * len(STREAMS) and st["failed"] == 0
    assert st["slices"] == sum(sum(s) for s in sizes)
    assert 0 < st["latency_p50_ms"] <= st["latency_p99_ms"]
    assert 0 < st["busy_fraction"] <= 1.0
    assert st["peak_resident_bytes"] <= st["mem_budget"]
    for q in range(len(STREAMS)):
        mix = srv.stream(sids[q]).factors()
        for a, b in zip(alone[q], mix):
            assert np.array_equal(a, b)
    assert srv.stream(sids[1]).K == K0 + sum(sizes[1])
    srv.close()


def test_budget_admission_and_release(sbt):
    """A batch whose workspace does not fit waits until another stream is
    closed; a stream that does not fit is refused."""
    I, J, R = 90, 70, 4
    X1 = _data(I, J, R, 7, [8])
    X2 = _data(I, J, R, 8, [8])
    o = {**_opts("bf16", 7), "max_batch": 0, "K_capacity": 40}
    # measure the footprints on a throwaway context of the same shape
    probe = sbt.SamBaTen(X1[:K0], R, **o)
    opened = probe.device_bytes()
    after = probe.update_bytes(8)
    probe.close()
    assert opened > after - opened > 0  # a third stream is larger than one update's growth
    budget = 2 * opened + (after - opened) - 1  # both streams fit, one update's growth does not
    srv = sbt.Server(slots=2, mem_budget=budget)
    s1 = srv.open_stream(X1[:K0], R, **o)
    s2 = srv.open_stream(X2[:K0], R, **{**o, "seed": 8})
    st, _ = srv.open_stream_status(X2[:K0], R, **o)
    assert st == sbt.SBT_E_NOMEM
    torch.cuda.synchronize()
    t = srv.submit(s1, X1[K0:K0 + 8])
    with pytest.raises(sbt.SbtError) as e:
        srv.wait(t, 300)
    assert e.value.status == sbt.SBT_E_TIMEOUT
    assert srv.stats()["queued"] == 1
    srv.close_stream(s2)  # frees memory: the batch is admitted
    res = srv.wait(t, 120000)
    assert res["status"] == sbt.SBT_OK and res["K"] == K0 + 8
    st = srv.stats()
    assert st["peak_resident_bytes"] <= budget
    assert st["resident_bytes"] == after
    srv.close()


def test_failed_batch_leaves_its_stream_usable(sbt):
    I, J, R, prec, seed = STREAMS[0]
    sizes = _batch_sizes(seed)
    X = _data(I, J, R, seed, sizes)
    srv = sbt.Server(slots=2, mem_budget=4 << 30)
    sid = srv.open_stream(X[:K0], R, **_opts(prec, seed))
    bad = X[K0:K0 + 3].clone()
    bad[1, 2, 3] = float("nan")
    torch.cuda.synchronize()
    t_bad = srv.submit(sid, bad)
    ts, k = [], K0
    for b in sizes:
        ts.append(srv.submit(sid, X[k:k + b]))
        k += b
    assert srv.wait(t_bad)["status"] == sbt.SBT_E_NONFINITE
    # the failed batch's message reaches the waiting thread
    assert b"non-finite" in sbt.lib().sbt_last_error()
    for t in ts:
        assert srv.wait(t)["status"] == sbt.SBT_OK
    got = srv.stream(sid).factors()
    for a, b in zip(_alone(sbt, I, J, R, prec, seed), got):
        assert np.array_equal(a, b)
    assert srv.stats()["failed"] == 1
    srv.close()


# batch_als: f32 and f64 streams with the persistent ALS (the CUDA-core path),
# ranks in two ranges (1-8 and 9-16), and a bf16 stream that runs whole
BATCHED = [(60, 50, 3, "f32", 11), (80, 70, 5, "f32", 12), (45, 64, 8, "f32", 13), (70, 40, 12, "f32", 14),
           (50, 52, 4, "f64", 15), (64, 48, 6, "f32", 16), (40, 44, 3, "bf16", 17)]


def _bopts(prec, seed):
    o = _opts(prec, seed)
    if prec != "bf16":
        o["persistent_als"] = 1
    return o


def _alone_b(sbt, I, J, R, prec, seed):
    sizes = _batch_sizes(seed)
    X = _data(I, J, R, seed, sizes)
    if prec == "f64":
        X = X.double()
    ctx = sbt.SamBaTen(X[:K0], R, **_bopts(prec, seed))
    k = K0
    for b in sizes:
        ctx.update(X[k:k + b])
        k += b
    out = ctx.factors()
    ctx.close()
    return out


def test_batched_als_each_stream_same_as_alone(sbt):
    """A server with batch_als runs the summary ALS of several streams'
    updates in one persistent launch; every stream's factors are the same
    bits as the stream absorbed alone with the persistent ALS."""
    alone = [_alone_b(sbt, *s) for s in BATCHED]
    srv = sbt.Server(slots=8, mem_budget=8 << 30, batch_als=1)
    data, sids, sizes = [], [], []
    for (I, J, R, prec, seed) in BATCHED:
        sz = _batch_sizes(seed)
        X = _data(I, J, R, seed, sz)
        if prec == "f64":
            X = X.double()
        data.append(X)
        sizes.append(sz)
        sids.append(srv.open_stream(X[:K0], R, **_bopts(prec, seed)))
    torch.cuda.synchronize()
    srv.stats_reset()
    tickets = []
    offs = [K0] * len(BATCHED)
    for b in range(4):
        for q in range(len(BATCHED)):
            n = sizes[q][b]
            tickets.append((q, srv.submit(sids[q], data[q][offs[q]:offs[q] + n]), offs[q] + n))
            offs[q] += n
    for q, t, k_after in tickets:
        res = srv.wait(t, 120000)
        assert res["status"] == sbt.SBT_OK, res
        assert res["K"] == k_after
    st = srv.stats()
    assert st["completed"] == 4 * len(BATCHED) and st["failed"] == 0
    # the six persistent streams' 24 updates went through batched launches,
    # more than one set per launch on average
    assert st["als_sets"] == 4 * 6
    assert 0 < st["als_launches"] < st["als_sets"]
    for q in range(len(BATCHED)):
        mix = srv.stream(sids[q]).factors()
        for a, b in zip(alone[q], mix):
            assert np.array_equal(a, b), BATCHED[q]
    srv.close()


def test_batched_als_failed_batch_leaves_the_others(sbt):
    """batch_als: a batch with a non-finite value fails alone (SBT_E_NONFINITE);
    the other updates admitted with it, and the failing stream's later
    batches, give the same bits as each stream absorbed alone."""
    picks = [BATCHED[0], BATCHED[1], BATCHED[4]]
    alone = [_alone_b(sbt, *s) for s in picks]
    srv = sbt.Server(slots=8, mem_budget=8 << 30, batch_als=1)
    data, sids, sizes = [], [], []
    for (I, J, R, prec, seed) in picks:
        sz = _batch_sizes(seed)
        X = _data(I, J, R, seed, sz)
        if prec == "f64":
            X = X.double()
        data.append(X)
        sizes.append(sz)
        sids.append(srv.open_stream(X[:K0], R, **_bopts(prec, seed)))
    bad = data[0][K0:K0 + 3].clone()
    bad[1, 2, 3] = float("nan")
    torch.cuda.synchronize()
    t_bad = srv.submit(sids[0], bad)
    tickets, offs = [], [K0] * len(picks)
    for b in range(4):
        for q in range(len(picks)):
            n = sizes[q][b]
            tickets.append(srv.submit(sids[q], data[q][offs[q]:offs[q] + n]))
            offs[q] += n
    assert srv.wait(t_bad)["status"] == sbt.SBT_E_NONFINITE
    for t in tickets:
        assert srv.wait(t)["status"] == sbt.SBT_OK
    for q in range(len(picks)):
        for a, b in zip(alone[q], srv.stream(sids[q]).factors()):
            assert np.array_equal(a, b), picks[q]
    srv.close()
