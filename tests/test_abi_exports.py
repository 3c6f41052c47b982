"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/sambaten.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sambaten.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sbt_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1709_00668_gb300 import build, sbt
    build.build()
    return sbt.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("sbt_init", "sbt_update", "sbt_factors", "sbt_fit", "sbt_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_1709_00668_gb300 import sbt
    assert sorted(sbt.EXPORTS) == declared_symbols()


def test_default_options_and_version(lib):
    from paper_1709_00668_gb300 import sbt
    o = sbt.sbt_default_options()
    assert (o.s_I, o.s_J, o.s_K, o.r, o.max_iters) == (2, 2, 2, 4, 50)
    assert o.tol == 1e-6 and o.prec == sbt.SBT_PREC_F32
    assert "sm_103a" in sbt.version()


def test_invalid_arguments_rejected_without_gpu(lib):
    """Argument checks run before any device call."""
    from paper_1709_00668_gb300 import sbt
    h = ctypes.c_void_p()
    o = sbt.sbt_default_options()
    t = sbt.SbtTensor(sbt.SBT_F32, 0, 4, 4, 4, None)
    assert lib.sbt_init(ctypes.byref(t), 3, ctypes.byref(o), ctypes.byref(h)) == sbt.SBT_E_INVALID
    o.r = 0
    buf = (ctypes.c_float * 64)()
    t = sbt.SbtTensor(sbt.SBT_F32, 0, 4, 4, 4, ctypes.cast(buf, ctypes.c_void_p))
    assert lib.sbt_init(ctypes.byref(t), 3, ctypes.byref(o), ctypes.byref(h)) == sbt.SBT_E_INVALID
    o.r = 2
    assert lib.sbt_init(ctypes.byref(t), 40, ctypes.byref(o), ctypes.byref(h)) == sbt.SBT_E_INVALID
    assert lib.sbt_update(None, ctypes.byref(t)) == sbt.SBT_E_INVALID
    assert b"null" in lib.sbt_last_error()


@pytest.mark.parametrize("field,value", [("mode3_pass", 2), ("als_groups", -1), ("als_groups", 65),
                                         ("warm_start", 3), ("refine_sweeps", -1), ("check_every", 0)])
def test_invalid_options_rejected_without_gpu(lib, field, value):
    """Each option's range is checked before any device call (check_every 0
    is valid: the default poll interval)."""
    from paper_1709_00668_gb300 import sbt
    h = ctypes.c_void_p()
    buf = (ctypes.c_float * 64)()
    t = sbt.SbtTensor(sbt.SBT_F32, 0, 4, 4, 4, ctypes.cast(buf, ctypes.c_void_p))
    o = sbt.sbt_default_options()
    setattr(o, field, value)
    rc = lib.sbt_init(ctypes.byref(t), 3, ctypes.byref(o), ctypes.byref(h))
    if field == "check_every":
        assert rc != sbt.SBT_E_INVALID or b"check_every" not in lib.sbt_last_error()
    else:
        assert rc == sbt.SBT_E_INVALID, (field, rc)
        assert field.encode() in lib.sbt_last_error()


def test_core_consistency_rejects_bad_arguments_without_gpu(lib):
    from paper_1709_00668_gb300 import sbt
    cc = ctypes.c_double()
    buf = (ctypes.c_double * 64)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert lib.sbt_core_consistency(sbt.SBT_F64, None, 4, 4, 4, 4, p, p, p, p, 2, ctypes.byref(cc),
                                    None) == sbt.SBT_E_INVALID
    assert lib.sbt_core_consistency(sbt.SBT_BF16, p, 4, 4, 4, 4, p, p, p, p, 2, ctypes.byref(cc),
                                    None) == sbt.SBT_E_INVALID
    assert lib.sbt_core_consistency(sbt.SBT_F64, p, 4, 4, 4, 4, p, p, p, p, 0, ctypes.byref(cc),
                                    None) == sbt.SBT_E_INVALID
    assert lib.sbt_core_consistency(sbt.SBT_F64, p, 1, 4, 4, 4, p, p, p, p, 2, ctypes.byref(cc),
                                    None) == sbt.SBT_E_SHAPE


def test_recompute_rejects_bad_arguments_without_gpu(lib):
    from paper_1709_00668_gb300 import sbt
    f = ctypes.c_double()
    assert lib.sbt_recompute(None, 10, 1e-6, 0, None, None, None, None, ctypes.byref(f)) == sbt.SBT_E_INVALID


def test_package_import_does_not_need_the_library():
    import importlib
    m = importlib.import_module("paper_1709_00668_gb300")
    assert hasattr(m, "__all__")


def test_server_host_logic_without_gpu(lib):
    """The serving loop's bookkeeping: unknown streams and tickets are
    rejected, counters start at zero, destroy joins the workers."""
    from paper_1709_00668_gb300 import sbt
    o = sbt.SbtServerOptions()
    assert lib.sbt_server_default_options(ctypes.byref(o)) == sbt.SBT_OK
    assert (o.slots, o.mem_budget, o.device) == (4, 0, -1)
    o.slots, o.mem_budget, o.device = 3, 1 << 30, 0
    srv = ctypes.c_void_p()
    assert lib.sbt_server_create(ctypes.byref(o), ctypes.byref(srv)) == sbt.SBT_OK
    buf = (ctypes.c_float * 16)()
    t = sbt.SbtTensor(sbt.SBT_F32, 0, 2, 2, 4, ctypes.cast(buf, ctypes.c_void_p))
    ticket = ctypes.c_uint64()
    assert lib.sbt_server_submit(srv, 7, ctypes.byref(t), ctypes.byref(ticket)) == sbt.SBT_E_INVALID
    t0 = sbt.SbtTensor(sbt.SBT_F32, 0, 2, 2, 0, ctypes.cast(buf, ctypes.c_void_p))
    assert lib.sbt_server_submit(srv, 7, ctypes.byref(t0), ctypes.byref(ticket)) == sbt.SBT_E_SHAPE
    res = sbt.SbtRequestResult()
    assert lib.sbt_server_wait(srv, 12345, 0, ctypes.byref(res)) == sbt.SBT_E_INVALID
    ctx = ctypes.c_void_p()
    assert lib.sbt_server_stream_ctx(srv, 1, ctypes.byref(ctx)) == sbt.SBT_E_INVALID
    assert lib.sbt_server_close_stream(srv, 1) == sbt.SBT_E_INVALID
    # a store larger than the budget is refused before anything is allocated
    big = sbt.SbtTensor(sbt.SBT_F32, 0, 4096, 4096, 64, ctypes.cast(buf, ctypes.c_void_p))
    so = sbt.sbt_default_options(K_capacity=128)
    sid = ctypes.c_int32()
    assert lib.sbt_server_open_stream(srv, ctypes.byref(big), 3, ctypes.byref(so),
                                      ctypes.byref(sid)) == sbt.SBT_E_NOMEM
    st = sbt.SbtServingStats()
    assert lib.sbt_server_stats(srv, ctypes.byref(st)) == sbt.SBT_OK
    assert (st.submitted, st.completed, st.queued, st.in_flight, st.streams, st.resident_bytes) == (0,) * 6
    assert st.mem_budget == 1 << 30
    assert lib.sbt_server_stats_reset(srv) == sbt.SBT_OK
    lib.sbt_server_destroy(srv)
    slots_bad = sbt.SbtServerOptions(65, 1, 0)
    assert lib.sbt_server_create(ctypes.byref(slots_bad), ctypes.byref(srv)) == sbt.SBT_E_INVALID


def test_tile_table_host_logic(lib):
    """The MTTKRP tile table: merge, read back, replace by key, reject bad
    choices, clear (host only)."""
    from paper_1709_00668_gb300 import sbt
    sbt.tile_table_clear()
    assert sbt.tile_table() == []
    e1 = dict(fp8=0, R=10, NP=200, NC=200, Kp_bucket=6, nrep=8, epi=0, ctas_per_sm=1, stages=6)
    e2 = dict(e1, epi=1, ctas_per_sm=2, stages=0)
    sbt.tile_table_merge([e1, e2])
    got = sbt.tile_table()
    assert len(got) == 2 and e1 in got and e2 in got
    sbt.tile_table_merge([dict(e1, stages=3)])
    got = sbt.tile_table()
    assert len(got) == 2 and dict(e1, stages=3) in got
    with pytest.raises(sbt.SbtError):
        sbt.tile_table_merge([dict(e1, ctas_per_sm=3)])
    with pytest.raises(sbt.SbtError):
        sbt.tile_table_merge([dict(e1, stages=9)])
    n = ctypes.c_int32()
    assert lib.sbt_tile_table(7, None, 0, ctypes.byref(n)) == sbt.SBT_E_INVALID
    sbt.tile_table_clear()
    assert sbt.tile_table() == []


def test_nmode_and_get_rank_arguments_rejected_without_gpu(lib):
    """The order-N calls and the GetRank options check their arguments
    before any device call."""
    from paper_1709_00668_gb300 import sbt
    h = ctypes.c_void_p()
    buf = (ctypes.c_double * 4096)()
    dims = (ctypes.c_int64 * sbt.SBT_NMODE_MAX)(6, 5, 4, 3, 0, 0, 0, 0)
    o = sbt.sbt_default_options(prec="f64")
    lam = (ctypes.c_double * 2)(1.0, 1.0)
    U = (ctypes.c_void_p * 4)(*([ctypes.cast(buf, ctypes.c_void_p)] * 4))
    t2 = sbt.SbtTensorN(sbt.SBT_F64, 0, 2, dims, ctypes.cast(buf, ctypes.c_void_p))  # N below 3
    assert lib.sbt_nmode_init_factors(ctypes.byref(t2), 2, lam, U, ctypes.byref(o), ctypes.byref(h)) == \
        sbt.SBT_E_INVALID
    t4 = sbt.SbtTensorN(sbt.SBT_F64, 0, 4, dims, ctypes.cast(buf, ctypes.c_void_p))
    assert lib.sbt_nmode_init_factors(ctypes.byref(t4), 2, lam, None, ctypes.byref(o), ctypes.byref(h)) == \
        sbt.SBT_E_INVALID
    o32 = sbt.sbt_default_options(prec="f32")  # a float32 summary needs a float32 tensor
    assert lib.sbt_nmode_init_factors(ctypes.byref(t4), 2, lam, U, ctypes.byref(o32), ctypes.byref(h)) == \
        sbt.SBT_E_INVALID
    ow = sbt.sbt_default_options(prec="f64", warm_start=1)
    assert lib.sbt_nmode_init_factors(ctypes.byref(t4), 2, lam, U, ctypes.byref(ow), ctypes.byref(h)) == \
        sbt.SBT_E_INVALID
    assert lib.sbt_nmode_update(None, ctypes.byref(t4)) == sbt.SBT_E_INVALID
    # GetRank: float8 summaries, refinement and out-of-range trial counts are rejected
    t = sbt.SbtTensor(sbt.SBT_F32, 0, 4, 4, 4, ctypes.cast(buf, ctypes.c_void_p))
    for kw in (dict(get_rank=1, prec="fp8"), dict(get_rank=1, prec="bf16", refine_sweeps=2),
               dict(get_rank=2), dict(get_rank=1, get_rank_trials=17)):
        og = sbt.sbt_default_options(**kw)
        assert lib.sbt_init(ctypes.byref(t), 3, ctypes.byref(og), ctypes.byref(h)) == sbt.SBT_E_INVALID


def test_persistent_and_batch_options_rejected_without_gpu(lib):
    """persistent_als and the server's batch_als take 0 or 1, checked before
    any device call."""
    from paper_1709_00668_gb300 import sbt
    h = ctypes.c_void_p()
    buf = (ctypes.c_double * 64)()
    t = sbt.SbtTensor(sbt.SBT_F32, 0, 4, 4, 4, ctypes.cast(buf, ctypes.c_void_p))
    o = sbt.sbt_default_options(persistent_als=2)
    assert lib.sbt_init(ctypes.byref(t), 3, ctypes.byref(o), ctypes.byref(h)) == sbt.SBT_E_INVALID
    so = sbt.SbtServerOptions()
    assert lib.sbt_server_default_options(ctypes.byref(so)) == sbt.SBT_OK
    assert so.batch_als == 0
    so.batch_als = 3
    srv = ctypes.c_void_p()
    assert lib.sbt_server_create(ctypes.byref(so), ctypes.byref(srv)) == sbt.SBT_E_INVALID
