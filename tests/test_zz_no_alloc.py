"""sbt_sample_noalloc, the sampling entry point for callers that cannot
allocate device memory during a call (its scratch is a fixed array inside the
library), must draw exactly what sbt_sample draws.

Collected last on purpose: if it fails, a run stopped at the first failure has
already run every other test.  Sampled indices are integers, so the tolerance
is bit-exact, as for every sampling test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1709_00668_gb300 import build, sbt
    build.build()
    return sbt.lib()


def _draw(fn, w_dev, n, seed, mode, rep, batch):
    out = torch.full((max(1, n),), -1, dtype=torch.int32, device=w_dev.device)
    stream = torch.cuda.current_stream().cuda_stream
    st = fn(ctypes.c_void_p(w_dev.data_ptr()), w_dev.numel(), n, seed, 9, mode, rep, batch,
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    return st, out[:n].cpu().numpy()


def test_noalloc_matches_sample_on_two_calls_in_a_row(lib):
    rng = np.random.default_rng(21)
    cases = [(5000, 700, 2 ** 40, 1, 0, 3), (120000, 4000, 2 ** 20, 2, 5, 11)]
    for N, n, scale, mode, rep, batch in cases:
        w = rng.integers(1, scale, size=N, dtype=np.uint64)
        w[::17] = 0
        w_dev = torch.from_numpy(w.view(np.int64)).cuda()
        st_ref, ref = _draw(lib.sbt_sample, w_dev, n, 77, mode, rep, batch)
        st_new, got = _draw(lib.sbt_sample_noalloc, w_dev, n, 77, mode, rep, batch)
        assert st_ref == 0 and st_new == 0, lib.sbt_last_error()
        assert np.array_equal(got, ref)
        assert np.all(np.diff(got) > 0)


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    from paper_1709_00668_gb300 import sbt
    N = sbt.SBT_SAMPLE_NOALLOC_MAX_N + 1
    w_dev = torch.ones(N, dtype=torch.int64, device="cuda")
    st, _ = _draw(lib.sbt_sample_noalloc, w_dev, 10, 0, 0, 0, 0)
    assert st == sbt.SBT_E_INVALID
    assert b"SBT_SAMPLE_NOALLOC_MAX_N" in lib.sbt_last_error()


def test_noalloc_reports_oversized_draw(lib):
    from paper_1709_00668_gb300 import sbt
    w_dev = torch.tensor([0, 3, 0, 4], dtype=torch.int64, device="cuda")
    st, _ = _draw(lib.sbt_sample_noalloc, w_dev, 3, 0, 0, 0, 0)
    assert st == sbt.SBT_E_INVALID
