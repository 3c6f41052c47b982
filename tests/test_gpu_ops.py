"""GPU parity of the device-level operations against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import csampling
from oracle import sambaten as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbt():
    from paper_1709_00668_gb300 import build, sbt as s
    build.build()
    s.lib()
    return s


def test_philox_matches_oracle(sbt):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4099, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    for key in ([0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [0x12345678, 0x9abcdef0]):
        want = csampling.philox4x32_10(ctr, key)
        got = sbt.sbt_philox4x32_10(torch.from_numpy(ctr.view(np.int32)).cuda(), key)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("N,n,zero_every,scale", [
    (1, 1, 0, 1), (7, 3, 0, 1), (200, 50, 7, 1 << 30), (1000, 200, 0, 1 << 40),
    (2000, 400, 13, 3), (4097, 1000, 0, 1 << 50), (5000, 1, 3, 1 << 20), (100, 100, 0, 5),
])
def test_sample_matches_oracle_bit_exact(sbt, N, n, zero_every, scale):
    rng = np.random.default_rng(N + n)
    w = rng.integers(1, max(2, scale), size=N, dtype=np.uint64)
    if zero_every:
        w[::zero_every] = 0
    n = min(n, int(np.count_nonzero(w)))
    for mode, rep, batch, seed in [(0, 0, 0, 0), (2, 5, 9, 123456789123), (1, 63, 0xFFFFFFFF, 7)]:
        want = csampling.sample_mode(w, n, seed, 3, mode, rep, batch)
        got = sbt.sbt_sample(torch.from_numpy(w.view(np.int64)).cuda(), n, seed=seed, stream_id=3,
                             mode=mode, rep=rep, batch=batch)
        assert np.array_equal(got.cpu().numpy(), want), (mode, rep, batch)


def test_sample_equal_weights_and_ties(sbt):
    w = np.full(300, 1 << 33, np.uint64)
    want = csampling.sample_mode(w, 150, 1, 0, 0, 0, 0)
    got = sbt.sbt_sample(torch.from_numpy(w.view(np.int64)).cuda(), 150, seed=1)
    assert np.array_equal(got.cpu().numpy(), want)


def test_sample_rejects_oversize(sbt):
    w = np.array([0, 1, 0, 2], np.uint64)
    with pytest.raises(sbt.SbtError) as e:
        sbt.sbt_sample(torch.from_numpy(w.view(np.int64)).cuda(), 3)
    assert e.value.status == sbt.SBT_E_INVALID


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("K,I,J,R", [(2, 3, 5, 1), (9, 17, 33, 5), (37, 45, 29, 10), (20, 70, 300, 16),
                                     (11, 13, 130, 20), (6, 9, 41, 32), (300, 8, 8, 3)])
def test_mttkrp_matches_oracle(sbt, dtype, K, I, J, R):
    rng = np.random.default_rng(K * I + J + R)
    X = rng.standard_normal((K, I, J))
    U = [rng.standard_normal((I, R)), rng.standard_normal((J, R)), rng.standard_normal((K, R))]
    ld = (J + 7) // 8 * 8
    Xp = np.zeros((K, I, ld))
    Xp[:, :, :J] = X
    Xd = torch.from_numpy(Xp).to(dtype).cuda()
    Ud = [torch.from_numpy(u).to(dtype).cuda() for u in U]
    Xv = Xd[:, :, :J].double().cpu().numpy()
    Uv = [u.double().cpu().numpy() for u in Ud]
    tol = 1e-12 if dtype == torch.float64 else 2e-5
    for mode in range(3):
        want = O.mttkrp(Xv, Uv, mode)
        got = sbt.sbt_mttkrp(Xd, *Ud, mode).double().cpu().numpy()
        scale = np.max(np.abs(want)) + 1e-300
        assert np.max(np.abs(got - want)) / scale < tol, mode


def test_mttkrp_ignores_padding(sbt):
    """Values in the row padding [J, ld) never reach the result (NaN there)."""
    rng = np.random.default_rng(1)
    K, I, J, R = 5, 6, 13, 4
    Xp = np.full((K, I, 16), np.nan)
    Xp[:, :, :J] = rng.standard_normal((K, I, J))
    U = [rng.standard_normal((I, R)), rng.standard_normal((J, R)), rng.standard_normal((K, R))]
    Xd = torch.from_numpy(Xp).float().cuda()
    Ud = [torch.from_numpy(u).float().cuda() for u in U]
    for mode in range(3):
        got = sbt.sbt_mttkrp(Xd, *Ud, mode).cpu().numpy()
        assert np.all(np.isfinite(got))
        want = O.mttkrp(Xd[:, :, :J].double().cpu().numpy(), [u.double().cpu().numpy() for u in Ud], mode)
        assert np.allclose(got, want, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("K,I,J,R", [(3, 5, 7, 1), (9, 130, 70, 10), (24, 200, 200, 10), (7, 256, 64, 16),
                                     (13, 100, 300, 20), (5, 129, 129, 32), (40, 64, 520, 8)])
def test_mttkrp_bf16_tensor_cores_match_oracle(sbt, K, I, J, R):
    """tcgen05 path: bfloat16 X (exact in float64), float32 factors, all three modes."""
    rng = np.random.default_rng(K + I + J + R)
    ld = (J + 7) // 8 * 8
    Xp = torch.zeros(K, I, ld, dtype=torch.bfloat16)
    Xp[:, :, :J] = torch.from_numpy(rng.standard_normal((K, I, J))).to(torch.bfloat16)
    Xd = Xp.cuda()
    U = [torch.from_numpy(rng.standard_normal((n, R))).float().cuda() for n in (I, J, K)]
    Xv = Xp[:, :, :J].double().numpy()
    Uv = [u.double().cpu().numpy() for u in U]
    for mode in range(3):
        want = O.mttkrp(Xv, Uv, mode)
        got = sbt.sbt_mttkrp(Xd, *U, mode).double().cpu().numpy()
        scale = np.max(np.abs(want)) + 1e-300
        # bf16 x (hi + lo) keeps ~2^-16 of each factor; float32 accumulation
        assert np.max(np.abs(got - want)) / scale < 2e-4, mode
