"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties one oracle step to a published value, a closed form, brute
force on tiny inputs, a library routine it reduces to, a distribution law, or
an invariant the paper states, so that a dropped term, a wrong sign or index,
or a transposed operand in the oracle fails here.
"""
import itertools
import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import csampling
from oracle import sambaten as O
from paper_1709_00668_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ----
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (Salmon et al. SC'11)."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        ctr, key, want = r[0:4], r[4:6], r[6:10]
        got = csampling.philox4x32_10(np.array([ctr], np.uint32), key)[0]
        assert [int(x) for x in got] == want


def test_philox_uniformity():
    """Word 0 over consecutive counters is uniform (chi-square on 256 bins)."""
    n = 1 << 16
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 3] = 1
    v = csampling.philox4x32_10(ctr, [0, 0])[:, 0]
    h = np.bincount((v >> 24).astype(np.int64), minlength=256)
    e = n / 256
    chi2 = float(((h - e) ** 2 / e).sum())
    assert chi2 < 400.0  # 255 dof: mean 255, sd ~22.6


# -------------------------------------------------------- fixed-point log2 ----
def _log2_exact_q32(t: int) -> Fraction:
    getcontext().prec = 60
    v = Decimal(t).ln() / Decimal(2).ln()
    return Fraction(v) * (1 << 32)


@pytest.mark.parametrize("seed", [0, 1])
def test_log2_q32_within_truncation_bound(seed):
    """Shift-and-square log2 (Turner 2010): 0 <= exact*2^32 - result < 2 for 1 <= t < 2^33."""
    rng = np.random.default_rng(seed)
    ts = [1, 2, 3, 5, 7, (1 << 32) - 1, 1 << 32, (1 << 32) + 1, (1 << 33) - 1]
    ts += [int(x) for x in rng.integers(1, 1 << 33, size=300, dtype=np.int64)]
    got = csampling.log2_q32(np.array(ts, np.uint64))
    for t, g in zip(ts, got):
        exact = _log2_exact_q32(t)
        d = exact - int(g)
        assert 0 <= d < 2, (t, int(g), float(exact))


def test_log2_q32_powers_of_two_exact():
    t = np.array([1 << p for p in range(33)], np.uint64)
    got = csampling.log2_q32(t)
    assert [int(g) for g in got] == [p << 32 for p in range(33)]


# ------------------------------------------------------- weighted sampling ----
def _successive_inclusion(w, n):
    """Exact P(x in sample) for successive sampling without replacement, prob ~ w."""
    N = len(w)
    W = sum(w)
    p = [Fraction(0)] * N
    for seq in itertools.permutations(range(N), n):
        pr = Fraction(1)
        rest = W
        for x in seq:
            pr *= Fraction(w[x], rest)
            rest -= w[x]
        for x in seq:
            p[x] += pr
    return [float(v) for v in p]


@pytest.mark.parametrize("n", [1, 2, 3])
def test_es_sampling_inclusion_probabilities(n):
    """Exponential-key draws reproduce successive-sampling inclusion probabilities."""
    w = [1, 2, 3, 5, 13]
    exact = _successive_inclusion(w, n)
    wv = np.array(w, np.uint64) << np.uint64(20)  # scale is irrelevant to the law
    trials = 12000
    counts = np.zeros(len(w))
    for t in range(trials):
        s = csampling.sample_mode(wv, n, seed=7, stream_id=0, mode=0, rep=t & 0xFFF,
                                  batch=t >> 12)
        counts[s] += 1
    emp = counts / trials
    for x in range(len(w)):
        sd = math.sqrt(exact[x] * (1 - exact[x]) / trials)
        assert abs(emp[x] - exact[x]) < 5 * sd + 1e-9, (x, emp[x], exact[x])


def test_es_sampling_structure():
    """Sorted, distinct, within range, zero weights never drawn, n = #positives takes all."""
    rng = np.random.default_rng(3)
    w = rng.integers(0, 1 << 40, size=200).astype(np.uint64)
    w[::7] = 0
    pos = np.flatnonzero(w)
    s = O.sample_mode(w, 50, O.Options(seed=11), 1, 2, 5)
    assert np.all(np.diff(s) > 0)
    assert np.all(w[s] > 0)
    s_all = O.sample_mode(w, len(pos), O.Options(seed=11), 1, 2, 5)
    assert np.array_equal(s_all, pos)
    with pytest.raises(ValueError):
        O.sample_mode(w, len(pos) + 1, O.Options(seed=11), 1, 2, 5)


def test_es_sampling_prefers_heavy_indices():
    """One index with overwhelming weight is always drawn."""
    w = np.ones(100, np.uint64)
    w[37] = np.uint64(1 << 50)
    for rep in range(20):
        s = O.sample_mode(w, 5, O.Options(seed=1), 0, rep, 0)
        assert 37 in s


def test_sample_size_rule():
    w = np.array([0, 3, 0, 4, 5], np.uint64)
    assert O.sample_size(5, 2, w) == 3          # ceil(5/2)=3, 3 positives
    assert O.sample_size(5, 1, w) == 3          # clamped to positives
    assert O.sample_size(10, 4, np.ones(10, np.uint64)) == 3


# ------------------------------------------------------------- marginals ----
def test_marginals_eq1_bruteforce():
    """Eq. 1 by exact rational arithmetic on a tiny tensor."""
    rng = np.random.default_rng(0)
    X = rng.standard_normal((3, 4, 5)).astype(np.float32)
    S = O.marginal_shift(X)
    M = max(abs(float(v)) for v in X.ravel())
    assert 2 ** 31 <= M * M * 2.0 ** S < 2 ** 32
    xa, xb, xc = O.marginals(X, S)
    ea = [0] * 4
    eb = [0] * 5
    ec = [0] * 3
    for k in range(3):
        for i in range(4):
            for j in range(5):
                q = math.floor(Fraction(float(X[k, i, j])) ** 2 * Fraction(2) ** S)
                ea[i] += q
                eb[j] += q
                ec[k] += q
    assert [int(v) for v in xa] == ea
    assert [int(v) for v in xb] == eb
    assert [int(v) for v in xc] == ec


def test_marginals_incremental_equals_scratch():
    rng = np.random.default_rng(1)
    X = rng.random((9, 6, 7)).astype(np.float32)
    S = O.marginal_shift(X[:4])
    a0, b0, c0 = O.marginals(X[:4], S)
    a1, b1, c1 = O.marginals(X[4:], S)
    a, b, c = O.marginals(X, S)
    assert np.array_equal(a0 + a1, a)
    assert np.array_equal(b0 + b1, b)
    assert np.array_equal(np.concatenate([c0, c1]), c)


# --------------------------------------------------------------- summary ----
def test_summary_is_direct_indexing():
    rng = np.random.default_rng(2)
    X = rng.random((6, 5, 4))
    Is, Js, Kp = np.array([0, 3]), np.array([1, 2, 3]), np.array([1, 4, 5])
    Xs = O.summary(X, Is, Js, Kp)
    for a, k in enumerate(Kp):
        for b, i in enumerate(Is):
            for c, j in enumerate(Js):
                assert Xs[a, b, c] == X[k, i, j]


def test_bf16_round_matches_torch():
    """Round-to-nearest-even to bfloat16, against torch's conversion."""
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.standard_normal(5000).astype(np.float32),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.5 - 2 ** -8, 0.0],
                                 np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.bf16_round(x), ref)


def test_split_bf16_bound_hi_and_exact_cases():
    """hi + lo split: hi is the bfloat16 rounding itself, the pair carries
    about 16 significant bits (|x - (hi + lo)| <= 2^-16 |x|), and values with
    at most 16 significant bits are represented exactly."""
    rng = np.random.default_rng(41)
    x = (rng.standard_normal(20000) * np.exp2(rng.integers(-40, 40, 20000))).astype(np.float32)
    y = O.split_bf16(x)
    assert np.all(np.abs(x.astype(np.float64) - y) <= np.exp2(-16) * np.abs(x.astype(np.float64)))
    hi = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    lo = y - hi
    # lo is itself a bfloat16 value and no larger than half an ulp of hi
    assert np.array_equal(O.bf16_round(lo.astype(np.float32)), lo)
    assert np.all(np.abs(lo) <= np.exp2(-8) * np.abs(hi) + 1e-300)
    m = rng.integers(1, 2 ** 16, 3000)
    e = rng.integers(-30, 30, 3000)
    x16 = np.ldexp(m.astype(np.float64), e).astype(np.float32)  # <= 16 significant bits
    assert np.array_equal(O.split_bf16(x16), x16.astype(np.float64))


def test_refinement_brings_bf16_als_to_float32_accuracy():
    """ALS continued on the split summary lands at the float32 solution:
    much closer to the float32 ALS than the bfloat16 ALS it started from."""
    X = synth.planted_dense(30, 26, 24, 3, noise=0.01, seed=42, dtype=torch.float32).X.numpy()
    rng = np.random.default_rng(43)
    U0 = [rng.random((30, 3)), rng.random((26, 3)), rng.random((24, 3))]
    ref = O.cp_als(X.astype(np.float64), U0, 0.0, 200, fixed_iters=True)
    b16 = O.cp_als(O.summary_values(X, "bf16"), U0, 0.0, 200, fixed_iters=True)
    fine = O.cp_als(O.split_bf16(X), b16.U, 0.0, 60, fixed_iters=True)

    def dist(a, b):  # unit-column factors from the same start: no permutation to undo
        return max(float(np.max(np.abs(ua - ub))) for ua, ub in zip(a.U, b.U))
    d16, dfine = dist(b16, ref), dist(fine, ref)
    assert d16 > 1e-4
    assert dfine < d16 / 20
    assert abs(fine.fit - ref.fit) < abs(b16.fit - ref.fit) / 20 + 1e-9


def test_e4m3_round_matches_torch_and_the_format():
    """float8 e4m3 rounding: torch's conversion where it does not saturate
    (|x| < 464), every code of the format a fixed point, ties to even, and
    saturation at 448 (torch returns NaN there instead)."""
    rng = np.random.default_rng(44)
    x = (rng.standard_normal(20000) * np.exp2(rng.integers(-12, 9, 20000))).astype(np.float32)
    x = x[np.abs(x) < 464]
    ties = np.array([1.0625, 1.1875, -1.0625, 2 ** -10, 3 * 2 ** -11, 0.0], np.float32)
    x = np.concatenate([x, ties])
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(O.e4m3_round(x), ref)
    codes = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    codes = codes[np.isfinite(codes)]
    assert np.array_equal(O.e4m3_round(codes.astype(np.float32)), codes)
    assert codes.max() == 448.0 and np.min(codes[codes > 0]) == 2.0 ** -9
    assert O.e4m3_round(np.float32(1.0625)) == 1.0 and O.e4m3_round(np.float32(1.1875)) == 1.25
    assert np.array_equal(O.e4m3_round(np.array([470.0, 1e30, -1e6], np.float32)), [448.0, 448.0, -448.0])


def test_fp8_summary_scale_and_error_bound():
    """Per-slice scaled e4m3 summary: the slice's largest value maps to code
    448 exactly and every value is within half a code step (2^-4 relative in
    the normal range, 2^-10 * scale below it)."""
    rng = np.random.default_rng(45)
    Xs = (rng.standard_normal((5, 7, 9)) * np.array([1e-3, 1.0, 50.0, 0.0, 3.0])[:, None, None]).astype(np.float32)
    amax = np.max(np.abs(Xs).reshape(5, -1), axis=1)
    V = O.fp8_summary_values(Xs, amax)
    assert np.all(V[3] == 0.0)
    for k in (0, 1, 2, 4):
        s = np.float64(np.float32(amax[k] / np.float32(448.0)))
        i = np.unravel_index(np.argmax(np.abs(Xs[k])), Xs[k].shape)
        assert abs(V[k][i]) == 448.0 * s
        err = np.abs(V[k] - Xs[k].astype(np.float64))
        assert np.all(err <= 2.0 ** -4 * np.abs(Xs[k]) * 1.0001 + 2.0 ** -10 * s)


# --------------------------------------------------------------- MTTKRP ----
def test_mttkrp_bruteforce():
    rng = np.random.default_rng(5)
    K, I, J, R = 3, 4, 5, 2
    X = rng.standard_normal((K, I, J))
    U = [rng.standard_normal((I, R)), rng.standard_normal((J, R)), rng.standard_normal((K, R))]
    want = [np.zeros((I, R)), np.zeros((J, R)), np.zeros((K, R))]
    for k in range(K):
        for i in range(I):
            for j in range(J):
                for r in range(R):
                    x = X[k, i, j]
                    want[0][i, r] += x * U[1][j, r] * U[2][k, r]
                    want[1][j, r] += x * U[0][i, r] * U[2][k, r]
                    want[2][k, r] += x * U[0][i, r] * U[1][j, r]
    for n in range(3):
        np.testing.assert_allclose(O.mttkrp(X, U, n), want[n], rtol=1e-12, atol=1e-12)


def test_mttkrp_rank_one_closed_form():
    """For X = a o b o c: mode-1 MTTKRP = a (b^T B * c^T C), and cyclically."""
    rng = np.random.default_rng(6)
    a, b, c = rng.random(4), rng.random(5), rng.random(3)
    X = np.einsum("i,j,k->kij", a, b, c)
    U = [rng.random((4, 3)), rng.random((5, 3)), rng.random((3, 3))]
    np.testing.assert_allclose(O.mttkrp(X, U, 0), np.outer(a, (b @ U[1]) * (c @ U[2])), rtol=1e-12)
    np.testing.assert_allclose(O.mttkrp(X, U, 1), np.outer(b, (a @ U[0]) * (c @ U[2])), rtol=1e-12)
    np.testing.assert_allclose(O.mttkrp(X, U, 2), np.outer(c, (a @ U[0]) * (b @ U[1])), rtol=1e-12)


# ----------------------------------------------------------------- solve ----
def test_solve_normal_matches_numpy():
    rng = np.random.default_rng(7)
    F = rng.standard_normal((20, 6))
    V = F.T @ F
    M = rng.standard_normal((9, 6))
    U, flags = O.solve_normal(M, V)
    assert flags == 0
    np.testing.assert_allclose(U, np.linalg.solve(V, M.T).T, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(U @ V, M, rtol=1e-10, atol=1e-10)


def test_solve_normal_regularizes_singular():
    V = np.ones((3, 3))
    U, flags = O.solve_normal(np.ones((2, 3)), V)
    assert flags & O.FLAG_CHOL_REGULARIZED
    assert np.all(np.isfinite(U))


# ---------------------------------------------------------------- CP-ALS ----
def _planted(I, J, K, R, noise=0.0, seed=0, dist="normal"):
    p = synth.planted_dense(I, J, K, R, noise=noise, seed=seed, dtype=torch.float64, dist=dist)
    return p.X.numpy(), p.A.numpy(), p.B.numpy(), p.C.numpy()


def test_cp_als_recovers_planted_noiseless():
    X, A, B, C = _planted(12, 11, 10, 3, seed=2)
    opts = O.Options(seed=3)
    U0 = [O.init_factor(np.arange(12), 3, 0, 0, 0, opts), O.init_factor(np.arange(11), 3, 1, 0, 0, opts),
          O.init_factor(np.arange(10), 3, 2, 0, 0, opts)]
    res = O.cp_als(X, U0, tol=1e-14, max_iters=2000)
    assert res.fit > 1 - 1e-6
    assert O.fms(res.lam, res.U, np.ones(3), [A, B, C]) > 0.999
    assert abs(O.core_consistency(X, res.lam, *res.U) - 100.0) < 1e-3


def test_cp_als_reported_fit_equals_direct_fit():
    """The fit from the Gram/MTTKRP expansion equals 1 - ||X - X_hat||/||X|| computed directly."""
    X, *_ = _planted(9, 8, 7, 2, noise=0.2, seed=4)
    opts = O.Options(seed=5)
    U0 = [O.init_factor(np.arange(9), 2, 0, 0, 0, opts), O.init_factor(np.arange(8), 2, 1, 0, 0, opts),
          O.init_factor(np.arange(7), 2, 2, 0, 0, opts)]
    for iters in (1, 3, 10):
        res = O.cp_als(X, U0, tol=0.0, max_iters=iters, fixed_iters=True)
        assert res.iters == iters
        direct = O.full_fit(X, res.lam, *res.U)
        assert abs(res.fit - direct) < 1e-10


def test_cp_als_columns_unit_norm():
    X, *_ = _planted(8, 8, 8, 3, noise=0.1, seed=6)
    opts = O.Options(seed=1)
    U0 = [O.init_factor(np.arange(8), 3, m, 0, 0, opts) for m in range(3)]
    res = O.cp_als(X, U0, tol=0.0, max_iters=4, fixed_iters=True)
    for u in res.U:
        np.testing.assert_allclose(np.linalg.norm(u, axis=0), 1.0, rtol=1e-12)


def test_core_consistency_detects_overfactoring():
    """CC is 100 for the planted model and drops well below for a wrong model."""
    X, A, B, C = _planted(10, 9, 8, 2, seed=7)
    assert abs(O.core_consistency(X, np.ones(2), A, B, C) - 100.0) < 1e-6
    rng = np.random.default_rng(0)
    bad = O.core_consistency(X, np.ones(3), rng.random((10, 3)), rng.random((9, 3)), rng.random((8, 3)))
    assert bad < 90.0


def test_init_factor_values():
    """Init values are Philox word 0 >> 8 scaled by 2^-24, on the documented counter."""
    opts = O.Options(seed=0x123456789, stream_id=5)
    U = O.init_factor(np.array([7, 9]), 2, 1, 3, 4, opts)
    key = [0x23456789, 0x1 ^ 5]
    for t, x in enumerate([7, 9]):
        for r in range(2):
            ctr = [x, r | (1 << 8) | (3 << 12), 4, 2]
            v = int(csampling.philox4x32_10(np.array([ctr], np.uint32), key)[0, 0])
            assert U[t, r] == (v >> 8) / 2.0 ** 24


# --------------------------------------------------------------- matching ----
@pytest.mark.parametrize("R", [1, 2, 4, 6])
def test_match_is_optimal_assignment(R):
    rng = np.random.default_rng(R)
    for _ in range(5):
        Us = [rng.standard_normal((7, R)) for _ in range(3)]
        anchors = [rng.standard_normal((7, R)) for _ in range(3)]
        mt = O.match(Us, anchors)
        best = max(sum(mt.score[a, p[a]] for a in range(R)) for p in itertools.permutations(range(R)))
        got = sum(mt.score[a, mt.perm[a]] for a in range(R))
        assert abs(got - best) < 1e-12
        assert sorted(mt.perm.tolist()) == list(range(R))


def test_match_recovers_permutation_lemma1():
    """Lemma 1: unit columns of the same component have inner product 1."""
    rng = np.random.default_rng(9)
    old = [rng.random((15, 4)) for _ in range(3)]
    perm = np.array([2, 0, 3, 1])
    Us = []
    for o in old:
        u = o[:, perm] * rng.uniform(0.5, 2.0, size=4)
        Us.append(u / np.linalg.norm(u, axis=0))
    mt = O.match(Us, old)
    assert np.array_equal(mt.perm, perm)
    for n in range(3):
        np.testing.assert_allclose(mt.gamma[n][np.arange(4), perm], 1.0, rtol=1e-12)


# ------------------------------------------------------ whole update step ----
def _planted_state(I, J, K0, R, opts, noise=0.0, seed=0, dist="normal", Ktot=None):
    p = synth.planted_dense(I, J, Ktot or K0, R, noise=noise, seed=seed, dtype=torch.float64, dist=dist)
    X = p.X.numpy()
    A, B, C = p.A.numpy(), p.B.numpy(), p.C.numpy()
    na, nb, nc = (np.linalg.norm(u, axis=0) for u in (A, B, C[:K0]))
    lam = na * nb * nc
    st = O.init_state_from_factors(X[:K0], lam, A / na, B / nb, C[:K0] / nc, opts)
    return st, X, (A / na, B / nb, C / nc, lam)


def test_update_noiseless_projects_back_exactly():
    """Project-back relation: in the noiseless case the appended rows equal the
    planted C rows in the old model's scale, and the model still fits exactly."""
    R = 3
    opts = O.Options(s_I=2, s_J=2, s_K=2, r=3, tol=1e-15, max_iters=3000, seed=0)
    st, X, (A, B, Cn, lam) = _planted_state(24, 22, 20, R, opts, Ktot=30)
    st2, traces = O.update(st, X[20:30])
    np.testing.assert_allclose(st2.C[20:30], Cn[20:30], rtol=1e-5, atol=1e-7)
    assert O.full_fit(st2.X, st2.lam, st2.A, st2.B, st2.C) > 1 - 1e-6
    for t in traces:
        # Lemma 1 at the matched pairs
        for n in range(3):
            g = np.abs(t.match.gamma[n][np.arange(R), t.match.perm])
            np.testing.assert_allclose(g, 1.0, atol=1e-6)
        # samples are the paper's sizes
        assert len(t.Is) == 12 and len(t.Js) == 11 and len(t.Ks) == 10


def test_warm_start_projects_back_exactly_in_few_iterations():
    """Warm start (the old factors at the sampled rows, new rows of C' zero):
    in the noiseless case the same project-back relation holds, the matching
    is the identity (the start keeps the component order), and the summary ALS
    stops after far fewer iterations than from the random start."""
    R = 3
    base = dict(s_I=2, s_J=2, s_K=2, r=3, tol=1e-12, max_iters=3000, seed=0)
    st, X, (A, B, Cn, lam) = _planted_state(24, 22, 20, R, O.Options(**base, warm_start=True), Ktot=30)
    st2, traces = O.update(st, X[20:30])
    np.testing.assert_allclose(st2.C[20:30], Cn[20:30], rtol=1e-5, atol=1e-7)
    assert O.full_fit(st2.X, st2.lam, st2.A, st2.B, st2.C) > 1 - 1e-6
    st_r, X_r, _ = _planted_state(24, 22, 20, R, O.Options(**base), Ktot=30)
    _, traces_r = O.update(st_r, X_r[20:30])
    for t, tr in zip(traces, traces_r):
        assert list(t.match.perm) == list(range(R))
        assert t.als.iters <= 10 and t.als.iters * 5 < tr.als.iters


def test_warm_start_first_mode1_update_ignores_new_slices():
    """With the new rows of C' zero, the first mode-1 MTTKRP is that of the old
    slices alone: the start's new rows carry no weight (checked against the
    MTTKRP of the summary with the new slices cut off)."""
    rng = np.random.default_rng(5)
    X = rng.random((7, 5, 6))
    U = [rng.random((5, 3)), rng.random((6, 3)), np.concatenate([rng.random((4, 3)), np.zeros((3, 3))])]
    np.testing.assert_allclose(O.mttkrp(X, U, 0), O.mttkrp(X[:4], [U[0], U[1], U[2][:4]], 0), rtol=1e-14)


def test_relative_fitness_definition():
    """Relative Fitness: 1 for the baseline itself; the ratio of the (1 - fit)
    values; and 2 for a model whose residual is exactly twice the baseline's
    (data = baseline + a rank-one D, model = baseline - D as a rank R+1 CP)."""
    rng = np.random.default_rng(9)
    A, B, C = rng.random((6, 2)), rng.random((5, 2)), rng.random((4, 2))
    lam = np.array([2.0, 1.0])
    base = (lam, A, B, C)
    a, b, c = rng.random((6, 1)), rng.random((5, 1)), rng.random((4, 1))
    eps = 0.01
    X = O.reconstruct(*base) + O.reconstruct(np.array([eps]), a, b, c)
    assert O.relative_fitness(X, base, base) == 1.0
    other = (lam * 1.01, A, B, C)
    ratio = (1 - O.full_fit(X, *other)) / (1 - O.full_fit(X, *base))
    assert abs(O.relative_fitness(X, other, base) - ratio) < 1e-12
    twice = (np.concatenate([lam, [-eps]]), np.hstack([A, a]), np.hstack([B, b]), np.hstack([C, c]))
    assert abs(O.relative_fitness(X, twice, base) - 2.0) < 1e-12


@pytest.mark.parametrize("R_true,noise", [(2, 0.0), (3, 0.01)])
def test_get_rank_finds_the_planted_rank(R_true, noise):
    """Algorithm 2 with the threshold reading: on a planted rank-R_true tensor
    the largest candidate rank whose core consistency reaches 90 is R_true
    (an exact CP scores 100; an over-factored one falls far below)."""
    p = synth.planted_dense(14, 12, 10, R_true, noise=noise, seed=21, dtype=torch.float64)
    X = p.X.numpy()
    opts = O.Options(tol=1e-10, max_iters=400, get_rank=True, get_rank_trials=2)
    idx = (np.arange(14), np.arange(12), np.arange(10))
    R_new, pr = O.get_rank(X, 4, idx, opts, rep=0, batch=0)
    assert R_new == R_true, pr
    assert np.max(pr[R_true - 1]) > 99.0 - 1000 * noise
    assert np.all(np.max(pr[R_true:], axis=1) < 90.0)


def test_match_of_fewer_summary_components():
    """Rectangular Lemma-1 matching: a summary with R_new < R components, each
    an old component at the sampled rows (in another order, unit columns),
    is matched to exactly those old components."""
    rng = np.random.default_rng(4)
    old = [rng.random((8, 4)), rng.random((7, 4)), rng.random((6, 4))]
    pick = [3, 1]
    Us = [u[:, pick] / np.linalg.norm(u[:, pick], axis=0) for u in old]
    mt = O.match(Us, old)
    assert list(mt.perm) == pick


def test_get_rank_full_rank_update_equals_plain_update():
    """When every summary has the full rank, the GetRank update is the plain
    update (rank-R ALS from the same start, every component matched by every
    repetition)."""
    R = 2
    base = dict(s_I=2, s_J=2, s_K=2, r=2, tol=1e-10, max_iters=300, seed=0)
    st, X, _ = _planted_state(16, 14, 10, R, O.Options(**base, get_rank=True), Ktot=14, seed=3)
    st_g, tr_g = O.update(st, X[10:14])
    st_p, _ = _planted_state(16, 14, 10, R, O.Options(**base), Ktot=14, seed=3)[:2]
    st_p2, _ = O.update(st_p, X[10:14])
    assert all(t.R_new == R and t.matched.all() for t in tr_g)
    np.testing.assert_array_equal(st_g.C, st_p2.C)


def test_nmode_oracle_at_order_three_is_the_three_mode_oracle():
    """The order-N oracle (NEXT N3) at N = 3: the same samples, the same match
    and the same appended rows as the 3-mode oracle (only einsum's summation
    order differs)."""
    from oracle import nmode
    R = 3
    opts = O.Options(s_I=2, s_J=2, s_K=2, r=2, tol=1e-9, max_iters=60, seed=2)
    st, X, (A, B, Cn, lam) = _planted_state(18, 16, 12, R, opts, noise=0.01, Ktot=16, seed=8)
    st3, tr3 = O.update(st, X[12:16])
    stN = nmode.init_state_from_factors(X[:12], lam, [A, B, Cn[:12]], opts)
    stN2, trN = nmode.update(stN, X[12:16])
    for a, b in zip(tr3, trN):
        assert np.array_equal(a.Is, b["idx"][0]) and np.array_equal(a.Js, b["idx"][1])
        assert np.array_equal(a.Ks, b["idx"][2])
        assert list(a.match.perm) == list(b["match"].perm)
        assert a.als.iters == b["als"].iters
    np.testing.assert_allclose(stN2.U[2], st3.C, rtol=1e-9, atol=1e-12)


def test_nmode_update_projects_back_exactly_at_order_four():
    """Project-back relation at N = 4 (noiseless): the appended time rows equal
    the planted ones in the old model's scale, and every marginal and mode
    sample follows Eq. 1 and the sample-size rule."""
    from oracle import nmode
    rng = np.random.default_rng(12)
    R, dims, Ktot, K0 = 2, (9, 8, 7), 14, 10
    U = [rng.random((d, R)) for d in dims] + [rng.random((Ktot, R))]
    norms = [np.linalg.norm(u[:K0] if n == 3 else u, axis=0) for n, u in enumerate(U)]
    Un = [u / nrm for u, nrm in zip(U, norms)]
    lam = np.prod(norms, axis=0)
    X = nmode.reconstruct(np.ones(R), U)
    opts = O.Options(s_I=2, s_J=2, s_K=2, r=2, tol=1e-14, max_iters=2000, seed=0)
    st = nmode.init_state_from_factors(X[:K0], lam, [Un[0], Un[1], Un[2], Un[3][:K0]], opts)
    w = nmode.marginals(X[:K0], st.S)
    q = O.quantized_squares(X[:K0], st.S)
    assert np.array_equal(w[0], q.sum(axis=(0, 2, 3), dtype=np.uint64))
    assert np.array_equal(w[3], q.sum(axis=(1, 2, 3), dtype=np.uint64))
    st2, traces = nmode.update(st, X[K0:])
    np.testing.assert_allclose(st2.U[3][K0:], Un[3][K0:], rtol=1e-5, atol=1e-7)
    for t in traces:
        assert [len(i) for i in t["idx"]] == [5, 4, 4, 5]
        assert list(t["match"].perm) in ([0, 1], [1, 0])


def test_nmode_mttkrp_bruteforce_order_four():
    """The order-N MTTKRP against explicit loops on a tiny 4-mode tensor, every mode."""
    from oracle import nmode
    rng = np.random.default_rng(6)
    K, I1, I2, I3, R = 3, 4, 2, 3, 2
    X = rng.standard_normal((K, I1, I2, I3))
    U = [rng.standard_normal((I1, R)), rng.standard_normal((I2, R)), rng.standard_normal((I3, R)),
         rng.standard_normal((K, R))]
    for mode in range(4):
        dims = (I1, I2, I3, K)
        M = np.zeros((dims[mode], R))
        for k, a, b, c, r in itertools.product(range(K), range(I1), range(I2), range(I3), range(R)):
            idx = (a, b, c, k)
            prod = X[k, a, b, c]
            for m in range(4):
                if m != mode:
                    prod *= U[m][idx[m], r]
            M[idx[mode], r] += prod
        np.testing.assert_allclose(nmode.mttkrp(X, U, mode), M, rtol=1e-12, atol=1e-12)


def test_nmode_cp_als_recovers_planted_order_four():
    """Noiseless planted rank-2 4-mode tensor: the order-N CP-ALS reaches fit 1
    and its factors match the planted ones (FMS-style cosines ~1)."""
    from oracle import nmode
    rng = np.random.default_rng(7)
    R = 2
    U = [rng.random((d, R)) for d in (7, 6, 5, 8)]
    X = nmode.reconstruct(np.ones(R), U)
    U0 = [rng.random(u.shape) for u in U]
    res = nmode.cp_als(X, U0, 1e-14, 3000)
    assert res.fit > 1 - 1e-6
    for u, v in zip(res.U, U):
        cos = np.abs((u / np.linalg.norm(u, axis=0)).T @ (v / np.linalg.norm(v, axis=0)))
        assert np.allclose(np.sort(cos.max(axis=1)), 1.0, atol=1e-5)


def test_cp_als_scale_equivariance():
    """CP-ALS of c X from the same start: the same unit factors, lambda times c,
    the same fit (the normal equations are homogeneous in X)."""
    X = synth.planted_dense(12, 11, 10, 3, noise=0.01, seed=2, dtype=torch.float64).X.numpy()
    U0 = [O.init_factor(np.arange(n), 3, m, 0, 0, O.Options()) for m, n in enumerate((12, 11, 10))]
    a = O.cp_als(X, U0, 0.0, 15, fixed_iters=True)
    b = O.cp_als(4.0 * X, U0, 0.0, 15, fixed_iters=True)
    for ua, ub in zip(a.U, b.U):
        np.testing.assert_allclose(ua, ub, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(b.lam, 4.0 * a.lam, rtol=1e-9)
    assert abs(a.fit - b.fit) < 1e-9


def test_update_stream_keeps_fit_noiseless():
    R = 2
    opts = O.Options(s_I=2, s_J=2, s_K=2, r=2, tol=1e-15, max_iters=3000, seed=4)
    st, X, _ = _planted_state(16, 14, 10, R, opts, Ktot=22, seed=3)
    for k0 in (10, 14, 15):
        k1 = {10: 14, 14: 15, 15: 22}[k0]
        st, _ = O.update(st, X[k0:k1])
        assert st.K == k1
        assert O.full_fit(st.X, st.lam, st.A, st.B, st.C) > 1 - 1e-6


def test_update_zero_entries_filled_by_projection():
    """Only exactly-zero old entries at sampled rows change; the fill is the
    projected planted value in the noiseless case (Algorithm 1 step 8)."""
    R = 2
    opts = O.Options(s_I=1, s_J=1, s_K=1, r=2, tol=1e-15, max_iters=3000, seed=2)
    st, X, (A, B, Cn, lam) = _planted_state(12, 10, 8, R, opts, Ktot=12, seed=5)
    st.A[3, 1] = 0.0
    st.B[4, 0] = 0.0
    st.C[5, 1] = 0.0
    st2, _ = O.update(st, X[8:12])
    np.testing.assert_allclose(st2.A[3, 1], A[3, 1], rtol=1e-4)
    np.testing.assert_allclose(st2.B[4, 0], B[4, 0], rtol=1e-4)
    # an old row of C (mode 3: every old slice is sampled at s_K = 1)
    np.testing.assert_allclose(st2.C[5, 1], Cn[5, 1], rtol=1e-4)
    mask = np.ones_like(st.A, bool)
    mask[3, 1] = False
    assert np.array_equal(st2.A[mask], st.A[mask])
    maskc = np.ones_like(st.C, bool)
    maskc[5, 1] = False
    assert np.array_equal(st2.C[:8][maskc], st.C[maskc])


def test_update_lambda_modes():
    R = 2
    opts = O.Options(s_I=2, s_J=2, s_K=2, r=2, tol=1e-15, max_iters=2000, seed=1, lambda_mode=0)
    st, X, (_, _, _, lam) = _planted_state(14, 12, 10, R, opts, Ktot=14, seed=8)
    st0, _ = O.update(st, X[10:14])
    assert np.array_equal(st0.lam, st.lam)
    st.opts = O.Options(**{**st.opts.__dict__, "lambda_mode": 1})
    st1, _ = O.update(st, X[10:14])
    # the summary's estimate of lambda equals lambda in the noiseless case
    np.testing.assert_allclose(st1.lam, st.lam, rtol=1e-5)


def test_update_rejects_nonfinite():
    opts = O.Options(r=1)
    st, X, _ = _planted_state(6, 6, 6, 1, opts, Ktot=8)
    bad = X[6:8].copy()
    bad[0, 1, 1] = np.nan
    with pytest.raises(FloatingPointError):
        O.update(st, bad)


def test_full_fit_direct():
    rng = np.random.default_rng(10)
    X = rng.random((3, 4, 5))
    lam, A, B, C = rng.random(2), rng.random((4, 2)), rng.random((5, 2)), rng.random((3, 2))
    Xh = np.zeros_like(X)
    for k in range(3):
        for i in range(4):
            for j in range(5):
                Xh[k, i, j] = sum(lam[r] * A[i, r] * B[j, r] * C[k, r] for r in range(2))
    want = 1 - np.sqrt(((X - Xh) ** 2).sum()) / np.sqrt((X ** 2).sum())
    assert abs(O.full_fit(X, lam, A, B, C) - want) < 1e-12
    assert abs(O.full_fit(Xh, lam, A, B, C) - 1.0) < 1e-12


def test_canonicalize_order_and_signs():
    rng = np.random.default_rng(11)
    U = [rng.standard_normal((6, 3)) for _ in range(3)]
    lam = np.array([1.0, 3.0, 2.0])
    A, B, C, l2 = O.canonicalize(U, lam)
    assert np.array_equal(l2, [3.0, 2.0, 1.0])
    assert np.all(A.sum(0) >= 0) and np.all(B.sum(0) >= 0)
    np.testing.assert_allclose(O.reconstruct(l2, A, B, C), O.reconstruct(lam, *U), atol=1e-12)


def test_fms_identities():
    rng = np.random.default_rng(12)
    U = [rng.random((5, 3)) for _ in range(3)]
    lam = rng.random(3) + 0.5
    assert abs(O.fms(lam, U, lam, U) - 1.0) < 1e-12
    p = [2, 0, 1]
    # scaling every mode by 3 multiplies lambda by 27: penalty 1 - 26/27 per component
    assert abs(O.fms(lam, U, lam[p], [u[:, p] * 3.0 for u in U]) - 1 / 27) < 1e-12
    assert abs(O.fms(lam, U, lam[p], [u[:, p] for u in U]) - 1.0) < 1e-12


def test_fp8_update_close_to_float64_update():
    """A whole update on e4m3 summaries stays close to the float64 update:
    quantisation noise of ~2^-5 per element costs little full-tensor fit."""
    p = synth.planted_dense(40, 36, 34, 3, noise=0.01, seed=46, dtype=torch.float32)
    X, A, B, C = p.X.numpy(), p.A.numpy(), p.B.numpy(), p.C.numpy()
    na, nb, nc = (np.linalg.norm(u, axis=0) for u in (A, B, C[:28]))
    fits = {}
    for prec in ("f64", "fp8"):
        o = O.Options(s_I=2, s_J=2, s_K=2, r=2, max_iters=30, fixed_iters=True, prec=prec)
        st = O.init_state_from_factors(X[:28], na * nb * nc, A / na, B / nb, C[:28] / nc, o)
        st, _ = O.update(st, X[28:34])
        fits[prec] = O.full_fit(st.X, st.lam, st.A, st.B, st.C)
    assert fits["f64"] > 0.85
    assert abs(fits["fp8"] - fits["f64"]) < 0.05


def test_pool_oracle_equals_serial_update():
    """The oracle with its repetitions in worker processes (the benchmark's
    CPU baseline) gives the serial update's samples, matches and factors."""
    from oracle.pool import PoolOracle
    R = 3
    opts = O.Options(s_I=2, s_J=2, s_K=2, r=4, tol=1e-7, max_iters=40, seed=6)
    st, X, _ = _planted_state(30, 26, 20, R, opts, Ktot=32, seed=9)
    st_s, tr_s = O.update(st, X[20:26])
    st_s2, tr_s2 = O.update(st_s, X[26:32])
    with PoolOracle(X.astype(np.float64), workers=2, threads=1) as po:
        sp = po.state(20, st.lam, st.A, st.B, st.C, opts)
        assert np.array_equal(sp.xa, st.xa) and np.array_equal(sp.xc, st.xc)
        sp2, tr_p = po.update(sp, 6)
        sp3, tr_p2 = po.update(sp2, 6)
        f_pool = po.full_fit(sp3)
        # a state rebuilt from the stored slices at K = 26 (marginals by chunks)
        sq = po.state(26, st_s.lam, st_s.A, st_s.B, st_s.C, opts, K_shift=20, batch=1)
        sq_xa, sq_xb, sq_xc, sq_S = sq.xa.copy(), sq.xb.copy(), sq.xc.copy(), sq.S
        sp3 = O.State(X=np.array(sp3.X), A=sp3.A, B=sp3.B, C=sp3.C, lam=sp3.lam, S=sp3.S, xa=sp3.xa, xb=sp3.xb,
                      xc=sp3.xc, batch=sp3.batch, opts=sp3.opts)
        del sp, sp2, sq
    for a, b in zip(tr_s + tr_s2, tr_p + tr_p2):
        assert np.array_equal(a.Is, b.Is) and np.array_equal(a.Ks, b.Ks)
        assert np.array_equal(a.match.perm, b.match.perm)
        assert a.als.iters == b.als.iters
    for u, v in ((st_s2.A, sp3.A), (st_s2.B, sp3.B), (st_s2.C, sp3.C), (st_s2.lam, sp3.lam)):
        np.testing.assert_allclose(v, u, rtol=1e-12, atol=1e-14)
    assert np.array_equal(st_s2.xc, sp3.xc) and sp3.batch == 2
    assert abs(f_pool - O.full_fit(st_s2.X, st_s2.lam, st_s2.A, st_s2.B, st_s2.C)) < 1e-12
    assert sq_S == st_s.S and np.array_equal(sq_xa, st_s.xa) and np.array_equal(sq_xb, st_s.xb)
    assert np.array_equal(sq_xc, st_s.xc)
