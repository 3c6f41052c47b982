"""FP64 CPU oracle of SamBaTen's batch-incremental CP update (arxiv 1709.00668).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA path: the integer sampling primitives live in `oracle/sampling.c`,
everything else is plain numpy/scipy in float64, written as the paper's steps
in the paper's order.

Section map (paper arxiv 1709.00668):
  * Eq. 1 (Section 3.1, "Sample")      -> marginals()
  * Section 3.1 + Algorithm 1 step 3   -> sample_sizes(), sample_mode() (oracle/sampling.c)
  * Section 3.1 + Algorithm 1 step 4   -> summary()
  * Algorithm 1 step 5, Section 3.1 "Decompose" (ALS, Kolda & Bader 2009)
                                       -> init_factors(), mttkrp(), cp_als()
  * Algorithm 1 step 6, Section 3.1 "Project back" (shared-row normalisation)
                                       -> normalize_shared()
  * Lemma 1 + Algorithm 1 step 7       -> match()
  * Section 3.1 "Project back" relation + Algorithm 1 steps 8-10
                                       -> project_back()
  * Algorithm 1 steps 12-13            -> commit inside update()
  * Section 2.2 problem statement      -> init_decomposition(), update()
  * Section 4.2 relative error         -> full_fit()
  * Bro & Kiers 2003 (cited, Section 3.2) core consistency, FMS (Section 4.4)
                                       -> core_consistency(), fms() (test utilities)

Readings where the paper is silent or ambiguous (each is restated in the
repository's design notes):
  R1  sampling weights are the marginals of the tensor before the update;
  R2  weighted sampling without replacement = successive sampling through
      exponential keys (oracle/sampling.c);
  R3  sample size ceil(N/s), clamped to the number of positive weights;
  R4  the time-mode sample is drawn from the old slices, the new slices are
      always appended whole;
  R5  summary ALS starts from Philox uniforms keyed by the global index;
  R6  ALS normalises every column to unit 2-norm after each mode update and
      stops when |fit - fit_prev| < tol (or at max_iters);
  R7  C' is normalised over the shared old rows only;
  R8  matching maximises the sum over components of |G1|*|G2|*|G3| (cosine
      matrices of the three modes) with the Hungarian method;
  R9  new rows of C and zero-entry fills are least-squares projections of the
      summary component onto the matched old component (signs carried);
  R10 old entries are updated only where they are exactly 0, to the mean of
      the proposing repetitions;
  R11 lambda is kept (lambda_mode 0) or averaged with the summary estimate
      (lambda_mode 1, the literal reading of Algorithm 1 step 13);
  R12 all repetitions anchor on the pre-update factors.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field, replace

import numpy as np
import scipy.linalg
import scipy.optimize

from . import csampling

DOMAIN_SAMPLE = 1
DOMAIN_INIT = 2
DOMAIN_GETRANK = 3
INIT_BATCH = 0xFFFFFFFF  # batch number used by the initial decomposition

FLAG_CHOL_REGULARIZED = 1
FLAG_ZERO_COLUMN = 2
FLAG_SAMPLE_LT_RANK = 4


@dataclass
class Options:
    s_I: int = 2
    s_J: int = 2
    s_K: int = 2
    r: int = 4
    tol: float = 1e-6
    max_iters: int = 50
    max_iters_init: int = 50
    seed: int = 0
    stream_id: int = 0
    lambda_mode: int = 0
    fixed_iters: bool = False
    prec: str = "f64"          # values the summary ALS sees: f64 | f32 | bf16 | fp8
    refine_sweeps: int = 0     # bf16 only: ALS iterations on the split summary after the bf16 ALS
    warm_start: bool = False   # start the summary ALS from the old factors at the sampled rows
    get_rank: bool = False     # Section 3.2: estimate R_new per summary (Algorithm 2) and match R_new components
    get_rank_trials: int = 2   # Algorithm 2's `it`: decompositions per candidate rank
    get_rank_threshold: float = 90.0  # CorConDia a candidate rank must reach


@dataclass
class State:
    X: np.ndarray              # (K, I, J) stored slices, float32 or float64
    A: np.ndarray              # (I, R) float64
    B: np.ndarray              # (J, R)
    C: np.ndarray              # (K, R)
    lam: np.ndarray            # (R,)
    S: int                     # fixed-point shift of the marginals
    xa: np.ndarray             # (I,) uint64
    xb: np.ndarray             # (J,) uint64
    xc: np.ndarray             # (K,) uint64
    batch: int
    opts: Options = field(default_factory=Options)

    @property
    def K(self) -> int:
        return self.X.shape[0]

    @property
    def R(self) -> int:
        return self.A.shape[1]


# --------------------------------------------------------------------------
# Eq. 1: measure of importance, as exact fixed-point integers
# --------------------------------------------------------------------------
def marginal_shift(X0: np.ndarray) -> int:
    """S such that M*M*2^S lies in [2^31, 2^32), M = max |x| over X0."""
    M = float(np.max(np.abs(X0))) if X0.size else 0.0
    if M == 0.0:
        return 0
    m2 = np.float64(M) * np.float64(M)
    _, e = math.frexp(float(m2))
    return 32 - e


def quantized_squares(X: np.ndarray, S: int) -> np.ndarray:
    """q(x) = floor((x*x) * 2^S) as uint64: one rounded float64 product, exact scaling."""
    x = X.astype(np.float64)
    sq = np.ldexp(x * x, S)
    if np.any(sq >= 2.0 ** 64):
        raise OverflowError("quantised square exceeds 64 bits")
    return np.floor(sq).astype(np.uint64)


def marginals(X: np.ndarray, S: int):
    """Eq. 1 for all three modes: x_a(i) = sum_{j,k} X(i,j,k)^2 (and x_b, x_c).

    X is slice-major (K, I, J).  Returns uint64 (x_a, x_b, x_c).  Integer sums
    are exact, so slices are processed in blocks to bound memory."""
    K, I, J = X.shape
    xa = np.zeros(I, np.uint64)
    xb = np.zeros(J, np.uint64)
    xc = np.zeros(K, np.uint64)
    step = max(1, (1 << 24) // max(1, I * J))
    for k0 in range(0, K, step):
        q = quantized_squares(X[k0:k0 + step], S)
        xa += q.sum(axis=(0, 2), dtype=np.uint64)
        xb += q.sum(axis=(0, 1), dtype=np.uint64)
        xc[k0:k0 + step] = q.sum(axis=(1, 2), dtype=np.uint64)
    return xa, xb, xc


# --------------------------------------------------------------------------
# Section 3.1 / Algorithm 1 step 3: weighted sampling without replacement
# --------------------------------------------------------------------------
def sample_size(N_old: int, s: int, w: np.ndarray) -> int:
    """|I_s| = N/s (rounded up), clamped to the number of positive weights."""
    return int(min(-(-int(N_old) // int(s)), int(np.count_nonzero(w))))


def sample_mode(w, n, opts: Options, mode: int, rep: int, batch: int) -> np.ndarray:
    return csampling.sample_mode(w, n, opts.seed, opts.stream_id, mode, rep, batch)


# --------------------------------------------------------------------------
# Algorithm 1 step 4: the summary X(I_s, J_s, K_s U [K+1 .. K+K_new])
# --------------------------------------------------------------------------
def summary(X_all: np.ndarray, Is: np.ndarray, Js: np.ndarray, Kprime: np.ndarray) -> np.ndarray:
    """Sub-tensor at the sampled indices, slice-major (len(K'), len(I_s), len(J_s))."""
    return X_all[np.ix_(Kprime, Is, Js)]


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even); returns float64."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def split_bf16(Xs: np.ndarray) -> np.ndarray:
    """hi + lo with hi = bf16(x) and lo = bf16(x - hi), x as float32 (the
    difference is exact in float32); returns float64.  |x - (hi + lo)| is at
    most one half unit in the last place of lo: about 2^-17 |x|."""
    x = np.ascontiguousarray(Xs, dtype=np.float32)
    hi = bf16_round(x)
    lo = bf16_round((x - hi.astype(np.float32)).astype(np.float32))
    return hi + lo


E4M3_MAX = 448.0


def e4m3_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to float8 e4m3 (the finite variant: 4 exponent
    bits with bias 7, 3 mantissa bits, largest value 448, subnormals spaced
    2^-9 below 2^-6), to nearest with ties to even, saturating at +-448;
    returns float64."""
    v = np.asarray(x, dtype=np.float32).astype(np.float64)
    a = np.abs(v)
    _, ex = np.frexp(a)                                  # a = m 2^ex, m in [0.5, 1)
    binade = np.maximum(np.where(a > 0, ex - 1, -6), -6)  # below 2^-6 the spacing stays 2^-9
    ulp = np.ldexp(1.0, binade - 3)
    q = np.minimum(np.rint(a / ulp) * ulp, E4M3_MAX)
    return np.copysign(q, v)


def slice_amax(X: np.ndarray) -> np.ndarray:
    """max |x| of every stored slice (float32 values)."""
    return np.max(np.abs(X.astype(np.float32)).reshape(X.shape[0], -1), axis=1).astype(np.float32)


def fp8_summary_values(Xs: np.ndarray, amax: np.ndarray) -> np.ndarray:
    """e4m3 codes with one scale per summary slice: in float32, inv = 448 /
    amax and q = e4m3(x * inv); the value is q * (amax / 448).  amax[kk] is
    the max |x| of the stored slice behind summary slice kk (0: all zero)."""
    x = np.ascontiguousarray(Xs, dtype=np.float32)
    amax = np.asarray(amax, dtype=np.float32)
    pos = amax > 0
    inv = np.where(pos, np.float32(E4M3_MAX) / np.where(pos, amax, np.float32(1)), np.float32(0)).astype(np.float32)
    scale = (amax / np.float32(E4M3_MAX)).astype(np.float32)
    q = e4m3_round((x * inv[:, None, None]).astype(np.float32))
    return q * scale.astype(np.float64)[:, None, None]


def summary_values(Xs: np.ndarray, prec: str) -> np.ndarray:
    """The values the summary ALS computes with, as float64."""
    if prec == "bf16":
        return bf16_round(Xs.astype(np.float32))
    if prec == "f32":
        return Xs.astype(np.float32).astype(np.float64)
    return Xs.astype(np.float64)


# --------------------------------------------------------------------------
# Algorithm 1 step 5: CP(X_s, R) by alternating least squares
# --------------------------------------------------------------------------
def init_factor(global_idx: np.ndarray, R: int, mode: int, rep: int, batch: int,
                opts: Options, trial: int = -1) -> np.ndarray:
    """U(x, r) = (Philox word 0 >> 8) * 2^-24 with counter (x, r | mode<<8 | rep<<12, batch, 2);
    GetRank's trial t (>= 0) uses (x, r | mode<<8 | rep<<12 | t<<20, batch, 3)."""
    gi = np.asarray(global_idx, dtype=np.uint64)
    n = gi.shape[0]
    ctr = np.zeros((n, R, 4), np.uint32)
    ctr[:, :, 0] = gi[:, None].astype(np.uint32)
    ctr[:, :, 1] = (np.arange(R, dtype=np.uint32)[None, :] | np.uint32(mode << 8)
                    | np.uint32((rep << 12) & 0xFFFFFFFF) | np.uint32((max(trial, 0) << 20) & 0xFFFFFFFF))
    ctr[:, :, 2] = np.uint32(batch & 0xFFFFFFFF)
    ctr[:, :, 3] = DOMAIN_INIT if trial < 0 else DOMAIN_GETRANK
    key = [opts.seed & 0xFFFFFFFF, ((opts.seed >> 32) & 0xFFFFFFFF) ^ (opts.stream_id & 0xFFFFFFFF)]
    out = csampling.philox4x32_10(ctr.reshape(-1, 4), key)
    return np.ldexp((out[:, 0] >> 8).astype(np.float64), -24).reshape(n, R)


def mttkrp(X: np.ndarray, U, mode: int) -> np.ndarray:
    """Matricised tensor times Khatri-Rao product, by its definition.

    X is slice-major (K, I, J) = X(i, j, k) at [k, i, j]; U = [A, B, C].
      mode 0: M(i,r) = sum_{j,k} X(i,j,k) B(j,r) C(k,r)
      mode 1: M(j,r) = sum_{i,k} X(i,j,k) A(i,r) C(k,r)
      mode 2: M(k,r) = sum_{i,j} X(i,j,k) A(i,r) B(j,r)
    """
    A, B, C = U
    if mode == 0:
        return np.einsum("kij,jr,kr->ir", X, B, C, optimize=True)
    if mode == 1:
        return np.einsum("kij,ir,kr->jr", X, A, C, optimize=True)
    return np.einsum("kij,ir,jr->kr", X, A, B, optimize=True)


def solve_normal(M: np.ndarray, V: np.ndarray):
    """U = M V^{-1} for symmetric positive (semi)definite V via Cholesky.

    If the factorisation fails, V + 1e-12 tr(V)/R I is used and a flag is raised."""
    R = V.shape[0]
    flags = 0
    try:
        cf = scipy.linalg.cho_factor(V, lower=True, check_finite=False)
        if not np.all(np.isfinite(cf[0])):
            raise np.linalg.LinAlgError
    except (np.linalg.LinAlgError, scipy.linalg.LinAlgError):
        flags |= FLAG_CHOL_REGULARIZED
        Vr = V + (1e-12 * np.trace(V) / R) * np.eye(R)
        cf = scipy.linalg.cho_factor(Vr, lower=True, check_finite=False)
    U = scipy.linalg.cho_solve(cf, M.T, check_finite=False).T
    return U, flags


@dataclass
class ALSResult:
    U: list
    lam: np.ndarray
    iters: int
    fit: float
    flags: int


def cp_als(X: np.ndarray, U0, tol: float, max_iters: int, fixed_iters: bool = False) -> ALSResult:
    """CP-ALS (Kolda & Bader 2009) from the given starting factors.

    Per iteration, for modes 1, 2, 3 in turn: M = MTTKRP, V = Hadamard product
    of the other two Grams, U_n = M V^{-1}, lambda = column 2-norms, U_n /=
    lambda.  After mode 3: fit = 1 - ||X - X_hat|| / ||X|| from
    ||X||^2 + lambda^T (G1*G2*G3) lambda - 2 sum_r lambda_r <M3(:,r), U3(:,r)>;
    stop when |fit - fit_prev| < tol unless fixed_iters."""
    U = [np.array(u, dtype=np.float64, copy=True) for u in U0]
    R = U[0].shape[1]
    normX2 = float(np.sum(X * X))
    normX = math.sqrt(normX2)
    G = [u.T @ u for u in U]
    lam = np.ones(R)
    fit_prev = 0.0
    fit = 0.0
    flags = 0
    it = 0
    for it in range(1, max_iters + 1):
        M = None
        for n in range(3):
            M = mttkrp(X, U, n)
            V = np.ones((R, R))
            for m in range(3):
                if m != n:
                    V = V * G[m]
            Un, f = solve_normal(M, V)
            flags |= f
            lam = np.sqrt(np.sum(Un * Un, axis=0))
            if np.any(lam == 0.0):
                flags |= FLAG_ZERO_COLUMN
                lam = np.where(lam == 0.0, 1.0, lam)
            U[n] = Un / lam
            G[n] = U[n].T @ U[n]
        inner = float(np.sum(lam * np.sum(M * U[2], axis=0)))
        normXhat2 = float(lam @ (G[0] * G[1] * G[2]) @ lam)
        resid2 = max(normX2 + normXhat2 - 2.0 * inner, 0.0)
        fit = 1.0 - math.sqrt(resid2) / normX if normX > 0 else 0.0
        if not fixed_iters and abs(fit - fit_prev) < tol:
            break
        fit_prev = fit
    return ALSResult(U=U, lam=lam, iters=it, fit=fit, flags=flags)


# --------------------------------------------------------------------------
# Algorithm 1 step 6: normalise over the rows shared with the old factors
# --------------------------------------------------------------------------
def normalize_shared(U, lam, nK: int):
    """Unit 2-norm of each column over the shared rows (all rows of A', B';
    the first nK rows of C'), scale absorbed into lambda."""
    out = []
    lam = lam.copy()
    flags = 0
    for n, u in enumerate(U):
        rows = u[:nK] if n == 2 else u
        nu = np.sqrt(np.sum(rows * rows, axis=0))
        if np.any(nu == 0.0):
            flags |= FLAG_ZERO_COLUMN
            nu = np.where(nu == 0.0, 1.0, nu)
        out.append(u / nu)
        lam = lam * nu
    return out, lam, flags


# --------------------------------------------------------------------------
# Lemma 1 + Algorithm 1 step 7: match summary components to old components
# --------------------------------------------------------------------------
@dataclass
class Match:
    perm: np.ndarray           # perm[r'] = old component matched to summary component r'
    gamma: list                # Gamma_n (R x R): cosine of summary col r' with old col r
    norms: list                # N_n(r) = ||U_old(S_n, r)||
    score: np.ndarray          # |G1| * |G2| * |G3|


def match(Us, anchors) -> Match:
    """Us: normalised summary factors over the shared rows; anchors: the old
    factors at the sampled rows (A_old(I_s), B_old(J_s), C_old(K_s)).  The old
    columns are normalised to unit norm; by Lemma 1 the inner product of
    matching unit columns is 1 in the noiseless case."""
    gam, norms = [], []
    for u, a in zip(Us, anchors):
        N = np.sqrt(np.sum(a * a, axis=0))
        Ns = np.where(N == 0.0, 1.0, N)
        gam.append(u.T @ (a / Ns))
        norms.append(N)
    score = np.abs(gam[0]) * np.abs(gam[1]) * np.abs(gam[2])
    rows, cols = scipy.optimize.linear_sum_assignment(score, maximize=True)
    perm = np.empty(score.shape[0], np.int64)
    perm[rows] = cols
    return Match(perm=perm, gamma=gam, norms=norms, score=score)


# --------------------------------------------------------------------------
# Section 3.1 "Project back" relation + Algorithm 1 steps 8-10
# --------------------------------------------------------------------------
def project_coef(mt: Match, lam_s, lam_old, skip_mode: int) -> np.ndarray:
    """coef(r') = lam'_{r'} prod_{m != skip} Gamma_m(r', r) / (lam_r prod_{m != skip} N_m(r)),
    r = perm[r']: the least-squares scale that carries a summary column of mode
    `skip_mode` into the matched old component's scale."""
    R = lam_s.shape[0]
    coef = np.zeros(R)
    for rp in range(R):
        r = mt.perm[rp]
        num = lam_s[rp]
        den = lam_old[r]
        for m in range(3):
            if m != skip_mode:
                num *= mt.gamma[m][rp, r]
                den *= mt.norms[m][r]
        coef[rp] = num / den if den != 0.0 else 0.0
    return coef


def project_back(Us_full, lam_s, lam_old, mt: Match, nK: int, K_new: int,
                 old_rows, sampled):
    """Returns (C_new in old scale (K_new x R_old), zero-fill proposals per
    mode: dict {(row, r): value} for old entries that are exactly 0, the
    summary's estimate of lambda, and the mask of old components matched).
    With GetRank the summary has R_new <= R_old components; old components
    no summary component matched get no new rows from this repetition."""
    R = lam_s.shape[0]
    R_old = lam_old.shape[0]
    c3 = project_coef(mt, lam_s, lam_old, 2)
    Cnew = np.zeros((K_new, R_old))
    matched = np.zeros(R_old, bool)
    for rp in range(R):
        Cnew[:, mt.perm[rp]] = c3[rp] * Us_full[2][nK:nK + K_new, rp]
        matched[mt.perm[rp]] = True
    props = []
    for n in range(3):
        cn = project_coef(mt, lam_s, lam_old, n)
        rows = sampled[n]
        d = {}
        for t, x in enumerate(rows):
            for rp in range(R):
                r = mt.perm[rp]
                if old_rows[n][t, r] == 0.0:
                    d[(int(x), int(r))] = cn[rp] * Us_full[n][t, rp]
        props.append(d)
    lam_est = np.zeros(R_old)
    for rp in range(R):
        r = mt.perm[rp]
        den = mt.norms[0][r] * mt.norms[1][r] * mt.norms[2][r]
        lam_est[r] = (lam_s[rp] * mt.gamma[0][rp, r] * mt.gamma[1][rp, r]
                      * mt.gamma[2][rp, r] / den) if den != 0.0 else 0.0
    return Cnew, props, lam_est, matched


# --------------------------------------------------------------------------
# Section 2.2: the pre-existing decomposition, and Algorithm 1 as a whole
# --------------------------------------------------------------------------
def canonicalize(U, lam):
    """Sort components by lambda (descending, stable) and fix signs so that
    sum A(:,r) >= 0 and sum B(:,r) >= 0, pushing signs into C."""
    order = np.argsort(-lam, kind="stable")
    A, B, C = (u[:, order].copy() for u in U)
    lam = lam[order].copy()
    for r in range(A.shape[1]):
        if A[:, r].sum() < 0:
            A[:, r] *= -1.0
            C[:, r] *= -1.0
        if B[:, r].sum() < 0:
            B[:, r] *= -1.0
            C[:, r] *= -1.0
    return A, B, C, lam


def init_state_from_factors(X0: np.ndarray, lam, A, B, C, opts: Options) -> State:
    """State for a given pre-existing decomposition of X0 (Section 2.2, (a))."""
    S = marginal_shift(X0)
    xa, xb, xc = marginals(X0, S)
    return State(X=np.array(X0, copy=True), A=np.array(A, np.float64), B=np.array(B, np.float64),
                 C=np.array(C, np.float64), lam=np.array(lam, np.float64), S=S,
                 xa=xa, xb=xb, xc=xc, batch=0, opts=replace(opts))


def init_decomposition(X0: np.ndarray, R: int, opts: Options):
    """CP-ALS of the initial tensor from Philox-uniform factors (batch 0xFFFFFFFF),
    then canonical order and signs.  Returns (State, ALSResult)."""
    K0, I, J = X0.shape
    U0 = [init_factor(np.arange(I), R, 0, 0, INIT_BATCH, opts),
          init_factor(np.arange(J), R, 1, 0, INIT_BATCH, opts),
          init_factor(np.arange(K0), R, 2, 0, INIT_BATCH, opts)]
    Xv = X0.astype(np.float64)
    res = cp_als(Xv, U0, opts.tol, opts.max_iters_init, opts.fixed_iters)
    A, B, C, lam = canonicalize(res.U, res.lam)
    return init_state_from_factors(X0, lam, A, B, C, opts), res


def get_rank(X: np.ndarray, R_max: int, idx, opts: Options, rep: int, batch: int):
    """Algorithm 2 (GetRank): for every candidate rank i = 1..R_max and trial
    j = 1..it, a CP decomposition of X at rank i (from trial j's start) and its
    CorConDia p(i, j).  The algorithm's last step (sort p, take the top index)
    is read as: R_new = the largest rank whose best trial reaches the
    threshold (CorConDia of a rank-1 model is 100, so the literal top entry
    would always be rank 1); 1 if none does.  idx: the global indices of the
    summary's rows per mode (they key the starts).  Returns (R_new, p)."""
    p = np.zeros((R_max, opts.get_rank_trials))
    for i in range(1, R_max + 1):
        for j in range(opts.get_rank_trials):
            U0 = [init_factor(idx[m], i, m, rep, batch, opts, trial=j) for m in range(3)]
            res = cp_als(X, U0, opts.tol, opts.max_iters, opts.fixed_iters)
            p[i - 1, j] = core_consistency(X, res.lam, res.U[0], res.U[1], res.U[2])
    ok = [i for i in range(1, R_max + 1) if np.max(p[i - 1]) >= opts.get_rank_threshold]
    return (max(ok) if ok else 1), p


@dataclass
class RepTrace:
    Is: np.ndarray
    Js: np.ndarray
    Ks: np.ndarray
    als: ALSResult
    Us: list                   # summary factors after shared-row normalisation
    lam_s: np.ndarray
    match: Match
    Cnew: np.ndarray
    flags: int


def batch_sample_sizes(state: State):
    """Algorithm 1 step 2 on the tensor before the update: the sample sizes
    (n_I, n_J, n_K) of Section 3.1 from the measure of importance."""
    opts = state.opts
    K_old, I, J = state.X.shape
    return (sample_size(I, opts.s_I, state.xa), sample_size(J, opts.s_J, state.xb),
            sample_size(K_old, opts.s_K, state.xc))


def update_rep(state: State, X_all: np.ndarray, sizes, K_new: int, rho: int,
               keep_summaries: bool = False) -> RepTrace:
    """Steps 3-9 of Algorithm 1 for repetition rho: sample, gather the
    summary, CP of the summary, shared-row normalisation, match, project
    back.  X_all holds the K_old stored slices followed by the K_new new ones
    (slice-major); every repetition anchors on the pre-update factors of
    `state`, so repetitions do not depend on one another."""
    opts = state.opts
    nI, nJ, nK = sizes
    K_old = X_all.shape[0] - K_new
    R = state.R
    t_rep = time.perf_counter()
    flags = FLAG_SAMPLE_LT_RANK if min(nI, nJ, nK) < R else 0
    # step 3: sample each mode without replacement
    Is = sample_mode(state.xa, nI, opts, 0, rho, state.batch)
    Js = sample_mode(state.xb, nJ, opts, 1, rho, state.batch)
    Ks = sample_mode(state.xc, nK, opts, 2, rho, state.batch)
    Kp = np.concatenate([Ks.astype(np.int64), np.arange(K_old, K_old + K_new)])
    # step 4: the summary
    if opts.prec == "fp8":
        Xs = fp8_summary_values(summary(X_all, Is, Js, Kp), slice_amax(X_all[Kp]))
    else:
        Xs = summary_values(summary(X_all, Is, Js, Kp), opts.prec)
    # step 5: CP of the summary, from random factors (the paper leaves
    # the start open), or warm: the old factors at the sampled rows, the
    # new slices' rows of C' zero (their first mode-3 update fills them)
    # GetRank (Section 3.2, Algorithm 2): the summary's rank R_new <= R
    R_s, p_rank = R, None
    if opts.get_rank:
        R_s, p_rank = get_rank(Xs, R, (Is, Js, Kp), opts, rho, state.batch)
    if opts.warm_start and not opts.get_rank:
        U0 = [state.A[Is].copy(), state.B[Js].copy(),
              np.concatenate([state.C[Ks], np.zeros((K_new, R))], axis=0)]
    else:
        U0 = [init_factor(Is, R_s, 0, rho, state.batch, opts),
              init_factor(Js, R_s, 1, rho, state.batch, opts),
              init_factor(Kp, R_s, 2, rho, state.batch, opts)]
    res = cp_als(Xs, U0, opts.tol, opts.max_iters, opts.fixed_iters)
    if opts.prec == "bf16" and opts.refine_sweeps > 0:
        # refinement: continue the same ALS from its factors for a fixed
        # number of iterations on the split (hi + lo) summary
        Xr = split_bf16(summary(X_all, Is, Js, Kp))
        ref = cp_als(Xr, res.U, opts.tol, opts.refine_sweeps, fixed_iters=True)
        res = ALSResult(U=ref.U, lam=ref.lam, iters=res.iters, fit=ref.fit, flags=res.flags | ref.flags)
    flags |= res.flags
    # step 6: normalise over shared rows
    Us, lam_s, f = normalize_shared(res.U, res.lam, nK)
    flags |= f
    # step 7: match against the anchors (old factors at the sampled rows)
    old_rows = [state.A[Is], state.B[Js], state.C[Ks]]
    mt = match([Us[0], Us[1], Us[2][:nK]], old_rows)
    # steps 8-9: project back
    Cnew, props, lam_est, matched = project_back(Us, lam_s, state.lam, mt, nK, K_new,
                                                 old_rows, [Is, Js, Ks])
    t = RepTrace(Is=Is, Js=Js, Ks=Ks, als=res, Us=Us, lam_s=lam_s, match=mt, Cnew=Cnew, flags=flags)
    t.props = props
    t.lam_est = lam_est
    t.matched = matched
    t.R_new = R_s
    t.p_rank = p_rank
    if keep_summaries:
        t.Xs = Xs
    t.seconds = time.perf_counter() - t_rep
    return t


def commit(state: State, X_all: np.ndarray, K_new: int, traces) -> State:
    """Steps 10-13 of Algorithm 1: average the repetitions' new rows of C
    (in repetition order), fill zero entries of the old factors with the mean
    of the proposals, keep or average lambda, fold the new slices into the
    measure of importance.  The new State holds X_all as its slices."""
    opts = state.opts
    R = state.R
    # step 10 and 12: average C_new over the repetitions (with GetRank, over
    # those that matched the component; none: zero rows), append to C
    Cnew = np.zeros((K_new, R))
    cnt = np.zeros(R)
    for t in traces:
        Cnew = Cnew + t.Cnew
        cnt = cnt + t.matched
    Cnew = Cnew / np.where(cnt > 0, cnt, 1.0)
    # step 8 (commit): zero entries of the old factors take the mean of the proposals
    A, B, C = state.A.copy(), state.B.copy(), state.C.copy()
    for n, F in enumerate((A, B, C)):
        acc = {}
        for t in traces:
            for key, val in t.props[n].items():
                s, c = acc.get(key, (0.0, 0))
                acc[key] = (s + val, c + 1)
        for (x, r), (s, c) in acc.items():
            F[x, r] = s / c
    lam = state.lam.copy()
    if opts.lambda_mode == 1:
        est = np.zeros(R)
        for t in traces:
            est = est + t.lam_est
        lam = np.where(cnt > 0, 0.5 * (lam + est / np.where(cnt > 0, cnt, 1.0)), lam)
    # fold the new slices into the measure of importance
    qa, qb, qc = marginals(X_all[X_all.shape[0] - K_new:], state.S)
    return State(X=X_all, A=A, B=B, C=np.concatenate([C, Cnew], axis=0), lam=lam, S=state.S,
                 xa=state.xa + qa, xb=state.xb + qb, xc=np.concatenate([state.xc, qc]),
                 batch=state.batch + 1, opts=state.opts)


def update(state: State, X_new: np.ndarray, keep_summaries: bool = False):
    """Algorithm 1 for one batch of new slices X_new (K_new, I, J): step 2
    (sample sizes), steps 3-9 per repetition (update_rep), steps 10-13
    (commit).

    Returns (new State, list of per-repetition traces)."""
    K_old, I, J = state.X.shape
    K_new = X_new.shape[0]
    if X_new.shape[1:] != (I, J) or K_new < 1:
        raise ValueError("bad batch shape")
    if not np.all(np.isfinite(X_new)):
        raise FloatingPointError("non-finite value in the new slices")
    # step 2: the measure of importance of X (the tensor before the update)
    sizes = batch_sample_sizes(state)
    X_all = np.concatenate([state.X, X_new.astype(state.X.dtype)], axis=0)
    traces = [update_rep(state, X_all, sizes, K_new, rho, keep_summaries) for rho in range(state.opts.r)]
    return commit(state, X_all, K_new, traces), traces


# --------------------------------------------------------------------------
# Section 4.2: relative error / fit of the full model
# --------------------------------------------------------------------------
def reconstruct(lam, A, B, C) -> np.ndarray:
    return np.einsum("r,ir,jr,kr->kij", lam, A, B, C, optimize=True)


def full_fit(X: np.ndarray, lam, A, B, C) -> float:
    """1 - ||X - X_hat||_F / ||X||_F, element by element (slice loop)."""
    num = 0.0
    den = 0.0
    for k in range(X.shape[0]):
        Xk = X[k].astype(np.float64)
        Xh = (A * (lam * C[k])) @ B.T
        D = Xk - Xh
        num += float(np.sum(D * D))
        den += float(np.sum(Xk * Xk))
    return 1.0 - math.sqrt(num) / math.sqrt(den)


# --------------------------------------------------------------------------
# Test utilities: core consistency (Bro & Kiers 2003) and FMS (Section 4.4)
# --------------------------------------------------------------------------
def relative_fitness(X: np.ndarray, model, baseline) -> float:
    """Relative Fitness (Section 4.2): ||X - X_model|| / ||X - X_baseline||,
    each model a tuple (lam, A, B, C); the baseline is the decomposition
    recomputed on the whole tensor."""
    ra = np.linalg.norm((X - reconstruct(*model)).ravel())
    rb = np.linalg.norm((X - reconstruct(*baseline)).ravel())
    return float(ra / rb) if rb > 0 else float("inf")


def core_consistency(X: np.ndarray, lam, A, B, C) -> float:
    """100 (1 - ||G - T||^2 / R): G the least-squares Tucker core for the fixed
    CP factors (lambda absorbed into C), T the superdiagonal of ones."""
    R = A.shape[1]
    Cl = C * lam
    Xv = X.astype(np.float64)
    G = np.einsum("kij,ai,bj,ck->abc", Xv, np.linalg.pinv(A), np.linalg.pinv(B),
                  np.linalg.pinv(Cl), optimize=True)
    T = np.zeros((R, R, R))
    for r in range(R):
        T[r, r, r] = 1.0
    return 100.0 * (1.0 - float(np.sum((G - T) ** 2)) / R)


def fms(lam_a, Ua, lam_b, Ub) -> float:
    """Factor match score after the best one-to-one matching:
    (1/R) sum_r (1 - |la - lb| / max(la, lb)) prod_n |a_r^(n)T b_r^(n)|,
    columns scaled to unit norm with the scale folded into lambda."""
    def unit(lam, U):
        lam = np.array(lam, np.float64).copy()
        out = []
        for u in U:
            nrm = np.sqrt(np.sum(u * u, axis=0))
            nrm = np.where(nrm == 0, 1.0, nrm)
            out.append(u / nrm)
            lam = lam * nrm
        return lam, out
    la, ua = unit(lam_a, Ua)
    lb, ub = unit(lam_b, Ub)
    R = la.shape[0]
    cong = np.ones((R, R))
    for x, y in zip(ua, ub):
        cong = cong * np.abs(x.T @ y)
    pen = 1.0 - np.abs(la[:, None] - lb[None, :]) / np.maximum(np.maximum(la[:, None], lb[None, :]), 1e-300)
    score = pen * cong
    rows, cols = scipy.optimize.linear_sum_assignment(score, maximize=True)
    return float(score[rows, cols].sum() / R)
