"""Order-N SamBaTen (plain FP64 CPU oracle): Algorithm 1 for a tensor with
N >= 3 modes, one of which (the last factor, the first array axis) grows
with time.  Section 2.2 states that the problem and the method extend to any
number of modes; the steps are those of the 3-mode oracle (`sambaten.py`)
with every "three modes" replaced by "all modes":

  Eq. 1 marginals for every mode; each non-time mode and the old time slices
  sampled by the same exponential keys (Philox counter mode index = the
  mode's position, the time mode last); the summary at the sampled indices
  plus the new slices; CP-ALS over all N modes; shared-row normalisation;
  Lemma 1 matching with the product of the N |cosine| matrices; the
  project-back scale over the N-1 modes other than the one being placed.

Test infrastructure only (see `sambaten.py`).  Layout: X[k, i_1, ..., i_{N-1}]
(time first), factors U = [U_1, ..., U_{N-1}, C].  For N = 3 every function
reduces to the 3-mode oracle's, which the tests check value for value.
"""
from __future__ import annotations

import math
import string
from dataclasses import dataclass, field, replace

import numpy as np
import scipy.optimize

from . import sambaten as O

_LETTERS = string.ascii_lowercase


def _axes(N: int):
    """einsum letters: array axes (time first) and the matching factor order
    (non-time modes, then time)."""
    ltr = _LETTERS[:N]  # ltr[0] = time axis, ltr[1..] = modes 1..N-1
    factor_ax = [ltr[n + 1] for n in range(N - 1)] + [ltr[0]]
    return ltr, factor_ax


@dataclass
class StateN:
    X: np.ndarray              # (K, I_1, ..., I_{N-1})
    U: list                    # [U_1, ..., U_{N-1}, C], float64
    lam: np.ndarray
    S: int
    w: list                    # uint64 marginals per factor (same order as U)
    batch: int
    opts: O.Options = field(default_factory=O.Options)

    @property
    def N(self) -> int:
        return self.X.ndim


def marginals(X: np.ndarray, S: int):
    """Eq. 1 for every mode: w_n(i) = sum over all other indices of q(x);
    returned in factor order (non-time modes, then time)."""
    q = O.quantized_squares(X, S)
    N = X.ndim
    out = []
    for n in range(N - 1):
        ax = n + 1
        out.append(q.sum(axis=tuple(a for a in range(N) if a != ax), dtype=np.uint64))
    out.append(q.sum(axis=tuple(range(1, N)), dtype=np.uint64))
    return out


def mttkrp(X: np.ndarray, U, mode: int) -> np.ndarray:
    """M(x, r) = sum over the other indices of X times the product of the other
    factors' entries, by its definition (an einsum over all modes)."""
    N = X.ndim
    ltr, fax = _axes(N)
    ops, subs = [X], [ltr]
    for m in range(N):
        if m != mode:
            ops.append(U[m])
            subs.append(fax[m] + "z")
    return np.einsum(",".join(subs) + "->" + fax[mode] + "z", *ops, optimize=True)


def cp_als(X: np.ndarray, U0, tol: float, max_iters: int, fixed_iters: bool = False) -> O.ALSResult:
    """CP-ALS over all N modes in turn (Kolda & Bader 2009), as the 3-mode
    cp_als: U_n = M V^{-1} with V the Hadamard product of the other Grams,
    unit columns, fit after the last mode from ||X||^2 + lam^T (*G) lam -
    2 sum_r lam_r <M_last(:, r), U_last(:, r)>."""
    U = [np.array(u, dtype=np.float64, copy=True) for u in U0]
    N = len(U)
    R = U[0].shape[1]
    normX2 = float(np.sum(X.astype(np.float64) ** 2))
    normX = math.sqrt(normX2)
    G = [u.T @ u for u in U]
    lam = np.ones(R)
    fit_prev = fit = 0.0
    flags = 0
    it = 0
    for it in range(1, max_iters + 1):
        M = None
        for n in range(N):
            M = mttkrp(X, U, n)
            V = np.ones((R, R))
            for m in range(N):
                if m != n:
                    V = V * G[m]
            Un, f = O.solve_normal(M, V)
            flags |= f
            lam = np.sqrt(np.sum(Un * Un, axis=0))
            if np.any(lam == 0.0):
                flags |= O.FLAG_ZERO_COLUMN
                lam = np.where(lam == 0.0, 1.0, lam)
            U[n] = Un / lam
            G[n] = U[n].T @ U[n]
        inner = float(np.sum(lam * np.sum(M * U[N - 1], axis=0)))
        H = np.ones((R, R))
        for g in G:
            H = H * g
        resid2 = max(normX2 + float(lam @ H @ lam) - 2.0 * inner, 0.0)
        fit = 1.0 - math.sqrt(resid2) / normX if normX > 0 else 0.0
        if not fixed_iters and abs(fit - fit_prev) < tol:
            break
        fit_prev = fit
    return O.ALSResult(U=U, lam=lam, iters=it, fit=fit, flags=flags)


def normalize_shared(U, lam, nK: int):
    """Unit columns over the shared rows: all rows of the non-time factors,
    the first nK rows of C'; the scale goes into lambda."""
    out, lam, flags = [], lam.copy(), 0
    N = len(U)
    for n, u in enumerate(U):
        rows = u[:nK] if n == N - 1 else u
        nu = np.sqrt(np.sum(rows * rows, axis=0))
        if np.any(nu == 0.0):
            flags |= O.FLAG_ZERO_COLUMN
            nu = np.where(nu == 0.0, 1.0, nu)
        out.append(u / nu)
        lam = lam * nu
    return out, lam, flags


def match(Us, anchors) -> O.Match:
    """Lemma 1 over N modes: score = prod_n |Gamma_n|, Hungarian maximum."""
    gam, norms = [], []
    for u, a in zip(Us, anchors):
        nrm = np.sqrt(np.sum(a * a, axis=0))
        gam.append(u.T @ (a / np.where(nrm == 0.0, 1.0, nrm)))
        norms.append(nrm)
    score = np.ones_like(gam[0])
    for g in gam:
        score = score * np.abs(g)
    rows, cols = scipy.optimize.linear_sum_assignment(score, maximize=True)
    perm = np.empty(score.shape[0], np.int64)
    perm[rows] = cols
    return O.Match(perm=perm, gamma=gam, norms=norms, score=score)


def project_coef(mt: O.Match, lam_s, lam_old, skip_mode: int) -> np.ndarray:
    """coef(r') = lam'_{r'} prod_{m != skip} Gamma_m(r', r) / (lam_r prod_{m != skip} N_m(r))."""
    R = lam_s.shape[0]
    coef = np.zeros(R)
    for rp in range(R):
        r = mt.perm[rp]
        num, den = lam_s[rp], lam_old[r]
        for m in range(len(mt.gamma)):
            if m != skip_mode:
                num *= mt.gamma[m][rp, r]
                den *= mt.norms[m][r]
        coef[rp] = num / den if den != 0.0 else 0.0
    return coef


def init_state_from_factors(X0: np.ndarray, lam, U, opts: O.Options) -> StateN:
    S = O.marginal_shift(X0)
    return StateN(X=np.array(X0, copy=True), U=[np.array(u, np.float64) for u in U],
                  lam=np.array(lam, np.float64), S=S, w=marginals(X0, S), batch=0, opts=replace(opts))


def update(state: StateN, X_new: np.ndarray):
    """Algorithm 1 for one batch of new slices X_new (K_new, I_1, ..., I_{N-1}).
    Sampling factors: s_I and s_J for the first two non-time modes, s_I for
    any further one, s_K for time.  The zero-entry fills and the lambda
    options of the 3-mode oracle are not carried over.  Returns (new StateN,
    per-repetition traces)."""
    opts = state.opts
    N = state.N
    K_old = state.X.shape[0]
    K_new = X_new.shape[0]
    R = state.lam.shape[0]
    if X_new.shape[1:] != state.X.shape[1:] or K_new < 1:
        raise ValueError("bad batch shape")
    dims = [state.X.shape[n + 1] for n in range(N - 1)] + [K_old]
    s_of = [opts.s_I, opts.s_J] + [opts.s_I] * (N - 3) + [opts.s_K]
    sizes = [O.sample_size(dims[n], s_of[n], state.w[n]) for n in range(N)]
    X_all = np.concatenate([state.X, X_new.astype(state.X.dtype)], axis=0)
    traces = []
    for rho in range(opts.r):
        idx = [O.sample_mode(state.w[n], sizes[n], opts, n, rho, state.batch) for n in range(N)]
        Kp = np.concatenate([idx[N - 1].astype(np.int64), np.arange(K_old, K_old + K_new)])
        Xs = X_all[np.ix_(Kp, *idx[:N - 1])]
        Xs = O.summary_values(Xs, opts.prec)
        gidx = idx[:N - 1] + [Kp]
        U0 = [O.init_factor(gidx[n], R, n, rho, state.batch, opts) for n in range(N)]
        res = cp_als(Xs, U0, opts.tol, opts.max_iters, opts.fixed_iters)
        Us, lam_s, _ = normalize_shared(res.U, res.lam, sizes[N - 1])
        anchors = [state.U[n][idx[n]] for n in range(N)]
        mt = match(Us[:N - 1] + [Us[N - 1][:sizes[N - 1]]], anchors)
        c = project_coef(mt, lam_s, state.lam, N - 1)
        Cnew = np.zeros((K_new, R))
        for rp in range(R):
            Cnew[:, mt.perm[rp]] = c[rp] * Us[N - 1][sizes[N - 1]:sizes[N - 1] + K_new, rp]
        traces.append(dict(idx=idx, als=res, match=mt, Cnew=Cnew))
    Cnew = sum(t["Cnew"] for t in traces) / opts.r
    w_new = marginals(X_new, state.S)
    w = [state.w[n] + w_new[n] for n in range(N - 1)] + [np.concatenate([state.w[N - 1], w_new[N - 1]])]
    U = [u.copy() for u in state.U[:N - 1]] + [np.concatenate([state.U[N - 1], Cnew], axis=0)]
    return StateN(X=X_all, U=U, lam=state.lam.copy(), S=state.S, w=w, batch=state.batch + 1,
                  opts=state.opts), traces


def reconstruct(lam, U, time_first: bool = True) -> np.ndarray:
    """sum_r lam_r U_1(:, r) o ... o C(:, r), array axes time first."""
    N = len(U)
    ltr, fax = _axes(N)
    subs = ",".join(f + "z" for f in fax)
    return np.einsum("z," + subs + "->" + ltr, lam, *U, optimize=True)
