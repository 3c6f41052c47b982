"""Seeded synthetic tensors shaped like the paper's planted workloads.

This module is the one piece shared by the FP64 oracle's tests and the CUDA
path's tests and benchmark.  It holds no arithmetic of the method itself: it
only draws planted CP factors and noise (Section 4.1.1 of the paper: tensors
built from known, randomly generated factors) and hands out the same bytes to
both sides.

Recipe (dense):
    A, B, C  ~ U[0, 1) i.i.d., lambda = 1
    X(i, j, k) = sum_r A(i, r) B(j, r) C(k, r) + eps,
    eps ~ N(0, sigma^2), sigma = c * RMS(noiseless X over the full final tensor)
Layout: slice-major, X[k, i, j] (k = time mode), i.e. element (i, j, k) sits at
offset (k * I + i) * J + j.

Optionally (`cond`), the factors are mixed toward a shared direction,
a_r <- (1 - beta) u_r + beta u_0, with beta found by bisection so that the
condition number of each factor Gram is about `cond` (values stay in [0, 1]).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch


@dataclass
class Planted:
    X: torch.Tensor          # (K_total, I, J), slice-major, requested dtype
    A: torch.Tensor          # (I, R) float64, planted
    B: torch.Tensor          # (J, R)
    C: torch.Tensor          # (K_total, R)
    sigma: float             # noise standard deviation actually used

    def slices(self, k0: int, k1: int) -> torch.Tensor:
        return self.X[k0:k1]


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _mix_to_condition(U: torch.Tensor, target: float) -> torch.Tensor:
    """Mix columns toward the first one until cond(U^T U) ~= target."""
    if target is None or U.shape[1] < 2:
        return U
    u0 = U[:, :1]

    def cond_of(beta: float) -> float:
        M = (1.0 - beta) * U + beta * u0
        ev = torch.linalg.eigvalsh(M.T @ M)
        return float(ev[-1] / ev[0].clamp_min(1e-300))

    lo, hi = 0.0, 0.999
    if cond_of(lo) >= target:
        return U
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if cond_of(mid) < target:
            lo = mid
        else:
            hi = mid
    beta = 0.5 * (lo + hi)
    return (1.0 - beta) * U + beta * u0


def planted_dense(I: int, J: int, K: int, R: int, *, noise: float = 0.01,
                  seed: int = 0, dtype=torch.float32, device="cpu",
                  cond: float | None = None, dist: str = "uniform") -> Planted:
    """Planted rank-R dense tensor (K slices of I x J), seeded.

    `dist` is "uniform" (U[0,1) factors, the paper's recipe) or "normal"
    (N(0,1) factors, better conditioned; used by small pin tests).
    The noiseless tensor is formed in float32 on CUDA devices (float64 on the
    CPU), the noise in the same type; the result is cast to `dtype`.
    """
    dev = torch.device(device)
    g = _gen(seed, dev)
    draw = torch.rand if dist == "uniform" else torch.randn
    A = draw(I, R, generator=g, device=dev, dtype=torch.float64)
    B = draw(J, R, generator=g, device=dev, dtype=torch.float64)
    C = draw(K, R, generator=g, device=dev, dtype=torch.float64)
    if cond is not None:
        A = _mix_to_condition(A, cond)
        B = _mix_to_condition(B, cond)
        C = _mix_to_condition(C, cond)
    work = torch.float64 if dev.type == "cpu" else torch.float32
    # noiseless X_(3) = C (A kr B)^T, slice by slice to bound memory
    AB = (A[:, None, :] * B[None, :, :]).reshape(I * J, R).to(work)
    X = torch.empty(K, I, J, dtype=work, device=dev)
    step = max(1, (1 << 28) // max(1, I * J))
    sumsq = 0.0
    for k0 in range(0, K, step):
        k1 = min(K, k0 + step)
        blk = (C[k0:k1].to(work) @ AB.T).reshape(k1 - k0, I, J)
        X[k0:k1] = blk
        sumsq += float((blk.double() ** 2).sum())
    rms = math.sqrt(sumsq / max(1, I * J * K))
    sigma = float(noise) * rms
    if sigma > 0:
        for k0 in range(0, K, step):
            k1 = min(K, k0 + step)
            X[k0:k1] += sigma * torch.randn(k1 - k0, I, J, generator=g,
                                             device=dev, dtype=work)
    return Planted(X=X.to(dtype), A=A, B=B, C=C, sigma=sigma)


def poisson_arrivals(n: int, rate: float, seed: int = 0) -> list[float]:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    g = _gen(seed, "cpu")
    gaps = torch.empty(n, dtype=torch.float64).exponential_(1.0, generator=g)
    t = torch.cumsum(gaps / float(rate), 0)
    return [float(x) for x in t]


@dataclass
class SparsePlanted:
    k: torch.Tensor          # (nnz,) int32 time slice, sorted (time-major order)
    i: torch.Tensor          # (nnz,) int32
    j: torch.Tensor          # (nnz,) int32
    v: torch.Tensor          # (nnz,) float32: planted model + noise at the coordinate
    A: torch.Tensor          # (I, R) float64, zero off the component supports
    B: torch.Tensor          # (J, R)
    C: torch.Tensor          # (K, R)
    sigma: float

    def batch(self, k0: int, k1: int):
        """Nonzeros of slices [k0, k1) with k relative to k0."""
        lo = int(torch.searchsorted(self.k, torch.tensor(k0, dtype=self.k.dtype, device=self.k.device)))
        hi = int(torch.searchsorted(self.k, torch.tensor(k1, dtype=self.k.dtype, device=self.k.device)))
        return self.i[lo:hi], self.j[lo:hi], self.k[lo:hi] - k0, self.v[lo:hi]

    def dense(self, k0: int = 0, k1: int = None) -> torch.Tensor:
        """The slices [k0, k1) as a dense (K, I, J) float32 array on the CPU (small tensors only)."""
        k1 = self.C.shape[0] if k1 is None else k1
        I, J = self.A.shape[0], self.B.shape[0]
        ii, jj, kk, vv = (t.cpu() for t in self.batch(k0, k1))
        X = torch.zeros(k1 - k0, I, J, dtype=torch.float32)
        X[kk.long(), ii.long(), jj.long()] = vv
        return X


def planted_sparse(I: int, J: int, K: int, R: int, *, support: int, coords: int, noise: float = 0.01,
                   seed: int = 0, device="cpu") -> SparsePlanted:
    """Planted sparse CP tensor, seeded: component r has `support` random
    indices in each mode with factor values U[0, 1) there (0 elsewhere);
    `coords` coordinates are drawn uniformly from its support box; the value
    at a coordinate is the full planted model plus N(0, noise^2); coordinates
    drawn more than once are kept once.  Time-sorted."""
    dev = torch.device(device)
    g = _gen(seed, dev)
    U = []
    sup = []
    for n in (I, J, K):
        Un = torch.zeros(n, R, dtype=torch.float64, device=dev)
        Sn = torch.stack([torch.randperm(n, generator=g, device=dev)[:support] for _ in range(R)])  # (R, support)
        vals = torch.rand(R, support, generator=g, device=dev, dtype=torch.float64)
        for r in range(R):
            Un[Sn[r], r] = vals[r]
        U.append(Un)
        sup.append(Sn)
    keys = []
    for r in range(R):
        t = [sup[m][r][torch.randint(0, support, (coords,), generator=g, device=dev)].long() for m in range(3)]
        keys.append((t[2] * I + t[0]) * J + t[1])
    key = torch.unique(torch.cat(keys))  # sorted: time-major
    k = key // (I * J)
    i = (key // J) % I
    j = key % J
    A, B, C = U
    v = torch.empty(key.shape[0], dtype=torch.float32, device=dev)
    step = 1 << 22
    for a in range(0, key.shape[0], step):
        b = min(a + step, key.shape[0])
        model = (A[i[a:b]] * B[j[a:b]] * C[k[a:b]]).sum(dim=1)
        v[a:b] = (model + noise * torch.randn(model.shape, generator=g, device=dev, dtype=torch.float64)).to(
            torch.float32)
    return SparsePlanted(k=k.to(torch.int32), i=i.to(torch.int32), j=j.to(torch.int32), v=v, A=A, B=B, C=C,
                         sigma=noise)


@dataclass
class PlantedN:
    X: torch.Tensor          # (K, I_1, ..., I_{N-1}), time first, requested dtype
    U: list                  # [U_1, ..., U_{N-1}, C] float64, planted (factor order)
    sigma: float


def planted_dense_n(dims, K: int, R: int, *, noise: float = 0.01, seed: int = 0,
                    dtype=torch.float64, device="cpu") -> PlantedN:
    """Planted rank-R order-N tensor, seeded: factors U_m ~ U[0, 1) i.i.d.
    for the modes of `dims` = (I_1, ..., I_{N-1}) and for time (K rows);
    X(k, i_1, ...) = sum_r prod_m U_m(i_m, r) + N(0, sigma^2), sigma = noise *
    RMS of the noiseless tensor.  Time-first layout."""
    dev = torch.device(device)
    g = _gen(seed, dev)
    U = [torch.rand(d, R, generator=g, device=dev, dtype=torch.float64) for d in dims]
    C = torch.rand(K, R, generator=g, device=dev, dtype=torch.float64)
    # noiseless X: outer products built up one mode at a time, time first
    X = C
    for u in U:
        X = (X.unsqueeze(-2) * u.reshape((1,) * (X.dim() - 1) + u.shape))
    X = X.sum(dim=-1)
    rms = float(X.pow(2).mean().sqrt())
    sigma = float(noise) * rms
    if sigma > 0:
        X = X + sigma * torch.randn(X.shape, generator=g, device=dev, dtype=torch.float64)
    return PlantedN(X=X.to(dtype).contiguous(), U=U + [C], sigma=sigma)
