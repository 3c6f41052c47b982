// After the ALS: shared-row normalisation, matching (Lemma 1), project back,
// commit of the averaged new rows; full-tensor fit; canonical order at init.
#include "sbt_internal.cuh"
#include "sbt_hungarian.cuh"

#include <cmath>

namespace sbt {

// ---------------------------------------------------------------------------
// Dot products of k_match.  Summary factors of the float32 / bfloat16 path are
// float32 and the anchors (the old factors) float64: the products are summed
// in double-float on the float32 pipes (float64 is a slow unit here); the
// float64 path sums in float64.
template <typename TF> struct MatchAcc;
template <> struct MatchAcc<double> {
    using Anchor = double;
    double v = 0.0;
    __device__ __forceinline__ static Anchor anchor(double a) { return a; }
    __device__ __forceinline__ void add_prod(double u, Anchor a) { v = fma(u, a, v); }
    __device__ __forceinline__ void add_sq(double u) { v = fma(u, u, v); }
    __device__ __forceinline__ void add_sq_anchor(Anchor a) { v = fma(a, a, v); }
    __device__ __forceinline__ void merge(const MatchAcc &o) { v += o.v; }
    __device__ __forceinline__ double value() const { return v; }
};
template <> struct MatchAcc<float> {
    using Anchor = DF;
    DF v{0.f, 0.f};
    __device__ __forceinline__ static Anchor anchor(double a) { return df_from_double(a); }
    __device__ __forceinline__ void add_prod(float u, Anchor a) { v = df_fma(v, DF{u, 0.f}, a); }
    __device__ __forceinline__ void add_sq(float u) { v = df_add_sq(v, u); }
    __device__ __forceinline__ void add_sq_anchor(Anchor a) { v = df_fma(v, a, a); }
    __device__ __forceinline__ void merge(const MatchAcc &o) { v = df_add(v, o.v); }
    __device__ __forceinline__ double value() const { return df_value(v); }
};

// rows staged per tile (the float64 path has twice the bytes per row and
// stays within 48 KB of static shared memory with 16)
template <typename TF> constexpr int match_ts() { return sizeof(TF) == 8 ? 16 : 32; }
constexpr int MATCH_ITEMS = (32 * 32 + 2 * 32 + 255) / 256;      // accumulators per thread
constexpr int MATCH_SLOTS = 32 * 32 + 2 * 32;                     // per-mode sums of a repetition

// The per-mode sums of k_match (one CTA per repetition and mode): over the
// shared rows, U'(:,r')^T anchor(:,r), |U'(:,r')|^2 and |anchor(:,r)|^2,
// each item's rows added in order; m.dots[rep][mode][item].
template <typename TF>
__global__ void __launch_bounds__(256) k_match_dots(MergeDesc m) {
    using Acc = MatchAcc<TF>;
    using Anchor = typename Acc::Anchor;
    const int rep = blockIdx.x;
    const int R = m.R;
    const int Rs = m.rnew ? m.rnew[rep] : R;
    const int Kp = m.nK + m.K_new;
    const int n[3] = {m.nI, m.nJ, Kp};
    const int nsh[3] = {m.nI, m.nJ, m.nK};
    constexpr int MATCH_TS = match_ts<TF>();
    __shared__ TF su[MATCH_TS * 32];
    __shared__ Anchor sa[MATCH_TS * 32];
    const TF *U[3];
    const int *S[3];
    const double *old[3] = {m.A, m.B, m.C};
    for (int q = 0; q < 3; ++q) {
        U[q] = (const TF *)m.U[q] + (long long)rep * n[q] * R;
        S[q] = m.samples + (long long)(rep * 3 + q) * m.samp_stride;
    }
    const int nitems = R * R + 2 * R;
    // few items (small R): `split` threads per item, each over the rows
    // t = part (mod split); the parts are merged in order 0..split-1
    const int split = nitems <= 64 ? 4 : (nitems <= 128 ? 2 : 1);
    const int part = threadIdx.x % split;
    static_assert(sizeof(TF) * MATCH_TS * 32 >= 256 * sizeof(Acc), "the merge reuses the staging buffer");
    Acc *parts = reinterpret_cast<Acc *>(su);  // free between a mode's last tile and the next mode's first
    // per mode over the shared rows: U'(:,r')^T anchor(:,r), |U'(:,r')|^2, |anchor(:,r)|^2
    {
        const int q = blockIdx.y;
        Acc acc[MATCH_ITEMS];
        // tiles of as many rows as R columns fill (the staged rows are packed
        // by R): few global round trips per mode; each item still adds the
        // rows in order
        const int TR = (MATCH_TS * 32) / R;
        for (int t0 = 0; t0 < nsh[q]; t0 += TR) {
            const int rows = min(TR, nsh[q] - t0);
            __syncthreads();
            // four entries per thread and round: the sampled indices, then
            // the anchor rows, all loads of a round in flight together
            for (int e0 = threadIdx.x; e0 < rows * R; e0 += 4 * blockDim.x) {
                int row[4];
                TF uv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + u * blockDim.x;
                    if (e < rows * R) {
                        const int t = t0 + e / R, c = e % R;
                        row[u] = S[q][t];
                        uv[u] = c < Rs ? U[q][(long long)t * Rs + c] : (TF)0;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + u * blockDim.x;
                    if (e < rows * R) {
                        su[e] = uv[u];
                        sa[e] = Acc::anchor(old[q][(long long)row[u] * R + e % R]);
                    }
                }
            }
            __syncthreads();
            // this thread's first row of the tile among rows = part (mod split)
            const int tb = ((part - t0) % split + split) % split;
#pragma unroll
            for (int u = 0; u < MATCH_ITEMS; ++u) {
                const int item = (threadIdx.x + u * 256) / split;
                if (item >= nitems || (split > 1 && u > 0)) break;
                if (item < R * R) {
                    const int rp = item / R, r = item % R;
                    for (int t = tb; t < rows; t += split) acc[u].add_prod(su[t * R + rp], sa[t * R + r]);
                } else if (item < R * R + R) {
                    const int rp = item - R * R;
                    for (int t = tb; t < rows; t += split) acc[u].add_sq(su[t * R + rp]);
                } else {
                    const int r = item - R * R - R;
                    for (int t = tb; t < rows; t += split) acc[u].add_sq_anchor(sa[t * R + r]);
                }
            }
        }
        if (split > 1) {
            __syncthreads();
            parts[threadIdx.x] = acc[0];
            __syncthreads();
            if (part == 0 && threadIdx.x / split < nitems)
                for (int k = 1; k < split; ++k) acc[0].merge(parts[threadIdx.x + k]);
        }
#pragma unroll
        for (int u = 0; u < MATCH_ITEMS; ++u) {
            const int item = (threadIdx.x + u * 256) / split;
            if (item >= nitems || (split > 1 && (u > 0 || part != 0))) break;
            m.dots[((long long)rep * 3 + q) * MATCH_SLOTS + item] = acc[u].value();
        }
    }
}

// One CTA per repetition: shared-row norms (Alg. 1 step 6), cosines and the
// matching (Lemma 1, Alg. 1 step 7), project back (steps 8-9).
template <typename TF>
__global__ void __launch_bounds__(256) k_match(MergeDesc m) {
    const int rep = blockIdx.x;
    const int R = m.R;
    const int Rs = m.rnew ? m.rnew[rep] : R;  // summary components (GetRank: R_new <= R)
    const int Kp = m.nK + m.K_new;
    const int n[3] = {m.nI, m.nJ, Kp};
    const int nsh[3] = {m.nI, m.nJ, m.nK};  // shared rows per mode
    __shared__ double nu[3][32], Nn[3][32], gam[3][32][32], score[32 * 32], lsp[32], scale[3][32];
    __shared__ int perm[32], iperm[32];
    __shared__ int zflag;
    __shared__ HungarianWork hw;  // in shared memory rather than the thread's stack
    const TF *U[3];
    const int *S[3];
    const double *old[3] = {m.A, m.B, m.C};
    for (int q = 0; q < 3; ++q) {
        // the repetition's n x R slot holds rows of Rs values
        U[q] = (const TF *)m.U[q] + (long long)rep * n[q] * R;
        S[q] = m.samples + (long long)(rep * 3 + q) * m.samp_stride;
    }
    if (threadIdx.x == 0) zflag = 0;
    const int nitems = R * R + 2 * R;
    // the per-mode sums (k_match_dots): dot products, then norms
    for (int e = threadIdx.x; e < 3 * nitems; e += blockDim.x) {
        const int q = e / nitems, item = e % nitems;
        const double v = m.dots[((long long)rep * 3 + q) * MATCH_SLOTS + item];
        if (item < R * R) {
            gam[q][item / R][item % R] = v;  // the dot product; divided by the norms below
        } else if (item < R * R + R) {
            double s = sqrt(v);
            if (s == 0.0) {
                s = 1.0;
                if (item - R * R < Rs) zflag = 1;  // columns past Rs are absent, not zero
            }
            nu[q][item - R * R] = s;
        } else {
            const double s = sqrt(v);
            Nn[q][item - R * R - R] = s == 0.0 ? 1.0 : s;
        }
    }
    __syncthreads();
    // cosines Gamma_q(r', r) between unit summary and unit anchor columns
    for (int e = threadIdx.x; e < 3 * R * R; e += blockDim.x) {
        const int q = e / (R * R), rp = (e / R) % R, r = e % R;
        gam[q][rp][r] /= nu[q][rp] * Nn[q][r];
    }
    __syncthreads();
    // the scores (one entry per thread) and the summary's lambda in its own scale
    for (int e = threadIdx.x; e < Rs * R; e += blockDim.x) {
        const int rp = e / R, r = e % R;
        score[rp * 32 + r] = fabs(gam[0][rp][r]) * fabs(gam[1][rp][r]) * fabs(gam[2][rp][r]);
    }
    if (threadIdx.x < Rs) {
        const int rp = threadIdx.x;
        lsp[rp] = m.lam_s[rep * R + rp] * nu[0][rp] * nu[1][rp] * nu[2][rp];
    }
    __syncthreads();
    if (threadIdx.x < 32) hungarian_max_warp(score, 32, Rs, R, perm, hw, threadIdx.x);
    __syncthreads();
    if (threadIdx.x < R) iperm[threadIdx.x] = -1;
    __syncthreads();
    if (threadIdx.x < Rs) iperm[perm[threadIdx.x]] = threadIdx.x;
    if (threadIdx.x < R) m.perm[rep * R + threadIdx.x] = threadIdx.x < Rs ? perm[threadIdx.x] : -1;
    for (int e = threadIdx.x; e < 3 * R; e += blockDim.x) m.nu[rep * 3 * R + e] = nu[e / R][e % R];
    if (threadIdx.x == 0) {
        double mn = INFINITY;
        for (int rp = 0; rp < Rs; ++rp) mn = fmin(mn, score[rp * 32 + perm[rp]]);
        m.min_score[rep] = mn;
        if (zflag) m.flags[rep] |= SBT_FLAG_ZERO_COLUMN_DEV;
    }
    __syncthreads();
    // the summary's estimate of lambda in the old scale; NaN: not matched
    if (threadIdx.x < R) {
        const int r = threadIdx.x, rp = iperm[r];
        const double den = Nn[0][r] * Nn[1][r] * Nn[2][r];
        m.lam_est[rep * R + r] =
            rp < 0 ? NAN : (den != 0.0 ? lsp[rp] * gam[0][rp][r] * gam[1][rp][r] * gam[2][rp][r] / den : 0.0);
    }
    // least-squares scale of a summary column of mode q in the matched old
    // scale, per unit of the raw summary value
    if (threadIdx.x < 3 * R) {
        const int q = threadIdx.x / R, rp = threadIdx.x % R;
        if (rp < Rs) {
            const int r = perm[rp];
            double num = lsp[rp], den = m.lam[r];
            for (int o = 0; o < 3; ++o)
                if (o != q) {
                    num *= gam[o][rp][r];
                    den *= Nn[o][r];
                }
            scale[q][rp] = den != 0.0 ? num / den / nu[q][rp] : 0.0;
        }
    }
    __syncthreads();
    // new rows of C (Alg. 1 step 9); NaN in the columns no summary component matched
    double *cn = m.cnew + (long long)rep * m.K_new * R;
    for (int e = threadIdx.x; e < m.K_new * R; e += blockDim.x) {
        const int k = e / R, r = e % R, rp = iperm[r];
        cn[e] = rp < 0 ? NAN : scale[2][rp] * (double)U[2][(long long)(m.nK + k) * Rs + rp];
    }
    // zero-entry proposals (Alg. 1 step 8): the three modes' entries as one
    // sequence, four per thread and round, the sampled indices and then the
    // old and summary values of a round in flight together
    const int tot0 = nsh[0] * R, tot01 = tot0 + nsh[1] * R, tot = tot01 + nsh[2] * R;
    for (int e0 = threadIdx.x; e0 < tot; e0 += 4 * blockDim.x) {
        int qv[4], ev[4], row[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int g = e0 + u * blockDim.x;
            qv[u] = g < tot0 ? 0 : (g < tot01 ? 1 : 2);
            ev[u] = g - (qv[u] == 0 ? 0 : (qv[u] == 1 ? tot0 : tot01));
            row[u] = g < tot ? S[qv[u]][ev[u] / R] : 0;
        }
        double ov[4], uv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int g = e0 + u * blockDim.x;
            const int q = qv[u], t = ev[u] / R, r = ev[u] % R;
            const int rp = g < tot ? iperm[r] : -1;
            ov[u] = rp >= 0 ? old[q][(long long)row[u] * R + r] : 1.0;
            uv[u] = rp >= 0 ? (double)U[q][(long long)t * Rs + rp] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int g = e0 + u * blockDim.x;
            if (g >= tot) continue;
            const int q = qv[u], r = ev[u] % R, rp = iperm[r];
            double val = NAN;
            if (rp >= 0 && ov[u] == 0.0) val = scale[q][rp] * uv[u];
            m.prop[((long long)rep * 3 + q) * m.pmax * R + ev[u]] = val;
        }
    }
}

cudaError_t launch_match(const MergeDesc &m, cudaStream_t st) {
    count_launches(2);
    if (m.elem == 0) {
        k_match_dots<double><<<dim3(m.nrep, 3), 256, 0, st>>>(m);
        k_match<double><<<m.nrep, 256, 0, st>>>(m);
    } else {
        k_match_dots<float><<<dim3(m.nrep, 3), 256, 0, st>>>(m);
        k_match<float><<<m.nrep, 256, 0, st>>>(m);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// overflow check of x_a + dx_a, x_b + dx_b (before anything is written)
__global__ void k_precommit(MergeDesc m) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    bool bad = false;
    if (e < m.I) bad = m.xa[e] + m.dxa[e] < m.xa[e];
    else if (e < m.I + m.J) bad = m.xb[e - m.I] + m.dxb[e - m.I] < m.xb[e - m.I];
    if (bad) atomicOr(&m.status->err, ERR_RANGE);
}

cudaError_t launch_precommit(const MergeDesc &m, cudaStream_t st) {
    long long n = (long long)m.I + m.J;
    count_launches(1);
    k_precommit<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m);
    return cudaGetLastError();
}

// lower_bound of x in ascending S[0..n)
__device__ __forceinline__ int find_sorted(const int *S, int n, int x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (S[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && S[lo] == x) ? lo : -1;
}

// Commit (Alg. 1 steps 8, 10, 12, 13): new rows of C = mean over repetitions;
// exactly-zero old entries = mean of the proposing repetitions; lambda; fold
// the marginal deltas.  Skipped entirely when the status word holds an error.
__global__ void k_commit(MergeDesc m) {
    if (m.status->err) return;
    const int R = m.R;
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nC = (long long)m.K_new * R;
    const long long nA = (long long)m.I * R, nB = (long long)m.J * R, nCo = (long long)m.K_old * R;
    if (e < nC) {
        // mean over the repetitions that matched the component (all of them
        // without GetRank); none: zero
        const int k = (int)(e / R), r = (int)(e % R);
        double s = 0.0;
        int c = 0;
        for (int q = 0; q < m.nrep; ++q) {
            const double v = m.cnew[((long long)q * m.K_new + k) * R + r];
            if (!isnan(v)) {
                s += v;
                ++c;
            }
        }
        m.C[(long long)(m.K_old + k) * R + r] = c ? s / c : 0.0;
        return;
    }
    e -= nC;
    if (e < nA + nB + nCo) {
        int q;
        double *F;
        int nsh;
        if (e < nA) {
            q = 0; F = m.A; nsh = m.nI;
        } else if (e < nA + nB) {
            e -= nA; q = 1; F = m.B; nsh = m.nJ;
        } else {
            e -= nA + nB; q = 2; F = m.C; nsh = m.nK;
        }
        if (F[e] != 0.0) return;
        const int x = (int)(e / R), r = (int)(e % R);
        double s = 0.0;
        int c = 0;
        for (int rep = 0; rep < m.nrep; ++rep) {
            const int *S = m.samples + (long long)(rep * 3 + q) * m.samp_stride;
            const int t = find_sorted(S, nsh, x);
            if (t < 0) continue;
            const double v = m.prop[(((long long)rep * 3 + q) * m.pmax + t) * R + r];
            if (!isnan(v)) {
                s += v;
                ++c;
            }
        }
        if (c) F[e] = s / c;
        return;
    }
    e -= nA + nB + nCo;
    if (e < R) {
        if (m.lambda_mode == 1) {
            double s = 0.0;
            int c = 0;
            for (int rep = 0; rep < m.nrep; ++rep) {
                const double v = m.lam_est[rep * R + e];
                if (!isnan(v)) {
                    s += v;
                    ++c;
                }
            }
            if (c) m.lam[e] = 0.5 * (m.lam[e] + s / c);
        }
        return;
    }
    e -= R;
    if (e < m.I) {
        unsigned long long v = m.xa[e] + m.dxa[e];
        m.xa[e] = v;
        if (v) atomicAdd(&m.status->npos[0], 1ull);
        return;
    }
    e -= m.I;
    if (e < m.J) {
        unsigned long long v = m.xb[e] + m.dxb[e];
        m.xb[e] = v;
        if (v) atomicAdd(&m.status->npos[1], 1ull);
        return;
    }
    e -= m.J;
    if (e < (long long)m.K_old + m.K_new) {
        unsigned long long v = e < m.K_old ? m.xc[e] : m.xc_new[e - m.K_old];
        if (e >= m.K_old) m.xc[e] = v;
        if (v) atomicAdd(&m.status->npos[2], 1ull);
    }
}

cudaError_t launch_commit(const MergeDesc &m, cudaStream_t st) {
    const long long R = m.R;
    long long n = (long long)m.K_new * R + (long long)m.I * R + (long long)m.J * R + (long long)m.K_old * R + R +
                  m.I + m.J + m.K_old + m.K_new;
    k_commit<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Full-tensor fit: 1 - ||X - X_hat|| / ||X|| (Section 4.2).  A warp per row
// (k, i): x_hat(j) = sum_r lambda_r A(i,r) C(k,r) B(j,r); residual squares and
// squares accumulate per lane, then per CTA, then in fixed order.
template <typename TS> struct FitAcc;
template <> struct FitAcc<float> {
    DF r{0.f, 0.f}, x{0.f, 0.f};
    __device__ void add(float xv, float xh) {
        float d = xv - xh;
        r = df_add_sq(r, d);
        x = df_add_sq(x, xv);
    }
    __device__ void total(double &rr, double &xx) {
        rr = df_value(warp_df_sum(r));
        xx = df_value(warp_df_sum(x));
    }
};
template <> struct FitAcc<double> {
    double r = 0.0, x = 0.0;
    __device__ void add(double xv, double xh) {
        double d = xv - xh;
        r += d * d;
        x += xv * xv;
    }
    __device__ void total(double &rr, double &xx) {
        rr = warp_sum(r);
        xx = warp_sum(x);
    }
};

template <typename TS>
__global__ void k_bcast_b(const double *B, TS *Bt, int J, int R) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < (long long)J * R) Bt[e] = (TS)B[e];
}

template <typename TS>
__global__ void __launch_bounds__(256) k_fit_rows(const TS *X, int K, int I, int J, int lds, const double *A,
                                                  const TS *Bc, const double *C, const double *lam, int R,
                                                  double *part) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ double red_r[8], red_x[8];
    const long long rows = (long long)K * I;
    double tr = 0.0, tx = 0.0;
    for (long long row = (long long)blockIdx.x * 8 + warp; row < rows; row += (long long)gridDim.x * 8) {
        const int k = (int)(row / I), i = (int)(row % I);
        TS w[32];
        for (int r = 0; r < R; ++r) w[r] = (TS)(lam[r] * A[(long long)i * R + r] * C[(long long)k * R + r]);
        const TS *xr = X + row * lds;
        FitAcc<TS> acc;
        for (int j = lane; j < J; j += 32) {
            TS xh = 0;
            const TS *b = Bc + (long long)j * R;
            for (int r = 0; r < R; ++r) xh = fmadd(w[r], b[r], xh);
            acc.add(xr[j], xh);
        }
        double rr, xx;
        acc.total(rr, xx);
        tr += rr;
        tx += xx;
    }
    if (lane == 0) {
        red_r[warp] = tr;
        red_x[warp] = tx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < 8; ++q) {
            a += red_r[q];
            b += red_x[q];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_fit_final(const double *part, int nb, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < nb; ++q) {
            a += part[2 * q];
            b += part[2 * q + 1];
        }
        out[0] = a;
        out[1] = b;
    }
}

static const int FIT_BLOCKS = 1216;

long long fit_scratch_doubles(int K, int I, int J, int R) {
    (void)K;
    (void)I;
    return 2LL * FIT_BLOCKS + (long long)J * R + 16;
}

cudaError_t launch_full_fit(const void *store, int sdtype, int K, int I, int J, int lds, const double *A,
                            const double *B, const double *C, const double *lam, int R, double *out,
                            double *scratch, cudaStream_t st) {
    double *part = scratch;
    void *bc = scratch + 2 * FIT_BLOCKS;
    const long long nb = (long long)J * R;
    if (sdtype == 0) {
        k_bcast_b<double><<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(B, (double *)bc, J, R);
        k_fit_rows<double><<<FIT_BLOCKS, 256, 0, st>>>((const double *)store, K, I, J, lds, A, (const double *)bc,
                                                       C, lam, R, part);
    } else {
        k_bcast_b<float><<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(B, (float *)bc, J, R);
        k_fit_rows<float><<<FIT_BLOCKS, 256, 0, st>>>((const float *)store, K, I, J, lds, A, (const float *)bc, C,
                                                      lam, R, part);
    }
    k_fit_final<<<1, 32, 0, st>>>(part, FIT_BLOCKS, out);
    count_launches(3);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Init: sort components by lambda (descending, stable) and fix signs so that
// sum A(:,r) >= 0 and sum B(:,r) >= 0, pushing signs into C.
template <typename TF>
__global__ void __launch_bounds__(256) k_canon(AlsDesc d, double *A, double *B, double *C, double *lam) {
    const int R = d.R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ int order[32];
    __shared__ double sgn[2][32];
    const TF *U0 = (const TF *)d.U[0], *U1 = (const TF *)d.U[1], *U2 = (const TF *)d.U[2];
    if (threadIdx.x == 0) {
        for (int r = 0; r < R; ++r) order[r] = r;
        for (int a = 1; a < R; ++a) {  // stable insertion sort, descending
            int v = order[a], b = a - 1;
            while (b >= 0 && d.lam[order[b]] < d.lam[v]) {
                order[b + 1] = order[b];
                --b;
            }
            order[b + 1] = v;
        }
    }
    __syncthreads();
    for (int pr = warp; pr < 2 * R; pr += 8) {
        const int q = pr / R, r = pr % R;
        const TF *U = q == 0 ? U0 : U1;
        const int n = d.n[q];
        double s = 0.0;
        for (int x = lane; x < n; x += 32) s += (double)U[(long long)x * R + order[r]];
        s = warp_sum(s);
        if (lane == 0) sgn[q][r] = s < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)d.n[0] * R; e += blockDim.x) {
        int x = (int)(e / R), r = (int)(e % R);
        A[e] = sgn[0][r] * (double)U0[(long long)x * R + order[r]];
    }
    for (long long e = threadIdx.x; e < (long long)d.n[1] * R; e += blockDim.x) {
        int x = (int)(e / R), r = (int)(e % R);
        B[e] = sgn[1][r] * (double)U1[(long long)x * R + order[r]];
    }
    for (long long e = threadIdx.x; e < (long long)d.n[2] * R; e += blockDim.x) {
        int x = (int)(e / R), r = (int)(e % R);
        C[e] = sgn[0][r] * sgn[1][r] * (double)U2[(long long)x * R + order[r]];
    }
    if (threadIdx.x < R) lam[threadIdx.x] = d.lam[order[threadIdx.x]];
}

cudaError_t launch_canonicalize(const AlsDesc &d, double *A, double *B, double *C, double *lam,
                                cudaStream_t st) {
    count_launches(1);
    if (d.elem == 0) k_canon<double><<<1, 256, 0, st>>>(d, A, B, C, lam);
    else k_canon<float><<<1, 256, 0, st>>>(d, A, B, C, lam);
    return cudaGetLastError();
}

}  // namespace sbt
