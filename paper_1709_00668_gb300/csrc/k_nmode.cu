// Order-N tensors: Algorithm 1 for a dense tensor with N = 3..SBT_NMODE_MAX
// modes, the first array axis being time (the mode that grows).  Section 2.2
// states that the problem and the method extend to any number of modes; every
// step is the 3-mode step with "three modes" replaced by "all modes":
//   append + Eq. 1 marginals of every mode (exact 64-bit fixed point),
//   sampling of every mode by exponential keys (the 3-mode sampler, one mode
//   per launch; mode ids in factor order, time last),
//   the summary gather, CP-ALS over all N modes (MTTKRP with the Khatri-Rao
//   rows of the other N-1 factors formed on the fly, Hadamard product of the
//   other N-1 Grams, float64 Cholesky solve, unit columns, fit),
//   shared-row normalisation, Lemma 1 matching with the product of the N
//   |cosine| matrices, project back of the new time rows, commit.
// Layouts: the store X[k][i_1]...[i_{N-1}] (row-major, time first, innermost
// axis contiguous); a summary the same with the sampled sizes; factors in
// factor order U[0..N-2] = modes 1..N-1, U[N-1] = C (time), each n x R
// row-major float64.  The MTTKRP of a float32 summary multiplies and sums in
// float32 within a lane and in float64 across lanes, warps and CTAs; the
// float64 path is float64 throughout.  Every reduction has a fixed order or
// is an exact integer sum, so results do not depend on timing.
#include "sambaten.h"
#include "sbt_internal.cuh"
#include "sbt_hungarian.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace sbt {

constexpr int NM_MAX = SBT_NMODE_MAX;
constexpr int NM_THREADS = 256;

// Shape of an order-N array in factor order: mode m < N-1 is array axis m+1,
// mode N-1 (time) is axis 0.  st[m] = element stride of mode m.
struct NmShape {
    int N;
    int n[NM_MAX];
    long long st[NM_MAX];
    long long total;
};

__host__ __device__ inline NmShape nm_shape(int N, const int *n) {
    NmShape s;
    s.N = N;
    for (int m = 0; m < NM_MAX; ++m) {
        s.n[m] = m < N ? n[m] : 1;
        s.st[m] = 0;
    }
    long long stride = 1;
    for (int m = N - 2; m >= 0; --m) {  // axes N-1 .. 1 (modes N-2 .. 0), innermost first
        s.st[m] = stride;
        stride *= s.n[m];
    }
    s.st[N - 1] = stride;  // time, outermost
    s.total = stride * s.n[N - 1];
    return s;
}

// ---------------------------------------------------------------------------
// Append + marginals (Eq. 1): copy K_new slices into the store and add the
// fixed-point squares q(x) = floor((x * x) 2^S) of every element to the
// marginal of its index in every mode.  A CTA takes NM_ROWS consecutive rows
// (a row = the innermost axis at fixed other indices); each thread keeps its
// columns' sums over those rows, rows are summed in shared memory; all sums
// are exact 64-bit integers, so their order does not matter.
constexpr int NM_ROWS = 16;

struct NmW {
    unsigned long long *w[NM_MAX];  // marginal of every mode in factor order (time: of the slices written)
};

template <typename T>
__global__ void __launch_bounds__(NM_THREADS) k_nm_append(const T *in, T *out, NmShape s, int S, NmW mw,
                                                          DevStatus *status) {
    unsigned long long *const *w = mw.w;
    const int N = s.N, inner = N - 2;
    const int J = s.n[inner];
    const long long rows = s.total / J;
    const long long r0 = (long long)blockIdx.x * NM_ROWS;
    const int nr = (int)(rows - r0 < NM_ROWS ? rows - r0 : NM_ROWS);
    __shared__ unsigned long long rsum[NM_ROWS];
    if (threadIdx.x < NM_ROWS) rsum[threadIdx.x] = 0ull;
    __syncthreads();
    bool bad = false, over = false;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        unsigned long long cs = 0ull;
        for (int t = 0; t < nr; ++t) {
            const long long e = (r0 + t) * J + j;
            const T x = in[e];
            out[e] = x;
            const double xd = (double)x;
            if (!isfinite(xd)) {
                bad = true;
                continue;
            }
            const double sq = ldexp(__dmul_rn(xd, xd), S);
            if (sq >= 18446744073709551616.0) {
                over = true;
                continue;
            }
            const unsigned long long q = (unsigned long long)floor(sq);
            cs += q;
            atomicAdd(&rsum[t], q);
        }
        if (cs) atomicAdd(&w[inner][j], cs);
    }
    if (bad) atomicOr(&status->err, ERR_NONFINITE);
    if (over) atomicOr(&status->err, ERR_RANGE);
    __syncthreads();
    if (threadIdx.x < nr) {
        const unsigned long long v = rsum[threadIdx.x];
        if (v) {
            // the row's index in every mode but the innermost
            long long row = r0 + threadIdx.x;
            for (int m = N - 3; m >= 0; --m) {
                const int i = (int)(row % s.n[m]);
                row /= s.n[m];
                atomicAdd(&w[m][i], v);
            }
            atomicAdd(&w[N - 1][row], v);  // time: the slice
        }
    }
}

cudaError_t launch_nm_append(const void *in, void *out, int dtype, const NmShape &s, int S, const NmW &w,
                             DevStatus *status, cudaStream_t st) {
    const long long rows = s.total / s.n[s.N - 2];
    const unsigned blocks = (unsigned)((rows + NM_ROWS - 1) / NM_ROWS);
    count_launches(1);
    if (dtype == SBT_F64)
        k_nm_append<double><<<blocks, NM_THREADS, 0, st>>>((const double *)in, (double *)out, s, S, w, status);
    else
        k_nm_append<float><<<blocks, NM_THREADS, 0, st>>>((const float *)in, (float *)out, s, S, w, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Summary gather (Alg. 1 step 4): Xs[rep][kk][ii_1]...[ii_{N-1}] =
// X(K'[kk], I_1[ii_1], ...), K' = the sampled old slices then the new ones.
// samples: [mode][rep][stride]; the time mode's list holds the old slices.
template <typename T>
__global__ void __launch_bounds__(NM_THREADS) k_nm_gather(const T *X, NmShape sx, NmShape ss, const int *samples,
                                                          long long sstride, int nrep, int nK, int K_old, T *Xs) {
    const int N = ss.N;
    const long long total = ss.total * nrep;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int rep = (int)(e / ss.total);
        long long rem = e % ss.total;
        long long src = 0;
        for (int m = N - 2; m >= 0; --m) {
            const int ii = (int)(rem % ss.n[m]);
            rem /= ss.n[m];
            src += (long long)samples[((long long)m * nrep + rep) * sstride + ii] * sx.st[m];
        }
        const int kk = (int)rem;
        const int k = kk < nK ? samples[((long long)(N - 1) * nrep + rep) * sstride + kk] : K_old + (kk - nK);
        src += (long long)k * sx.st[N - 1];
        Xs[e] = X[src];
    }
}

cudaError_t launch_nm_gather(const void *X, int dtype, const NmShape &sx, const NmShape &ss, const int *samples,
                             long long sstride, int nrep, int nK, int K_old, void *Xs, cudaStream_t st) {
    const long long total = ss.total * nrep;
    const unsigned blocks = (unsigned)std::min<long long>((total + NM_THREADS - 1) / NM_THREADS, 152LL * 16);
    count_launches(1);
    if (dtype == SBT_F64)
        k_nm_gather<double><<<blocks, NM_THREADS, 0, st>>>((const double *)X, sx, ss, samples, sstride, nrep, nK,
                                                           K_old, (double *)Xs);
    else
        k_nm_gather<float><<<blocks, NM_THREADS, 0, st>>>((const float *)X, sx, ss, samples, sstride, nrep, nK,
                                                          K_old, (float *)Xs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CP-ALS of the r summaries over all N modes (Alg. 1 step 5).
struct NmAls {
    int nrep, R, nK;
    NmShape s;               // one summary, factor order (s.n[N-1] = Kp)
    const void *X;           // [rep][s.total], float or double (elem)
    int elem;                // 0 float64, 1 float32
    double *U[NM_MAX];       // [rep][n_m][R]
    double *part;            // [rep][P][n_max][R] MTTKRP partial sums
    long long prs;           // doubles per repetition of part
    int P[NM_MAX];           // partials per mode
    double *G;               // [rep][N][R][R] Grams of the unit-column factors
    double *lam;             // [rep][R]
    double *fit, *fit_prev, *normX2;  // [rep]
    int *iters, *conv, *flags;        // [rep]
    double tol;
    int max_iters, fixed_iters;
};

// Start: Philox uniforms keyed by the global index in every mode (counter
// (x, r | mode << 8 | rep << 12, batch, 2), mode in factor order), the Grams,
// ||X_s||^2 (fixed order), the iteration state.  One CTA per repetition.
template <typename T>
__global__ void __launch_bounds__(NM_THREADS) k_nm_prepare(NmAls d, const int *samples, long long sstride, int K_old,
                                                           uint64_t seed, uint32_t stream_id, uint32_t batch) {
    const int rep = blockIdx.x, R = d.R, N = d.s.N;
    const uint2 key = philox_key(seed, stream_id);
    for (int m = 0; m < N; ++m) {
        const int n = d.s.n[m];
        double *U = d.U[m] + (long long)rep * n * R;
        const int *S = samples + ((long long)m * d.nrep + rep) * sstride;
        for (long long e = threadIdx.x; e < (long long)n * R; e += blockDim.x) {
            const int x = (int)(e / R), r = (int)(e % R);
            const uint32_t gx = (uint32_t)(m < N - 1 || x < d.nK ? S[x] : K_old + (x - d.nK));
            U[e] = init_value(key, gx, r, m, rep, batch);
        }
    }
    __syncthreads();
    for (int m = 0; m < N; ++m) {
        const int n = d.s.n[m];
        const double *U = d.U[m] + (long long)rep * n * R;
        double *G = d.G + ((long long)rep * NM_MAX + m) * R * R;
        for (int pq = threadIdx.x; pq < R * R; pq += blockDim.x) {
            const int a = pq / R, b = pq % R;
            double g = 0.0;
            for (int x = 0; x < n; ++x) g = fma(U[(long long)x * R + a], U[(long long)x * R + b], g);
            G[pq] = g;
        }
    }
    const T *X = (const T *)d.X + (long long)rep * d.s.total;
    __shared__ double red[NM_THREADS];
    double a = 0.0;
    for (long long e = threadIdx.x; e < d.s.total; e += blockDim.x) {
        const double v = (double)X[e];
        a = fma(v, v, a);
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int h = NM_THREADS / 2; h; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        d.normX2[rep] = red[0];
        d.fit[rep] = 0.0;
        d.fit_prev[rep] = 0.0;
        d.iters[rep] = 0;
        d.conv[rep] = 0;
        int nmin = d.nK;
        for (int m = 0; m < N - 1; ++m) nmin = min(nmin, d.s.n[m]);
        d.flags[rep] = nmin < R ? SBT_FLAG_SAMPLE_LT_RANK_DEV : 0;
    }
}

// Outer modes of an MTTKRP: every mode but `skip1` and `skip2`, innermost
// axis first (modes N-3 .. 0), time last.  Returns their count.
__device__ inline int nm_outer_modes(int N, int skip1, int skip2, int *om) {
    int c = 0;
    for (int m = N - 3; m >= 0; --m)
        if (m != skip1 && m != skip2) om[c++] = m;
    if (N - 1 != skip1 && N - 1 != skip2) om[c++] = N - 1;
    return c;
}

// Compute type of the MTTKRP products: float32 summaries multiply in float32
template <typename T> struct NmCompute { using C = double; };
template <> struct NmCompute<float> { using C = float; };

// MTTKRP of mode n != N-2 (the innermost axis): M(x, r) = sum over the other
// indices of X times the product of the other factors' entries.  CTA (x, p):
// row x of the output, partial p; its warps take the outer index tuples o
// (all modes but n and the innermost) p*8 + warp, stepping by P*8; for each
// o the lanes run along the contiguous innermost axis, z(r) = sum_j x(o, j)
// U_inner(j, r), then acc(r) += z(r) * prod over the outer modes of U(i, r).
// Lanes, then warps (in order) are added in float64; partial p of row x goes
// to part[rep][p][x][r].
template <typename T, int RP>
__global__ void __launch_bounds__(NM_THREADS) k_nm_mtt_outer(NmAls d, int n) {
    using TC = typename NmCompute<T>::C;
    const int rep = blockIdx.y, R = d.R, N = d.s.N, inner = N - 2;
    if (d.conv[rep]) return;
    const int P = d.P[n];
    const int x = blockIdx.x / P, p = blockIdx.x % P;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int J = d.s.n[inner];
    extern __shared__ __align__(16) unsigned char nm_smem[];
    TC *uin = reinterpret_cast<TC *>(nm_smem);  // [J][RP] innermost factor
    const double *Ui = d.U[inner] + (long long)rep * J * R;
    for (int e = threadIdx.x; e < J * RP; e += blockDim.x) {
        const int j = e / RP, r = e % RP;
        uin[e] = r < R ? (TC)Ui[(long long)j * R + r] : (TC)0;
    }
    __syncthreads();
    int om[NM_MAX];
    const int no = nm_outer_modes(N, n, inner, om);
    long long O = 1;
    for (int q = 0; q < no; ++q) O *= d.s.n[om[q]];
    const T *X = (const T *)d.X + (long long)rep * d.s.total + (long long)x * d.s.st[n];
    double acc[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) acc[r] = 0.0;
    for (long long o = (long long)p * 8 + warp; o < O; o += (long long)P * 8) {
        long long rem = o, base = 0;
        TC pr[RP];
#pragma unroll
        for (int r = 0; r < RP; ++r) pr[r] = (TC)1;
        for (int q = 0; q < no; ++q) {
            const int m = om[q];
            const int i = (int)(rem % d.s.n[m]);
            rem /= d.s.n[m];
            base += (long long)i * d.s.st[m];
            const double *Um = d.U[m] + ((long long)rep * d.s.n[m] + i) * R;
#pragma unroll
            for (int r = 0; r < RP; ++r)
                if (r < R) pr[r] *= (TC)Um[r];
        }
        TC z[RP];
#pragma unroll
        for (int r = 0; r < RP; ++r) z[r] = (TC)0;
        for (int j = lane; j < J; j += 32) {
            const TC v = (TC)X[base + j];
            const TC *u = uin + j * RP;
#pragma unroll
            for (int r = 0; r < RP; ++r) z[r] = fma(v, u[r], z[r]);
        }
#pragma unroll
        for (int r = 0; r < RP; ++r) acc[r] = fma((double)z[r], (double)pr[r], acc[r]);
    }
    __shared__ double wred[8][RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) {
        const double v = warp_sum(acc[r]);
        if (lane == 0) wred[warp][r] = v;
    }
    __syncthreads();
    if (threadIdx.x < R) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += wred[w][threadIdx.x];
        d.part[(long long)rep * d.prs + ((long long)p * d.s.n[n] + x) * R + threadIdx.x] = s;
    }
}

// MTTKRP of the innermost mode (n = N-2): CTA (jb, p) takes the 32 output
// rows jb*32 + lane (one per lane) and partial p; its warps take the outer
// index tuples o (all modes but the innermost) p*8 + warp, stepping by P*8:
// acc(r) += x(o, j) * prod over the other modes of U(i, r).  Warps are added
// in order through shared memory.
template <typename T, int RP>
__global__ void __launch_bounds__(NM_THREADS) k_nm_mtt_inner(NmAls d) {
    using TC = typename NmCompute<T>::C;
    const int rep = blockIdx.y, R = d.R, N = d.s.N, inner = N - 2;
    if (d.conv[rep]) return;
    const int P = d.P[inner];
    const int jb = blockIdx.x / P, p = blockIdx.x % P;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int J = d.s.n[inner];
    const int j = jb * 32 + lane;
    int om[NM_MAX];
    const int no = nm_outer_modes(N, inner, inner, om);
    long long O = 1;
    for (int q = 0; q < no; ++q) O *= d.s.n[om[q]];
    const T *X = (const T *)d.X + (long long)rep * d.s.total;
    double acc[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) acc[r] = 0.0;
    for (long long o = (long long)p * 8 + warp; o < O; o += (long long)P * 8) {
        long long rem = o, base = 0;
        TC pr[RP];
#pragma unroll
        for (int r = 0; r < RP; ++r) pr[r] = (TC)1;
        for (int q = 0; q < no; ++q) {
            const int m = om[q];
            const int i = (int)(rem % d.s.n[m]);
            rem /= d.s.n[m];
            base += (long long)i * d.s.st[m];
            const double *Um = d.U[m] + ((long long)rep * d.s.n[m] + i) * R;
#pragma unroll
            for (int r = 0; r < RP; ++r)
                if (r < R) pr[r] *= (TC)Um[r];
        }
        if (j < J) {
            const TC v = (TC)X[base + j];
#pragma unroll
            for (int r = 0; r < RP; ++r) acc[r] += (double)(v * pr[r]);
        }
    }
    __shared__ double red[32][RP + 1];
    for (int w = 0; w < 8; ++w) {
        if (warp == w) {
#pragma unroll
            for (int r = 0; r < RP; ++r) red[lane][r] = (w == 0 ? 0.0 : red[lane][r]) + acc[r];
        }
        __syncthreads();
    }
    if (warp == 0 && j < J)
        for (int r = 0; r < R; ++r) d.part[(long long)rep * d.prs + ((long long)p * J + j) * R + r] = red[lane][r];
}

// Tail of mode n, one CTA per repetition, float64: M = the partials summed in
// order; V = Hadamard product of the other N-1 Grams; Cholesky V = L L^T (a
// pivot <= 0: V + 1e-12 tr(V)/R I and a flag); U_n = M V^-1 row by row;
// lambda = column 2-norms (zero: 1 and a flag); U_n /= lambda; the new Gram;
// after the last mode the fit 1 - sqrt(||X||^2 + lambda^T (*G) lambda -
// 2 <M, U_raw>) / ||X|| and the stopping test |fit - fit_prev| < tol.
__global__ void __launch_bounds__(NM_THREADS) k_nm_tail(NmAls d, int n) {
    const int rep = blockIdx.x, R = d.R, N = d.s.N;
    if (d.conv[rep]) return;
    const int rows = d.s.n[n], P = d.P[n];
    __shared__ double V[32][33], V0[32][33];
    __shared__ double lam_s[32], red[8][32];
    __shared__ int bad;
    double *Gr = d.G + (long long)rep * NM_MAX * R * R;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const int a = e / R, b = e % R;
        double v = 1.0;
        for (int m = 0; m < N; ++m)
            if (m != n) v *= Gr[(long long)m * R * R + e];
        V[a][b] = v;
        V0[a][b] = v;
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (attempt == 1) {
            if (!bad) break;
            // regularised retry from the original V
            double tr = 0.0;
            for (int a = 0; a < R; ++a) tr += V0[a][a];
            __syncthreads();
            for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
                const int a = e / R, b = e % R;
                V[a][b] = V0[a][b] + (a == b ? 1e-12 * tr / R : 0.0);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                bad = 0;
                d.flags[rep] |= SBT_FLAG_CHOL_REGULARIZED_DEV;
            }
            __syncthreads();
        }
        // right-looking Cholesky, lower triangle in place
        for (int k = 0; k < R; ++k) {
            if (threadIdx.x == 0) {
                const double piv = V[k][k];
                if (!(piv > 0.0) || !isfinite(piv)) bad = 1;
                V[k][k] = piv > 0.0 ? sqrt(piv) : 1.0;
            }
            __syncthreads();
            for (int i = k + 1 + threadIdx.x; i < R; i += blockDim.x) V[i][k] /= V[k][k];
            __syncthreads();
            for (int e = threadIdx.x; e < (R - k - 1) * (R - k - 1); e += blockDim.x) {
                const int i = k + 1 + e / (R - k - 1), j = k + 1 + e % (R - k - 1);
                if (j <= i) V[i][j] -= V[i][k] * V[j][k];
            }
            __syncthreads();
        }
    }
    // U_raw = M V^-1 by forward and back substitution, one row per thread;
    // <M, U_raw> and the column squares per thread
    double *U = d.U[n] + (long long)rep * rows * R;
    const double *part = d.part + (long long)rep * d.prs;
    double sq[32], inner_p = 0.0;
    for (int r = 0; r < R; ++r) sq[r] = 0.0;
    for (int x = threadIdx.x; x < rows; x += blockDim.x) {
        double m[32], y[32];
        for (int r = 0; r < R; ++r) {
            double a = 0.0;
            for (int q = 0; q < P; ++q) a += part[((long long)q * rows + x) * R + r];
            m[r] = a;
        }
        for (int i = 0; i < R; ++i) {
            double a = m[i];
            for (int k = 0; k < i; ++k) a -= V[i][k] * y[k];
            y[i] = a / V[i][i];
        }
        for (int i = R - 1; i >= 0; --i) {
            double a = y[i];
            for (int k = i + 1; k < R; ++k) a -= V[k][i] * y[k];
            y[i] = a / V[i][i];
        }
        for (int r = 0; r < R; ++r) {
            U[(long long)x * R + r] = y[r];
            sq[r] = fma(y[r], y[r], sq[r]);
            inner_p = fma(m[r], y[r], inner_p);
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = 0; r < R; ++r) {
        const double v = warp_sum(sq[r]);
        if (lane == 0) red[warp][r] = v;
    }
    __syncthreads();
    __shared__ int zflag;
    if (threadIdx.x == 0) zflag = 0;
    __syncthreads();
    if (threadIdx.x < R) {
        double s = 0.0;
        for (int w = 0; w < NM_THREADS / 32; ++w) s += red[w][threadIdx.x];
        double l = sqrt(s);
        if (l == 0.0) {
            l = 1.0;
            zflag = 1;
        }
        lam_s[threadIdx.x] = l;
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)rows * R; e += blockDim.x) U[e] /= lam_s[e % R];
    __syncthreads();
    double *Gn = Gr + (long long)n * R * R;
    for (int pq = threadIdx.x; pq < R * R; pq += blockDim.x) {
        const int a = pq / R, b = pq % R;
        double g = 0.0;
        for (int x = 0; x < rows; ++x) g = fma(U[(long long)x * R + a], U[(long long)x * R + b], g);
        Gn[pq] = g;
    }
    if (threadIdx.x < R) d.lam[rep * R + threadIdx.x] = lam_s[threadIdx.x];
    if (threadIdx.x == 0 && zflag) d.flags[rep] |= SBT_FLAG_ZERO_COLUMN_DEV;
    if (n != N - 1) return;
    // after the last mode: the fit and the stopping test
    __shared__ double ired[8];
    const double iv = warp_sum(inner_p);
    if (lane == 0) ired[warp] = iv;
    __syncthreads();
    if (threadIdx.x == 0) {
        double inner = 0.0;
        for (int w = 0; w < NM_THREADS / 32; ++w) inner += ired[w];
        double xh = 0.0;
        for (int a = 0; a < R; ++a)
            for (int b = 0; b < R; ++b) {
                double h = 1.0;
                for (int m = 0; m < N; ++m) h *= Gr[(long long)m * R * R + a * R + b];
                xh += lam_s[a] * h * lam_s[b];
            }
        const double nx2 = d.normX2[rep];
        const double res2 = fmax(nx2 + xh - 2.0 * inner, 0.0);
        const double fit = nx2 > 0.0 ? 1.0 - sqrt(res2) / sqrt(nx2) : 0.0;
        const int it = d.iters[rep] + 1;
        d.iters[rep] = it;
        d.fit[rep] = fit;
        bool stop = it >= d.max_iters;
        if (!d.fixed_iters && fabs(fit - d.fit_prev[rep]) < d.tol) stop = true;
        d.fit_prev[rep] = fit;
        if (stop) d.conv[rep] = 1;
    }
}

// ---------------------------------------------------------------------------
// Steps 6-9 for order N, one CTA per repetition: shared-row norms nu_m (all
// rows of the non-time factors, the first nK rows of C'), cosines Gamma_m
// between unit summary columns and unit anchor columns (the old factors at the
// sampled rows), score = prod_m |Gamma_m|, Hungarian maximum (Lemma 1), and
// the new rows of C projected back: C_new(k, perm r') = lambda'_{r'}
// prod_{m != time} Gamma_m(r', r) / (lambda_r prod_{m != time} N_m(r)) *
// C'(nK + k, r') / nu_time(r').
struct NmMerge {
    int nrep, R, nK, K_new, K_old;
    NmShape s;                  // summary shape
    const double *U[NM_MAX];    // summary factors [rep][n_m][R]
    const double *lam_s;        // [rep][R]
    const double *old[NM_MAX];  // model factors (C with K_old rows)
    const double *lam;          // [R]
    const int *samples;         // [mode][rep][sstride]
    long long sstride;
    double *cnew;               // [rep][K_new][R]
    int *perm;                  // [rep][R]
    double *min_score;          // [rep]
    int *flags;                 // [rep]
};

__global__ void __launch_bounds__(NM_THREADS) k_nm_match(NmMerge g) {
    const int rep = blockIdx.x, R = g.R, N = g.s.N;
    // the N cosine matrices in dynamic shared memory: gam(m, r', r)
    extern __shared__ double nm_gam[];
    auto gam = [&](int m, int rp, int r) -> double & { return nm_gam[((long long)m * 32 + rp) * 32 + r]; };
    __shared__ double nu[NM_MAX][32], Nn[NM_MAX][32], score[32 * 32], coef[32];
    __shared__ int perm[32];
    __shared__ int zflag;
    __shared__ HungarianWork hw;
    if (threadIdx.x == 0) zflag = 0;
    __syncthreads();
    for (int m = 0; m < N; ++m) {
        const int sh = m == N - 1 ? g.nK : g.s.n[m];
        const double *U = g.U[m] + (long long)rep * g.s.n[m] * R;
        const int *S = g.samples + ((long long)m * g.nrep + rep) * g.sstride;
        const double *A = g.old[m];
        for (int it = threadIdx.x; it < R * R + 2 * R; it += blockDim.x) {
            double a = 0.0;
            if (it < R * R) {
                const int rp = it / R, r = it % R;
                for (int t = 0; t < sh; ++t) a = fma(U[(long long)t * R + rp], A[(long long)S[t] * R + r], a);
                gam(m, rp, r) = a;
            } else if (it < R * R + R) {
                const int rp = it - R * R;
                for (int t = 0; t < sh; ++t) a = fma(U[(long long)t * R + rp], U[(long long)t * R + rp], a);
                double s = sqrt(a);
                if (s == 0.0) {
                    s = 1.0;
                    zflag = 1;
                }
                nu[m][rp] = s;
            } else {
                const int r = it - R * R - R;
                for (int t = 0; t < sh; ++t) {
                    const double v = A[(long long)S[t] * R + r];
                    a = fma(v, v, a);
                }
                Nn[m][r] = sqrt(a);  // 0 stays 0 (its scale divides by it below)
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N * R * R; e += blockDim.x) {
        const int m = e / (R * R), rp = (e / R) % R, r = e % R;
        gam(m, rp, r) /= nu[m][rp] * (Nn[m][r] == 0.0 ? 1.0 : Nn[m][r]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const int rp = e / R, r = e % R;
        double sc = 1.0;
        for (int m = 0; m < N; ++m) sc *= fabs(gam(m, rp, r));
        score[rp * 32 + r] = sc;
    }
    __syncthreads();
    if (threadIdx.x < 32) hungarian_max_warp(score, 32, R, R, perm, hw, threadIdx.x);
    __syncthreads();
    if (threadIdx.x == 0) {
        double mn = INFINITY;
        for (int rp = 0; rp < R; ++rp) {
            mn = fmin(mn, score[rp * 32 + perm[rp]]);
            g.perm[rep * R + rp] = perm[rp];
        }
        g.min_score[rep] = mn;
        for (int rp = 0; rp < R; ++rp) {
            const int r = perm[rp];
            double num = g.lam_s[rep * R + rp], den = g.lam[r];
            for (int m = 0; m < N; ++m) num *= nu[m][rp];  // lambda' after the shared-row normalisation
            for (int m = 0; m < N - 1; ++m) {
                num *= gam(m, rp, r);
                den *= Nn[m][r];
            }
            coef[rp] = den != 0.0 ? num / den / nu[N - 1][rp] : 0.0;
        }
        if (zflag) g.flags[rep] |= SBT_FLAG_ZERO_COLUMN_DEV;
    }
    __syncthreads();
    const double *Ct = g.U[N - 1] + (long long)rep * g.s.n[N - 1] * R;
    double *cn = g.cnew + (long long)rep * g.K_new * R;
    for (int e = threadIdx.x; e < g.K_new * R; e += blockDim.x) {
        const int k = e / R, rp = e % R;
        cn[(long long)k * R + perm[rp]] = coef[rp] * Ct[(long long)(g.nK + k) * R + rp];
    }
}

// Marginal fold overflow check (before anything changes), then the commit:
// C rows K_old.. = mean over repetitions in order; marginals += the batch's.
__global__ void k_nm_precommit(NmW w, NmW dw, NmShape store, int N, DevStatus *status) {
    for (int m = 0; m < N - 1; ++m)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < store.n[m]; i += gridDim.x * blockDim.x)
            if (w.w[m][i] + dw.w[m][i] < w.w[m][i]) atomicOr(&status->err, ERR_RANGE);
}

__global__ void k_nm_commit(NmW w, NmW dw, NmShape store, int N, int K_old, int K_new, int nrep, int R,
                            const double *cnew, double *C, const DevStatus *status) {
    if (status->err) return;
    const long long e0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, step = (long long)gridDim.x * blockDim.x;
    for (long long e = e0; e < (long long)K_new * R; e += step) {
        double s = 0.0;
        for (int q = 0; q < nrep; ++q) s += cnew[(long long)q * K_new * R + e];
        C[(long long)K_old * R + e] = s / nrep;
    }
    for (int m = 0; m < N - 1; ++m)
        for (long long i = e0; i < store.n[m]; i += step) w.w[m][i] += dw.w[m][i];
    for (long long k = e0; k < K_new; k += step) w.w[N - 1][K_old + k] = dw.w[N - 1][k];
}

// Full-tensor fit (Section 4.2): a warp per row of the store (the innermost
// axis at fixed other indices): x_hat(j) = sum_r lambda_r prod_{m != inner}
// U_m(i_m, r) U_inner(j, r); per-warp sums of (x - x_hat)^2 and x^2 to
// scratch, added in row order by k_nm_fit_sum.
struct NmFactors {
    const double *U[NM_MAX];  // factor order, n_m x R each
};

template <typename T>
__global__ void __launch_bounds__(NM_THREADS) k_nm_fit_rows(const T *X, NmShape s, NmFactors F, const double *lam,
                                                            int R, double *scratch) {
    const double *const *Ug = F.U;
    const int N = s.N, inner = N - 2, J = s.n[inner];
    const long long rows = s.total / J;
    const long long row = (long long)blockIdx.x * (NM_THREADS / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    double pr[32];
    for (int r = 0; r < R; ++r) pr[r] = lam[r];
    long long rem = row;
    for (int m = N - 3; m >= 0; --m) {
        const int i = (int)(rem % s.n[m]);
        rem /= s.n[m];
        for (int r = 0; r < R; ++r) pr[r] *= Ug[m][(long long)i * R + r];
    }
    for (int r = 0; r < R; ++r) pr[r] *= Ug[N - 1][rem * R + r];
    double a = 0.0, b = 0.0;
    const T *x = X + row * J;
    for (int j = lane; j < J; j += 32) {
        double xh = 0.0;
        for (int r = 0; r < R; ++r) xh = fma(pr[r], Ug[inner][(long long)j * R + r], xh);
        const double xv = (double)x[j], dd = xv - xh;
        a = fma(dd, dd, a);
        b = fma(xv, xv, b);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        scratch[2 * row] = a;
        scratch[2 * row + 1] = b;
    }
}

__global__ void __launch_bounds__(NM_THREADS) k_nm_fit_sum(const double *scratch, long long rows, double *out) {
    __shared__ double ra[NM_THREADS], rb[NM_THREADS];
    double a = 0.0, b = 0.0;
    for (long long e = threadIdx.x; e < rows; e += blockDim.x) {
        a += scratch[2 * e];
        b += scratch[2 * e + 1];
    }
    ra[threadIdx.x] = a;
    rb[threadIdx.x] = b;
    __syncthreads();
    for (int h = NM_THREADS / 2; h; h >>= 1) {
        if (threadIdx.x < h) {
            ra[threadIdx.x] += ra[threadIdx.x + h];
            rb[threadIdx.x] += rb[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = ra[0];
        out[1] = rb[0];
    }
}

// ---------------------------------------------------------------------------
// launchers
static int nm_rp(int R) { return R <= 8 ? 8 : (R <= 16 ? 16 : 32); }

// partials per mode: about 4 CTAs per SM over all repetitions, at most one
// outer tuple per warp
void nm_partials(NmAls &d, int num_sms) {
    const int N = d.s.N, inner = N - 2;
    for (int n = 0; n < N; ++n) {
        const long long rowsb = n == inner ? (d.s.n[inner] + 31) / 32 : d.s.n[n];
        const long long O = d.s.total / d.s.n[n] / (n == inner ? 1 : d.s.n[inner]);
        long long P = ((long long)num_sms * 4 + rowsb * d.nrep - 1) / (rowsb * d.nrep);
        P = std::max(1LL, std::min(P, (O + 7) / 8));
        d.P[n] = (int)std::min<long long>(P, 1 << 16);
    }
}

long long nm_part_doubles(const NmAls &d) {
    long long best = 0;
    for (int n = 0; n < d.s.N; ++n) best = std::max(best, (long long)d.P[n] * d.s.n[n] * d.R);
    return best;
}

template <typename T, int RP>
static cudaError_t nm_mtt_rp(const NmAls &d, int n, cudaStream_t st) {
    const int inner = d.s.N - 2;
    if (n == inner) {
        dim3 grid((unsigned)(((d.s.n[inner] + 31) / 32) * d.P[n]), d.nrep);
        k_nm_mtt_inner<T, RP><<<grid, NM_THREADS, 0, st>>>(d);
    } else {
        using TC = typename NmCompute<T>::C;
        const size_t smem = (size_t)d.s.n[inner] * RP * sizeof(TC);
        dim3 grid((unsigned)(d.s.n[n] * d.P[n]), d.nrep);
        k_nm_mtt_outer<T, RP><<<grid, NM_THREADS, smem, st>>>(d, n);
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t nm_mtt_t(const NmAls &d, int n, cudaStream_t st) {
    const int RP = nm_rp(d.R);
    if (RP == 8) return nm_mtt_rp<T, 8>(d, n, st);
    if (RP == 16) return nm_mtt_rp<T, 16>(d, n, st);
    return nm_mtt_rp<T, 32>(d, n, st);
}

// shared memory of the outer MTTKRP (the innermost factor), above 48 KB on request
template <typename T, int RP>
static cudaError_t nm_attr_rp() {
    return cudaFuncSetAttribute(k_nm_mtt_outer<T, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t nm_set_attributes() {
    cudaError_t e = cudaFuncSetAttribute(k_nm_match, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         NM_MAX * 32 * 32 * (int)sizeof(double));
    if (e == cudaSuccess) e = nm_attr_rp<double, 8>();
    if (e == cudaSuccess) e = nm_attr_rp<double, 16>();
    if (e == cudaSuccess) e = nm_attr_rp<double, 32>();
    if (e == cudaSuccess) e = nm_attr_rp<float, 8>();
    if (e == cudaSuccess) e = nm_attr_rp<float, 16>();
    if (e == cudaSuccess) e = nm_attr_rp<float, 32>();
    return e;
}

// largest innermost summary dimension the outer MTTKRP stages (200 KB)
bool nm_supported(int J, int R, int elem) {
    return (size_t)J * nm_rp(R) * (elem == 0 ? 8 : 4) <= 200 * 1024;
}

cudaError_t launch_nm_mode(const NmAls &d, int n, cudaStream_t st) {
    count_launches(2);
    cudaError_t e = d.elem == 0 ? nm_mtt_t<double>(d, n, st) : nm_mtt_t<float>(d, n, st);
    if (e != cudaSuccess) return e;
    k_nm_tail<<<d.nrep, NM_THREADS, 0, st>>>(d, n);
    return cudaGetLastError();
}

cudaError_t launch_nm_prepare(const NmAls &d, const int *samples, long long sstride, int K_old, uint64_t seed,
                              uint32_t stream_id, uint32_t batch, cudaStream_t st) {
    count_launches(1);
    if (d.elem == 0)
        k_nm_prepare<double><<<d.nrep, NM_THREADS, 0, st>>>(d, samples, sstride, K_old, seed, stream_id, batch);
    else
        k_nm_prepare<float><<<d.nrep, NM_THREADS, 0, st>>>(d, samples, sstride, K_old, seed, stream_id, batch);
    return cudaGetLastError();
}

cudaError_t launch_nm_merge(const NmMerge &g, const NmW &w, const NmW &dw, const NmShape &store, DevStatus *status,
                            cudaStream_t st) {
    count_launches(3);
    k_nm_match<<<g.nrep, NM_THREADS, (size_t)g.s.N * 32 * 32 * sizeof(double), st>>>(g);
    k_nm_precommit<<<64, 256, 0, st>>>(w, dw, store, g.s.N, status);
    k_nm_commit<<<64, 256, 0, st>>>(w, dw, store, g.s.N, g.K_old, g.K_new, g.nrep, g.R, g.cnew,
                                    const_cast<double *>(g.old[g.s.N - 1]), status);
    return cudaGetLastError();
}

cudaError_t launch_nm_fit(const void *X, int dtype, const NmShape &s, const NmFactors &F, const double *lam, int R,
                          double *scratch, double *out, cudaStream_t st) {
    const long long rows = s.total / s.n[s.N - 2];
    const unsigned blocks = (unsigned)((rows + NM_THREADS / 32 - 1) / (NM_THREADS / 32));
    count_launches(2);
    if (dtype == SBT_F64)
        k_nm_fit_rows<double><<<blocks, NM_THREADS, 0, st>>>((const double *)X, s, F, lam, R, scratch);
    else
        k_nm_fit_rows<float><<<blocks, NM_THREADS, 0, st>>>((const float *)X, s, F, lam, R, scratch);
    k_nm_fit_sum<<<1, NM_THREADS, 0, st>>>(scratch, rows, out);
    return cudaGetLastError();
}

}  // namespace sbt

// ===========================================================================
// C ABI of the order-N path
using namespace sbt;

namespace {

sbt_status nfail(sbt_status s, const std::string &msg) {
    set_last_error(msg);
    return s;
}

#define NCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return nfail(e_ == cudaErrorMemoryAllocation ? SBT_E_NOMEM : SBT_E_CUDA,                \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

#define NTRY(expr)                    \
    do {                              \
        sbt_status s_ = (expr);       \
        if (s_ != SBT_OK) return s_;  \
    } while (0)

// device buffer that only grows (contents are not kept when it grows)
struct NBuf {
    void *p = nullptr;
    size_t cap = 0;
    ~NBuf() {
        if (p) cudaFree(p);
    }
    sbt_status ensure(size_t bytes) {
        if (bytes <= cap) return SBT_OK;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        const size_t want = std::max<size_t>(bytes, 256);
        const cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            p = nullptr;
            return nfail(SBT_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        cap = want;
        return SBT_OK;
    }
    template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

// pinned host buffer (status words and statistics read back by the host)
struct NHBuf {
    void *p = nullptr;
    size_t cap = 0;
    ~NHBuf() {
        if (p) cudaFreeHost(p);
    }
    sbt_status ensure(size_t bytes) {
        if (bytes <= cap) return SBT_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        const size_t want = std::max<size_t>(bytes, 256);
        if (cudaMallocHost(&p, want) != cudaSuccess) {
            p = nullptr;
            return nfail(SBT_E_NOMEM, "cudaMallocHost failed");
        }
        cap = want;
        return SBT_OK;
    }
    template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

std::mutex g_nm_attr_mu;
bool g_nm_attr_done[64] = {};

}  // namespace

struct sbt_nmode {
    int device = 0, num_sms = 0;
    cudaStream_t user = nullptr, stream = nullptr;
    cudaEvent_t ev_user = nullptr;
    sbt_options opt{};
    int N = 3, R = 0, sdtype = SBT_F32, S = 0;
    int dims[NM_MAX] = {};   // factor order; dims[N-1] = K
    int64_t K = 0, Kcap = 0;
    uint32_t batch = 0;
    int64_t npos[NM_MAX] = {};
    NBuf store, lam, status, U[NM_MAX], w[NM_MAX], dw[NM_MAX];
    NBuf samples, khi, klo, Xs, Us[NM_MAX], part, G, lam_s, fit, fit_prev, normX2, iters, conv, flags;
    NBuf cnew, perm, min_score, fitscr;
    NHBuf hstat;  // host
    bool have_last = false;
    int last_n[NM_MAX] = {};
    long long last_sstride = 0;
    sbt_update_stats stats{};
    ~sbt_nmode() {
        if (ev_user) cudaEventDestroy(ev_user);
        if (stream) cudaStreamDestroy(stream);
    }
    size_t es() const { return sdtype == SBT_F64 ? 8 : 4; }
    long long slice_elems() const {
        long long e = 1;
        for (int m = 0; m < N - 1; ++m) e *= dims[m];
        return e;
    }
    NmShape store_shape(long long K_rows) const {
        int n[NM_MAX];
        for (int m = 0; m < N - 1; ++m) n[m] = dims[m];
        n[N - 1] = (int)K_rows;
        return nm_shape(N, n);
    }
    NmW marg() {
        NmW a{};
        for (int m = 0; m < N; ++m) a.w[m] = w[m].as<unsigned long long>();
        return a;
    }
};

static sbt_status nm_check_tensor(const sbt_tensor_n *X) {
    if (!X) return nfail(SBT_E_INVALID, "null tensor");
    if (X->N < 3 || X->N > SBT_NMODE_MAX) return nfail(SBT_E_INVALID, "N out of range [3, SBT_NMODE_MAX]");
    if (!X->data) return nfail(SBT_E_INVALID, "null tensor data");
    if (X->dtype != SBT_F64 && X->dtype != SBT_F32) return nfail(SBT_E_INVALID, "dtype must be SBT_F64 or SBT_F32");
    long long total = 1;
    for (int a = 0; a < X->N; ++a) {
        if (X->dims[a] < 1 || X->dims[a] > (1 << 30)) return nfail(SBT_E_SHAPE, "dimensions must be in [1, 2^30]");
        total *= X->dims[a];
        if (total > (1LL << 40)) return nfail(SBT_E_SHAPE, "tensor too large");
    }
    return SBT_OK;
}

static sbt_status nm_check_options(const sbt_options *o, int R) {
    if (!o) return nfail(SBT_E_INVALID, "null options");
    if (o->s_I < 1 || o->s_J < 1 || o->s_K < 1) return nfail(SBT_E_INVALID, "sampling factors must be >= 1");
    if (o->r < 1 || o->r > SBT_MAX_REPS) return nfail(SBT_E_INVALID, "r out of range [1, SBT_MAX_REPS]");
    if (R < 1 || R > SBT_MAX_RANK) return nfail(SBT_E_INVALID, "R out of range [1, SBT_MAX_RANK]");
    if (o->max_iters < 1) return nfail(SBT_E_INVALID, "max_iters must be >= 1");
    if (!(o->tol >= 0.0)) return nfail(SBT_E_INVALID, "tol must be >= 0");
    if (o->prec != SBT_PREC_F64 && o->prec != SBT_PREC_F32)
        return nfail(SBT_E_INVALID, "order-N tensors take SBT_PREC_F64 or SBT_PREC_F32");
    if (o->lambda_mode || o->refine_sweeps || o->autotune || o->mode3_pass || o->warm_start || o->get_rank ||
        o->max_batch)
        return nfail(SBT_E_INVALID, "option not available for order-N tensors");
    return SBT_OK;
}

// upload (or copy) K slices to the store at slice K0 and add their Eq. 1
// marginals into w (non-time modes) and wt (the slices')
static sbt_status nm_append(sbt_nmode *c, const sbt_tensor_n *X, int64_t K0, const NmW &w) {
    const long long se = c->slice_elems();
    char *dst = c->store.as<char>() + (size_t)K0 * se * c->es();
    const size_t bytes = (size_t)X->dims[0] * se * c->es();
    NCK(cudaMemcpyAsync(dst, X->data, bytes, X->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        c->stream));
    NCK(launch_nm_append(dst, dst, c->sdtype, c->store_shape(X->dims[0]), c->S, w, c->status.as<DevStatus>(),
                         c->stream));
    return SBT_OK;
}

static sbt_status nm_read_status(sbt_nmode *c, DevStatus *out) {
    NCK(cudaMemcpyAsync(c->hstat.p, c->status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
    NCK(cudaStreamSynchronize(c->stream));
    std::memcpy(out, c->hstat.p, sizeof(DevStatus));
    return SBT_OK;
}

// positive-weight counts of every mode's marginal (the time mode over K slices)
static sbt_status nm_count_positive(sbt_nmode *c) {
    for (int m = 0; m < c->N; ++m) {
        const int64_t len = m == c->N - 1 ? c->K : c->dims[m];
        std::vector<unsigned long long> h(len);
        NCK(cudaMemcpy(h.data(), c->w[m].p, (size_t)len * 8, cudaMemcpyDeviceToHost));
        int64_t cnt = 0;
        for (auto v : h) cnt += v != 0;
        c->npos[m] = cnt;
    }
    return SBT_OK;
}

extern "C" sbt_status sbt_nmode_init_factors(const sbt_tensor_n *X0, int32_t R, const double *lambda,
                                             const double *const *U, const sbt_options *opt, sbt_nmode **out) {
    if (!out) return nfail(SBT_E_INVALID, "null output pointer");
    *out = nullptr;
    NTRY(nm_check_tensor(X0));
    NTRY(nm_check_options(opt, R));
    if (!lambda || !U) return nfail(SBT_E_INVALID, "null factors");
    for (int m = 0; m < X0->N; ++m)
        if (!U[m]) return nfail(SBT_E_INVALID, "null factor");
    if ((opt->prec == SBT_PREC_F64) != (X0->dtype == SBT_F64))
        return nfail(SBT_E_INVALID, "SBT_PREC_F64 takes a float64 tensor, SBT_PREC_F32 a float32 one");
    sbt_nmode *c = new sbt_nmode();
    auto bail = [&](sbt_status s) {
        delete c;
        return s;
    };
    c->opt = *opt;
    c->N = X0->N;
    c->R = R;
    c->sdtype = X0->dtype;
    for (int m = 0; m < c->N - 1; ++m) c->dims[m] = (int)X0->dims[m + 1];
    c->K = X0->dims[0];
    c->dims[c->N - 1] = (int)c->K;
    c->Kcap = std::max<int64_t>(opt->K_capacity > 0 ? opt->K_capacity : 2 * c->K, c->K + 1);
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return bail(nfail(SBT_E_CUDA, "no usable CUDA device"));
    {
        std::lock_guard<std::mutex> lock(g_nm_attr_mu);
        if (c->device >= 0 && c->device < 64 && !g_nm_attr_done[c->device]) {
            if (nm_set_attributes() != cudaSuccess) return bail(nfail(SBT_E_CUDA, "kernel attributes"));
            g_nm_attr_done[c->device] = true;
        }
    }
    c->user = (cudaStream_t)opt->cuda_stream;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_user, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(c->ev_user, c->user) != cudaSuccess || cudaStreamWaitEvent(c->stream, c->ev_user, 0) != cudaSuccess)
        return bail(nfail(SBT_E_CUDA, "stream set-up failed"));
    sbt_status s = c->store.ensure((size_t)c->Kcap * c->slice_elems() * c->es());
    if (s == SBT_OK) s = c->lam.ensure((size_t)R * 8);
    if (s == SBT_OK) s = c->status.ensure(sizeof(DevStatus));
    if (s == SBT_OK) s = c->hstat.ensure(sizeof(DevStatus));
    for (int m = 0; m < c->N && s == SBT_OK; ++m) {
        const int64_t rows = m == c->N - 1 ? c->Kcap : c->dims[m];
        s = c->U[m].ensure((size_t)rows * R * 8);
        if (s == SBT_OK) s = c->w[m].ensure((size_t)rows * 8);
        if (s == SBT_OK) s = c->dw[m].ensure((size_t)rows * 8);
    }
    if (s != SBT_OK) return bail(s);
    for (int m = 0; m < c->N; ++m)
        if (cudaMemsetAsync(c->w[m].p, 0, c->w[m].cap, c->stream) != cudaSuccess)
            return bail(nfail(SBT_E_CUDA, "memset"));
    if (cudaMemsetAsync(c->status.p, 0, sizeof(DevStatus), c->stream) != cudaSuccess)
        return bail(nfail(SBT_E_CUDA, "memset"));
    // X0 into the store, the shift S from max |x| (Eq. 1 fixed point), then the marginals
    const size_t bytes = (size_t)c->K * c->slice_elems() * c->es();
    if (cudaMemcpyAsync(c->store.p, X0->data, bytes, X0->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess ||
        launch_absmax(c->store.p, c->sdtype, (long long)(bytes / c->es()), c->status.as<DevStatus>(), c->stream) !=
            cudaSuccess)
        return bail(nfail(SBT_E_CUDA, "X0 upload"));
    DevStatus hs;
    s = nm_read_status(c, &hs);
    if (s != SBT_OK) return bail(s);
    if (hs.err & ERR_NONFINITE) return bail(nfail(SBT_E_NONFINITE, "non-finite value in X0"));
    double M;
    std::memcpy(&M, &hs.amax_bits, 8);
    int e2 = 0;
    if (M != 0.0) std::frexp(M * M, &e2);
    c->S = M == 0.0 ? 0 : 32 - e2;
    if (launch_nm_append(c->store.p, c->store.p, c->sdtype, c->store_shape(c->K), c->S, c->marg(),
                         c->status.as<DevStatus>(), c->stream) != cudaSuccess)
        return bail(nfail(SBT_E_CUDA, "marginals"));
    s = nm_read_status(c, &hs);
    if (s != SBT_OK) return bail(s);
    if (hs.err & ERR_NONFINITE) return bail(nfail(SBT_E_NONFINITE, "non-finite value in X0"));
    if (hs.err & ERR_RANGE) return bail(nfail(SBT_E_RANGE, "fixed-point marginal would overflow 64 bits"));
    for (int m = 0; m < c->N; ++m) {
        const int64_t rows = m == c->N - 1 ? c->K : c->dims[m];
        if (cudaMemcpy(c->U[m].p, U[m], (size_t)rows * R * 8, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(nfail(SBT_E_CUDA, "factor upload"));
    }
    if (cudaMemcpy(c->lam.p, lambda, (size_t)R * 8, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(nfail(SBT_E_CUDA, "lambda upload"));
    s = nm_count_positive(c);
    if (s != SBT_OK) return bail(s);
    *out = c;
    return SBT_OK;
}

// grow the store, C and the time marginal to at least `need` slices
static sbt_status nm_grow(sbt_nmode *c, int64_t need) {
    if (need <= c->Kcap) return SBT_OK;
    const int64_t ncap = std::max<int64_t>(need, 2 * c->Kcap);
    const size_t slice = (size_t)c->slice_elems() * c->es();
    const int T = c->N - 1;
    NBuf ns, nC, nw;
    NTRY(ns.ensure((size_t)ncap * slice));
    NTRY(nC.ensure((size_t)ncap * c->R * 8));
    NTRY(nw.ensure((size_t)ncap * 8));
    NTRY(c->dw[T].ensure((size_t)ncap * 8));
    NCK(cudaMemcpyAsync(ns.p, c->store.p, (size_t)c->K * slice, cudaMemcpyDeviceToDevice, c->stream));
    NCK(cudaMemcpyAsync(nC.p, c->U[T].p, (size_t)c->K * c->R * 8, cudaMemcpyDeviceToDevice, c->stream));
    NCK(cudaMemsetAsync(nw.p, 0, (size_t)ncap * 8, c->stream));
    NCK(cudaMemcpyAsync(nw.p, c->w[T].p, (size_t)c->K * 8, cudaMemcpyDeviceToDevice, c->stream));
    NCK(cudaStreamSynchronize(c->stream));
    std::swap(c->store.p, ns.p);
    std::swap(c->store.cap, ns.cap);
    std::swap(c->U[T].p, nC.p);
    std::swap(c->U[T].cap, nC.cap);
    std::swap(c->w[T].p, nw.p);
    std::swap(c->w[T].cap, nw.cap);
    c->Kcap = ncap;
    return SBT_OK;
}

extern "C" sbt_status sbt_nmode_update(sbt_nmode *c, const sbt_tensor_n *X) {
    if (!c) return nfail(SBT_E_INVALID, "null context");
    NTRY(nm_check_tensor(X));
    if (X->N != c->N || X->dtype != c->sdtype) return nfail(SBT_E_SHAPE, "N and dtype must match the initial tensor");
    for (int m = 0; m < c->N - 1; ++m)
        if (X->dims[m + 1] != c->dims[m]) return nfail(SBT_E_SHAPE, "non-time dimensions must match the initial tensor");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    struct Restore {
        int d;
        ~Restore() {
            if (d >= 0) cudaSetDevice(d);
        }
    } restore{prev};
    NCK(cudaEventRecord(c->ev_user, c->user));
    NCK(cudaStreamWaitEvent(c->stream, c->ev_user, 0));
    const int N = c->N, R = c->R, r = c->opt.r, T = N - 1;
    const int K_new = (int)X->dims[0];
    const int64_t K_old = c->K;
    NTRY(nm_grow(c, K_old + K_new));
    // sample sizes (Section 3.1): ceil(dim / s), clamped to the positive weights
    int n[NM_MAX];
    long long sstride = 0, kstride = K_old;
    for (int m = 0; m < N; ++m) {
        const int sm = m == T ? c->opt.s_K : (m == 1 ? c->opt.s_J : c->opt.s_I);
        const int64_t dim = m == T ? K_old : c->dims[m];
        n[m] = (int)std::min<int64_t>((dim + sm - 1) / sm, c->npos[m]);
        if (n[m] < 1) return nfail(SBT_E_STATE, "a mode has no positive weight to sample");
        sstride = std::max<long long>(sstride, n[m]);
        if (m < T) kstride = std::max<long long>(kstride, c->dims[m]);
    }
    const int nK = n[T];
    int ns[NM_MAX];
    for (int m = 0; m < N; ++m) ns[m] = n[m];
    ns[T] = nK + K_new;
    const NmShape ss = nm_shape(N, ns);
    const int elem = c->sdtype == SBT_F64 ? 0 : 1;
    if (!nm_supported(ns[N - 2], R, elem))
        return nfail(SBT_E_INVALID, "the summary's last dimension is beyond the order-N MTTKRP's shared-memory plan");
    NmAls d{};
    d.nrep = r;
    d.R = R;
    d.nK = nK;
    d.s = ss;
    d.elem = elem;
    d.tol = c->opt.tol;
    d.max_iters = c->opt.max_iters;
    d.fixed_iters = c->opt.fixed_iters;
    nm_partials(d, c->num_sms);
    d.prs = nm_part_doubles(d);
    // workspace
    NTRY(c->samples.ensure((size_t)N * r * sstride * 4));
    NTRY(c->khi.ensure((size_t)r * kstride * 8));
    NTRY(c->klo.ensure((size_t)r * kstride * 8));
    NTRY(c->Xs.ensure((size_t)r * ss.total * c->es()));
    for (int m = 0; m < N; ++m) NTRY(c->Us[m].ensure((size_t)r * ns[m] * R * 8));
    NTRY(c->part.ensure((size_t)r * d.prs * 8));
    NTRY(c->G.ensure((size_t)r * NM_MAX * R * R * 8));
    NTRY(c->lam_s.ensure((size_t)r * R * 8));
    NTRY(c->fit.ensure((size_t)r * 8));
    NTRY(c->fit_prev.ensure((size_t)r * 8));
    NTRY(c->normX2.ensure((size_t)r * 8));
    NTRY(c->iters.ensure((size_t)r * 4));
    NTRY(c->conv.ensure((size_t)r * 4));
    NTRY(c->flags.ensure((size_t)r * 4));
    NTRY(c->cnew.ensure((size_t)r * K_new * R * 8));
    NTRY(c->perm.ensure((size_t)r * R * 4));
    NTRY(c->min_score.ensure((size_t)r * 8));
    NTRY(c->hstat.ensure(sizeof(DevStatus) + (size_t)r * (4 + 8 + 8 + 4 + 4 * R)));
    // 1. append + marginal deltas
    NmW dw{};
    for (int m = 0; m < N; ++m) {
        dw.w[m] = c->dw[m].as<unsigned long long>();
        NCK(cudaMemsetAsync(c->dw[m].p, 0, (size_t)(m == T ? K_new : c->dims[m]) * 8, c->stream));
    }
    NCK(cudaMemsetAsync(c->status.p, 0, sizeof(DevStatus), c->stream));
    NTRY(nm_append(c, X, K_old, dw));
    // 2. sampling from the marginals before the update, one launch per mode
    int *smp = c->samples.as<int>();
    for (int m = 0; m < N; ++m) {
        SampleParams sp;
        std::memset(&sp, 0, sizeof(sp));
        sp.w[0] = c->w[m].as<unsigned long long>();
        sp.N[0] = m == T ? (int)K_old : c->dims[m];
        sp.n[0] = n[m];
        sp.mode_id[0] = m;
        sp.nmodes = 1;
        sp.nrep = r;
        sp.rep0 = 0;
        sp.out = smp + (long long)m * r * sstride;
        sp.out_stride = sstride;
        sp.khi = c->khi.as<unsigned long long>();
        sp.klo = c->klo.as<unsigned long long>();
        sp.key_stride = kstride;
        sp.seed = c->opt.seed;
        sp.stream_id = c->opt.stream_id;
        sp.batch = c->batch;
        sp.status = c->status.as<DevStatus>();
        NCK(launch_sample(sp, c->stream));
    }
    // 3. the summaries
    NCK(launch_nm_gather(c->store.p, c->sdtype, c->store_shape(c->Kcap), ss, smp, sstride, r, nK, (int)K_old,
                         c->Xs.p, c->stream));
    // 4. CP-ALS over all N modes
    d.X = c->Xs.p;
    for (int m = 0; m < N; ++m) d.U[m] = c->Us[m].as<double>();
    d.part = c->part.as<double>();
    d.G = c->G.as<double>();
    d.lam = c->lam_s.as<double>();
    d.fit = c->fit.as<double>();
    d.fit_prev = c->fit_prev.as<double>();
    d.normX2 = c->normX2.as<double>();
    d.iters = c->iters.as<int>();
    d.conv = c->conv.as<int>();
    d.flags = c->flags.as<int>();
    NCK(launch_nm_prepare(d, smp, sstride, (int)K_old, c->opt.seed, c->opt.stream_id, c->batch, c->stream));
    const int every = c->opt.check_every > 0 ? c->opt.check_every : 4;
    std::vector<int> hconv(r);
    for (int it = 0; it < d.max_iters; it += every) {
        const int nit = std::min(every, d.max_iters - it);
        for (int q = 0; q < nit; ++q)
            for (int m = 0; m < N; ++m) NCK(launch_nm_mode(d, m, c->stream));
        if (d.fixed_iters && it + nit < d.max_iters) continue;
        NCK(cudaMemcpyAsync(hconv.data(), d.conv, (size_t)r * 4, cudaMemcpyDeviceToHost, c->stream));
        NCK(cudaStreamSynchronize(c->stream));
        bool all = true;
        for (int q = 0; q < r; ++q) all = all && hconv[q];
        if (all) break;
    }
    // 5.-6. normalise, match, project back; commit
    NmMerge g{};
    g.nrep = r;
    g.R = R;
    g.nK = nK;
    g.K_new = K_new;
    g.K_old = (int)K_old;
    g.s = ss;
    for (int m = 0; m < N; ++m) {
        g.U[m] = c->Us[m].as<double>();
        g.old[m] = c->U[m].as<double>();
    }
    g.lam_s = d.lam;
    g.lam = c->lam.as<double>();
    g.samples = smp;
    g.sstride = sstride;
    g.cnew = c->cnew.as<double>();
    g.perm = c->perm.as<int>();
    g.min_score = c->min_score.as<double>();
    g.flags = d.flags;
    NCK(launch_nm_merge(g, c->marg(), dw, c->store_shape(c->Kcap), c->status.as<DevStatus>(), c->stream));
    // status and statistics, one synchronisation
    char *hb = c->hstat.as<char>();
    size_t off = 0;
    NCK(cudaMemcpyAsync(hb, c->status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
    off += sizeof(DevStatus);
    NCK(cudaMemcpyAsync(hb + off, d.iters, (size_t)r * 4, cudaMemcpyDeviceToHost, c->stream));
    NCK(cudaMemcpyAsync(hb + off + (size_t)r * 4, d.fit, (size_t)r * 8, cudaMemcpyDeviceToHost, c->stream));
    NCK(cudaMemcpyAsync(hb + off + (size_t)r * 12, g.min_score, (size_t)r * 8, cudaMemcpyDeviceToHost, c->stream));
    NCK(cudaMemcpyAsync(hb + off + (size_t)r * 20, d.flags, (size_t)r * 4, cudaMemcpyDeviceToHost, c->stream));
    NCK(cudaMemcpyAsync(hb + off + (size_t)r * 24, g.perm, (size_t)r * R * 4, cudaMemcpyDeviceToHost, c->stream));
    NCK(cudaStreamSynchronize(c->stream));
    DevStatus hs;
    std::memcpy(&hs, hb, sizeof(DevStatus));
    if (hs.err & ERR_NONFINITE) return nfail(SBT_E_NONFINITE, "non-finite value in the new slices");
    if (hs.err & ERR_RANGE) return nfail(SBT_E_RANGE, "fixed-point marginal would overflow 64 bits");
    if (hs.err & ERR_SAMPLE) return nfail(SBT_E_STATE, "sample size above the number of positive weights");
    if (hs.err) return nfail(SBT_E_CUDA, "device error in the update");
    c->K = K_old + K_new;
    c->dims[T] = (int)c->K;
    c->batch += 1;
    NTRY(nm_count_positive(c));
    sbt_update_stats &st = c->stats;
    std::memset(&st, 0, sizeof(st));
    st.K = c->K;
    st.r = r;
    st.R = R;
    st.n_I = n[0];
    st.n_J = n[1];
    st.n_K = nK;
    const int *it = (const int *)(hb + off);
    const double *ft = (const double *)(hb + off + (size_t)r * 4);
    const double *ms = (const double *)(hb + off + (size_t)r * 12);
    const int *fl = (const int *)(hb + off + (size_t)r * 20);
    const int *pm = (const int *)(hb + off + (size_t)r * 24);
    int nmin = nK;
    for (int m = 0; m < T; ++m) nmin = std::min(nmin, n[m]);
    if (nmin < R) st.flags |= SBT_FLAG_SAMPLE_LT_RANK;
    for (int q = 0; q < r; ++q) {
        st.iters[q] = it[q];
        st.fit[q] = ft[q];
        st.min_score[q] = ms[q];
        st.flags |= fl[q];
        st.rank[q] = R;
        for (int a = 0; a < R; ++a) st.perm[q][a] = pm[q * R + a];
    }
    c->have_last = true;
    for (int m = 0; m < N; ++m) c->last_n[m] = n[m];
    c->last_sstride = sstride;
    return SBT_OK;
}

extern "C" sbt_status sbt_nmode_factors(const sbt_nmode *c, double *lambda, double *const *U, int64_t *K_out) {
    if (!c) return nfail(SBT_E_INVALID, "null context");
    NCK(cudaStreamSynchronize(c->stream));
    if (lambda) NCK(cudaMemcpy(lambda, c->lam.p, (size_t)c->R * 8, cudaMemcpyDeviceToHost));
    if (U)
        for (int m = 0; m < c->N; ++m)
            if (U[m]) {
                const int64_t rows = m == c->N - 1 ? c->K : c->dims[m];
                NCK(cudaMemcpy(U[m], c->U[m].p, (size_t)rows * c->R * 8, cudaMemcpyDeviceToHost));
            }
    if (K_out) *K_out = c->K;
    return SBT_OK;
}

extern "C" sbt_status sbt_nmode_fit(sbt_nmode *c, double *fit) {
    if (!c || !fit) return nfail(SBT_E_INVALID, "null argument");
    const NmShape s = c->store_shape(c->K);
    const long long rows = s.total / s.n[c->N - 2];
    NTRY(c->fitscr.ensure((size_t)(2 * rows + 2) * 8));
    double *scr = c->fitscr.as<double>();
    NmFactors F{};
    for (int m = 0; m < c->N; ++m) F.U[m] = c->U[m].as<double>();
    NCK(launch_nm_fit(c->store.p, c->sdtype, s, F, c->lam.as<double>(), c->R, scr, scr + 2 * rows, c->stream));
    double h[2];
    NCK(cudaMemcpyAsync(h, scr + 2 * rows, 16, cudaMemcpyDeviceToHost, c->stream));
    NCK(cudaStreamSynchronize(c->stream));
    *fit = h[1] > 0.0 ? 1.0 - std::sqrt(h[0]) / std::sqrt(h[1]) : 0.0;
    return SBT_OK;
}

extern "C" sbt_status sbt_nmode_stats(const sbt_nmode *c, sbt_update_stats *st) {
    if (!c || !st) return nfail(SBT_E_INVALID, "null argument");
    if (!c->have_last) return nfail(SBT_E_STATE, "no update has run");
    *st = c->stats;
    return SBT_OK;
}

extern "C" sbt_status sbt_nmode_last_samples(const sbt_nmode *c, int32_t rep, int32_t mode, int32_t *out,
                                             int64_t cap, int64_t *n) {
    if (!c || !n) return nfail(SBT_E_INVALID, "null argument");
    if (!c->have_last) return nfail(SBT_E_STATE, "no update has run");
    if (rep < 0 || rep >= c->opt.r || mode < 0 || mode >= c->N) return nfail(SBT_E_INVALID, "rep or mode out of range");
    *n = c->last_n[mode];
    if (out && cap > 0) {
        const int64_t cnt = std::min<int64_t>(cap, *n);
        NCK(cudaMemcpy(out, c->samples.as<int>() + ((long long)mode * c->opt.r + rep) * c->last_sstride,
                       (size_t)cnt * 4, cudaMemcpyDeviceToHost));
    }
    return SBT_OK;
}

extern "C" void sbt_nmode_destroy(sbt_nmode *c) { delete c; }
