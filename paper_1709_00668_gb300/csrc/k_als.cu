// CP-ALS on the r summaries (Alg. 1 step 5), batched over repetitions.
//
// Per iteration and mode n: MTTKRP partial sums (one CTA per tile, no atomics)
// and a tail that solves U_n = M_n V^-1 with V the Hadamard product of the
// other modes' Grams, normalises the columns (lambda) and refreshes the Gram;
// after mode 3 the tail also computes the fit and the convergence flag.
//
// float64 summaries: a fixed-order reduction of the partials, then one CTA per
// repetition factors V (float64 Cholesky in one warp) and does the rest.
// float32 / bfloat16 summaries (float32 factors): float64 is a slow unit on
// this GPU, so the R x R work is done in double-float (pairs of floats with
// error-free sums and products, ~44 significant bits).  V^-1 (Gauss-Jordan)
// is computed by k_xinv on a side stream while the MTTKRP runs (for a mode 3
// formed from the mode-2 pass's products, by k_mtt_memo beside that
// contraction); k_tail_rows then reduces the partials of 16 rows per CTA,
// forms U = M V^-1 and the chunk's share of the new Gram.  The chunks of a
// repetition form one thread-block cluster (up to 16 CTAs): every CTA adds
// the shares from distributed shared memory in chunk order, takes lambda and
// writes its rows of U normalised.  Larger modes use an atomic ticket: the
// last CTA to finish combines the shares, takes lambda, rescales U and, after
// mode 3, computes the fit.
// Every reduction runs in a fixed order, so results do not depend on timing.
#include "sbt_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

namespace sbt {

static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void count_launches(int n) { g_launches += n; }

// ---------------------------------------------------------------------------
// vector loads of summary elements (16 bytes) widened to the factor type
template <typename TX, typename TF> struct VecLd;
template <> struct VecLd<float, float> {
    static constexpr int V = 4;
    static __device__ __forceinline__ void ld(const float *p, float (&o)[4]) {
        float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <> struct VecLd<double, double> {
    static constexpr int V = 2;
    static __device__ __forceinline__ void ld(const double *p, double (&o)[2]) {
        double2 v = *reinterpret_cast<const double2 *>(p);
        o[0] = v.x; o[1] = v.y;
    }
};
template <> struct VecLd<__nv_bfloat16, float> {
    static constexpr int V = 8;
    static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, float (&o)[8]) {
        uint4 v = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            o[2 * t] = __uint_as_float(w[t] << 16);
            o[2 * t + 1] = __uint_as_float(w[t] & 0xFFFF0000u);
        }
    }
};

// Reduce-scatter of RP per-lane values over a warp: lane l ends with the
// total of value l / (32 / RP).  log2(RP) halving exchanges, then plain sums.
template <int RP, typename T>
__device__ __forceinline__ T warp_reduce_scatter(T (&v)[RP], int lane) {
    int o = 16;
#pragma unroll
    for (int half = RP / 2; half >= 1; half >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int t = 0; t < half; ++t) {
            T send = up ? v[t] : v[t + half];
            T keep = up ? v[t + half] : v[t];
            v[t] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
        o >>= 1;
    }
    for (; o >= 1; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    return v[0];
}

template <typename TF>
__global__ void k_store_m(const double *M, TF *out, long long cnt) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < cnt) out[e] = (TF)M[e];
}

template <typename TX> struct FactorOf { using T = float; };
template <> struct FactorOf<double> { using T = double; };

// ---------------------------------------------------------------------------
// Row kernel: modes 1 and 3.  A CTA owns 8 rows ii (one per warp) and a range
// of slices kk; z(kk, ii, :) = X[kk][ii][:] . B is formed with B^T staged in
// shared memory (column chunks of jc), then
//   mode 1: part[ks][ii][r] = sum_kk z(kk,ii,r) C(kk,r)
//   mode 3: part[ib][kk][r] = sum_ii z(kk,ii,r) A(ii,r)
template <typename TX, int RP>
__device__ void mtt_row_block(const AlsDesc &d, int mode, int bx, int rep, unsigned char *smem_raw) {
    using TF = typename FactorOf<TX>::T;
    constexpr int V = VecLd<TX, TF>::V;
    if (d.conv[rep]) return;
    const int NI = d.n[0], NJ = d.n[1], Kp = d.n[2], R = d.R, ldj = d.ldj;
    const int ib = bx % d.nib, ks = bx / d.nib;
    const int k0 = ks * d.spc, k1 = min(Kp, k0 + d.spc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ii = ib * 8 + warp;
    const int jc = d.jc;
    TF *Bt = reinterpret_cast<TF *>(smem_raw);               // [RP][jc]
    TF *z = Bt + (size_t)RP * jc;                            // [spc][8][RP]
    const TF *A = (const TF *)d.U[0] + (long long)rep * NI * R;
    const TF *B = (const TF *)d.U[1] + (long long)rep * NJ * R;
    const TF *C = (const TF *)d.U[2] + (long long)rep * Kp * R;
    const TX *X = (const TX *)d.X + rep * d.xrs;
    const int nkk = max(0, k1 - k0);
    if (d.bytes_ctr && threadIdx.x == 0) {
        const int rows = min(8, NI - ib * 8);
        atomicAdd(d.bytes_ctr, (unsigned long long)rows * nkk * NJ * sizeof(TX));
    }
    const int lane_r = lane / (32 / RP);
    const bool lane_writes = (lane % (32 / RP)) == 0 && lane_r < R;

    for (int c0 = 0; c0 < NJ; c0 += jc) {
        const int c1 = min(NJ, c0 + jc);
        __syncthreads();
        for (int e = threadIdx.x; e < RP * jc; e += blockDim.x) {
            int r = e / jc, j = c0 + e % jc;
            Bt[e] = (r < R && j < c1) ? B[(long long)j * R + r] : TF(0);
        }
        __syncthreads();
        if (ii < NI) {
            for (int t = 0; t < nkk; ++t) {
                const TX *xr = X + ((long long)(k0 + t) * NI + ii) * ldj;
                TF acc[RP];
#pragma unroll
                for (int r = 0; r < RP; ++r) acc[r] = TF(0);
                for (int jj = c0 + lane * V; jj < c1; jj += 32 * V) {
                    TF xv[V];
                    VecLd<TX, TF>::ld(xr + jj, xv);
#pragma unroll
                    for (int u = 0; u < V; ++u)
                        if (jj + u >= c1) xv[u] = TF(0);
                    const TF *bt = Bt + (jj - c0);
#pragma unroll
                    for (int r = 0; r < RP; ++r) {
                        if (r < R) {
#pragma unroll
                            for (int u = 0; u < V; ++u) acc[r] = fmadd(xv[u], bt[r * jc + u], acc[r]);
                        }
                    }
                }
                TF zr = warp_reduce_scatter<RP>(acc, lane);
                if (lane_writes) {
                    TF *zp = z + ((size_t)t * 8 + warp) * RP + lane_r;
                    *zp = (c0 == 0) ? zr : *zp + zr;
                }
            }
        }
    }
    __syncthreads();
    TF *part = (TF *)d.part + rep * d.prs;
    if (mode == 0) {
        // part[ks][ii][r]
        if (ii < NI && lane < R) {
            TF s = TF(0);
            for (int t = 0; t < nkk; ++t) s = fmadd(z[((size_t)t * 8 + warp) * RP + lane], C[(long long)(k0 + t) * R + lane], s);
            part[((long long)ks * NI + ii) * d.pr + lane] = s;
        }
    } else {
        // part[ib][kk][r]
        for (int e = threadIdx.x; e < nkk * R; e += blockDim.x) {
            int t = e / R, r = e % R;
            TF s = TF(0);
            for (int w = 0; w < 8; ++w) {
                int i = ib * 8 + w;
                if (i < NI) s = fmadd(z[((size_t)t * 8 + w) * RP + r], A[(long long)i * R + r], s);
            }
            part[((long long)ib * Kp + (k0 + t)) * d.pr + r] = s;
        }
    }
}

template <typename TX, int RP>
__global__ void __launch_bounds__(256) k_mtt_row(AlsDesc d, int mode) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    mtt_row_block<TX, RP>(d, mode, blockIdx.x, blockIdx.y, smem_raw);
}

// ---------------------------------------------------------------------------
// Column kernel: mode 2.  A CTA owns 32*COLS columns jj and a range of
// flattened rows (kk, ii); M2(jj, r) += X[kk][ii][jj] A(ii,r) C(kk,r).  Each
// warp takes every 8th row; warps are summed in shared memory in fixed order.
template <typename TX, int RP, int COLS>
__device__ void mtt_col_block(const AlsDesc &d, int bx, int rep, unsigned char *smem_raw) {
    using TF = typename FactorOf<TX>::T;
    if (d.conv[rep]) return;
    const int NI = d.n[0], NJ = d.n[1], Kp = d.n[2], R = d.R, ldj = d.ldj;
    const int njb = (NJ + 32 * COLS - 1) / (32 * COLS);
    const int jb = bx % njb, rs = bx / njb;
    const long long rows = (long long)Kp * NI;
    const long long r0 = (long long)rs * d.rows_per, r1 = min(rows, r0 + d.rows_per);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = jb * 32 * COLS + lane * COLS;
    if (d.bytes_ctr && threadIdx.x == 0) {
        const int cols = min(NJ, (jb + 1) * 32 * COLS) - jb * 32 * COLS;
        atomicAdd(d.bytes_ctr, (unsigned long long)max(0LL, r1 - r0) * cols * sizeof(TX));
    }
    TF *red = reinterpret_cast<TF *>(smem_raw);  // [8][32*COLS][RP]
    const TF *A = (const TF *)d.U[0] + (long long)rep * NI * R;
    const TF *C = (const TF *)d.U[2] + (long long)rep * Kp * R;
    const TX *X = (const TX *)d.X + rep * d.xrs;
    TF acc[COLS][RP];
#pragma unroll
    for (int c = 0; c < COLS; ++c)
#pragma unroll
        for (int r = 0; r < RP; ++r) acc[c][r] = TF(0);
    for (long long row = r0 + warp; row < r1; row += 8) {
        const int kk = (int)(row / NI), ii = (int)(row % NI);
        TF w[RP];
#pragma unroll
        for (int r = 0; r < RP; ++r) w[r] = (r < R) ? A[(long long)ii * R + r] * C[(long long)kk * R + r] : TF(0);
        const TX *xr = X + row * ldj + j0;
        TF xv[COLS];
#pragma unroll
        for (int c = 0; c < COLS; ++c) xv[c] = (j0 + c < NJ) ? (TF)widen_elem(xr[c]) : TF(0);
#pragma unroll
        for (int c = 0; c < COLS; ++c)
#pragma unroll
            for (int r = 0; r < RP; ++r)
                if (r < R) acc[c][r] = fmadd(xv[c], w[r], acc[c][r]);
    }
#pragma unroll
    for (int c = 0; c < COLS; ++c)
#pragma unroll
        for (int r = 0; r < RP; ++r) red[((size_t)warp * 32 * COLS + lane * COLS + c) * RP + r] = acc[c][r];
    __syncthreads();
    TF *part = (TF *)d.part + rep * d.prs;
    for (int e = threadIdx.x; e < 32 * COLS * R; e += blockDim.x) {
        int cl = e / R, r = e % R;
        int jj = jb * 32 * COLS + cl;
        if (jj >= NJ) continue;
        TF s = TF(0);
        for (int w = 0; w < 8; ++w) s += red[((size_t)w * 32 * COLS + cl) * RP + r];
        part[((long long)rs * NJ + jj) * d.pr + r] = s;
    }
}

template <typename TX, int RP, int COLS>
__global__ void __launch_bounds__(256) k_mtt_col(AlsDesc d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    mtt_col_block<TX, RP, COLS>(d, blockIdx.x, blockIdx.y, smem_raw);
}

// ---------------------------------------------------------------------------
// Fixed-order reduction of the partials: M[rep][e] = sum_p part[rep][p][e]

// sum_{q < P} p[q * stride] in q order, in float64, eight loads in flight
template <typename TF>
__device__ __forceinline__ double sum_partials(const TF *p, int P, long long stride) {
    double s = 0.0;
    int q = 0;
    for (; q + 8 <= P; q += 8) {
        TF v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = p[(long long)(q + u) * stride];
#pragma unroll
        for (int u = 0; u < 8; ++u) s += (double)v[u];
    }
    for (; q < P; ++q) s += (double)p[(long long)q * stride];
    return s;
}

// M(x, r) = sum of the P partials in order; partials [rep][P][n][pr] (row
// stride pr >= R), M [rep][n][R]
template <typename TF>
__global__ void k_reduce(const TF *part, long long prs, int P, int n, int R, int pr, double *M, long long mrs,
                         const int *conv) {
    const int rep = blockIdx.y;
    if (conv[rep]) return;
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * R) return;
    const long long x = e / R, r = e % R;
    M[rep * mrs + e] = sum_partials(part + rep * prs + x * pr + r, P, (long long)n * pr);
}

// ---------------------------------------------------------------------------
// float64 helpers of the tail: Cholesky, inverse, by one warp (R <= 32).
// L lower triangular, row-major 32 x 32; rinv[j] = 1 / L(j, j), so that the
// other lanes of a column and both triangular solves multiply instead of
// dividing (float64 division is a long chain of dependent operations here).
__device__ bool warp_cholesky(const double *V, double *L, double *rinv, int R, int lane) {
    bool ok = true;
    for (int j = 0; j < R; ++j) {
        if (lane == j) {
            double s = V[j * 32 + j];
            for (int k = 0; k < j; ++k) s -= L[j * 32 + k] * L[j * 32 + k];
            const bool pos = s > 0.0 && isfinite(s);
            const double dj = pos ? sqrt(s) : -1.0;
            L[j * 32 + j] = dj;
            rinv[j] = pos ? 1.0 / dj : 0.0;
        }
        __syncwarp();
        if (!(L[j * 32 + j] > 0.0)) ok = false;
        if (ok && lane > j && lane < R) {
            double s = V[lane * 32 + j];
            for (int k = 0; k < j; ++k) s -= L[lane * 32 + k] * L[j * 32 + k];
            L[lane * 32 + j] = s * rinv[j];
        }
        __syncwarp();
        if (!ok) break;
    }
    return ok;
}

// Vi = (L L^T)^-1: lane c solves L y = e_c, then L^T x = y; up to RP = 8
// y in registers (the loops unrolled over RP >= R), above in lane c's column
// of Vi itself.
template <int RP>
__device__ void warp_chol_inverse(const double *L, const double *rinv, double *Vi, int R, int lane) {
    if constexpr (RP > 8) {
        if (lane < R) {
            for (int i = 0; i < R; ++i) {
                double s = (i == lane) ? 1.0 : 0.0;
                for (int k = 0; k < i; ++k) s -= L[i * 32 + k] * Vi[k * 32 + lane];
                Vi[i * 32 + lane] = s * rinv[i];
            }
            for (int i = R - 1; i >= 0; --i) {
                double s = Vi[i * 32 + lane];
                for (int k = i + 1; k < R; ++k) s -= L[k * 32 + i] * Vi[k * 32 + lane];
                Vi[i * 32 + lane] = s * rinv[i];
            }
        }
        __syncwarp();
        return;
    }
    if (lane < R) {
        double y[RP];
#pragma unroll
        for (int i = 0; i < RP; ++i) {
            double s = (i == lane) ? 1.0 : 0.0;
#pragma unroll
            for (int k = 0; k < RP; ++k)
                if (k < i) s -= L[i * 32 + k] * y[k];
            y[i] = i < R ? s * rinv[i] : 0.0;
        }
#pragma unroll
        for (int i = RP - 1; i >= 0; --i) {
            if (i < R) {
                double s = y[i];
#pragma unroll
                for (int k = 0; k < RP; ++k)
                    if (k > i && k < R) s -= L[k * 32 + i] * y[k];
                y[i] = s * rinv[i];
            }
        }
#pragma unroll
        for (int i = 0; i < RP; ++i)
            if (i < R) Vi[i * 32 + lane] = y[i];
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Tail of one mode for one repetition (one CTA of 256 threads): the float64
// normal-equation solve, unit columns, the Gram and (mode 3) the fit.
struct TailShared {
    double V[32 * 32], L[32 * 32], Vi[32 * 32];
    double lam_s[32], rinv[32], red[8];
    int chol_ok, reg_flag, zero_flag;
};

template <typename TF, int RP>
__device__ void tail_rep_rp(const AlsDesc &d, int mode, int rep, TailShared &ts) {
    const int R = d.R, n = d.n[mode];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *V = ts.V, *L = ts.L, *Vi = ts.Vi, *lam_s = ts.lam_s;
    double *G = d.G + (long long)rep * 3 * R * R;
    const double *M = d.M + rep * d.mrs;
    TF *U = (TF *)d.U[mode] + (long long)rep * n * R;

    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        int r = e / R, s = e % R;
        double v = 1.0;
        for (int m = 0; m < 3; ++m)
            if (m != mode) v *= G[m * R * R + e];
        V[r * 32 + s] = v;
    }
    if (threadIdx.x == 0) {
        ts.reg_flag = 0;
        ts.zero_flag = 0;
    }
    __syncthreads();
    if (warp == 0) {
        bool ok = warp_cholesky(V, L, ts.rinv, R, lane);
        if (!ok) {
            // V + 1e-12 tr(V)/R I
            double tr = 0.0;
            for (int i = 0; i < R; ++i) tr += V[i * 32 + i];
            __syncwarp();
            if (lane < R) V[lane * 32 + lane] += 1e-12 * tr / R;
            __syncwarp();
            ok = warp_cholesky(V, L, ts.rinv, R, lane);
            if (lane == 0) ts.reg_flag = 1;
        }
        if (lane == 0) ts.chol_ok = ok;
        __syncwarp();
        if (ok) warp_chol_inverse<RP>(L, ts.rinv, Vi, R, lane);
    }
    __syncthreads();
    if (!ts.chol_ok) {
        // singular even after the shift: leave the factor, flag
        if (threadIdx.x == 0) atomicOr(&d.flags[rep], SBT_FLAG_CHOL_REGULARIZED_DEV);
        return;
    }
    // U = M Vi (float64 arithmetic, stored as TF)
    for (int x = threadIdx.x; x < n && RP > 8; x += blockDim.x) {
        for (int r = 0; r < R; ++r) {
            double acc = 0.0;
            for (int s = 0; s < R; ++s) acc += M[(long long)x * R + s] * Vi[s * 32 + r];
            U[(long long)x * R + r] = (TF)acc;
        }
    }
    for (int x = threadIdx.x; x < n && RP <= 8; x += blockDim.x) {
        double m[RP <= 8 ? RP : 1];
        constexpr int Q = RP <= 8 ? RP : 1;
#pragma unroll
        for (int s = 0; s < Q; ++s) m[s] = s < R ? M[(long long)x * R + s] : 0.0;
#pragma unroll
        for (int r = 0; r < Q; ++r) {
            if (r < R) {
                double acc = 0.0;
#pragma unroll
                for (int s = 0; s < Q; ++s)
                    if (s < R) acc += m[s] * Vi[s * 32 + r];
                U[(long long)x * R + r] = (TF)acc;
            }
        }
    }
    __syncthreads();
    // lambda_r = ||U(:, r)||
    for (int r = warp; r < R; r += 8) {
        double a = 0.0;
        for (int x = lane; x < n; x += 32) {
            double u = (double)U[(long long)x * R + r];
            a += u * u;
        }
        a = warp_sum(a);
        if (lane == 0) {
            double l = sqrt(a);
            if (l == 0.0) {
                l = 1.0;
                ts.zero_flag = 1;
            }
            lam_s[r] = l;
            ts.rinv[r] = 1.0 / l;
        }
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)n * R; e += blockDim.x) {
        int r = (int)(e % R);
        U[e] = (TF)((double)U[e] * ts.rinv[r]);
    }
    __syncthreads();
    // Gram of the normalised factor
    const int npairs = R * (R + 1) / 2;
    for (int pq = warp; pq < npairs; pq += 8) {
        int r = 0, rem = pq;
        while (rem >= R - r) {
            rem -= R - r;
            ++r;
        }
        int s = r + rem;
        double a = 0.0;
        for (int x = lane; x < n; x += 32) a += (double)U[(long long)x * R + r] * (double)U[(long long)x * R + s];
        a = warp_sum(a);
        if (lane == 0) {
            G[mode * R * R + r * R + s] = a;
            G[mode * R * R + s * R + r] = a;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int f = 0;
        if (ts.reg_flag) f |= SBT_FLAG_CHOL_REGULARIZED_DEV;
        if (ts.zero_flag) f |= SBT_FLAG_ZERO_COLUMN_DEV;
        if (f) d.flags[rep] |= f;
    }
    if (mode == 2) {
        // fit = 1 - ||X - X_hat|| / ||X||
        double inner = 0.0;
        for (long long e = threadIdx.x; e < (long long)n * R; e += blockDim.x) {
            int r = (int)(e % R);
            inner += lam_s[r] * M[e] * (double)U[e];
        }
        inner = warp_sum(inner);
        if (lane == 0) ts.red[warp] = inner;
        __syncthreads();
        if (warp == 0) {
            // ||X_hat||^2 = sum_{r,s} lam_r lam_s G1 G2 G3, a term per lane in turn
            double xh = 0.0;
            for (int e = lane; e < R * R; e += 32) {
                const int r = e / R, s = e % R;
                xh += lam_s[r] * lam_s[s] * G[e] * G[R * R + e] * G[2 * R * R + e];
            }
            xh = warp_sum(xh);
            if (lane == 0) {
                double in = 0.0;
                for (int w = 0; w < 8; ++w) in += ts.red[w];
                double nx2 = d.normX2[rep];
                double res2 = fmax(nx2 + xh - 2.0 * in, 0.0);
                double fit = nx2 > 0.0 ? 1.0 - sqrt(res2) / sqrt(nx2) : 0.0;
                int it = d.iters[rep] + 1;
                d.iters[rep] = it;
                d.fit[rep] = fit;
                bool stop = it >= d.max_iters;
                if (!d.fixed_iters && fabs(fit - d.fit_prev[rep]) < d.tol) stop = true;
                d.fit_prev[rep] = fit;
                if (stop) d.conv[rep] = 1;
                for (int r = 0; r < R; ++r) d.lam[rep * R + r] = lam_s[r];
            }
        }
    }
}

template <typename TF>
__device__ void tail_rep(const AlsDesc &d, int mode, int rep) {
    __shared__ TailShared ts;
    if (d.conv[rep]) return;
    if (d.R <= 8) tail_rep_rp<TF, 8>(d, mode, rep, ts);
    else if (d.R <= 16) tail_rep_rp<TF, 16>(d, mode, rep, ts);
    else tail_rep_rp<TF, 32>(d, mode, rep, ts);
}

template <typename TF>
__global__ void __launch_bounds__(256) k_tail(AlsDesc d, int mode) {
    tail_rep<TF>(d, mode, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Tail of one mode for float32 factors.  float64 is a slow unit here, so the
// R x R work (Hadamard of Grams, inverse, fit) runs in double-float like the
// n x R work, on the float32 pipes.
//
// k_tail_rows: grid (row chunks of TAIL_ROWS, repetitions).  V^-1 of the
// mode comes from k_xinv (beside the MTTKRP pass) or k_mtt_memo.  Every CTA
// sums the MTTKRP partials of its rows in fixed order, forms U_raw = M V^-1
// (written unnormalised) and the chunk's share of U_raw^T U_raw and of
// <M, U_raw>; the last CTA to finish combines the shares (tail_finish).
constexpr int TAIL_PB = 32;        // partials staged per block
constexpr int TAIL_THREADS = 256;
constexpr int TAIL_MAX_CLUSTER = 16;  // chunks of one repetition in one cluster (non-portable size)

__device__ void tail_finish(const AlsDesc &d, int mode, int rep, size_t smem_bytes);

// dynamic shared memory of k_tail_rows
struct TailSmem {
    float xh[32][33], xl[32][33];   // V^-1 in double-float
    float nh[32][33], nl[32][33];   // chunk shares before the fixed-order combine
    float in_h[256], in_l[256];
};

template <int RP>
__host__ __device__ constexpr size_t tail_smem_bytes() {
    return sizeof(TailSmem) + (size_t)3 * TAIL_ROWS * (RP + 1) * sizeof(float) + 16 +
           (size_t)TAIL_PB * TAIL_ROWS * RP * sizeof(float);
}

template <int RP>
__device__ void tail_finish_cluster(const AlsDesc &d, int mode, int rep, const DF *csh, int nch, int rows, int x0,
                                    const float (*ur)[RP + 1]);

template <int RP, bool CL>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail_rows(AlsDesc d, int mode) {
    const int rep = blockIdx.y, chunk = blockIdx.x;
    // programmatic dependent launch: let the next MTTKRP pass be scheduled,
    // then wait for the pass this tail reduces (and its memory)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (d.conv[rep]) return;
    const int R = d.R, n = d.n[mode], P = d.P[mode];
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    TailSmem &S = *reinterpret_cast<TailSmem *>(tsm_raw);
    auto xh = S.xh, xl = S.xl, nh = S.nh, nl = S.nl;
    float *in_h = S.in_h, *in_l = S.in_l;
    float (*mh)[RP + 1] = reinterpret_cast<float (*)[RP + 1]>(tsm_raw + sizeof(TailSmem));
    float (*ml)[RP + 1] = mh + TAIL_ROWS;
    float (*ur)[RP + 1] = ml + TAIL_ROWS;
    const float *part = (const float *)d.part + rep * d.prs;
    float *U = (float *)d.U[mode] + (long long)rep * n * R;
    const int x0 = chunk * TAIL_ROWS;
    const int rows = min(TAIL_ROWS, n - x0);

    // V^-1 of this mode (double-float planes, computed beside the MTTKRP
    // pass): its R x R entries, all loads in flight before the stores
    {
        const float *Xg = d.xinv + (long long)rep * 2048;
        constexpr int XPT = 32 * 32 / TAIL_THREADS;
        float vh[XPT], vl[XPT];
#pragma unroll
        for (int u = 0; u < XPT; ++u) {
            const int e = threadIdx.x + u * TAIL_THREADS;
            const int k = e / R, r = e % R;
            vh[u] = e < R * R ? Xg[k * 32 + r] : 0.f;
            vl[u] = e < R * R ? Xg[1024 + k * 32 + r] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < XPT; ++u) {
            const int e = threadIdx.x + u * TAIL_THREADS;
            if (e < R * R) {
                xh[e / R][e % R] = vh[u];
                xl[e / R][e % R] = vl[u];
            }
        }
    }
    // partial sums in fixed order per (row, r) item.  The chunk's share of
    // each partial is one contiguous, 16-byte aligned run of rows*pr floats
    // (rows padded to pr), so blocks of TAIL_PB partials are staged in shared
    // memory with coalesced float4 loads (four in flight per thread), then
    // summed item by item.
    const int pr = d.pr;
    const int nitems = rows * R;
    const int nrun = rows * pr;          // floats per partial in this chunk (multiple of 4)
    const long long pstride4 = (long long)n * pr;
    float *stage = reinterpret_cast<float *>(
        (reinterpret_cast<uintptr_t>(ur + TAIL_ROWS) + 15) & ~(uintptr_t)15);  // [TAIL_PB][rows*pr]
    constexpr int IPT = (TAIL_ROWS * RP + TAIL_THREADS - 1) / TAIL_THREADS;  // items per thread
    DF acc[IPT];
    int soff[IPT];  // offset of each item in a staged partial (row * pr + r)
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
        acc[u] = DF{0.f, 0.f};
        const int it = threadIdx.x + u * TAIL_THREADS;
        soff[u] = it < nitems ? (it / R) * pr + it % R : -1;
    }
    for (int q0 = 0; q0 < P; q0 += TAIL_PB) {
        const int pb = min(TAIL_PB, P - q0);
        const int n4 = nrun / 4, total4 = pb * n4;
        for (int e0 = threadIdx.x; e0 < total4; e0 += 4 * blockDim.x) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * blockDim.x;
                if (e < total4) {
                    const int q = e / n4, w = e % n4;
                    v[u] = *reinterpret_cast<const float4 *>(part + (long long)(q0 + q) * pstride4 +
                                                             (long long)x0 * pr + 4 * w);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * blockDim.x;
                if (e < total4) reinterpret_cast<float4 *>(stage)[e] = v[u];
            }
        }
        __syncthreads();
        for (int q = 0; q < pb; ++q) {
            const float *sq = stage + q * nrun;
#pragma unroll
            for (int u = 0; u < IPT; ++u)
                if (soff[u] >= 0) acc[u] = df_add(acc[u], DF{sq[soff[u]], 0.f});
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
        const int it = threadIdx.x + u * TAIL_THREADS;
        if (it < nitems) {
            mh[it / R][it % R] = acc[u].hi;
            ml[it / R][it % R] = acc[u].lo;
        }
    }
    __syncthreads();
    // U_raw = M X for the chunk's rows; <M, U_raw> per thread
    DF inner{0.f, 0.f};
    for (int it = threadIdx.x; it < rows * R; it += blockDim.x) {
        const int t = it / R, r = it % R;
        DF a{0.f, 0.f};
        for (int k = 0; k < R; ++k) a = df_fma(a, DF{mh[t][k], ml[t][k]}, DF{xh[k][r], xl[k][r]});
        const float uf = __fadd_rn(a.hi, a.lo);
        ur[t][r] = uf;
        if (!CL) U[(long long)(x0 + t) * R + r] = uf;  // a cluster writes its rows once, normalised
        inner = df_fma(inner, DF{mh[t][r], ml[t][r]}, DF{uf, 0.f});
    }
    inner = warp_df_sum(inner);
    if ((threadIdx.x & 31) == 0) {
        in_h[threadIdx.x >> 5] = inner.hi;
        in_l[threadIdx.x >> 5] = inner.lo;
    }
    __syncthreads();
    // chunk shares: (U_raw^T U_raw)(r, s) for r <= s, and <M, U_raw> (slot npairs);
    // tps threads per slot each take every tps-th row, combined in fixed order
    const int npairs = R * (R + 1) / 2;
    const int slots = npairs + 1;
    const int tps = slots >= (int)blockDim.x ? 1 : (slots * 4 <= (int)blockDim.x ? 4 : (slots * 2 <= (int)blockDim.x ? 2 : 1));
    DF *tp = d.tpart + ((long long)rep * d.tchunks + chunk) * (npairs + 1);
    __syncthreads();
    for (int w0 = threadIdx.x; w0 < slots * tps; w0 += blockDim.x) {
        const int pq = w0 / tps, sub = w0 % tps;
        DF a{0.f, 0.f};
        if (pq < npairs) {
            int r = 0, rem = pq;
            while (rem >= R - r) {
                rem -= R - r;
                ++r;
            }
            const int s2 = r + rem;
            for (int t = sub; t < rows; t += tps) a = df_add_prod(a, ur[t][r], ur[t][s2]);
        } else {
            for (int t = sub; t < (int)(blockDim.x >> 5); t += tps) a = df_add(a, DF{in_h[t], in_l[t]});
        }
        // park the share in the (now unused) matrices: slot-major, sub-minor
        (&nh[0][0])[w0] = a.hi;
        (&nl[0][0])[w0] = a.lo;
    }
    __syncthreads();
    if constexpr (CL) {
        // the repetition's chunk CTAs are one cluster: shares stay in shared
        // memory and every CTA completes the mode for its own rows
        __shared__ DF csh[32 * 33 / 2 + 1];
        for (int pq = threadIdx.x; pq < slots; pq += blockDim.x) {
            DF a{0.f, 0.f};
            for (int sub = 0; sub < tps; ++sub) a = df_add(a, DF{(&nh[0][0])[pq * tps + sub], (&nl[0][0])[pq * tps + sub]});
            csh[pq] = a;
        }
        tail_finish_cluster<RP>(d, mode, rep, csh, (int)gridDim.x, rows, x0, ur);
    } else {
        for (int pq = threadIdx.x; pq < slots; pq += blockDim.x) {
            DF a{0.f, 0.f};
            for (int sub = 0; sub < tps; ++sub) a = df_add(a, DF{(&nh[0][0])[pq * tps + sub], (&nl[0][0])[pq * tps + sub]});
            tp[pq] = a;
        }
        // the last chunk CTA of this repetition to finish completes the mode
        __shared__ int is_last;
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const int nch = (n + TAIL_ROWS - 1) / TAIL_ROWS;
            const int old = atomicAdd(&d.tail_cnt[rep], 1);
            is_last = (old == nch - 1);
            if (is_last) d.tail_cnt[rep] = 0;
        }
        __syncthreads();
        if (!is_last) return;
        __threadfence();
        tail_finish(d, mode, rep, tail_smem_bytes<RP>());
    }
}

// Finish of one mode for one repetition (the last chunk CTA), in double-float:
// sums the chunk shares in fixed order: lambda_r = sqrt((U_raw^T U_raw)(r,r)),
// the Gram of the normalised factor, U /= lambda; after mode 3 the fit
// 1 - sqrt(||X||^2 + lambda^T (G1*G2*G3) lambda - 2 <M, U_raw>) / ||X|| and the
// convergence flag.  Shares and rows of the other CTAs are read through L2.
__device__ __forceinline__ DF ldcg_df(const DF *p) {
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return DF{v.x, v.y};
}

__device__ void tail_finish(const AlsDesc &d, int mode, int rep, size_t smem_bytes) {
    const int R = d.R, n = d.n[mode];
    const int npairs = R * (R + 1) / 2;
    const int nch = (n + TAIL_ROWS - 1) / TAIL_ROWS;
    __shared__ DF graw[32 * 33 / 2 + 1];
    __shared__ DF lam_s[32], inv_l[32];
    __shared__ float inv_lam[32];
    __shared__ DF gm[32 * 32];
    __shared__ DF xh_part[32];
    __shared__ int zero_flag;
    DF *Gf = d.Gf + (long long)rep * 3 * R * R;
    const DF *tp = d.tpart + (long long)rep * d.tchunks * (npairs + 1);
    // chunk shares: as many as the CTA's dynamic shared memory holds (free
    // now: this CTA's own chunk is done) loaded with all loads in flight,
    // then added per pair in chunk order
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    DF *shr = reinterpret_cast<DF *>(tsm_raw);
    const int blk = max(1, (int)(smem_bytes / ((size_t)(npairs + 1) * sizeof(DF))));
    if (threadIdx.x == 0) zero_flag = 0;
    for (int pq = threadIdx.x; pq <= npairs; pq += blockDim.x) graw[pq] = DF{0.f, 0.f};
    for (int c0 = 0; c0 < nch; c0 += blk) {
        const int cn = min(blk, nch - c0);
        const int items = cn * (npairs + 1);
        for (int e = threadIdx.x; e < items; e += blockDim.x)
            shr[e] = ldcg_df(&tp[(long long)c0 * (npairs + 1) + e]);
        __syncthreads();
        for (int pq = threadIdx.x; pq <= npairs; pq += blockDim.x) {
            DF a = graw[pq];
            for (int c = 0; c < cn; ++c) a = df_add(a, shr[c * (npairs + 1) + pq]);
            graw[pq] = a;
        }
        __syncthreads();
    }
    if (threadIdx.x < R) {
        const int r = threadIdx.x;
        DF l = df_sqrt(graw[r * R - r * (r - 1) / 2]);  // diagonal pair (r, r)
        if (l.hi == 0.f) {
            l = DF{1.f, 0.f};
            zero_flag = 1;
        }
        lam_s[r] = l;
        inv_l[r] = df_div(DF{1.f, 0.f}, l);
        inv_lam[r] = __fadd_rn(inv_l[r].hi, inv_l[r].lo);
    }
    __syncthreads();
    for (int pq = threadIdx.x; pq < npairs; pq += blockDim.x) {
        int r = 0, rem = pq;
        while (rem >= R - r) {
            rem -= R - r;
            ++r;
        }
        const int s2 = r + rem;
        const DF g = df_mul(df_mul(graw[pq], inv_l[r]), inv_l[s2]);
        Gf[mode * R * R + r * R + s2] = g;
        Gf[mode * R * R + s2 * R + r] = g;
        gm[r * R + s2] = g;
        gm[s2 * R + r] = g;
    }
    float *U = (float *)d.U[mode] + (long long)rep * n * R;
    {
        // U /= lambda column-wise: eight loads in flight per thread, then the
        // stores (column index tracked incrementally, no division per element)
        const long long total = (long long)n * R;
        const int step = (int)(blockDim.x % R);
        int r = (int)(threadIdx.x % R);
        for (long long e0 = threadIdx.x; e0 < total; e0 += 8LL * blockDim.x) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const long long e = e0 + (long long)u * blockDim.x;
                v[u] = e < total ? __ldcg(&U[e]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const long long e = e0 + (long long)u * blockDim.x;
                if (e < total) U[e] = v[u] * inv_lam[r];
                r += step;
                if (r >= R) r -= R;
            }
        }
    }
    __syncthreads();
    if (mode == 2) {
        DF a{0.f, 0.f};
        for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
            const int r = e / R, s2 = e % R;
            DF t = df_mul(df_mul(lam_s[r], lam_s[s2]), df_mul(df_mul(Gf[e], Gf[R * R + e]), gm[e]));
            a = df_add(a, t);
        }
        a = warp_df_sum(a);
        if ((threadIdx.x & 31) == 0) xh_part[threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            DF xh{0.f, 0.f};
            for (int t = 0; t < (int)(blockDim.x >> 5); ++t) xh = df_add(xh, xh_part[t]);
            const DF in = graw[npairs];  // <X, X_hat> = sum_r lambda_r <M(:,r), U(:,r)> = <M, U_raw>
            const DF nx2 = d.nx2f[rep];
            DF res2 = df_sub(df_add(nx2, xh), df_add(in, in));
            if (!(res2.hi > 0.f)) res2 = DF{0.f, 0.f};
            const DF ratio = nx2.hi > 0.f ? df_div(df_sqrt(res2), df_sqrt(nx2)) : DF{1.f, 0.f};
            const DF fit = df_sub(DF{1.f, 0.f}, ratio);
            const DF diff = df_sub(fit, d.fitpf[rep]);
            const int it = d.iters[rep] + 1;
            d.iters[rep] = it;
            d.fit[rep] = df_value(fit);
            bool stop = it >= d.max_iters;
            if (!d.fixed_iters && fabsf(__fadd_rn(diff.hi, diff.lo)) < (float)d.tol) stop = true;
            d.fitpf[rep] = fit;
            if (stop) d.conv[rep] = 1;
        }
        if (threadIdx.x < R) d.lam[rep * R + threadIdx.x] = df_value(lam_s[threadIdx.x]);
    }
    if (threadIdx.x == 0 && zero_flag) d.flags[rep] |= SBT_FLAG_ZERO_COLUMN_DEV;
}

// tail_finish for a cluster of the repetition's chunk CTAs (rank = chunk):
// after a cluster barrier every CTA adds the shares of all chunks in chunk
// order from their shared memory (the same sums as tail_finish), forms
// lambda and the normalised Gram, and writes its own rows of U divided by
// lambda; rank 0 writes the repetition's state (Gram, lambda, fit,
// convergence).  A second barrier keeps every CTA's shares readable until
// all have been read.
template <int RP>
__device__ void tail_finish_cluster(const AlsDesc &d, int mode, int rep, const DF *csh, int nch, int rows, int x0,
                                    const float (*ur)[RP + 1]) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int R = d.R, n = d.n[mode];
    const int npairs = R * (R + 1) / 2;
    const bool lead = cluster.block_rank() == 0;
    __shared__ DF graw[32 * 33 / 2 + 1];
    __shared__ DF lam_s[32], inv_l[32];
    __shared__ float inv_lam[32];
    __shared__ DF gm[32 * 32];
    __shared__ DF xh_part[32];
    __shared__ int zero_flag;
    if (threadIdx.x == 0) zero_flag = 0;
    cluster.sync();
    for (int pq = threadIdx.x; pq <= npairs; pq += blockDim.x) {
        DF v[TAIL_MAX_CLUSTER];
#pragma unroll
        for (int c = 0; c < TAIL_MAX_CLUSTER; ++c)
            v[c] = c < nch ? cluster.map_shared_rank(csh, c)[pq] : DF{0.f, 0.f};
        DF a{0.f, 0.f};
#pragma unroll
        for (int c = 0; c < TAIL_MAX_CLUSTER; ++c)
            if (c < nch) a = df_add(a, v[c]);
        graw[pq] = a;
    }
    __syncthreads();
    if (threadIdx.x < R) {
        const int r = threadIdx.x;
        DF l = df_sqrt(graw[r * R - r * (r - 1) / 2]);  // diagonal pair (r, r)
        if (l.hi == 0.f) {
            l = DF{1.f, 0.f};
            zero_flag = 1;
        }
        lam_s[r] = l;
        inv_l[r] = df_div(DF{1.f, 0.f}, l);
        inv_lam[r] = __fadd_rn(inv_l[r].hi, inv_l[r].lo);
    }
    __syncthreads();
    DF *Gf = d.Gf + (long long)rep * 3 * R * R;
    for (int pq = threadIdx.x; pq < npairs; pq += blockDim.x) {
        int r = 0, rem = pq;
        while (rem >= R - r) {
            rem -= R - r;
            ++r;
        }
        const int s2 = r + rem;
        const DF g = df_mul(df_mul(graw[pq], inv_l[r]), inv_l[s2]);
        if (lead) {
            Gf[mode * R * R + r * R + s2] = g;
            Gf[mode * R * R + s2 * R + r] = g;
        }
        gm[r * R + s2] = g;
        gm[s2 * R + r] = g;
    }
    float *U = (float *)d.U[mode] + (long long)rep * n * R;
    for (int it = threadIdx.x; it < rows * R; it += blockDim.x) {
        const int t = it / R, r = it % R;
        U[(long long)(x0 + t) * R + r] = ur[t][r] * inv_lam[r];
    }
    __syncthreads();
    if (mode == 2 && lead) {
        DF a{0.f, 0.f};
        for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
            const int r = e / R, s2 = e % R;
            DF t = df_mul(df_mul(lam_s[r], lam_s[s2]), df_mul(df_mul(Gf[e], Gf[R * R + e]), gm[e]));
            a = df_add(a, t);
        }
        a = warp_df_sum(a);
        if ((threadIdx.x & 31) == 0) xh_part[threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            DF xh{0.f, 0.f};
            for (int t = 0; t < (int)(blockDim.x >> 5); ++t) xh = df_add(xh, xh_part[t]);
            const DF in = graw[npairs];  // <X, X_hat> = sum_r lambda_r <M(:,r), U(:,r)> = <M, U_raw>
            const DF nx2 = d.nx2f[rep];
            DF res2 = df_sub(df_add(nx2, xh), df_add(in, in));
            if (!(res2.hi > 0.f)) res2 = DF{0.f, 0.f};
            const DF ratio = nx2.hi > 0.f ? df_div(df_sqrt(res2), df_sqrt(nx2)) : DF{1.f, 0.f};
            const DF fit = df_sub(DF{1.f, 0.f}, ratio);
            const DF diff = df_sub(fit, d.fitpf[rep]);
            const int it = d.iters[rep] + 1;
            d.iters[rep] = it;
            d.fit[rep] = df_value(fit);
            bool stop = it >= d.max_iters;
            if (!d.fixed_iters && fabsf(__fadd_rn(diff.hi, diff.lo)) < (float)d.tol) stop = true;
            d.fitpf[rep] = fit;
            if (stop) d.conv[rep] = 1;
        }
        if (threadIdx.x < R) d.lam[rep * R + threadIdx.x] = df_value(lam_s[threadIdx.x]);
    }
    if (lead && threadIdx.x == 0 && zero_flag) d.flags[rep] |= SBT_FLAG_ZERO_COLUMN_DEV;
    cluster.sync();
}

// V^-1 for mode `mode` from the Grams of the other two modes, by Gauss-Jordan
// elimination on [V | I] in double-float (R pivot steps).  For symmetric V
// the pivots are the squared Cholesky diagonals, so a non-positive pivot
// means V is not positive definite: then V + 1e-12 tr(V)/R I is used and
// `reg` is set; if that fails too, X = 0 and `reg` is set.  Called by
// INV_THREADS threads, each holding up to INV_EPT entries (e = t + 128 u,
// row-major over R x 2R; EPT >= 2 R^2 / 128) with straight-line code per
// pivot step; W (shared memory, 32 x 64 values) exchanges the pivot row and
// column.  X is written as two float planes (hi, lo) of 32 x 32.
constexpr int INV_THREADS = 128;
template <int EPT>
__device__ void cta_inverse_df_t(const DF *Gf, int R, int mode, float *X, int *reg, DF *W) {
    constexpr int INV_EPT = EPT;
    const int t = threadIdx.x, ld = 64;
    const int m0 = mode == 0 ? 1 : 0, m1 = mode == 2 ? 1 : 2;  // the two other modes, in order
    const int ne = 2 * R * R;
    int ei[INV_EPT], ej[INV_EPT];
    DF init[INV_EPT];
#pragma unroll
    for (int u = 0; u < INV_EPT; ++u) {
        const int e = t + INV_THREADS * u;
        const int ec = e < ne ? e : 0;
        ei[u] = ec / (2 * R);
        ej[u] = ec % (2 * R);
        const int jc = ej[u] < R ? ej[u] : 0;
        const DF v = df_mul(df_mul(DF{1.f, 0.f}, Gf[m0 * R * R + ei[u] * R + jc]), Gf[m1 * R * R + ei[u] * R + jc]);
        init[u] = ej[u] < R ? v : DF{(ej[u] - R == ei[u]) ? 1.f : 0.f, 0.f};
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
#pragma unroll
        for (int u = 0; u < INV_EPT; ++u)
            if (t + INV_THREADS * u < ne) W[ei[u] * ld + ej[u]] = init[u];
        __syncthreads();
        if (attempt == 1) {
            if (t == 0) {
                DF tr{0.f, 0.f};
                for (int i = 0; i < R; ++i) tr = df_add(tr, W[i * ld + i]);
                const DF shift = df_mul(tr, DF{1e-12f / (float)R, 0.f});
                for (int i = 0; i < R; ++i) W[i * ld + i] = df_add(W[i * ld + i], shift);
            }
            __syncthreads();
        }
        bool ok = true;
        for (int k = 0; k < R; ++k) {
            const DF piv = W[k * ld + k];
            const DF inv = df_div(DF{1.f, 0.f}, piv);
            DF nv[INV_EPT];
#pragma unroll
            for (int u = 0; u < INV_EPT; ++u) {
                const DF rk = W[k * ld + ej[u]];
                const DF ck = W[ei[u] * ld + k];
                const DF tt = df_mul(rk, inv);
                nv[u] = ei[u] == k ? tt : df_sub(W[ei[u] * ld + ej[u]], df_mul(ck, tt));
            }
            ok = ok && piv.hi > 0.f && isfinite(piv.hi);
            __syncthreads();
#pragma unroll
            for (int u = 0; u < INV_EPT; ++u)
                if (t + INV_THREADS * u < ne) W[ei[u] * ld + ej[u]] = nv[u];
            __syncthreads();
        }
        if (ok) {
            for (int e = t; e < 32 * 32; e += INV_THREADS) {
                const int i = e / 32, j = e % 32;
                const DF v = (i < R && j < R) ? W[i * ld + R + j] : DF{0.f, 0.f};
                X[e] = v.hi;
                X[1024 + e] = v.lo;
            }
            if (attempt == 1 && t == 0) *reg = 1;
            return;
        }
        __syncthreads();
    }
    for (int e = t; e < 2 * 32 * 32; e += INV_THREADS) X[e] = 0.f;
    if (t == 0) *reg = 1;
}

// entries per thread: 2 R^2 <= 128 EPT
__device__ void cta_inverse_df(const DF *Gf, int R, int mode, float *X, int *reg, DF *W) {
    if (R <= 8) cta_inverse_df_t<1>(Gf, R, mode, X, reg, W);
    else if (R <= 11) cta_inverse_df_t<2>(Gf, R, mode, X, reg, W);
    else if (R <= 16) cta_inverse_df_t<4>(Gf, R, mode, X, reg, W);
    else cta_inverse_df_t<16>(Gf, R, mode, X, reg, W);
}

// V^-1 of mode `mode` (its Grams are final): one CTA per repetition, run on
// a side stream while the mode's MTTKRP pass runs.
__global__ void __launch_bounds__(INV_THREADS) k_xinv(AlsDesc d, int mode) {
    const int rep = blockIdx.x;
    if (d.conv[rep]) return;
    __shared__ DF W[32 * 64];
    int reg = 0;
    cta_inverse_df(d.Gf + (long long)rep * 3 * d.R * d.R, d.R, mode, d.xinv + (long long)rep * 2048, &reg, W);
    if (threadIdx.x == 0 && reg) atomicOr(&d.flags[rep], SBT_FLAG_CHOL_REGULARIZED_DEV);
}

// Mode 3 after a memoised mode-2 pass: M3(kk, r) = sum_j Y_kk(j, r) B(j, r)
// with the new B, one CTA per summary slice: every thread loads its rows of
// Y and of B together (two rows per round), then a fixed-order reduction
// (lane tree, then the warps in order) gives the single partial sum of the
// mode-3 tail.  CTA 0 of each repetition forms V^-1 of mode 3 (the Grams of
// A and B are final) meanwhile.
constexpr int MEMO_THREADS = INV_THREADS;
template <int RP>
__global__ void __launch_bounds__(MEMO_THREADS) k_mtt_memo(AlsDesc d) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int rep = blockIdx.y;
    if (d.conv[rep]) return;
    const int R = d.R, nj = d.n[1], pr = d.pr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (blockIdx.x == 0) {
        if (!d.tail64) {  // the float64 tail solves with its own Cholesky factorisation
            __shared__ DF W[32 * 64];
            int reg = 0;
            cta_inverse_df(d.Gf + (long long)rep * 3 * R * R, R, 2, d.xinv + (long long)rep * 2048, &reg, W);
            if (threadIdx.x == 0 && reg) atomicOr(&d.flags[rep], SBT_FLAG_CHOL_REGULARIZED_DEV);
        }
        return;
    }
    const int kk = blockIdx.x - 1;
    constexpr int NQ = RP / 4;  // float4 per row of Y (pr <= RP)
    const int pq = pr / 4;
    const float4 *y = reinterpret_cast<const float4 *>(d.ymem + rep * d.yrs + (long long)kk * nj * pr);
    const float *Bf = (const float *)d.U[1] + (long long)rep * nj * R;
    float a[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) a[r] = 0.f;
    for (int jb = threadIdx.x; jb < nj; jb += 2 * MEMO_THREADS) {
        float4 v[2][NQ];
        float b[2][RP];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int j = jb + u * MEMO_THREADS;
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                v[u][q] = (j < nj && q < pq) ? __ldcg(y + (long long)j * pq + q) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int r = 0; r < RP; ++r) b[u][r] = (j < nj && r < R) ? __ldg(Bf + (long long)j * R + r) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const float e[4] = {v[u][q].x, v[u][q].y, v[u][q].z, v[u][q].w};
#pragma unroll
                for (int c = 0; c < 4; ++c) a[4 * q + c] = fmaf(e[c], b[u][4 * q + c], a[4 * q + c]);
            }
        }
    }
    __shared__ float red[MEMO_THREADS / 32][RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) {
        const float v = warp_sum(a[r]);
        if (lane == 0) red[warp][r] = v;
    }
    __syncthreads();
    if (threadIdx.x < R) {
        float sum = red[0][threadIdx.x];
        for (int w = 1; w < MEMO_THREADS / 32; ++w) sum += red[w][threadIdx.x];
        ((float *)d.part + rep * d.prs + (long long)kk * pr)[threadIdx.x] = sum;
    }
}

// Sum of the thread's entries q[t], q[t + blockDim.x], ... in that order,
// eight loads in flight before their additions (the order, and so the
// result, of a plain strided loop).
__device__ __forceinline__ double sum_strided(const double *q, long long n) {
    double a = 0.0;
    long long e = threadIdx.x;
    const long long step = blockDim.x;
    for (; e + 7 * step < n; e += 8 * step) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = q[e + u * step];
#pragma unroll
        for (int u = 0; u < 8; ++u) a += v[u];
    }
    for (; e < n; e += step) a += q[e];
    return a;
}

// ---------------------------------------------------------------------------
// Start values, Grams and ||X_s||^2: grid (repetitions, 4); CTA (rep, m < 3)
// starts mode m's factor and its Gram, CTA (rep, 3) takes ||X_s||^2 and the
// per-repetition words
template <typename TF>
__global__ void __launch_bounds__(256) k_prepare(AlsDesc d, const int *samples, long long samp_stride,
                                                 int K_old, int identity, uint64_t seed,
                                                 uint32_t stream_id, uint32_t batch,
                                                 const double *rowsq, WarmStart ws) {
    const int rep = blockIdx.x;
    const int R = d.R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint2 key = philox_key(seed, stream_id);
    const int m = blockIdx.y;
    if (m < 3) {
        const int n = d.n[m];
        TF *U = (TF *)d.U[m] + (long long)rep * n * R;
        const int *S = samples ? samples + (long long)(rep * 3 + m) * samp_stride : nullptr;
        for (long long e = threadIdx.x; e < (long long)n * R; e += blockDim.x) {
            int x = (int)(e / R), r = (int)(e % R);
            uint32_t gx;
            if (identity) gx = (uint32_t)x;
            else if (m < 2) gx = (uint32_t)S[x];
            else gx = (uint32_t)(x < d.nK ? S[x] : K_old + (x - d.nK));
            if (ws.F[0])  // warm: the old factor at the sampled row; new slices' rows zero
                U[e] = (m < 2 || x < d.nK) ? (TF)ws.F[m][(long long)gx * R + r] : (TF)0;
            else if (ws.trial >= 0)  // GetRank's trial start (Algorithm 2)
                U[e] = (TF)init_value_trial(key, gx, r, m, rep + d.rep0, batch, ws.trial);
            else
                U[e] = (TF)init_value(key, gx, r, m, rep + d.rep0, batch);
        }
        __syncthreads();
        double *G = d.G + (long long)rep * 3 * R * R;
        const int npairs = R * (R + 1) / 2;
        for (int pq = warp; pq < npairs; pq += 8) {
            int r = 0, rem = pq;
            while (rem >= R - r) {
                rem -= R - r;
                ++r;
            }
            int s = r + rem;
            if (d.Gf && !d.tail64) {
                // float32 factors: exact products, double-float sums
                DF a{0.f, 0.f};
                for (int x = lane; x < n; x += 32)
                    a = df_add_prod(a, (float)U[(long long)x * R + r], (float)U[(long long)x * R + s]);
                a = warp_df_sum(a);
                if (lane == 0) {
                    d.Gf[((long long)rep * 3 + m) * R * R + r * R + s] = a;
                    d.Gf[((long long)rep * 3 + m) * R * R + s * R + r] = a;
                }
            } else {
                double a = 0.0;
                for (int x = lane; x < n; x += 32) a += (double)U[(long long)x * R + r] * (double)U[(long long)x * R + s];
                a = warp_sum(a);
                if (lane == 0) {
                    G[m * R * R + r * R + s] = a;
                    G[m * R * R + s * R + r] = a;
                }
            }
        }
        return;
    }
    // ||X_s||^2 from the row sums, fixed order
    __shared__ double red[256];
    const long long rows = d.rq_rows ? d.rq_rows : (long long)d.n[2] * d.n[0];
    const double *rq = rowsq + rep * rows;
    const double a = sum_strided(rq, rows);
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s = 128; s; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        d.normX2[rep] = red[0];
        if (d.nx2f) {
            d.nx2f[rep] = df_from_double(red[0]);
            d.fitpf[rep] = DF{0.f, 0.f};
        }
        d.fit_prev[rep] = 0.0;
        d.fit[rep] = 0.0;
        d.iters[rep] = 0;
        d.conv[rep] = 0;
        d.flags[rep] = (min(min(d.n[0], d.n[1]), d.nK) < R) ? SBT_FLAG_SAMPLE_LT_RANK_DEV : 0;
    }
}

// Start of the refinement sweeps (one CTA per repetition): ||X_s||^2 of the
// split summary (hi + lo) from its row sums, fixed order as in k_prepare;
// the fit history, iteration counts and convergence flags start again.  The
// factors and Grams carry over from the bfloat16 ALS.
__global__ void __launch_bounds__(256) k_refine_start(AlsDesc d, const double *rowsq2) {
    const int rep = blockIdx.x;
    __shared__ double red[256];
    const long long rows = (long long)d.n[2] * d.n[0];
    const double *rq = rowsq2 + rep * rows;
    const double a = sum_strided(rq, rows);
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s = 128; s; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        d.normX2[rep] = red[0];
        if (d.nx2f) {
            d.nx2f[rep] = df_from_double(red[0]);
            d.fitpf[rep] = DF{0.f, 0.f};
        }
        d.fit_prev[rep] = 0.0;
        d.iters[rep] = 0;
        d.conv[rep] = 0;
    }
}

cudaError_t launch_refine_start(const AlsDesc &d, const double *rowsq2, cudaStream_t st) {
    k_refine_start<<<d.nrep, 256, 0, st>>>(d, rowsq2);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host side
static int rp_of(int R) { return R <= 8 ? 8 : (R <= 16 ? 16 : 32); }
static int vec_of(int elem) { return elem == 0 ? 2 : (elem == 1 ? 4 : 8); }
static int tf_size(int elem) { return elem == 0 ? 8 : 4; }
static int cols_of(int elem, int RP) { return std::min(vec_of(elem), std::max(1, 64 / RP)); }

void choose_tiles(AlsDesc &d, int num_sms) {
    const int NI = d.n[0], NJ = d.n[1], Kp = d.n[2];
    const int RP = rp_of(d.R);
    const long long target = (long long)num_sms * 8;
    d.nib = (NI + 7) / 8;
    long long nks = target / std::max(1LL, (long long)d.nib * d.nrep);
    nks = std::max(1LL, std::min<long long>(nks, Kp));
    int spc = (int)((Kp + nks - 1) / nks);
    spc = std::max(1, std::min(spc, 32));
    d.spc = spc;
    d.nks = (Kp + spc - 1) / spc;
    // column chunk of the row kernel: all of NJ if it fits next to z
    const int V = vec_of(d.elem);
    int jc = (NJ + V - 1) / V * V;
    const int tfs = tf_size(d.elem);
    const int zbytes = d.spc * 8 * RP * tfs;
    const int budget = 160 * 1024 - zbytes;
    int jmax = budget / (RP * tfs);
    jmax = std::max(32 * V, jmax / (32 * V) * (32 * V));
    d.jc = std::min(jc, jmax);
    // column kernel
    const int cols = cols_of(d.elem, RP);
    d.cols = cols;
    const int njb = (NJ + 32 * cols - 1) / (32 * cols);
    const long long rows = (long long)Kp * NI;
    long long nrs = target / std::max(1LL, (long long)njb * d.nrep);
    nrs = std::max(1LL, std::min(nrs, rows));
    // small summaries: at least 64 rows (8 per warp) per column block, so
    // that the partial sums the reduction adds one by one stay few (split
    // finer, each block would do almost nothing)
    d.rows_per = std::max<long long>((rows + nrs - 1) / nrs, std::min<long long>(64, rows));
    d.nrs = (int)((rows + d.rows_per - 1) / d.rows_per);
    d.P[0] = d.nks;
    d.P[1] = d.nrs;
    d.P[2] = d.nib;
}

long long partial_elems(const AlsDesc &d) {
    long long a = (long long)d.nks * d.n[0];
    long long b = (long long)d.nrs * d.n[1];
    long long c = (long long)d.nib * d.n[2];
    return std::max(a, std::max(b, c)) * (d.pr > 0 ? d.pr : d.R);
}

static size_t row_smem(const AlsDesc &d) {
    const int RP = rp_of(d.R);
    return (size_t)RP * d.jc * tf_size(d.elem) + (size_t)d.spc * 8 * RP * tf_size(d.elem);
}
static size_t col_smem(const AlsDesc &d) {
    const int RP = rp_of(d.R);
    return (size_t)8 * 32 * d.cols * RP * tf_size(d.elem);
}

template <typename TX, int RP>
static cudaError_t run_row(const AlsDesc &d, int mode, cudaStream_t st) {
    size_t sm = row_smem(d);
    dim3 grid(d.nib * d.nks, d.nrep);
    k_mtt_row<TX, RP><<<grid, 256, sm, st>>>(d, mode);
    return cudaGetLastError();
}

template <typename TX, int RP, int COLS>
static cudaError_t run_col(const AlsDesc &d, cudaStream_t st) {
    size_t sm = col_smem(d);
    const int njb = (d.n[1] + 32 * COLS - 1) / (32 * COLS);
    dim3 grid(njb * d.nrs, d.nrep);
    k_mtt_col<TX, RP, COLS><<<grid, 256, sm, st>>>(d);
    return cudaGetLastError();
}

// columns per lane of the column kernel: one 16-byte vector, at most 64 accumulators
template <typename TX, int RP>
constexpr int cols_for() {
    constexpr int v = 16 / (int)sizeof(TX);
    return v < 64 / RP ? v : 64 / RP;
}

template <typename TX, int RP>
static cudaError_t run_col_any(const AlsDesc &d, cudaStream_t st) {
    return run_col<TX, RP, cols_for<TX, RP>()>(d, st);
}

template <typename TX>
static cudaError_t run_mtt(const AlsDesc &d, int mode, cudaStream_t st) {
    const int RP = rp_of(d.R);
    if (mode == 1) {
        if (RP == 8) return run_col_any<TX, 8>(d, st);
        if (RP == 16) return run_col_any<TX, 16>(d, st);
        return run_col_any<TX, 32>(d, st);
    }
    if (RP == 8) return run_row<TX, 8>(d, mode, st);
    if (RP == 16) return run_row<TX, 16>(d, mode, st);
    return run_row<TX, 32>(d, mode, st);
}

static cudaError_t mtt_dispatch(const AlsDesc &d, int mode, cudaStream_t st) {
    if (d.elem == 0) return run_mtt<double>(d, mode, st);
    if (d.elem == 1) return run_mtt<float>(d, mode, st);
    return run_mtt<__nv_bfloat16>(d, mode, st);
}

static cudaError_t reduce_dispatch(const AlsDesc &d, int mode, cudaStream_t st) {
    const int P = d.P[mode];
    const long long cnt = (long long)d.n[mode] * d.R;
    dim3 grid((unsigned)((cnt + 255) / 256), d.nrep);
    if (d.elem == 0)
        k_reduce<double><<<grid, 256, 0, st>>>((const double *)d.part, d.prs, P, d.n[mode], d.R, d.pr, d.M, d.mrs,
                                               d.conv);
    else
        k_reduce<float><<<grid, 256, 0, st>>>((const float *)d.part, d.prs, P, d.n[mode], d.R, d.pr, d.M, d.mrs,
                                              d.conv);
    return cudaGetLastError();
}

cudaError_t launch_mttkrp(const AlsDesc &d, int mode, cudaStream_t st) {
    count_launches(1);
    return mtt_dispatch(d, mode, st);
}

cudaError_t launch_reduce_only(const AlsDesc &d, int mode, cudaStream_t st) {
    count_launches(1);
    return reduce_dispatch(d, mode, st);
}

cudaError_t launch_store_m(const AlsDesc &d, int mode, void *Mout, cudaStream_t st) {
    const long long cnt = (long long)d.n[mode] * d.R;
    unsigned blocks = (unsigned)((cnt + 255) / 256);
    count_launches(1);
    if (d.elem == 0) k_store_m<double><<<blocks, 256, 0, st>>>(d.M, (double *)Mout, cnt);
    else k_store_m<float><<<blocks, 256, 0, st>>>(d.M, (float *)Mout, cnt);
    return cudaGetLastError();
}

cudaError_t launch_reduce_tail(const AlsDesc &d, int mode, cudaStream_t st) {
    if (d.elem != 0 && !d.tail64) {
        // float32 factors: row kernel (partial reduction fused) + finish kernel
        const int RP = rp_of(d.R);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((d.n[mode] + TAIL_ROWS - 1) / TAIL_ROWS, d.nrep);
        cfg.blockDim = dim3(TAIL_THREADS);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        count_launches(1);
        // a repetition's chunks as one cluster (up to 16 CTAs) when they fit
        const int nch = (d.n[mode] + TAIL_ROWS - 1) / TAIL_ROWS;
        const bool cl = nch <= TAIL_MAX_CLUSTER;
        cudaLaunchAttribute attr2[2] = {attr[0], {}};
        if (cl) {
            attr2[1].id = cudaLaunchAttributeClusterDimension;
            attr2[1].val.clusterDim.x = (unsigned)nch;
            attr2[1].val.clusterDim.y = 1;
            attr2[1].val.clusterDim.z = 1;
            cfg.attrs = attr2;
            cfg.numAttrs = 2;
        }
        if (RP == 8) {
            cfg.dynamicSmemBytes = tail_smem_bytes<8>();
            return cl ? cudaLaunchKernelEx(&cfg, k_tail_rows<8, true>, d, mode)
                      : cudaLaunchKernelEx(&cfg, k_tail_rows<8, false>, d, mode);
        }
        if (RP == 16) {
            cfg.dynamicSmemBytes = tail_smem_bytes<16>();
            return cl ? cudaLaunchKernelEx(&cfg, k_tail_rows<16, true>, d, mode)
                      : cudaLaunchKernelEx(&cfg, k_tail_rows<16, false>, d, mode);
        }
        cfg.dynamicSmemBytes = tail_smem_bytes<32>();
        return cl ? cudaLaunchKernelEx(&cfg, k_tail_rows<32, true>, d, mode)
                  : cudaLaunchKernelEx(&cfg, k_tail_rows<32, false>, d, mode);
    }
    cudaError_t e = reduce_dispatch(d, mode, st);
    if (e != cudaSuccess) return e;
    if (d.elem == 0) k_tail<double><<<d.nrep, 256, 0, st>>>(d, mode);
    else k_tail<float><<<d.nrep, 256, 0, st>>>(d, mode);
    count_launches(2);
    return cudaGetLastError();
}

template <typename TX, int RP>
static cudaError_t raise_smem_limits() {
    cudaError_t e = cudaFuncSetAttribute(k_mtt_row<TX, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mtt_col<TX, RP, cols_for<TX, RP>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
    return e;
}

// Raise the dynamic shared-memory limits of every ALS kernel once, outside any
// stream capture.

// dynamic shared memory of both tail variants; clusters of up to 16 CTAs
template <int RP>
static cudaError_t tail_attributes() {
    const int smem = (int)tail_smem_bytes<RP>();
    const cudaFuncAttribute co = cudaFuncAttributePreferredSharedMemoryCarveout;
    cudaError_t e = cudaFuncSetAttribute(k_tail_rows<RP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tail_rows<RP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tail_rows<RP, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    // the largest carveout, like the tensor-core MTTKRP they alternate with
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tail_rows<RP, false>, co, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tail_rows<RP, true>, co, cudaSharedmemCarveoutMaxShared);
    return e;
}

cudaError_t set_als_kernel_attributes() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = raise_smem_limits<double, 8>();
    if (e == cudaSuccess) e = raise_smem_limits<double, 16>();
    if (e == cudaSuccess) e = raise_smem_limits<double, 32>();
    if (e == cudaSuccess) e = raise_smem_limits<float, 8>();
    if (e == cudaSuccess) e = raise_smem_limits<float, 16>();
    if (e == cudaSuccess) e = raise_smem_limits<float, 32>();
    if (e == cudaSuccess) e = raise_smem_limits<__nv_bfloat16, 8>();
    if (e == cudaSuccess) e = raise_smem_limits<__nv_bfloat16, 16>();
    if (e == cudaSuccess) e = raise_smem_limits<__nv_bfloat16, 32>();
    if (e == cudaSuccess) e = tail_attributes<8>();
    if (e == cudaSuccess) e = tail_attributes<16>();
    if (e == cudaSuccess) e = tail_attributes<32>();
    const cudaFuncAttribute co = cudaFuncAttributePreferredSharedMemoryCarveout;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xinv, co, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mtt_memo<16>, co, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mtt_memo<32>, co, cudaSharedmemCarveoutMaxShared);
    return e;
}

// Condition of the device-side ALS loop (the WHILE node of the ALS graph):
// run another pass while some repetition has not converged, at most
// max_passes passes (the counter is advanced here, every pass, so the loop
// always ends).
__global__ void k_als_continue(cudaGraphConditionalHandle h, const int *conv, int nrep, int *passes,
                               int max_passes) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int p = *passes + 1;
    *passes = p;
    bool more = false;
    for (int q = 0; q < nrep; ++q) more = more || conv[q] == 0;
    cudaGraphSetConditional(h, (more && p < max_passes) ? 1u : 0u);
}

cudaError_t launch_als_continue(cudaGraphConditionalHandle h, const int *conv, int nrep, int *passes,
                                int max_passes, cudaStream_t st) {
    k_als_continue<<<1, 32, 0, st>>>(h, conv, nrep, passes, max_passes);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_xinv(const AlsDesc &d, int mode, cudaStream_t st) {
    k_xinv<<<d.nrep, INV_THREADS, 0, st>>>(d, mode);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mtt_memo(const AlsDesc &d, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(d.n[2] + 1, d.nrep);
    cfg.blockDim = dim3(MEMO_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launches(1);
    if (d.R <= 16) return cudaLaunchKernelEx(&cfg, k_mtt_memo<16>, d);
    return cudaLaunchKernelEx(&cfg, k_mtt_memo<32>, d);
}

cudaError_t launch_als_mode(const AlsDesc &d, int mode, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (d.elem != 0) e = launch_xinv(d, mode, st);
    if (e == cudaSuccess) e = launch_mttkrp(d, mode, st);
    if (e != cudaSuccess) return e;
    return launch_reduce_tail(d, mode, st);
}

cudaError_t launch_als_iteration(const AlsDesc &d, cudaStream_t st) {
    for (int mode = 0; mode < 3; ++mode) {
        cudaError_t e = launch_als_mode(d, mode, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_als_prepare(const AlsDesc &d, const int *samples, long long samp_stride, int K_old,
                               bool identity, uint64_t seed, uint32_t stream_id, uint32_t batch,
                               const double *rowsq, cudaStream_t st, const WarmStart &ws) {
    if (d.elem == 0)
        k_prepare<double><<<dim3(d.nrep, 4), 256, 0, st>>>(d, samples, samp_stride, K_old, identity ? 1 : 0, seed,
                                                  stream_id, batch, rowsq, ws);
    else
        k_prepare<float><<<dim3(d.nrep, 4), 256, 0, st>>>(d, samples, samp_stride, K_old, identity ? 1 : 0, seed,
                                                 stream_id, batch, rowsq, ws);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The whole ALS of all repetitions as one persistent launch (CUDA-core
// MTTKRP path): every CTA stays resident (cooperative launch) and the
// iterations' steps are separated by a grid barrier instead of kernel
// boundaries.  Per iteration and mode: the MTTKRP's blocks (the row or column
// kernel's, as virtual blocks spread over the CTAs) -> barrier -> per
// repetition the partials summed in order and the float64 tail (CTA b takes
// repetitions b, b + grid, ...) -> barrier; after mode 3 every CTA reads the
// convergence flags and all leave together.  The same device functions and
// summation orders as the separate kernels (k_mtt_row / k_mtt_col, k_reduce,
// k_tail), so the results are the same bits as the kernel-per-step ALS with
// the float64 tail.
constexpr unsigned PA_SPIN_LIMIT = 1u << 22;

struct PersistSync {
    unsigned *words;  // PA_SYNC_WORDS, zero at launch: [0] groups arrived, [1] generation, [2] abort,
                      // [32 (1 + g)] arrivals of CTA group g (a 128-byte line each)
};

// Grid barrier in two levels: the CTAs arrive on PA_GROUPS counters (CTA b
// on counter b mod groups), the last of a group on the top counter, and the
// last group's CTA resets it and advances the generation, which the others
// poll (bounded; on timeout the error word gets ERR_TIMEOUT and every CTA
// leaves at its next barrier).  Each counter sees at most ~grid / groups
// contending atomics instead of grid.  Writes before the barrier are visible
// to every thread after it (fence, arrive, poll, fence, then the CTA
// barrier; every counter is reset before the arrival that follows it).
// Returns false if the launch is giving up.
__device__ bool pa_barrier(const PersistSync &ps, unsigned *err) {
    __shared__ int go;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned *w = ps.words;
        volatile unsigned *gen = w + 1;
        volatile int *ab = reinterpret_cast<volatile int *>(w + 2);
        const unsigned ng = min(gridDim.x, (unsigned)PA_GROUPS);
        const unsigned grp = blockIdx.x % ng;
        const unsigned gsize = gridDim.x / ng + (grp < gridDim.x % ng ? 1u : 0u);
        unsigned *gc = w + 32 * (1 + grp);
        const unsigned g = *gen;
        __threadfence();
        bool flip = false;
        if (atomicAdd(gc, 1u) == gsize - 1) {  // the last of its group
            *gc = 0;
            __threadfence();
            if (atomicAdd(w, 1u) == ng - 1) {  // the last group
                *w = 0;
                __threadfence();
                atomicAdd(w + 1, 1u);
                flip = true;
            }
        }
        if (!flip) {
            unsigned it = 0;
            while (*gen == g && !*ab) {
                if (++it > PA_SPIN_LIMIT) {
                    atomicExch(reinterpret_cast<int *>(w + 2), 1);
                    atomicOr(err, ERR_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        go = !*ab;
    }
    __syncthreads();
    return go != 0;
}

// One grid-strided pass over the items [base, base + cnt) of a sequence that
// concatenates the summary sets: the first item of this CTA at or after base.
__device__ __forceinline__ long long pa_first(long long base) {
    const long long g = gridDim.x;
    return base + (((long long)blockIdx.x - base) % g + g) % g;
}

// Copy of descriptor i into shared memory (the CTA's threads, then a barrier).
__device__ __forceinline__ void pa_load_desc(AlsDesc &sd, const AlsDesc *descs, int i) {
    static_assert(sizeof(AlsDesc) % 4 == 0, "AlsDesc copied as 32-bit words");
    const int *src = reinterpret_cast<const int *>(descs + i);
    int *dst = reinterpret_cast<int *>(&sd);
    for (int w = threadIdx.x; w < (int)(sizeof(AlsDesc) / 4); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
}

// The summary sets' descriptors, nd of them, in device memory (one context's
// update, or several contexts' updates that a server runs together).  Per
// iteration and mode: the MTTKRP's virtual blocks of every set, set after
// set, spread over the CTAs -> barrier -> the (set, repetition) pairs' partial
// sums and float64 tails -> barrier; after mode 3 every CTA reads every
// convergence flag.  Each set's arithmetic is its own: a set gives the same
// bits alone and in any batch.
template <typename TX, int RP, int COLS>
__global__ void __launch_bounds__(256) k_als_persistent(const AlsDesc *__restrict__ descs, int nd, PersistSync ps,
                                                        unsigned *err, int max_iters) {
    using TF = typename FactorOf<TX>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ AlsDesc sd;
    for (int it = 0; it < max_iters; ++it) {
        for (int mode = 0; mode < 3; ++mode) {
            long long base = 0;
            for (int i = 0; i < nd; ++i) {
                const AlsDesc &g = descs[i];
                const int njb = (g.n[1] + 32 * COLS - 1) / (32 * COLS);
                const int per = mode == 1 ? njb * g.nrs : g.nib * g.nks;
                const long long cnt = (long long)per * g.nrep;
                long long vb = pa_first(base);
                if (vb < base + cnt) {
                    pa_load_desc(sd, descs, i);
                    for (; vb < base + cnt; vb += gridDim.x) {
                        const int local = (int)(vb - base);
                        if (mode == 1) mtt_col_block<TX, RP, COLS>(sd, local % per, local / per, smem_raw);
                        else mtt_row_block<TX, RP>(sd, mode, local % per, local / per, smem_raw);
                        __syncthreads();  // shared memory (and sd) are reused next
                    }
                }
                base += cnt;
            }
            if (!pa_barrier(ps, err)) return;
            base = 0;
            for (int i = 0; i < nd; ++i) {
                const int nrep = descs[i].nrep;
                long long q = pa_first(base);
                if (q < base + nrep) {
                    pa_load_desc(sd, descs, i);
                    for (; q < base + nrep; q += gridDim.x) {
                        const int rep = (int)(q - base);
                        if (!sd.conv[rep]) {
                            // k_reduce's sums for this repetition, in partial order
                            const int n = sd.n[mode], P = sd.P[mode];
                            const TF *part = (const TF *)sd.part + rep * sd.prs;
                            for (long long e = threadIdx.x; e < (long long)n * sd.R; e += blockDim.x) {
                                const long long x = e / sd.R, r = e % sd.R;
                                sd.M[rep * sd.mrs + e] = sum_partials(part + x * sd.pr + r, P, (long long)n * sd.pr);
                            }
                        }
                        __syncthreads();
                        tail_rep<TF>(sd, mode, rep);
                        __syncthreads();
                    }
                }
                base += nrep;
            }
            if (!pa_barrier(ps, err)) return;
        }
        bool all = true;
        for (int i = 0; i < nd && all; ++i)
            for (int q = 0; q < descs[i].nrep; ++q) all = all && ((volatile const int *)descs[i].conv)[q] != 0;
        if (all) break;
    }
}

static_assert(sizeof(AlsSetArg) <= 3072, "the descriptors travel as a kernel parameter (4 KB limit)");

// descriptors into device memory, stream-ordered (block i writes set i)
__global__ void k_put_descs(AlsSetArg s, AlsDesc *dst) {
    const int *src = reinterpret_cast<const int *>(&s.d[blockIdx.x]);
    int *out = reinterpret_cast<int *>(dst + blockIdx.x);
    for (int w = threadIdx.x; w < (int)(sizeof(AlsDesc) / 4); w += blockDim.x) out[w] = src[w];
}

template <typename TX, int RP>
static cudaError_t persistent_rp(const AlsDesc *hd, const AlsDesc *dd, int nd, int max_iters, const PersistSync &ps,
                                 unsigned *err, int num_sms, cudaStream_t st) {
    constexpr int COLS = cols_for<TX, RP>();
    auto kern = k_als_persistent<TX, RP, COLS>;
    size_t smem = 0;
    long long want = 1, w3[3] = {0, 0, 0}, reps = 0;
    for (int i = 0; i < nd; ++i) {
        const AlsDesc &d = hd[i];
        smem = std::max(smem, std::max(row_smem(d), col_smem(d)));
        const int njb = (d.n[1] + 32 * COLS - 1) / (32 * COLS);
        w3[0] += (long long)d.nib * d.nks * d.nrep;
        w3[1] += (long long)njb * d.nrs * d.nrep;
        reps += d.nrep;
    }
    want = std::max(std::max(w3[0], w3[1]), reps);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // as many CTAs as the largest step has blocks, at most all co-resident
    const int grid = (int)std::min<long long>(want, (long long)per_sm * num_sms);
    const AlsDesc *dp = dd;
    int n = nd;
    PersistSync pp = ps;
    unsigned *ee = err;
    int mi = max_iters;
    void *args[] = {&dp, &n, &pp, &ee, &mi};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(256), args, smem, st);
}

template <typename TX>
static cudaError_t persistent_tx(const AlsDesc *hd, const AlsDesc *dd, int nd, int max_iters, const PersistSync &ps,
                                 unsigned *err, int num_sms, cudaStream_t st) {
    const int RP = rp_of(hd[0].R);
    if (RP == 8) return persistent_rp<TX, 8>(hd, dd, nd, max_iters, ps, err, num_sms, st);
    if (RP == 16) return persistent_rp<TX, 16>(hd, dd, nd, max_iters, ps, err, num_sms, st);
    return persistent_rp<TX, 32>(hd, dd, nd, max_iters, ps, err, num_sms, st);
}

bool persistent_compatible(const AlsDesc &a, const AlsDesc &b) { return a.elem == b.elem && rp_of(a.R) == rp_of(b.R); }

cudaError_t launch_als_persistent(const AlsDesc *descs, int nd, AlsDesc *dev_descs, int max_iters,
                                  unsigned *sync_words, unsigned *err, int num_sms, cudaStream_t st) {
    if (nd < 1 || nd > PA_MAX_SETS) return cudaErrorInvalidValue;
    for (int i = 1; i < nd; ++i)
        if (!persistent_compatible(descs[0], descs[i])) return cudaErrorInvalidValue;
    AlsSetArg s;
    for (int i = 0; i < nd; ++i) s.d[i] = descs[i];
    k_put_descs<<<nd, 64, 0, st>>>(s, dev_descs);
    count_launches(1);
    // sync_words: PA_SYNC_WORDS, zeroed here
    cudaError_t e = cudaMemsetAsync(sync_words, 0, PA_SYNC_WORDS * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    PersistSync ps{sync_words};
    if (descs[0].elem == 0) return persistent_tx<double>(descs, dev_descs, nd, max_iters, ps, err, num_sms, st);
    if (descs[0].elem == 1) return persistent_tx<float>(descs, dev_descs, nd, max_iters, ps, err, num_sms, st);
    return persistent_tx<__nv_bfloat16>(descs, dev_descs, nd, max_iters, ps, err, num_sms, st);
}

// ---------------------------------------------------------------------------
// MTTKRP op: one mode, one tensor, result in the factor type.

cudaError_t launch_mttkrp_op(AlsDesc &d, int mode, void *Mout, cudaStream_t st) {
    count_launches(3);
    cudaError_t e = mtt_dispatch(d, mode, st);
    if (e != cudaSuccess) return e;
    e = reduce_dispatch(d, mode, st);
    if (e != cudaSuccess) return e;
    const long long cnt = (long long)d.n[mode] * d.R;
    unsigned blocks = (unsigned)((cnt + 255) / 256);
    if (d.elem == 0) k_store_m<double><<<blocks, 256, 0, st>>>(d.M, (double *)Mout, cnt);
    else k_store_m<float><<<blocks, 256, 0, st>>>(d.M, (float *)Mout, cnt);
    return cudaGetLastError();
}

}  // namespace sbt
