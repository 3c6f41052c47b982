// CP-ALS on the r summaries (Alg. 1 step 5), batched over repetitions.
//
// Per iteration and mode n: MTTKRP partial sums (one CTA per tile, no atomics),
// a fixed-order reduction of the partials, and a per-repetition tail that
// forms V = Hadamard of the other Grams, factors it (float64 Cholesky),
// inverts it, solves U_n = M_n V^-1, normalises columns (lambda) and refreshes
// the Gram; after mode 3 the tail computes the fit and the convergence flag.
// Every reduction runs in a fixed order, so results do not depend on timing.
#include "sbt_internal.cuh"

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
__global__ void __launch_bounds__(256) k_mtt_row(AlsDesc d, int mode) {
    using TF = typename FactorOf<TX>::T;
    constexpr int V = VecLd<TX, TF>::V;
    const int rep = blockIdx.y;
    if (d.conv[rep]) return;
    const int NI = d.n[0], NJ = d.n[1], Kp = d.n[2], R = d.R, ldj = d.ldj;
    const int ib = blockIdx.x % d.nib, ks = blockIdx.x / d.nib;
    const int k0 = ks * d.spc, k1 = min(Kp, k0 + d.spc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ii = ib * 8 + warp;
    const int jc = d.jc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
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
            part[((long long)ks * NI + ii) * R + lane] = s;
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
            part[((long long)ib * Kp + (k0 + t)) * R + r] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// Column kernel: mode 2.  A CTA owns 32*COLS columns jj and a range of
// flattened rows (kk, ii); M2(jj, r) += X[kk][ii][jj] A(ii,r) C(kk,r).  Each
// warp takes every 8th row; warps are summed in shared memory in fixed order.
template <typename TX, int RP, int COLS>
__global__ void __launch_bounds__(256) k_mtt_col(AlsDesc d) {
    using TF = typename FactorOf<TX>::T;
    const int rep = blockIdx.y;
    if (d.conv[rep]) return;
    const int NI = d.n[0], NJ = d.n[1], Kp = d.n[2], R = d.R, ldj = d.ldj;
    const int njb = (NJ + 32 * COLS - 1) / (32 * COLS);
    const int jb = blockIdx.x % njb, rs = blockIdx.x / njb;
    const long long rows = (long long)Kp * NI;
    const long long r0 = (long long)rs * d.rows_per, r1 = min(rows, r0 + d.rows_per);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = jb * 32 * COLS + lane * COLS;
    if (d.bytes_ctr && threadIdx.x == 0) {
        const int cols = min(NJ, (jb + 1) * 32 * COLS) - jb * 32 * COLS;
        atomicAdd(d.bytes_ctr, (unsigned long long)max(0LL, r1 - r0) * cols * sizeof(TX));
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
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
        part[((long long)rs * NJ + jj) * R + r] = s;
    }
}

// ---------------------------------------------------------------------------
// Fixed-order reduction of the partials: M[rep][e] = sum_p part[rep][p][e]
template <typename TF>
__global__ void k_reduce(const TF *part, long long prs, int P, long long cnt, double *M, long long mrs,
                         const int *conv) {
    const int rep = blockIdx.y;
    if (conv[rep]) return;
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    const TF *p = part + rep * prs + e;
    double s = 0.0;
    for (int q = 0; q < P; ++q) s += (double)p[(long long)q * cnt];
    M[rep * mrs + e] = s;
}

// ---------------------------------------------------------------------------
// float64 helpers of the tail: Cholesky, inverse, by one warp (R <= 32)
__device__ bool warp_cholesky(const double *V, double *L, int R, int lane) {
    // L lower triangular, row-major 32x32
    bool ok = true;
    for (int j = 0; j < R; ++j) {
        if (lane == j) {
            double s = V[j * 32 + j];
            for (int k = 0; k < j; ++k) s -= L[j * 32 + k] * L[j * 32 + k];
            L[j * 32 + j] = (s > 0.0 && isfinite(s)) ? sqrt(s) : -1.0;
        }
        __syncwarp();
        const double djj = L[j * 32 + j];
        if (!(djj > 0.0)) ok = false;
        if (ok && lane > j && lane < R) {
            double s = V[lane * 32 + j];
            for (int k = 0; k < j; ++k) s -= L[lane * 32 + k] * L[j * 32 + k];
            L[lane * 32 + j] = s / djj;
        }
        __syncwarp();
        if (!ok) break;
    }
    return ok;
}

// Vi = (L L^T)^-1: lane c solves L y = e_c, then L^T x = y.
__device__ void warp_chol_inverse(const double *L, double *Vi, int R, int lane) {
    if (lane < R) {
        double y[32];
        for (int i = 0; i < R; ++i) {
            double s = (i == lane) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i * 32 + k] * y[k];
            y[i] = s / L[i * 32 + i];
        }
        for (int i = R - 1; i >= 0; --i) {
            double s = y[i];
            for (int k = i + 1; k < R; ++k) s -= L[k * 32 + i] * y[k];
            y[i] = s / L[i * 32 + i];
        }
        for (int i = 0; i < R; ++i) Vi[i * 32 + lane] = y[i];
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Tail of one mode for one repetition (one CTA per repetition).
template <typename TF>
__global__ void __launch_bounds__(256) k_tail(AlsDesc d, int mode) {
    const int rep = blockIdx.x;
    if (d.conv[rep]) return;
    const int R = d.R, n = d.n[mode];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ double V[32 * 32], L[32 * 32], Vi[32 * 32];
    __shared__ double lam_s[32];
    __shared__ int chol_ok, reg_flag, zero_flag;
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
        reg_flag = 0;
        zero_flag = 0;
    }
    __syncthreads();
    if (warp == 0) {
        bool ok = warp_cholesky(V, L, R, lane);
        if (!ok) {
            // V + 1e-12 tr(V)/R I
            double tr = 0.0;
            for (int i = 0; i < R; ++i) tr += V[i * 32 + i];
            __syncwarp();
            if (lane < R) V[lane * 32 + lane] += 1e-12 * tr / R;
            __syncwarp();
            ok = warp_cholesky(V, L, R, lane);
            if (lane == 0) reg_flag = 1;
        }
        if (lane == 0) chol_ok = ok;
        __syncwarp();
        if (ok) warp_chol_inverse(L, Vi, R, lane);
    }
    __syncthreads();
    if (!chol_ok) {
        // singular even after the shift: leave the factor, flag
        if (threadIdx.x == 0) atomicOr(&d.flags[rep], SBT_FLAG_CHOL_REGULARIZED_DEV);
        return;
    }
    // U = M Vi (float64 arithmetic, stored as TF)
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        double m[32];
        for (int s = 0; s < R; ++s) m[s] = M[(long long)x * R + s];
        for (int r = 0; r < R; ++r) {
            double acc = 0.0;
            for (int s = 0; s < R; ++s) acc += m[s] * Vi[s * 32 + r];
            U[(long long)x * R + r] = (TF)acc;
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
                zero_flag = 1;
            }
            lam_s[r] = l;
        }
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)n * R; e += blockDim.x) {
        int r = (int)(e % R);
        U[e] = (TF)((double)U[e] / lam_s[r]);
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
        if (reg_flag) f |= SBT_FLAG_CHOL_REGULARIZED_DEV;
        if (zero_flag) f |= SBT_FLAG_ZERO_COLUMN_DEV;
        if (f) d.flags[rep] |= f;
    }
    if (mode == 2) {
        // fit = 1 - ||X - X_hat|| / ||X||
        __shared__ double red[8];
        double inner = 0.0;
        for (long long e = threadIdx.x; e < (long long)n * R; e += blockDim.x) {
            int r = (int)(e % R);
            inner += lam_s[r] * M[e] * (double)U[e];
        }
        inner = warp_sum(inner);
        if (lane == 0) red[warp] = inner;
        __syncthreads();
        if (threadIdx.x == 0) {
            double in = 0.0;
            for (int w = 0; w < 8; ++w) in += red[w];
            double xh = 0.0;
            for (int r = 0; r < R; ++r)
                for (int s = 0; s < R; ++s)
                    xh += lam_s[r] * lam_s[s] * G[r * R + s] * G[R * R + r * R + s] * G[2 * R * R + r * R + s];
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

// ---------------------------------------------------------------------------
// Start values, Grams and ||X_s||^2 (one CTA per repetition)
template <typename TF>
__global__ void __launch_bounds__(256) k_prepare(AlsDesc d, const int *samples, long long samp_stride,
                                                 int K_old, int identity, uint64_t seed,
                                                 uint32_t stream_id, uint32_t batch,
                                                 const double *rowsq) {
    const int rep = blockIdx.x;
    const int R = d.R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint2 key = philox_key(seed, stream_id);
    for (int m = 0; m < 3; ++m) {
        const int n = d.n[m];
        TF *U = (TF *)d.U[m] + (long long)rep * n * R;
        const int *S = samples ? samples + (long long)(rep * 3 + m) * samp_stride : nullptr;
        for (long long e = threadIdx.x; e < (long long)n * R; e += blockDim.x) {
            int x = (int)(e / R), r = (int)(e % R);
            uint32_t gx;
            if (identity) gx = (uint32_t)x;
            else if (m < 2) gx = (uint32_t)S[x];
            else gx = (uint32_t)(x < d.nK ? S[x] : K_old + (x - d.nK));
            U[e] = (TF)init_value(key, gx, r, m, rep, batch);
        }
    }
    __syncthreads();
    double *G = d.G + (long long)rep * 3 * R * R;
    const int npairs = R * (R + 1) / 2;
    for (int m = 0; m < 3; ++m) {
        const int n = d.n[m];
        const TF *U = (const TF *)d.U[m] + (long long)rep * n * R;
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
                G[m * R * R + r * R + s] = a;
                G[m * R * R + s * R + r] = a;
            }
        }
    }
    // ||X_s||^2 from the row sums, fixed order
    __shared__ double red[256];
    const long long rows = (long long)d.n[2] * d.n[0];
    const double *rq = rowsq + rep * rows;
    double a = 0.0;
    for (long long e = threadIdx.x; e < rows; e += blockDim.x) a += rq[e];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s = 128; s; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        d.normX2[rep] = red[0];
        d.fit_prev[rep] = 0.0;
        d.fit[rep] = 0.0;
        d.iters[rep] = 0;
        d.conv[rep] = 0;
        d.flags[rep] = (min(min(d.n[0], d.n[1]), d.nK) < R) ? SBT_FLAG_SAMPLE_LT_RANK_DEV : 0;
    }
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
    d.rows_per = (rows + nrs - 1) / nrs;
    d.nrs = (int)((rows + d.rows_per - 1) / d.rows_per);
    d.P[0] = d.nks;
    d.P[1] = d.nrs;
    d.P[2] = d.nib;
}

long long partial_elems(const AlsDesc &d) {
    long long a = (long long)d.nks * d.n[0];
    long long b = (long long)d.nrs * d.n[1];
    long long c = (long long)d.nib * d.n[2];
    return std::max(a, std::max(b, c)) * d.R;
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
    static bool attr = false;  // per instantiation
    if (!attr) {
        cudaFuncSetAttribute(k_mtt_row<TX, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    dim3 grid(d.nib * d.nks, d.nrep);
    k_mtt_row<TX, RP><<<grid, 256, sm, st>>>(d, mode);
    return cudaGetLastError();
}

template <typename TX, int RP, int COLS>
static cudaError_t run_col(const AlsDesc &d, cudaStream_t st) {
    size_t sm = col_smem(d);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_mtt_col<TX, RP, COLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
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
        k_reduce<double><<<grid, 256, 0, st>>>((const double *)d.part, d.prs, P, cnt, d.M, d.mrs, d.conv);
    else
        k_reduce<float><<<grid, 256, 0, st>>>((const float *)d.part, d.prs, P, cnt, d.M, d.mrs, d.conv);
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
    cudaError_t e = reduce_dispatch(d, mode, st);
    if (e != cudaSuccess) return e;
    if (d.elem == 0) k_tail<double><<<d.nrep, 256, 0, st>>>(d, mode);
    else k_tail<float><<<d.nrep, 256, 0, st>>>(d, mode);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_als_mode(const AlsDesc &d, int mode, cudaStream_t st) {
    cudaError_t e = launch_mttkrp(d, mode, st);
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
                               const double *rowsq, cudaStream_t st) {
    if (d.elem == 0)
        k_prepare<double><<<d.nrep, 256, 0, st>>>(d, samples, samp_stride, K_old, identity ? 1 : 0, seed,
                                                  stream_id, batch, rowsq);
    else
        k_prepare<float><<<d.nrep, 256, 0, st>>>(d, samples, samp_stride, K_old, identity ? 1 : 0, seed,
                                                 stream_id, batch, rowsq);
    count_launches(1);
    return cudaGetLastError();
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
