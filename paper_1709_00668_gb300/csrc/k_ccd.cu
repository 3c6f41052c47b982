// Core consistency diagnostic (CorConDia, Bro & Kiers 2003) of a CP model of
// a dense slice-major tensor: the quality rating GetRank scores every
// candidate decomposition with (Section 3.2, Algorithm 2).
//
//   CorConDia = 100 (1 - ||G - T||^2 / R),
//   G = X x_1 A+ x_2 B+ x_3 (C diag(lambda))+,   T = superdiagonal of ones,
//
// with F+ = (F^T F)^-1 F^T the least-squares inverse of a full-column-rank
// factor.  Everything runs in float64 (a diagnostic, not the per-iteration
// path), every sum in a fixed order:
//   k_ccd_pinv   one CTA per factor: Gram, Gauss-Jordan inverse (pivots
//                checked), F+ (R x n)
//   k_ccd_z      Z[k][i][q] = sum_j X[k][i][j] B+[q][j]   (warp per row)
//   k_ccd_t1     T1[k][p][q] = sum_i A+[p][i] Z[k][i][q]
//   k_ccd_core   G[p][q][s] = sum_k C+[s][k] T1[k][p][q]
//   k_ccd_final  the diagnostic from G
#include "sbt_internal.cuh"

namespace sbt {

constexpr int CCD_THREADS = 256;

// value of a summary element as float64 (bfloat16 widened exactly)
__device__ __forceinline__ double ccd_value(double v) { return v; }
__device__ __forceinline__ double ccd_value(float v) { return (double)v; }
__device__ __forceinline__ double ccd_value(__nv_bfloat16 v) { return (double)__bfloat162float(v); }


// F+ = (F^T F)^-1 F^T of F' = F diag(scale) (scale null: ones); F row-major n x R.
// status bit 1: a pivot of the Gram was not positive (F' rank-deficient).
__global__ void __launch_bounds__(CCD_THREADS) k_ccd_pinv(const double *F, long long n, int R, const double *scale,
                                                         double *P, int *status) {
    __shared__ double W[32][65];  // [G | I], R x 2R
    const int t = threadIdx.x;
    for (int pq = t; pq < R * R; pq += blockDim.x) {
        const int p = pq / R, q = pq % R;
        double a = 0.0;
        for (long long x = 0; x < n; ++x) a = fma(F[x * R + p], F[x * R + q], a);
        if (scale) a *= scale[p] * scale[q];
        W[p][q] = a;
        W[p][R + q] = p == q ? 1.0 : 0.0;
    }
    __syncthreads();
    __shared__ int bad;
    if (t == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < R; ++k) {
        const double piv = W[k][k];
        if (!(piv > 0.0)) {
            if (t == 0) bad = 1;
            break;  // uniform: every thread read the same pivot
        }
        const double inv = 1.0 / piv;
        constexpr int EPT = 2 * 32 * 32 / CCD_THREADS;  // entries of [G | I] per thread
        double nv[EPT];
#pragma unroll
        for (int c = 0; c < EPT; ++c) {
            const int e = t + c * CCD_THREADS;
            if (e < R * 2 * R) {
                const int i = e / (2 * R), j = e % (2 * R);
                const double tt = W[k][j] * inv;
                nv[c] = i == k ? tt : W[i][j] - W[i][k] * tt;
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < EPT; ++c) {
            const int e = t + c * CCD_THREADS;
            if (e < R * 2 * R) W[e / (2 * R)][e % (2 * R)] = nv[c];
        }
        __syncthreads();
    }
    __syncthreads();
    if (bad) {
        if (t == 0) atomicOr(status, 1);
        return;
    }
    // P[p][x] = sum_q Ginv[p][q] F'(x, q)
    for (long long x = t; x < n; x += blockDim.x) {
        for (int p = 0; p < R; ++p) {
            double a = 0.0;
            for (int q = 0; q < R; ++q) a = fma(W[p][R + q], F[x * R + q] * (scale ? scale[q] : 1.0), a);
            P[(long long)p * n + x] = a;
        }
    }
}

// Z[k][i][q] = sum_j X[k][i][j] B+[q][j]: a warp per row (k, i), lanes over j,
// a lane-order tree per q
template <typename T>
__global__ void __launch_bounds__(CCD_THREADS) k_ccd_z(const T *X, long long K, long long I, long long J,
                                                      long long ld, const double *PB, int R, double *Z) {
    const int lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * (CCD_THREADS / 32) + (threadIdx.x >> 5);
    if (row >= K * I) return;
    const T *x = X + row * ld;
    double z[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) z[q] = 0.0;
    for (long long j = lane; j < J; j += 32) {
        const double v = ccd_value(x[j]);
#pragma unroll
        for (int q = 0; q < 32; ++q)
            if (q < R) z[q] = fma(v, PB[(long long)q * J + j], z[q]);
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        if (q < R) {
            const double s = warp_sum(z[q]);
            if (lane == 0) Z[row * R + q] = s;
        }
    }
}

// T1[k][p][q] = sum_i A+[p][i] Z[k][i][q], one thread per (k, p, q)
__global__ void __launch_bounds__(CCD_THREADS) k_ccd_t1(const double *Z, const double *PA, long long K, long long I,
                                                       int R, double *T1) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= K * R * R) return;
    const long long k = e / (R * R);
    const int p = (int)(e / R % R), q = (int)(e % R);
    double a = 0.0;
    for (long long i = 0; i < I; ++i) a = fma(PA[(long long)p * I + i], Z[(k * I + i) * R + q], a);
    T1[e] = a;
}

// G[p][q][s] = sum_k C+[s][k] T1[k][p][q], one thread per (p, q, s)
__global__ void __launch_bounds__(CCD_THREADS) k_ccd_core(const double *T1, const double *PC, long long K, int R,
                                                         double *G) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= R * R * R) return;
    const int p = e / (R * R), q = e / R % R, s = e % R;
    double a = 0.0;
    for (long long k = 0; k < K; ++k) a = fma(PC[(long long)s * K + k], T1[(k * R + p) * R + q], a);
    G[e] = a;
}

// 100 (1 - sum (G - T)^2 / R), one CTA, a fixed-order tree
__global__ void __launch_bounds__(CCD_THREADS) k_ccd_final(const double *G, int R, double *out) {
    __shared__ double red[CCD_THREADS / 32];
    double a = 0.0;
    for (int e = threadIdx.x; e < R * R * R; e += blockDim.x) {
        const int p = e / (R * R), q = e / R % R, s = e % R;
        const double d = G[e] - ((p == q && q == s) ? 1.0 : 0.0);
        a = fma(d, d, a);
    }
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < CCD_THREADS / 32; ++w) s += red[w];
        *out = 100.0 * (1.0 - s / R);
    }
}

// float32 factor rows widened to float64 (the GetRank candidates' factors)
__global__ void k_ccd_widen(const float *in, double *out, long long n) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = (double)in[e];
}

cudaError_t launch_widen(const float *in, double *out, long long n, cudaStream_t st) {
    count_launches(1);
    k_ccd_widen<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_core_consistency(int elem, const void *X, long long K, long long I, long long J, long long ld,
                                    const double *lam, const double *A, const double *B, const double *C, int R,
                                    double *scratch, int *status, double *out, cudaStream_t st) {
    double *PA = scratch, *PB = PA + (size_t)R * I, *PC = PB + (size_t)R * J, *Z = PC + (size_t)R * K;
    double *T1 = Z + (size_t)K * I * R, *G = T1 + (size_t)K * R * R;
    k_ccd_pinv<<<1, CCD_THREADS, 0, st>>>(A, I, R, nullptr, PA, status);
    k_ccd_pinv<<<1, CCD_THREADS, 0, st>>>(B, J, R, nullptr, PB, status);
    k_ccd_pinv<<<1, CCD_THREADS, 0, st>>>(C, K, R, lam, PC, status);
    const long long rows = K * I;
    const unsigned zb = (unsigned)((rows + CCD_THREADS / 32 - 1) / (CCD_THREADS / 32));
    if (elem == 0) k_ccd_z<double><<<zb, CCD_THREADS, 0, st>>>((const double *)X, K, I, J, ld, PB, R, Z);
    else if (elem == 1) k_ccd_z<float><<<zb, CCD_THREADS, 0, st>>>((const float *)X, K, I, J, ld, PB, R, Z);
    else k_ccd_z<__nv_bfloat16><<<zb, CCD_THREADS, 0, st>>>((const __nv_bfloat16 *)X, K, I, J, ld, PB, R, Z);
    const long long n1 = K * R * R;
    k_ccd_t1<<<(unsigned)((n1 + CCD_THREADS - 1) / CCD_THREADS), CCD_THREADS, 0, st>>>(Z, PA, K, I, R, T1);
    k_ccd_core<<<(R * R * R + CCD_THREADS - 1) / CCD_THREADS, CCD_THREADS, 0, st>>>(T1, PC, K, R, G);
    k_ccd_final<<<1, CCD_THREADS, 0, st>>>(G, R, out);
    count_launches(7);
    return cudaGetLastError();
}

size_t core_consistency_scratch_doubles(long long K, long long I, long long J, int R) {
    return (size_t)R * (I + J + K) + (size_t)K * I * R + (size_t)K * R * R + (size_t)R * R * R + 1;
}

}  // namespace sbt
