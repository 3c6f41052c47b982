// Kernels before the ALS: Philox op, max |x|, append + Eq. 1 marginals,
// weighted sampling without replacement, summary gather.
#include "sbt_internal.cuh"

namespace sbt {

// ---------------------------------------------------------------------------
// Philox op
__global__ void k_philox(const uint4 *ctr, uint2 key, uint4 *out, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

cudaError_t launch_philox(const uint32_t *ctr, uint2 key, uint32_t *out, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    k_philox<<<(unsigned)blocks, 256, 0, st>>>((const uint4 *)ctr, key, (uint4 *)out, n);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// max |x| (as ordered bits of a non-negative double) and non-finite detection
template <typename T>
__global__ void k_absmax(const T *X, long long n, DevStatus *status) {
    T m = 0;
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const T v = X[i];
        if (!isfinite(v)) bad = true;
        else m = fmax(m, fabs(v));
    }
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    unsigned anybad = __ballot_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&status->amax_bits, (unsigned long long)__double_as_longlong((double)m));
        if (anybad) atomicOr(&status->err, ERR_NONFINITE);
    }
}

cudaError_t launch_absmax(const void *X, int dtype, long long n, DevStatus *status, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    count_launches(1);
    if (dtype == 0)
        k_absmax<double><<<(unsigned)blocks, 256, 0, st>>>((const double *)X, n, status);
    else
        k_absmax<float><<<(unsigned)blocks, 256, 0, st>>>((const float *)X, n, status);
    return cudaGetLastError();
}

constexpr int APPEND_ROWS = 128;  // rows (k, i) of the new slices per CTA
constexpr int APPEND_THREADS = 256;

// One pass over the new slices: copy them into the store and add the
// fixed-point squares q(x) to x_a (per row i), x_b (per column j) and x_c
// (per slice k).  A CTA covers APPEND_ROWS consecutive rows (k, i) and one
// chunk of 256 * V columns; each thread owns V adjacent columns (one 16-byte
// vector when the rows are aligned), so its column sums stay in registers.
// Row sums are reduced per warp, then over the CTA's warps.  All sums are
// exact 64-bit integers, so the atomics may land in any order.
template <typename T>
__global__ void __launch_bounds__(APPEND_THREADS) k_append(const T *Xin, long long nrows, int I, int J, int ldin,
                                                           T *store, int lds, int S, int vec_ok, int inplace,
                                                           unsigned long long *dxa, unsigned long long *dxb,
                                                           unsigned long long *xc_new, unsigned *samax,
                                                           DevStatus *status) {
    constexpr int V = 16 / sizeof(T);
    constexpr int NW = APPEND_THREADS / 32;
    const long long r0 = (long long)blockIdx.x * APPEND_ROWS;
    const int rows = (int)min((long long)APPEND_ROWS, nrows - r0);
    const int jc = blockIdx.y * (APPEND_THREADS * V) + threadIdx.x * V;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ unsigned long long rowp[APPEND_ROWS][NW];
    __shared__ unsigned long long slice_acc[APPEND_ROWS + 1];
    __shared__ unsigned slice_max[APPEND_ROWS + 1];  // max |x| per slice (float bits: ordered as integers)
    __shared__ int range_flag;
    if (threadIdx.x == 0) range_flag = 0;
    for (int t = threadIdx.x; t <= APPEND_ROWS; t += APPEND_THREADS) {
        slice_acc[t] = 0;
        slice_max[t] = 0;
    }
    __syncthreads();
    const long long k_first = r0 / I;
    unsigned long long cs[V];
#pragma unroll
    for (int v = 0; v < V; ++v) cs[v] = 0;
    bool bad = false, range = false;
    const bool vec = vec_ok && jc + V <= J;
    // rows in groups of AU: the loads of a group are issued before any of
    // its rows is processed (several vectors in flight per thread)
    constexpr int AU = 4;
    for (int t0 = 0; t0 < rows; t0 += AU) {
        T xs[AU][V];
#pragma unroll
        for (int u = 0; u < AU; ++u) {
            const long long r = r0 + t0 + u;
            if (t0 + u < rows && jc < J) {
                const T *src = Xin + r * ldin + jc;
                if (vec) {
                    *reinterpret_cast<uint4 *>(xs[u]) = *reinterpret_cast<const uint4 *>(src);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) xs[u][v] = jc + v < J ? src[v] : T(0);
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) xs[u][v] = T(0);
            }
        }
        if (!inplace) {
#pragma unroll
            for (int u = 0; u < AU; ++u) {
                const long long r = r0 + t0 + u;
                if (t0 + u < rows && jc < J) {
                    T *dst = store + r * lds + jc;
                    if (vec) {
                        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(xs[u]);
                    } else {
#pragma unroll
                        for (int v = 0; v < V; ++v)
                            if (jc + v < J) dst[v] = xs[u][v];
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < AU; ++u) {
            const int t = t0 + u;
            if (t >= rows) break;
            const long long r = r0 + t;
            unsigned long long rp = 0;
            float am = 0.f;
            if (jc < J) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const T x = xs[u][v];
                    unsigned long long q = 0;
                    if (samax) am = fmaxf(am, fabsf((float)x));
                    if (!isfinite(x)) bad = true;
                    else if (!qsquare(x, S, &q)) range = true;
                    if (cs[v] + q < cs[v]) range = true;
                    cs[v] += q;
                    if (rp + q < rp) range = true;
                    rp += q;
                }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, rp, o);
                if (rp + other < rp) range = true;
                rp += other;
            }
            if (lane == 0) rowp[t][warp] = rp;
            if (samax) {
#pragma unroll
                for (int o = 16; o; o >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
                if (lane == 0 && am > 0.f) atomicMax(&slice_max[r / I - k_first], __float_as_uint(am));
            }
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&status->err, ERR_NONFINITE);
    if (range) range_flag = 1;
    __syncthreads();
    // rows: x_a[i] += row sum; slice sums gathered per slice in shared memory
    for (int t = threadIdx.x; t < rows; t += APPEND_THREADS) {
        unsigned long long s = 0;
        bool ov = false;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            if (s + rowp[t][w] < s) ov = true;
            s += rowp[t][w];
        }
        const long long r = r0 + t;
        const long long k = r / I;
        const int i = (int)(r - k * I);
        add_checked(&dxa[i], s, status);
        if (s) {
            const unsigned long long old = atomicAdd(&slice_acc[k - k_first], s);
            if (old + s < old) ov = true;
        }
        if (ov) range_flag = 1;
    }
    __syncthreads();
    const int nslices = (int)((r0 + rows - 1) / I - k_first) + 1;
    for (int t = threadIdx.x; t < nslices; t += APPEND_THREADS) {
        add_checked(&xc_new[k_first + t], slice_acc[t], status);
        if (samax && slice_max[t]) atomicMax(&samax[k_first + t], slice_max[t]);
    }
    // columns: x_b[j] += column sums of this CTA's rows
#pragma unroll
    for (int v = 0; v < V; ++v)
        if (jc + v < J) add_checked(&dxb[jc + v], cs[v], status);
    if (threadIdx.x == 0 && range_flag) atomicOr(&status->err, ERR_RANGE);
}

cudaError_t launch_append(const void *Xin, int dtype, long long K_new, int I, int J, int ldin, void *store,
                          int lds, int S, unsigned long long *dxa, unsigned long long *dxb,
                          unsigned long long *xc_new, unsigned *samax, DevStatus *status, cudaStream_t st) {
    if (K_new <= 0) return cudaSuccess;
    const long long nrows = K_new * I;
    const int V = dtype == 0 ? 2 : 4;
    dim3 grid((unsigned)((nrows + APPEND_ROWS - 1) / APPEND_ROWS), (J + APPEND_THREADS * V - 1) / (APPEND_THREADS * V));
    const int vec_ok = ldin % V == 0 && lds % V == 0 && ((uintptr_t)Xin & 15) == 0 && ((uintptr_t)store & 15) == 0;
    const int inplace = Xin == store && ldin == lds;  // the initial tensor is already in the store
    count_launches(1);
    if (dtype == 0)
        k_append<double><<<grid, APPEND_THREADS, 0, st>>>((const double *)Xin, nrows, I, J, ldin, (double *)store, lds,
                                                          S, vec_ok, inplace, dxa, dxb, xc_new, samax, status);
    else
        k_append<float><<<grid, APPEND_THREADS, 0, st>>>((const float *)Xin, nrows, I, J, ldin, (float *)store, lds,
                                                         S, vec_ok, inplace, dxa, dxb, xc_new, samax, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Weighted sampling without replacement (Section 3.1, Alg. 1 step 3).
// Exponential keys: key = floor(L * 2^64 / w), L = -log2(u) in Q.32 with
// u = (2v+1) / 2^33 and v Philox word 0 on counter (x, mode | rep<<4, batch, 1).
// The n smallest (key, x) are found by an MSB-first radix select over the
// composite (key_hi:40 | key_lo:64 | x:32) and compacted in index order.

// Q.32 binary logarithm of 1 <= t < 2^33 by repeated squaring (Turner 2010):
// y = t / 2^p held as Q1.62; each squaring is truncated back to Q2.62 and a
// square at or above 2 emits a one bit and is halved.
__device__ __forceinline__ unsigned long long log2_q32(unsigned long long t) {
    int p = 63 - __clzll((long long)t);
    unsigned long long y = t << (62 - p);
    unsigned long long f = 0;
#pragma unroll 4
    for (int b = 0; b < 32; ++b) {
        unsigned long long hi = __umul64hi(y, y), lo = y * y;
        y = (hi << 2) | (lo >> 62);
        f <<= 1;
        if (y >> 63) {
            f |= 1ull;
            y >>= 1;
        }
    }
    return ((unsigned long long)p << 32) | f;
}

// floor(L * 2^64 / w) for L < 2^38, w >= 1: high word L / w; the low word by
// restoring division of (L mod w) * 2^64.
__device__ __forceinline__ void key_div(unsigned long long L, unsigned long long w,
                                        unsigned long long *qhi, unsigned long long *qlo) {
    *qhi = L / w;
    unsigned long long rem = L % w, q = 0;
    for (int b = 0; b < 64; ++b) {
        bool carry = rem >> 63;
        rem <<= 1;
        q <<= 1;
        if (carry || rem >= w) {
            rem -= w;
            q |= 1ull;
        }
    }
    *qlo = q;
}

constexpr unsigned long long KEY_HI_MAX = 0xFFFFFFFFFFull;  // 40 bits: never drawn

__device__ __forceinline__ unsigned digit_of(int d, unsigned long long hi, unsigned long long lo,
                                             unsigned x) {
    if (d < 5) return (unsigned)(hi >> (32 - 8 * d)) & 0xFFu;
    if (d < 13) return (unsigned)(lo >> (56 - 8 * (d - 5))) & 0xFFu;
    return (x >> (24 - 8 * (d - 13))) & 0xFFu;
}

struct Prefix {
    unsigned long long m2, m1, v2, v1;
    unsigned m0, v0;
};

__device__ __forceinline__ bool prefix_eq(const Prefix &p, unsigned long long hi,
                                          unsigned long long lo, unsigned x) {
    return ((hi & p.m2) == p.v2) && ((lo & p.m1) == p.v1) && ((x & p.m0) == p.v0);
}
__device__ __forceinline__ bool prefix_le(const Prefix &p, unsigned long long hi,
                                          unsigned long long lo, unsigned x) {
    unsigned long long a2 = hi & p.m2, a1 = lo & p.m1;
    unsigned a0 = x & p.m0;
    if (a2 != p.v2) return a2 < p.v2;
    if (a1 != p.v1) return a1 < p.v1;
    return a0 <= p.v0;
}

__global__ void __launch_bounds__(1024) k_sample(SampleParams sp) {
    const int nm = sp.nmodes;
    const int b = blockIdx.x;
    const int rep_local = b / nm, mi = b % nm;
    const int rep = sp.rep0 + rep_local;
    const int mode = sp.mode_id[mi];
    const unsigned long long *w = sp.w[mi];
    const int N = sp.N[mi], n = sp.n[mi];
    int *out = sp.out + (long long)b * sp.out_stride;
    unsigned long long *khi = sp.khi + (long long)b * sp.key_stride;
    unsigned long long *klo = sp.klo + (long long)b * sp.key_stride;
    const uint2 key = philox_key(sp.seed, sp.stream_id);

    __shared__ unsigned hist[256];
    __shared__ Prefix pre;
    __shared__ int krem, done, npos_s;
    __shared__ int warp_tot[32];
    __shared__ int base_s, chunk_s;

    if (threadIdx.x == 0) {
        npos_s = 0;
        pre.m2 = pre.m1 = pre.v2 = pre.v1 = 0;
        pre.m0 = pre.v0 = 0;
        krem = n;
        done = 0;
        base_s = 0;
    }
    __syncthreads();
    int mypos = 0;
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        unsigned long long wx = w[x];
        if (wx == 0) {
            khi[x] = KEY_HI_MAX;
            klo[x] = ~0ull;
        } else {
            uint4 r = philox4x32_10(make_uint4((uint32_t)x, (uint32_t)mode | ((uint32_t)rep << 4),
                                               sp.batch, 1u), key);
            unsigned long long t = 2ull * r.x + 1ull;
            unsigned long long L = (33ull << 32) - log2_q32(t);
            unsigned long long qh, ql;
            key_div(L, wx, &qh, &ql);
            khi[x] = qh;
            klo[x] = ql;
            ++mypos;
        }
    }
    atomicAdd(&npos_s, mypos);
    __syncthreads();
    if (n > npos_s) {
        if (threadIdx.x == 0) atomicOr(&sp.status->err, ERR_SAMPLE);
        return;
    }
    if (n == 0) return;
    __threadfence_block();

    for (int d = 0; d < 17; ++d) {
        for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[t] = 0;
        __syncthreads();
        Prefix p = pre;
        for (int x = threadIdx.x; x < N; x += blockDim.x) {
            unsigned long long hi = khi[x], lo = klo[x];
            if (prefix_eq(p, hi, lo, (unsigned)x)) atomicAdd(&hist[digit_of(d, hi, lo, (unsigned)x)], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int cum = 0, bsel = 0;
            for (bsel = 0; bsel < 255; ++bsel) {
                if (cum + (int)hist[bsel] >= krem) break;
                cum += hist[bsel];
            }
            krem -= cum;
            unsigned long long dm = 0xFFull;
            if (d < 5) {
                int sh = 32 - 8 * d;
                pre.m2 |= dm << sh;
                pre.v2 |= (unsigned long long)bsel << sh;
            } else if (d < 13) {
                int sh = 56 - 8 * (d - 5);
                pre.m1 |= dm << sh;
                pre.v1 |= (unsigned long long)bsel << sh;
            } else {
                int sh = 24 - 8 * (d - 13);
                pre.m0 |= 0xFFu << sh;
                pre.v0 |= (unsigned)bsel << sh;
            }
            if ((int)hist[bsel] == krem) done = 1;
        }
        __syncthreads();
        if (done) break;
    }

    // compaction in index order
    const Prefix p = pre;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = 0; c < N; c += blockDim.x) {
        int x = c + threadIdx.x;
        bool f = (x < N) && prefix_le(p, khi[x], klo[x], (unsigned)x);
        unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_tot[wid] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int q = 0; q < nw; ++q) {
                int v = warp_tot[q];
                warp_tot[q] = s;
                s += v;
            }
            chunk_s = s;
        }
        __syncthreads();
        const int chunk_total = chunk_s;
        const int pos = base_s + warp_tot[wid] + __popc(bal & ((1u << lane) - 1u));
        if (f && pos < n) out[pos] = x;
        __syncthreads();
        if (threadIdx.x == 0) base_s += chunk_total;
        __syncthreads();
    }
}

cudaError_t launch_sample(const SampleParams &sp, cudaStream_t st) {
    int blocks = sp.nmodes * sp.nrep;
    if (blocks <= 0) return cudaSuccess;
    k_sample<<<blocks, 1024, 0, st>>>(sp);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Summary gather (Alg. 1 step 4): Xs[kk][ii][jj] = X(K'[kk], I_s[ii], J_s[jj]),
// K' = K_s (old, ascending) followed by the new slices in arrival order.
// Also the exact-product, double-float sum of squares of every summary row.
template <typename TX> struct Quant;
template <> struct Quant<double> {
    template <typename TS> static __device__ __forceinline__ double q(TS v) { return (double)v; }
};
template <> struct Quant<float> {
    template <typename TS> static __device__ __forceinline__ float q(TS v) { return (float)v; }
};
template <> struct Quant<__nv_bfloat16> {
    // float64 stores round to float32 first, then to bfloat16 (both nearest-even)
    template <typename TS> static __device__ __forceinline__ __nv_bfloat16 q(TS v) {
        return __float2bfloat16_rn((float)v);
    }
};

// sum of squares accumulators: float64 for float64 summaries, double-float otherwise
struct SqD {
    double a = 0.0;
    __device__ void add(double v) { a = __fma_rn(v, v, a); }
    __device__ double total() { return warp_sum(a); }
};
struct SqF {
    DF a{0.f, 0.f};
    __device__ void add(float v) { a = df_add_sq(a, v); }
    __device__ double total() { return df_value(warp_df_sum(a)); }
};
template <typename TX> struct SqOf { using T = SqF; };
template <> struct SqOf<double> { using T = SqD; };

template <typename TS, typename TX>
__global__ void __launch_bounds__(256) k_gather(GatherParams g) {
    const int rep = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Kp = g.nK + g.K_new;
    const long long row = (long long)blockIdx.x * 8 + warp;
    if (row >= (long long)Kp * g.nI) return;
    const int kk = (int)(row / g.nI), ii = (int)(row % g.nI);
    const int *Is = g.samples + (long long)(rep * 3 + 0) * g.samp_stride;
    const int *Js = g.samples + (long long)(rep * 3 + 1) * g.samp_stride;
    const int *Ks = g.samples + (long long)(rep * 3 + 2) * g.samp_stride;
    const int gk = kk < g.nK ? Ks[kk] : g.K_old + (kk - g.nK);
    const TS *src = (const TS *)g.store + ((long long)gk * g.I + Is[ii]) * g.lds;
    TX *dst = (TX *)g.Xs + rep * g.xrs + row * g.ldj;
    typename SqOf<TX>::T acc;
    for (int jj = lane; jj < g.ldj; jj += 32) {
        TX v = Quant<TX>::q(jj < g.nJ ? src[Js[jj]] : (TS)0);
        dst[jj] = v;
        acc.add(widen_elem(v));
    }
    double t = acc.total();
    if (lane == 0) g.rowsq[(long long)rep * Kp * g.nI + row] = t;
}

// bfloat16 summaries with their transposed copy in one pass: a CTA gathers
// 32 rows x 256 columns of one summary slice into shared memory, writes them
// row-major (Xs) and column-major (Xt, the operand of the mode-2 MTTKRP).
// Repetitions are the fastest grid index, so the CTAs of one slice in every
// summary run together (the new slices are in all of them).  Each lane sums
// its columns in the same order as k_gather, so the row sums of squares are
// the same numbers.
constexpr int GT_ROWS = 32, GT_COLS = 256;

template <typename TS, bool SPLIT>
__global__ void __launch_bounds__(256) k_gather_bf16_t(GatherParams g) {
    const int tiles_i = (g.nI + GT_ROWS - 1) / GT_ROWS;
    const int rep = (int)(blockIdx.x % g.nrep);
    const long long tix = blockIdx.x / g.nrep;
    const int kk = (int)(tix / tiles_i), ii0 = (int)(tix % tiles_i) * GT_ROWS;
    const int Kp = g.nK + g.K_new;
    if (kk >= Kp) return;
    const int rows = min(GT_ROWS, g.nI - ii0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int *Is = g.samples + (long long)(rep * 3 + 0) * g.samp_stride;
    const int *Js = g.samples + (long long)(rep * 3 + 1) * g.samp_stride;
    const int *Ks = g.samples + (long long)(rep * 3 + 2) * g.samp_stride;
    const int gk = kk < g.nK ? Ks[kk] : g.K_old + (kk - g.nK);
    __shared__ __nv_bfloat16 tile[GT_ROWS][GT_COLS + 2];
    __shared__ __nv_bfloat16 tlo[SPLIT ? GT_ROWS : 1][GT_COLS + 2];
    SqF acc[GT_ROWS / 8], acc2[SPLIT ? GT_ROWS / 8 : 1];
    const long long soff = rep * g.xrs + (long long)kk * g.nI * g.ldj;
    const long long toff = rep * g.xtrs + (long long)kk * g.nJ * g.ldi;
    __nv_bfloat16 *xs = (__nv_bfloat16 *)g.Xs + soff;
    __nv_bfloat16 *xt = (__nv_bfloat16 *)g.Xt + toff;
    for (int j0 = 0; j0 < g.ldj; j0 += GT_COLS) {
#pragma unroll
        for (int rr = 0; rr < GT_ROWS / 8; ++rr) {
            const int r = warp + 8 * rr;
            if (r < rows) {
                const TS *src = (const TS *)g.store + ((long long)gk * g.I + Is[ii0 + r]) * g.lds;
                __nv_bfloat16 *dst = xs + (long long)(ii0 + r) * g.ldj;
                for (int c = lane; c < GT_COLS && j0 + c < g.ldj; c += 32) {
                    const int jj = j0 + c;
                    const TS x = jj < g.nJ ? src[Js[jj]] : (TS)0;
                    const __nv_bfloat16 v = Quant<__nv_bfloat16>::q(x);
                    dst[jj] = v;
                    tile[r][c] = v;
                    acc[rr].add(widen_elem(v));
                    if constexpr (SPLIT) {
                        // lo = bf16(x - hi), x as float32 (the difference is exact)
                        const float hf = __bfloat162float(v);
                        const __nv_bfloat16 lo = __float2bfloat16_rn((float)x - hf);
                        ((__nv_bfloat16 *)g.Xlo + soff)[(long long)(ii0 + r) * g.ldj + jj] = lo;
                        tlo[r][c] = lo;
                        acc2[rr].add(hf + __bfloat162float(lo));
                    }
                }
            }
        }
        __syncthreads();
        // Xt[kk][jj][ii0 + r]: 16 threads per column jj, two rows each
        const int jn = min(GT_COLS, g.nJ - j0);
        for (int e = threadIdx.x; e < jn * 16; e += blockDim.x) {
            const int c = e >> 4, r = (e & 15) * 2;
            if (r < rows) {
                const long long oi = (long long)(j0 + c) * g.ldi + ii0 + r;
                __nv_bfloat16 *o = xt + oi;
                if (r + 1 < rows) {
                    *reinterpret_cast<__nv_bfloat162 *>(o) = __halves2bfloat162(tile[r][c], tile[r + 1][c]);
                } else {
                    o[0] = tile[r][c];
                }
                if constexpr (SPLIT) {
                    __nv_bfloat16 *ol = (__nv_bfloat16 *)g.Xtlo + toff + oi;
                    if (r + 1 < rows) {
                        *reinterpret_cast<__nv_bfloat162 *>(ol) = __halves2bfloat162(tlo[r][c], tlo[r + 1][c]);
                    } else {
                        ol[0] = tlo[r][c];
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int rr = 0; rr < GT_ROWS / 8; ++rr) {
        const int r = warp + 8 * rr;
        if (r < rows) {
            const long long ri = (long long)rep * Kp * g.nI + (long long)kk * g.nI + ii0 + r;
            const double t = acc[rr].total();
            if (lane == 0) g.rowsq[ri] = t;
            if constexpr (SPLIT) {
                const double t2 = acc2[rr].total();
                if (lane == 0) g.rowsq2[ri] = t2;
            }
        }
    }
}

// float8 e4m3 summaries with their transposed copy (the same tiling as
// k_gather_bf16_t): summary slice kk of stored slice k gets the scale
// amax_k / 448 and codes e4m3(x * (448 / amax_k)), all in float32 with round
// to nearest; the row sums of squares are sum(q^2) * scale^2.
template <typename TS>
__global__ void __launch_bounds__(256) k_gather_fp8_t(GatherParams g) {
    const int tiles_i = (g.nI + GT_ROWS - 1) / GT_ROWS;
    const int rep = (int)(blockIdx.x % g.nrep);
    const long long tix = blockIdx.x / g.nrep;
    const int kk = (int)(tix / tiles_i), ii0 = (int)(tix % tiles_i) * GT_ROWS;
    const int Kp = g.nK + g.K_new;
    if (kk >= Kp) return;
    const int rows = min(GT_ROWS, g.nI - ii0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int *Is = g.samples + (long long)(rep * 3 + 0) * g.samp_stride;
    const int *Js = g.samples + (long long)(rep * 3 + 1) * g.samp_stride;
    const int *Ks = g.samples + (long long)(rep * 3 + 2) * g.samp_stride;
    const int gk = kk < g.nK ? Ks[kk] : g.K_old + (kk - g.nK);
    const float amax = __uint_as_float(g.samax[gk]);
    const float inv = amax > 0.f ? __fdiv_rn(448.f, amax) : 0.f;
    const float scale = __fdiv_rn(amax, 448.f);
    if (ii0 == 0 && threadIdx.x == 0) g.sscale[(long long)rep * Kp + kk] = scale;
    __shared__ unsigned char tile[GT_ROWS][GT_COLS + 4];
    SqF acc[GT_ROWS / 8];
    unsigned char *xs = (unsigned char *)g.Xs + rep * g.xrs + (long long)kk * g.nI * g.ldj;
    unsigned char *xt = (unsigned char *)g.Xt + rep * g.xtrs + (long long)kk * g.nJ * g.ldi;
    for (int j0 = 0; j0 < g.ldj; j0 += GT_COLS) {
#pragma unroll
        for (int rr = 0; rr < GT_ROWS / 8; ++rr) {
            const int r = warp + 8 * rr;
            if (r < rows) {
                const TS *src = (const TS *)g.store + ((long long)gk * g.I + Is[ii0 + r]) * g.lds;
                unsigned char *dst = xs + (long long)(ii0 + r) * g.ldj;
                for (int c = lane; c < GT_COLS && j0 + c < g.ldj; c += 32) {
                    const int jj = j0 + c;
                    const float x = jj < g.nJ ? (float)src[Js[jj]] : 0.f;
                    const unsigned char q = to_e4m3(__fmul_rn(x, inv));
                    dst[jj] = q;
                    tile[r][c] = q;
                    acc[rr].add(from_e4m3(q));
                }
            }
        }
        __syncthreads();
        // Xt[kk][jj][ii0 + r]: 16 threads per column jj, two rows each
        const int jn = min(GT_COLS, g.nJ - j0);
        for (int e = threadIdx.x; e < jn * 16; e += blockDim.x) {
            const int c = e >> 4, r = (e & 15) * 2;
            if (r < rows) {
                unsigned char *o = xt + (long long)(j0 + c) * g.ldi + ii0 + r;
                if (r + 1 < rows) {
                    *reinterpret_cast<uchar2 *>(o) = make_uchar2(tile[r][c], tile[r + 1][c]);
                } else {
                    o[0] = tile[r][c];
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int rr = 0; rr < GT_ROWS / 8; ++rr) {
        const int r = warp + 8 * rr;
        if (r < rows) {
            const double t = acc[rr].total() * (double)scale * (double)scale;
            if (lane == 0) g.rowsq[(long long)rep * Kp * g.nI + (long long)kk * g.nI + ii0 + r] = t;
        }
    }
}

cudaError_t launch_gather(const GatherParams &g, int sdtype, int xelem, cudaStream_t st) {
    const long long rows = (long long)(g.nK + g.K_new) * g.nI;
    if (rows <= 0 || g.nrep <= 0) return cudaSuccess;
    if (xelem == 3) {
        if (!g.Xt || !g.samax || !g.sscale) return cudaErrorInvalidValue;
        const long long tiles = (long long)(g.nK + g.K_new) * ((g.nI + GT_ROWS - 1) / GT_ROWS) * g.nrep;
        count_launches(1);
        if (sdtype == 0) k_gather_fp8_t<double><<<(unsigned)tiles, 256, 0, st>>>(g);
        else k_gather_fp8_t<float><<<(unsigned)tiles, 256, 0, st>>>(g);
        return cudaGetLastError();
    }
    if (xelem == 2 && g.Xt) {
        const long long tiles = (long long)(g.nK + g.K_new) * ((g.nI + GT_ROWS - 1) / GT_ROWS) * g.nrep;
        count_launches(1);
        const bool split = g.Xlo && g.Xtlo && g.rowsq2;
        if (sdtype == 0) {
            if (split) k_gather_bf16_t<double, true><<<(unsigned)tiles, 256, 0, st>>>(g);
            else k_gather_bf16_t<double, false><<<(unsigned)tiles, 256, 0, st>>>(g);
        } else {
            if (split) k_gather_bf16_t<float, true><<<(unsigned)tiles, 256, 0, st>>>(g);
            else k_gather_bf16_t<float, false><<<(unsigned)tiles, 256, 0, st>>>(g);
        }
        return cudaGetLastError();
    }
    dim3 grid((unsigned)((rows + 7) / 8), g.nrep);
    count_launches(1);
    if (sdtype == 0) {
        if (xelem == 0) k_gather<double, double><<<grid, 256, 0, st>>>(g);
        else if (xelem == 1) k_gather<double, float><<<grid, 256, 0, st>>>(g);
        else k_gather<double, __nv_bfloat16><<<grid, 256, 0, st>>>(g);
    } else {
        if (xelem == 0) k_gather<float, double><<<grid, 256, 0, st>>>(g);
        else if (xelem == 1) k_gather<float, float><<<grid, 256, 0, st>>>(g);
        else k_gather<float, __nv_bfloat16><<<grid, 256, 0, st>>>(g);
    }
    return cudaGetLastError();
}

// Row sums of squares of a dense store (the identity summary of sbt_init).
template <typename TS>
__global__ void __launch_bounds__(256) k_rowsq(const TS *X, long long rows, int J, int lds,
                                               double *rowsq) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * 8 + warp;
    if (row >= rows) return;
    const TS *src = X + row * lds;
    typename SqOf<TS>::T acc;
    for (int j = lane; j < J; j += 32) acc.add(src[j]);
    double t = acc.total();
    if (lane == 0) rowsq[row] = t;
}

cudaError_t launch_rowsq(const void *X, int sdtype, long long rows, int J, int lds, double *rowsq,
                         cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)((rows + 7) / 8);
    count_launches(1);
    if (sdtype == 0) k_rowsq<double><<<blocks, 256, 0, st>>>((const double *)X, rows, J, lds, rowsq);
    else k_rowsq<float><<<blocks, 256, 0, st>>>((const float *)X, rows, J, lds, rowsq);
    return cudaGetLastError();
}

}  // namespace sbt
