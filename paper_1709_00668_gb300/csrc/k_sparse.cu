// Sparse (COO) tensors: the store, the summaries and the MTTKRP.
//
// The method is the same as for dense tensors (Alg. 1); only the layout
// differs.  The store holds the nonzeros of every time slice k contiguously
// (row index, column index, value) at [sptr[k], sptr[k+1]).  A summary is the
// list of nonzeros of the sampled slices whose row and column were sampled,
// in summary coordinates (kk, ii, jj), grouped by kk.  Modes 1 and 2 need the
// entries grouped by ii and by jj: those groupings are built once per update
// by counting and placing entries with atomic slot claims, so the order of
// entries inside a group is arbitrary.  The MTTKRP therefore adds its
// products as 64-bit fixed-point integers (each float32 product rounded to
// 2^-F, F chosen from max |v| and the entry count so that no sum can
// overflow), which makes every result independent of that order, and of the
// order of the input nonzeros.
#include "sbt_internal.cuh"

#include <algorithm>

namespace sbt {

// ---------------------------------------------------------------------------
// store append
__global__ void k_coo_count(const int *kk, long long nnz, int K, int *cnt, DevStatus *status) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz; e += (long long)gridDim.x * blockDim.x) {
        const int k = kk[e];
        if (k < 0 || k >= K) {
            atomicOr(&status->err, ERR_INDEX);
            continue;
        }
        atomicAdd(&cnt[k], 1);
    }
}

// Exclusive prefix sums of n counts per segment (one CTA per segment):
// out[seg][t] = base + sum_{u < t} in[seg][u], out[seg][n] = base + total.
__global__ void __launch_bounds__(1024) k_exscan(const int *in, long long in_stride, long long *out,
                                                  long long out_stride, int n, long long base) {
    const int seg = blockIdx.x;
    const int *a = in + seg * in_stride;
    long long *o = out + seg * out_stride;
    __shared__ long long wsum[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = base;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t0 = 0; t0 <= n; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        long long v = t < n ? (long long)a[t] : 0;
        long long x = v;  // inclusive warp scan
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            long long w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += y;
            }
            wsum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const long long before = carry + (warp ? wsum[warp - 1] : 0) + x - v;
        if (t <= n) o[t] = before;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + v;
        __syncthreads();
    }
}

// Place a batch's nonzeros into the store at their slices (sptr already
// holds the slices' start offsets) and add their fixed-point squares to the
// marginal deltas.  Indices outside the shape and non-finite values raise
// the status word (the update is then not committed).
__global__ void k_coo_scatter(const int *ii, const int *jj, const int *kk, const float *val, long long nnz, int I,
                              int J, int K_new, int S, const long long *sptr_new, int *fill, int *si, int *sj,
                              float *sv, unsigned long long *dxa, unsigned long long *dxb,
                              unsigned long long *xc_new, DevStatus *status) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz; e += (long long)gridDim.x * blockDim.x) {
        const int i = ii[e], j = jj[e], k = kk[e];
        if (i < 0 || i >= I || j < 0 || j >= J || k < 0 || k >= K_new) {
            atomicOr(&status->err, ERR_INDEX);
            continue;
        }
        const float v = val[e];
        unsigned long long q = 0;
        if (!isfinite(v)) {
            atomicOr(&status->err, ERR_NONFINITE);
        } else if (!qsquare(v, S, &q)) {
            atomicOr(&status->err, ERR_RANGE);
        }
        const long long pos = sptr_new[k] + atomicAdd(&fill[k], 1);
        si[pos] = i;
        sj[pos] = j;
        sv[pos] = v;
        add_checked(&dxa[i], q, status);
        add_checked(&dxb[j], q, status);
        add_checked(&xc_new[k], q, status);
    }
}

// largest |v| of n values (float bits, atomically maxed into *out)
__global__ void k_abs_max_f(const float *v, long long n, unsigned *out) {
    float m = 0.f;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(v[e]));
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

// ---------------------------------------------------------------------------
// summaries
// pos[rep][x] = position of x in the sample of that mode (-1 elsewhere; the
// array is cleared to -1 first)
__global__ void k_coo_pos(const int *samples, long long samp_stride, int nI, int nJ, int I, int J, int *posI,
                          int *posJ) {
    const int rep = blockIdx.y;
    const int *Is = samples + (long long)(rep * 3 + 0) * samp_stride;
    const int *Js = samples + (long long)(rep * 3 + 1) * samp_stride;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nI + nJ; t += gridDim.x * blockDim.x) {
        if (t < nI) posI[(long long)rep * I + Is[t]] = t;
        else posJ[(long long)rep * J + Js[t - nI]] = t - nI;
    }
}

// One CTA per (summary slice kk, repetition): the nonzeros of stored slice
// K'[kk] whose row and column were sampled.  Pass 0 counts them, sums their
// fixed-point squares (the row sum of squares of the summary slice) and
// raises the repetition's max |v|; pass 1 writes them, in store order, at
// off[rep][kk].
__global__ void __launch_bounds__(256) k_coo_gather(CooGather g, int pass) {
    const int kk = blockIdx.x, rep = blockIdx.y;
    const int Kp = g.nK + g.K_new;
    const int *Ks = g.samples + (long long)(rep * 3 + 2) * g.samp_stride;
    const int gk = kk < g.nK ? Ks[kk] : g.K_old + (kk - g.nK);
    const long long b = g.sptr[gk], e = g.sptr[gk + 1];
    const int *pI = g.posI + (long long)rep * g.I, *pJ = g.posJ + (long long)rep * g.J;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ int wcnt[8];
    __shared__ unsigned long long wq[8];
    __shared__ long long base;
    if (pass == 0) {
        int cnt = 0;
        unsigned long long qs = 0;
        float m = 0.f;
        for (long long t = b + threadIdx.x; t < e; t += blockDim.x) {
            const int ii = pI[g.si[t]], jj = pJ[g.sj[t]];
            if (ii >= 0 && jj >= 0) {
                const float v = g.sv[t];
                unsigned long long q = 0;
                qsquare(v, g.S, &q);
                ++cnt;
                qs += q;
                m = fmaxf(m, fabsf(v));
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            qs += __shfl_xor_sync(0xffffffffu, qs, o);
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        }
        if (lane == 0) {
            wcnt[warp] = cnt;
            wq[warp] = qs;
            if (m > 0.f) atomicMax(&g.vmax[rep], __float_as_uint(m));
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int c = 0;
            unsigned long long s = 0;
            for (int w = 0; w < 8; ++w) {
                c += wcnt[w];
                s += wq[w];
            }
            g.cnt[(long long)rep * (Kp + 1) + kk] = c;
            g.rowsq[(long long)rep * Kp + kk] = ldexp((double)s, -g.S);
        }
        return;
    }
    // pass 1: order-preserving compaction, 256 entries per step
    if (threadIdx.x == 0) base = g.off[(long long)rep * (Kp + 1) + kk];
    __syncthreads();
    const long long eo = (long long)rep * g.ecap;
    for (long long t0 = b; t0 < e; t0 += blockDim.x) {
        const long long t = t0 + threadIdx.x;
        int ii = -1, jj = -1;
        if (t < e) {
            ii = pI[g.si[t]];
            jj = pJ[g.sj[t]];
        }
        const bool keep = ii >= 0 && jj >= 0;
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wcnt[warp] = __popc(mask);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < 8; ++w) {
            if (w < warp) before += wcnt[w];
            total += wcnt[w];
        }
        if (keep) {
            const long long pos = eo + base + before + __popc(mask & ((1u << lane) - 1u));
            g.eii[pos] = ii;
            g.ejj[pos] = jj;
            g.ekk[pos] = kk;
            g.ev[pos] = g.sv[t];
        }
        __syncthreads();
        if (threadIdx.x == 0) base += total;
        __syncthreads();
    }
}

// Fixed-point exponent F of every repetition: 2^F * (max |v| * entries)
// stays below 2^61, so no row sum of |v * f * w| <= |v| can overflow.
__global__ void k_coo_fexp(const unsigned *vmax, const long long *total, int nrep, int *fexp) {
    const int rep = threadIdx.x;
    if (rep >= nrep) return;
    const double bound = (double)__uint_as_float(vmax[rep]) * (double)max(1LL, total[rep]) + 1.0;
    int e2;
    frexp(bound, &e2);  // bound < 2^e2
    fexp[rep] = max(0, min(100, 61 - e2));
}

// Entries grouped by row of mode 1 (ii) or 2 (jj): count, then place with
// atomic slot claims (the order inside a row is arbitrary).
__global__ void k_coo_group_count(const int *key, long long ecap, const long long *total, int nrows, int *cnt) {
    const int rep = blockIdx.y;
    const long long n = total[rep];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[(long long)rep * (nrows + 1) + key[rep * ecap + t]], 1);
}

__global__ void k_coo_group_fill(const int *key, long long ecap, const long long *total, int nrows,
                                 const long long *rowptr, int *fill, int *perm) {
    const int rep = blockIdx.y;
    const long long n = total[rep];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int r = key[rep * ecap + t];
        const long long pos = rowptr[(long long)rep * (nrows + 1) + r] + atomicAdd(&fill[(long long)rep * nrows + r], 1);
        perm[rep * ecap + pos] = (int)t;
    }
}

// The summary slice of every entry for the identity summary (the whole
// tensor, at the initial decomposition): ekk[t] = k for t in [sptr[k], sptr[k+1]).
__global__ void k_coo_expand_k(const long long *sptr, int K, int *ekk) {
    const int k = blockIdx.x;
    if (k >= K) return;
    for (long long t = sptr[k] + threadIdx.x; t < sptr[k + 1]; t += blockDim.x) ekk[t] = k;
}

// ---------------------------------------------------------------------------
// MTTKRP: one warp per output row, products of float32 values rounded to
// 2^-F and added as 64-bit integers (order-free), one partial (P = 1).
template <int RP>
__global__ void __launch_bounds__(256) k_mtt_coo(AlsDesc d, CooDesc s, int mode) {
    const int rep = blockIdx.y;
    if (d.conv[rep]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = d.n[mode];
    const int row = blockIdx.x * 8 + warp;
    if (row >= n) return;
    const int R = d.R;
    const float *U0 = (const float *)d.U[0] + (long long)rep * d.n[0] * R;
    const float *U1 = (const float *)d.U[1] + (long long)rep * d.n[1] * R;
    const float *U2 = (const float *)d.U[2] + (long long)rep * d.n[2] * R;
    const long long eo = (long long)rep * s.ecap;
    long long b, e;
    const int *perm = nullptr;
    if (mode == 0) {
        b = s.rp1[(long long)rep * (d.n[0] + 1) + row];
        e = s.rp1[(long long)rep * (d.n[0] + 1) + row + 1];
        perm = s.perm1 + eo;
    } else if (mode == 1) {
        b = s.rp2[(long long)rep * (d.n[1] + 1) + row];
        e = s.rp2[(long long)rep * (d.n[1] + 1) + row + 1];
        perm = s.perm2 + eo;
    } else {
        b = s.off[(long long)rep * (d.n[2] + 1) + row];
        e = s.off[(long long)rep * (d.n[2] + 1) + row + 1];
    }
    const int F = s.fexp[rep];
    const float scale = ldexpf(1.f, min(F, 120));
    long long acc[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) acc[r] = 0;
    for (long long t = b + lane; t < e; t += 32) {
        const long long ent = eo + (perm ? perm[t] : t);
        const float v = s.ev[ent];
        const float *f, *w;
        if (mode == 0) {
            f = U1 + (long long)s.ejj[ent] * R;
            w = U2 + (long long)s.ekk[ent] * R;
        } else if (mode == 1) {
            f = U0 + (long long)s.eii[ent] * R;
            w = U2 + (long long)s.ekk[ent] * R;
        } else {
            f = U0 + (long long)s.eii[ent] * R;
            w = U1 + (long long)s.ejj[ent] * R;
        }
#pragma unroll
        for (int r = 0; r < RP; ++r)
            if (r < R) acc[r] += __float2ll_rn(__fmul_rn(__fmul_rn(__fmul_rn(v, f[r]), w[r]), scale));
    }
#pragma unroll
    for (int r = 0; r < RP; ++r) {
#pragma unroll
        for (int o = 16; o; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    }
    if (lane == 0) {
        float *out = (float *)d.part + rep * d.prs + (long long)row * d.pr;
        const double inv = ldexp(1.0, -F);
#pragma unroll
        for (int r = 0; r < RP; ++r)
            if (r < R) out[r] = (float)((double)acc[r] * inv);
    }
}

// ---------------------------------------------------------------------------
// <X, X_hat> over the stored nonzeros, X_hat = sum_r lambda_r A(i,r) B(j,r) C(k,r):
// float64 terms rounded to 2^-F and added as integers (order-free).
__global__ void __launch_bounds__(256) k_coo_inner(const int *si, const int *sj, const float *sv,
                                                    const long long *sptr, int K, const double *A, const double *B,
                                                    const double *C, const double *lam, int R, int F,
                                                    unsigned long long *acc_u) {
    const int k = blockIdx.x;
    if (k >= K) return;
    long long acc = 0;
    const double sc = ldexp(1.0, F);
    for (long long t = sptr[k] + threadIdx.x; t < sptr[k + 1]; t += blockDim.x) {
        const int i = si[t], j = sj[t];
        double m = 0.0;
        for (int r = 0; r < R; ++r) m += lam[r] * A[(long long)i * R + r] * B[(long long)j * R + r] * C[(long long)k * R + r];
        acc += __double2ll_rn((double)sv[t] * m * sc);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(acc_u, (unsigned long long)acc);
}

// ---------------------------------------------------------------------------
// launchers
static unsigned blocks_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (unsigned)std::max(1LL, std::min(b, 4096LL * 8));
}

cudaError_t launch_coo_count(const int *kk, long long nnz, int K, int *cnt, DevStatus *status, cudaStream_t st) {
    if (nnz <= 0) return cudaSuccess;
    k_coo_count<<<blocks_for(nnz, 256), 256, 0, st>>>(kk, nnz, K, cnt, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_exscan(const int *in, long long in_stride, long long *out, long long out_stride, int n, int nseg,
                          long long base, cudaStream_t st) {
    k_exscan<<<nseg, 1024, 0, st>>>(in, in_stride, out, out_stride, n, base);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_coo_scatter(const int *ii, const int *jj, const int *kk, const float *val, long long nnz, int I,
                               int J, int K_new, int S, const long long *sptr_new, int *fill, int *si, int *sj,
                               float *sv, unsigned long long *dxa, unsigned long long *dxb,
                               unsigned long long *xc_new, DevStatus *status, cudaStream_t st) {
    if (nnz <= 0) return cudaSuccess;
    k_coo_scatter<<<blocks_for(nnz, 256), 256, 0, st>>>(ii, jj, kk, val, nnz, I, J, K_new, S, sptr_new, fill, si, sj,
                                                         sv, dxa, dxb, xc_new, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_abs_max_f(const float *v, long long n, unsigned *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_abs_max_f<<<blocks_for(n, 256), 256, 0, st>>>(v, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_coo_pos(const int *samples, long long samp_stride, int nI, int nJ, int I, int J, int nrep,
                           int *posI, int *posJ, cudaStream_t st) {
    dim3 grid((unsigned)std::min<long long>((nI + nJ + 255) / 256, 4096), nrep);
    k_coo_pos<<<grid, 256, 0, st>>>(samples, samp_stride, nI, nJ, I, J, posI, posJ);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_coo_gather(const CooGather &g, int pass, cudaStream_t st) {
    dim3 grid(g.nK + g.K_new, g.nrep);
    k_coo_gather<<<grid, 256, 0, st>>>(g, pass);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_coo_fexp(const unsigned *vmax, const long long *total, int nrep, int *fexp, cudaStream_t st) {
    k_coo_fexp<<<1, 32, 0, st>>>(vmax, total, nrep, fexp);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_coo_group(const int *key, long long ecap, const long long *total, long long max_total, int nrows,
                             int nrep, int *cnt, long long *rowptr, int *fill, int *perm, cudaStream_t st) {
    dim3 grid(blocks_for(max_total, 256), nrep);
    k_coo_group_count<<<grid, 256, 0, st>>>(key, ecap, total, nrows, cnt);
    k_exscan<<<nrep, 1024, 0, st>>>(cnt, nrows + 1, rowptr, nrows + 1, nrows, 0);
    k_coo_group_fill<<<grid, 256, 0, st>>>(key, ecap, total, nrows, rowptr, fill, perm);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_coo_expand_k(const long long *sptr, int K, int *ekk, cudaStream_t st) {
    if (K <= 0) return cudaSuccess;
    k_coo_expand_k<<<K, 256, 0, st>>>(sptr, K, ekk);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mttkrp_coo(const AlsDesc &d, const CooDesc &s, int mode, cudaStream_t st) {
    dim3 grid((d.n[mode] + 7) / 8, d.nrep);
    const int R = d.R;
    if (R <= 8) k_mtt_coo<8><<<grid, 256, 0, st>>>(d, s, mode);
    else if (R <= 16) k_mtt_coo<16><<<grid, 256, 0, st>>>(d, s, mode);
    else k_mtt_coo<32><<<grid, 256, 0, st>>>(d, s, mode);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_coo_inner(const int *si, const int *sj, const float *sv, const long long *sptr, int K,
                             const double *A, const double *B, const double *C, const double *lam, int R, int F,
                             unsigned long long *acc, cudaStream_t st) {
    if (K <= 0) return cudaSuccess;
    k_coo_inner<<<K, 256, 0, st>>>(si, sj, sv, sptr, K, A, B, C, lam, R, F, acc);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sbt
