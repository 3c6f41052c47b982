// Internal declarations shared by the translation units of libsambaten.
// Device helpers (Philox, fixed-point log2, reductions) and the host-side
// launchers of every kernel family.
#pragma once

#include "sambaten.h"

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <string>

namespace sbt {

// message returned by sbt_last_error() on this thread
void set_last_error(const std::string &msg);

// kernels launched by the library (process-wide), for the launch counter
long long launch_count();
void count_launches(int n);

// ---------------------------------------------------------------------------
// update flags, same values as SBT_FLAG_* of the public header
constexpr int SBT_FLAG_CHOL_REGULARIZED_DEV = 1;
constexpr int SBT_FLAG_ZERO_COLUMN_DEV = 2;
constexpr int SBT_FLAG_SAMPLE_LT_RANK_DEV = 4;

// error bits of the device status word
enum : unsigned {
    ERR_NONFINITE = 1u,  // new slices hold NaN/Inf
    ERR_RANGE = 2u,      // fixed-point marginal overflow
    ERR_SAMPLE = 4u,     // sample size above the number of positive weights
    ERR_TIMEOUT = 8u,    // a bounded device wait gave up
    ERR_INDEX = 16u,     // a coordinate outside the tensor (COO input)
};

// Device status block (mirrored to pinned host memory once per call).
struct DevStatus {
    unsigned err;
    unsigned pad;
    unsigned long long npos[3];  // positive-weight counts of x_a, x_b, x_c after commit
    unsigned long long amax_bits;  // max |x| of a tensor, as ordered double bits
};


// ---------------------------------------------------------------------------
// Fixed-point squares of the marginals (Eq. 1).  q(x) = floor((x*x) * 2^S): one correctly rounded
// float64 product (never contracted), exact power-of-two scaling, truncation.
__device__ __forceinline__ bool qsquare(double x, int S, unsigned long long *q) {
    double sq = ldexp(__dmul_rn(x, x), S);
    if (!(sq < 18446744073709551616.0)) return false;
    *q = __double2ull_rz(sq);
    return true;
}

// The same q for a float32 x without float64 arithmetic: x = m * 2^e with a
// 24-bit integer m, so x*x = m^2 * 2^(2e) exactly and q = floor(m^2 * 2^(2e+S))
// is an integer shift of the 48-bit m^2.  Returns false on overflow (q >= 2^64).
__device__ __forceinline__ bool qsquare(float x, int S, unsigned long long *q) {
    const uint32_t b = __float_as_uint(x) & 0x7FFFFFFFu;
    const int be = (int)(b >> 23);
    uint32_t m = b & 0x7FFFFFu;
    int e;
    if (be == 0) {
        e = -149;  // subnormal: no implicit bit
    } else {
        m |= 0x800000u;
        e = be - 150;
    }
    const unsigned long long m2 = (unsigned long long)m * (unsigned long long)m;  // < 2^48
    const int sh = 2 * e + S;
    if (m2 == 0) {
        *q = 0;
        return true;
    }
    if (sh >= 0) {
        if (sh >= 64 || (m2 >> (63 - sh)) >> 1) return false;  // m2 * 2^sh >= 2^64
        *q = m2 << sh;
    } else {
        *q = sh <= -64 ? 0ull : (m2 >> (-sh));
    }
    return true;
}

__device__ __forceinline__ void add_checked(unsigned long long *dst, unsigned long long v,
                                            DevStatus *status) {
    if (v == 0) return;
    unsigned long long old = atomicAdd(dst, v);
    if (old + v < old) atomicOr(&status->err, ERR_RANGE);
}




// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies with xor-folding, key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t lo0 = m0 * c.x, hi0 = __umulhi(m0, c.x);
        uint32_t lo1 = m1 * c.z, hi1 = __umulhi(m1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint2 philox_key(uint64_t seed, uint32_t stream_id) {
    return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32) ^ stream_id);
}

// Start value of the ALS factors: Philox word 0 >> 8, scaled by 2^-24, counter
// (global index, r | mode << 8 | rep << 12, batch, 2).
__device__ __forceinline__ double init_value(uint2 key, uint32_t gx, int r, int mode, int rep,
                                             uint32_t batch) {
    uint4 c = make_uint4(gx, (uint32_t)r | ((uint32_t)mode << 8) | ((uint32_t)rep << 12), batch, 2u);
    uint4 o = philox4x32_10(c, key);
    return (double)(o.x >> 8) * (1.0 / 16777216.0);
}

// Start value of GetRank's trial t (Section 3.2, Algorithm 2): counter
// (global index, r | mode << 8 | rep << 12 | t << 20, batch, 3).
__device__ __forceinline__ double init_value_trial(uint2 key, uint32_t gx, int r, int mode, int rep,
                                                   uint32_t batch, int trial) {
    uint4 c = make_uint4(gx, (uint32_t)r | ((uint32_t)mode << 8) | ((uint32_t)rep << 12) | ((uint32_t)trial << 20),
                         batch, 3u);
    uint4 o = philox4x32_10(c, key);
    return (double)(o.x >> 8) * (1.0 / 16777216.0);
}

// ---------------------------------------------------------------------------
// Reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// fused multiply-add in the operand type (never promoted)
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// widening loads of summary elements
__device__ __forceinline__ double widen_elem(double v) { return v; }
__device__ __forceinline__ float widen_elem(float v) { return v; }
__device__ __forceinline__ float widen_elem(__nv_bfloat16 v) { return __bfloat162float(v); }

// ---------------------------------------------------------------------------
// Double-float accumulation on the float32 pipes (float64 is a slow unit on
// this part): a value is the unevaluated sum hi + lo, sums use Knuth's
// two-sum, products of squares are split exactly with an FMA.
// float8 e4m3 code of x (nearest, ties to even, saturating at +-448) and its value
__device__ __forceinline__ unsigned char to_e4m3(float x) {
    return (unsigned char)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float from_e4m3(unsigned char c) {
    return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)c, __NV_E4M3)));
}

struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, DF b) {
    float s = __fadd_rn(a.hi, b.hi);
    float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    float h = __fadd_rn(s, e);
    float l = __fsub_rn(e, __fsub_rn(h, s));
    return DF{h, l};
}
__device__ __forceinline__ DF df_add_sq(DF a, float v) {
    float p = __fmul_rn(v, v);
    float pe = __fmaf_rn(v, v, -p);
    return df_add(a, DF{p, pe});
}
__device__ __forceinline__ DF df_add_prod(DF a, float u, float v) {
    float p = __fmul_rn(u, v);
    float pe = __fmaf_rn(u, v, -p);
    return df_add(a, DF{p, pe});
}
__device__ __forceinline__ DF warp_df_sum(DF a) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        DF b{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
        a = df_add(a, b);
    }
    return a;
}
__device__ __forceinline__ double df_value(DF a) { return (double)a.hi + (double)a.lo; }
// acc + a * b with a, b double-float: exact leading product by FMA, cross terms in float
__device__ __forceinline__ DF df_fma(DF acc, DF a, DF b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_add(acc, DF{p, e});
}
__device__ __forceinline__ DF df_from_double(double v) {
    float h = (float)v;
    return DF{h, (float)(v - (double)h)};
}
__device__ __forceinline__ DF df_quick(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_quick(p, e);
}
// a / b: quotient of the leading parts, corrected once by the remainder
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const DF r = df_sub(a, df_mul(DF{q1, 0.f}, b));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return df_quick(q1, q2);
}
// sqrt(a) for a >= 0: float square root, corrected once by the remainder
__device__ __forceinline__ DF df_sqrt(DF a) {
    if (!(a.hi > 0.f)) return DF{0.f, 0.f};
    const float s = __fsqrt_rn(a.hi);
    const float p = __fmul_rn(s, s);
    const DF r = df_sub(a, DF{p, __fmaf_rn(s, s, -p)});
    return df_quick(s, __fdiv_rn(r.hi, __fmul_rn(2.f, s)));
}
__device__ __forceinline__ DF warp_df_sum2(DF a) { return warp_df_sum(a); }

// ---------------------------------------------------------------------------
// Parameters of the sampling and gather kernels
struct SampleParams {
    const unsigned long long *w[3];  // weights per listed mode
    int N[3], n[3], mode_id[3];
    int nmodes, nrep, rep0;
    int *out;                 // [rep][nmodes][out_stride]
    long long out_stride;
    unsigned long long *khi, *klo;  // key scratch [rep][nmodes][key_stride]
    long long key_stride;
    uint64_t seed;
    uint32_t stream_id, batch;
    DevStatus *status;
};

struct GatherParams {
    const void *store;
    int I, lds;
    const int *samples;       // [rep][3][samp_stride]
    long long samp_stride;
    int nI, nJ, nK, K_old, K_new, nrep;
    void *Xs;                 // [rep][Kp][nI][ldj]
    int ldj;
    long long xrs;
    double *rowsq;            // [rep][Kp * nI]
    void *Xt;                 // bfloat16 only, may be null: transposed copy [rep][Kp][nJ][ldi]
    int ldi;
    long long xtrs;
    void *Xlo, *Xtlo;         // bfloat16 with Xt only, may be null: lo parts bf16(x - hi), same layouts
    double *rowsq2;           // with Xlo: row sums of (hi + lo)^2
    const unsigned *samax;    // float8: max |x| of every stored slice (float bits)
    float *sscale;            // float8: scale of every summary slice [rep][Kp] (written here)
};

// COO summaries: gather of the sampled nonzeros
struct CooGather {
    const int *si, *sj;       // store: row, column of every nonzero, grouped by slice
    const float *sv;
    const long long *sptr;    // slice k at [sptr[k], sptr[k+1])
    const int *samples;       // [rep][3][samp_stride]
    long long samp_stride;
    const int *posI, *posJ;   // [rep][I], [rep][J]: position in the sample or -1
    int I, J, nK, K_old, K_new, nrep, S;
    int *cnt;                 // [rep][Kp + 1] kept nonzeros per summary slice (pass 0)
    const long long *off;     // [rep][Kp + 1] their offsets (pass 1)
    double *rowsq;            // [rep][Kp] sum of squares per summary slice
    unsigned *vmax;           // [rep] max |v| (float bits)
    long long ecap;           // entries capacity per repetition
    int *eii, *ejj, *ekk;     // [rep][ecap] summary coordinates
    float *ev;
};

// COO summaries as the MTTKRP reads them
struct CooDesc {
    long long ecap;
    const int *eii, *ejj, *ekk;
    const float *ev;
    const long long *off;     // [rep][Kp + 1]: entries of summary slice kk (mode 3 rows)
    const long long *rp1;     // [rep][nI + 1]: row offsets into perm1 (mode 1 rows)
    const long long *rp2;     // [rep][nJ + 1]
    const int *perm1, *perm2; // [rep][ecap]: entries grouped by ii / by jj
    const int *fexp;          // [rep]: fixed-point exponent F of the sums
};

// rows of one tail CTA (float32 / bfloat16 summaries): the partial-sum
// reduction after each MTTKRP pass is spread over ceil(n / TAIL_ROWS) CTAs
// per repetition
constexpr int TAIL_ROWS = 16;

// ---------------------------------------------------------------------------
// Problem description handed to the ALS kernels.  All repetitions share the
// summary shape (n[0] = n_I, n[1] = n_J, n[2] = Kp).
struct AlsDesc {
    int nrep, R;
    int n[3];
    int ldj;          // row pitch of the summary (elements)
    int nK;           // shared old rows of the time mode
    int elem;         // 0 f64, 1 f32, 2 bf16
    long long xrs;    // elements per repetition of X
    const void *X;
    void *U[3];       // [rep][n_m][R], double (elem 0) or float
    double *M;        // [rep][nmax][R] reduced MTTKRP
    void *part;       // [rep][P][nmax][R] partial sums (float or double)
    long long prs;    // elements per repetition of part
    int pr;           // row stride of the partials: R (float64 path) or R rounded up to 4
    long long mrs;    // elements per repetition of M
    double *G;        // [rep][3][R][R]
    double *lam;      // [rep][R]
    double *fit, *fit_prev, *normX2;  // [rep]
    int *iters, *conv, *flags;        // [rep]
    double tol;
    int max_iters, fixed_iters;
    unsigned long long *bytes_ctr;  // algorithmic bytes read by MTTKRP passes (nullable)
    int P[3];              // partial sums per mode (set by the chosen MTTKRP kernels)
    DF *tpart;             // tail chunk shares [rep][tchunks][R(R+1)/2 + 1]
    float *xinv;           // V^-1 of the mode being solved, double-float planes [rep][2][32][32]
    DF *Gf;                // Grams in double-float [rep][3][R][R] (float32 factor path)
    DF *nx2f, *fitpf;      // ||X_s||^2 and the previous fit in double-float [rep]
    int *tail_cnt;         // [rep] chunk CTAs finished (the last one completes the mode; zero between uses)
    int tchunks;           // row chunks of TAIL_ROWS for the largest mode
    long long rq_rows;     // row sums of squares per repetition (0: n[2] * n[0], the dense summary rows)
    float *ymem;           // nullable: Y_kk = X_kk^T A of the mode-2 pass, [rep][n[2]][n[1]][pr]; the
                           // mode-3 MTTKRP is then M3(kk, r) = sum_j Y_kk(j, r) B(j, r) (k_mtt_memo)
    long long yrs;         // floats per repetition of ymem
    int rep0;              // repetition index of the first repetition (Philox counters of the start)
    int tail64;            // float32 factor path with the float64 tail (k_reduce + k_tail): Grams in G,
                           // no V^-1 beside the passes
    // tile choices
    int spc, nks, nib, jc; // row kernel: slices per CTA, slice splits, row blocks, column chunk
    long long rows_per;    // column kernel: rows per CTA
    int nrs, cols;         // column kernel: row splits, columns per lane
};

// Start of a summary ALS: F[0] null -> Philox uniforms; else the old factors
// A, B, C (float64, row-major, R columns) at the sampled rows, the new
// slices' rows of C' zero
struct WarmStart {
    const double *F[3] = {nullptr, nullptr, nullptr};
    int trial = -1;  // >= 0 (F null): GetRank's trial start, init_value_trial
};

// ---------------------------------------------------------------------------
// Launchers (all asynchronous on `st`)
cudaError_t launch_philox(const uint32_t *ctr, uint2 key, uint32_t *out, long long n, cudaStream_t st);

cudaError_t launch_absmax(const void *X, int dtype, long long n, DevStatus *status, cudaStream_t st);

// Copy K_new slices (row pitch ldin; may alias the store) into the store and
// add their fixed-point squares to the marginals: dxa (I), dxb (J), xc_new (K_new).
// samax: null, or the max |x| of every new slice (float bits, atomically maxed; zero it first)
cudaError_t launch_append(const void *Xin, int dtype, long long K_new, int I, int J, int ldin, void *store,
                          int lds, int S, unsigned long long *dxa, unsigned long long *dxb,
                          unsigned long long *xc_new, unsigned *samax, DevStatus *status, cudaStream_t st);

cudaError_t launch_sample(const SampleParams &sp, cudaStream_t st);

// Summaries: Xs[rep][kk][ii][jj], kk over K_s (n_K old) then K_old..K_old+K_new-1.
cudaError_t launch_gather(const GatherParams &g, int sdtype, int xelem, cudaStream_t st);
// Row sums of squares of a dense store (identity summary of sbt_init).
cudaError_t launch_rowsq(const void *X, int sdtype, long long rows, int J, int lds, double *rowsq,
                         cudaStream_t st);

// ALS: start values, Grams, ||X_s||^2; then the iterations.
cudaError_t launch_als_prepare(const AlsDesc &d, const int *samples, long long samp_stride, int K_old,
                               bool identity, uint64_t seed, uint32_t stream_id, uint32_t batch,
                               const double *rowsq, cudaStream_t st,
                               const WarmStart &ws = WarmStart{});
cudaError_t launch_als_iteration(const AlsDesc &d, cudaStream_t st);
cudaError_t launch_als_mode(const AlsDesc &d, int mode, cudaStream_t st);
// the two halves of launch_als_mode: the MTTKRP pass, then reduction + tail
cudaError_t launch_mttkrp(const AlsDesc &d, int mode, cudaStream_t st);
cudaError_t launch_reduce_tail(const AlsDesc &d, int mode, cudaStream_t st);
// dynamic shared-memory limits of the ALS and tensor-core kernels (call once
// per process and device, outside any stream capture)
cudaError_t set_als_kernel_attributes();
cudaError_t set_tc_kernel_attributes();
// V^-1 of `mode` for the float32 factor path (run beside the mode's MTTKRP)
cudaError_t launch_xinv(const AlsDesc &d, int mode, cudaStream_t st);
// CorConDia of a CP model (float64; X slice-major, element kind elem: 0 f64,
// 1 f32, 2 bf16); scratch: core_consistency_scratch_doubles(K, I, J, R)
// doubles; status bit 1 when a factor's Gram is not positive definite; *out
// device double
cudaError_t launch_core_consistency(int elem, const void *X, long long K, long long I, long long J, long long ld,
                                    const double *lam, const double *A, const double *B, const double *C, int R,
                                    double *scratch, int *status, double *out, cudaStream_t st);
size_t core_consistency_scratch_doubles(long long K, long long I, long long J, int R);
cudaError_t launch_widen(const float *in, double *out, long long n, cudaStream_t st);
// The whole ALS (CUDA-core MTTKRP, float64 tail) of every repetition of nd
// summary sets (1..PA_MAX_SETS descriptors, one per update, all of one
// element type and one rp_of(R)) as one persistent cooperative launch.
// dev_descs: room for nd descriptors in device memory (written here, in
// stream order); sync_words: PA_SYNC_WORDS device words (zeroed here); err: a device
// status word (ERR_TIMEOUT if a grid barrier gave up); max_iters: the largest
// of the sets' caps (each set stops at its own).
constexpr int PA_MAX_SETS = 8;
constexpr int PA_GROUPS = 16;                        // arrival counters of the grid barrier
constexpr int PA_SYNC_WORDS = 32 * (1 + PA_GROUPS);  // one 128-byte line each, and the top line
struct AlsSetArg {
    AlsDesc d[PA_MAX_SETS];
};
bool persistent_compatible(const AlsDesc &a, const AlsDesc &b);

// Updates whose summary ALS a server runs in one batched persistent launch
// (api.cu).  update_deferred: sbt_update, stopped before the ALS when the
// context's options allow (persistent_als, the CUDA-core path, no per-launch
// timing; *deferred tells), else the whole update.  deferred_als: the pending
// ALS's descriptor, the context's stream and SM count.  update_complete: the
// match and the commit after the ALS ran (synchronises the context's stream).
// update_abandon: drop the pending update (the model and K are unchanged).
sbt_status update_deferred(sbt_ctx *c, const sbt_tensor *X, bool *deferred);
sbt_status deferred_als(sbt_ctx *c, AlsDesc *d, cudaStream_t *st, int *num_sms);
sbt_status update_complete(sbt_ctx *c);
void update_abandon(sbt_ctx *c);
cudaError_t launch_als_persistent(const AlsDesc *descs, int nd, AlsDesc *dev_descs, int max_iters,
                                  unsigned *sync_words, unsigned *err, int num_sms, cudaStream_t st);

// mode 3 after a memoised mode-2 pass: M3 from d.ymem and the new B as the
// single partial of the mode-3 tail, and V^-1 of mode 3 (PDL launch)
cudaError_t launch_mtt_memo(const AlsDesc &d, cudaStream_t st);
cudaError_t launch_refine_start(const AlsDesc &d, const double *rowsq2, cudaStream_t st);
// COO path
cudaError_t launch_coo_count(const int *kk, long long nnz, int K, int *cnt, DevStatus *status, cudaStream_t st);
cudaError_t launch_exscan(const int *in, long long in_stride, long long *out, long long out_stride, int n, int nseg,
                          long long base, cudaStream_t st);
cudaError_t launch_coo_scatter(const int *ii, const int *jj, const int *kk, const float *val, long long nnz, int I,
                               int J, int K_new, int S, const long long *sptr_new, int *fill, int *si, int *sj,
                               float *sv, unsigned long long *dxa, unsigned long long *dxb,
                               unsigned long long *xc_new, DevStatus *status, cudaStream_t st);
cudaError_t launch_abs_max_f(const float *v, long long n, unsigned *out, cudaStream_t st);
cudaError_t launch_coo_pos(const int *samples, long long samp_stride, int nI, int nJ, int I, int J, int nrep,
                           int *posI, int *posJ, cudaStream_t st);
cudaError_t launch_coo_gather(const CooGather &g, int pass, cudaStream_t st);
cudaError_t launch_coo_fexp(const unsigned *vmax, const long long *total, int nrep, int *fexp, cudaStream_t st);
cudaError_t launch_coo_group(const int *key, long long ecap, const long long *total, long long max_total, int nrows,
                             int nrep, int *cnt, long long *rowptr, int *fill, int *perm, cudaStream_t st);
cudaError_t launch_coo_expand_k(const long long *sptr, int K, int *ekk, cudaStream_t st);
cudaError_t launch_mttkrp_coo(const AlsDesc &d, const CooDesc &s, int mode, cudaStream_t st);
cudaError_t launch_coo_inner(const int *si, const int *sj, const float *sv, const long long *sptr, int K,
                             const double *A, const double *B, const double *C, const double *lam, int R, int F,
                             unsigned long long *acc, cudaStream_t st);
cudaError_t launch_als_continue(cudaGraphConditionalHandle h, const int *conv, int nrep, int *passes,
                                int max_passes, cudaStream_t st);
void choose_tiles(AlsDesc &d, int num_sms);
long long partial_elems(const AlsDesc &d);  // per repetition

// tcgen05 MTTKRP of bfloat16 summaries (k_tc.cu)
bool tc_supported(int R, int NC, bool fp8);
// tile choice of one tensor-core MTTKRP launch shape: CTAs per SM (1 or 2),
// pipeline stages (0: as many as fit)
struct TileChoice {
    int per_sm, stages;
};
TileChoice tile_choice(bool fp8, int R, int NP, int NC, int Kp, int nrep, int epi);
bool tile_known(bool fp8, int R, int NP, int NC, int Kp, int nrep, int epi);
void tile_store(bool fp8, int R, int NP, int NC, int Kp, int nrep, int epi, TileChoice c);
int tile_table_read(int *out, int cap);
void tile_table_merge(const int *in, int n);
void tile_table_clear();
void tc_tiles(int nrep, int NP, int Kp, int num_sms, int per_sm, int *npb, int *nks, int *spc);
void tc_plan(bool fp8, int R, int nrep, int NP, int NC, int Kp, int epi, int num_sms, int *npb, int *nks, int *spc);
cudaError_t make_summary_tmap(CUtensorMap *m, const void *base, int NC, int NP, int ld, long long nslices,
                              bool fp8);
// tmap_lo: null, or the map of the lo part of a split summary (added into
// every product); sscale: null for bfloat16 summaries, else float8 e4m3
// summaries with one scale per summary slice [rep][Kp]
cudaError_t launch_mttkrp_tc(const CUtensorMap &tmap, const CUtensorMap *tmap_lo, int epi, int nrep, int R, int NP,
                             int NC, int Kp,
                             const float *F, long long frs, const float *W, long long wrs, float *part, long long prs,
                             int pr,
                             const int *conv, unsigned long long *bytes_ctr, unsigned *err, const float *sscale,
                             int num_sms, int *P_out, cudaStream_t st, float *Y = nullptr, long long yrs = 0,
                             const TileChoice *force = nullptr);
cudaError_t launch_transpose_bf16(const void *X, void *Y, int NI, int NJ, int ldx, int ldy, long long nslices,
                                  cudaStream_t st);
// reduction of d.P[mode] partials into d.M, then the tail
cudaError_t launch_reduce_only(const AlsDesc &d, int mode, cudaStream_t st);
cudaError_t launch_store_m(const AlsDesc &d, int mode, void *Mout, cudaStream_t st);

// MTTKRP of one mode of a single tensor (d.nrep == 1, d.conv zero) into Mout
// (factor type), through d.part and d.M.
cudaError_t launch_mttkrp_op(AlsDesc &d, int mode, void *Mout, cudaStream_t st);

// Match + project back (one CTA per repetition) and commit.
struct MergeDesc {
    int nrep, R, I, J, K_old, K_new, nI, nJ, nK;
    const int *samples;  // [rep][3][samp_stride]
    long long samp_stride;
    const void *U[3];    // summary factors (float or double by elem)
    int elem;
    const double *lam_s; // [rep][R]
    double *A, *B, *C, *lam;   // state (C has K_old + K_new rows after commit)
    double *nu;          // [rep][3][R]   shared-row norms of the summary factors
    double *cnew;        // [rep][K_new][R]
    double *prop;        // [rep][3][pmax][R] zero-fill proposals (NaN = none)
    int pmax;
    double *lam_est;     // [rep][R]
    int *perm;           // [rep][R]
    double *min_score;   // [rep]
    double *dots;        // [rep][3][32 * 32 + 64] per-mode sums of the matching (dot products, norms)
    int *flags;          // [rep]
    int lambda_mode;
    unsigned long long *xa, *xb, *xc, *dxa, *dxb, *xc_new;
    DevStatus *status;
    const int *rnew;     // nullable: components of each summary (GetRank's R_new <= R), [rep];
                         // summary factor rows then hold rnew[rep] values (stride rnew[rep]) in
                         // the repetition's n x R slot
};
cudaError_t launch_match(const MergeDesc &m, cudaStream_t st);
// overflow check of the marginal fold; sets ERR_RANGE before anything changes
cudaError_t launch_precommit(const MergeDesc &m, cudaStream_t st);
cudaError_t launch_commit(const MergeDesc &m, cudaStream_t st);

// Full fit: out[0] = sum (x - x_hat)^2, out[1] = sum x^2 over K slices of the
// store.  scratch: at least fit_scratch_doubles(K, I, J, R) doubles.
long long fit_scratch_doubles(int K, int I, int J, int R);
cudaError_t launch_full_fit(const void *store, int sdtype, int K, int I, int J, int lds,
                            const double *A, const double *B, const double *C, const double *lam,
                            int R, double *out, double *scratch, cudaStream_t st);

// Init: canonical order and signs of the ALS result, written to the state.
cudaError_t launch_canonicalize(const AlsDesc &d, double *A, double *B, double *C, double *lam,
                                cudaStream_t st);

}  // namespace sbt
