// C ABI of libsambaten: context management and the per-batch pipeline of
// Algorithm 1 (sample -> gather -> CP-ALS -> normalise/match -> project back ->
// commit) on the context's stream (the ALS forks side streams for V^-1 and
// for groups of repetitions, and joins them), one host synchronisation per
// update.
#include "sambaten.h"
#include "sbt_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace sbt;

namespace {

thread_local std::string g_err;

sbt_status fail(sbt_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

#define CK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            return fail(e_ == cudaErrorMemoryAllocation ? SBT_E_NOMEM : SBT_E_CUDA,   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));          \
        }                                                                             \
    } while (0)

#define TRY(expr)                      \
    do {                               \
        sbt_status s_ = (expr);        \
        if (s_ != SBT_OK) return s_;   \
    } while (0)

// device buffer that only grows
struct Buf {
    void *p = nullptr;
    size_t cap = 0;
    ~Buf() {
        if (p) cudaFree(p);
    }
    sbt_status ensure(size_t bytes) {
        if (bytes <= cap) return SBT_OK;
        if (p) {
            cudaFree(p);
            p = nullptr;
            cap = 0;
        }
        size_t want = std::max<size_t>(bytes, 256);
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            p = nullptr;
            return fail(SBT_E_NOMEM, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e));
        }
        cap = want;
        return SBT_OK;
    }
    template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

// host pinned buffer
struct HBuf {
    void *p = nullptr;
    size_t cap = 0;
    ~HBuf() {
        if (p) cudaFreeHost(p);
    }
    sbt_status ensure(size_t bytes) {
        if (bytes <= cap) return SBT_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        if (cudaMallocHost(&p, std::max<size_t>(bytes, 256)) != cudaSuccess)
            return fail(SBT_E_NOMEM, "cudaMallocHost failed");
        cap = std::max<size_t>(bytes, 256);
        return SBT_OK;
    }
    template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int round8(int64_t x) { return (int)((x + 7) / 8 * 8); }
inline int round16(int64_t x) { return (int)((x + 15) / 16 * 16); }
inline int esize_store(int dt) { return dt == SBT_F64 ? 8 : 4; }
inline int esize_elem(int elem) { return elem == 0 ? 8 : (elem == 1 ? 4 : (elem == 2 ? 2 : 1)); }
// summary row pitch: 16 bytes at least (TMA strides), 8 elements (vector loads)
inline int summary_ld(int n, int elem) { return elem == 3 ? round16(n) : round8(n); }

// value of a float8 e4m3 code (4 exponent bits, bias 7, 3 mantissa bits;
// exponent 0 is subnormal, 0x7F / 0xFF are NaN)
double e4m3_value(unsigned char c) {
    const int sgn = c >> 7, e = (c >> 3) & 15, m = c & 7;
    if (e == 15 && m == 7) return std::nan("");
    const double v = e == 0 ? std::ldexp((double)m, -9) : std::ldexp(1.0 + m / 8.0, e - 7);
    return sgn ? -v : v;
}
inline int esize_tf(int elem) { return elem == 0 ? 8 : 4; }

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// tensor-core plan for bfloat16 summaries: tensor maps over the summary and
// its transposed copy
struct TcPlan {
    bool on = false;
    bool split = false;  // refinement: add the lo parts (m1lo, m2lo) into every product
    CUtensorMap m1;      // [slice][ii][jj]: contraction over jj
    CUtensorMap m2;      // [slice][jj][ii]: contraction over ii
    CUtensorMap m1lo, m2lo;
    const float *sscale = nullptr;  // float8 summaries: scale of every summary slice
    const TileChoice *force = nullptr;  // autotuning: the candidate being timed
    int sms = 0;                    // SMs a launch sizes its grid for (0: all; a group of the ALS: its share)
    // the summaries the maps cover, so that a group of repetitions gets maps of its own
    const void *xs = nullptr, *xt = nullptr, *xlo = nullptr, *xtlo = nullptr;
    int nI = 0, nJ = 0, ldj = 0, ldi = 0, Kp = 0;
    bool fp8 = false;
};

// The ALS of the repetitions as independent groups, each its own chain of
// kernels on its own stream; each group's launches size their grids for its
// share of the SMs, so the groups' passes run side by side and the kernel
// boundaries of one chain overlap the other's work.
struct AlsGroupRt {
    cudaStream_t st = nullptr, side = nullptr;   // the group's chain; V^-1 beside its passes
    cudaEvent_t fork = nullptr, join = nullptr;  // around V^-1
    cudaEvent_t done = nullptr;                  // end of the group's chain in a loop body
};

// one group: its descriptor (per-repetition pointers offset to its first
// repetition) and its tensor-core plan
struct AlsPlan {
    AlsDesc d;
    TcPlan tc;
    bool has_tc = false;
};

}  // namespace

void sbt::set_last_error(const std::string &msg) { g_err = msg; }

// Raise the kernels' shared-memory limits once per device (outside any capture).
static cudaError_t ensure_kernel_attributes(int device) {
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (device < 0 || device >= 64 || done[device]) return cudaSuccess;
    cudaError_t e = set_als_kernel_attributes();
    if (e == cudaSuccess) e = set_tc_kernel_attributes();
    if (e == cudaSuccess) done[device] = true;
    return e;
}

// An update stopped before its summary ALS, which a server runs in a batched
// persistent launch with other contexts' (steps 1-4 and the ALS start done;
// the ALS, the match and the commit pending).
struct PendingAls {
    bool on = false;
    AlsDesc d{};
    int64_t K_old = 0;
    int K_new = 0, nI = 0, nJ = 0, nK = 0, ldj = 0;
    long long samp_stride = 0;
};

struct sbt_ctx {
    PendingAls pend;
    int device = 0;
    int num_sms = 0;
    cudaStream_t user = nullptr;    // the caller's stream (inputs are ordered on it)
    cudaStream_t stream = nullptr;  // the library's own stream (capturable)
    cudaEvent_t ev_user = nullptr;
    sbt_options opt{};
    int I = 0, J = 0, R = 0;
    int64_t K = 0, Kcap = 0;
    int sdtype = SBT_F32;
    int lds = 0;
    int S = 0;
    int elem = 1;  // summary element: 0 f64, 1 f32, 2 bf16, 3 float8 e4m3 (scaled per slice)
    uint32_t batch = 0;
    int64_t npos[3] = {0, 0, 0};
    // resident state
    Buf store, A, B, C, lam, xa, xb, xc, dxa, dxb, xc_new, status;
    HBuf h_status, h_poll, h_stats;
    // workspace
    Buf samples, khi, klo, Xs, rowsq, U[3], M, part, G, lam_s, fit, fit_prev, normX2, iters, conv, flags;
    Buf nu, cnew, prop, lam_est, perm, min_score, mdots, fitscr, staging, Xt, tpart, xinv, tail_cnt, Gf, dfs;
    Buf Xlo, Xtlo, rowsq2, iters_main;  // refinement: lo parts of the split summary
    Buf ymem;                           // mode-2 pass products for the mode-3 MTTKRP (mode3_pass 0)
    Buf grscr, gcc, rnew;               // GetRank: CorConDia scratch, scores + status words, R_new per repetition
    Buf psync, pdesc;                   // grid-barrier words and the descriptor of the persistent ALS
    std::vector<int> last_rank;         // components of each summary of the last update
    Buf samax, sscale;  // float8: max |x| of every stored slice (float bits); scale of every summary slice
    // COO contexts (sbt_init_coo): nonzeros grouped by slice, and the summary workspace
    bool coo = false;
    int64_t nnz = 0;
    Buf si, sj, sv, sptr;                   // store [nnz cap] x 3, slice offsets [K cap + 1]
    Buf cin_i, cin_j, cin_k, cin_v;         // host input staged on the device
    Buf ccnt, cfill, cmax;                  // per new slice counts / fill; max |v| of the input
    Buf posI, posJ, gcnt, goff, gtot, vmax, fexp;
    Buf eii, ejj, ekk, ev, perm1, perm2, rp1, rp2, gc1, gc2, gf1, gf2;
    HBuf h_tot;
    CooDesc cd{};
    cudaStream_t side = nullptr;  // runs V^-1 of a mode beside its MTTKRP pass
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    TcPlan tc;
    std::vector<AlsGroupRt> grt;   // groups 1.. of the ALS (group 0 runs on stream / side)
    cudaEvent_t ev_groups = nullptr;  // start of a loop body, for the groups' streams
    // profiling
    Buf prof_bytes;  // unsigned long long, device
    Buf passes;      // pass counter of the device-side ALS loop
    HBuf h_passes;
    bool passes_pending = false;
    long long launches_per_pass = 0;
    int pass_iters = 0;
    int timing = 0;  // 0 off; 1 events, each chunk of iterations as a graph; 2 events, direct launches
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> gev;  // MTTKRP timing slots of the ALS graph
    double mtt_ms = 0.0, mtt_busy_ms = 0.0, mtt_launch_ms = 0.0;
    long long launch_base = 0, updates = 0, mtt_launches = 0, mtt_passes = 0;
    int mtt_per_iter = 3;  // MTTKRP launches per ALS iteration of the last loop (2 with the memoised mode 3)
    ~sbt_ctx() {
        for (auto &e : gev) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
        for (auto &g : grt) {
            if (g.fork) cudaEventDestroy(g.fork);
            if (g.join) cudaEventDestroy(g.join);
            if (g.done) cudaEventDestroy(g.done);
            if (g.side) cudaStreamDestroy(g.side);
            if (g.st) cudaStreamDestroy(g.st);
        }
        if (ev_groups) cudaEventDestroy(ev_groups);
        if (ev_user) cudaEventDestroy(ev_user);
        if (stream) cudaStreamDestroy(stream);
    }
    // last update
    bool have_last = false;
    int last_nI = 0, last_nJ = 0, last_nK = 0, last_Knew = 0, last_ldj = 0;
    long long last_samp_stride = 0;
    sbt_update_stats stats{};
};

// ---------------------------------------------------------------------------
extern "C" const char *sbt_version(void) { return "sambaten-gb300 0.1 (sm_103a)"; }

extern "C" const char *sbt_last_error(void) { return g_err.c_str(); }

extern "C" sbt_status sbt_default_options(sbt_options *o) {
    if (!o) return fail(SBT_E_INVALID, "null options");
    std::memset(o, 0, sizeof(*o));
    o->s_I = o->s_J = o->s_K = 2;
    o->r = 4;
    o->tol = 1e-6;
    o->max_iters = 50;
    o->max_iters_init = 50;
    o->seed = 0;
    o->stream_id = 0;
    o->prec = SBT_PREC_F32;
    o->lambda_mode = 0;
    o->fixed_iters = 0;
    o->K_capacity = 0;
    o->max_batch = 0;
    o->cuda_stream = nullptr;
    o->check_every = 4;
    o->get_rank = 0;
    o->get_rank_trials = 2;
    o->get_rank_threshold = 90.0;
    return SBT_OK;
}

static sbt_status check_options(const sbt_options *o, int R) {
    if (!o) return fail(SBT_E_INVALID, "null options");
    if (o->s_I < 1 || o->s_J < 1 || o->s_K < 1) return fail(SBT_E_INVALID, "sampling factors must be >= 1");
    if (o->r < 1 || o->r > SBT_MAX_REPS) return fail(SBT_E_INVALID, "r out of range [1, SBT_MAX_REPS]");
    if (R < 1 || R > SBT_MAX_RANK) return fail(SBT_E_INVALID, "R out of range [1, SBT_MAX_RANK]");
    if (o->max_iters < 1 || o->max_iters_init < 1) return fail(SBT_E_INVALID, "iteration caps must be >= 1");
    if (!(o->tol >= 0.0)) return fail(SBT_E_INVALID, "tol must be >= 0");
    if (o->prec < SBT_PREC_F64 || o->prec > SBT_PREC_FP8) return fail(SBT_E_INVALID, "unknown precision");
    if (o->lambda_mode != 0 && o->lambda_mode != 1) return fail(SBT_E_INVALID, "lambda_mode must be 0 or 1");
    if (o->refine_sweeps < 0 || o->refine_sweeps > 1000) return fail(SBT_E_INVALID, "refine_sweeps out of [0, 1000]");
    if (o->mode3_pass != 0 && o->mode3_pass != 1) return fail(SBT_E_INVALID, "mode3_pass must be 0 or 1");
    if (o->als_groups < 0 || o->als_groups > SBT_MAX_REPS) return fail(SBT_E_INVALID, "als_groups out of [0, SBT_MAX_REPS]");
    if (o->warm_start != 0 && o->warm_start != 1) return fail(SBT_E_INVALID, "warm_start must be 0 or 1");
    if (o->get_rank != 0 && o->get_rank != 1) return fail(SBT_E_INVALID, "get_rank must be 0 or 1");
    if (o->fp64_tail != 0 && o->fp64_tail != 1) return fail(SBT_E_INVALID, "fp64_tail must be 0 or 1");
    if (o->persistent_als != 0 && o->persistent_als != 1) return fail(SBT_E_INVALID, "persistent_als must be 0 or 1");
    if (o->get_rank_trials < 0 || o->get_rank_trials > 16) return fail(SBT_E_INVALID, "get_rank_trials out of [0, 16]");
    if (!std::isfinite(o->get_rank_threshold)) return fail(SBT_E_INVALID, "get_rank_threshold must be finite");
    if (o->get_rank && (o->prec == SBT_PREC_FP8 || o->refine_sweeps > 0))
        return fail(SBT_E_INVALID, "get_rank takes float64, float32 or bfloat16 summaries without refinement");
    return SBT_OK;
}

static sbt_status check_tensor(const sbt_tensor *X) {
    if (!X) return fail(SBT_E_INVALID, "null tensor");
    if (X->I < 1 || X->J < 1 || X->K < 1) return fail(SBT_E_SHAPE, "tensor dimensions must be >= 1");
    if (!X->data) return fail(SBT_E_INVALID, "null tensor data");
    if (X->dtype != SBT_F64 && X->dtype != SBT_F32) return fail(SBT_E_INVALID, "unknown dtype");
    if (X->I > (1 << 30) || X->J > (1 << 30) || X->K > (1 << 30)) return fail(SBT_E_SHAPE, "dimension too large");
    return SBT_OK;
}

// Order the library's stream after the caller's stream (device inputs).
static sbt_status order_after_user(sbt_ctx *c) {
    CK(cudaEventRecord(c->ev_user, c->user));
    CK(cudaStreamWaitEvent(c->stream, c->ev_user, 0));
    return SBT_OK;
}

// Move K_new slices (host or device) into the store at slice K0 and add their
// marginals into (ma, mb, mc).
static sbt_status append_slices(sbt_ctx *c, const sbt_tensor *X, int64_t K0, unsigned long long *ma,
                                unsigned long long *mb, unsigned long long *mc) {
    const size_t es = esize_store(c->sdtype);
    char *dst = c->store.as<char>() + (size_t)K0 * c->I * c->lds * es;
    const void *src = X->data;
    int ldin = c->J;
    if (!X->on_device) {
        // page-locked host memory is mapped into the device's address space:
        // the append kernel then reads the batch over the host link and
        // writes the store in the same pass (no separate copy, no second
        // read of the copied slices); pageable memory is copied first
        cudaPointerAttributes pa;
        const void *mapped = nullptr;
        if (cudaPointerGetAttributes(&pa, X->data) == cudaSuccess) {
            if (pa.type == cudaMemoryTypeHost && pa.devicePointer) mapped = pa.devicePointer;
        } else {
            cudaGetLastError();  // an unregistered pointer is not an error here
        }
        if (mapped) {
            src = mapped;
        } else {
            if (c->lds == c->J)  // rows already at the store's pitch: one contiguous copy
                CK(cudaMemcpyAsync(dst, X->data, (size_t)X->K * c->I * c->J * es, cudaMemcpyHostToDevice,
                                   c->stream));
            else
                CK(cudaMemcpy2DAsync(dst, (size_t)c->lds * es, X->data, (size_t)c->J * es, (size_t)c->J * es,
                                     (size_t)X->K * c->I, cudaMemcpyHostToDevice, c->stream));
            src = dst;
            ldin = c->lds;
        }
    }
    CK(launch_append(src, c->sdtype, X->K, c->I, c->J, ldin, dst, c->lds, c->S, ma, mb, mc,
                     c->samax.p ? c->samax.as<unsigned>() + K0 : nullptr, c->status.as<DevStatus>(), c->stream));
    return SBT_OK;
}

static sbt_status read_status(sbt_ctx *c, DevStatus *out) {
    CK(cudaMemcpyAsync(c->h_status.p, c->status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *out = *c->h_status.as<DevStatus>();
    return SBT_OK;
}

static sbt_status status_error(unsigned err) {
    if (err & ERR_NONFINITE) return fail(SBT_E_NONFINITE, "non-finite value in the input slices");
    if (err & ERR_RANGE) return fail(SBT_E_RANGE, "fixed-point marginal would overflow 64 bits");
    if (err & ERR_SAMPLE) return fail(SBT_E_STATE, "sample size above the number of positive weights");
    if (err & ERR_TIMEOUT) return fail(SBT_E_TIMEOUT, "a bounded device wait gave up");
    if (err & ERR_INDEX) return fail(SBT_E_SHAPE, "a COO coordinate lies outside the tensor");
    return SBT_OK;
}

// Workspace sizing: every per-call buffer goes through one Sizer, which either
// allocates (Buf::ensure) or, in a dry run, records what would be needed so
// that a context's footprint after a call can be predicted exactly.
struct Sizer {
    bool dry = false;
    std::vector<std::pair<const Buf *, size_t>> want;
    sbt_status need(Buf &b, size_t bytes) {
        if (!dry) return b.ensure(bytes);
        want.emplace_back(&b, std::max<size_t>(bytes, 256));
        return SBT_OK;
    }
};

// ALS descriptor scalars and tiles for nrep summaries of shape n[3] (no memory)
// element kind the ALS kernels see: float8 summaries run the float-factor ALS
// of the tensor-core path, as bfloat16 ones do
static int als_elem(const sbt_ctx *c) { return c->elem == 3 ? 2 : c->elem; }

static void als_shape(const sbt_ctx *c, AlsDesc &d, int nrep, const int n[3], int ldj, int nK, int elem,
                      int max_iters, int rank = 0) {
    std::memset(&d, 0, sizeof(d));
    d.nrep = nrep;
    d.R = rank > 0 ? rank : c->R;
    d.n[0] = n[0];
    d.n[1] = n[1];
    d.n[2] = n[2];
    d.ldj = ldj;
    d.nK = nK;
    d.elem = elem;
    d.tol = c->opt.tol;
    d.max_iters = max_iters;
    d.fixed_iters = c->opt.fixed_iters;
    // the float64 tail: asked for, or part of the persistent ALS (which a
    // tensor-core plan, decided later, turns off again)
    d.tail64 = elem != 0 && (c->opt.fp64_tail || c->opt.persistent_als) ? 1 : 0;
    d.pr = elem == 0 ? d.R : (d.R + 3) / 4 * 4;
    choose_tiles(d, c->num_sms);
    const int nmax = std::max(n[0], std::max(n[1], n[2]));
    d.mrs = (long long)nmax * d.R;
    d.prs = partial_elems(d);
    d.tchunks = (nmax + TAIL_ROWS - 1) / TAIL_ROWS;
}

// ALS workspace of a descriptor from als_shape; part_bytes covers the partial
// sums of every MTTKRP kernel that will run on it
static sbt_status als_sizes(sbt_ctx *c, const AlsDesc &d, size_t part_bytes, Sizer &z) {
    const int R = c->R, nrep = d.nrep;
    const size_t tfs = esize_tf(d.elem);
    for (int m = 0; m < 3; ++m) TRY(z.need(c->U[m], (size_t)nrep * d.n[m] * R * tfs));
    TRY(z.need(c->M, (size_t)nrep * d.mrs * 8));
    TRY(z.need(c->part, part_bytes));
    TRY(z.need(c->G, (size_t)nrep * 3 * R * R * 8));
    TRY(z.need(c->lam_s, (size_t)nrep * R * 8));
    TRY(z.need(c->fit, (size_t)nrep * 8));
    TRY(z.need(c->fit_prev, (size_t)nrep * 8));
    TRY(z.need(c->normX2, (size_t)nrep * 8));
    TRY(z.need(c->iters, (size_t)nrep * 4));
    TRY(z.need(c->conv, (size_t)nrep * 4));
    TRY(z.need(c->flags, (size_t)nrep * 4));
    TRY(z.need(c->tpart, (size_t)nrep * d.tchunks * (R * (R + 1) / 2 + 1) * sizeof(DF)));
    if (d.elem != 0) {
        TRY(z.need(c->xinv, (size_t)nrep * 2048 * 4));
        TRY(z.need(c->Gf, (size_t)nrep * 3 * R * R * sizeof(DF)));
        TRY(z.need(c->dfs, (size_t)nrep * 2 * sizeof(DF)));
    }
    TRY(z.need(c->tail_cnt, (size_t)nrep * 4));
    if (!z.dry) TRY(c->h_poll.ensure((size_t)nrep * 4));
    return SBT_OK;
}

// Point the descriptor at the (already sized) workspace
static sbt_status als_bind(sbt_ctx *c, AlsDesc &d, const void *X, long long xrs) {
    const int nrep = d.nrep;
    d.X = X;
    d.xrs = xrs;
    d.tpart = c->tpart.as<DF>();
    if (d.elem != 0) {
        d.xinv = c->xinv.as<float>();
        d.Gf = c->Gf.as<DF>();
        d.nx2f = c->dfs.as<DF>();
        d.fitpf = d.nx2f + nrep;
        if (!c->side) {
            CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
        }
    }
    CK(cudaMemsetAsync(c->tail_cnt.p, 0, (size_t)nrep * 4, c->stream));
    d.tail_cnt = c->tail_cnt.as<int>();
    for (int m = 0; m < 3; ++m) d.U[m] = c->U[m].p;
    d.M = c->M.as<double>();
    d.part = c->part.p;
    d.G = c->G.as<double>();
    d.lam = c->lam_s.as<double>();
    d.fit = c->fit.as<double>();
    d.fit_prev = c->fit_prev.as<double>();
    d.normX2 = c->normX2.as<double>();
    d.iters = c->iters.as<int>();
    d.conv = c->conv.as<int>();
    d.flags = c->flags.as<int>();
    d.bytes_ctr = c->prof_bytes.as<unsigned long long>();
    return SBT_OK;
}

// ALS descriptor over the ctx workspace for nrep summaries of shape n[3]
static sbt_status setup_als(sbt_ctx *c, AlsDesc &d, int nrep, const int n[3], int ldj, int nK, int elem,
                            const void *X, long long xrs, int max_iters) {
    als_shape(c, d, nrep, n, ldj, nK, elem, max_iters);
    Sizer z;
    TRY(als_sizes(c, d, (size_t)nrep * d.prs * esize_tf(elem), z));
    return als_bind(c, d, X, xrs);
}

// Run ALS iterations until every repetition converged (polled every
// check_every iterations) or max_iters.
static cudaError_t mttkrp_mode(sbt_ctx *c, const AlsDesc &d, const TcPlan *tc, int mode, cudaStream_t st) {
    if (c->coo) return launch_mttkrp_coo(d, c->cd, mode, st);
    if (!tc || !tc->on) return launch_mttkrp(d, mode, st);
    const int R = d.R, NI = d.n[0], NJ = d.n[1], Kp = d.n[2];
    const int sms = tc->sms > 0 ? tc->sms : c->num_sms;
    const float *U0 = (const float *)d.U[0], *U1 = (const float *)d.U[1], *U2 = (const float *)d.U[2];
    unsigned *err = &c->status.as<DevStatus>()->err;
    int P = 0;
    if (mode == 0)
        return launch_mttkrp_tc(tc->m1, tc->split ? &tc->m1lo : nullptr, 0, d.nrep, R, NI, NJ, Kp, U1, (long long)NJ * R, U2, (long long)Kp * R,
                                (float *)d.part, d.prs, d.pr, d.conv, d.bytes_ctr, err, tc->sscale, sms, &P, st,
                                nullptr, 0, tc->force);
    if (mode == 1)  // keeps Y_kk = X_kk^T A for the memoised mode 3
        return launch_mttkrp_tc(tc->m2, tc->split ? &tc->m2lo : nullptr, 0, d.nrep, R, NJ, NI, Kp, U0, (long long)NI * R, U2, (long long)Kp * R,
                                (float *)d.part, d.prs, d.pr, d.conv, d.bytes_ctr, err, tc->sscale, sms, &P, st,
                                d.ymem, d.yrs, tc->force);
    if (d.ymem) return launch_mtt_memo(d, st);  // mode 3 from Y and the new B (one partial), and its V^-1
    return launch_mttkrp_tc(tc->m1, tc->split ? &tc->m1lo : nullptr, 1, d.nrep, R, NI, NJ, Kp, U1, (long long)NJ * R, U0, (long long)NI * R,
                            (float *)d.part, d.prs, d.pr, d.conv, d.bytes_ctr, err, tc->sscale, sms, &P, st,
                            nullptr, 0, tc->force);
}

// partial counts of the tensor-core kernels, fixed by the shapes and the tile choices
static void tc_partials(AlsDesc &d, int num_sms, bool fp8) {
    int npb, nks, spc;
    tc_plan(fp8, d.R, d.nrep, d.n[0], d.n[1], d.n[2], 0, num_sms, &npb, &nks, &spc);
    d.P[0] = nks;
    const long long e0 = (long long)nks * d.n[0];
    tc_plan(fp8, d.R, d.nrep, d.n[0], d.n[1], d.n[2], 1, num_sms, &npb, &nks, &spc);
    d.P[2] = npb;
    const long long e2 = (long long)npb * d.n[2];
    tc_plan(fp8, d.R, d.nrep, d.n[1], d.n[0], d.n[2], 0, num_sms, &npb, &nks, &spc);
    d.P[1] = nks;
    const long long e1 = (long long)nks * d.n[1];
    d.prs = std::max(e0, std::max(e1, e2)) * d.pr;
}

// Autotuning of the tensor-core MTTKRP tiles: for every launch shape of this
// update that has no recorded choice, time each candidate (CTAs per SM,
// pipeline stages) on the live summaries with CUDA events and keep the
// fastest.  Runs before the ALS; the passes it times count no bytes and
// their partial sums are overwritten by the ALS.
static sbt_status autotune_tiles(sbt_ctx *c, const AlsDesc &d, TcPlan &tc) {
    const bool fp8 = c->elem == 3;
    const int R = d.R, nrep = d.nrep, Kp = d.n[2];
    static const TileChoice cands[] = {{2, 3}, {2, 4}, {2, 6}, {2, 0}, {1, 6}, {1, 0}};
    AlsDesc dq = d;
    dq.bytes_ctr = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    sbt_status st = SBT_OK;
    for (int mode = 0; mode < 3 && st == SBT_OK; ++mode) {
        const int NP = mode == 1 ? d.n[1] : d.n[0], NC = mode == 1 ? d.n[0] : d.n[1], epi = mode == 2 ? 1 : 0;
        if (tile_known(fp8, R, NP, NC, Kp, nrep, epi) || (mode == 2 && d.ymem)) continue;
        TileChoice best{2, 0};
        float best_ms = 1e30f;
        for (const TileChoice &cand : cands) {
            tc.force = &cand;
            cudaError_t e = mttkrp_mode(c, dq, &tc, mode, c->stream);  // warm
            if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
            for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = mttkrp_mode(c, dq, &tc, mode, c->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                st = fail(SBT_E_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
                break;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
        tc.force = nullptr;
        if (st == SBT_OK) tile_store(fp8, R, NP, NC, Kp, nrep, epi, best);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// Groups the ALS of nrep repetitions runs in: the tensor-core path splits
// them (default 2 groups, option als_groups) so that the groups' passes and
// tails overlap; every other path runs one group.
static int als_group_count(const sbt_ctx *c, int nrep, bool tc) {
    if (!tc || nrep < 2) return 1;
    const int g = c->opt.als_groups > 0 ? c->opt.als_groups : 2;
    return std::min(g, nrep);
}

// SMs a group's MTTKRP launch sizes its grid for: its share, so that the
// groups' concurrent passes fit the GPU together in one wave (a group's
// pass alone, one CTA per SM, streams at about half the HBM bandwidth)
static int group_sms(const sbt_ctx *c, int G) { return c->num_sms / G; }

// Partial counts of a tensor-core ALS of nrep repetitions in G groups, and
// the per-repetition stride of the partials that covers every group (the
// smallest group splits its slices most).
static void tc_group_partials(const sbt_ctx *c, AlsDesc &d, int G) {
    AlsDesc dm = d;
    dm.nrep = d.nrep / G;
    tc_partials(dm, group_sms(c, G), c->elem == 3);
    d.prs = dm.prs;
    for (int m = 0; m < 3; ++m) d.P[m] = dm.P[m];
}

// descriptor of repetitions [rep0, rep0 + ng): every per-repetition pointer
// offset to rep0 (the kernels index repetitions from blockIdx)
static AlsDesc group_desc(const AlsDesc &d, int rep0, int ng, size_t xbytes_per_rep) {
    AlsDesc s = d;
    const int R = d.R;
    const size_t tfs = esize_tf(d.elem);
    const long long r0 = rep0;
    s.nrep = ng;
    s.rep0 = d.rep0 + rep0;
    if (d.X) s.X = (const char *)d.X + r0 * xbytes_per_rep;
    for (int m = 0; m < 3; ++m) s.U[m] = (char *)d.U[m] + r0 * d.n[m] * R * tfs;
    if (d.M) s.M = d.M + r0 * d.mrs;
    s.part = (char *)d.part + r0 * d.prs * tfs;
    s.G = d.G + r0 * 3 * R * R;
    s.lam = d.lam + r0 * R;
    s.fit = d.fit + r0;
    s.fit_prev = d.fit_prev + r0;
    s.normX2 = d.normX2 + r0;
    s.iters = d.iters + r0;
    s.conv = d.conv + r0;
    s.flags = d.flags + r0;
    s.tpart = d.tpart + r0 * d.tchunks * (R * (R + 1) / 2 + 1);
    if (d.xinv) s.xinv = d.xinv + r0 * 2048;
    if (d.Gf) s.Gf = d.Gf + r0 * 3 * R * R;
    if (d.nx2f) s.nx2f = d.nx2f + r0;
    if (d.fitpf) s.fitpf = d.fitpf + r0;
    s.tail_cnt = d.tail_cnt + r0;
    if (d.ymem) s.ymem = d.ymem + r0 * d.yrs;
    return s;
}

// the groups of one ALS run (one group unless the tensor-core path splits)
static sbt_status als_plans(sbt_ctx *c, const AlsDesc &d, const TcPlan *tc, std::vector<AlsPlan> &out) {
    out.clear();
    const bool on = tc && tc->on;
    const int G = als_group_count(c, d.nrep, on);
    if (G == 1) {
        AlsPlan p;
        p.d = d;
        if (tc) {
            p.tc = *tc;
            p.has_tc = true;
            p.tc.sms = c->num_sms;
        }
        out.push_back(p);
        return SBT_OK;
    }
    const size_t es = tc->fp8 ? 1 : 2;
    const size_t xb = (size_t)tc->Kp * tc->nI * tc->ldj * es, xtb = (size_t)tc->Kp * tc->nJ * tc->ldi * es;
    const size_t xlb = (size_t)tc->Kp * tc->nI * tc->ldj * 2, xtlb = (size_t)tc->Kp * tc->nJ * tc->ldi * 2;
    for (int g = 0; g < G; ++g) {
        const int rep0 = g * d.nrep / G, ng = (g + 1) * d.nrep / G - rep0;
        AlsPlan p;
        p.d = group_desc(d, rep0, ng, xb);
        p.tc = *tc;
        p.has_tc = true;
        p.tc.sms = group_sms(c, G);
        const long long ns = (long long)ng * tc->Kp;
        CK(make_summary_tmap(&p.tc.m1, (const char *)tc->xs + rep0 * xb, tc->nJ, tc->nI, tc->ldj, ns, tc->fp8));
        CK(make_summary_tmap(&p.tc.m2, (const char *)tc->xt + rep0 * xtb, tc->nI, tc->nJ, tc->ldi, ns, tc->fp8));
        if (tc->split) {
            CK(make_summary_tmap(&p.tc.m1lo, (const char *)tc->xlo + rep0 * xlb, tc->nJ, tc->nI, tc->ldj, ns, false));
            CK(make_summary_tmap(&p.tc.m2lo, (const char *)tc->xtlo + rep0 * xtlb, tc->nI, tc->nJ, tc->ldi, ns, false));
        }
        if (tc->sscale) p.tc.sscale = tc->sscale + (long long)rep0 * tc->Kp;
        tc_partials(p.d, p.tc.sms, tc->fp8);
        p.d.prs = d.prs;  // the stride of the shared buffer (covers this group's partials)
        out.push_back(p);
    }
    return SBT_OK;
}

// streams and events of groups 1 .. G-1 (created outside any capture)
static sbt_status ensure_group_rt(sbt_ctx *c, int G) {
    if (G > 1 && !c->ev_groups) CK(cudaEventCreateWithFlags(&c->ev_groups, cudaEventDisableTiming));
    while ((int)c->grt.size() < G - 1) {
        AlsGroupRt g;
        CK(cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&g.side, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming));
        c->grt.push_back(g);
    }
    return SBT_OK;
}

// The kernels of G ALS iterations: group 0 on the library's stream, group g
// on its own stream, forked from and joined back to the library's stream.
// Per mode and group: V^-1 on the group's side stream beside its MTTKRP
// pass, then the tail.  With timed != 0, CUDA events bracket every MTTKRP
// launch on the stream it runs on (slots from 0); timed == 2 records them as
// event nodes of the graph being captured.
static cudaError_t launch_iterations(sbt_ctx *c, const std::vector<AlsPlan> &plans, int G, int timed) {
    cudaError_t e = cudaSuccess;
    auto record = [timed](cudaEvent_t ev, cudaStream_t s) {
        return timed == 2 ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal) : cudaEventRecord(ev, s);
    };
    const int ng = (int)plans.size();
    if (ng > 1) {
        e = cudaEventRecord(c->ev_groups, c->stream);
        for (int g = 1; g < ng && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(c->grt[g - 1].st, c->ev_groups, 0);
    }
    int slot = 0;
    for (int it = 0; it < G && e == cudaSuccess; ++it) {
        for (int mode = 0; mode < 3 && e == cudaSuccess; ++mode) {
            for (int g = 0; g < ng && e == cudaSuccess; ++g, ++slot) {
                const AlsDesc &d = plans[g].d;
                const TcPlan *tc = plans[g].has_tc ? &plans[g].tc : nullptr;
                cudaStream_t st = g == 0 ? c->stream : c->grt[g - 1].st;
                cudaStream_t side = g == 0 ? c->side : c->grt[g - 1].side;
                cudaEvent_t fork = g == 0 ? c->ev_fork : c->grt[g - 1].fork;
                cudaEvent_t join = g == 0 ? c->ev_join : c->grt[g - 1].join;
                // V^-1 beside the pass; a memoised mode 3 has no pass over the
                // summary, and k_mtt_memo forms its inverse
                const bool xinv = d.xinv && !(mode == 2 && d.ymem) && !d.tail64;
                if (xinv) {
                    e = cudaEventRecord(fork, st);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork, 0);
                    if (e == cudaSuccess) e = launch_xinv(d, mode, side);
                    if (e == cudaSuccess) e = cudaEventRecord(join, side);
                }
                const bool pass = !(mode == 2 && d.ymem);  // a memoised mode 3 launches no pass
                if (e == cudaSuccess && timed && pass) e = record(c->gev[slot].first, st);
                if (e == cudaSuccess) e = mttkrp_mode(c, d, tc, mode, st);
                if (e == cudaSuccess && timed && pass) e = record(c->gev[slot].second, st);
                if (e == cudaSuccess && xinv) e = cudaStreamWaitEvent(st, join, 0);
                if (e == cudaSuccess) e = launch_reduce_tail(d, mode, st);
            }
        }
    }
    for (int g = 1; g < ng && e == cudaSuccess; ++g) {
        e = cudaEventRecord(c->grt[g - 1].done, c->grt[g - 1].st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->grt[g - 1].done, 0);
    }
    return e;
}

// The whole ALS as one CUDA graph: a WHILE node whose body runs G iterations
// and then k_als_continue, which keeps the loop going while a repetition has
// not converged, for at most ceil(max_iters / G) passes.  The convergence
// test runs on the device: no host round trip inside the ALS.
static sbt_status build_als_loop(sbt_ctx *c, const AlsDesc &d, const std::vector<AlsPlan> &plans, int G,
                                 int max_passes, cudaGraphExec_t *exec, long long *launches_per_pass) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    cudaGraphConditionalHandle h = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    const long long base = launch_count();
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = launch_iterations(c, plans, G, 0);
            if (el == cudaSuccess)
                el = launch_als_continue(h, d.conv, d.nrep, c->passes.as<int>(), max_passes, c->stream);
            cudaGraph_t got = nullptr;
            e = cudaStreamEndCapture(c->stream, &got);
            if (el != cudaSuccess) e = el;
        }
    }
    *launches_per_pass = launch_count() - base;
    count_launches(-(int)*launches_per_pass);
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(SBT_E_CUDA, std::string("ALS loop graph: ") + cudaGetErrorString(e));
    return SBT_OK;
}

// Launches and MTTKRP passes of the last device-side ALS loop, known once
// its pass counter has been read back (after the caller's synchronisation).
static void settle_als_counts(sbt_ctx *c) {
    if (!c->passes_pending) return;
    const int passes = *c->h_passes.as<int>();
    count_launches((int)(passes * c->launches_per_pass));
    c->mtt_launches += (long long)c->mtt_per_iter * c->pass_iters * passes;
    c->passes_pending = false;
}

// Run ALS iterations until every repetition has converged or max_iters.
// Throughput path: one graph launch of the device-side loop; the pass count
// is read back with the caller's next synchronisation.  Timing path (CUDA
// events around every MTTKRP launch): the same kernels in chunks of
// check_every iterations, convergence polled from the host after each chunk;
// a chunk is one launch of a graph captured once (timing 1: the kernels and
// events run back to back, so no interval holds host submission time) or its
// kernels issued one by one (timing 2).  Kernels of converged repetitions
// exit at once, so iterations past convergence cost only their launches.
static sbt_status run_als(sbt_ctx *c, const AlsDesc &d, int max_iters, const TcPlan *tc = nullptr) {
    const int every = c->opt.check_every > 0 ? c->opt.check_every : 4;
    const int G = std::max(1, std::min(every, max_iters));
    const int nl = (max_iters + G - 1) / G;
    std::vector<AlsPlan> plans;
    TRY(als_plans(c, d, tc, plans));
    for (AlsPlan &pl : plans)
        if (pl.d.ymem) pl.d.P[2] = 1;  // the memoised mode 3 writes one partial
    const int ngr = (int)plans.size();
    TRY(ensure_group_rt(c, ngr));
    c->mtt_per_iter = (d.ymem ? 2 : 3) * ngr;
    if (c->passes_pending) {  // an earlier loop's count not read yet (its call failed before syncing)
        CK(cudaStreamSynchronize(c->stream));
        settle_als_counts(c);
    }
    if (c->opt.persistent_als && !(tc && tc->on) && !c->coo && !c->timing) {
        // one cooperative launch for every iteration and repetition
        TRY(c->psync.ensure(PA_SYNC_WORDS * sizeof(unsigned)));
        TRY(c->pdesc.ensure(sizeof(AlsDesc)));
        CK(launch_als_persistent(&d, 1, c->pdesc.as<AlsDesc>(), max_iters, c->psync.as<unsigned>(),
                                 &c->status.as<DevStatus>()->err, c->num_sms, c->stream));
        return SBT_OK;
    }
    if (!c->timing) {
        TRY(c->passes.ensure(sizeof(int)));
        TRY(c->h_passes.ensure(sizeof(int)));
        cudaGraphExec_t exec = nullptr;
        long long lpp = 0;
        TRY(build_als_loop(c, d, plans, G, nl, &exec, &lpp));
        cudaError_t e = cudaMemsetAsync(c->passes.p, 0, sizeof(int), c->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->h_passes.p, c->passes.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) return fail(SBT_E_CUDA, std::string("ALS loop launch: ") + cudaGetErrorString(e));
        c->passes_pending = true;
        c->launches_per_pass = lpp;
        c->pass_iters = G;
        return SBT_OK;
    }
    const int nslots = 3 * G * ngr;
    while ((int)c->gev.size() < nslots) {
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        c->gev.emplace_back(a, b);
    }
    struct ExecGuard {
        cudaGraphExec_t x = nullptr;
        ~ExecGuard() {
            if (x) cudaGraphExecDestroy(x);
        }
    } chunk;
    long long chunk_launches = 0;
    if (c->timing == 1) {
        cudaGraph_t graph = nullptr;
        const long long base = launch_count();
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = launch_iterations(c, plans, G, 2);
            e = cudaStreamEndCapture(c->stream, &graph);
            if (el != cudaSuccess) e = el;
        }
        chunk_launches = launch_count() - base;
        count_launches(-(int)chunk_launches);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&chunk.x, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(SBT_E_CUDA, std::string("ALS (timed) graph: ") + cudaGetErrorString(e));
    }
    for (int k = 0; k < nl; ++k) {
        cudaError_t e = cudaSuccess;
        if (chunk.x) {
            e = cudaGraphLaunch(chunk.x, c->stream);
            count_launches((int)chunk_launches);
        } else {
            e = launch_iterations(c, plans, G, 1);
        }
        c->mtt_launches += (long long)c->mtt_per_iter * G;
        const bool poll = (k == nl - 1) || !c->opt.fixed_iters;
        if (e == cudaSuccess && poll)
            e = cudaMemcpyAsync(c->h_poll.p, d.conv, sizeof(int) * d.nrep, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return fail(SBT_E_CUDA, std::string("ALS (timed): ") + cudaGetErrorString(e));
        // a pass (one launch per group, concurrent on the groups' streams)
        // lasts from the earliest start to the latest end, taken relative
        // to the first start event of the body; the busy time is the union
        // of all the body's launch intervals
        std::vector<std::pair<float, float>> iv;
        for (int q = 0; q < nslots; ++q) {
            if ((q / ngr) % 3 == 2 && d.ymem) continue;
            float a = 0.f, b = 0.f;
            if (cudaEventElapsedTime(&a, c->gev[0].first, c->gev[q].first) == cudaSuccess &&
                cudaEventElapsedTime(&b, c->gev[0].first, c->gev[q].second) == cudaSuccess)
                iv.emplace_back(a, b);
        }
        std::sort(iv.begin(), iv.end());
        for (size_t q = 0; q < iv.size();) {
            float lo = iv[q].first, hi = iv[q].second;
            c->mtt_launch_ms += iv[q].second - iv[q].first;
            size_t u = q + 1;
            for (; u < iv.size() && iv[u].first <= hi; ++u) {
                hi = std::max(hi, iv[u].second);
                c->mtt_launch_ms += iv[u].second - iv[u].first;
            }
            c->mtt_busy_ms += hi - lo;
            q = u;
        }
        for (int q0 = 0; q0 < nslots; q0 += ngr) {
            if ((q0 / ngr) % 3 == 2 && d.ymem) continue;
            float t0 = 0.f, t1 = 0.f;
            bool okp = true;
            for (int g = 0; g < ngr; ++g) {
                float a = 0.f, b = 0.f;
                okp = okp && cudaEventElapsedTime(&a, c->gev[0].first, c->gev[q0 + g].first) == cudaSuccess &&
                      cudaEventElapsedTime(&b, c->gev[0].first, c->gev[q0 + g].second) == cudaSuccess;
                t0 = g == 0 ? a : std::min(t0, a);
                t1 = g == 0 ? b : std::max(t1, b);
            }
            if (okp) {
                c->mtt_ms += t1 - t0;
                ++c->mtt_passes;
            }
        }
        if (poll) {
            const int *h = c->h_poll.as<int>();
            bool all = true;
            for (int q = 0; q < d.nrep; ++q) all = all && h[q];
            if (all) break;
        }
    }
    return SBT_OK;
}

static sbt_status ctx_alloc(sbt_ctx *c, const sbt_tensor *X0, int32_t R, const sbt_options *opt) {
    TRY(check_tensor(X0));
    TRY(check_options(opt, R));
    if (opt->prec == SBT_PREC_F64 && X0->dtype != SBT_F64)
        return fail(SBT_E_INVALID, "SBT_PREC_F64 needs a float64 store");
    c->opt = *opt;
    CK(cudaGetDevice(&c->device));
    CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    CK(ensure_kernel_attributes(c->device));
    c->user = (cudaStream_t)opt->cuda_stream;
    CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_user, cudaEventDisableTiming));
    TRY(order_after_user(c));
    c->I = (int)X0->I;
    c->J = (int)X0->J;
    c->R = R;
    c->K = X0->K;
    c->sdtype = X0->dtype;
    c->lds = round8(c->J);
    c->elem = opt->prec == SBT_PREC_F64 ? 0 : (opt->prec == SBT_PREC_F32 ? 1 : (opt->prec == SBT_PREC_BF16 ? 2 : 3));
    c->Kcap = std::max<int64_t>(opt->K_capacity > 0 ? opt->K_capacity : 2 * X0->K, X0->K + 1);
    const size_t es = esize_store(c->sdtype);
    TRY(c->store.ensure((size_t)c->Kcap * c->I * c->lds * es));
    CK(cudaMemsetAsync(c->store.p, 0, (size_t)c->Kcap * c->I * c->lds * es, c->stream));
    TRY(c->A.ensure((size_t)c->I * R * 8));
    TRY(c->B.ensure((size_t)c->J * R * 8));
    TRY(c->C.ensure((size_t)c->Kcap * R * 8));
    TRY(c->lam.ensure((size_t)R * 8));
    TRY(c->xa.ensure((size_t)c->I * 8));
    TRY(c->xb.ensure((size_t)c->J * 8));
    TRY(c->xc.ensure((size_t)c->Kcap * 8));
    TRY(c->dxa.ensure((size_t)c->I * 8));
    TRY(c->dxb.ensure((size_t)c->J * 8));
    TRY(c->status.ensure(sizeof(DevStatus)));
    TRY(c->h_status.ensure(sizeof(DevStatus)));
    if (c->elem == 3) {  // float8 summaries: max |x| of every stored slice, kept by the appends
        TRY(c->samax.ensure((size_t)c->Kcap * 4));
        CK(cudaMemsetAsync(c->samax.p, 0, (size_t)c->Kcap * 4, c->stream));
    }
    TRY(c->prof_bytes.ensure(8));
    CK(cudaMemsetAsync(c->prof_bytes.p, 0, 8, c->stream));
    CK(cudaMemsetAsync(c->status.p, 0, sizeof(DevStatus), c->stream));
    CK(cudaMemsetAsync(c->xa.p, 0, (size_t)c->I * 8, c->stream));
    CK(cudaMemsetAsync(c->xb.p, 0, (size_t)c->J * 8, c->stream));
    CK(cudaMemsetAsync(c->xc.p, 0, (size_t)c->Kcap * 8, c->stream));
    // X0 into the store, then the shift S from max |x| (Eq. 1 fixed point)
    const size_t sbytes = (size_t)X0->K * c->I * c->lds * es;
    if (X0->on_device) {
        CK(cudaMemcpy2DAsync(c->store.p, (size_t)c->lds * es, X0->data, (size_t)c->J * es, (size_t)c->J * es,
                             (size_t)X0->K * c->I, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        CK(cudaMemcpy2DAsync(c->store.p, (size_t)c->lds * es, X0->data, (size_t)c->J * es, (size_t)c->J * es,
                             (size_t)X0->K * c->I, cudaMemcpyHostToDevice, c->stream));
    }
    CK(launch_absmax(c->store.p, c->sdtype, (long long)(sbytes / es), c->status.as<DevStatus>(), c->stream));
    DevStatus hs;
    TRY(read_status(c, &hs));
    if (hs.err & ERR_NONFINITE) return fail(SBT_E_NONFINITE, "non-finite value in X0");
    double M;
    std::memcpy(&M, &hs.amax_bits, 8);
    if (M == 0.0) {
        c->S = 0;
    } else {
        int e2;
        std::frexp(M * M, &e2);
        c->S = 32 - e2;
    }
    CK(launch_append(c->store.p, c->sdtype, X0->K, c->I, c->J, c->lds, c->store.p, c->lds, c->S,
                     c->xa.as<unsigned long long>(), c->xb.as<unsigned long long>(),
                     c->xc.as<unsigned long long>(), c->samax.as<unsigned>(), c->status.as<DevStatus>(), c->stream));
    TRY(read_status(c, &hs));
    TRY(status_error(hs.err));
    // positive-weight counts
    std::vector<unsigned long long> h(std::max<int64_t>(std::max(c->I, c->J), X0->K));
    const unsigned long long *src[3] = {c->xa.as<unsigned long long>(), c->xb.as<unsigned long long>(),
                                        c->xc.as<unsigned long long>()};
    const int64_t len[3] = {c->I, c->J, X0->K};
    for (int m = 0; m < 3; ++m) {
        CK(cudaMemcpy(h.data(), src[m], (size_t)len[m] * 8, cudaMemcpyDeviceToHost));
        int64_t cnt = 0;
        for (int64_t x = 0; x < len[m]; ++x) cnt += h[x] != 0;
        c->npos[m] = cnt;
    }
    return SBT_OK;
}

static sbt_status reserve(sbt_ctx *c, int64_t K_max, int64_t K_new_max);

extern "C" sbt_status sbt_init(const sbt_tensor *X0, int32_t R, const sbt_options *opt, sbt_ctx **out) {
    if (!out) return fail(SBT_E_INVALID, "null output pointer");
    *out = nullptr;
    sbt_ctx *c = new sbt_ctx();
    sbt_status s = ctx_alloc(c, X0, R, opt);
    if (s != SBT_OK) {
        delete c;
        return s;
    }
    // CP-ALS of X0 in the store's own precision (the identity summary)
    AlsDesc d;
    const int n[3] = {c->I, c->J, (int)c->K};
    const int elem = c->sdtype == SBT_F64 ? 0 : 1;
    s = setup_als(c, d, 1, n, c->lds, (int)c->K, elem, c->store.p, 0, opt->max_iters_init);
    if (s == SBT_OK) s = c->rowsq.ensure((size_t)c->K * c->I * 8);
    if (s != SBT_OK) {
        delete c;
        return s;
    }
    cudaError_t e = launch_rowsq(c->store.p, c->sdtype, c->K * c->I, c->J, c->lds, c->rowsq.as<double>(), c->stream);
    if (e == cudaSuccess)
        e = launch_als_prepare(d, nullptr, 0, (int)c->K, true, opt->seed, opt->stream_id, 0xFFFFFFFFu,
                               c->rowsq.as<double>(), c->stream);
    if (e != cudaSuccess) {
        delete c;
        return fail(SBT_E_CUDA, std::string("init ALS launch: ") + cudaGetErrorString(e));
    }
    s = run_als(c, d, opt->max_iters_init);
    if (s == SBT_OK) {
        e = launch_canonicalize(d, c->A.as<double>(), c->B.as<double>(), c->C.as<double>(), c->lam.as<double>(),
                                c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) s = fail(SBT_E_CUDA, std::string("init canonicalize: ") + cudaGetErrorString(e));
        else settle_als_counts(c);
    }
    if (s == SBT_OK && opt->max_batch > 0) s = reserve(c, c->Kcap, opt->max_batch);
    if (s != SBT_OK) {
        delete c;
        return s;
    }
    *out = c;
    return SBT_OK;
}

extern "C" sbt_status sbt_init_factors(const sbt_tensor *X0, int32_t R, const double *lambda, const double *A,
                                       const double *B, const double *C, const sbt_options *opt, sbt_ctx **out) {
    if (!out) return fail(SBT_E_INVALID, "null output pointer");
    *out = nullptr;
    if (!lambda || !A || !B || !C) return fail(SBT_E_INVALID, "null factor pointer");
    sbt_ctx *c = new sbt_ctx();
    sbt_status s = ctx_alloc(c, X0, R, opt);
    if (s == SBT_OK) {
        cudaError_t e = cudaMemcpy(c->A.p, A, (size_t)c->I * R * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->B.p, B, (size_t)c->J * R * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->C.p, C, (size_t)c->K * R * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->lam.p, lambda, (size_t)R * 8, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) s = fail(SBT_E_CUDA, std::string("factor upload: ") + cudaGetErrorString(e));
    }
    if (s == SBT_OK && opt->max_batch > 0) s = reserve(c, c->Kcap, opt->max_batch);
    if (s != SBT_OK) {
        delete c;
        return s;
    }
    *out = c;
    return SBT_OK;
}

// Grow the store (and C, x_c) to hold at least `need` slices.
static sbt_status grow_store(sbt_ctx *c, int64_t need) {
    if (need <= c->Kcap) return SBT_OK;
    int64_t ncap = std::max<int64_t>(need, c->Kcap * 2);
    const size_t es = esize_store(c->sdtype);
    const size_t slice = (size_t)c->I * c->lds * es;
    Buf ns, nC, nxc, nam;
    TRY(ns.ensure(ncap * slice));
    TRY(nC.ensure((size_t)ncap * c->R * 8));
    TRY(nxc.ensure((size_t)ncap * 8));
    if (c->samax.p) {
        TRY(nam.ensure((size_t)ncap * 4));
        CK(cudaMemsetAsync(nam.p, 0, (size_t)ncap * 4, c->stream));
        CK(cudaMemcpyAsync(nam.p, c->samax.p, (size_t)c->K * 4, cudaMemcpyDeviceToDevice, c->stream));
    }
    CK(cudaMemsetAsync(ns.p, 0, ncap * slice, c->stream));
    CK(cudaMemsetAsync(nxc.p, 0, (size_t)ncap * 8, c->stream));
    CK(cudaMemcpyAsync(ns.p, c->store.p, c->K * slice, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(nC.p, c->C.p, (size_t)c->K * c->R * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(nxc.p, c->xc.p, (size_t)c->K * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::swap(c->store.p, ns.p);
    std::swap(c->store.cap, ns.cap);
    std::swap(c->C.p, nC.p);
    std::swap(c->C.cap, nC.cap);
    std::swap(c->xc.p, nxc.p);
    std::swap(c->xc.cap, nxc.cap);
    if (c->samax.p) {
        std::swap(c->samax.p, nam.p);
        std::swap(c->samax.cap, nam.cap);
    }
    c->Kcap = ncap;
    return SBT_OK;
}

// Shapes of one update of K_new slices on K_old old ones: the sample sizes of
// Section 3.1 (ceil(N / s), clamped to the positive weights) and everything
// the workspace depends on.  With `bound` the clamps are replaced by their
// largest possible values (used to size for future updates).
struct UpdShape {
    int64_t K_old = 0;
    int K_new = 0, nI = 0, nJ = 0, nK = 0, Kp = 0, ldj = 0, ldi = 0;
    long long samp_stride = 0, key_stride = 0, xrs = 0;
    bool tc = false;
};

static sbt_status update_shape(const sbt_ctx *c, int64_t K_old, int K_new, bool bound, UpdShape &u) {
    u.K_old = K_old;
    u.K_new = K_new;
    const int64_t pos[3] = {bound ? c->I : c->npos[0], bound ? c->J : c->npos[1], bound ? K_old : c->npos[2]};
    u.nI = (int)std::min<int64_t>(ceil_div(c->I, c->opt.s_I), pos[0]);
    u.nJ = (int)std::min<int64_t>(ceil_div(c->J, c->opt.s_J), pos[1]);
    u.nK = (int)std::min<int64_t>(ceil_div(K_old, c->opt.s_K), pos[2]);
    if (u.nI < 1 || u.nJ < 1 || u.nK < 1) return fail(SBT_E_STATE, "a mode has no positive weight to sample");
    u.Kp = u.nK + K_new;
    u.ldj = summary_ld(u.nJ, c->elem);
    u.ldi = summary_ld(u.nI, c->elem);
    u.samp_stride = std::max(u.nI, std::max(u.nJ, u.nK));
    u.key_stride = std::max<int64_t>(std::max(c->I, c->J), K_old);
    u.xrs = (long long)u.Kp * u.nI * u.ldj;
    u.tc = (c->elem == 2 || c->elem == 3) && tc_supported(c->R, u.nI, c->elem == 3) &&
           tc_supported(c->R, u.nJ, c->elem == 3);
    return SBT_OK;
}

// start of the summary ALS: the old factors at the sampled rows (option
// warm_start), else Philox uniforms
static WarmStart warm_start_of(const sbt_ctx *c) {
    WarmStart w;
    if (c->opt.warm_start) {
        w.F[0] = c->A.as<double>();
        w.F[1] = c->B.as<double>();
        w.F[2] = c->C.as<double>();
    }
    return w;
}

// mode 3 formed from the mode-2 pass's products (tensor-core path) unless
// the option asks for its own pass
static bool memo_mode3(const sbt_ctx *c, int) { return !c->opt.mode3_pass; }

// bytes of MTTKRP partial sums for an update of this shape; with `bound`, the
// largest over all summary lengths up to u.Kp (tile counts are not monotone)
static size_t update_part_bytes(const sbt_ctx *c, const UpdShape &u, bool bound) {
    const int r = c->opt.r;
    size_t best = 0;
    for (int Kp = bound ? 1 : u.Kp; Kp <= u.Kp; ++Kp) {
        AlsDesc d;
        const int n[3] = {u.nI, u.nJ, Kp};
        als_shape(c, d, r, n, u.ldj, u.nK, als_elem(c), c->opt.max_iters);
        best = std::max<size_t>(best, (size_t)r * d.prs * esize_tf(als_elem(c)));
        if (c->opt.get_rank) {  // GetRank's final ALS runs one repetition at a time
            AlsDesc d1;
            als_shape(c, d1, 1, n, u.ldj, u.nK, als_elem(c), c->opt.max_iters);
            best = std::max<size_t>(best, (size_t)d1.prs * esize_tf(als_elem(c)));
        }
        if (u.tc) {
            tc_group_partials(c, d, als_group_count(c, r, true));
            best = std::max<size_t>(best, (size_t)r * d.prs * 4);
        }
    }
    return best;
}

// every device buffer an update of shape u uses (the store and its growth
// included only in a dry run: grow_store moves the contents itself)
static sbt_status size_update(sbt_ctx *c, const UpdShape &u, bool bound, Sizer &z) {
    const int r = c->opt.r, R = c->R;
    TRY(z.need(c->samples, (size_t)r * 3 * u.samp_stride * 4));
    TRY(z.need(c->khi, (size_t)r * 3 * u.key_stride * 8));
    TRY(z.need(c->klo, (size_t)r * 3 * u.key_stride * 8));
    TRY(z.need(c->Xs, (size_t)r * u.xrs * esize_elem(c->elem)));
    TRY(z.need(c->rowsq, (size_t)r * u.Kp * u.nI * 8));
    TRY(z.need(c->xc_new, (size_t)u.K_new * 8));
    AlsDesc d;
    const int n[3] = {u.nI, u.nJ, u.Kp};
    als_shape(c, d, r, n, u.ldj, u.nK, als_elem(c), c->opt.max_iters);
    TRY(als_sizes(c, d, update_part_bytes(c, u, bound), z));
    if (u.tc) TRY(z.need(c->Xt, (size_t)r * u.Kp * u.nJ * u.ldi * esize_elem(c->elem)));
    if (u.tc && memo_mode3(c, u.nJ)) TRY(z.need(c->ymem, (size_t)r * u.Kp * u.nJ * d.pr * 4));
    if (c->elem == 3) TRY(z.need(c->sscale, (size_t)r * u.Kp * 4));
    if (u.tc && c->opt.refine_sweeps > 0) {
        TRY(z.need(c->Xlo, (size_t)r * u.xrs * 2));
        TRY(z.need(c->Xtlo, (size_t)r * u.Kp * u.nJ * u.ldi * 2));
        TRY(z.need(c->rowsq2, (size_t)r * u.Kp * u.nI * 8));
        TRY(z.need(c->iters_main, (size_t)r * 4));
    }
    if (c->opt.persistent_als) {  // barrier words and the descriptor of the persistent ALS
        TRY(z.need(c->psync, PA_SYNC_WORDS * sizeof(unsigned)));
        TRY(z.need(c->pdesc, sizeof(AlsDesc)));
    }
    if (c->opt.get_rank) {
        // CorConDia scratch of one candidate and the widened factors; scores
        // and status words of every (repetition, rank, trial); R_new
        const int T = c->opt.get_rank_trials > 0 ? c->opt.get_rank_trials : 2;
        const size_t nd = core_consistency_scratch_doubles(u.Kp, u.nI, u.nJ, R) +
                          (size_t)(u.nI + u.nJ + u.Kp) * R;
        TRY(z.need(c->grscr, nd * 8));
        TRY(z.need(c->gcc, (size_t)r * R * T * (8 + 4)));
        TRY(z.need(c->rnew, (size_t)r * 4));
    }
    const size_t pmax = (size_t)u.samp_stride;
    TRY(z.need(c->nu, (size_t)r * 3 * R * 8));
    TRY(z.need(c->cnew, (size_t)r * u.K_new * R * 8));
    TRY(z.need(c->prop, (size_t)r * 3 * pmax * R * 8));
    TRY(z.need(c->lam_est, (size_t)r * R * 8));
    TRY(z.need(c->perm, (size_t)r * R * 4));
    TRY(z.need(c->min_score, (size_t)r * 8));
    TRY(z.need(c->mdots, (size_t)r * 3 * (32 * 32 + 64) * 8));
    if (z.dry && u.K_old + u.K_new > c->Kcap) {
        const int64_t ncap = std::max<int64_t>(u.K_old + u.K_new, c->Kcap * 2);
        TRY(z.need(c->store, (size_t)ncap * c->I * c->lds * esize_store(c->sdtype)));
        TRY(z.need(c->C, (size_t)ncap * R * 8));
        TRY(z.need(c->xc, (size_t)ncap * 8));
    }
    return SBT_OK;
}

// all device buffers of a context
static std::vector<Buf *> ctx_bufs(sbt_ctx *c) {
    return {&c->store, &c->A, &c->B, &c->C, &c->lam, &c->xa, &c->xb, &c->xc, &c->dxa, &c->dxb, &c->xc_new,
            &c->status, &c->samples, &c->khi, &c->klo, &c->Xs, &c->rowsq, &c->U[0], &c->U[1], &c->U[2], &c->M,
            &c->part, &c->G, &c->lam_s, &c->fit, &c->fit_prev, &c->normX2, &c->iters, &c->conv, &c->flags,
            &c->nu, &c->cnew, &c->prop, &c->lam_est, &c->perm, &c->min_score, &c->mdots, &c->fitscr, &c->staging,
            &c->Xt, &c->tpart, &c->xinv, &c->tail_cnt, &c->Gf, &c->dfs, &c->prof_bytes, &c->passes,
            &c->Xlo, &c->Xtlo, &c->rowsq2, &c->iters_main, &c->samax, &c->sscale, &c->ymem,
            &c->grscr, &c->gcc, &c->rnew, &c->psync, &c->pdesc,
            &c->si, &c->sj, &c->sv, &c->sptr, &c->cin_i, &c->cin_j, &c->cin_k, &c->cin_v, &c->ccnt, &c->cfill,
            &c->cmax, &c->posI, &c->posJ, &c->gcnt, &c->goff, &c->gtot, &c->vmax, &c->fexp, &c->eii, &c->ejj,
            &c->ekk, &c->ev, &c->perm1, &c->perm2, &c->rp1, &c->rp2, &c->gc1, &c->gc2, &c->gf1, &c->gf2};
}

// device bytes after the needs of z (every buffer at max(capacity, need))
static uint64_t footprint(sbt_ctx *c, const Sizer &z) {
    uint64_t total = 0;
    for (Buf *b : ctx_bufs(c)) {
        size_t cap = b->cap;
        for (const auto &w : z.want)
            if (w.first == b) cap = std::max(cap, w.second);
        total += cap;
    }
    return total;
}

// Size the store and the workspace so that every update that keeps K <= K_max
// with K_new <= K_new_max allocates nothing.
static sbt_status reserve(sbt_ctx *c, int64_t K_max, int64_t K_new_max) {
    if (K_new_max < 1 || K_max <= c->K) return fail(SBT_E_INVALID, "sbt_reserve: need K_new_max >= 1, K_max > K");
    K_new_max = std::min<int64_t>(K_new_max, K_max - c->K);
    TRY(grow_store(c, K_max));
    Sizer z;
    // sizes grow with K_old and K_new except the tile counts, which
    // update_part_bytes bounds over every summary length
    UpdShape u;
    TRY(update_shape(c, K_max - 1, 1, true, u));
    TRY(size_update(c, u, true, z));
    TRY(update_shape(c, K_max - K_new_max, (int)K_new_max, true, u));
    TRY(size_update(c, u, true, z));
    return SBT_OK;
}

extern "C" sbt_status sbt_tile_table(int32_t op, sbt_tile_entry *entries, int32_t cap, int32_t *n) {
    static_assert(sizeof(sbt_tile_entry) == 9 * sizeof(int32_t), "sbt_tile_entry layout");
    if (op == 0) {
        if (!n || (cap > 0 && !entries)) return fail(SBT_E_INVALID, "sbt_tile_table: bad arguments");
        *n = tile_table_read(reinterpret_cast<int *>(entries), cap);
        return SBT_OK;
    }
    if (op == 1) {
        if (cap < 0 || (cap > 0 && !entries)) return fail(SBT_E_INVALID, "sbt_tile_table: bad arguments");
        for (int q = 0; q < cap; ++q) {
            const sbt_tile_entry &e = entries[q];
            if ((e.ctas_per_sm != 1 && e.ctas_per_sm != 2) || e.stages < 0 || e.stages > 8)
                return fail(SBT_E_INVALID, "sbt_tile_table: ctas_per_sm must be 1 or 2, stages 0..8");
        }
        tile_table_merge(reinterpret_cast<const int *>(entries), cap);
        return SBT_OK;
    }
    if (op == 2) {
        tile_table_clear();
        return SBT_OK;
    }
    return fail(SBT_E_INVALID, "sbt_tile_table: op must be 0 (read), 1 (merge) or 2 (clear)");
}

extern "C" sbt_status sbt_device_bytes(sbt_ctx *c, uint64_t *bytes) {
    if (!c || !bytes) return fail(SBT_E_INVALID, "null argument");
    Sizer z;
    *bytes = footprint(c, z);
    return SBT_OK;
}

extern "C" sbt_status sbt_update_bytes(sbt_ctx *c, int64_t K_new, uint64_t *bytes) {
    if (!c || !bytes || K_new < 1 || K_new > INT32_MAX) return fail(SBT_E_INVALID, "sbt_update_bytes: bad arguments");
    if (c->coo) return fail(SBT_E_INVALID, "sbt_update_bytes: dense contexts only");
    UpdShape u;
    TRY(update_shape(c, c->K, (int)K_new, false, u));
    Sizer z;
    z.dry = true;
    TRY(size_update(c, u, false, z));
    *bytes = footprint(c, z);
    return SBT_OK;
}

extern "C" sbt_status sbt_reserve(sbt_ctx *c, int64_t K_max, int64_t K_new_max) {
    if (!c) return fail(SBT_E_INVALID, "null context");
    if (c->coo) return fail(SBT_E_INVALID, "sbt_reserve: dense contexts only");
    DeviceGuard dg(c->device);
    return reserve(c, K_max, K_new_max);
}

// Steps 5 and 6 of an update (shared-row normalisation, matching, project
// back, commit) and its statistics; shared by the dense and the COO updates.
static sbt_status match_commit(sbt_ctx *c, const AlsDesc &d, int64_t K_old, int K_new, int nI, int nJ, int nK,
                               long long samp_stride, int ldj, bool refined, bool no_refine,
                               const std::vector<int> *rnew = nullptr) {
    const int R = c->R, r = c->opt.r;
    // 5. normalise, match, project back; 6. commit
    const int pmax = (int)samp_stride;
    MergeDesc m;
    std::memset(&m, 0, sizeof(m));
    m.nrep = r;
    m.R = R;
    m.I = c->I;
    m.J = c->J;
    m.K_old = (int)K_old;
    m.K_new = K_new;
    m.nI = nI;
    m.nJ = nJ;
    m.nK = nK;
    m.samples = c->samples.as<int>();
    m.samp_stride = samp_stride;
    for (int q = 0; q < 3; ++q) m.U[q] = c->U[q].p;
    m.elem = c->elem == 0 ? 0 : 1;
    m.lam_s = c->lam_s.as<double>();
    m.A = c->A.as<double>();
    m.B = c->B.as<double>();
    m.C = c->C.as<double>();
    m.lam = c->lam.as<double>();
    m.nu = c->nu.as<double>();
    m.cnew = c->cnew.as<double>();
    m.prop = c->prop.as<double>();
    m.pmax = pmax;
    m.lam_est = c->lam_est.as<double>();
    m.perm = c->perm.as<int>();
    m.min_score = c->min_score.as<double>();
    m.dots = c->mdots.as<double>();
    m.flags = c->flags.as<int>();
    m.lambda_mode = c->opt.lambda_mode;
    m.xa = c->xa.as<unsigned long long>();
    m.xb = c->xb.as<unsigned long long>();
    m.xc = c->xc.as<unsigned long long>();
    m.dxa = c->dxa.as<unsigned long long>();
    m.dxb = c->dxb.as<unsigned long long>();
    m.xc_new = c->xc_new.as<unsigned long long>();
    m.status = c->status.as<DevStatus>();
    m.rnew = rnew ? c->rnew.as<int>() : nullptr;
    CK(launch_match(m, c->stream));
    CK(launch_precommit(m, c->stream));
    CK(launch_commit(m, c->stream));
    // 7. one synchronisation: status and statistics
    const size_t stat_bytes = sizeof(DevStatus) + (size_t)r * (4 + 8 + 8 + 4 + 4 * R);
    TRY(c->h_stats.ensure(stat_bytes));
    char *hb = c->h_stats.as<char>();
    CK(cudaMemcpyAsync(hb, c->status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
    size_t off = sizeof(DevStatus);
    CK(cudaMemcpyAsync(hb + off, refined ? c->iters_main.p : (void *)d.iters, (size_t)r * 4,
                       cudaMemcpyDeviceToHost, c->stream));
    off += (size_t)r * 4;
    CK(cudaMemcpyAsync(hb + off, d.fit, (size_t)r * 8, cudaMemcpyDeviceToHost, c->stream));
    off += (size_t)r * 8;
    CK(cudaMemcpyAsync(hb + off, m.min_score, (size_t)r * 8, cudaMemcpyDeviceToHost, c->stream));
    off += (size_t)r * 8;
    CK(cudaMemcpyAsync(hb + off, d.flags, (size_t)r * 4, cudaMemcpyDeviceToHost, c->stream));
    off += (size_t)r * 4;
    CK(cudaMemcpyAsync(hb + off, m.perm, (size_t)r * R * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    settle_als_counts(c);
    DevStatus hs;
    std::memcpy(&hs, hb, sizeof(DevStatus));
    if (hs.err) return status_error(hs.err);
    // the update is committed
    c->updates += 1;
    c->K = K_old + K_new;
    c->batch += 1;
    for (int q = 0; q < 3; ++q) c->npos[q] = (int64_t)hs.npos[q];
    sbt_update_stats &st = c->stats;
    std::memset(&st, 0, sizeof(st));
    st.K = c->K;
    st.r = r;
    st.R = R;
    st.n_I = nI;
    st.n_J = nJ;
    st.n_K = nK;
    off = sizeof(DevStatus);
    const int *it = (const int *)(hb + off);
    off += (size_t)r * 4;
    const double *ft = (const double *)(hb + off);
    off += (size_t)r * 8;
    const double *ms = (const double *)(hb + off);
    off += (size_t)r * 8;
    const int *fl = (const int *)(hb + off);
    off += (size_t)r * 4;
    const int *pm = (const int *)(hb + off);
    if (no_refine) st.flags |= SBT_FLAG_NO_REFINE;
    if (std::min(nI, std::min(nJ, nK)) < R) st.flags |= SBT_FLAG_SAMPLE_LT_RANK;
    c->last_rank.assign(r, R);
    if (rnew) c->last_rank = *rnew;
    for (int q = 0; q < r; ++q) {
        st.rank[q] = c->last_rank[q];
        st.iters[q] = it[q];
        st.fit[q] = ft[q];
        st.min_score[q] = ms[q];
        st.flags |= fl[q];
        for (int a = 0; a < R; ++a) st.perm[q][a] = pm[q * R + a];
    }
    c->have_last = true;
    c->last_nI = nI;
    c->last_nJ = nJ;
    c->last_nK = nK;
    c->last_Knew = K_new;
    c->last_ldj = ldj;
    c->last_samp_stride = samp_stride;
    return SBT_OK;
}

// The rank-dependent fields of a descriptor (tiles, partial and M strides,
// tail chunks) for rank `rank`, its pointers kept.
static void set_rank(const sbt_ctx *c, AlsDesc &d, int rank) {
    AlsDesc t;
    als_shape(c, t, d.nrep, d.n, d.ldj, d.nK, d.elem, d.max_iters, rank);
    d.R = t.R;
    d.pr = t.pr;
    d.mrs = t.mrs;
    d.prs = t.prs;
    d.tchunks = t.tchunks;
    d.spc = t.spc;
    d.nks = t.nks;
    d.nib = t.nib;
    d.jc = t.jc;
    d.rows_per = t.rows_per;
    d.nrs = t.nrs;
    d.cols = t.cols;
    for (int m = 0; m < 3; ++m) d.P[m] = t.P[m];
}

// GetRank (Section 3.2, Algorithm 2) on the r summaries, then step 5 of
// Algorithm 1 at each repetition's estimated rank.  For every trial t and
// candidate rank i = 1..R: one batched CP-ALS of all r summaries at rank i
// from trial t's Philox start (CUDA-core MTTKRP), then the core consistency
// (float64) of every repetition's model.  R_new(rho) = the largest rank whose
// best trial reaches the threshold (1 if none; a candidate whose factor Gram
// is singular does not reach it).  The summary ALS of repetition rho then
// runs alone at rank R_new(rho) from the usual start, its factors in the
// repetition's n x R slot as rows of R_new(rho) values.
static sbt_status get_rank_als(sbt_ctx *c, const UpdShape &u, const AlsDesc &d_full, std::vector<int> &rnew) {
    const int R = c->R, r = c->opt.r;
    const int T = c->opt.get_rank_trials > 0 ? c->opt.get_rank_trials : 2;
    const double thr = c->opt.get_rank_threshold != 0.0 ? c->opt.get_rank_threshold : 90.0;
    const int elem = als_elem(c);
    const int n[3] = {u.nI, u.nJ, u.Kp};
    const size_t xes = esize_elem(c->elem);
    const size_t nslots = (size_t)r * R * T;
    double *cc = c->gcc.as<double>();
    int *cst = reinterpret_cast<int *>(cc + nslots);
    CK(cudaMemsetAsync(cst, 0, nslots * 4, c->stream));
    double *scr = c->grscr.as<double>();
    const size_t nd = core_consistency_scratch_doubles(u.Kp, u.nI, u.nJ, R);
    double *F64[3] = {scr + nd, scr + nd + (size_t)u.nI * R, scr + nd + (size_t)(u.nI + u.nJ) * R};
    const int *samples = c->samples.as<int>();
    const double *rowsq = c->rowsq.as<double>();
    for (int t = 0; t < T; ++t) {
        for (int i = 1; i <= R; ++i) {
            AlsDesc dc;
            als_shape(c, dc, r, n, u.ldj, u.nK, elem, c->opt.max_iters, i);
            TRY(als_bind(c, dc, c->Xs.p, u.xrs));
            WarmStart ws;
            ws.trial = t;
            CK(launch_als_prepare(dc, samples, u.samp_stride, (int)u.K_old, false, c->opt.seed, c->opt.stream_id,
                                  c->batch, rowsq, c->stream, ws));
            TRY(run_als(c, dc, c->opt.max_iters));
            for (int rho = 0; rho < r; ++rho) {
                const double *Fd[3];
                for (int m = 0; m < 3; ++m) {
                    const long long cnt = (long long)n[m] * i;
                    if (elem == 0) {
                        Fd[m] = (const double *)dc.U[m] + rho * cnt;
                    } else {
                        CK(launch_widen((const float *)dc.U[m] + rho * cnt, F64[m], cnt, c->stream));
                        Fd[m] = F64[m];
                    }
                }
                const size_t slot = ((size_t)rho * R + (i - 1)) * T + t;
                CK(launch_core_consistency(elem, (const char *)c->Xs.p + (size_t)rho * u.xrs * xes, u.Kp, u.nI,
                                           u.nJ, u.ldj, dc.lam + (size_t)rho * i, Fd[0], Fd[1], Fd[2], i, scr,
                                           cst + slot, cc + slot, c->stream));
            }
        }
    }
    std::vector<double> h(nslots);
    std::vector<int> hs(nslots);
    CK(cudaMemcpyAsync(h.data(), cc, nslots * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(hs.data(), cst, nslots * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    settle_als_counts(c);
    rnew.assign(r, 1);
    for (int rho = 0; rho < r; ++rho)
        for (int i = 1; i <= R; ++i) {
            double best = -INFINITY;
            for (int t = 0; t < T; ++t) {
                const size_t slot = ((size_t)rho * R + (i - 1)) * T + t;
                if (!hs[slot] && std::isfinite(h[slot])) best = std::max(best, h[slot]);
            }
            if (best >= thr) rnew[rho] = i;
        }
    CK(cudaMemcpyAsync(c->rnew.p, rnew.data(), (size_t)r * 4, cudaMemcpyHostToDevice, c->stream));
    // the summary ALS of each repetition at its rank (the partial sums are
    // scratch of one run, so every run takes them from the start of the buffer)
    for (int rho = 0; rho < r; ++rho) {
        AlsDesc d1 = group_desc(d_full, rho, 1, (size_t)u.xrs * xes);
        set_rank(c, d1, rnew[rho]);
        d1.part = c->part.p;
        CK(launch_als_prepare(d1, samples + (size_t)rho * 3 * u.samp_stride, u.samp_stride, (int)u.K_old, false,
                              c->opt.seed, c->opt.stream_id, c->batch, rowsq + (size_t)rho * u.Kp * u.nI,
                              c->stream, WarmStart{}));
        TRY(run_als(c, d1, c->opt.max_iters));
    }
    return SBT_OK;
}

// Alg. 1 for one batch.  deferred non-null: an update whose ALS can join a
// batched persistent launch (persistent_als, the CUDA-core path, no
// per-launch timing) stops before it, with *deferred = true.
static sbt_status update_impl(sbt_ctx *c, const sbt_tensor *X, bool *deferred) {
    if (!c) return fail(SBT_E_INVALID, "null context");
    if (c->pend.on) return fail(SBT_E_STATE, "an update of this context is pending");
    if (c->coo) return fail(SBT_E_INVALID, "a COO context takes sbt_update_coo");
    TRY(check_tensor(X));
    if (X->I != c->I || X->J != c->J) return fail(SBT_E_SHAPE, "I and J must match the initial tensor");
    if (X->dtype != c->sdtype) return fail(SBT_E_INVALID, "dtype must match the initial tensor");
    DeviceGuard dg(c->device);
    TRY(order_after_user(c));
    const int R = c->R, r = c->opt.r;
    const int K_new = (int)X->K;
    const int64_t K_old = c->K;
    UpdShape u;
    TRY(update_shape(c, K_old, K_new, false, u));
    TRY(grow_store(c, K_old + K_new));
    {
        Sizer z;
        TRY(size_update(c, u, false, z));
    }
    if (c->elem == 3 && !u.tc) return fail(SBT_E_INVALID, "float8 summaries need the tensor-core MTTKRP (R <= 32)");
    if (c->opt.get_rank && (c->elem == 3 || c->opt.refine_sweeps > 0))
        return fail(SBT_E_INVALID, "get_rank takes float64, float32 or bfloat16 summaries without refinement");
    const int nI = u.nI, nJ = u.nJ, nK = u.nK, Kp = u.Kp, ldj = u.ldj;
    const long long samp_stride = u.samp_stride, key_stride = u.key_stride, xrs = u.xrs;
    // 1. append + marginal deltas
    CK(cudaMemsetAsync(c->status.p, 0, sizeof(DevStatus), c->stream));
    CK(cudaMemsetAsync(c->dxa.p, 0, (size_t)c->I * 8, c->stream));
    CK(cudaMemsetAsync(c->dxb.p, 0, (size_t)c->J * 8, c->stream));
    CK(cudaMemsetAsync(c->xc_new.p, 0, (size_t)K_new * 8, c->stream));
    if (c->samax.p) CK(cudaMemsetAsync(c->samax.as<unsigned>() + K_old, 0, (size_t)K_new * 4, c->stream));
    TRY(append_slices(c, X, K_old, c->dxa.as<unsigned long long>(), c->dxb.as<unsigned long long>(),
                      c->xc_new.as<unsigned long long>()));
    // 2. sampling from the marginals of the tensor before the update
    SampleParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.w[0] = c->xa.as<unsigned long long>();
    sp.w[1] = c->xb.as<unsigned long long>();
    sp.w[2] = c->xc.as<unsigned long long>();
    sp.N[0] = c->I;
    sp.N[1] = c->J;
    sp.N[2] = (int)K_old;
    sp.n[0] = nI;
    sp.n[1] = nJ;
    sp.n[2] = nK;
    sp.mode_id[0] = 0;
    sp.mode_id[1] = 1;
    sp.mode_id[2] = 2;
    sp.nmodes = 3;
    sp.nrep = r;
    sp.rep0 = 0;
    sp.out = c->samples.as<int>();
    sp.out_stride = samp_stride;
    sp.khi = c->khi.as<unsigned long long>();
    sp.klo = c->klo.as<unsigned long long>();
    sp.key_stride = key_stride;
    sp.seed = c->opt.seed;
    sp.stream_id = c->opt.stream_id;
    sp.batch = c->batch;
    sp.status = c->status.as<DevStatus>();
    CK(launch_sample(sp, c->stream));
    // 3. gather the summaries
    GatherParams g;
    std::memset(&g, 0, sizeof(g));
    g.store = c->store.p;
    g.I = c->I;
    g.lds = c->lds;
    g.samples = c->samples.as<int>();
    g.samp_stride = samp_stride;
    g.nI = nI;
    g.nJ = nJ;
    g.nK = nK;
    g.K_old = (int)K_old;
    g.K_new = K_new;
    g.nrep = r;
    g.Xs = c->Xs.p;
    g.ldj = ldj;
    g.xrs = xrs;
    g.rowsq = c->rowsq.as<double>();
    if (u.tc) {  // the transposed copy for the mode-2 tensor-core pass, written by the gather
        g.Xt = c->Xt.p;
        g.ldi = u.ldi;
        g.xtrs = (long long)Kp * nJ * u.ldi;
        if (c->elem == 3) {  // float8: per-slice scales from the stored slices' max |x|
            g.samax = c->samax.as<unsigned>();
            g.sscale = c->sscale.as<float>();
        }
        if (c->opt.refine_sweeps > 0 && c->elem == 2) {  // and the lo parts of the split summary
            g.Xlo = c->Xlo.p;
            g.Xtlo = c->Xtlo.p;
            g.rowsq2 = c->rowsq2.as<double>();
        }
    }
    CK(launch_gather(g, c->sdtype, c->elem, c->stream));
    // 4. CP-ALS on the r summaries
    AlsDesc d;
    const int n[3] = {nI, nJ, Kp};
    als_shape(c, d, r, n, ldj, nK, als_elem(c), c->opt.max_iters);
    TRY(als_bind(c, d, c->Xs.p, xrs));
    // bfloat16 summaries: tensor-core MTTKRP over the summary and its transposed copy
    TcPlan &tc = c->tc;
    tc.on = u.tc && !c->opt.get_rank;
    if (tc.on && !c->opt.fp64_tail) d.tail64 = 0;  // the persistent ALS does not apply to the tensor-core plan
    if (c->opt.get_rank) {  // Section 3.2: the rank of every summary first (Algorithm 2)
        std::vector<int> rn;
        TRY(get_rank_als(c, u, d, rn));
        return match_commit(c, d, K_old, K_new, nI, nJ, nK, samp_stride, ldj, false, false, &rn);
    }
    if (tc.on) {
        const int ldi = u.ldi;
        CK(make_summary_tmap(&tc.m1, c->Xs.p, nJ, nI, ldj, (long long)r * Kp, c->elem == 3));
        CK(make_summary_tmap(&tc.m2, c->Xt.p, nI, nJ, ldi, (long long)r * Kp, c->elem == 3));
        tc.sscale = c->elem == 3 ? c->sscale.as<float>() : nullptr;
        tc.xs = c->Xs.p;
        tc.xt = c->Xt.p;
        tc.nI = nI;
        tc.nJ = nJ;
        tc.ldj = ldj;
        tc.ldi = ldi;
        tc.Kp = Kp;
        tc.fp8 = c->elem == 3;
        tc_group_partials(c, d, als_group_count(c, r, true));
        if (memo_mode3(c, nJ)) {
            d.ymem = c->ymem.as<float>();
            d.yrs = (long long)Kp * nJ * d.pr;
        }
    }
    CK(launch_als_prepare(d, c->samples.as<int>(), samp_stride, (int)K_old, false, c->opt.seed, c->opt.stream_id,
                          c->batch, c->rowsq.as<double>(), c->stream, warm_start_of(c)));
    if (tc.on && c->opt.autotune) {  // tile choices for the groups' launch shapes not seen before
        std::vector<AlsPlan> plans;
        TRY(als_plans(c, d, &tc, plans));
        for (AlsPlan &pl : plans) TRY(autotune_tiles(c, pl.d, pl.tc));
    }
    if (deferred && c->opt.persistent_als && !tc.on && !c->timing) {
        c->pend.d = d;
        c->pend.K_old = K_old;
        c->pend.K_new = K_new;
        c->pend.nI = nI;
        c->pend.nJ = nJ;
        c->pend.nK = nK;
        c->pend.ldj = ldj;
        c->pend.samp_stride = samp_stride;
        c->pend.on = true;
        *deferred = true;
        return SBT_OK;
    }
    TRY(run_als(c, d, c->opt.max_iters, tc.on ? &tc : nullptr));
    // refinement sweeps: the same ALS continued for refine_sweeps iterations
    // with every MTTKRP on the split summary (hi + lo)
    bool refined = false, no_refine = false;
    if (c->opt.refine_sweeps > 0 && c->elem == 2) {
        if (!tc.on) {
            no_refine = true;
        } else {
            CK(make_summary_tmap(&tc.m1lo, c->Xlo.p, nJ, nI, ldj, (long long)r * Kp, false));
            CK(make_summary_tmap(&tc.m2lo, c->Xtlo.p, nI, nJ, u.ldi, (long long)r * Kp, false));
            tc.xlo = c->Xlo.p;
            tc.xtlo = c->Xtlo.p;
            CK(cudaMemcpyAsync(c->iters_main.p, d.iters, (size_t)r * 4, cudaMemcpyDeviceToDevice, c->stream));
            CK(launch_refine_start(d, c->rowsq2.as<double>(), c->stream));
            AlsDesc dr = d;
            dr.fixed_iters = 1;
            dr.max_iters = c->opt.refine_sweeps;
            tc.split = true;
            const sbt_status rs = run_als(c, dr, c->opt.refine_sweeps, &tc);
            tc.split = false;
            TRY(rs);
            refined = true;
        }
    }
    return match_commit(c, d, K_old, K_new, nI, nJ, nK, samp_stride, ldj, refined, no_refine);
}

extern "C" sbt_status sbt_update(sbt_ctx *c, const sbt_tensor *X) { return update_impl(c, X, nullptr); }

namespace sbt {

sbt_status update_deferred(sbt_ctx *c, const sbt_tensor *X, bool *deferred) {
    *deferred = false;
    return update_impl(c, X, deferred);
}

sbt_status deferred_als(sbt_ctx *c, AlsDesc *d, cudaStream_t *st, int *num_sms) {
    if (!c || !c->pend.on) return fail(SBT_E_STATE, "no pending update");
    *d = c->pend.d;
    *st = c->stream;
    *num_sms = c->num_sms;
    return SBT_OK;
}

sbt_status update_complete(sbt_ctx *c) {
    if (!c || !c->pend.on) return fail(SBT_E_STATE, "no pending update");
    DeviceGuard dg(c->device);
    PendingAls p = c->pend;
    c->pend.on = false;
    return match_commit(c, p.d, p.K_old, p.K_new, p.nI, p.nJ, p.nK, p.samp_stride, p.ldj, false, false);
}

void update_abandon(sbt_ctx *c) {
    // the model and K are untouched until the commit: nothing to undo
    if (c) c->pend.on = false;
}

}  // namespace sbt

extern "C" sbt_status sbt_factors(const sbt_ctx *c, double *lambda, double *A, double *B, double *C, int64_t *K_out) {
    if (!c) return fail(SBT_E_INVALID, "null context");
    DeviceGuard dg(c->device);
    CK(cudaStreamSynchronize(c->stream));
    if (lambda) CK(cudaMemcpy(lambda, c->lam.p, (size_t)c->R * 8, cudaMemcpyDeviceToHost));
    if (A) CK(cudaMemcpy(A, c->A.p, (size_t)c->I * c->R * 8, cudaMemcpyDeviceToHost));
    if (B) CK(cudaMemcpy(B, c->B.p, (size_t)c->J * c->R * 8, cudaMemcpyDeviceToHost));
    if (C) CK(cudaMemcpy(C, c->C.p, (size_t)c->K * c->R * 8, cudaMemcpyDeviceToHost));
    if (K_out) *K_out = c->K;
    return SBT_OK;
}

static sbt_status coo_fit(sbt_ctx *c, double *fit);

extern "C" sbt_status sbt_fit(sbt_ctx *c, double *fit) {
    if (!c || !fit) return fail(SBT_E_INVALID, "null argument");
    DeviceGuard dg(c->device);
    if (c->coo) return coo_fit(c, fit);
    const long long need = fit_scratch_doubles((int)c->K, c->I, c->J, c->R) + 2;
    TRY(c->fitscr.ensure((size_t)need * 8));
    double *scr = c->fitscr.as<double>();
    CK(launch_full_fit(c->store.p, c->sdtype, (int)c->K, c->I, c->J, c->lds, c->A.as<double>(), c->B.as<double>(),
                       c->C.as<double>(), c->lam.as<double>(), c->R, scr + need - 2, scr, c->stream));
    double h[2];
    CK(cudaMemcpyAsync(h, scr + need - 2, 16, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *fit = h[1] > 0.0 ? 1.0 - std::sqrt(h[0]) / std::sqrt(h[1]) : 0.0;
    return SBT_OK;
}

extern "C" sbt_status sbt_recompute(sbt_ctx *c, int32_t max_iters, double tol, uint64_t seed, double *lambda,
                                    double *A, double *B, double *C, double *fit) {
    if (!c) return fail(SBT_E_INVALID, "null context");
    if (c->coo) return fail(SBT_E_STATE, "sbt_recompute takes dense contexts");
    if (max_iters < 1 || !(tol >= 0.0)) return fail(SBT_E_INVALID, "max_iters >= 1 and tol >= 0 required");
    DeviceGuard dg(c->device);
    CK(cudaStreamSynchronize(c->stream));
    settle_als_counts(c);
    const int R = c->R, K = (int)c->K;
    // the same CP-ALS as sbt_init, on the whole store
    AlsDesc d;
    const int n[3] = {c->I, c->J, K};
    const int elem = c->sdtype == SBT_F64 ? 0 : 1;
    TRY(setup_als(c, d, 1, n, c->lds, K, elem, c->store.p, 0, max_iters));
    d.tol = tol;
    TRY(c->rowsq.ensure((size_t)K * c->I * 8));
    Buf tA, tB, tC, tl, scr;
    TRY(tA.ensure((size_t)c->I * R * 8));
    TRY(tB.ensure((size_t)c->J * R * 8));
    TRY(tC.ensure((size_t)K * R * 8));
    TRY(tl.ensure((size_t)R * 8));
    CK(launch_rowsq(c->store.p, c->sdtype, (long long)K * c->I, c->J, c->lds, c->rowsq.as<double>(), c->stream));
    CK(launch_als_prepare(d, nullptr, 0, K, true, seed, c->opt.stream_id, 0xFFFFFFFFu, c->rowsq.as<double>(),
                          c->stream));
    TRY(run_als(c, d, max_iters));
    CK(launch_canonicalize(d, tA.as<double>(), tB.as<double>(), tC.as<double>(), tl.as<double>(), c->stream));
    const long long need = fit_scratch_doubles(K, c->I, c->J, R) + 2;
    TRY(scr.ensure((size_t)need * 8));
    double *sp = scr.as<double>();
    CK(launch_full_fit(c->store.p, c->sdtype, K, c->I, c->J, c->lds, tA.as<double>(), tB.as<double>(),
                       tC.as<double>(), tl.as<double>(), R, sp + need - 2, sp, c->stream));
    double h[2];
    CK(cudaMemcpyAsync(h, sp + need - 2, 16, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    settle_als_counts(c);
    if (lambda) CK(cudaMemcpy(lambda, tl.p, (size_t)R * 8, cudaMemcpyDeviceToHost));
    if (A) CK(cudaMemcpy(A, tA.p, (size_t)c->I * R * 8, cudaMemcpyDeviceToHost));
    if (B) CK(cudaMemcpy(B, tB.p, (size_t)c->J * R * 8, cudaMemcpyDeviceToHost));
    if (C) CK(cudaMemcpy(C, tC.p, (size_t)K * R * 8, cudaMemcpyDeviceToHost));
    if (fit) *fit = h[1] > 0.0 ? 1.0 - std::sqrt(h[0]) / std::sqrt(h[1]) : 0.0;
    return SBT_OK;
}

extern "C" sbt_status sbt_stats(const sbt_ctx *c, sbt_update_stats *st) {
    if (!c || !st) return fail(SBT_E_INVALID, "null argument");
    if (!c->have_last) return fail(SBT_E_STATE, "no update has run");
    *st = c->stats;
    return SBT_OK;
}

extern "C" sbt_status sbt_last_samples(const sbt_ctx *c, int32_t rep, int32_t mode, int32_t *out, int64_t cap,
                                       int64_t *n) {
    if (!c || !n) return fail(SBT_E_INVALID, "null argument");
    if (!c->have_last) return fail(SBT_E_STATE, "no update has run");
    if (rep < 0 || rep >= c->opt.r || mode < 0 || mode > 2) return fail(SBT_E_INVALID, "rep or mode out of range");
    DeviceGuard dg(c->device);
    const int cnt = mode == 0 ? c->last_nI : (mode == 1 ? c->last_nJ : c->last_nK);
    *n = cnt;
    if (out && cap > 0) {
        const int64_t w = std::min<int64_t>(cap, cnt);
        CK(cudaMemcpy(out, c->samples.as<int>() + (size_t)(rep * 3 + mode) * c->last_samp_stride, (size_t)w * 4,
                      cudaMemcpyDeviceToHost));
    }
    return SBT_OK;
}

static inline float bf16_bits_to_float(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

extern "C" sbt_status sbt_last_summary(const sbt_ctx *c, int32_t rep, double *out, int64_t cap, int64_t dims[3]) {
    if (!c || !dims) return fail(SBT_E_INVALID, "null argument");
    if (!c->have_last) return fail(SBT_E_STATE, "no update has run");
    if (c->coo) return fail(SBT_E_STATE, "COO summaries are lists of nonzeros, not dense arrays");
    if (rep < 0 || rep >= c->opt.r) return fail(SBT_E_INVALID, "rep out of range");
    DeviceGuard dg(c->device);
    const int nI = c->last_nI, nJ = c->last_nJ, Kp = c->last_nK + c->last_Knew, ldj = c->last_ldj;
    dims[0] = nI;
    dims[1] = nJ;
    dims[2] = Kp;
    const int64_t total = (int64_t)Kp * nI * nJ;
    if (!out) return SBT_OK;
    if (cap < total) return fail(SBT_E_INVALID, "output buffer too small");
    const size_t es = esize_elem(c->elem);
    const long long xrs = (long long)Kp * nI * ldj;
    std::vector<unsigned char> h((size_t)xrs * es);
    CK(cudaMemcpy(h.data(), c->Xs.as<unsigned char>() + (size_t)rep * xrs * es, (size_t)xrs * es,
                  cudaMemcpyDeviceToHost));
    std::vector<float> sc(c->elem == 3 ? Kp : 0);
    if (c->elem == 3)
        CK(cudaMemcpy(sc.data(), c->sscale.as<float>() + (size_t)rep * Kp, (size_t)Kp * 4, cudaMemcpyDeviceToHost));
    for (int64_t row = 0; row < (int64_t)Kp * nI; ++row)
        for (int jj = 0; jj < nJ; ++jj) {
            const size_t idx = (size_t)row * ldj + jj;
            double v;
            if (c->elem == 0) std::memcpy(&v, &h[idx * 8], 8);
            else if (c->elem == 1) {
                float f;
                std::memcpy(&f, &h[idx * 4], 4);
                v = f;
            } else if (c->elem == 2) {
                uint16_t b;
                std::memcpy(&b, &h[idx * 2], 2);
                v = bf16_bits_to_float(b);
            } else {
                v = e4m3_value(h[idx]) * (double)sc[row / nI];
            }
            out[row * nJ + jj] = v;
        }
    return SBT_OK;
}

extern "C" sbt_status sbt_last_summary_factors(const sbt_ctx *c, int32_t rep, double *lambda, double *A, double *B,
                                               double *C) {
    if (!c) return fail(SBT_E_INVALID, "null context");
    if (!c->have_last) return fail(SBT_E_STATE, "no update has run");
    if (rep < 0 || rep >= c->opt.r) return fail(SBT_E_INVALID, "rep out of range");
    DeviceGuard dg(c->device);
    const int R = c->R;
    const int n[3] = {c->last_nI, c->last_nJ, c->last_nK + c->last_Knew};
    std::vector<double> nu(3 * R), ls(R);
    CK(cudaMemcpy(nu.data(), c->nu.as<double>() + (size_t)rep * 3 * R, 3 * R * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(ls.data(), c->lam_s.as<double>() + (size_t)rep * R, R * 8, cudaMemcpyDeviceToHost));
    // the repetition's n x R slot holds rows of Rs values (Rs < R with GetRank)
    const int Rs = rep < (int)c->last_rank.size() ? c->last_rank[rep] : R;
    double *outs[3] = {A, B, C};
    for (int q = 0; q < 3; ++q) {
        if (!outs[q]) continue;
        const size_t slot = (size_t)n[q] * R, cnt = (size_t)n[q] * Rs;
        std::vector<double> v(cnt);
        if (c->elem == 0) {
            CK(cudaMemcpy(v.data(), c->U[q].as<double>() + (size_t)rep * slot, cnt * 8, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> f(cnt);
            CK(cudaMemcpy(f.data(), c->U[q].as<float>() + (size_t)rep * slot, cnt * 4, cudaMemcpyDeviceToHost));
            for (size_t e = 0; e < cnt; ++e) v[e] = f[e];
        }
        for (int x = 0; x < n[q]; ++x)
            for (int a = 0; a < R; ++a) outs[q][(size_t)x * R + a] = a < Rs ? v[(size_t)x * Rs + a] / nu[q * R + a] : 0.0;
    }
    if (lambda)
        for (int a = 0; a < R; ++a) lambda[a] = a < Rs ? ls[a] * nu[a] * nu[R + a] * nu[2 * R + a] : 0.0;
    return SBT_OK;
}

extern "C" sbt_status sbt_profile_reset(sbt_ctx *c, int32_t timing) {
    if (!c) return fail(SBT_E_INVALID, "null context");
    if (timing < 0 || timing > 2) return fail(SBT_E_INVALID, "timing must be 0, 1 or 2");
    DeviceGuard dg(c->device);
    CK(cudaStreamSynchronize(c->stream));
    settle_als_counts(c);
    CK(cudaMemsetAsync(c->prof_bytes.p, 0, 8, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->timing = timing;
    c->mtt_ms = 0.0;
    c->mtt_busy_ms = 0.0;
    c->mtt_launch_ms = 0.0;
    c->launch_base = launch_count();
    c->updates = 0;
    c->mtt_launches = 0;
    c->mtt_passes = 0;
    return SBT_OK;
}

extern "C" sbt_status sbt_profile_read(sbt_ctx *c, sbt_profile *out) {
    if (!c || !out) return fail(SBT_E_INVALID, "null argument");
    DeviceGuard dg(c->device);
    CK(cudaStreamSynchronize(c->stream));
    settle_als_counts(c);
    unsigned long long bytes = 0;
    CK(cudaMemcpy(&bytes, c->prof_bytes.p, 8, cudaMemcpyDeviceToHost));
    const double ms = c->mtt_ms;
    out->launches = launch_count() - c->launch_base;
    out->updates = c->updates;
    out->mttkrp_launches = c->mtt_launches;
    out->mttkrp_ms = ms;
    out->mttkrp_bytes = (double)bytes;
    out->mttkrp_passes = c->mtt_passes;
    out->mttkrp_busy_ms = c->mtt_busy_ms;
    out->mttkrp_launch_ms = c->mtt_launch_ms;
    return SBT_OK;
}

// ---------------------------------------------------------------------------
// COO tensors: the same method (Alg. 1) on a store of nonzeros grouped by
// time slice; the sparse workloads of Section 4.1.

static sbt_status check_coo(const sbt_coo *X) {
    if (!X) return fail(SBT_E_INVALID, "null tensor");
    if (X->I < 1 || X->J < 1 || X->K < 1) return fail(SBT_E_SHAPE, "tensor dimensions must be >= 1");
    if (X->I > INT32_MAX || X->J > INT32_MAX || X->K > (1 << 30)) return fail(SBT_E_SHAPE, "dimension too large");
    if (X->nnz < 0 || X->nnz > INT32_MAX) return fail(SBT_E_SHAPE, "nnz out of range");
    if (X->nnz > 0 && (!X->ii || !X->jj || !X->kk || !X->val)) return fail(SBT_E_INVALID, "null COO array");
    return SBT_OK;
}

// device arrays of a COO input: host arrays are copied to staging buffers
static sbt_status coo_device(sbt_ctx *c, const sbt_coo *X, const int **ii, const int **jj, const int **kk,
                             const float **v) {
    if (X->on_device || X->nnz == 0) {
        *ii = X->ii;
        *jj = X->jj;
        *kk = X->kk;
        *v = X->val;
        return SBT_OK;
    }
    const size_t n = (size_t)X->nnz;
    TRY(c->cin_i.ensure(n * 4));
    TRY(c->cin_j.ensure(n * 4));
    TRY(c->cin_k.ensure(n * 4));
    TRY(c->cin_v.ensure(n * 4));
    CK(cudaMemcpyAsync(c->cin_i.p, X->ii, n * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->cin_j.p, X->jj, n * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->cin_k.p, X->kk, n * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->cin_v.p, X->val, n * 4, cudaMemcpyHostToDevice, c->stream));
    *ii = c->cin_i.as<int>();
    *jj = c->cin_j.as<int>();
    *kk = c->cin_k.as<int>();
    *v = c->cin_v.as<float>();
    return SBT_OK;
}

// room for `need` stored nonzeros (doubling; the first nnz are kept)
static sbt_status coo_grow_nnz(sbt_ctx *c, int64_t need) {
    const int64_t cap = (int64_t)(c->sv.cap / 4);
    if (need <= cap && c->sv.p) return SBT_OK;
    const int64_t ncap = std::max<int64_t>(std::max<int64_t>(need, 2 * cap), 1024);
    Buf ni, nj, nv;
    TRY(ni.ensure((size_t)ncap * 4));
    TRY(nj.ensure((size_t)ncap * 4));
    TRY(nv.ensure((size_t)ncap * 4));
    if (c->nnz > 0) {
        CK(cudaMemcpyAsync(ni.p, c->si.p, (size_t)c->nnz * 4, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(nj.p, c->sj.p, (size_t)c->nnz * 4, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(nv.p, c->sv.p, (size_t)c->nnz * 4, cudaMemcpyDeviceToDevice, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    std::swap(c->si.p, ni.p);
    std::swap(c->si.cap, ni.cap);
    std::swap(c->sj.p, nj.p);
    std::swap(c->sj.cap, nj.cap);
    std::swap(c->sv.p, nv.p);
    std::swap(c->sv.cap, nv.cap);
    return SBT_OK;
}

// room for `need` slices: C, x_c and the slice offsets
static sbt_status coo_grow_slices(sbt_ctx *c, int64_t need) {
    if (need <= c->Kcap) return SBT_OK;
    const int64_t ncap = std::max<int64_t>(need, c->Kcap * 2);
    Buf nC, nxc, nsp;
    TRY(nC.ensure((size_t)ncap * c->R * 8));
    TRY(nxc.ensure((size_t)ncap * 8));
    TRY(nsp.ensure((size_t)(ncap + 1) * 8));
    CK(cudaMemsetAsync(nxc.p, 0, (size_t)ncap * 8, c->stream));
    CK(cudaMemcpyAsync(nC.p, c->C.p, (size_t)c->K * c->R * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(nxc.p, c->xc.p, (size_t)c->K * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(nsp.p, c->sptr.p, (size_t)(c->K + 1) * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::swap(c->C.p, nC.p);
    std::swap(c->C.cap, nC.cap);
    std::swap(c->xc.p, nxc.p);
    std::swap(c->xc.cap, nxc.cap);
    std::swap(c->sptr.p, nsp.p);
    std::swap(c->sptr.cap, nsp.cap);
    c->Kcap = ncap;
    return SBT_OK;
}

// Context of a COO tensor: the store of X0's nonzeros and its marginals (Eq. 1)
static sbt_status coo_begin(const sbt_coo *X0, int32_t R, const sbt_options *opt, sbt_ctx *c) {
    TRY(check_coo(X0));
    TRY(check_options(opt, R));
    if (opt->prec != SBT_PREC_F32)
        return fail(SBT_E_INVALID, "COO tensors take SBT_PREC_F32 (float32 values, fixed-point MTTKRP sums)");
    c->opt = *opt;
    c->coo = true;
    CK(cudaGetDevice(&c->device));
    CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    CK(ensure_kernel_attributes(c->device));
    c->user = (cudaStream_t)opt->cuda_stream;
    CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_user, cudaEventDisableTiming));
    TRY(order_after_user(c));
    c->I = (int)X0->I;
    c->J = (int)X0->J;
    c->R = R;
    c->K = X0->K;
    c->sdtype = SBT_F32;
    c->elem = 1;
    c->Kcap = std::max<int64_t>(opt->K_capacity > 0 ? opt->K_capacity : 2 * X0->K, X0->K + 1);
    TRY(c->A.ensure((size_t)c->I * R * 8));
    TRY(c->B.ensure((size_t)c->J * R * 8));
    TRY(c->C.ensure((size_t)c->Kcap * R * 8));
    TRY(c->lam.ensure((size_t)R * 8));
    TRY(c->xa.ensure((size_t)c->I * 8));
    TRY(c->xb.ensure((size_t)c->J * 8));
    TRY(c->xc.ensure((size_t)c->Kcap * 8));
    TRY(c->dxa.ensure((size_t)c->I * 8));
    TRY(c->dxb.ensure((size_t)c->J * 8));
    TRY(c->sptr.ensure((size_t)(c->Kcap + 1) * 8));
    TRY(c->status.ensure(sizeof(DevStatus)));
    TRY(c->h_status.ensure(sizeof(DevStatus)));
    TRY(c->prof_bytes.ensure(8));
    TRY(c->cmax.ensure(4));
    CK(cudaMemsetAsync(c->prof_bytes.p, 0, 8, c->stream));
    CK(cudaMemsetAsync(c->status.p, 0, sizeof(DevStatus), c->stream));
    CK(cudaMemsetAsync(c->xa.p, 0, (size_t)c->I * 8, c->stream));
    CK(cudaMemsetAsync(c->xb.p, 0, (size_t)c->J * 8, c->stream));
    CK(cudaMemsetAsync(c->xc.p, 0, (size_t)c->Kcap * 8, c->stream));
    CK(cudaMemsetAsync(c->cmax.p, 0, 4, c->stream));
    TRY(coo_grow_nnz(c, std::max<int64_t>(X0->nnz, 1)));
    const int *ii, *jj, *kk;
    const float *v;
    TRY(coo_device(c, X0, &ii, &jj, &kk, &v));
    // the shift S from max |x| (zeros do not matter), as for dense tensors
    CK(launch_abs_max_f(v, X0->nnz, c->cmax.as<unsigned>(), c->stream));
    unsigned mb = 0;
    CK(cudaMemcpyAsync(c->h_status.p, c->cmax.p, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::memcpy(&mb, c->h_status.p, 4);
    float mf;
    std::memcpy(&mf, &mb, 4);
    const double M = (double)mf;
    if (M == 0.0) {
        c->S = 0;
    } else {
        int e2;
        std::frexp(M * M, &e2);
        c->S = 32 - e2;
    }
    // nonzeros into the store by slice; marginals straight into x_a, x_b, x_c
    const int K = (int)c->K;
    TRY(c->ccnt.ensure((size_t)K * 4));
    TRY(c->cfill.ensure((size_t)K * 4));
    CK(cudaMemsetAsync(c->ccnt.p, 0, (size_t)K * 4, c->stream));
    CK(cudaMemsetAsync(c->cfill.p, 0, (size_t)K * 4, c->stream));
    CK(launch_coo_count(kk, X0->nnz, K, c->ccnt.as<int>(), c->status.as<DevStatus>(), c->stream));
    CK(launch_exscan(c->ccnt.as<int>(), 0, c->sptr.as<long long>(), 0, K, 1, 0, c->stream));
    CK(launch_coo_scatter(ii, jj, kk, v, X0->nnz, c->I, c->J, K, c->S, c->sptr.as<long long>(), c->cfill.as<int>(),
                          c->si.as<int>(), c->sj.as<int>(), c->sv.as<float>(), c->xa.as<unsigned long long>(),
                          c->xb.as<unsigned long long>(), c->xc.as<unsigned long long>(), c->status.as<DevStatus>(),
                          c->stream));
    DevStatus hs;
    TRY(read_status(c, &hs));
    TRY(status_error(hs.err));
    c->nnz = X0->nnz;
    std::vector<unsigned long long> h(std::max<int64_t>(std::max(c->I, c->J), c->K));
    const unsigned long long *src[3] = {c->xa.as<unsigned long long>(), c->xb.as<unsigned long long>(),
                                        c->xc.as<unsigned long long>()};
    const int64_t len[3] = {c->I, c->J, c->K};
    for (int m = 0; m < 3; ++m) {
        CK(cudaMemcpy(h.data(), src[m], (size_t)len[m] * 8, cudaMemcpyDeviceToHost));
        int64_t cnt = 0;
        for (int64_t x = 0; x < len[m]; ++x) cnt += h[x] != 0;
        c->npos[m] = cnt;
    }
    return SBT_OK;
}

// entries of every repetition grouped by ii (mode 1) and jj (mode 2), and the
// fixed-point exponents; the MTTKRP descriptor of the summaries
static sbt_status coo_groups(sbt_ctx *c, int nrep, int nI, int nJ, long long ecap, long long max_total,
                             const int *eii, const int *ejj) {
    TRY(c->gc1.ensure((size_t)nrep * (nI + 1) * 4));
    TRY(c->gc2.ensure((size_t)nrep * (nJ + 1) * 4));
    TRY(c->gf1.ensure((size_t)nrep * nI * 4));
    TRY(c->gf2.ensure((size_t)nrep * nJ * 4));
    TRY(c->rp1.ensure((size_t)nrep * (nI + 1) * 8));
    TRY(c->rp2.ensure((size_t)nrep * (nJ + 1) * 8));
    TRY(c->perm1.ensure((size_t)nrep * std::max(1LL, ecap) * 4));
    TRY(c->perm2.ensure((size_t)nrep * std::max(1LL, ecap) * 4));
    TRY(c->fexp.ensure((size_t)nrep * 4));
    CK(cudaMemsetAsync(c->gc1.p, 0, (size_t)nrep * (nI + 1) * 4, c->stream));
    CK(cudaMemsetAsync(c->gc2.p, 0, (size_t)nrep * (nJ + 1) * 4, c->stream));
    CK(cudaMemsetAsync(c->gf1.p, 0, (size_t)nrep * nI * 4, c->stream));
    CK(cudaMemsetAsync(c->gf2.p, 0, (size_t)nrep * nJ * 4, c->stream));
    const long long *tot = c->gtot.as<long long>();
    CK(launch_coo_group(eii, ecap, tot, max_total, nI, nrep, c->gc1.as<int>(), c->rp1.as<long long>(),
                        c->gf1.as<int>(), c->perm1.as<int>(), c->stream));
    CK(launch_coo_group(ejj, ecap, tot, max_total, nJ, nrep, c->gc2.as<int>(), c->rp2.as<long long>(),
                        c->gf2.as<int>(), c->perm2.as<int>(), c->stream));
    CK(launch_coo_fexp(c->vmax.as<unsigned>(), tot, nrep, c->fexp.as<int>(), c->stream));
    return SBT_OK;
}

// ALS descriptor of COO summaries: one partial per mode (the MTTKRP writes
// whole rows)
static void coo_partials(AlsDesc &d) {
    d.P[0] = d.P[1] = d.P[2] = 1;
    d.prs = (long long)std::max(d.n[0], std::max(d.n[1], d.n[2])) * d.pr;
}

// CP-ALS of the whole stored tensor (the identity summary), or nothing when
// the factors are given
static sbt_status coo_init_als(sbt_ctx *c) {
    const int K = (int)c->K;
    const long long nnz = c->nnz;
    TRY(c->ekk.ensure((size_t)std::max(1LL, nnz) * 4));
    CK(launch_coo_expand_k(c->sptr.as<long long>(), K, c->ekk.as<int>(), c->stream));
    TRY(c->gtot.ensure(8));
    TRY(c->vmax.ensure(4));
    CK(cudaMemcpy(c->gtot.p, &nnz, 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpyAsync(c->vmax.p, c->cmax.p, 4, cudaMemcpyDeviceToDevice, c->stream));
    TRY(coo_groups(c, 1, c->I, c->J, nnz, nnz, c->si.as<int>(), c->sj.as<int>()));
    c->cd = CooDesc{nnz, c->si.as<int>(), c->sj.as<int>(), c->ekk.as<int>(), c->sv.as<float>(),
                    c->sptr.as<long long>(), c->rp1.as<long long>(), c->rp2.as<long long>(), c->perm1.as<int>(),
                    c->perm2.as<int>(), c->fexp.as<int>()};
    AlsDesc d;
    const int n[3] = {c->I, c->J, K};
    TRY(setup_als(c, d, 1, n, 0, K, 1, nullptr, 0, c->opt.max_iters_init));
    coo_partials(d);
    d.rq_rows = K;
    // ||X||^2 per slice from the exact marginals: x_c(k) 2^-S
    std::vector<unsigned long long> hx(K);
    CK(cudaMemcpy(hx.data(), c->xc.p, (size_t)K * 8, cudaMemcpyDeviceToHost));
    std::vector<double> rq(K);
    for (int k = 0; k < K; ++k) rq[k] = std::ldexp((double)hx[k], -c->S);
    TRY(c->rowsq.ensure((size_t)K * 8));
    CK(cudaMemcpy(c->rowsq.p, rq.data(), (size_t)K * 8, cudaMemcpyHostToDevice));
    CK(launch_als_prepare(d, nullptr, 0, K, true, c->opt.seed, c->opt.stream_id, 0xFFFFFFFFu, c->rowsq.as<double>(),
                          c->stream));
    TRY(run_als(c, d, c->opt.max_iters_init));
    CK(launch_canonicalize(d, c->A.as<double>(), c->B.as<double>(), c->C.as<double>(), c->lam.as<double>(),
                           c->stream));
    CK(cudaStreamSynchronize(c->stream));
    settle_als_counts(c);
    return SBT_OK;
}

extern "C" sbt_status sbt_init_coo(const sbt_coo *X0, int32_t R, const sbt_options *opt, sbt_ctx **out) {
    if (!out) return fail(SBT_E_INVALID, "null output pointer");
    *out = nullptr;
    sbt_ctx *c = new sbt_ctx();
    sbt_status s = coo_begin(X0, R, opt, c);
    if (s == SBT_OK) s = coo_init_als(c);
    if (s != SBT_OK) {
        delete c;
        return s;
    }
    *out = c;
    return SBT_OK;
}

extern "C" sbt_status sbt_init_coo_factors(const sbt_coo *X0, int32_t R, const double *lambda, const double *A,
                                           const double *B, const double *C, const sbt_options *opt, sbt_ctx **out) {
    if (!out) return fail(SBT_E_INVALID, "null output pointer");
    *out = nullptr;
    if (!lambda || !A || !B || !C) return fail(SBT_E_INVALID, "null factor pointer");
    sbt_ctx *c = new sbt_ctx();
    sbt_status s = coo_begin(X0, R, opt, c);
    if (s == SBT_OK) {
        cudaError_t e = cudaMemcpy(c->A.p, A, (size_t)c->I * R * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->B.p, B, (size_t)c->J * R * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->C.p, C, (size_t)c->K * R * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->lam.p, lambda, (size_t)R * 8, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) s = fail(SBT_E_CUDA, std::string("factor upload: ") + cudaGetErrorString(e));
    }
    if (s != SBT_OK) {
        delete c;
        return s;
    }
    *out = c;
    return SBT_OK;
}

extern "C" sbt_status sbt_update_coo(sbt_ctx *c, const sbt_coo *X) {
    if (!c) return fail(SBT_E_INVALID, "null context");
    if (!c->coo) return fail(SBT_E_INVALID, "not a COO context (sbt_update takes dense slices)");
    if (c->opt.get_rank) return fail(SBT_E_INVALID, "get_rank takes dense contexts");
    TRY(check_coo(X));
    if (X->I != c->I || X->J != c->J) return fail(SBT_E_SHAPE, "I and J must match the initial tensor");
    DeviceGuard dg(c->device);
    TRY(order_after_user(c));
    const int R = c->R, r = c->opt.r;
    const int K_new = (int)X->K;
    const int64_t K_old = c->K;
    // sample sizes (Section 3.1): ceil(N / s), clamped to the positive weights
    const int nI = (int)std::min<int64_t>(ceil_div(c->I, c->opt.s_I), c->npos[0]);
    const int nJ = (int)std::min<int64_t>(ceil_div(c->J, c->opt.s_J), c->npos[1]);
    const int nK = (int)std::min<int64_t>(ceil_div(K_old, c->opt.s_K), c->npos[2]);
    if (nI < 1 || nJ < 1 || nK < 1) return fail(SBT_E_STATE, "a mode has no positive weight to sample");
    const int Kp = nK + K_new;
    const long long samp_stride = std::max(nI, std::max(nJ, nK));
    const long long key_stride = std::max<int64_t>(std::max(c->I, c->J), K_old);
    TRY(coo_grow_slices(c, K_old + K_new));
    TRY(coo_grow_nnz(c, c->nnz + X->nnz));
    const int *ii, *jj, *kk;
    const float *v;
    TRY(coo_device(c, X, &ii, &jj, &kk, &v));
    TRY(c->samples.ensure((size_t)r * 3 * samp_stride * 4));
    TRY(c->khi.ensure((size_t)r * 3 * key_stride * 8));
    TRY(c->klo.ensure((size_t)r * 3 * key_stride * 8));
    TRY(c->xc_new.ensure((size_t)K_new * 8));
    TRY(c->ccnt.ensure((size_t)K_new * 4));
    TRY(c->cfill.ensure((size_t)K_new * 4));
    // 1. append the nonzeros and their marginal deltas
    CK(cudaMemsetAsync(c->status.p, 0, sizeof(DevStatus), c->stream));
    CK(cudaMemsetAsync(c->dxa.p, 0, (size_t)c->I * 8, c->stream));
    CK(cudaMemsetAsync(c->dxb.p, 0, (size_t)c->J * 8, c->stream));
    CK(cudaMemsetAsync(c->xc_new.p, 0, (size_t)K_new * 8, c->stream));
    CK(cudaMemsetAsync(c->ccnt.p, 0, (size_t)K_new * 4, c->stream));
    CK(cudaMemsetAsync(c->cfill.p, 0, (size_t)K_new * 4, c->stream));
    long long *sptr_new = c->sptr.as<long long>() + K_old;
    CK(launch_coo_count(kk, X->nnz, K_new, c->ccnt.as<int>(), c->status.as<DevStatus>(), c->stream));
    CK(launch_exscan(c->ccnt.as<int>(), 0, sptr_new, 0, K_new, 1, c->nnz, c->stream));
    CK(launch_coo_scatter(ii, jj, kk, v, X->nnz, c->I, c->J, K_new, c->S, sptr_new, c->cfill.as<int>(),
                          c->si.as<int>(), c->sj.as<int>(), c->sv.as<float>(), c->dxa.as<unsigned long long>(),
                          c->dxb.as<unsigned long long>(), c->xc_new.as<unsigned long long>(),
                          c->status.as<DevStatus>(), c->stream));
    // 2. sampling from the marginals of the tensor before the update
    SampleParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.w[0] = c->xa.as<unsigned long long>();
    sp.w[1] = c->xb.as<unsigned long long>();
    sp.w[2] = c->xc.as<unsigned long long>();
    sp.N[0] = c->I;
    sp.N[1] = c->J;
    sp.N[2] = (int)K_old;
    sp.n[0] = nI;
    sp.n[1] = nJ;
    sp.n[2] = nK;
    sp.mode_id[0] = 0;
    sp.mode_id[1] = 1;
    sp.mode_id[2] = 2;
    sp.nmodes = 3;
    sp.nrep = r;
    sp.out = c->samples.as<int>();
    sp.out_stride = samp_stride;
    sp.khi = c->khi.as<unsigned long long>();
    sp.klo = c->klo.as<unsigned long long>();
    sp.key_stride = key_stride;
    sp.seed = c->opt.seed;
    sp.stream_id = c->opt.stream_id;
    sp.batch = c->batch;
    sp.status = c->status.as<DevStatus>();
    CK(launch_sample(sp, c->stream));
    // 3. the summaries: sampled nonzeros of the sampled and the new slices
    TRY(c->posI.ensure((size_t)r * c->I * 4));
    TRY(c->posJ.ensure((size_t)r * c->J * 4));
    CK(cudaMemsetAsync(c->posI.p, 0xFF, (size_t)r * c->I * 4, c->stream));
    CK(cudaMemsetAsync(c->posJ.p, 0xFF, (size_t)r * c->J * 4, c->stream));
    CK(launch_coo_pos(c->samples.as<int>(), samp_stride, nI, nJ, c->I, c->J, r, c->posI.as<int>(), c->posJ.as<int>(),
                      c->stream));
    TRY(c->gcnt.ensure((size_t)r * (Kp + 1) * 4));
    TRY(c->goff.ensure((size_t)r * (Kp + 1) * 8));
    TRY(c->gtot.ensure((size_t)r * 8));
    TRY(c->vmax.ensure((size_t)r * 4));
    TRY(c->rowsq.ensure((size_t)r * Kp * 8));
    CK(cudaMemsetAsync(c->gcnt.p, 0, (size_t)r * (Kp + 1) * 4, c->stream));
    CK(cudaMemsetAsync(c->vmax.p, 0, (size_t)r * 4, c->stream));
    CooGather g;
    std::memset(&g, 0, sizeof(g));
    g.si = c->si.as<int>();
    g.sj = c->sj.as<int>();
    g.sv = c->sv.as<float>();
    g.sptr = c->sptr.as<long long>();
    g.samples = c->samples.as<int>();
    g.samp_stride = samp_stride;
    g.posI = c->posI.as<int>();
    g.posJ = c->posJ.as<int>();
    g.I = c->I;
    g.J = c->J;
    g.nK = nK;
    g.K_old = (int)K_old;
    g.K_new = K_new;
    g.nrep = r;
    g.S = c->S;
    g.cnt = c->gcnt.as<int>();
    g.off = c->goff.as<long long>();
    g.rowsq = c->rowsq.as<double>();
    g.vmax = c->vmax.as<unsigned>();
    CK(launch_coo_gather(g, 0, c->stream));
    CK(launch_exscan(c->gcnt.as<int>(), Kp + 1, c->goff.as<long long>(), Kp + 1, Kp, r, 0, c->stream));
    CK(cudaMemcpy2DAsync(c->gtot.p, 8, c->goff.as<long long>() + Kp, (size_t)(Kp + 1) * 8, 8, r,
                         cudaMemcpyDeviceToDevice, c->stream));
    TRY(c->h_tot.ensure((size_t)r * 8));
    CK(cudaMemcpyAsync(c->h_tot.p, c->gtot.p, (size_t)r * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    long long max_total = 0;
    for (int q = 0; q < r; ++q) max_total = std::max(max_total, c->h_tot.as<long long>()[q]);
    const long long ecap = std::max(1LL, max_total);
    TRY(c->eii.ensure((size_t)r * ecap * 4));
    TRY(c->ejj.ensure((size_t)r * ecap * 4));
    TRY(c->ekk.ensure((size_t)r * ecap * 4));
    TRY(c->ev.ensure((size_t)r * ecap * 4));
    g.ecap = ecap;
    g.eii = c->eii.as<int>();
    g.ejj = c->ejj.as<int>();
    g.ekk = c->ekk.as<int>();
    g.ev = c->ev.as<float>();
    CK(launch_coo_gather(g, 1, c->stream));
    TRY(coo_groups(c, r, nI, nJ, ecap, max_total, c->eii.as<int>(), c->ejj.as<int>()));
    c->cd = CooDesc{ecap, c->eii.as<int>(), c->ejj.as<int>(), c->ekk.as<int>(), c->ev.as<float>(),
                    c->goff.as<long long>(), c->rp1.as<long long>(), c->rp2.as<long long>(), c->perm1.as<int>(),
                    c->perm2.as<int>(), c->fexp.as<int>()};
    // 4. CP-ALS on the r summaries
    AlsDesc d;
    const int n[3] = {nI, nJ, Kp};
    als_shape(c, d, r, n, 0, nK, 1, c->opt.max_iters);
    {
        Sizer z;
        TRY(als_sizes(c, d, (size_t)r * std::max(nI, std::max(nJ, Kp)) * d.pr * 4 + (size_t)r * d.prs * 4, z));
    }
    TRY(als_bind(c, d, nullptr, 0));
    coo_partials(d);
    d.rq_rows = Kp;
    CK(launch_als_prepare(d, c->samples.as<int>(), samp_stride, (int)K_old, false, c->opt.seed, c->opt.stream_id,
                          c->batch, c->rowsq.as<double>(), c->stream, warm_start_of(c)));
    TRY(run_als(c, d, c->opt.max_iters));
    // 5-6. normalise, match, project back, commit
    const size_t pmax = (size_t)samp_stride;
    TRY(c->nu.ensure((size_t)r * 3 * R * 8));
    TRY(c->cnew.ensure((size_t)r * K_new * R * 8));
    TRY(c->prop.ensure((size_t)r * 3 * pmax * R * 8));
    TRY(c->lam_est.ensure((size_t)r * R * 8));
    TRY(c->perm.ensure((size_t)r * R * 4));
    TRY(c->min_score.ensure((size_t)r * 8));
    TRY(c->mdots.ensure((size_t)r * 3 * (32 * 32 + 64) * 8));
    const int64_t nnz_in = X->nnz;
    TRY(match_commit(c, d, K_old, K_new, nI, nJ, nK, samp_stride, 0, false, false));
    c->nnz += nnz_in;
    return SBT_OK;
}

// Full-tensor fit of a COO context: ||X||^2 from the exact marginals,
// ||X_hat||^2 from the Grams, <X, X_hat> over the nonzeros in fixed point.
static sbt_status coo_fit(sbt_ctx *c, double *fit) {
    const int R = c->R, I = c->I, J = c->J, K = (int)c->K;
    std::vector<double> lam(R), A((size_t)I * R), B((size_t)J * R), C((size_t)K * R);
    std::vector<unsigned long long> xc(K);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(lam.data(), c->lam.p, (size_t)R * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(A.data(), c->A.p, A.size() * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(B.data(), c->B.p, B.size() * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(C.data(), c->C.p, C.size() * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(xc.data(), c->xc.p, (size_t)K * 8, cudaMemcpyDeviceToHost));
    double nx2 = 0.0;
    for (int k = 0; k < K; ++k) nx2 += std::ldexp((double)xc[k], -c->S);
    auto gram = [R](const std::vector<double> &U, int n) {
        std::vector<double> G((size_t)R * R, 0.0);
        for (int x = 0; x < n; ++x)
            for (int a = 0; a < R; ++a)
                for (int b = 0; b < R; ++b) G[a * R + b] += U[(size_t)x * R + a] * U[(size_t)x * R + b];
        return G;
    };
    const std::vector<double> GA = gram(A, I), GB = gram(B, J), GC = gram(C, K);
    double nh2 = 0.0;
    for (int a = 0; a < R; ++a)
        for (int b = 0; b < R; ++b) nh2 += lam[a] * lam[b] * GA[a * R + b] * GB[a * R + b] * GC[a * R + b];
    // a bound on |v * model| over the nonzeros picks the fixed-point exponent
    auto colmax = [R](const std::vector<double> &U, int r) {
        double m = 0.0;
        for (size_t x = r; x < U.size(); x += R) m = std::max(m, std::fabs(U[x]));
        return m;
    };
    double mb = 0.0;
    for (int a = 0; a < R; ++a) mb += std::fabs(lam[a]) * colmax(A, a) * colmax(B, a) * colmax(C, a);
    CK(cudaMemsetAsync(c->cmax.p, 0, 4, c->stream));
    CK(launch_abs_max_f(c->sv.as<float>(), c->nnz, c->cmax.as<unsigned>(), c->stream));
    unsigned vb = 0;
    CK(cudaMemcpyAsync(c->h_status.p, c->cmax.p, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::memcpy(&vb, c->h_status.p, 4);
    float vf;
    std::memcpy(&vf, &vb, 4);
    int e2 = 0;
    std::frexp((double)vf * mb * (double)std::max<int64_t>(1, c->nnz) + 1.0, &e2);
    const int F = std::max(0, std::min(100, 61 - e2));
    TRY(c->fitscr.ensure(16));
    CK(cudaMemsetAsync(c->fitscr.p, 0, 8, c->stream));
    CK(launch_coo_inner(c->si.as<int>(), c->sj.as<int>(), c->sv.as<float>(), c->sptr.as<long long>(), K,
                        c->A.as<double>(), c->B.as<double>(), c->C.as<double>(), c->lam.as<double>(), R, F,
                        c->fitscr.as<unsigned long long>(), c->stream));
    unsigned long long acc = 0;
    CK(cudaMemcpyAsync(c->h_status.p, c->fitscr.p, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::memcpy(&acc, c->h_status.p, 8);
    const double inner = std::ldexp((double)(long long)acc, -F);
    const double resid2 = std::max(nx2 + nh2 - 2.0 * inner, 0.0);
    *fit = nx2 > 0.0 ? 1.0 - std::sqrt(resid2) / std::sqrt(nx2) : 0.0;
    return SBT_OK;
}

extern "C" void sbt_destroy(sbt_ctx *c) {
    if (!c) return;
    {
        DeviceGuard dg(c->device);
        cudaStreamSynchronize(c->stream);
        delete c;
    }
}

// ---------------------------------------------------------------------------
// device-level operations
extern "C" sbt_status sbt_philox4x32_10(const uint32_t *ctr, uint32_t key0, uint32_t key1, uint32_t *out, int64_t n,
                                        void *stream) {
    if (n < 0 || (n > 0 && (!ctr || !out))) return fail(SBT_E_INVALID, "bad arguments");
    CK(launch_philox(ctr, make_uint2(key0, key1), out, n, (cudaStream_t)stream));
    return SBT_OK;
}

extern "C" sbt_status sbt_sample(const uint64_t *w, int64_t N, int64_t n, uint64_t seed, uint32_t stream_id,
                                 int32_t mode, int32_t rep, uint32_t batch, int32_t *out, void *stream) {
    if (!w || !out || N < 1 || n < 0 || n > N || N > (1 << 30)) return fail(SBT_E_INVALID, "bad arguments");
    if (mode < 0 || mode > 15 || rep < 0) return fail(SBT_E_INVALID, "mode or rep out of range");
    cudaStream_t st = (cudaStream_t)stream;
    void *scr = nullptr;
    const size_t bytes = (size_t)N * 16 + sizeof(DevStatus);
    CK(cudaMallocAsync(&scr, bytes, st));
    DevStatus *ds = (DevStatus *)((char *)scr + (size_t)N * 16);
    cudaError_t e = cudaMemsetAsync(ds, 0, sizeof(DevStatus), st);
    SampleParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.w[0] = (const unsigned long long *)w;
    sp.N[0] = (int)N;
    sp.n[0] = (int)n;
    sp.mode_id[0] = mode;
    sp.nmodes = 1;
    sp.nrep = 1;
    sp.rep0 = rep;
    sp.out = out;
    sp.out_stride = n;
    sp.khi = (unsigned long long *)scr;
    sp.klo = (unsigned long long *)scr + N;
    sp.key_stride = N;
    sp.seed = seed;
    sp.stream_id = stream_id;
    sp.batch = batch;
    sp.status = ds;
    if (e == cudaSuccess) e = launch_sample(sp, st);
    unsigned herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, &ds->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(scr, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SBT_E_CUDA, std::string("sbt_sample: ") + cudaGetErrorString(e));
    if (herr & ERR_SAMPLE) return fail(SBT_E_INVALID, "sample size above the number of positive weights");
    return SBT_OK;
}

static sbt_status mttkrp_bf16_op(const void *X, int64_t K, int64_t I, int64_t J, int64_t ld, const void *A,
                                 const void *B, const void *C, int32_t R, int32_t mode, void *M, cudaStream_t st) {
    const int NP = (int)(mode == 1 ? J : I), NC = (int)(mode == 1 ? I : J);
    if (!tc_supported(R, NC, false)) return fail(SBT_E_INVALID, "R or the contraction length exceeds the tensor-core plan");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    AlsDesc d;
    std::memset(&d, 0, sizeof(d));
    d.nrep = 1;
    d.R = R;
    d.n[0] = (int)I;
    d.n[1] = (int)J;
    d.n[2] = (int)K;
    d.elem = 2;
    d.pr = R;
    int npb, nks, spc;
    tc_plan(false, R, 1, NP, NC, (int)K, mode == 2 ? 1 : 0, sms, &npb, &nks, &spc);
    const int P = mode == 2 ? npb : nks;
    d.P[mode] = P;
    d.prs = (long long)P * (mode == 2 ? K : NP) * R;
    d.mrs = (long long)std::max(I, std::max(J, K)) * R;
    const int ldi = round8(I);
    const size_t xt_bytes = mode == 1 ? (size_t)K * J * ldi * 2 : 0;
    const size_t off_m = 256, off_part = off_m + (size_t)d.mrs * 8, off_xt = (off_part + (size_t)d.prs * 4 + 255) / 256 * 256;
    char *scr = nullptr;
    CK(cudaMallocAsync((void **)&scr, off_xt + xt_bytes + 256, st));
    d.conv = (int *)scr;
    unsigned *err = (unsigned *)(scr + 64);
    d.M = (double *)(scr + off_m);
    d.part = scr + off_part;
    cudaError_t e = cudaMemsetAsync(scr, 0, 256, st);
    CUtensorMap map;
    int Pk = 0;
    if (e == cudaSuccess) {
        if (mode == 1) {
            e = launch_transpose_bf16(X, scr + off_xt, (int)I, (int)J, (int)ld, ldi, K, st);
            if (e == cudaSuccess) e = make_summary_tmap(&map, scr + off_xt, (int)I, (int)J, ldi, K, false);
        } else {
            e = make_summary_tmap(&map, X, (int)J, (int)I, (int)ld, K, false);
        }
    }
    if (e == cudaSuccess) {
        if (mode == 0)
            e = launch_mttkrp_tc(map, nullptr, 0, 1, R, (int)I, (int)J, (int)K, (const float *)B, 0, (const float *)C, 0,
                                 (float *)d.part, d.prs, d.pr, d.conv, nullptr, err, nullptr, sms, &Pk, st);
        else if (mode == 1)
            e = launch_mttkrp_tc(map, nullptr, 0, 1, R, (int)J, (int)I, (int)K, (const float *)A, 0, (const float *)C, 0,
                                 (float *)d.part, d.prs, d.pr, d.conv, nullptr, err, nullptr, sms, &Pk, st);
        else
            e = launch_mttkrp_tc(map, nullptr, 1, 1, R, (int)I, (int)J, (int)K, (const float *)B, 0, (const float *)A, 0,
                                 (float *)d.part, d.prs, d.pr, d.conv, nullptr, err, nullptr, sms, &Pk, st);
    }
    if (e == cudaSuccess) e = launch_reduce_only(d, mode, st);
    if (e == cudaSuccess) e = launch_store_m(d, mode, M, st);
    unsigned herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st);
    cudaError_t e2 = cudaFreeAsync(scr, st);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SBT_E_CUDA, std::string("sbt_mttkrp (bf16): ") + cudaGetErrorString(e));
    if (herr) return fail(SBT_E_TIMEOUT, "sbt_mttkrp (bf16): a bounded device wait gave up");
    return SBT_OK;
}

extern "C" sbt_status sbt_core_consistency(int32_t dtype, const void *X, int64_t K, int64_t I, int64_t J,
                                           int64_t ld, const double *lambda, const double *A, const double *B,
                                           const double *C, int32_t R, double *cc, void *stream) {
    if (!X || !lambda || !A || !B || !C || !cc) return fail(SBT_E_INVALID, "null pointer");
    if (dtype != SBT_F64 && dtype != SBT_F32) return fail(SBT_E_INVALID, "dtype must be SBT_F64 or SBT_F32");
    if (R < 1 || R > SBT_MAX_RANK) return fail(SBT_E_INVALID, "R out of range [1, SBT_MAX_RANK]");
    if (K < R || I < R || J < R || ld < J) return fail(SBT_E_SHAPE, "need K, I, J >= R and ld >= J");
    if (K > (1 << 30) || I > (1 << 30) || J > (1 << 30)) return fail(SBT_E_SHAPE, "dimension too large");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nd = core_consistency_scratch_doubles(K, I, J, R);
    char *scr = nullptr;
    CK(cudaMallocAsync((void **)&scr, 16 + (nd + 1) * sizeof(double), st));
    int *status = (int *)scr;
    double *out = (double *)(scr + 8), *scratch = out + 1;
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = launch_core_consistency(dtype == SBT_F64 ? 0 : 1, X, K, I, J, ld, lambda, A, B, C, R, scratch, status,
                                    out, st);
    double h_out = 0.0;
    int h_status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_out, out, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t ef = cudaFreeAsync(scr, st);
    if (e == cudaSuccess) e = ef;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SBT_E_CUDA, std::string("core consistency: ") + cudaGetErrorString(e));
    if (h_status) return fail(SBT_E_STATE, "a factor's Gram is not positive definite");
    *cc = h_out;
    return SBT_OK;
}

extern "C" sbt_status sbt_mttkrp(int32_t dtype, const void *X, int64_t K, int64_t I, int64_t J, int64_t ld,
                                 const void *A, const void *B, const void *C, int32_t R, int32_t mode, void *M,
                                 void *stream) {
    if (!X || !A || !B || !C || !M) return fail(SBT_E_INVALID, "null pointer");
    if (dtype != SBT_F64 && dtype != SBT_F32 && dtype != SBT_BF16)
        return fail(SBT_E_INVALID, "dtype must be SBT_F64, SBT_F32 or SBT_BF16");
    if (K < 1 || I < 1 || J < 1 || ld < J || ld % 8 != 0) return fail(SBT_E_SHAPE, "need K, I, J >= 1 and ld >= J, ld % 8 == 0");
    if (((uintptr_t)X) % 16 != 0) return fail(SBT_E_INVALID, "X must be 16-byte aligned");
    if (R < 1 || R > SBT_MAX_RANK || mode < 0 || mode > 2) return fail(SBT_E_INVALID, "R or mode out of range");
    if (K > (1 << 30) || I > (1 << 30) || J > (1 << 30)) return fail(SBT_E_SHAPE, "dimension too large");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(ensure_kernel_attributes(dev));
    if (dtype == SBT_BF16) return mttkrp_bf16_op(X, K, I, J, ld, A, B, C, R, mode, M, st);
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    AlsDesc d;
    std::memset(&d, 0, sizeof(d));
    d.nrep = 1;
    d.R = R;
    d.n[0] = (int)I;
    d.n[1] = (int)J;
    d.n[2] = (int)K;
    d.ldj = (int)ld;
    d.nK = (int)K;
    d.elem = dtype == SBT_F64 ? 0 : 1;
    d.pr = R;
    d.X = X;
    d.xrs = 0;
    d.U[0] = (void *)A;
    d.U[1] = (void *)B;
    d.U[2] = (void *)C;
    choose_tiles(d, sms);
    d.prs = partial_elems(d);
    const int nmax = (int)std::max(I, std::max(J, K));
    d.mrs = (long long)nmax * R;
    const size_t tfs = dtype == SBT_F64 ? 8 : 4;
    const size_t bytes = 256 + (size_t)d.prs * tfs + (size_t)d.mrs * 8 + 256;
    char *scr = nullptr;
    CK(cudaMallocAsync((void **)&scr, bytes, st));
    d.conv = (int *)scr;
    d.M = (double *)(scr + 256);
    d.part = scr + 256 + (size_t)d.mrs * 8;
    cudaError_t e = cudaMemsetAsync(scr, 0, 256, st);
    if (e == cudaSuccess) e = launch_mttkrp_op(d, mode, M, st);
    cudaError_t e2 = cudaFreeAsync(scr, st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail(SBT_E_CUDA, std::string("sbt_mttkrp: ") + cudaGetErrorString(e));
    return SBT_OK;
}
