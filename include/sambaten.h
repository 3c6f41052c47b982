/*
 * sambaten.h -- C ABI of a GB300-native (sm_103a) batch-incremental CP update,
 * after SamBaTen: "Sampling-based Batch Incremental Tensor Decomposition"
 * (Gujral, Pasricha, Papalexakis; arxiv 1709.00668).
 *
 * The calls follow the paper's problem statement (Section 2.2): given a CP
 * decomposition A, B, C, lambda of an I x J x K1 tensor and a batch of K2 new
 * slices along the third (time) mode, return A, B and a C with K1 + K2 rows.
 * One sbt_update runs Algorithm 1 once on the GPU: sample each mode by its
 * measure of importance (Eq. 1), gather r summaries, CP-ALS each summary,
 * normalise over the shared rows, match components (Lemma 1), project back and
 * append the averaged new rows of C.
 *
 * Conventions shared by every call:
 *   - Every call returns an sbt_status; SBT_OK is 0.  On any error a message
 *     is available from sbt_last_error() (thread-local).
 *   - Dense tensors are slice-major: element (i, j, k) of an I x J x K tensor
 *     sits at data[(k * I + i) * J + j] (k is the time mode).
 *   - Factor matrices are row-major n x R doubles: U[x * R + r].
 *   - Input buffers are borrowed for the duration of the call and copied; the
 *     caller keeps ownership.  on_device = 1 means the pointer is device memory
 *     of the context's device, ordered on the context's CUDA stream.  Host
 *     input in page-locked (pinned) memory is read by the device in place
 *     during the call; pageable host input is copied first.
 *   - Output buffers are caller-owned host memory unless stated otherwise.
 *   - R <= SBT_MAX_RANK, r <= SBT_MAX_REPS.
 *   - Everything computes on the GPU; there is no CPU fallback.  A missing
 *     GPU or a CUDA failure is reported as SBT_E_CUDA.
 */
#ifndef SAMBATEN_H
#define SAMBATEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SBT_MAX_RANK 32
#define SBT_MAX_REPS 64

typedef struct sbt_ctx sbt_ctx; /* opaque; owned by the library */

typedef enum {
    SBT_OK = 0,
    SBT_E_INVALID = 1,   /* bad argument (null pointer, out-of-range option) */
    SBT_E_SHAPE = 2,     /* shape mismatch (I, J differ from init; K_new < 1) */
    SBT_E_NOMEM = 3,     /* device allocation failed */
    SBT_E_CUDA = 4,      /* CUDA runtime error or no usable device */
    SBT_E_NONFINITE = 5, /* the new slices hold NaN or Inf; state unchanged */
    SBT_E_RANGE = 6,     /* a fixed-point marginal would overflow 64 bits; state unchanged */
    SBT_E_TIMEOUT = 7,   /* a bounded device wait gave up */
    SBT_E_STATE = 8      /* call not valid in the context's current state */
} sbt_status;

/* Storage type of X.  SBT_BF16 is accepted by sbt_mttkrp only. */
typedef enum { SBT_F64 = 0, SBT_F32 = 1, SBT_BF16 = 2 } sbt_dtype;

/* Arithmetic of the summary ALS.  F64: float64 throughout (needs an F64
 * store), the R x R solve by a float64 Cholesky factorisation.  F32: float32
 * values, float32 accumulation.  BF16: summary rounded to bfloat16
 * (nearest-even), tensor-core MTTKRP with float32 accumulation.  FP8: float8
 * e4m3 codes with one scale per stored slice (scale = max|x| of the slice /
 * 448, code = e4m3(x * 448 / max|x|), ties to even, saturating; needs
 * R <= 32).  For F32, BF16 and FP8 the R x R work (Grams, V^-1, column norms,
 * the fit) runs in double-float, pairs of floats with ~44 significant bits,
 * float64 being a slow unit on this GPU. */
typedef enum { SBT_PREC_F64 = 0, SBT_PREC_F32 = 1, SBT_PREC_BF16 = 2, SBT_PREC_FP8 = 3 } sbt_prec;

/* Update flags (sbt_update_stats.flags), OR-ed over repetitions. */
#define SBT_FLAG_CHOL_REGULARIZED 1 /* a Gram Hadamard product was not positive definite */
#define SBT_FLAG_ZERO_COLUMN 2      /* a factor column had zero norm */
#define SBT_FLAG_SAMPLE_LT_RANK 4   /* a sample had fewer indices than R */
#define SBT_FLAG_NO_REFINE 8        /* refine_sweeps requested but not run (no tensor-core plan) */

typedef struct {
    int32_t dtype;     /* sbt_dtype of data */
    int32_t on_device; /* 1: data is device memory; 0: host memory */
    int64_t I, J, K;   /* dense, slice-major */
    const void *data;
} sbt_tensor;

typedef struct {
    int32_t s_I, s_J, s_K; /* sampling factors: a sample keeps ceil(N/s) indices (Section 3.1) */
    int32_t r;             /* repetitions (independent summaries per batch) */
    double tol;            /* ALS stops when |fit - previous fit| < tol */
    int32_t max_iters;     /* ALS iteration cap per summary */
    int32_t max_iters_init;/* ALS iteration cap of sbt_init */
    uint64_t seed;         /* Philox key (low and high words) */
    uint32_t stream_id;    /* xor-ed into the Philox key's high word */
    int32_t prec;          /* sbt_prec of the summary MTTKRP */
    int32_t lambda_mode;   /* 0: keep lambda; 1: average with the summaries' estimate (Alg. 1 step 13) */
    int32_t fixed_iters;   /* 1: ignore tol, run exactly max_iters iterations (parity mode) */
    int64_t K_capacity;    /* slices the store is sized for up front (0: 2 * K0); grows on demand */
    int64_t max_batch;     /* > 0: at init, size the workspace for every K_new <= max_batch
                              up to K_capacity slices (sbt_reserve); 0: size on demand */
    void *cuda_stream;     /* cudaStream_t for all device work; NULL: the legacy default stream */
    int32_t check_every;   /* ALS convergence poll interval in iterations (0: 4) */
    int32_t refine_sweeps; /* SBT_PREC_BF16 only: after the bf16 ALS, this many ALS iterations whose
                              MTTKRP reads the split summary x ~ hi + lo (hi = bf16(x), lo =
                              bf16(x - hi), ~16 significant bits); 0: none.  Needs the
                              tensor-core MTTKRP (R <= 32); otherwise flagged and skipped */
    int32_t autotune;      /* 1: before the ALS of an update, time the tile candidates of every
                              tensor-core MTTKRP launch shape not in the tile table and record
                              the fastest (see sbt_tile_table); 0: use the table / default rule */
    int32_t mode3_pass;    /* tensor-core MTTKRP (bf16 / fp8 summaries) only.  0 (default): the
                              mode-2 pass keeps every slice's product Y_k = X_k^T A (float32,
                              K_s' x n_J x R per repetition) and the mode-3 MTTKRP is formed from
                              it and the new B, M3(k, r) = sum_j Y_k(j, r) B(j, r): two passes
                              over the summary per ALS iteration instead of three (the same sums
                              as the definition, in another order).  1: mode 3 reads the summary
                              in its own pass */
    int32_t als_groups;    /* tensor-core MTTKRP only: the r independent summary ALS run as this
                              many groups of repetitions, each its own chain of kernels on its
                              own stream, so that one group's MTTKRP pass overlaps another
                              group's latency-bound tail; 0: 2 (1 when r = 1).  Results depend
                              on it only through the order of partial sums */
    int32_t warm_start;    /* 0 (default): the summary ALS starts from Philox uniforms keyed by the
                              global index (the paper leaves the start open).  1: it starts from
                              the old factors at the sampled rows, A(I_s), B(J_s), C(K_s), with
                              the new slices' rows of C' zero; it then converges in a few
                              iterations and keeps the component order */
    int32_t get_rank;      /* 1: quality control of Section 3.2 (Algorithm 2, GetRank) on every
                              summary: for each candidate rank i = 1..R and trial t <
                              get_rank_trials, a CP-ALS of the summary at rank i from Philox
                              uniforms (counter (x, r | mode << 8 | rep << 12 | t << 20, batch, 3)),
                              scored by its core consistency (sbt_core_consistency); R_new = the
                              largest i whose best trial reaches get_rank_threshold (1 if none).
                              The summary ALS then runs at rank R_new from the usual start, its
                              components are matched to R_new distinct old components, and a new
                              row of C averages each component over the repetitions that matched
                              it (none: zero).  MTTKRP on the CUDA cores; SBT_PREC_FP8,
                              refine_sweeps and COO contexts are rejected (SBT_E_INVALID).
                              0 (default): every summary at rank R */
    int32_t get_rank_trials;   /* GetRank decompositions per candidate rank (Algorithm 2's `it`); 0: 2 */
    double get_rank_threshold; /* core consistency a candidate rank must reach; 0: 90 */
    int32_t fp64_tail;     /* SBT_PREC_F32 / BF16 / FP8: 1 runs the R x R work of every ALS step in
                              float64 -- the Hadamard product of the Grams, its Cholesky factorisation
                              and the solve U = M V^-1, the column norms, the Grams and the fit --
                              one CTA per repetition, after the MTTKRP partials are summed in float64;
                              0 (default): double-float (~44 bits) on the float32 pipes, V^-1 beside
                              the MTTKRP pass */
    int32_t persistent_als;/* 1: the summary ALS of all repetitions, when its MTTKRP runs on the CUDA
                              cores (SBT_PREC_F64 / F32, or BF16 without the tensor-core plan) and the
                              context is dense, is one persistent cooperative launch: the steps of
                              every iteration separated by bounded grid barriers instead of kernel
                              boundaries, the float64 tail (as fp64_tail); the same results as the
                              launch-per-step ALS with the float64 tail.  Ignored with per-launch
                              profiling timing.  0 (default): a CUDA graph of per-step kernels */
} sbt_options;

typedef struct {
    int64_t K;                 /* slices held after the update */
    int32_t r, R;
    int32_t n_I, n_J, n_K;     /* sample sizes of the update */
    int32_t flags;             /* SBT_FLAG_* */
    int32_t iters[SBT_MAX_REPS];     /* ALS iterations per repetition */
    double fit[SBT_MAX_REPS];        /* summary fit at the last ALS iteration */
    double min_score[SBT_MAX_REPS];  /* smallest |G1|*|G2|*|G3| over matched pairs */
    int32_t perm[SBT_MAX_REPS][SBT_MAX_RANK]; /* summary component -> old component (-1 past rank[rep]) */
    int32_t rank[SBT_MAX_REPS];      /* components of each summary: R, or R_new with get_rank */
} sbt_update_stats;

/* Library version string. */
const char *sbt_version(void);

/* Thread-local message of the last failing call on this thread. */
const char *sbt_last_error(void);

/* Fill *opt with defaults: s = 2 in every mode, r = 4, tol = 1e-6, 50
 * iterations (init: 50), seed 0, F32 MTTKRP, lambda kept. */
sbt_status sbt_default_options(sbt_options *opt);

/* Decompose X0 (I x J x K0) at rank R with CP-ALS on the GPU (Philox-uniform
 * start), sort components by lambda, fix signs (sum A(:,r) >= 0, sum B(:,r)
 * >= 0) and keep X0, the factors and the Eq. 1 marginals resident on the
 * device.  This is the pre-existing decomposition of Section 2.2, (a). */
sbt_status sbt_init(const sbt_tensor *X0, int32_t R, const sbt_options *opt, sbt_ctx **out);

/* Same, but the pre-existing decomposition is given: lambda (R), A (I x R),
 * B (J x R), C (K0 x R), host doubles, row-major.  No ALS runs. */
sbt_status sbt_init_factors(const sbt_tensor *X0, int32_t R, const double *lambda,
                            const double *A, const double *B, const double *C,
                            const sbt_options *opt, sbt_ctx **out);

/* Absorb K_new >= 1 new slices (I x J x K_new): Algorithm 1 once.  Sampling
 * uses the marginals of the tensor before the update.  Transactional: on any
 * error the factors, marginals and K are unchanged.  Returns after the GPU
 * finished (one host synchronisation per call). */
sbt_status sbt_update(sbt_ctx *ctx, const sbt_tensor *X_new);

/* Copy the current model to host buffers (any may be NULL): lambda (R),
 * A (I x R), B (J x R), C (K x R); *K_out receives K. */
sbt_status sbt_factors(const sbt_ctx *ctx, double *lambda, double *A, double *B, double *C,
                       int64_t *K_out);

/* Fit of the full model against the full resident tensor:
 * 1 - ||X - X_hat||_F / ||X||_F (Section 4.2, relative error = 1 - fit). */
sbt_status sbt_fit(sbt_ctx *ctx, double *fit);

/* The recompute comparator of Section 4.2 (Relative Fitness): CP-ALS of the
 * whole resident tensor from scratch, as sbt_init runs it (the store's
 * precision, Philox start with `seed` and the context's stream id, at most
 * max_iters iterations, stop when the fit changes by less than tol), without
 * touching the context's factors.  Outputs are caller-owned host buffers,
 * each nullable: lambda (R), A (I x R), B (J x R), C (K x R), row-major; *fit
 * = 1 - ||X - X_cp|| / ||X|| of the recomputed model.  Relative Fitness =
 * ||X - X_sbt|| / ||X - X_cp|| = (1 - sbt_fit) / (1 - *fit).  Dense
 * contexts only (SBT_E_STATE for COO).  Synchronises the context's stream;
 * may grow the context's ALS workspace. */
sbt_status sbt_recompute(sbt_ctx *ctx, int32_t max_iters, double tol, uint64_t seed, double *lambda, double *A,
                         double *B, double *C, double *fit);

/* Statistics of the last sbt_update. */
sbt_status sbt_stats(const sbt_ctx *ctx, sbt_update_stats *st);

/* ---- sparse (COO) tensors -------------------------------------------------
 * The same method (Alg. 1) on tensors stored as nonzeros (the sparse
 * workloads of Section 4.1).  The context keeps the nonzeros grouped by time
 * slice; summaries are the lists of nonzeros of the sampled slices whose row
 * and column were sampled.  Results equal the dense definitions applied to the
 * densified tensor; the MTTKRP adds its float32 products in 64-bit fixed point,
 * so results do not depend on the order of the input nonzeros.  Coordinates
 * must be unique (duplicates are not merged).  Options: prec must be
 * SBT_PREC_F32; refine_sweeps, autotune, max_batch do not apply. */
typedef struct {
    int64_t I, J, K;           /* shape (K: slices of this tensor or batch) */
    int64_t nnz;               /* nonzeros, < 2^31 */
    const int32_t *ii, *jj, *kk;  /* coordinates; kk relative to this tensor (batch): 0 <= kk < K */
    const float *val;
    int32_t on_device;         /* arrays in device memory (ordered on opts.cuda_stream) or host */
} sbt_coo;

/* CP-ALS of X0 (max_iters_init iterations) and a context for updates.
 * SBT_E_SHAPE: a coordinate outside the shape; SBT_E_NONFINITE; SBT_E_INVALID. */
sbt_status sbt_init_coo(const sbt_coo *X0, int32_t R, const sbt_options *opts, sbt_ctx **out);

/* As sbt_init_coo with the decomposition of X0 given (host, row-major, as
 * sbt_init_factors). */
sbt_status sbt_init_coo_factors(const sbt_coo *X0, int32_t R, const double *lambda, const double *A,
                                const double *B, const double *C, const sbt_options *opts, sbt_ctx **out);

/* One batch of K_new new slices given as nonzeros (kk relative to the batch);
 * transactional like sbt_update.  sbt_factors, sbt_fit, sbt_stats,
 * sbt_last_samples and sbt_last_summary_factors apply to COO contexts too. */
sbt_status sbt_update_coo(sbt_ctx *ctx, const sbt_coo *X_new);

/* ---- order-N tensors ------------------------------------------------------
 * Section 2.2: the problem and the method extend to tensors with any number
 * of modes, one of which grows with time.  These calls run Algorithm 1 on a
 * dense tensor with N = 3..SBT_NMODE_MAX modes: Eq. 1 marginals of every mode,
 * each non-time mode and the old slices sampled by exponential keys (Philox
 * counter (x, mode | rep << 4, batch, 1), mode = the factor's position below),
 * the summary at the sampled indices plus the new slices, CP-ALS over all N
 * modes (Philox start (x, r | mode << 8 | rep << 12, batch, 2); MTTKRP with the
 * Khatri-Rao rows of the other N-1 factors formed on the fly; the Hadamard
 * product of the other N-1 Grams solved by a float64 Cholesky factorisation;
 * unit columns; the fit after the last mode), shared-row normalisation,
 * Lemma 1 matching with the product of the N |cosine| matrices, and the new
 * time rows projected back and averaged over the repetitions.  Zero-entry
 * fills and lambda_mode are not applied (lambda is kept).
 *
 * Layout: time first, row-major: element (k, i_1, ..., i_{N-1}) of a tensor
 * with dims = (K, I_1, ..., I_{N-1}) sits at
 * data[((k * I_1 + i_1) * I_2 + i_2) ... * I_{N-1} + i_{N-1}].  Factors are in
 * factor order: U[0..N-2] = the modes of I_1..I_{N-1} (I_m x R), U[N-1] = C
 * (K x R), row-major float64.  Sampling factors: s_I for I_1 and for I_3 and
 * later modes, s_J for I_2, s_K for time.  Options used: s_I, s_J, s_K, r, tol,
 * max_iters, seed, stream_id, prec (SBT_PREC_F64 with a float64 tensor or
 * SBT_PREC_F32 with a float32 one: the summary keeps the stored values; the
 * float32 MTTKRP multiplies and adds in float32 within a lane, float64
 * beyond), fixed_iters, K_capacity, cuda_stream, check_every; the others must
 * be at their defaults (SBT_E_INVALID otherwise).  R <= SBT_MAX_RANK; the
 * summary's last dimension I_{N-1} / s must fit the MTTKRP's shared-memory
 * plan (I_{N-1} / s x 32 x 8 bytes <= 200 KB).  Every call returns a status. */
#define SBT_NMODE_MAX 8

typedef struct {
    int32_t dtype;                  /* SBT_F64 or SBT_F32 */
    int32_t on_device;              /* 1: device memory of the context's device */
    int32_t N;                      /* modes, 3..SBT_NMODE_MAX */
    int64_t dims[SBT_NMODE_MAX];    /* dims[0] = K (slices), dims[1..N-1] = I_1..I_{N-1} */
    const void *data;
} sbt_tensor_n;

typedef struct sbt_nmode sbt_nmode; /* opaque; owned by the library */

/* A context for the pre-existing decomposition lambda (R), U[0..N-1] (host
 * float64, factor order, U[N-1] with K0 rows) of X0; X0, the factors and the
 * marginals are kept on the device.  SBT_E_NONFINITE, SBT_E_SHAPE,
 * SBT_E_INVALID, SBT_E_NOMEM, SBT_E_CUDA. */
sbt_status sbt_nmode_init_factors(const sbt_tensor_n *X0, int32_t R, const double *lambda, const double *const *U,
                                  const sbt_options *opt, sbt_nmode **out);

/* Absorb K_new = X_new->dims[0] >= 1 new slices (the other dims as at init):
 * Algorithm 1 once.  Transactional like sbt_update (non-finite values,
 * marginal overflow: SBT_E_NONFINITE / SBT_E_RANGE, state unchanged).  One
 * host synchronisation per ALS convergence poll and one at the end. */
sbt_status sbt_nmode_update(sbt_nmode *c, const sbt_tensor_n *X_new);

/* Copy the model to caller-owned host buffers (any may be NULL; U may hold
 * NULL entries): lambda (R), U[m] (n_m x R, U[N-1] with K rows); *K_out = K. */
sbt_status sbt_nmode_factors(const sbt_nmode *c, double *lambda, double *const *U, int64_t *K_out);

/* 1 - ||X - X_hat||_F / ||X||_F over the whole resident tensor (Section 4.2). */
sbt_status sbt_nmode_fit(sbt_nmode *c, double *fit);

/* Statistics of the last update: n_I, n_J = the sample sizes of I_1 and I_2,
 * n_K = of the old slices; iters, fit, min_score, perm per repetition. */
sbt_status sbt_nmode_stats(const sbt_nmode *c, sbt_update_stats *st);

/* Sampled indices of repetition rep in mode `mode` (factor order; N-1: the
 * old slices), ascending; *n receives the count, at most cap written. */
sbt_status sbt_nmode_last_samples(const sbt_nmode *c, int32_t rep, int32_t mode, int32_t *out, int64_t cap,
                                  int64_t *n);

/* Free the context.  NULL is a no-op. */
void sbt_nmode_destroy(sbt_nmode *c);

/* ---- device memory of a context ------------------------------------------
 * No counterpart in the paper: these let a caller (the server below) admit
 * work by a device-memory budget and keep allocation out of the update path. */

/* Device bytes the context holds now (store, factors, marginals, workspace). */
sbt_status sbt_device_bytes(sbt_ctx *ctx, uint64_t *bytes);

/* Device bytes the context would hold after an sbt_update of K_new slices,
 * computed on the host without allocating (buffers only grow).
 * SBT_E_INVALID for K_new < 1; SBT_E_STATE if a mode has no positive weight. */
sbt_status sbt_update_bytes(sbt_ctx *ctx, int64_t K_new, uint64_t *bytes);

/* Size the store for K_max slices and the workspace for every update that
 * keeps K <= K_max with K_new <= K_new_max, so that those updates allocate
 * and free nothing (cudaFree waits for the whole device).  The init calls do
 * this when opts.max_batch > 0, with K_max = the store capacity.
 * SBT_E_INVALID unless K_new_max >= 1 and K_max > K; SBT_E_NOMEM. */
sbt_status sbt_reserve(sbt_ctx *ctx, int64_t K_max, int64_t K_new_max);

/* Inspection of the last sbt_update (for parity checks): the sampled indices
 * of repetition rep in mode (0: I_s, 1: J_s, 2: K_s over the old slices),
 * ascending.  *n receives the count; at most cap are written. */
sbt_status sbt_last_samples(const sbt_ctx *ctx, int32_t rep, int32_t mode, int32_t *out,
                            int64_t cap, int64_t *n);

/* The gathered summary of repetition rep as the values the ALS computed with
 * (bfloat16 / float32 / float64, widened exactly to double), slice-major
 * (Kp x n_I x n_J) with Kp = n_K + K_new; dims[3] receives (n_I, n_J, Kp). */
sbt_status sbt_last_summary(const sbt_ctx *ctx, int32_t rep, double *out, int64_t cap,
                            int64_t dims[3]);

/* Summary factors of repetition rep after the shared-row normalisation
 * (Alg. 1 step 6): lambda' (R), A' (n_I x R), B' (n_J x R), C' (Kp x R).
 * With get_rank the summary has rank[rep] components: columns beyond it
 * (and their lambda') are zero. */
sbt_status sbt_last_summary_factors(const sbt_ctx *ctx, int32_t rep, double *lambda,
                                    double *A, double *B, double *C);

/* Counters for measurement (the benchmark's roofline figure). */
typedef struct {
    int64_t launches;        /* kernels launched by the library (process-wide) since the reset */
    int64_t updates;         /* sbt_update calls committed since the reset */
    int64_t mttkrp_launches; /* MTTKRP kernel launches over the summaries (one per group of
                                repetitions per pass) */
    double mttkrp_ms;        /* device time of the passes from CUDA events (timing enabled), else
                                0: per pass, from the first group's launch start to the last
                                group's launch end (the groups' launches run concurrently) */
    double mttkrp_bytes;     /* algorithmic bytes of the passes: each summary element of every
                                repetition still iterating read once per pass */
    int64_t mttkrp_passes;   /* timed passes (mttkrp_ms covers these) */
    double mttkrp_busy_ms;   /* device time during which at least one timed MTTKRP launch ran: the
                                union of the launches' event intervals (a group's pass that overlaps
                                the other group's next pass is not counted twice) */
    double mttkrp_launch_ms; /* sum of the timed launches' own durations (concurrent launches of
                                the groups each counted in full) */
} sbt_profile;

/* Zero the counters.  timing != 0 also brackets every MTTKRP launch of this
 * context with CUDA events on the stream it runs on; the ALS then runs in
 * chunks of check_every iterations, polling convergence from the host after
 * each, rather than as one graph with a device-side loop (leave it off for
 * throughput).  timing = 1: each chunk is one launch of a graph of its
 * kernels and events, captured once per ALS, so that no event interval holds
 * host submission time; timing = 2: the chunk's kernels launched one by one
 * (visible to tools that trace kernel launches, intervals may include
 * submission gaps).  Other values: SBT_E_INVALID. */
sbt_status sbt_profile_reset(sbt_ctx *ctx, int32_t timing);

/* Read the counters (synchronises the context's stream). */
sbt_status sbt_profile_read(sbt_ctx *ctx, sbt_profile *out);

/* Free every device and host resource of the context.  NULL is a no-op. */
void sbt_destroy(sbt_ctx *ctx);

/* ---- MTTKRP tile table ----------------------------------------------------
 * No counterpart in the paper.  Process-wide choices for the tensor-core
 * MTTKRP (bf16 / fp8 summaries): per launch shape, CTAs per SM (1 or 2) and
 * pipeline stages (0: as many as fit).  Shapes without an entry use 2 CTAs
 * per SM and as many stages as fit.  Filled by the autotuner
 * (sbt_options.autotune) or imported (a tuning run can be saved and
 * reloaded).  Results depend on the choice only through the order in which
 * partial sums are added. */
typedef struct {
    int32_t fp8;          /* 0: bfloat16 summaries, 1: float8 */
    int32_t R;
    int32_t NP;           /* summary rows of the launch (n_I for modes 1 and 3, n_J for mode 2) */
    int32_t NC;           /* contraction length (n_J for modes 1 and 3, n_I for mode 2) */
    int32_t Kp_bucket;    /* ceil(summary slices / 32) */
    int32_t nrep;         /* repetitions in the launch */
    int32_t epi;          /* 0: rows of M (modes 1, 2), 1: M3 (mode 3) */
    int32_t ctas_per_sm;  /* 1 or 2 */
    int32_t stages;       /* 0..8 */
} sbt_tile_entry;

/* op 0: copy up to cap entries into entries, *n = number in the table;
 * op 1: merge cap entries from entries (same key: replaced);
 * op 2: clear.  SBT_E_INVALID on bad arguments or choices. */
sbt_status sbt_tile_table(int32_t op, sbt_tile_entry *entries, int32_t cap, int32_t *n);

/* ---- serving loop ---------------------------------------------------------
 * No counterpart in the paper, which absorbs one stream.  A server owns many
 * tensor streams, each a context whose store, factors and marginals stay
 * resident on the device, and runs their update batches concurrently:
 * `slots` worker threads each drive one sbt_update at a time on the CUDA
 * streams of that tensor stream's own context, so updates of different
 * streams overlap on the GPU.  A queued batch is admitted when a slot is free
 * and the device bytes its stream will hold after the update
 * (sbt_update_bytes) fit the budget together with every other stream's
 * bytes; a batch that cannot fit even alone fails with SBT_E_NOMEM.  Batches
 * of one stream run in submission order; batches of different streams are
 * admitted in arrival order, skipping those that do not fit yet (they wait
 * until a stream is closed).  Results do not depend on which batches share
 * the GPU: every kernel reduces in a fixed order.
 *
 * A batch is borrowed, not copied: the tensor given to sbt_server_submit must
 * stay valid until its ticket is done, and device data must be complete on
 * the stream named by the stream's options (cuda_stream; NULL: the legacy
 * default stream) when its update starts.  All calls are thread-safe except
 * sbt_server_destroy, which must not race with other calls on the server. */
typedef struct sbt_server sbt_server;

typedef struct {
    int32_t slots;        /* concurrent updates (worker threads), 1..64; 0: 4 */
    uint64_t mem_budget;  /* device bytes all streams may hold; 0: 90 % of the free memory at create */
    int32_t device;       /* CUDA device; -1: the calling thread's current device */
    int32_t batch_als;    /* 1: one worker admits up to `slots` batches together and runs the summary
                             ALS of those whose streams were opened with persistent_als (the CUDA-core
                             path: SBT_PREC_F64 / F32) in one persistent launch, up to 8 compatible
                             updates (same summary precision, R in the same range 1-8, 9-16, 17-32)
                             per launch; every other step of each update, and the whole update of other
                             streams, runs as in sbt_update.  Each stream's results are the same bits
                             as its update alone with persistent_als.  0 (default): `slots` workers,
                             one sbt_update each */
} sbt_server_options;

typedef struct {
    int32_t status;       /* sbt_status of the update (the stream is unchanged unless SBT_OK) */
    int32_t stream;       /* the stream id */
    int64_t K;            /* slices the stream held after the update */
    double queue_ms;      /* submit -> update started */
    double service_ms;    /* update started -> committed */
    double total_ms;      /* submit -> committed */
} sbt_request_result;

typedef struct {
    int64_t submitted, completed, failed;  /* batches since the last reset */
    int64_t queued, in_flight, streams;    /* now */
    int64_t slices;                        /* slices absorbed since the reset */
    uint64_t resident_bytes;               /* device bytes held by all streams now */
    uint64_t peak_resident_bytes;          /* the most held (or reserved) since the reset */
    uint64_t mem_budget;
    double latency_p50_ms, latency_p99_ms; /* submit -> committed, completed batches */
    double service_p50_ms, service_p99_ms; /* update started -> committed */
    double busy_fraction;                  /* wall time with an update in flight / elapsed */
    double elapsed_s;                      /* since the reset */
    int64_t als_launches;                  /* batch_als: persistent launches run since the reset */
    int64_t als_sets;                      /* batch_als: updates' summary ALS those launches ran */
} sbt_serving_stats;

/* Defaults: 4 slots, 90 % of free memory, the current device. */
sbt_status sbt_server_default_options(sbt_server_options *opts);

/* Start a server and its worker threads.  opts may be NULL (defaults). */
sbt_status sbt_server_create(const sbt_server_options *opts, sbt_server **out);

/* Open a tensor stream: sbt_init(X0, R, opts) on the server's device in the
 * calling thread, admitted only if the context fits the memory budget
 * (SBT_E_NOMEM otherwise, nothing kept).  Use opts.K_capacity and
 * opts.max_batch so that later updates allocate nothing.  *sid receives the
 * stream id. */
sbt_status sbt_server_open_stream(sbt_server *srv, const sbt_tensor *X0, int32_t R, const sbt_options *opts,
                                  int32_t *sid);

/* Queue one batch (sbt_update semantics) for stream sid; returns at once.
 * *ticket identifies it for sbt_server_wait.  SBT_E_INVALID: unknown or
 * closing stream; SBT_E_SHAPE: empty batch. */
sbt_status sbt_server_submit(sbt_server *srv, int32_t sid, const sbt_tensor *X_new, uint64_t *ticket);

/* Wait for a batch (timeout_ms < 0: no limit).  On SBT_OK *res (may be NULL)
 * receives its result and the ticket is released; if the batch failed
 * (res->status), its message becomes the calling thread's sbt_last_error().
 * SBT_E_TIMEOUT leaves it pending; SBT_E_INVALID: unknown ticket.  One thread
 * waits for a ticket. */
sbt_status sbt_server_wait(sbt_server *srv, uint64_t ticket, int32_t timeout_ms, sbt_request_result *res);

/* The stream's context, for sbt_factors / sbt_fit / sbt_stats while the
 * stream has no batch queued or in flight (SBT_E_STATE otherwise).  Owned by
 * the server; do not destroy it. */
sbt_status sbt_server_stream_ctx(sbt_server *srv, int32_t sid, sbt_ctx **ctx);

/* Wait for the stream's queued batches, then free its context and memory. */
sbt_status sbt_server_close_stream(sbt_server *srv, int32_t sid);

/* Counters and latency percentiles since the last reset. */
sbt_status sbt_server_stats(sbt_server *srv, sbt_serving_stats *st);
sbt_status sbt_server_stats_reset(sbt_server *srv);

/* Fail the batches not yet started (SBT_E_STATE), let the ones in flight
 * finish, stop the workers, wait until no thread is inside sbt_server_wait,
 * and free every stream.  No other call may start on the server once destroy
 * has begun.  NULL is a no-op. */
void sbt_server_destroy(sbt_server *srv);

/* ---- device-level operations (device pointers, ordered on `stream`) -------
 * These run one kernel family on caller buffers and return without a host
 * synchronisation unless stated.  Scratch is taken from the stream-ordered
 * allocator (cudaMallocAsync) and returned before the call returns. */

/* Philox4x32-10 (Salmon et al., SC'11) of n counters: ctr (n x 4 uint32),
 * out (n x 4 uint32); key = (key0, key1).  This is the counter-based
 * generator behind the sampler and the ALS start values. */
sbt_status sbt_philox4x32_10(const uint32_t *ctr, uint32_t key0, uint32_t key1, uint32_t *out,
                             int64_t n, void *stream);

/* Weighted sampling without replacement of one mode (Section 3.1, Alg. 1
 * step 3): draws n of the N indices with w[x] > 0, probability proportional
 * to w (successive sampling through exponential keys), writes them ascending
 * to out (device, n int32).  Philox key (lo32(seed), hi32(seed) ^ stream_id),
 * counter (x, mode | rep << 4, batch, 1).  SBT_E_INVALID if n exceeds the
 * number of positive weights (checked on the device; this call synchronises
 * to report it). */
sbt_status sbt_sample(const uint64_t *w, int64_t N, int64_t n, uint64_t seed,
                      uint32_t stream_id, int32_t mode, int32_t rep, uint32_t batch,
                      int32_t *out, void *stream);

/* MTTKRP of a dense slice-major tensor (K x I x J, row pitch ld >= J elements,
 * ld a multiple of 8, X 16-byte aligned) for one mode (0: M = X_(1)(C kr B)
 * -> I x R; 1: J x R; 2: K x R), the contraction inside every ALS step of
 * Alg. 1 step 5.  dtype SBT_F64 or SBT_F32 applies to X, the factors A (I x R),
 * B (J x R), C (K x R) and M (CUDA cores).  dtype SBT_BF16: X is bfloat16, the
 * factors and M are float32, and the product runs on the tensor cores
 * (tcgen05, factors split into three bfloat16 terms up to R = 16, two
 * above); SBT_E_INVALID if R or the contraction length is beyond that
 * kernel's shared-memory plan. */
sbt_status sbt_mttkrp(int32_t dtype, const void *X, int64_t K, int64_t I, int64_t J, int64_t ld,
                      const void *A, const void *B, const void *C, int32_t R, int32_t mode,
                      void *M, void *stream);

/* Core consistency diagnostic (CorConDia, Bro & Kiers 2003), the quality
 * rating GetRank gives each candidate decomposition (Section 3.2, Algorithm
 * 2): 100 (1 - ||G - T||^2 / R) with G = X x_1 A+ x_2 B+ x_3 (C diag(lambda))+
 * the least-squares Tucker core for the fixed factors (F+ = (F^T F)^-1 F^T)
 * and T the superdiagonal of ones; 100 for an exact CP, far below for an
 * over-factored one.  X: device, slice-major K x I x J, row pitch ld >= J
 * elements, dtype SBT_F64 or SBT_F32; lambda (R), A (I x R), B (J x R),
 * C (K x R): device float64, row-major; *cc: host.  Computed in float64 with
 * fixed-order sums; allocates scratch of about K I R + R (I + J + K) + K R^2
 * doubles on `stream` and synchronises it.  SBT_E_INVALID for a null
 * pointer, another dtype or R outside [1, SBT_MAX_RANK]; SBT_E_SHAPE unless
 * K, I, J >= R; SBT_E_STATE if a factor's Gram is not positive definite. */
sbt_status sbt_core_consistency(int32_t dtype, const void *X, int64_t K, int64_t I, int64_t J, int64_t ld,
                                const double *lambda, const double *A, const double *B, const double *C,
                                int32_t R, double *cc, void *stream);

/* The weighted draw of sbt_sample for callers that must not allocate device
 * memory during the call -- for example a serving process that gives the whole
 * device to its own pool at start-up, or a latency-critical loop where a
 * cudaMalloc (which may synchronise the device) is not allowed.  The paper has
 * no counterpart to this entry point; it is a deployment variant.
 *
 * Same arguments, results and errors as sbt_sample; N must not exceed
 * SBT_SAMPLE_NOALLOC_MAX_N (SBT_E_INVALID otherwise).  Scratch: one fixed
 * array of SBT_SAMPLE_NOALLOC_MAX_N * 16 + 256 bytes (about 4 MiB) in the
 * library's device memory, held by every GPU that loads the library until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress), so make the first call before any stream
 * capture; later calls outside a capture look it up again (a device reset
 * may move the array), calls inside a capture use the address found last.  All calls share the array and it keeps the last call's contents:
 * calls that overlap on the GPU (unordered streams or threads) race on it. */
#define SBT_SAMPLE_NOALLOC_MAX_N 262144
sbt_status sbt_sample_noalloc(const uint64_t *w, int64_t N, int64_t n, uint64_t seed,
                              uint32_t stream_id, int32_t mode, int32_t rep, uint32_t batch,
                              int32_t *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SAMBATEN_H */
