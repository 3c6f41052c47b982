// MTTKRP of bfloat16 summaries on the 5th-generation tensor cores (tcgen05).
//
// Per slice kk of a summary, Z = X_kk . F is a dense product: 128 rows of
// X_kk (an M = 128 tile, rows beyond the summary zero-filled by TMA) times the
// contraction factor F (K = the other summary dimension, N = NT * RH
// columns: F as NT bfloat16 terms, each the rounding of what the previous
// ones left, so that bf16 x (sum of the terms) keeps ~24 bits (three terms)
// or ~16 bits (two) of the float32 factor).  The accumulators
// live in tensor memory; four epilogue warps read them back and fold the
// ALS weights in:
//   ROWSUM (modes 1 and 2): M(p, r) += Z(p, r) C(kk, r), summed over the
//       CTA's slices in registers -> part[rep][ks][p][r];
//   COLSUM (mode 3): M3(kk, r) = sum_p Z(p, r) A(p, r) over the tile's rows
//       -> part[rep][pb][kk][r].
// Mode 2 reads a transposed copy of the summary ([kk][jj][ii]) so that every
// operand is K-major.  Warp roles: warp 0 issues TMA loads into a ring of
// 16 KB stages, warp 1 owns tensor memory and issues the MMAs (one thread),
// warps 2-5 are the epilogue.  Every mbarrier wait is bounded; a timeout sets
// an error word, stops the CTA's loops, waits for its outstanding copies and
// frees its tensor memory.
#include "sbt_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

namespace sbt {

constexpr int TC_M = 128;
constexpr int TC_BOX_BYTES = TC_M * 128;  // 128 rows x 64 bfloat16
constexpr unsigned TC_SPIN_LIMIT = 1u << 24;  // ~0.5 s of polling per wait

// ---------------------------------------------------------------------------
// PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// tiled 3-d load with an L2 eviction policy (`policy` from createpolicy)
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// L2 policy for data read once per pass: evicted before other lines, so the
// pass's outputs (partials, kept products) and the factors stay in L2
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand in the 128-byte swizzled layout: 8-row atoms of 128 B,
// atoms 1024 B apart (stride byte offset); the leading offset is unused.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;              // leading byte offset (16 B, ignored for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset: 1024 B between 8-row atoms
    d |= (uint64_t)1 << 46;              // descriptor version of the 5th-generation tensor core
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// Instruction descriptor, D float32, A and B K-major: kind::f16 with A and B
// bfloat16 (format 1), or kind::f8f6f4 with A and B float8 e4m3 (format 0).
template <bool FP8>
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4)                                  // D format: float32
           | ((FP8 ? 0u : 1u) << 7)                   // A format
           | ((FP8 ? 0u : 1u) << 10)                  // B format
           | ((uint32_t)(N >> 3) << 17)               // N / 8
           | ((uint32_t)(M >> 4) << 24);              // M / 16
}

template <bool FP8>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    if constexpr (FP8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}


__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// ---------------------------------------------------------------------------
struct TcParams {
    int nrep, R, NP, NC, Kp;
    int nkb, npb, spc, nks;
    int br;                  // summary rows per tile (tiles of equal height, a multiple of 8, <= 128)
    int split;               // 1: add the lo part of a split summary (second tensor map) into each product
    const float *sscale;     // float8 summaries: scale of every summary slice [rep][Kp]; else null
    int epi;                 // 0 ROWSUM (weights C(kk)), 1 COLSUM (weights A(p))
    const float *F;          // contraction factor [rep][NC][R]
    long long frs;
    const float *W;          // epilogue factor [rep][Kp][R] (ROWSUM) or [rep][NP][R] (COLSUM)
    long long wrs;
    float *part;
    long long prs;
    int pr;                  // row stride of the partials
    const int *conv;
    unsigned long long *bytes_ctr;
    unsigned *err;           // device status word (ERR_TIMEOUT on a wait that gave up)
    int stages;
    float *Y;                // ROWSUM only, nullable: every slice's product Z = X_kk F, [rep][Kp][NP][pr]
    long long yrs;
};

constexpr int TC_MAX_SPC = 64;  // slices per CTA (epilogue weights staged in shared memory)

struct TcShared {
    uint64_t full[8], empty[8], accf[2], acce[2];
    uint32_t tmem_base;
    int abort_flag;
    float red[4][32];
};

// bounded wait; on timeout raise the abort flag and the error word
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, unsigned *err) {
    for (unsigned it = 0; it < TC_SPIN_LIMIT; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (it > 64) __nanosleep(32);
    }
    *abort_flag = 1;
    atomicOr(err, ERR_TIMEOUT);
    return false;
}

// N columns: NT terms of RH columns each.  bfloat16 summaries: the factor
// as bf16 terms, hi + mid + lo (NT = 3, the float32 factor to ~24 bits) up
// to R = 16 and hi + lo (NT = 2, ~16 bits) above, where a third term would
// not leave room for two CTAs per SM; float8 summaries: the factor as three
// e4m3 terms at fixed scales, F = 2^-8 (e1 + 2^-4 e2 + 2^-8 e3) (NT = 3;
// factor entries are at most 1 in magnitude: unit columns or uniforms in
// [0, 1)).
template <int N, bool FP8>
__global__ void __launch_bounds__(192, 2) k_mtt_tc(const __grid_constant__ CUtensorMap tmap,
                                                   const __grid_constant__ CUtensorMap tmap_lo, TcParams p) {
    constexpr int NT = (FP8 || N == 48) ? 3 : 2;
    constexpr int RH = N / NT;
    constexpr int TS = N <= 32 ? 32 : (N <= 64 ? 64 : 128);  // tensor-memory columns per accumulator
    constexpr int KE = FP8 ? 128 : 64;                        // contraction elements per 128-byte row
    const int rep = blockIdx.y;
    // programmatic dependent launch: the next kernel of the stream may be
    // scheduled now.  This grid reads the previous kernel's results (the
    // factors, the convergence flags) only after griddepcontrol.wait below;
    // the summary tiles do not depend on it, so warp 0 starts streaming them
    // at once.  The flag read here may predate a convergence decided by the
    // kernel just before; it is read again after the wait.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // one decision for the whole CTA: the kernel before may be writing the
    // flag now, and threads that read it at different moments must not
    // split (some leaving, the rest waiting at a barrier for them)
    if (__syncthreads_or(p.conv[rep] != 0)) return;
    if (threadIdx.x == 0) {
        // fetch the tensor maps while the barriers and tensor memory are set up
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmap) : "memory");
        if (p.split) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmap_lo) : "memory");
    }
    const int pb = blockIdx.x % p.npb, ks = blockIdx.x / p.npb;
    const int k0 = ks * p.spc, k1 = min(p.Kp, k0 + p.spc);
    const int nsl = k1 - k0;
    if (nsl <= 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = p.stages;

    extern __shared__ unsigned char smem_dyn[];
    // 1024-byte alignment for the swizzled tiles
    const uint32_t base_u32 = smem_u32(smem_dyn);
    unsigned char *smem = smem_dyn + ((1024u - (base_u32 & 1023u)) & 1023u);
    unsigned char *ring = smem;                                   // S x 16 KB
    unsigned char *btile = ring + (size_t)S * TC_BOX_BYTES;        // nkb x N x 128 B
    TcShared *sh = reinterpret_cast<TcShared *>(btile + (size_t)p.nkb * N * 128);
    float *wst = reinterpret_cast<float *>(sh + 1);                // [TC_MAX_SPC][RH] epilogue weights
    volatile int *abort_flag = &sh->abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&sh->accf[a], 1);
            mbar_init(&sh->acce[a], 128);
        }
        sh->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    // the producer (thread 0, which initialised the barriers) issues its
    // first S boxes at once: every stage starts empty, so they need no wait,
    // and they fly while tensor memory and the B operand are set up
    const int nkb2 = p.nkb * (1 + p.split);
    const int nbox = nsl * nkb2;
    const int pre = min(S, nbox);
    const uint64_t pol = l2_evict_first_policy();
    auto issue_box = [&](int b, int stage) {
        const int t = b / nkb2, kb2 = b % nkb2;
        const int kb = kb2 < p.nkb ? kb2 : kb2 - p.nkb;
        mbar_expect_tx(&sh->full[stage], (uint32_t)p.br * 128u);
        tma_load_3d(ring + (size_t)stage * TC_BOX_BYTES, kb2 < p.nkb ? &tmap : &tmap_lo, kb * KE, pb * p.br,
                    rep * p.Kp + k0 + t, &sh->full[stage], pol);
    };
    if (threadIdx.x == 0)
        for (int b = 0; b < pre; ++b) issue_box(b, b);
    // TMA fills rows [0, br) of a stage; rows [br, 128) keep whatever the
    // shared memory held.  Row i of an M = 128 product depends on row i of A
    // only, so those rows reach accumulator rows the epilogue never reads.
    __syncthreads();  // the barriers' initialisation, seen by every warp
    uint32_t tmem = 0;
    const int R = p.R;
    if (warp != 0) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        // Tensor memory is allocated only now, once the grid this one depends
        // on has finished.  tcgen05.alloc blocks while the SM's 512 columns
        // are taken; a CTA launched early (the tail before it triggers at its
        // start) that held columns while it waited here could hold them
        // against a CTA of an earlier MTTKRP on the same SM, which that tail
        // waits for: a cycle.  After the wait, every holder depends only on
        // its own copies and products, so every allocation is served.
        if (warp == 1) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&sh->tmem_base)),
                         "r"(2 * TS));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
        if (threadIdx.x == 32 && p.conv[rep]) *abort_flag = 2;  // converged just before: skip, no error
        // warps 1-5 (160 threads), while warp 0 already streams X: the B operand
        // (row n of term q holds column n - q RH of the factor; K-major,
        // 128-byte swizzled), one thread per contraction index j, and the
        // epilogue weights C(kk, :) (times the slice scale for float8)
        const float *F = p.F + rep * p.frs;
        const int t = threadIdx.x - 32;
        // the epilogue weights' first round (up to 320 entries) is loaded
        // with the factor, so the two L2 round trips overlap
        const float *W = p.W + rep * p.wrs;
        float w0[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = t + u * 160, tt = e / RH, r = e % RH;
            w0[u] = (p.epi == 0 && e < nsl * RH && r < R) ? W[(long long)(k0 + tt) * R + r] : 0.f;
        }
        // two contraction indices per thread and round, all loads of a round
        // in flight before the conversions
        for (int j0 = t; j0 < p.nkb * KE; j0 += 2 * 160) {
            float fv[2][RH];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int j = j0 + u * 160;
#pragma unroll
                for (int r = 0; r < RH; ++r) fv[u][r] = (j < p.NC && r < R) ? F[(long long)j * R + r] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int j = j0 + u * 160;
                if (j >= p.nkb * KE) break;
                const int kb = j / KE, k = j % KE;
                unsigned char *blk = btile + (size_t)kb * N * 128;
#pragma unroll
                for (int r = 0; r < RH; ++r) {
                    const float f = fv[u][r];
                    if constexpr (!FP8) {
                        // successive bf16 roundings of the remainder (exact differences)
                        __nv_bfloat16 t[NT];
                        float rem = f;
#pragma unroll
                        for (int q = 0; q < NT; ++q) {
                            t[q] = __float2bfloat16_rn(rem);
                            rem -= __bfloat162float(t[q]);
                        }
                        unsigned char *col = blk + (k & 7) * 2;
#pragma unroll
                        for (int q = 0; q < NT; ++q) {
                            const int n = q * RH + r;
                            *reinterpret_cast<__nv_bfloat16 *>(col + n * 128 + (((k >> 3) ^ (n & 7)) << 4)) = t[q];
                        }
                    } else {
                        const unsigned char e1 = to_e4m3(f * 256.f);
                        const float r1 = f - from_e4m3(e1) * 0.00390625f;
                        const unsigned char e2 = to_e4m3(r1 * 4096.f);
                        const float r2 = r1 - from_e4m3(e2) * 0.000244140625f;
                        const unsigned char e3 = to_e4m3(r2 * 65536.f);
                        const unsigned char ev[3] = {e1, e2, e3};
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const int n = q * RH + r;
                            blk[n * 128 + (((k >> 4) ^ (n & 7)) << 4) + (k & 15)] = ev[q];
                        }
                    }
                }
            }
        }
        if (p.epi == 0) {
            for (int e0 = t; e0 < nsl * RH; e0 += 2 * 160) {
                float w[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int e = e0 + u * 160, tt = e / RH, r = e % RH;
                    w[u] = e0 == t ? w0[u] : ((e < nsl * RH && r < R) ? W[(long long)(k0 + tt) * R + r] : 0.f);
                    if (FP8 && e < nsl * RH) w[u] *= p.sscale[(long long)rep * p.Kp + k0 + tt];
                }
#pragma unroll
                for (int u = 0; u < 2; ++u)
                    if (e0 + u * 160 < nsl * RH) wst[e0 + u * 160] = w[u];
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        asm volatile("bar.sync 2, 160;" ::: "memory");
        tc_fence_after();
        tmem = sh->tmem_base;  // written by warp 1's allocation
    }

    if (warp == 0) {
        if (lane == 0) {
            // producer: the boxes after the first S, each into the stage the
            // MMA released
            int stage = pre % S;
            uint32_t phase = pre == S ? 1u : 0u;
            int issued = pre;
            for (int b = pre; b < nbox && !*abort_flag; ++b) {
                if (!tc_wait(&sh->empty[stage], phase ^ 1u, abort_flag, p.err)) break;
                issue_box(b, stage);
                ++issued;
                if (++stage == S) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (*abort_flag) {
                // let the copies in flight land before the CTA leaves (bounded)
                int s = stage;
                uint32_t ph = phase;
                for (int q = 0; q < min(issued, S); ++q) {
                    if (--s < 0) {
                        s = S - 1;
                        ph ^= 1u;
                    }
                    for (unsigned it = 0; it < TC_SPIN_LIMIT && !mbar_try_wait(&sh->full[s], ph); ++it) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc_idesc<FP8>(TC_M, N);
            int stage = 0;
            uint32_t phase = 0;
            const uint32_t bbase = smem_u32(btile);
            for (int t = 0; t < nsl && !*abort_flag; ++t) {
                const int a = t & 1;
                const uint32_t aph = (uint32_t)(t >> 1) & 1u;
                if (!tc_wait(&sh->acce[a], aph ^ 1u, abort_flag, p.err)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * TS);
                bool ok = true;
                const int nkb2 = p.nkb * (1 + p.split);
            const uint64_t pol = l2_evict_first_policy();
                for (int kb2 = 0; kb2 < nkb2; ++kb2) {
                    const int kb = kb2 < p.nkb ? kb2 : kb2 - p.nkb;
                    if (!tc_wait(&sh->full[stage], phase, abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t abase = smem_u32(ring + (size_t)stage * TC_BOX_BYTES);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        tc_mma<FP8>(d, sw128_desc(abase + k * 32), sw128_desc(bbase + kb * N * 128 + k * 32), idesc,
                                    (kb2 | k) != 0);
                    }
                    tc_commit(&sh->empty[stage]);
                    if (++stage == S) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                tc_commit(&sh->accf[a]);
            }
        }
    } else {
        // epilogue: thread <-> tile row
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const int pidx = pb * p.br + row;
        const bool valid = row < p.br && pidx < p.NP;
        const float *W = p.W + rep * p.wrs;
        float acc[RH];
        float arow[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            acc[r] = 0.f;
            arow[r] = (p.epi == 1 && valid && r < R) ? W[(long long)pidx * R + r] : 0.f;
        }
        float *part = p.part + rep * p.prs;
        const int etid = threadIdx.x - 64;
        for (int t = 0; t < nsl; ++t) {
            const int a = t & 1;
            const uint32_t aph = (uint32_t)(t >> 1) & 1u;
            const bool got = tc_wait(&sh->accf[a], aph, abort_flag, p.err);
            float z[RH];
            if (got) {
                tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * TS);
                float v[32];
#pragma unroll
                for (int r = 0; r < RH; ++r) z[r] = 0.f;
#pragma unroll
                for (int c = 0; c < N; c += 32) {
                    tmem_ld32(taddr + c, v);
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int col = c + i;
                        if (col < N) {
                            const int q = col / RH;
                            // bf16: sum of the terms; e4m3: 2^-8 (t1 + 2^-4 t2 + 2^-8 t3)
                            const float tw = FP8 ? (q == 0 ? 0.00390625f : (q == 1 ? 0.000244140625f : 1.52587890625e-05f))
                                                 : 1.f;
                            z[col - q * RH] = FP8 ? fmaf(v[i], tw, z[col - q * RH]) : z[col - q * RH] + v[i];
                        }
                    }
                }
                tc_fence_before();
            } else {
#pragma unroll
                for (int r = 0; r < RH; ++r) z[r] = 0.f;
            }
            mbar_arrive(&sh->acce[a]);
            const int kk = k0 + t;
            if (p.Y && got && valid) {
                // keep Z_kk (the slice scale applied): the mode-3 tail contracts it with the new factor
                const float sc = FP8 ? p.sscale[(long long)rep * p.Kp + kk] : 1.f;
                float4 *y = reinterpret_cast<float4 *>(p.Y + rep * p.yrs + ((long long)kk * p.NP + pidx) * p.pr);
#pragma unroll
                for (int r4 = 0; r4 < RH; r4 += 4)
                    if (r4 < p.pr) y[r4 / 4] = make_float4(z[r4] * sc, z[r4 + 1] * sc, z[r4 + 2] * sc, z[r4 + 3] * sc);
            }
            // after an abort every remaining wait returns at once; the loop
            // runs to its end so that all 128 threads meet the same barriers
            if (p.epi == 0) {
                if (valid) {
                    const float *c = wst + t * RH;
#pragma unroll
                    for (int r = 0; r < RH; ++r)
                        if (r < R) acc[r] = fmaf(z[r], c[r], acc[r]);
                }
            } else {
#pragma unroll
                for (int r = 0; r < RH; ++r) {
                    float v = warp_sum(valid ? z[r] * arow[r] : 0.f);  // rows past the tile hold no data
                    if (lane == 0) sh->red[quarter][r] = v;
                }
                epi_bar();
                if (etid < R && *abort_flag != 2) {
                    float s = ((sh->red[0][etid] + sh->red[1][etid]) + sh->red[2][etid]) + sh->red[3][etid];
                    if (FP8) s *= p.sscale[(long long)rep * p.Kp + kk];
                    part[((long long)pb * p.Kp + kk) * p.pr + etid] = s;
                }
                epi_bar();
            }
        }
        const bool skipped = *abort_flag == 2;
        if (p.epi == 0 && valid && !skipped) {
#pragma unroll
            for (int r = 0; r < RH; ++r)
                if (r < R) part[((long long)ks * p.NP + pidx) * p.pr + r] = acc[r];
        }
        if (p.bytes_ctr && etid == 0 && !skipped) {
            const int rows = min(p.br, p.NP - pb * p.br);
            // summary bytes read (the products a memoised mode-2 pass keeps
            // are an intermediate that stays in L2, not counted)
            atomicAdd(p.bytes_ctr, (unsigned long long)rows * p.NC * (FP8 ? 1ull : 2ull) * nsl * (1 + p.split));
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TS));
    }
}

// ---------------------------------------------------------------------------
// Transposed copy of bfloat16 summaries: Y[s][j][i] = X[s][i][j] (64 x 64 tiles)
__global__ void __launch_bounds__(256) k_transpose_bf16(const __nv_bfloat16 *X, __nv_bfloat16 *Y, int NI, int NJ,
                                                       int ldx, int ldy) {
    __shared__ __nv_bfloat16 tile[64][66];
    const long long s = blockIdx.z;
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    const __nv_bfloat16 *xs = X + s * NI * (long long)ldx;
    __nv_bfloat16 *ys = Y + s * NJ * (long long)ldy;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 x 4
    for (int i = ty; i < 64; i += 4) {
        const int gi = i0 + i, gj = j0 + tx;
        tile[i][tx] = (gi < NI && gj < NJ) ? xs[(long long)gi * ldx + gj] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int j = ty; j < 64; j += 4) {
        const int gj = j0 + j, gi = i0 + tx;
        if (gj < NJ && gi < NI) ys[(long long)gj * ldy + gi] = tile[tx][j];
    }
}

// ---------------------------------------------------------------------------
// host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

// Rows per tile: ceil(NP / 128) tiles of equal height (rounded up to a
// multiple of 8, the swizzle atom), so every CTA streams the same bytes.
int tc_box_rows(int NP) {
    const int npb = (NP + TC_M - 1) / TC_M;
    const int br = (NP + npb - 1) / npb;
    return std::min(TC_M, (br + 7) / 8 * 8);
}

// 3-D map over [slices][NP][ld] bfloat16 (or float8 codes), box of one
// 128-byte row (64 or 128 elements) x tc_box_rows(NP) x 1, 128-byte swizzle,
// zero fill outside (columns >= NC, rows >= NP).
cudaError_t make_summary_tmap(CUtensorMap *m, const void *base, int NC, int NP, int ld, long long nslices,
                              bool fp8) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int es = fp8 ? 1 : 2;
    if (((uintptr_t)base & 15) || (ld * es) % 16) return cudaErrorInvalidValue;
    cuuint64_t dims[3] = {(cuuint64_t)NC, (cuuint64_t)NP, (cuuint64_t)nslices};
    cuuint64_t strides[2] = {(cuuint64_t)ld * es, (cuuint64_t)NP * ld * es};
    cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)tc_box_rows(NP), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                     const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// B operand columns: terms of RH = 16 or 32 columns; three (e4m3, or bf16 up
// to R = 16) or two (bf16 above R = 16)
static int tc_rh_of(int R) { return R <= 16 ? 16 : 32; }
static int tc_n_of(int R, bool fp8) { return (fp8 || R <= 16 ? 3 : 2) * tc_rh_of(R); }
static int tc_nkb_of(int NC, bool fp8) { return (NC + (fp8 ? 127 : 63)) / (fp8 ? 128 : 64); }

static size_t tc_fixed_smem(int nkb, int N, int RH) {
    return 1024 + (size_t)nkb * N * 128 + sizeof(TcShared) + (size_t)TC_MAX_SPC * RH * sizeof(float);
}

bool tc_supported(int R, int NC, bool fp8) {
    return R <= 32 && (size_t)tc_nkb_of(NC, fp8) * tc_n_of(R, fp8) * 128 <= 96 * 1024;
}

// ---------------------------------------------------------------------------
// Tile choices: CTAs per SM (1 or 2) and pipeline stages for one launch shape,
// process-wide; filled by the autotuner (or imported), else the default rule.
namespace {
struct TileKey {
    int fp8, R, NP, NC, Kb, nrep, epi;
    bool operator<(const TileKey &o) const {
        return std::tie(fp8, R, NP, NC, Kb, nrep, epi) < std::tie(o.fp8, o.R, o.NP, o.NC, o.Kb, o.nrep, o.epi);
    }
};
std::mutex g_tile_mu;
std::map<TileKey, TileChoice> g_tiles;
TileKey tile_key(bool fp8, int R, int NP, int NC, int Kp, int nrep, int epi) {
    return TileKey{fp8 ? 1 : 0, R, NP, NC, (Kp + 31) / 32, nrep, epi};
}
}  // namespace

TileChoice tile_choice(bool fp8, int R, int NP, int NC, int Kp, int nrep, int epi) {
    std::lock_guard<std::mutex> lock(g_tile_mu);
    auto it = g_tiles.find(tile_key(fp8, R, NP, NC, Kp, nrep, epi));
    return it == g_tiles.end() ? TileChoice{2, 0} : it->second;
}

bool tile_known(bool fp8, int R, int NP, int NC, int Kp, int nrep, int epi) {
    std::lock_guard<std::mutex> lock(g_tile_mu);
    return g_tiles.count(tile_key(fp8, R, NP, NC, Kp, nrep, epi)) != 0;
}

void tile_store(bool fp8, int R, int NP, int NC, int Kp, int nrep, int epi, TileChoice c) {
    std::lock_guard<std::mutex> lock(g_tile_mu);
    g_tiles[tile_key(fp8, R, NP, NC, Kp, nrep, epi)] = c;
}

// entries [fp8, R, NP, NC, Kb, nrep, epi, per_sm, stages] x n
int tile_table_read(int *out, int cap) {
    std::lock_guard<std::mutex> lock(g_tile_mu);
    int n = 0;
    for (const auto &kv : g_tiles) {
        if (n < cap) {
            int *e = out + 9 * n;
            const TileKey &k = kv.first;
            e[0] = k.fp8; e[1] = k.R; e[2] = k.NP; e[3] = k.NC; e[4] = k.Kb; e[5] = k.nrep; e[6] = k.epi;
            e[7] = kv.second.per_sm;
            e[8] = kv.second.stages;
        }
        ++n;
    }
    return n;
}

void tile_table_merge(const int *in, int n) {
    std::lock_guard<std::mutex> lock(g_tile_mu);
    for (int q = 0; q < n; ++q) {
        const int *e = in + 9 * q;
        g_tiles[TileKey{e[0], e[1], e[2], e[3], e[4], e[5], e[6]}] = TileChoice{e[7], e[8]};
    }
}

void tile_table_clear() {
    std::lock_guard<std::mutex> lock(g_tile_mu);
    g_tiles.clear();
}

// Work split for one mode: CTAs = nrep x npb x nks, about per_sm per SM.
void tc_tiles(int nrep, int NP, int Kp, int num_sms, int per_sm, int *npb, int *nks, int *spc) {
    *npb = (NP + TC_M - 1) / TC_M;
    // one wave at per_sm CTAs per SM, less one slot per repetition for the
    // V^-1 kernel that runs beside the pass (a full grid would push CTAs
    // into a second wave behind it)
    long long target = (long long)per_sm * num_sms - nrep;
    long long n = target / std::max(1LL, (long long)nrep * *npb);
    n = std::max(1LL, std::min<long long>(n, Kp));
    *spc = std::min(TC_MAX_SPC, (int)((Kp + n - 1) / n));
    *nks = (Kp + *spc - 1) / *spc;
}

void tc_plan(bool fp8, int R, int nrep, int NP, int NC, int Kp, int epi, int num_sms, int *npb, int *nks,
             int *spc) {
    const TileChoice c = tile_choice(fp8, R, NP, NC, Kp, nrep, epi);
    tc_tiles(nrep, NP, Kp, num_sms, c.per_sm, npb, nks, spc);
}

cudaError_t launch_mttkrp_tc(const CUtensorMap &tmap, const CUtensorMap *tmap_lo, int epi, int nrep, int R, int NP,
                             int NC, int Kp,
                             const float *F, long long frs, const float *W, long long wrs, float *part, long long prs,
                             int pr,
                             const int *conv, unsigned long long *bytes_ctr, unsigned *err, const float *sscale,
                             int num_sms, int *P_out, cudaStream_t st, float *Y, long long yrs,
                             const TileChoice *force) {
    const bool fp8 = sscale != nullptr;
    const TileChoice tch = force ? *force : tile_choice(fp8, R, NP, NC, Kp, nrep, epi);
    TcParams p{};
    p.nrep = nrep;
    p.R = R;
    p.NP = NP;
    p.NC = NC;
    p.Kp = Kp;
    p.nkb = tc_nkb_of(NC, fp8);
    p.sscale = sscale;
    tc_tiles(nrep, NP, Kp, num_sms, tch.per_sm, &p.npb, &p.nks, &p.spc);
    p.br = tc_box_rows(NP);
    p.split = tmap_lo ? 1 : 0;
    const CUtensorMap &lo = tmap_lo ? *tmap_lo : tmap;
    p.epi = epi;
    p.F = F;
    p.frs = frs;
    p.W = W;
    p.wrs = wrs;
    p.part = part;
    p.prs = prs;
    p.pr = pr;
    p.conv = conv;
    p.bytes_ctr = bytes_ctr;
    p.err = err;
    p.Y = epi == 0 ? Y : nullptr;
    p.yrs = yrs;
    const int N = tc_n_of(R, fp8);
    const size_t budget = tch.per_sm == 1 ? 220 * 1024 : 110 * 1024;
    const size_t fixed = tc_fixed_smem(p.nkb, N, tc_rh_of(R));
    int stages = (int)std::min<size_t>(8, (budget > fixed ? (budget - fixed) : 0) / TC_BOX_BYTES);
    if (tch.stages > 0) stages = std::min(stages, tch.stages);
    p.stages = std::max(2, stages);
    const size_t smem = fixed + (size_t)p.stages * TC_BOX_BYTES;
    *P_out = epi == 0 ? p.nks : p.npb;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p.npb * p.nks, nrep);
    cfg.blockDim = dim3(192);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launches(1);
    if (!fp8) return N == 48 ? cudaLaunchKernelEx(&cfg, k_mtt_tc<48, false>, tmap, lo, p)
                             : cudaLaunchKernelEx(&cfg, k_mtt_tc<64, false>, tmap, lo, p);
    return N == 48 ? cudaLaunchKernelEx(&cfg, k_mtt_tc<48, true>, tmap, lo, p)
                   : cudaLaunchKernelEx(&cfg, k_mtt_tc<96, true>, tmap, lo, p);
}

// Raise the dynamic shared-memory limit of the tensor-core kernels once,
// outside any stream capture.
template <int N, bool FP8>
static cudaError_t tc_attributes() {
    cudaError_t e = cudaFuncSetAttribute(k_mtt_tc<N, FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    // the largest shared-memory carveout, as for the tails around it, so that
    // the SM is not reconfigured at every kernel boundary of the ALS chain
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mtt_tc<N, FP8>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

cudaError_t set_tc_kernel_attributes() {
    cudaError_t e = tc_attributes<48, false>();
    if (e == cudaSuccess) e = tc_attributes<64, false>();
    if (e == cudaSuccess) e = tc_attributes<48, true>();
    if (e == cudaSuccess) e = tc_attributes<96, true>();
    return e;
}

cudaError_t launch_transpose_bf16(const void *X, void *Y, int NI, int NJ, int ldx, int ldy, long long nslices,
                                  cudaStream_t st) {
    for (long long s0 = 0; s0 < nslices; s0 += 65535) {
        const long long ns = std::min<long long>(65535, nslices - s0);
        dim3 grid((NJ + 63) / 64, (NI + 63) / 64, (unsigned)ns);
        count_launches(1);
        k_transpose_bf16<<<grid, 256, 0, st>>>((const __nv_bfloat16 *)X + s0 * NI * (long long)ldx,
                                               (__nv_bfloat16 *)Y + s0 * NJ * (long long)ldy, NI, NJ, ldx, ldy);
    }
    return cudaGetLastError();
}

}  // namespace sbt
