/*
 * Oracle: integer sampling primitives of SamBaTen (arxiv 1709.00668).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg are its only users.  It shares no code with the CUDA path.
 *
 * Section 3.1 ("Sample") and Algorithm 1, step 3: each mode is sampled
 * without replacement with probabilities proportional to its measure of
 * importance (Eq. 1).  The oracle realises that draw as successive sampling
 * through exponential keys (Efraimidis & Spirakis, "Weighted random sampling
 * with a reservoir", IPL 2006): with u ~ U(0,1), key = -log(u) / w; the n
 * smallest keys are a draw of n items without replacement, each step picking
 * among the remaining items with probability proportional to w.
 *
 * Everything is integer so the CPU and GPU reach the same bits:
 *   - u comes from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 *     numbers: as easy as 1, 2, 3", SC'11), written from that paper;
 *   - -log2(u) is a Q.32 fixed-point number from the shift-and-square binary
 *     logarithm (Turner, "A Fast Binary Logarithm Algorithm", IEEE Signal
 *     Processing Magazine, 2010), every step truncating;
 *   - the key is floor(L * 2^64 / w) as an unsigned 128-bit integer.
 * Ties between equal keys go to the smaller index.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ---- Philox4x32-10 (Salmon et al. 2011) --------------------------------- */
static const uint32_t PHILOX_MUL_A = 0xD2511F53u; /* multiplies counter word 0 */
static const uint32_t PHILOX_MUL_B = 0xCD9E8D57u; /* multiplies counter word 2 */
static const uint32_t PHILOX_WEYL_0 = 0x9E3779B9u; /* key schedule increments */
static const uint32_t PHILOX_WEYL_1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { /* the key is bumped before every round but the first */
            k0 += PHILOX_WEYL_0;
            k1 += PHILOX_WEYL_1;
        }
        uint64_t pa = (uint64_t)PHILOX_MUL_A * x0;
        uint64_t pb = (uint64_t)PHILOX_MUL_B * x2;
        uint32_t y0 = (uint32_t)(pb >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)pb;
        uint32_t y2 = (uint32_t)(pa >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)pa;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Batch form for the Python wrapper: ctr is n x 4, out is n x 4. */
void orc_philox_batch(const uint32_t *ctr, const uint32_t key[2], uint32_t *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* ---- fixed-point binary logarithm (Turner 2010) -------------------------- */
/* For 1 <= t < 2^33, returns floor-ish log2(t) in Q.32: integer part p in the
 * upper bits, 32 fraction bits f.  y = t / 2^p in [1,2) is held as Q1.62; each
 * step squares y (128-bit product, truncated back to Q2.62); a square >= 2
 * yields fraction bit 1 and is halved. */
uint64_t orc_log2_q32(uint64_t t)
{
    int p = 63 - __builtin_clzll(t);
    uint64_t y = t << (62 - p);
    uint64_t f = 0;
    for (int b = 0; b < 32; ++b) {
        u128 sq = (u128)y * (u128)y;
        y = (uint64_t)(sq >> 62);
        f <<= 1;
        if (y >> 63) {
            f |= 1u;
            y >>= 1;
        }
    }
    return ((uint64_t)p << 32) | f;
}

void orc_log2_batch(const uint64_t *t, uint64_t *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_log2_q32(t[i]);
}

/* ---- exponential key ------------------------------------------------------ */
/* v is one uniform 32-bit word; u = (2v+1)/2^33 lies strictly inside (0,1).
 * L = -log2(u) in Q.32 = 33*2^32 - log2_q32(2v+1) >= 1.  key = floor(L*2^64/w). */
static u128 es_key(uint32_t v, uint64_t w)
{
    uint64_t t = 2u * (uint64_t)v + 1u;
    uint64_t L = ((uint64_t)33 << 32) - orc_log2_q32(t);
    return ((u128)L << 64) / (u128)w;
}

void orc_es_key_batch(const uint32_t *v, const uint64_t *w, uint64_t *hi, uint64_t *lo, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        u128 k = es_key(v[i], w[i]);
        hi[i] = (uint64_t)(k >> 64);
        lo[i] = (uint64_t)k;
    }
}

/* ---- one mode's draw ------------------------------------------------------ */
/* Philox stream of the sampling draw: key = (lo32(seed), hi32(seed) ^ stream_id),
 * counter = (x, mode | rep << 4, batch, 1); word 0 is v. */
typedef struct { u128 key; int64_t x; } keyed;

static int cmp_keyed(const void *pa, const void *pb)
{
    const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->x < b->x) ? -1 : (a->x > b->x);
}

static int cmp_i32(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return (a > b) - (a < b);
}

/* Draw n of the N indices whose weight w[x] is positive, without replacement,
 * with probability proportional to w; write them ascending to out.
 * Returns n, or -1 if n exceeds the number of positive weights. */
int64_t orc_sample_mode(const uint64_t *w, int64_t N, int64_t n, uint64_t seed,
                        uint32_t stream_id, uint32_t mode, uint32_t rep, uint32_t batch,
                        int32_t *out)
{
    keyed *cand = (keyed *)malloc(sizeof(keyed) * (size_t)(N > 0 ? N : 1));
    int64_t m = 0;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ stream_id};
    for (int64_t x = 0; x < N; ++x) {
        if (w[x] == 0) continue;
        uint32_t ctr[4] = {(uint32_t)x, mode | (rep << 4), batch, 1u}, r[4];
        orc_philox4x32_10(ctr, key, r);
        cand[m].key = es_key(r[0], w[x]);
        cand[m].x = x;
        ++m;
    }
    if (n > m) { free(cand); return -1; }
    qsort(cand, (size_t)m, sizeof(keyed), cmp_keyed);
    for (int64_t t = 0; t < n; ++t) out[t] = (int32_t)cand[t].x;
    qsort(out, (size_t)n, sizeof(int32_t), cmp_i32);
    free(cand);
    return n;
}
