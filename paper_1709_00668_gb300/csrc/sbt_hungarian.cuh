// Maximum-weight assignment used by the matching step (Lemma 1 and
// Algorithm 1 step 7) of the 3-mode and the order-N updates.
#pragma once

#include <cuda_runtime.h>

namespace sbt {

// Maximum-weight assignment of an nr x nc score matrix, nr <= nc <= 32:
// every row to a distinct column (Hungarian method, shortest augmenting
// paths with potentials; Kuhn 1955, Munkres 1957).  perm[row] = column.  Ties
// resolve to the lower column index.  nr = nc is the perfect matching of
// Lemma 1's square case; nr < nc is GetRank's R_new summary components
// against R old ones.
//
// One warp: lane c owns column c + 1 (its potential v, its slack minv, its
// "used" mark, its row p and its predecessor way); column 0 is the method's
// virtual column.  Each pass of a row is one step of the warp: every free
// column updates its slack from the row just reached, the warp takes the
// smallest slack (first column on ties) by shuffles, and every column
// updates its potential or slack by that amount.  Per entry these are the
// operations, in the order, of the textbook single-thread loop, so the
// result is the same; only the loop over columns runs across the lanes.  The
// float64 chain a row waits for is one pass per column reached instead of
// one pass times nc (float64 is a slow, long-latency unit on this GPU).
// Call from all 32 lanes of one converged warp; w in shared memory.
// Order-preserving map of a non-NaN double to an unsigned 64-bit key
// (negative values: all bits flipped; others: the sign bit set).
__device__ __forceinline__ unsigned long long order_key(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

struct HungarianWork {
    double u[33];  // row potentials (row 0 unused)
    int p[33], way[33];
};

__device__ inline void hungarian_max_warp(const double *score, int ld, int nr, int nc, int *perm, HungarianWork &w,
                                          int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    double *u = w.u;
    int *p = w.p, *way = w.way;
    const int j = lane + 1;
    const bool col = j <= nc;
    double vj = 0.0, minv = INFINITY;
    int pj = 0, wayj = 0;
    for (int i = lane; i <= nr; i += 32) u[i] = 0.0;
    __syncwarp();
    for (int i = 1; i <= nr; ++i) {
        const int p0 = i;  // the virtual column holds the row being placed
        int j0 = 0;
        bool used = false;
        minv = INFINITY;
        // each pass marks one more column used, so at most nc passes
        for (int guard = 0; guard <= nc; ++guard) {
            if (j0 == j) used = true;
            const int i0 = j0 == 0 ? p0 : __shfl_sync(FULL, pj, j0 - 1);
            const double ui0 = u[i0];
            double cand = INFINITY;
            if (col && !used) {
                double sc = score[(i0 - 1) * ld + (j - 1)];
                if (!isfinite(sc)) sc = 0.0;
                const double cur = -sc - ui0 - vj;
                if (cur < minv) {
                    minv = cur;
                    wayj = j0;
                }
                cand = minv;
            }
            // the smallest slack strictly below +inf, the first column on
            // ties: compared as order-preserving 64-bit keys (integer pipes;
            // -0 taken as +0 so that equal values give equal keys)
            const bool fin = cand < INFINITY;
            const double cz = cand == 0.0 ? 0.0 : cand;
            unsigned long long key = fin ? order_key(cz) : ~0ull;
            int dj = fin ? j : 0x7fffffff;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(FULL, key, o);
                const int oj = __shfl_xor_sync(FULL, dj, o);
                if (ok < key || (ok == key && oj < dj)) {
                    key = ok;
                    dj = oj;
                }
            }
            const int j1 = dj == 0x7fffffff ? 0 : dj;
            const double delta = j1 == 0 ? INFINITY : __shfl_sync(FULL, cand, j1 - 1);
            __syncwarp();  // every lane has read u[i0]
            // used columns hold distinct rows (and the virtual column the row
            // being placed), so no two lanes update the same potential
            if (col) {
                if (used) {
                    u[pj] += delta;
                    vj -= delta;
                } else {
                    minv -= delta;
                }
            }
            if (lane == 0) u[p0] += delta;
            __syncwarp();
            if (j1 == 0) break;  // no free column reachable (cannot happen for finite scores)
            j0 = j1;
            if (__shfl_sync(FULL, pj, j0 - 1) == 0) break;
        }
        // augment along the predecessors, from the free column reached back
        // to the virtual one
        if (col) {
            p[j] = pj;
            way[j] = wayj;
        }
        if (lane == 0) p[0] = p0;
        __syncwarp();
        if (lane == 0)
            for (int guard = 0; guard <= nc && j0; ++guard) {
                const int j1 = way[j0];
                p[j0] = p[j1];
                j0 = j1;
            }
        __syncwarp();
        if (col) pj = p[j];
    }
    if (lane == 0) {
        // rows that no column took (cannot happen for finite scores) take
        // the free columns in order
        bool row_done[33], col_used[33];
        for (int i = 0; i <= nr; ++i) row_done[i] = false;
        for (int c = 0; c <= nc; ++c) col_used[c] = false;
        for (int i = 0; i < nr; ++i) perm[i] = -1;
        for (int c = 1; c <= nc; ++c)
            if (p[c] >= 1 && p[c] <= nr && !row_done[p[c]]) {
                row_done[p[c]] = true;
                col_used[c] = true;
                perm[p[c] - 1] = c - 1;
            }
        for (int i = 1; i <= nr; ++i)
            if (!row_done[i])
                for (int c = 1; c <= nc; ++c)
                    if (!col_used[c]) {
                        col_used[c] = true;
                        perm[i - 1] = c - 1;
                        break;
                    }
    }
    __syncwarp();
}

}  // namespace sbt
