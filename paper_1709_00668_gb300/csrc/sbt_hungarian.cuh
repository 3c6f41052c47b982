// Maximum-weight assignment used by the matching step (Lemma 1 and
// Algorithm 1 step 7) of the 3-mode and the order-N updates.
#pragma once

#include <cuda_runtime.h>

namespace sbt {

// Maximum-weight assignment of an nr x nc score matrix, nr <= nc: every row
// to a distinct column (Hungarian method, shortest augmenting paths with
// potentials; Kuhn 1955, Munkres 1957), single thread.  perm[row] = column.
// Ties resolve to the lower column index.  nr = nc is the perfect matching of
// Lemma 1's square case; nr < nc is GetRank's R_new summary components
// against R old ones.
struct HungarianWork {
    double u[33], v[33], minv[33];
    int p[33], way[33];
    bool used[33];
};

__device__ inline void hungarian_max(const double *score, int ld, int nr, int nc, int *perm, HungarianWork &w) {
    double *u = w.u, *v = w.v, *minv = w.minv;
    int *p = w.p, *way = w.way;
    bool *used = w.used;
    for (int j = 0; j <= nc; ++j) {
        v[j] = 0.0;
        p[j] = 0;
        way[j] = 0;
    }
    for (int i = 0; i <= nr; ++i) u[i] = 0.0;
    for (int i = 1; i <= nr; ++i) {
        p[0] = i;
        int j0 = 0;
        for (int j = 0; j <= nc; ++j) {
            minv[j] = INFINITY;
            used[j] = false;
        }
        // each pass marks one more column used, so at most nc passes
        for (int guard = 0; guard <= nc; ++guard) {
            used[j0] = true;
            const int i0 = p[j0];
            double delta = INFINITY;
            int j1 = 0;
            for (int j = 1; j <= nc; ++j) {
                if (used[j]) continue;
                double sc = score[(i0 - 1) * ld + (j - 1)];
                if (!isfinite(sc)) sc = 0.0;
                const double cur = -sc - u[i0] - v[j];
                if (cur < minv[j]) {
                    minv[j] = cur;
                    way[j] = j0;
                }
                if (minv[j] < delta) {
                    delta = minv[j];
                    j1 = j;
                }
            }
            for (int j = 0; j <= nc; ++j) {
                if (used[j]) {
                    u[p[j]] += delta;
                    v[j] -= delta;
                } else {
                    minv[j] -= delta;
                }
            }
            if (j1 == 0) break;  // no free column reachable (cannot happen for finite scores)
            j0 = j1;
            if (p[j0] == 0) break;
        }
        for (int guard = 0; guard <= nc && j0; ++guard) {
            const int j1 = way[j0];
            p[j0] = p[j1];
            j0 = j1;
        }
    }
    // rows that no column took (cannot happen for finite scores) take the
    // free columns in order
    bool row_done[33], col_used[33];
    for (int i = 0; i <= nr; ++i) row_done[i] = false;
    for (int j = 0; j <= nc; ++j) col_used[j] = false;
    for (int i = 0; i < nr; ++i) perm[i] = -1;
    for (int j = 1; j <= nc; ++j)
        if (p[j] >= 1 && p[j] <= nr && !row_done[p[j]]) {
            row_done[p[j]] = true;
            col_used[j] = true;
            perm[p[j] - 1] = j - 1;
        }
    for (int i = 1; i <= nr; ++i)
        if (!row_done[i])
            for (int j = 1; j <= nc; ++j)
                if (!col_used[j]) {
                    col_used[j] = true;
                    perm[i - 1] = j - 1;
                    break;
                }
}

}  // namespace sbt
