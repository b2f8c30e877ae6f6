/*
 * Seeded synthetic graph generators for the walk-Laplacian workloads.
 *
 * Input generation only: nothing here evaluates a walk-generating function,
 * a Laplacian or a Krylov method. Both the CPU oracle and the CUDA library
 * consume the CSR arrays this file produces.
 *
 * Randomness comes from a counter-based hash (SplitMix64, Steele, Lea and
 * Flood, OOPSLA 2014): draw(seed, stream, i) depends only on its arguments,
 * so results are identical for any thread count and on x86 and Arm.
 *
 * Build: gcc -O3 -fopenmp -fPIC -shared (no architecture flags).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t i) {
    return mix64(mix64(seed ^ mix64(stream * 0x632BE59BD9B4E019ull)) + i);
}

/* uniform in [0,1) with 53 random bits */
static inline double unif(uint64_t seed, uint64_t stream, uint64_t i) {
    return (double)(draw(seed, stream, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* R-MAT edge list (Chakrabarti, Zhan, Faloutsos 2004): each of the m edges
 * descends `scale` levels choosing quadrant a | b | c | d. Vertex ids are then
 * relabelled by a seeded Fisher-Yates permutation (done by the caller via
 * wlgen_permutation) so that hubs are not clustered at low ids. */
int wlgen_rmat_edges(int scale, int64_t m, double a, double b, double c,
                     uint64_t seed, int32_t *src, int32_t *dst) {
    if (scale < 1 || scale > 30 || m < 0) return -1;
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint32_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            double r = unif(seed, 1, (uint64_t)e * 64u + (uint64_t)l);
            uint32_t bu, bv;
            if (r < a) { bu = 0; bv = 0; }
            else if (r < ab) { bu = 0; bv = 1; }
            else if (r < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        src[e] = (int32_t)u;
        dst[e] = (int32_t)v;
    }
    return 0;
}

/* Seeded Fisher-Yates permutation of 0..n-1 (sequential, O(n)). */
int wlgen_permutation(int64_t n, uint64_t seed, int32_t *perm) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        uint64_t r = draw(seed, 2, (uint64_t)i);
        int64_t j = (int64_t)(r % (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    return 0;
}

/* Apply a vertex relabelling in place: x -> perm[x]. */
int wlgen_relabel(int64_t m, const int32_t *perm, int32_t *src, int32_t *dst) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        src[e] = perm[src[e]];
        dst[e] = perm[dst[e]];
    }
    return 0;
}

/* Chung-Lu graph with expected degrees w (Miller and Hagberg 2011 skipping
 * sampler). Nodes must be given in non-increasing weight order through
 * `order` (order[r] = node of rank r). For each rank u, candidate partners
 * v > u are visited with geometric skips under the bound p = w_u w_v / S,
 * accepted with ratio q/p. Each u uses its own counter stream, so rows are
 * independent and the loop is parallel. Edges are written as (u, v) pairs
 * into per-u slots sized by `cap` (an upper bound computed by the caller);
 * returns the number of edges through *m_out, compacted. */
int wlgen_chung_lu_edges(int64_t n, const double *w, const int32_t *order,
                         uint64_t seed, int64_t cap, int32_t *src, int32_t *dst,
                         int64_t *m_out) {
    double S = 0.0;
    for (int64_t i = 0; i < n; ++i) S += w[i];
    if (!(S > 0.0)) { *m_out = 0; return 0; }
    /* two passes: count per u, then fill with a prefix offset */
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -2;
    for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t ru = 0; ru < n - 1; ++ru) {
            int64_t u = order[ru];
            double wu = w[u];
            int64_t rv = ru + 1;
            double p = wu * w[order[rv]] / S;
            if (p > 1.0) p = 1.0;
            uint64_t ctr = 0;
            int64_t k = 0;
            int64_t off = pass ? cnt[ru] : 0;
            while (rv < n && p > 0.0) {
                if (p < 1.0) {
                    double r = unif(seed, 3, ((uint64_t)ru << 32) + ctr++);
                    /* geometric skip */
                    double lr = log(1.0 - r) / log(1.0 - p);
                    if (lr > (double)(n)) break;
                    rv += (int64_t)floor(lr);
                }
                if (rv < n) {
                    double q = wu * w[order[rv]] / S;
                    if (q > 1.0) q = 1.0;
                    double r2 = unif(seed, 4, ((uint64_t)ru << 32) + ctr++);
                    if (r2 < q / p) {
                        if (pass) {
                            src[off + k] = (int32_t)u;
                            dst[off + k] = order[rv];
                        }
                        ++k;
                    }
                    p = q;
                    ++rv;
                }
            }
            if (!pass) cnt[ru] = k;
        }
        if (!pass) {
            int64_t run = 0;
            for (int64_t i = 0; i < n; ++i) { int64_t t = cnt[i]; cnt[i] = run; run += t; }
            cnt[n] = run;
            if (run > cap) { free(cnt); *m_out = run; return -3; }
        }
    }
    *m_out = cnt[n];
    free(cnt);
    return 0;
}

/* Build a simple undirected CSR from an edge list: each (u,v) with u != v
 * contributes u->v and v->u; duplicate entries are merged; self-loops are
 * dropped; column indices are sorted within each row. Two calls: with
 * col_idx == NULL it only fills row_ptr (n+1 entries) with the upper bound
 * of entries per row before deduplication and returns the bound total in
 * *nnz_out; the second call (col_idx sized by that bound) fills, sorts,
 * dedupes and rewrites row_ptr to the final counts. */
static int cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

int wlgen_csr_count(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                    int64_t *row_ptr, int64_t *nnz_out) {
    memset(row_ptr, 0, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = src[e], v = dst[e];
        if (u == v || u < 0 || v < 0 || u >= n || v >= n) continue;
        row_ptr[u + 1]++;
        row_ptr[v + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
    *nnz_out = row_ptr[n];
    return 0;
}

int wlgen_csr_fill(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                   int64_t *row_ptr, int32_t *col_idx, int64_t *nnz_out) {
    int64_t *fillp = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!fillp) return -2;
    memcpy(fillp, row_ptr, sizeof(int64_t) * (size_t)n);
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = src[e], v = dst[e];
        if (u == v || u < 0 || v < 0 || u >= n || v >= n) continue;
        col_idx[fillp[u]++] = v;
        col_idx[fillp[v]++] = u;
    }
    free(fillp);
    /* sort + unique per row, record new lengths */
    int64_t *len = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!len) return -2;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        int32_t *row = col_idx + row_ptr[i];
        int64_t L = row_ptr[i + 1] - row_ptr[i];
        if (L > 1) qsort(row, (size_t)L, sizeof(int32_t), cmp_i32);
        int64_t k = 0;
        for (int64_t t = 0; t < L; ++t)
            if (k == 0 || row[t] != row[k - 1]) row[k++] = row[t];
        len[i] = k;
    }
    /* compact in place (rows only move left) */
    int64_t out = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t beg = row_ptr[i];
        if (out != beg) memmove(col_idx + out, col_idx + beg, sizeof(int32_t) * (size_t)len[i]);
        row_ptr[i] = out;
        out += len[i];
    }
    row_ptr[n] = out;
    free(len);
    *nnz_out = out;
    return 0;
}

/* Uniform doubles for the caller-side recipes (weights, sources). */
int wlgen_uniform(int64_t count, uint64_t seed, uint64_t stream, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) out[i] = unif(seed, 100 + stream, (uint64_t)i);
    return 0;
}
