/*
 * Seeded synthetic graph generators (input synthesis only).
 *
 * Every generator returns an undirected graph as a CSR adjacency structure:
 * symmetric, loop-free, without duplicate edges, each row sorted by column.
 * This is the class of matrices the paper works with (Section 2.1: symmetric,
 * binary, zero diagonal).  Isolated nodes are kept.
 *
 * This file holds no arithmetic of the Monte Carlo method: it only draws
 * graphs.  Its random numbers come from a counter-based splitmix64 mix of
 * (seed, stream, index), so the output is independent of the OpenMP thread
 * count and identical on every host.
 *
 * Shapes follow the paper's workloads (Table 1: smallworld = Watts-Strogatz,
 * kronecker = Graph500 R-MAT) and the synthetic stand-ins for its real
 * networks: Barabasi-Albert, Erdos-Renyi and an erased configuration model
 * with a power-law degree sequence.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n;
    int64_t nnz;
    int64_t* row_ptr; /* n + 1 */
    int32_t* col_idx; /* nnz */
} gg_graph;

/* ---- counter-based random numbers (splitmix64 finaliser) ---- */
static inline uint64_t gg_mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline uint64_t gg_rand(uint64_t seed, uint64_t stream, uint64_t i) {
    return gg_mix(gg_mix(seed ^ gg_mix(stream * 0xD1B54A32D192ED03ull)) + i);
}
static inline double gg_u01(uint64_t seed, uint64_t stream, uint64_t i) {
    return (double)(gg_rand(seed, stream, i) >> 11) * (1.0 / 9007199254740992.0);
}
/* uniform integer in [0, m) */
static inline uint64_t gg_below(uint64_t seed, uint64_t stream, uint64_t i, uint64_t m) {
    return (uint64_t)(gg_u01(seed, stream, i) * (double)m) % m;
}

/* ---- edge list -> symmetric CSR ---- */
static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Builds the CSR of the undirected graph whose edges are (src[e], dst[e]).
 * Both directions are inserted, loops dropped, duplicates removed. */
static gg_graph* gg_build(int64_t n, int64_t m, const int32_t* src, const int32_t* dst) {
    gg_graph* g = (gg_graph*)calloc(1, sizeof(gg_graph));
    if (!g) return NULL;
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) { free(g); return NULL; }
    for (int64_t e = 0; e < m; ++e) {
        if (src[e] == dst[e]) continue;
        cnt[src[e] + 1]++;
        cnt[dst[e] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    int64_t tot = cnt[n];
    int32_t* col = (int32_t*)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int32_t));
    int64_t* pos = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!col || !pos) { free(cnt); free(col); free(pos); free(g); return NULL; }
    memcpy(pos, cnt, (size_t)n * sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = src[e], v = dst[e];
        if (u == v) continue;
        col[pos[u]++] = v;
        col[pos[v]++] = u;
    }
    free(pos);
    /* sort each row and count the distinct entries */
    int64_t* keep = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!keep) { free(cnt); free(col); free(g); return NULL; }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        int64_t b = cnt[i], e = cnt[i + 1];
        if (e - b > 1) qsort(col + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
        int64_t w = 0;
        for (int64_t p = b; p < e; ++p)
            if (w == 0 || col[b + w - 1] != col[p]) col[b + w++] = col[p];
        keep[i + 1] = w;
    }
    for (int64_t i = 0; i < n; ++i) keep[i + 1] += keep[i];
    int64_t nnz = keep[n];
    int32_t* out = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!out) { free(cnt); free(col); free(keep); free(g); return NULL; }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i)
        memcpy(out + keep[i], col + cnt[i], (size_t)(keep[i + 1] - keep[i]) * sizeof(int32_t));
    free(col);
    free(cnt);
    g->n = n;
    g->nnz = nnz;
    g->row_ptr = keep;
    g->col_idx = out;
    return g;
}

void gg_free(gg_graph* g) {
    if (!g) return;
    free(g->row_ptr);
    free(g->col_idx);
    free(g);
}
int64_t gg_n(const gg_graph* g) { return g->n; }
int64_t gg_nnz(const gg_graph* g) { return g->nnz; }
void gg_copy(const gg_graph* g, int64_t* row_ptr, int32_t* col_idx) {
    memcpy(row_ptr, g->row_ptr, (size_t)(g->n + 1) * sizeof(int64_t));
    if (g->nnz) memcpy(col_idx, g->col_idx, (size_t)g->nnz * sizeof(int32_t));
}

/* Random permutation of 0..n-1 (Fisher-Yates driven by the counter RNG). */
static int32_t* gg_perm(int64_t n, uint64_t seed, uint64_t stream) {
    int32_t* p = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!p) return NULL;
    for (int64_t i = 0; i < n; ++i) p[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)gg_below(seed, stream, (uint64_t)i, (uint64_t)(i + 1));
        int32_t t = p[i]; p[i] = p[j]; p[j] = t;
    }
    return p;
}

/*
 * R-MAT / Graph500 Kronecker generator: 2^scale nodes, edge_factor * 2^scale
 * directed edge draws; each draw descends `scale` levels choosing a quadrant
 * with probabilities (a, b, c, 1-a-b-c).  Node ids are randomly permuted when
 * `permute` is set (otherwise ids correlate with degree).
 */
gg_graph* gg_rmat(int scale, int edge_factor, double a, double b, double c, uint64_t seed, int permute) {
    int64_t n = (int64_t)1 << scale;
    int64_t m = (int64_t)edge_factor * n;
    int32_t* src = (int32_t*)malloc((size_t)m * sizeof(int32_t));
    int32_t* dst = (int32_t*)malloc((size_t)m * sizeof(int32_t));
    if (!src || !dst) { free(src); free(dst); return NULL; }
    double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        int64_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            double r = gg_u01(seed, 1, (uint64_t)e * (uint64_t)scale + (uint64_t)l);
            int bu, bv;
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
    if (permute) {
        int32_t* p = gg_perm(n, seed, 2);
        if (!p) { free(src); free(dst); return NULL; }
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < m; ++e) { src[e] = p[src[e]]; dst[e] = p[dst[e]]; }
        free(p);
    }
    gg_graph* g = gg_build(n, m, src, dst);
    free(src);
    free(dst);
    return g;
}

/*
 * Barabasi-Albert preferential attachment: start from the complete graph on
 * m + 1 nodes; every later node attaches to m distinct existing nodes chosen
 * with probability proportional to their degree.
 */
gg_graph* gg_ba(int64_t n, int m, uint64_t seed) {
    if (n < m + 1) return NULL;
    int64_t m0 = (int64_t)m + 1;
    int64_t edges = m0 * (m0 - 1) / 2 + (n - m0) * m;
    int32_t* src = (int32_t*)malloc((size_t)edges * sizeof(int32_t));
    int32_t* dst = (int32_t*)malloc((size_t)edges * sizeof(int32_t));
    int32_t* ends = (int32_t*)malloc((size_t)(2 * edges) * sizeof(int32_t));
    int32_t* pick = (int32_t*)malloc((size_t)m * sizeof(int32_t));
    if (!src || !dst || !ends || !pick) { free(src); free(dst); free(ends); free(pick); return NULL; }
    int64_t ne = 0, nends = 0;
    for (int64_t i = 0; i < m0; ++i)
        for (int64_t j = i + 1; j < m0; ++j) {
            src[ne] = (int32_t)i; dst[ne] = (int32_t)j; ++ne;
            ends[nends++] = (int32_t)i; ends[nends++] = (int32_t)j;
        }
    uint64_t draw = 0;
    for (int64_t v = m0; v < n; ++v) {
        int got = 0;
        while (got < m) {
            int32_t t = ends[gg_below(seed, 3, draw++, (uint64_t)nends)];
            int dup = 0;
            for (int q = 0; q < got; ++q) dup |= (pick[q] == t);
            if (!dup) pick[got++] = t;
        }
        for (int q = 0; q < m; ++q) {
            src[ne] = (int32_t)v; dst[ne] = pick[q]; ++ne;
            ends[nends++] = (int32_t)v; ends[nends++] = pick[q];
        }
    }
    gg_graph* g = gg_build(n, ne, src, dst);
    free(src); free(dst); free(ends); free(pick);
    return g;
}

/*
 * Erdos-Renyi G(n, p) with p = mean_degree / (n - 1), drawn by geometric
 * skipping over the pairs (i < j) in row-major order.
 */
gg_graph* gg_er(int64_t n, double mean_degree, uint64_t seed) {
    double p = n > 1 ? mean_degree / (double)(n - 1) : 0.0;
    if (p <= 0.0 || n < 2) { int32_t z = 0; return gg_build(n, 0, &z, &z); }
    if (p > 1.0) p = 1.0;
    int64_t cap = (int64_t)(p * (double)n * (double)(n - 1) / 2.0 * 1.1) + 1024;
    int32_t* src = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
    int32_t* dst = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
    if (!src || !dst) { free(src); free(dst); return NULL; }
    double lq = log(1.0 - p);
    int64_t ne = 0, v = 1, w = -1;
    uint64_t draw = 0;
    while (v < n) {
        double r = gg_u01(seed, 4, draw++);
        w += 1 + (p >= 1.0 ? 0 : (int64_t)floor(log(1.0 - r) / lq));
        while (w >= v && v < n) { w -= v; ++v; }
        if (v < n) {
            if (ne == cap) {
                cap = cap * 3 / 2;
                int32_t* s2 = (int32_t*)realloc(src, (size_t)cap * sizeof(int32_t));
                int32_t* d2 = (int32_t*)realloc(dst, (size_t)cap * sizeof(int32_t));
                if (!s2 || !d2) { free(s2 ? s2 : src); free(d2 ? d2 : dst); return NULL; }
                src = s2; dst = d2;
            }
            src[ne] = (int32_t)v; dst[ne] = (int32_t)w; ++ne;
        }
    }
    gg_graph* g = gg_build(n, ne, src, dst);
    free(src); free(dst);
    return g;
}

/*
 * Erased configuration model: degrees drawn i.i.d. from the discrete power
 * law P(k) ~ k^-exponent on [k_min, k_max]; stubs are paired by a random
 * shuffle; loops and multi-edges are erased.  k_min is the value in [1, 64]
 * whose truncated law has the mean closest to `mean_degree`, and
 * k_max = floor(sqrt(n * mean_degree)).
 */
gg_graph* gg_config_powerlaw(int64_t n, double exponent, double mean_degree, uint64_t seed) {
    int64_t kmax = (int64_t)floor(sqrt((double)n * mean_degree));
    if (kmax < 2) kmax = 2;
    int64_t best_kmin = 1;
    double best_err = 1e300;
    for (int64_t kmin = 1; kmin <= 64 && kmin < kmax; ++kmin) {
        double z = 0, s = 0;
        for (int64_t k = kmin; k <= kmax; ++k) {
            double w = pow((double)k, -exponent);
            z += w; s += w * (double)k;
        }
        double err = fabs(s / z - mean_degree);
        if (err < best_err) { best_err = err; best_kmin = kmin; }
    }
    int64_t nk = kmax - best_kmin + 1;
    double* cdf = (double*)malloc((size_t)nk * sizeof(double));
    int64_t* deg = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!cdf || !deg) { free(cdf); free(deg); return NULL; }
    double z = 0;
    for (int64_t t = 0; t < nk; ++t) { z += pow((double)(best_kmin + t), -exponent); cdf[t] = z; }
    int64_t stubs = 0;
    for (int64_t i = 0; i < n; ++i) {
        double r = gg_u01(seed, 5, (uint64_t)i) * z;
        int64_t lo = 0, hi = nk - 1;
        while (lo < hi) { int64_t mid = (lo + hi) / 2; if (cdf[mid] < r) lo = mid + 1; else hi = mid; }
        deg[i] = best_kmin + lo;
        stubs += deg[i];
    }
    if (stubs & 1) { deg[0] += 1; stubs += 1; }
    free(cdf);
    int32_t* st = (int32_t*)malloc((size_t)stubs * sizeof(int32_t));
    if (!st) { free(deg); return NULL; }
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i) for (int64_t q = 0; q < deg[i]; ++q) st[w++] = (int32_t)i;
    free(deg);
    for (int64_t i = stubs - 1; i > 0; --i) {
        int64_t j = (int64_t)gg_below(seed, 6, (uint64_t)i, (uint64_t)(i + 1));
        int32_t t = st[i]; st[i] = st[j]; st[j] = t;
    }
    int64_t m = stubs / 2;
    int32_t* src = (int32_t*)malloc((size_t)m * sizeof(int32_t));
    int32_t* dst = (int32_t*)malloc((size_t)m * sizeof(int32_t));
    if (!src || !dst) { free(st); free(src); free(dst); return NULL; }
    for (int64_t e = 0; e < m; ++e) { src[e] = st[2 * e]; dst[e] = st[2 * e + 1]; }
    free(st);
    gg_graph* g = gg_build(n, m, src, dst);
    free(src); free(dst);
    return g;
}

/*
 * Watts-Strogatz small world (the paper's `smallworld` graphs): ring lattice
 * where every node links to its k/2 nearest neighbours on each side; each
 * lattice edge (i, i+s) is rewired with probability p to (i, t), t uniform,
 * avoiding loops and edges already present in the lattice row of i.
 */
gg_graph* gg_smallworld(int64_t n, int k, double p, uint64_t seed) {
    int half = k / 2;
    int64_t m = n * half;
    int32_t* src = (int32_t*)malloc((size_t)m * sizeof(int32_t));
    int32_t* dst = (int32_t*)malloc((size_t)m * sizeof(int32_t));
    if (!src || !dst) { free(src); free(dst); return NULL; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int s = 1; s <= half; ++s) {
            int64_t e = i * half + (s - 1);
            int64_t t = (i + s) % n;
            if (gg_u01(seed, 7, (uint64_t)e) < p) {
                for (uint64_t tries = 0; tries < 64; ++tries) {
                    int64_t c = (int64_t)gg_below(seed, 8, (uint64_t)e * 64 + tries, (uint64_t)n);
                    int64_t dlt = (c - i + n) % n;
                    if (c != i && !(dlt >= 1 && dlt <= half) && !(dlt >= n - half)) { t = c; break; }
                }
            }
            src[e] = (int32_t)i;
            dst[e] = (int32_t)t;
        }
    }
    gg_graph* g = gg_build(n, m, src, dst);
    free(src); free(dst);
    return g;
}

/* Builds a graph from a caller's edge list (used for the small closed-form graphs). */
gg_graph* gg_from_edges(int64_t n, int64_t m, const int32_t* src, const int32_t* dst) {
    return gg_build(n, m, src, dst);
}
