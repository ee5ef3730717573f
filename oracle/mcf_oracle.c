/*
 * ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential CPU implementation of the randomized matrix
 * function estimators of Guidotti, Acebron and Monteiro, "A fast Monte Carlo
 * algorithm for evaluating matrix functions with application in complex
 * networks" (arXiv 2308.01037).  It exists to check the CUDA library: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code with the CUDA path.  Compile with -ffp-contract=off so that
 * every floating-point product is rounded on its own.
 *
 * Notation follows the paper: A is the n x n adjacency matrix, A' = gamma*A
 * the scaled matrix whose function is evaluated (Section 2.2, f(gamma A)),
 * zeta_0..zeta_K the power-series coefficients (Eq. power_series), N_s the
 * number of walks, W_c the weight cutoff (Eq. weight_cutoff).
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *  - W^(0) = 1 and the 1/N_i factor is applied after the walks; this equals
 *    the paper's W^(0) = 1/N_i (Algorithms 2 and 3) and 1/p_i (Eq. weights)
 *    because (1/N_s)(1/p_i) = 1/N_i, and the cutoff is relative.
 *  - N_i = 0 for an empty column, else max(1, llround(N_s * p_i)), or a fixed
 *    number of walks per node when the caller asks for one.
 *  - The series is truncated at K = n_coeffs - 1: a walk makes at most K - 2
 *    transitions; the paper's cutoff test |W| <= W_c stops it earlier.
 *  - SelectNextState takes its random words from Philox4x32-10 blocks keyed
 *    by the 64-bit seed, counter (block, walk id low, walk id high, request
 *    id).  A uniform row uses one 32-bit word per transition: transition k
 *    reads word k % 4 of block k / 4, and takes j = (w0 * deg) >> 32.  A
 *    weighted row uses two words per transition: words 2(k % 2) and
 *    2(k % 2) + 1 of block k / 2, bucket b = (w0 * deg) >> 32 and
 *    x = (w1 >> 8) * 2^-24 for Vose's alias table.
 *  - For a binary A the row sums and column norms are evaluated in closed
 *    form: sum_j |a'_ij| = gamma * deg_i, ||C_i||_2 = gamma * sqrt(indeg_i).
 *    For a weighted A: gamma * (sum_j |a_ij|) in CSR order and
 *    gamma * sqrt(sum_j a_ji^2) over column i in increasing row order.  A
 *    need not be symmetric: columns are read from a column-major copy (for
 *    a symmetric A with sorted rows it holds the same values in the same
 *    order as the rows).
 *  - r = A' v is evaluated as gamma * (sum_j a_ij v_j), the sum in CSR order.
 *  - Precision 0: every quantity is double.  Precision 1: walk weight W,
 *    coefficients, r and row-sum multipliers are float (round to nearest, no
 *    fused multiply-add); each contribution is widened to double before it is
 *    accumulated.
 *
 * Every function returns 0 on success and a negative value on bad input.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror and Shaw,    */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two  */
/* 32x32->64 multiplies by 0xD2511F53 and 0xCD9E8D57, the key bumped by the  */
/* Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds.                 */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* The Markov chain of Definition 1.                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    const int64_t* rp;
    const int32_t* ci;
    const float* val;   /* NULL: binary matrix */
    double gamma;       /* A' = gamma * A */
    double* rowabs;     /* sum_j |a'_ij|  (the weight multiplier of Eq. weights) */
    double* colnorm;    /* ||C'_i||_2     (Eq. initial_prob numerator) */
    int64_t* nw;        /* N_i */
    int64_t* off;       /* exclusive prefix of N_i: walk ids of start i are off[i] .. off[i+1]-1 */
    float* prob;        /* alias tables for weighted rows (nnz) */
    int32_t* alias;
    int64_t* cp;        /* column-major copy of A: column i holds rows ri[cp[i] .. cp[i+1]) */
    int32_t* ri;        /* in increasing row order, with values cv (NULL when binary)      */
    float* cv;
} chain_t;

static void chain_free(chain_t* c) {
    free(c->rowabs); free(c->colnorm); free(c->nw); free(c->off); free(c->prob); free(c->alias);
    free(c->cp); free(c->ri); free(c->cv);
    memset(c, 0, sizeof(*c));
}

/* Vose's alias method for the row distribution t_ij = |a_ij| / sum_k |a_ik|
 * (Eq. definition1).  Work lists are stacks filled in column order. */
static int build_alias_row(int64_t d, const float* a, float* prob, int32_t* alias) {
    double tot = 0.0;
    for (int64_t j = 0; j < d; ++j) tot += fabs((double)a[j]);
    double* s = (double*)malloc((size_t)d * sizeof(double));
    int64_t* small = (int64_t*)malloc((size_t)d * sizeof(int64_t));
    int64_t* large = (int64_t*)malloc((size_t)d * sizeof(int64_t));
    if (!s || !small || !large) { free(s); free(small); free(large); return -1; }
    int64_t ns = 0, nl = 0;
    for (int64_t j = 0; j < d; ++j) {
        s[j] = ((double)d * fabs((double)a[j])) / tot;
        if (s[j] < 1.0) small[ns++] = j; else large[nl++] = j;
    }
    while (ns > 0 && nl > 0) {
        int64_t l = small[--ns];
        int64_t g = large[--nl];
        prob[l] = (float)s[l];
        alias[l] = (int32_t)g;
        s[g] = (s[g] + s[l]) - 1.0;
        if (s[g] < 1.0) small[ns++] = g; else large[nl++] = g;
    }
    while (nl > 0) { int64_t g = large[--nl]; prob[g] = 1.0f; alias[g] = (int32_t)g; }
    while (ns > 0) { int64_t l = small[--ns]; prob[l] = 1.0f; alias[l] = (int32_t)l; }
    free(s); free(small); free(large);
    return 0;
}

static int chain_build(chain_t* c, int64_t n, const int64_t* rp, const int32_t* ci, const float* val,
                       double gamma, int64_t n_walks, int64_t walks_per_node) {
    memset(c, 0, sizeof(*c));
    if (n < 0 || !rp || (rp[n] > 0 && !ci)) return -1;
    c->n = n; c->rp = rp; c->ci = ci; c->val = val; c->gamma = gamma;
    c->rowabs = (double*)malloc((size_t)(n + 1) * sizeof(double));
    c->colnorm = (double*)malloc((size_t)(n + 1) * sizeof(double));
    c->nw = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    c->off = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    /* column-major copy by counting sort; rows are visited in increasing order */
    int64_t nnz = rp[n];
    c->cp = (int64_t*)calloc((size_t)(n + 2), sizeof(int64_t));
    c->ri = (int32_t*)malloc((size_t)(nnz + 1) * sizeof(int32_t));
    c->cv = val ? (float*)malloc((size_t)(nnz + 1) * sizeof(float)) : NULL;
    int64_t* cur = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!c->rowabs || !c->colnorm || !c->nw || !c->off || !c->cp || !c->ri || (val && !c->cv) || !cur) {
        free(cur); chain_free(c); return -2;
    }
    for (int64_t p = 0; p < nnz; ++p) {
        if (ci[p] < 0 || ci[p] >= n) { free(cur); chain_free(c); return -1; }
        c->cp[ci[p] + 1] += 1;
    }
    for (int64_t i = 0; i < n; ++i) c->cp[i + 1] += c->cp[i];
    for (int64_t i = 0; i < n; ++i) cur[i] = c->cp[i];
    for (int64_t r = 0; r < n; ++r)
        for (int64_t p = rp[r]; p < rp[r + 1]; ++p) {
            int64_t q = cur[ci[p]]++;
            c->ri[q] = (int32_t)r;
            if (val) c->cv[q] = val[p];
        }
    free(cur);
    for (int64_t i = 0; i < n; ++i) {
        int64_t d = rp[i + 1] - rp[i];
        if (!val) {
            c->rowabs[i] = gamma * (double)d;
            c->colnorm[i] = gamma * sqrt((double)(c->cp[i + 1] - c->cp[i]));
        } else {
            double sa = 0.0, sq = 0.0;
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) sa += fabs((double)val[p]);
            for (int64_t q = c->cp[i]; q < c->cp[i + 1]; ++q) {
                double a = (double)c->cv[q];
                sq += a * a;
            }
            c->rowabs[i] = gamma * sa;
            c->colnorm[i] = gamma * sqrt(sq);
        }
    }
    /* Eq. initial_prob: p_i = ||C_i|| / sum_k ||C_k||, N_i ~ N_s p_i. */
    double tot = 0.0;
    for (int64_t i = 0; i < n; ++i) tot += c->colnorm[i];
    for (int64_t i = 0; i < n; ++i) {
        if (!(c->colnorm[i] > 0.0)) c->nw[i] = 0;
        else if (walks_per_node > 0) c->nw[i] = walks_per_node;
        else {
            double x = (double)n_walks * (c->colnorm[i] / tot);
            long long r = llround(x);
            c->nw[i] = r < 1 ? 1 : (int64_t)r;
        }
    }
    c->off[0] = 0;
    for (int64_t i = 0; i < n; ++i) c->off[i + 1] = c->off[i] + c->nw[i];
    if (val && rp[n] > 0) {
        c->prob = (float*)malloc((size_t)rp[n] * sizeof(float));
        c->alias = (int32_t*)malloc((size_t)rp[n] * sizeof(int32_t));
        if (!c->prob || !c->alias) { chain_free(c); return -2; }
        for (int64_t i = 0; i < n; ++i) {
            int64_t d = rp[i + 1] - rp[i];
            if (d > 0 && build_alias_row(d, val + rp[i], c->prob + rp[i], c->alias + rp[i]) != 0) {
                chain_free(c); return -2;
            }
        }
    }
    return 0;
}

/* The random words of transition k of walk g: one word (w[0]) for a uniform
 * row, two (w[0], w[1]) for a weighted row. */
static void draw_words(int weighted, uint64_t g, int k, const uint32_t key[2], uint32_t req, uint32_t w[2]) {
    uint32_t u[4];
    if (!weighted) {
        uint32_t ctr[4] = {(uint32_t)(k / 4), (uint32_t)g, (uint32_t)(g >> 32), req};
        orc_philox4x32_10(ctr, key, u);
        w[0] = u[k % 4];
        w[1] = 0;
    } else {
        uint32_t ctr[4] = {(uint32_t)(k / 2), (uint32_t)g, (uint32_t)(g >> 32), req};
        orc_philox4x32_10(ctr, key, u);
        w[0] = u[2 * (k % 2)];
        w[1] = u[2 * (k % 2) + 1];
    }
}

/* SelectNextState: position j within row l, drawn from the words w. */
static int64_t select_next(const chain_t* c, int64_t l, const uint32_t w[2]) {
    int64_t d = c->rp[l + 1] - c->rp[l];
    int64_t b = (int64_t)(((uint64_t)w[0] * (uint64_t)d) >> 32);
    if (!c->val) return b;
    float x = (float)(w[1] >> 8) * 5.9604644775390625e-08f; /* 2^-24 */
    int64_t p = c->rp[l] + b;
    return x < c->prob[p] ? b : (int64_t)c->alias[p];
}

/* The weight ratio a'_{l l'} / t_{l l'} of Eq. weights: sign(a_{l l'}) * sum_k |a'_{lk}|. */
static double weight_ratio(const chain_t* c, int64_t l, int64_t pos) {
    double m = c->rowabs[l];
    if (c->val && c->val[pos] < 0.0f) m = -m;
    return m;
}

/*
 * One random walk of Algorithms 2/3 (the while loop), started at column i
 * with global walk id g.  For every visited state l_k with weight W^(k) it
 * calls visit(l_k, term) where term = zeta_{k+2} W^(k) in the chosen
 * precision.  Returns the number of transitions made.
 */
typedef void (*visit_fn)(void* ctx, int64_t l, double zw, float zw32);

static int64_t run_walk(const chain_t* c, int64_t i, int64_t g, const double* zeta, int K, double w_cutoff,
                        uint64_t seed, uint32_t req, int precision, visit_fn visit, void* ctx) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t l = i;
    double W = 1.0;   /* precision 0 */
    float W32 = 1.0f; /* precision 1 */
    int64_t steps = 0;
    for (int k = 0;; ++k) {
        double wabs = precision == 0 ? fabs(W) : (double)fabsf(W32);
        if (!(wabs > w_cutoff)) break;                   /* Eq. weight_cutoff */
        if (precision == 0) visit(ctx, l, zeta[k + 2] * W, 0.0f);
        else visit(ctx, l, 0.0, (float)zeta[k + 2] * W32);
        if (k + 2 >= K) break;                           /* truncation of the series */
        int64_t d = c->rp[l + 1] - c->rp[l];
        if (d == 0) break;
        uint32_t w[2];
        draw_words(c->val != NULL, (uint64_t)g, k, key, req, w);
        int64_t pos = c->rp[l] + select_next(c, l, w);
        double ratio = weight_ratio(c, l, pos);          /* Eq. weights */
        if (precision == 0) W = W * ratio;
        else W32 = W32 * (float)ratio;
        l = c->ci[pos];
        ++steps;
    }
    return steps;
}

/* ------------------------------------------------------------------------ */
/* RandFunmAction (Algorithm 3): y = zeta_0 v + zeta_1 r + A' q, r = A' v.   */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double* rr;   /* r in double */
    const float* rr32;  /* r in float */
    double acc;
} action_ctx;

static void action_visit(void* p, int64_t l, double zw, float zw32) {
    action_ctx* a = (action_ctx*)p;
    if (a->rr32) a->acc += (double)(zw32 * a->rr32[l]);
    else a->acc += zw * a->rr[l];
}

/* mark[k] = 1 for every start node k whose q_k enters an output y_i, i in S. */
static unsigned char* needed_starts(int64_t n, const int64_t* rp, const int32_t* ci, const int64_t* nodes,
                                    int64_t n_nodes) {
    unsigned char* mark = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!mark) return NULL;
    if (!nodes) { memset(mark, 1, (size_t)n); return mark; }
    for (int64_t t = 0; t < n_nodes; ++t) {
        int64_t i = nodes[t];
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) mark[ci[p]] = 1;
    }
    return mark;
}

int orc_action(int64_t n, const int64_t* rp, const int32_t* ci, const float* val, double gamma,
               const double* v, const double* zeta, int n_coeffs, int64_t n_walks, int64_t walks_per_node,
               double w_cutoff, uint64_t seed, uint32_t req, int precision, const int64_t* nodes,
               int64_t n_nodes, double* y, double* q_out, int64_t* stats) {
    if (n_coeffs < 1 || !zeta || !v || !y || (precision != 0 && precision != 1)) return -1;
    if (nodes) for (int64_t t = 0; t < n_nodes; ++t) if (nodes[t] < 0 || nodes[t] >= n) return -1;
    int K = n_coeffs - 1;
    chain_t c;
    int rc = chain_build(&c, n, rp, ci, val, gamma, n_walks, walks_per_node);
    if (rc) return rc;
    double* r = (double*)malloc((size_t)(n + 1) * sizeof(double));
    float* r32 = (float*)malloc((size_t)(n + 1) * sizeof(float));
    double* q = (double*)calloc((size_t)(n + 1), sizeof(double));
    unsigned char* mark = needed_starts(n, rp, ci, nodes, n_nodes);
    if (!r || !r32 || !q || !mark) { free(r); free(r32); free(q); free(mark); chain_free(&c); return -2; }
    /* r = A' v (Algorithm 3, before the walks) */
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += (val ? (double)val[p] : 1.0) * v[ci[p]];
        r[i] = gamma * s;
        r32[i] = (float)r[i];
    }
    int64_t walks = 0, steps = 0;
    if (K >= 2) {
        for (int64_t i = 0; i < n; ++i) {
            if (!mark[i] || c.nw[i] == 0) continue;
            action_ctx a = {r, precision == 1 ? r32 : NULL, 0.0};
            for (int64_t s = 0; s < c.nw[i]; ++s) {
                steps += run_walk(&c, i, c.off[i] + s, zeta, K, w_cutoff, seed, req, precision, action_visit, &a);
                ++walks;
            }
            q[i] = a.acc / (double)c.nw[i];
        }
    }
    /* y = zeta_0 v + zeta_1 r + A' q */
    int64_t cnt = nodes ? n_nodes : n;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = nodes ? nodes[t] : t;
        double aq = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) aq += (val ? (double)val[p] : 1.0) * q[ci[p]];
        double yi = zeta[0] * v[i];
        if (K >= 1) yi += zeta[1] * r[i];
        yi += gamma * aq;
        y[t] = yi;
    }
    if (q_out) memcpy(q_out, q, (size_t)n * sizeof(double));
    if (stats) { stats[0] = walks; stats[1] = steps; }
    free(r); free(r32); free(q); free(mark);
    chain_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Standard error of RandFunmAction (the estimator's variance, Section 3.5).  */
/* q_i is the mean of N_i independent walk sums X_s from column i, so        */
/* Var(y_j) = sum_i a'_ji^2 Var(X_i) / N_i.  Var(X_i) is estimated by the     */
/* sample variance s_i^2 = (sum_s X_s^2 - N_i q_i^2) / (N_i - 1), clamped at  */
/* 0, and taken as 0 when N_i < 2.  se[t] = sqrt(Var(y_j)) for j = nodes[t]   */
/* (or t); the walks, ids and precision are those of orc_action.            */
/* ------------------------------------------------------------------------ */
int orc_action_se(int64_t n, const int64_t* rp, const int32_t* ci, const float* val, double gamma, const double* v,
                  const double* zeta, int n_coeffs, int64_t n_walks, int64_t walks_per_node, double w_cutoff,
                  uint64_t seed, uint32_t req, int precision, const int64_t* nodes, int64_t n_nodes, double* se) {
    if (n_coeffs < 1 || !zeta || !v || !se || (precision != 0 && precision != 1)) return -1;
    if (nodes) for (int64_t t = 0; t < n_nodes; ++t) if (nodes[t] < 0 || nodes[t] >= n) return -1;
    int K = n_coeffs - 1;
    chain_t c;
    int rc = chain_build(&c, n, rp, ci, val, gamma, n_walks, walks_per_node);
    if (rc) return rc;
    double* r = (double*)malloc((size_t)(n + 1) * sizeof(double));
    float* r32 = (float*)malloc((size_t)(n + 1) * sizeof(float));
    double* w = (double*)calloc((size_t)(n + 1), sizeof(double));   /* s_i^2 / N_i */
    unsigned char* mark = needed_starts(n, rp, ci, nodes, n_nodes);
    if (!r || !r32 || !w || !mark) { free(r); free(r32); free(w); free(mark); chain_free(&c); return -2; }
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += (val ? (double)val[p] : 1.0) * v[ci[p]];
        r[i] = gamma * s;
        r32[i] = (float)r[i];
    }
    if (K >= 2) {
        for (int64_t i = 0; i < n; ++i) {
            int64_t N = c.nw[i];
            if (!mark[i] || N < 2) continue;
            double sum = 0.0, sum2 = 0.0;
            for (int64_t s = 0; s < N; ++s) {
                action_ctx a = {r, precision == 1 ? r32 : NULL, 0.0};   /* one walk's sum X_s */
                run_walk(&c, i, c.off[i] + s, zeta, K, w_cutoff, seed, req, precision, action_visit, &a);
                sum += a.acc;
                sum2 += a.acc * a.acc;
            }
            double mean = sum / (double)N;
            double ss = sum2 - (double)N * mean * mean;
            if (ss < 0.0) ss = 0.0;
            w[i] = ss / ((double)(N - 1) * (double)N);
        }
    }
    int64_t cnt = nodes ? n_nodes : n;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t j = nodes ? nodes[t] : t;
        double var = 0.0;
        for (int64_t p = rp[j]; p < rp[j + 1]; ++p) {
            double a = gamma * (val ? (double)val[p] : 1.0);
            var += a * a * w[ci[p]];
        }
        se[t] = sqrt(var);
    }
    free(r); free(r32); free(w); free(mark);
    chain_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* RandFunmDiag (Section 3.3, Eq. rand_funm_formula_diag):                   */
/* d_i = zeta_0 + zeta_1 a'_ii + sum_k a'_ik <Q_k, C'_i>.                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    double* Q;       /* row Q_k, dense (length n) */
    int64_t* touched;
    int64_t ntouched;
    unsigned char* seen;
    int precision;
} diag_ctx;

static void diag_visit(void* p, int64_t l, double zw, float zw32) {
    diag_ctx* d = (diag_ctx*)p;
    if (!d->seen[l]) { d->seen[l] = 1; d->touched[d->ntouched++] = l; }
    d->Q[l] += d->precision == 1 ? (double)zw32 : zw;
}

static double entry(const int64_t* rp, const int32_t* ci, const float* val, int64_t i, int64_t j) {
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
        if (ci[p] == j) return val ? (double)val[p] : 1.0;
    return 0.0;
}

int orc_diag(int64_t n, const int64_t* rp, const int32_t* ci, const float* val, double gamma,
             const double* zeta, int n_coeffs, int64_t n_walks, int64_t walks_per_node, double w_cutoff,
             uint64_t seed, uint32_t req, int precision, const int64_t* nodes, int64_t n_nodes, double* d,
             int64_t* stats) {
    if (n_coeffs < 1 || !zeta || !d || (precision != 0 && precision != 1)) return -1;
    if (nodes) for (int64_t t = 0; t < n_nodes; ++t) if (nodes[t] < 0 || nodes[t] >= n) return -1;
    int K = n_coeffs - 1;
    chain_t c;
    int rc = chain_build(&c, n, rp, ci, val, gamma, n_walks, walks_per_node);
    if (rc) return rc;
    /* pos[i] = index of i in the output, or -1 when i is not requested */
    int64_t* pos = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    double* acc = (double*)calloc((size_t)(n + 1), sizeof(double));
    diag_ctx dc;
    dc.Q = (double*)calloc((size_t)(n + 1), sizeof(double));
    dc.touched = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    dc.seen = (unsigned char*)calloc((size_t)(n + 1), 1);
    dc.ntouched = 0;
    dc.precision = precision;
    unsigned char* mark = needed_starts(n, rp, ci, nodes, n_nodes);
    if (!pos || !acc || !dc.Q || !dc.touched || !dc.seen || !mark) {
        free(pos); free(acc); free(dc.Q); free(dc.touched); free(dc.seen); free(mark); chain_free(&c);
        return -2;
    }
    for (int64_t i = 0; i < n; ++i) pos[i] = nodes ? -1 : i;
    if (nodes) for (int64_t t = 0; t < n_nodes; ++t) pos[nodes[t]] = t;
    int64_t walks = 0, steps = 0;
    if (K >= 2) {
        for (int64_t k = 0; k < n; ++k) {
            if (!mark[k] || c.nw[k] == 0) continue;
            /* row Q_k of Eq. rand_funm_Q (times N_k) from the N_k walks started at column k */
            for (int64_t s = 0; s < c.nw[k]; ++s) {
                steps += run_walk(&c, k, c.off[k] + s, zeta, K, w_cutoff, seed, req, precision, diag_visit, &dc);
                ++walks;
            }
            /* d_i += a'_ik <Q_k, C'_i> for every i with a_ik != 0 (the rows i of column k) */
            for (int64_t p = c.cp[k]; p < c.cp[k + 1]; ++p) {
                int64_t i = c.ri[p];
                if (pos[i] < 0) continue;
                double dot = 0.0;
                for (int64_t t = c.cp[i]; t < c.cp[i + 1]; ++t)   /* column i: entries a_ji */
                    dot += (gamma * (c.cv ? (double)c.cv[t] : 1.0)) * dc.Q[c.ri[t]];
                double aik = gamma * (c.cv ? (double)c.cv[p] : 1.0);
                acc[i] += (aik * dot) / (double)c.nw[k];
            }
            for (int64_t t = 0; t < dc.ntouched; ++t) { dc.Q[dc.touched[t]] = 0.0; dc.seen[dc.touched[t]] = 0; }
            dc.ntouched = 0;
        }
    }
    int64_t cnt = nodes ? n_nodes : n;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = nodes ? nodes[t] : t;
        double di = zeta[0];
        if (K >= 1) di += zeta[1] * (gamma * entry(rp, ci, val, i, i));
        d[t] = di + acc[i];
    }
    if (stats) { stats[0] = walks; stats[1] = steps; }
    free(pos); free(acc); free(dc.Q); free(dc.touched); free(dc.seen); free(mark);
    chain_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* RandFunm (Algorithm 2): F = zeta_0 I + zeta_1 A' + A' Q A', dense n x n.  */
/* Small graphs only; it shares walks (seeds, walk ids) with the two above.  */
/* ------------------------------------------------------------------------ */
int orc_funm_full(int64_t n, const int64_t* rp, const int32_t* ci, const float* val, double gamma,
                  const double* zeta, int n_coeffs, int64_t n_walks, int64_t walks_per_node, double w_cutoff,
                  uint64_t seed, uint32_t req, int precision, double* F /* n*n row-major */) {
    if (n_coeffs < 1 || !zeta || !F || n > 4096 || (precision != 0 && precision != 1)) return -1;
    int K = n_coeffs - 1;
    chain_t c;
    int rc = chain_build(&c, n, rp, ci, val, gamma, n_walks, walks_per_node);
    if (rc) return rc;
    double* Qm = (double*)calloc((size_t)(n * n + 1), sizeof(double));
    double* AQ = (double*)calloc((size_t)(n * n + 1), sizeof(double));
    diag_ctx dc;
    dc.touched = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    dc.seen = (unsigned char*)calloc((size_t)(n + 1), 1);
    dc.precision = precision;
    if (!Qm || !AQ || !dc.touched || !dc.seen) {
        free(Qm); free(AQ); free(dc.touched); free(dc.seen); chain_free(&c); return -2;
    }
    if (K >= 2) {
        for (int64_t i = 0; i < n; ++i) {
            if (c.nw[i] == 0) continue;
            dc.Q = Qm + i * n;
            dc.ntouched = 0;
            for (int64_t s = 0; s < c.nw[i]; ++s)
                run_walk(&c, i, c.off[i] + s, zeta, K, w_cutoff, seed, req, precision, diag_visit, &dc);
            for (int64_t t = 0; t < dc.ntouched; ++t) dc.seen[dc.touched[t]] = 0;
            for (int64_t j = 0; j < n; ++j) Qm[i * n + j] /= (double)c.nw[i];   /* Eq. rand_funm_Q */
        }
    }
    /* AQ = A' Q */
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            double a = gamma * (val ? (double)val[p] : 1.0);
            const double* qrow = Qm + (int64_t)ci[p] * n;
            for (int64_t j = 0; j < n; ++j) AQ[i * n + j] += a * qrow[j];
        }
    /* F = zeta_0 I + zeta_1 A' + (A' Q) A' */
    for (int64_t i = 0; i < n * n; ++i) F[i] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        F[i * n + i] += zeta[0];
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            double a = gamma * (val ? (double)val[p] : 1.0);
            if (K >= 1) F[i * n + ci[p]] += zeta[1] * a;
        }
    }
    for (int64_t j = 0; j < n; ++j)           /* column j of A': entries a'_mj */
        for (int64_t p = c.cp[j]; p < c.cp[j + 1]; ++p) {
            double a = gamma * (c.cv ? (double)c.cv[p] : 1.0);
            int64_t m = c.ri[p];
            for (int64_t i = 0; i < n; ++i) F[i * n + j] += AQ[i * n + m] * a;
        }
    free(Qm); free(AQ); free(dc.touched); free(dc.seen);
    chain_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The classical Monte Carlo method (Algorithm 1) for one entry of f(A')v:  */
/* N walks from row i, each adding zeta_k W^(k) v_{l_k}; W^(0) = 1 and the  */
/* 1/N factor after the walks.  Walk ids are i * N + s.                     */
/* ------------------------------------------------------------------------ */
typedef struct { const double* v; const double* zeta; double acc; int k; } mc_ctx;

int orc_mc_classic_action(int64_t n, const int64_t* rp, const int32_t* ci, const float* val, double gamma,
                          const double* v, const double* zeta, int n_coeffs, int64_t walks_per_row,
                          double w_cutoff, uint64_t seed, uint32_t req, const int64_t* nodes, int64_t n_nodes,
                          double* y) {
    if (n_coeffs < 1 || !zeta || !v || !y || walks_per_row < 1 || !nodes) return -1;
    int K = n_coeffs - 1;
    chain_t c;
    int rc = chain_build(&c, n, rp, ci, val, gamma, 0, 1);
    if (rc) return rc;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t t = 0; t < n_nodes; ++t) {
        int64_t i = nodes[t];
        if (i < 0 || i >= n) { chain_free(&c); return -1; }
        double acc = 0.0;
        for (int64_t s = 0; s < walks_per_row; ++s) {
            uint64_t g = (uint64_t)i * (uint64_t)walks_per_row + (uint64_t)s;
            int64_t l = i;
            double W = 1.0;
            for (int k = 0;; ++k) {
                if (!(fabs(W) > w_cutoff)) break;
                acc += zeta[k] * W * v[l];
                if (k >= K) break;
                int64_t d = rp[l + 1] - rp[l];
                if (d == 0) break;
                uint32_t w[2];
                draw_words(val != NULL, g, k, key, req, w);
                int64_t p = rp[l] + select_next(&c, l, w);
                W = W * weight_ratio(&c, l, p);
                l = ci[p];
            }
        }
        y[t] = acc / (double)walks_per_row;
    }
    chain_free(&c);
    return 0;
}

/* Counts the positions SelectNextState picks in row l over the transitions
 * k = 0 .. n_draws-1 of walk g (the random words every walk step uses), for
 * a frequency test of the sampler against t_lj = |a_lj| / sum_k |a_lk|. */
int orc_sample_counts(int64_t n, const int64_t* rp, const int32_t* ci, const float* val, int64_t l,
                      int64_t n_draws, uint64_t seed, uint32_t req, int64_t* counts) {
    if (l < 0 || l >= n || n_draws < 0 || !counts) return -1;
    chain_t c;
    int rc = chain_build(&c, n, rp, ci, val, 1.0, 0, 1);
    if (rc) return rc;
    int64_t d = rp[l + 1] - rp[l];
    if (d <= 0) { chain_free(&c); return -1; }
    for (int64_t j = 0; j < d; ++j) counts[j] = 0;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t t = 0; t < n_draws; ++t) {
        /* draw t: transition t % 256 of walk t / 256 */
        uint32_t w[2];
        draw_words(val != NULL, (uint64_t)(t / 256), (int)(t % 256), key, req, w);
        counts[select_next(&c, l, w)] += 1;
    }
    chain_free(&c);
    return 0;
}

/* Exposes the walk allocation of Definition 1 (for tests of the rule). */
int orc_allocation(int64_t n, const int64_t* rp, const int32_t* ci, const float* val, double gamma,
                   int64_t n_walks, int64_t walks_per_node, double* rowabs, double* colnorm, int64_t* nw,
                   int64_t* off) {
    chain_t c;
    int rc = chain_build(&c, n, rp, ci, val, gamma, n_walks, walks_per_node);
    if (rc) return rc;
    if (rowabs) memcpy(rowabs, c.rowabs, (size_t)n * sizeof(double));
    if (colnorm) memcpy(colnorm, c.colnorm, (size_t)n * sizeof(double));
    if (nw) memcpy(nw, c.nw, (size_t)n * sizeof(int64_t));
    if (off) memcpy(off, c.off, (size_t)(n + 1) * sizeof(int64_t));
    chain_free(&c);
    return 0;
}

/* Exposes the alias table of one weighted row (for tests of the sampler). */
int orc_alias_row(int64_t d, const float* a, float* prob, int32_t* alias) {
    if (d <= 0) return -1;
    return build_alias_row(d, a, prob, alias);
}
