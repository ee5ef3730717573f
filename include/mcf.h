/*
 * mcf.h -- C ABI of libmcf: Monte Carlo evaluation of matrix functions of a
 * sparse graph adjacency matrix on one NVIDIA GB300 (sm_103a).
 *
 * The library implements the randomized method of Guidotti, Acebron and
 * Monteiro (arXiv 2308.01037): a power series f(A') = sum_k zeta_k A'^k
 * (Eq. power_series) of the scaled adjacency matrix A' = scale * A is
 * estimated from random walks that sample a whole row or column of A' per
 * step (Lemma 2, Eq. random_walk_realization), with
 *   - f(A')v     by RandFunmAction (Algorithm 3, Section 3.4),
 *   - f(A')1     total communicability (Eq. total_comm),
 *   - diag f(A') subgraph centrality by RandFunmDiag (Section 3.3,
 *                Eq. rand_funm_formula_diag),
 *   - (I - gamma A)^{-1} 1, Katz centrality as the truncated Neumann series
 *                (Section 4.5).
 *
 * Conventions shared by every entry point
 *   - Matrices are symmetric (the paper's Section 2.1 class: undirected
 *     graphs; a digraph enters through its symmetrisation B = [0 A; A^T 0]),
 *     given in CSR: row_ptr int64[n+1] (row_ptr[0] = 0, non-decreasing),
 *     col_idx int32[nnz] strictly increasing within each row, optional
 *     values float32[nnz] (NULL = binary matrix, every entry 1).
 *   - Pointer arguments may point to host or device memory unless stated
 *     otherwise; the library tells them apart with cudaPointerGetAttributes.
 *     The caller keeps ownership of every array it passes.
 *   - Work is enqueued on params->stream (a cudaStream_t; NULL = the legacy
 *     default stream).  A call returns once its work is enqueued when every
 *     output is in device memory and `stats` is NULL; otherwise it waits for
 *     the stream before returning.
 *   - Every call returns an mcf_status; nothing aborts or throws across the
 *     ABI.  mcf_last_error() returns a thread-local message for the last
 *     failing call of this thread.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key =
 *     (seed low, seed high) and counter = (b, walk id low, walk id high,
 *     request_id), where b numbers the blocks of one walk.  A transition out
 *     of a row of a binary matrix uses one 32-bit word: transition k takes
 *     word k mod 4 of block b = floor(k / 4).  A transition out of a row of a
 *     weighted matrix uses two words (alias bucket and acceptance test):
 *     transition k takes words 2 (k mod 2) and 2 (k mod 2) + 1 of block
 *     b = floor(k / 2).  Walk ids are the exclusive prefix of N_i over the
 *     nodes (the classical method of Algorithm 1: i * N + s).  The same seed
 *     gives the same walks on every run and every launch configuration.
 */
#ifndef MCF_H
#define MCF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcf_graph* mcf_graph_t;

typedef enum {
    MCF_OK = 0,
    MCF_ERR_INVALID_ARG = 1,      /* a NULL, negative or out-of-range argument */
    MCF_ERR_INVALID_GRAPH = 2,    /* CSR not sorted / out of range / duplicate / not symmetric / non-finite */
    MCF_ERR_OOM = 3,              /* device or host allocation failed */
    MCF_ERR_CUDA = 4,             /* a CUDA runtime call failed; see mcf_last_error() */
    MCF_ERR_ADMISSION = 5,        /* a request does not fit the caller's memory budget */
    MCF_ERR_TIMEOUT = 6,          /* mcf_server_wait gave up before the request completed */
    MCF_ERR_CANCELLED = 7,        /* a queued server request was cancelled (mcf_server_cancel) */
    MCF_ERR_ACCURACY_BUDGET = 8,  /* an accuracy-targeted solve hit its walk cap above the target error */
    MCF_WARN_OVERFLOW = 9,        /* reserved: a float32 weight overflow sets bit 0 of mcf_stats.flags */
    MCF_ERR_UNSUPPORTED = 10      /* a valid request this build does not implement */
} mcf_status;

/* Arithmetic of the walk (Section 3.2's weights W^(k) and the sums of
 * Eq. rand_funm_Q):
 *   MCF_F64          every quantity in float64;
 *   MCF_F32W_F64ACC  W, zeta, r and the row-sum multipliers in float32
 *                    (round to nearest, no fused multiply-add), every
 *                    contribution widened to float64 before it is summed. */
typedef enum { MCF_F64 = 0, MCF_F32W_F64ACC = 1 } mcf_precision;

/* mcf_create_graph flags */
#define MCF_GRAPH_DEVICE_PTRS 1u   /* row_ptr/col_idx/values are device pointers (copied device to device) */
#define MCF_GRAPH_NONSYMMETRIC 2u  /* A is a general (e.g. directed) matrix: the symmetry check is skipped and a
                                      column-major copy is kept, since Definition 1 draws start columns from the
                                      column norms ||C_i|| and Eq. rand_funm_formula_diag and Algorithm 2 read
                                      columns of A.  The copy is built on the host at creation (a device-resident
                                      CSR is read back for it).  mcf_spectral_radius is then unsupported: pass
                                      the scale explicitly (mcf_gershgorin bounds the spectral radius). */

typedef struct {
    const double* coeffs;   /* zeta_0..zeta_K of Eq. power_series (host memory), K = n_coeffs - 1;
                               a walk makes at most K - 2 transitions                          */
    int32_t n_coeffs;       /* 1 .. MCF_MAX_COEFFS                                              */
    double scale;           /* A' = scale * A (the gamma of f(gamma A), Section 2.2); 0 means 1 */
    int64_t n_walks;        /* N_s: total walks, N_i = max(1, llround(N_s p_i)) for every
                               non-empty column i, p_i of Eq. initial_prob                      */
    int64_t walks_per_node; /* > 0: N_i = walks_per_node for every non-empty column instead     */
    double w_cutoff;        /* W_c of Eq. weight_cutoff (relative; W^(0) = 1); 0 = truncation only */
    uint64_t seed;          /* Philox key                                                        */
    uint32_t request_id;    /* fourth Philox counter word: independent streams per request       */
    int32_t precision;      /* mcf_precision                                                     */
    int32_t deterministic;  /* 1: RandFunmAction solves (mcf_action, mcf_action_nodes,
                               mcf_total_communicability, mcf_katz) give bit-identical results
                               on every run: each walk writes its value to a float64 slot of its
                               own (8 bytes of device scratch per walk) and the walks of a start
                               are summed in walk order with a fixed reduction tree, instead of
                               float64 atomics in arrival order.  Other solves return
                               MCF_ERR_UNSUPPORTED with 1.  0: atomics (faster).              */
    int32_t error_estimate; /* 1: also estimate the standard error (mcf_stats.max_rel_se) of a
                               single-query RandFunmAction solve (mcf_action, mcf_action_nodes,
                               mcf_total_communicability, mcf_katz); 0: off. Ignored elsewhere. */
    void* stream;           /* cudaStream_t                                                      */
    double target_rel_err;  /* > 0: accuracy-targeted solve (below); 0: the walks above, once    */
    int64_t max_walks;      /* accuracy-targeted solves: cap on the total walks (0: 2^34)        */
} mcf_params;

/* Accuracy-targeted solves (params.target_rel_err = t > 0; mcf_action,
 * mcf_action_nodes, mcf_total_communicability, mcf_katz,
 * mcf_subgraph_centrality, and batch queries, which then run through the
 * single-query path).  The solve runs independent replicas of the plain
 * solve with the walk budget above (replica r uses seed + r *
 * 0x9E3779B97F4A7C15, so replica 0 is the plain solve; every replica keeps
 * request_id) and returns their mean.  Replicas alternate between two
 * halves; est = max_i |mean of half 1 - mean of half 2|_i / 2 / max_i |mean|_i
 * estimates the relative l_inf error of the returned mean (its spread is that
 * error's: the estimator's error falls like N^-1/2, Theorem 1 and Section
 * 3.5).  Two replicas run first; while est > t the count grows to
 * R (est/t)^2 x 1.25 (even), within max_walks and 4096 replicas.  If est is
 * still above t at the cap the mean is returned with MCF_ERR_ACCURACY_BUDGET.
 * mcf_stats reports the total walks and steps, est_rel_err and replicas. */

#define MCF_MAX_COEFFS 256

typedef struct {
    int64_t walks;          /* walks run (sum of N_i over the start nodes used) */
    int64_t walk_steps;     /* transitions l_k -> l_{k+1} taken by all walks    */
    double kernel_ms;       /* device time of the walk kernel (CUDA events)     */
    uint32_t flags;         /* bit 0: float32 weight overflow seen              */
    /* With params.error_estimate = 1 (RandFunmAction solves): the largest
     * relative standard error max_j sqrt(V_j) / |y_j| over the entries with
     * y_j != 0, where V_j = sum_i a'_ji^2 s_i^2 / N_i is the variance of
     * y_j = ... + sum_i a'_ji q_i for independent walks (the estimator's
     * variance, Section 3.5) and s_i^2 the sample variance of the N_i walk
     * sums from column i (columns with N_i = 1 contribute 0); else 0. */
    double max_rel_se;
    double est_rel_err;     /* accuracy-targeted solves: the estimated relative l_inf error; else 0 */
    int32_t replicas;       /* accuracy-targeted solves: replicas run; else 1                      */
} mcf_stats;

/* ------------------------------------------------------------------ graphs */

/* Copies the CSR of a symmetric n x n matrix to the device, validates it
 * (sorted, in-range, duplicate-free columns; finite values; symmetric
 * pattern and values) and precomputes its per-row sums (the row sums of
 * Definition 1 before scaling) and, for a weighted matrix, the per-row alias
 * tables of the transition probabilities t_ij = |a_ij| / sum_k |a_ik|
 * (Eq. definition1).  Loops (a_ii != 0) are accepted.  n may be 0.
 * On success *out owns device memory until mcf_destroy_graph.
 * Errors: MCF_ERR_INVALID_ARG, MCF_ERR_INVALID_GRAPH, MCF_ERR_OOM, MCF_ERR_CUDA
 * (also when no usable CUDA device or driver is present: nothing runs on
 * the host instead). */
mcf_status mcf_create_graph(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const float* values,
                            uint32_t flags, mcf_graph_t* out);

/* Releases the graph's device memory (after synchronising the device). NULL is a no-op. */
mcf_status mcf_destroy_graph(mcf_graph_t g);

/* n, nnz, maximum degree and number of loops of the graph (any output may be NULL). */
mcf_status mcf_graph_info(mcf_graph_t g, int64_t* n, int64_t* nnz, int64_t* max_degree, int64_t* n_loops);

/* Largest eigenvalue of the symmetric matrix A (unscaled) by power iteration
 * on A + I in float64 on the device, until the Rayleigh quotient changes by
 * at most tol (relative) or max_iter iterations; used to set
 * scale = 1/lambda_max (the configurations of Section 4 scale A by gamma).
 * Cached on the graph.  Errors: MCF_ERR_INVALID_ARG, MCF_ERR_CUDA,
 * MCF_ERR_UNSUPPORTED (graph created with MCF_GRAPH_NONSYMMETRIC). */
mcf_status mcf_spectral_radius(mcf_graph_t g, double tol, int32_t max_iter, double* lambda_max);

/* Gershgorin bound max_i sum_k |a_ik| on the spectral radius of A (Section 4.5). */
mcf_status mcf_gershgorin(mcf_graph_t g, double* bound);

/* Spectral radius rho of M = diag(s') |A'|, s'_i = sum_j |a'_ij|, A' = scale * A
 * (scale 0 means 1): the second moment of a walk's weighted term at step k
 * grows like rho^k (E[W^(k)2 ...] = (M^k ...), from Definition 1 and
 * Eq. weights), so rho < 1 bounds the estimator's variance however long the
 * walks (the role of Theorem 1's condition alpha < 1, for which alpha >= rho);
 * with rho > 1 the variance grows geometrically with the truncation K (e.g.
 * Katz with gamma = 0.85 / lambda_max on graphs with hubs).  Power iteration
 * on the symmetric D^1/2 |A| D^1/2 (similar to M) in float64, shifted by the
 * current Rayleigh quotient, until it changes by at most tol (relative) or
 * max_iter iterations.  Errors: MCF_ERR_INVALID_ARG, MCF_ERR_UNSUPPORTED (A not
 * symmetric), MCF_ERR_OOM, MCF_ERR_CUDA. */
mcf_status mcf_second_moment_radius(mcf_graph_t g, double scale, double tol, int32_t max_iter, double* rho);

/* ------------------------------------------------------------------ solves */

/* RandFunmAction (Algorithm 3): y = zeta_0 v + zeta_1 r + A' q with r = A' v
 * and q_i the mean over the N_i walks from column i of
 * sum_k zeta_{k+2} W^(k) r_{l_k} (Eq. rand_funm_action_formula).
 * v, y: float64[n], host or device.  stats may be NULL.
 * Errors: MCF_ERR_INVALID_ARG (bad params, NULL arrays), MCF_ERR_OOM, MCF_ERR_CUDA. */
mcf_status mcf_action(mcf_graph_t g, const mcf_params* params, const double* v, double* y, mcf_stats* stats);

/* Entries nodes[0..n_nodes) of f(A')v (v = NULL means v = 1): single-entry
 * or subset total communicability, the setting of Section 4.3 (Table 3).
 * Only the columns adjacent to a requested node are walked, each with the
 * walk ids of the full run, so every entry equals the corresponding entry of
 * mcf_action / mcf_total_communicability.  nodes: int64, host or device;
 * y: float64[n_nodes], host or device.
 * Errors: MCF_ERR_INVALID_ARG (node out of range), as mcf_action. */
mcf_status mcf_action_nodes(mcf_graph_t g, const mcf_params* params, const double* v, const int64_t* nodes,
                            int64_t n_nodes, double* y, mcf_stats* stats);

/* Total communicability f(A')1 (Eq. total_comm): mcf_action with v = 1. */
mcf_status mcf_total_communicability(mcf_graph_t g, const mcf_params* params, double* y, mcf_stats* stats);

/* Subgraph centrality diag f(A') by RandFunmDiag (Eq. rand_funm_formula_diag):
 * d_i = zeta_0 + zeta_1 a'_ii + sum_k a'_ik <Q_k, C'_i>, with row Q_k built
 * from the N_k walks started at column k (Eq. rand_funm_Q).  nodes: int64
 * indices (host or device) of the requested entries, or NULL for all n;
 * only the columns k adjacent to a requested node are walked (Section 3.3's
 * skip of Q_k when a_ik = 0), with the walk ids of the full run, so a subset
 * reproduces the corresponding entries of the full result.
 * d: float64[n_nodes] (or [n]), host or device.
 * Errors: MCF_ERR_INVALID_ARG (node out of range), MCF_ERR_OOM, MCF_ERR_CUDA. */
mcf_status mcf_subgraph_centrality(mcf_graph_t g, const mcf_params* params, const int64_t* nodes, int64_t n_nodes,
                                   double* d, mcf_stats* stats);

/* Katz centrality (I - gamma A)^{-1} 1 as the Neumann series sum_{k<=K} (gamma A)^k 1
 * (Section 4.5) through RandFunmAction with zeta_k = 1 and scale = gamma;
 * params->coeffs and params->scale are ignored.  K = 0 picks the smallest K
 * with rho^(K+1) / (1 - rho) <= 1e-4, rho = gamma * lambda_max (computed
 * with mcf_spectral_radius if not cached); the series needs rho < 1.  A graph
 * created with MCF_GRAPH_NONSYMMETRIC needs an explicit K > 0.
 * Errors: MCF_ERR_INVALID_ARG (gamma <= 0, rho >= 1, K too large),
 * MCF_ERR_UNSUPPORTED (K = 0 on a non-symmetric graph), as mcf_action. */
mcf_status mcf_katz(mcf_graph_t g, double gamma, int32_t K, const mcf_params* params, double* y, mcf_stats* stats);

/* Largest n accepted by mcf_funm_full (its dense row of A'Q is staged in
 * shared memory: n float64 values per CTA). */
#define MCF_FULL_MAX_NODES 16384

/* RandFunm (Algorithm 2): the dense estimate F = zeta_0 I + zeta_1 A' + A' Q A'
 * of f(A'), where row k of Q is (1/N_k) sum over the N_k walks from column k
 * of sum_m zeta_{m+2} W^(m) e_{l_m} (Eq. rand_funm_Q; the walks, their ids and
 * the allocation are those of mcf_subgraph_centrality, so diag F equals its
 * result).  F: float64[n * n] row-major, host or device (a host F is staged
 * through n * n float64 of device memory).  Device scratch: n * n float64 for Q.
 * Errors: MCF_ERR_UNSUPPORTED (n > MCF_FULL_MAX_NODES), MCF_ERR_INVALID_ARG
 * (bad params, NULL F), MCF_ERR_OOM, MCF_ERR_CUDA. */
mcf_status mcf_funm_full(mcf_graph_t g, const mcf_params* params, double* F, mcf_stats* stats);

/* The classical Monte Carlo method (Algorithm 1), the paper's baseline: entry
 * y_t of f(A')v for row i = nodes[t] (or t when nodes is NULL) is the mean over
 * N = params->walks_per_node walks from i of sum_k zeta_k W^(k) v_{l_k}; each
 * step samples ONE entry of the current row (the chain of Definition 1) and
 * W^(k+1) = W^(k) sign(a_{l l'}) sum_j |a'_lj|, W^(0) = 1; a walk stops when
 * |W| <= params->w_cutoff or after K = n_coeffs - 1 steps.  Walk s of row i
 * has id i * N + s.  v: float64[n] (host or device) or NULL for v = 1;
 * y: float64[n_nodes] (or [n]), host or device.  Float64 only
 * (params->precision = MCF_F64); params->n_walks is ignored.
 * Errors: MCF_ERR_UNSUPPORTED (precision), MCF_ERR_INVALID_ARG (walks_per_node
 * < 1, node out of range), MCF_ERR_OOM, MCF_ERR_CUDA. */
mcf_status mcf_mc_classic(mcf_graph_t g, const mcf_params* params, const double* v, const int64_t* nodes,
                          int64_t n_nodes, double* y, mcf_stats* stats);

/* ------------------------------------------------------------------ batches */

typedef enum {
    MCF_QUERY_TOTAL_COMMUNICABILITY = 0, /* f(A')1 (Eq. total_comm)                          */
    MCF_QUERY_KATZ = 1,                  /* (I - gamma A)^{-1} 1 as a Neumann series (Sec. 4.5) */
    MCF_QUERY_SUBGRAPH_CENTRALITY = 2,   /* diag f(A'), all nodes or a subset (Sec. 3.3)    */
    MCF_QUERY_ACTION = 3                 /* f(A')v (Algorithm 3)                            */
} mcf_query_kind;

/* One request of a batch.  Every field means what it means for the single
 * call of the same kind (mcf_total_communicability, mcf_katz,
 * mcf_subgraph_centrality, mcf_action); params.stream is ignored. */
typedef struct {
    mcf_graph_t graph;
    int32_t kind;            /* mcf_query_kind                                      */
    int32_t katz_terms;      /* MCF_QUERY_KATZ: K (0 = from the tail bound)          */
    double katz_gamma;       /* MCF_QUERY_KATZ: gamma                                */
    mcf_params params;       /* coefficients, scale, walks, cutoff, seed, request id */
    const double* v;         /* MCF_QUERY_ACTION: float64[n], host or device         */
    const int64_t* nodes;    /* MCF_QUERY_SUBGRAPH_CENTRALITY: subset, or NULL       */
    int64_t n_nodes;
    double* out;             /* float64[n] (or [n_nodes]), host or device            */
} mcf_query;

typedef struct mcf_batch* mcf_batch_t;

#define MCF_BATCH_CUDA_GRAPH 1u  /* capture the fused launch sequence in a CUDA graph */
#define MCF_BATCH_AUTOTUNE 2u    /* time candidate launch shapes once per batch shape and keep the fastest */

/* Plans a batch of queries on any mix of resident graphs.  Total
 * communicability and Katz queries on binary graphs in MCF_F32W_F64ACC run
 * together in ONE persistent walk launch; subgraph-centrality queries on
 * binary graphs in MCF_F32W_F64ACC run together in one diag launch; their
 * preparation and epilogues are segmented kernels over all of them.  Other
 * queries (general v, weighted graphs, MCF_F64) run one after another with
 * the single-query path.  Every query keeps its own walk ids and Philox
 * streams, so each result equals the single call's result up to float64
 * summation order.  The plan owns its device scratch; query pointers must
 * stay valid until mcf_batch_destroy.  `stream` orders the planning work.
 * Errors: as the single calls; MCF_ERR_INVALID_ARG for an empty batch. */
mcf_status mcf_batch_create(const mcf_query* queries, int32_t n_queries, uint32_t flags, void* stream,
                            mcf_batch_t* out);

/* Runs the batch on `stream` (replaying the CUDA graph when captured) and
 * waits for it.  stats (may be NULL) receives the totals over the batch. */
mcf_status mcf_batch_run(mcf_batch_t batch, void* stream, mcf_stats* stats);

/* Releases the plan (after synchronising the device). NULL is a no-op. */
mcf_status mcf_batch_destroy(mcf_batch_t batch);

/* ------------------------------------------------------------------ serving */

typedef struct mcf_server* mcf_server_t;

typedef struct {
    size_t hbm_budget_bytes;   /* device memory the in-flight requests may use (scratch estimate) */
    int32_t max_inflight;      /* batches executing concurrently, one stream each (>= 1)         */
    int32_t max_batch;         /* requests per batch (>= 1)                                      */
    double batch_window_ms;    /* how long the scheduler waits for more arrivals before it forms
                                  a batch when a worker is free (0 = form at once)                */
} mcf_server_config;

typedef struct {
    int64_t submitted, completed, rejected, batches;   /* completed includes cancelled requests */
    int64_t cancelled;
    int64_t walk_steps;        /* over completed requests                          */
    double p50_ms, p99_ms, max_ms, mean_ms;  /* latency submit -> result ready      */
    double busy_s;             /* wall time from the first submit to the last completion */
    /* Device windows of the completed batches (the GPU's global timer read by
     * a kernel before a batch's first kernel and after its last one): the
     * time during which two or more batches' work was on the device, and the
     * largest number of batches whose windows overlapped at once. */
    double device_overlap_ms;
    int64_t max_concurrent_batches;
    double plan_s, run_s;      /* host time the workers spent planning (mcf_batch_create) and
                                  running (mcf_batch_run) batches, summed over the workers     */
} mcf_server_stats;

/* Starts a request server on the current device: a scheduler thread that
 * admits queued requests while their estimated device footprint fits the
 * budget, groups them into batches (mcf_batch_*), and hands each batch to a
 * free worker stream.  Requests that arrive while batches are running are
 * admitted as workers and memory free up, and their batches run on the
 * device concurrently with the running ones (continuous batching).  Graphs
 * stay resident; each request keeps its own walk ids and Philox streams, so
 * its result equals the single call's result.
 * Errors: MCF_ERR_INVALID_ARG (zero budget, max_inflight < 1), MCF_ERR_CUDA. */
mcf_status mcf_server_create(const mcf_server_config* config, mcf_server_t* out);

/* Device memory a request may take: the buffers mcf_batch_create allocates
 * for a batch holding only *query (for queries that batches run through the
 * single-query path, a bound on that path's scratch).  The server admits
 * requests while the sum of these over the requests in flight fits its
 * budget.  Errors: MCF_ERR_INVALID_ARG (as mcf_batch_create would refuse the
 * query), MCF_ERR_CUDA. */
mcf_status mcf_query_footprint(const mcf_query* query, size_t* bytes);

/* Device memory a batch plan holds (every buffer mcf_batch_create allocated). */
mcf_status mcf_batch_device_bytes(mcf_batch_t batch, size_t* bytes);

/* Queues a copy of *query (its arrays must stay valid until the request
 * completes) and returns a ticket.  A request whose footprint alone exceeds
 * the budget completes immediately with MCF_ERR_ADMISSION; a query the batch
 * planner would refuse returns MCF_ERR_INVALID_ARG and gets no ticket.
 * Completed requests stay listed, so every ticket can be polled or waited on
 * again, until mcf_server_release or mcf_server_destroy releases them. */
mcf_status mcf_server_submit(mcf_server_t s, const mcf_query* query, uint64_t* ticket);

/* Cancels a request that is still queued: it completes at once with status
 * MCF_ERR_CANCELLED and its output is not written.  A request that is already
 * running (or done) is not affected: the call returns MCF_ERR_INVALID_ARG.
 * Errors: MCF_ERR_INVALID_ARG (unknown ticket, or not queued). */
mcf_status mcf_server_cancel(mcf_server_t s, uint64_t ticket);

/* Forgets a completed request (its ticket becomes unknown), so a long-running
 * server does not keep every request it ever served.
 * Errors: MCF_ERR_INVALID_ARG (unknown ticket, or not completed yet). */
mcf_status mcf_server_release(mcf_server_t s, uint64_t ticket);

/* *done = 1 once the ticket's result is in query->out; *result is its status. */
mcf_status mcf_server_poll(mcf_server_t s, uint64_t ticket, int32_t* done, mcf_status* result);

/* Waits (at most timeout_s seconds; < 0 = no limit) for a ticket.  Returns
 * MCF_ERR_TIMEOUT if it is still running; *result is the request's status and
 * *latency_ms its submit-to-completion time (either may be NULL). */
mcf_status mcf_server_wait(mcf_server_t s, uint64_t ticket, double timeout_s, mcf_status* result,
                           double* latency_ms);

/* Counters and latency percentiles over the completed requests. */
mcf_status mcf_server_get_stats(mcf_server_t s, mcf_server_stats* out);

/* Waits for every queued request, then stops the server. NULL is a no-op. */
mcf_status mcf_server_destroy(mcf_server_t s);

/* ---------------------------------------------------------- allocation-free */

/* Size limits of mcf_total_communicability_noalloc (its fixed scratch array). */
#define MCF_NOALLOC_MAX_NODES (1LL << 17)
#define MCF_NOALLOC_MAX_WALKS (1LL << 25)

/* Total communicability f(A')1 for callers that cannot allocate device
 * memory -- for example code running inside a framework that owns every
 * device allocation, or a process whose allocator is already exhausted.  The
 * paper has no counterpart: this is the same computation as
 * mcf_total_communicability (same walks, same result), but the library
 * allocates nothing.  Its scratch is one file-scope device array of about
 * 17 MB that every GPU loading libmcf holds until the process exits; the
 * caller passes inputs and output:
 *   n, nnz           matrix size, n <= MCF_NOALLOC_MAX_NODES, nnz < 2^32;
 *   row_ptr, col_idx device pointers to a binary symmetric CSR (int64[n+1],
 *                    int32[nnz]); range and order are checked on the device
 *                    (MCF_ERR_INVALID_GRAPH, y left unchanged), symmetry is
 *                    the caller's duty;
 *   params           as for mcf_total_communicability; the walk count (N_s + n,
 *                    or walks_per_node * n) must not exceed MCF_NOALLOC_MAX_WALKS;
 *   y                device pointer to float64[n].
 * Sizes beyond the limits return MCF_ERR_INVALID_ARG with the limit in
 * mcf_last_error(), before any device work.  The first call on a device looks
 * up the array's device address (with that device current) and keeps it for
 * the life of the process, so make that first call before any stream capture,
 * and do not use the library across a cudaDeviceReset.  Every call uses the
 * same array and clears what must start at zero; calls that overlap on the
 * GPU (other streams, other threads) race on it and must be serialised by the
 * caller.  The call returns after its work is enqueued on params->stream
 * (after one short synchronisation for the CSR check). */
mcf_status mcf_total_communicability_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                                             const mcf_params* params, double* y);

/* ------------------------------------------------------------ measurement */

/* Measurement helpers; the paper has no counterpart.  A walk step reads one
 * record at a random position of an array of per-entry records, so the rate
 * at which this GPU serves random 8-byte reads bounds the walk kernels.
 * mcf_gather_probe allocates a device array of array_bytes (< 32 GiB), makes
 * about `reads` independent 8-byte reads at uniform random positions of it
 * (256-thread blocks, 2048 threads per SM, 16 reads in flight per thread,
 * L2 fetch granularity as the walk kernels use), times the launch with CUDA
 * events on `stream` after one warm-up launch, frees the array and returns
 * the reads per second.
 * Errors: MCF_ERR_INVALID_ARG, MCF_ERR_OOM, MCF_ERR_CUDA. */
mcf_status mcf_gather_probe(int64_t array_bytes, int64_t reads, void* stream, double* reads_per_s);

/* Number of kernel executions of this library on the current device since
 * the library was loaded: every kernel's first thread of block (0, 0, 0)
 * counts its own execution, so a replayed CUDA graph counts again.
 * Synchronises with the device (the counters are read back). */
mcf_status mcf_kernel_launches(uint64_t* count);

/* Host-side fault injection for testing callers' error paths; the paper has
 * no counterpart.  After `after` more successful device scratch allocations
 * of solves and batch plans (any thread), the next one fails as if the
 * device were full: the call returns MCF_ERR_OOM and releases what it had
 * taken; later allocations succeed again.
 * after < 0 switches the injection off.  Nothing runs on the GPU. */
mcf_status mcf_inject_allocation_failure(int64_t after);

/* Thread-local description of the last error of this thread ("" if none). */
const char* mcf_last_error(void);

/* Library version string. */
const char* mcf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MCF_H */
