// Internal declarations shared by the translation units of libmcf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/mcf.h"

namespace mcf {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
const char* get_error();

#define MCF_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess) {                                                        \
            ::mcf::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));       \
            return MCF_ERR_CUDA;                                                        \
        }                                                                               \
    } while (0)

#define MCF_TRY(expr)                          \
    do {                                       \
        mcf_status _s = (expr);                \
        if (_s != MCF_OK) return _s;           \
    } while (0)

inline mcf_status fail(mcf_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

// ---------------------------------------------------------------- device graph
// Per-row entry of a weighted matrix: Vose alias bucket (prob, alias) and the
// CSR entry itself (column, value), packed so one 16-byte load serves the
// accepted branch of the alias draw.
struct __align__(16) WEntry {
    float prob;
    int32_t alias;
    int32_t col;
    float val;
};

}  // namespace mcf

struct mcf_graph {
    int64_t n = 0;
    int64_t nnz = 0;
    int64_t max_degree = 0;
    int64_t n_loops = 0;
    bool weighted = false;
    int64_t* row_ptr = nullptr;   // n + 1
    int32_t* col_idx = nullptr;   // nnz
    float* values = nullptr;      // nnz (weighted only)
    double* row_abs = nullptr;    // n: sum_j |a_ij| (unscaled; weighted only, binary uses deg)
    double* row_sq = nullptr;     // n: sum_j a_ij^2 (unscaled; weighted only)
    double* diag = nullptr;       // n: a_ii
    mcf::WEntry* went = nullptr;  // nnz (weighted only)
    // Binary graphs with nnz < 2^32, built on the first solve that walks with
    // them: node_od[i] = {row offset, degree} of node i and, per CSR entry,
    // edge_od[p] = node_od[col_idx[p]], the record of the neighbour an entry
    // leads to -- so a walk step reads one random 8-byte word instead of a
    // column index and then a node record.
    uint2* node_od = nullptr;     // n
    uint2* edge_od = nullptr;     // nnz
    // Symmetric binary graphs, built on the first subgraph-centrality solve:
    // per CSR entry the row offset of the neighbour it leads to (the key of
    // that neighbour in a row Q_k), read by the dot phase.
    uint32_t* edge_key = nullptr; // nnz
    // Column-major copy of A (column i: rows row_idx[col_ptr[i] .. col_ptr[i+1])
    // in increasing order, values col_values) and sum_j a_ji^2 per column.
    // For a symmetric A these alias the row arrays; a general A (created with
    // MCF_GRAPH_NONSYMMETRIC) owns them.
    bool symmetric = true;
    int64_t* col_ptr = nullptr;   // n + 1
    int32_t* row_idx = nullptr;   // nnz
    float* col_values = nullptr;  // nnz (weighted only)
    double* col_sq = nullptr;     // n (weighted only)
    double lambda_max = 0.0;      // cached by mcf_spectral_radius (0 = unknown)
    double gershgorin = 0.0;
    int device = 0;
};

namespace mcf {

// ---------------------------------------------------------------- row sums
// sum_j a_ij x[j] for the 32 rows base .. base+31 of a warp: lane t owns row
// base + t and sums it alone when it has at most SHORT entries; longer rows
// are then summed by the whole warp, one at a time.  FP64 instructions on
// this part issue at a small fraction of the FP32 rate, so every lane keeps
// its own row instead of reducing across lanes for every row.  Must be called
// by all 32 lanes with the same base.  Returns the sum of row base + lane.
template <int SHORT>
__device__ __forceinline__ double warp_row_sums(int64_t base, int64_t n, const int64_t* __restrict__ rp,
                                                const int32_t* __restrict__ col, const float* __restrict__ val,
                                                const double* __restrict__ x) {
    const int lane = threadIdx.x & 31;
    const int64_t row = base + lane;
    int64_t b = 0, e = 0;
    if (row < n) {
        b = rp[row];
        e = rp[row + 1];
    }
    double s = 0.0;
    const bool is_short = e - b <= SHORT;
    if (is_short)
        for (int64_t p = b; p < e; ++p) s += (val ? (double)val[p] : 1.0) * x[col[p]];
    unsigned longs = __ballot_sync(0xffffffffu, !is_short);
    while (longs) {
        const int t = __ffs(longs) - 1;
        longs &= longs - 1;
        const int64_t lb = __shfl_sync(0xffffffffu, b, t);
        const int64_t le = __shfl_sync(0xffffffffu, e, t);
        double part = 0.0;
        for (int64_t p = lb + lane; p < le; p += 32) part += (val ? (double)val[p] : 1.0) * x[col[p]];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
        if (lane == t) s = part;
    }
    return s;
}

// sum_j a_ij x[j] for the nr <= EPI_ROWS consecutive rows r0 .. r0+nr-1 of a
// CSR matrix, by a CTA of EPI_ROWS threads (all of them must call it): the
// rows' entries are contiguous, so the CTA streams them through shared
// memory EPI_CHUNK at a time (coalesced column reads, one gather of x per
// entry), then each row adds up its part of the chunk, a row of at most 32
// entries by its own thread in entry order and a longer row by its warp; no
// thread sums a long row alone.  prod holds EPI_CHUNK doubles and off
// EPI_ROWS + 1 offsets (shared).  Returns the sum of row r0 + threadIdx.x
// (0 beyond nr).
constexpr int EPI_ROWS = 256;
constexpr int EPI_CHUNK = 2048;
__device__ __forceinline__ double tile_row_sums(int64_t r0, int nr, const int64_t* __restrict__ rp,
                                                const int32_t* __restrict__ col, const float* __restrict__ val,
                                                const double* __restrict__ x, double* prod, int64_t* off) {
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int t = tid; t <= nr; t += EPI_ROWS) off[t] = rp[r0 + t];
    __syncthreads();
    const int64_t E0 = off[0], E1 = off[nr];
    const int64_t rb = tid < nr ? off[tid] : 0, re = tid < nr ? off[tid + 1] : 0;
    const bool is_long = re - rb > 32;
    double s = 0.0;
    for (int64_t c0 = E0; c0 < E1; c0 += EPI_CHUNK) {
        const int64_t c1 = c0 + EPI_CHUNK < E1 ? c0 + EPI_CHUNK : E1;
        // the float64 pipe of this part, not memory, bounds the loop: a binary
        // A stores x itself (no multiply by 1), leaving one add per entry
        if (val) {
#pragma unroll 4
            for (int64_t e = c0 + tid; e < c1; e += EPI_ROWS) prod[e - c0] = (double)val[e] * __ldg(&x[col[e]]);
        } else {
#pragma unroll 4
            for (int64_t e = c0 + tid; e < c1; e += EPI_ROWS) prod[e - c0] = __ldg(&x[col[e]]);
        }
        __syncthreads();
        if (!is_long) {
            const int64_t a = rb > c0 ? rb : c0, b = re < c1 ? re : c1;
            for (int64_t p = a; p < b; ++p) s += prod[p - c0];
        }
        unsigned longs = __ballot_sync(FULL, is_long && rb < c1 && re > c0);
        while (longs) {
            const int t = __ffs(longs) - 1;
            longs &= longs - 1;
            const int64_t lb = __shfl_sync(FULL, rb, t), le = __shfl_sync(FULL, re, t);
            const int64_t a = lb > c0 ? lb : c0, b = le < c1 ? le : c1;
            double part = 0.0;
            for (int64_t p = a + lane; p < b; p += 32) part += prod[p - c0];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(FULL, part, d);
            if (lane == t) s += part;
        }
        __syncthreads();
    }
    return s;
}

// Row sums for 32 listed rows: lane t owns row rows[base + t] (t < m).
template <int SHORT>
__device__ __forceinline__ double warp_listed_row_sums(int64_t base, int64_t m, const int64_t* __restrict__ rows,
                                                       const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                       const float* __restrict__ val, const double* __restrict__ x) {
    const int lane = threadIdx.x & 31;
    const int64_t t = base + lane;
    int64_t b = 0, e = 0;
    if (t < m) {
        const int64_t row = rows[t];
        b = rp[row];
        e = rp[row + 1];
    }
    double s = 0.0;
    const bool is_short = e - b <= SHORT;
    if (is_short)
        for (int64_t p = b; p < e; ++p) s += (val ? (double)val[p] : 1.0) * x[col[p]];
    unsigned longs = __ballot_sync(0xffffffffu, !is_short);
    while (longs) {
        const int tl = __ffs(longs) - 1;
        longs &= longs - 1;
        const int64_t lb = __shfl_sync(0xffffffffu, b, tl);
        const int64_t le = __shfl_sync(0xffffffffu, e, tl);
        double part = 0.0;
        for (int64_t p = lb + lane; p < le; p += 32) part += (val ? (double)val[p] : 1.0) * x[col[p]];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
        if (lane == tl) s = part;
    }
    return s;
}

// ---------------------------------------------------------------- kernel execution count
// Every kernel of the library counts its own executions: its first thread
// of block (0, 0, 0) adds one to a per-translation-unit device counter (a
// CUDA graph replay counts again).  kernel_runs_<unit>() read the counters
// of the current device; mcf_kernel_launches() returns their sum.
static __device__ unsigned long long g_kernel_runs;
#define MCF_KERNEL_ENTRY()                                                                              \
    do {                                                                                                \
        if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0)     \
            atomicAdd(&g_kernel_runs, 1ull);                                                            \
    } while (0)
static inline uint64_t this_unit_kernel_runs() {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_kernel_runs, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}
uint64_t kernel_runs_walk();
uint64_t kernel_runs_batch();
uint64_t kernel_runs_graph();
uint64_t kernel_runs_probe();

// ---------------------------------------------------------------- helpers (host)
bool is_device_ptr(const void* p);
int num_sms();

// Exclusive scan of int64 values (in place allowed: out may equal in), n >= 0.
// Its partition: tiles of SCAN_TILE values, one block of SCAN_THREADS each;
// the scratch holds one total per tile plus one.
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr size_t scan_tmp_bytes_for(int64_t n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE + 1) * sizeof(int64_t); }
// Writes the total to *total_dev (device pointer) when non-null.  Deterministic.
mcf_status scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev, void* tmp, size_t tmp_bytes,
                    cudaStream_t st);
size_t scan_tmp_bytes(int64_t n);

// Float64 SpMV y = beta * (A x) (+ alpha * z if z), A the graph's matrix (values or binary).
mcf_status spmv_f64(const mcf_graph* g, const double* x, double* y, double beta, cudaStream_t st);

// Host-side allocation-failure injection (mcf_inject_allocation_failure):
// returns true when this device allocation is the one chosen to fail.
bool injected_allocation_failure();

// Stream-ordered scratch allocation helpers.
struct Scratch {
    cudaStream_t st;
    void* ptrs[48];
    int n = 0;
    explicit Scratch(cudaStream_t s) : st(s) {}
    ~Scratch() {
        for (int i = 0; i < n; ++i) cudaFreeAsync(ptrs[i], st);
    }
    template <class T>
    mcf_status get(T** p, size_t count) {
        if (n >= 48) return fail(MCF_ERR_OOM, "too many scratch buffers");
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        if (injected_allocation_failure()) return fail(MCF_ERR_OOM, "device allocation failed (injected)");
        void* q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, bytes, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(MCF_ERR_OOM, std::string("cudaMallocAsync failed: ") + cudaGetErrorString(e));
        }
        ptrs[n++] = q;
        *p = static_cast<T*>(q);
        return MCF_OK;
    }
};

// ---------------------------------------------------------------- launch helpers (host)
inline int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 32));
}

template <class KernelT>
inline int persistent_grid(KernelT kernel, int threads, size_t smem) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1) per_sm = 1;
    return per_sm * num_sms();
}

// The largest float f <= W_c: for every float x, x > f exactly when
// (double)x > W_c, so the walks take the cutoff decision in float32.
inline float cutoff_f32(double wc) {
    float f = (float)wc;
    if ((double)f > wc) f = nextafterf(f, -INFINITY);
    return f;
}

inline uint2 philox_key(uint64_t seed) { return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)); }

// Every walk step reads one random 4- to 16-byte word; by default the L2
// fetches a whole line from DRAM on such a miss, moving about four times the
// bytes the step uses.  The walk kernels are launched with the context's L2
// fetch granularity lowered to 32 bytes (a per-context launch limit), and the
// previous value is put back right after the launch.
// Destroys the events it watches when the scope ends (also on early returns).
struct EventGuard {
    cudaEvent_t* a;
    cudaEvent_t* b;
    ~EventGuard() {
        if (a && *a) cudaEventDestroy(*a);
        if (b && *b) cudaEventDestroy(*b);
    }
};

struct ScopedL2Fetch {
    // The limit belongs to the whole context: concurrent solves (server
    // workers, user threads) share one setting, taken by the first entrant
    // and restored by the last one to leave.
    bool active = false;
    explicit ScopedL2Fetch(int bytes) {
        if (bytes <= 0) return;
        std::lock_guard<std::mutex> lk(state().mu);
        State& s = state();
        if (s.users++ == 0) {
            s.saved = cudaDeviceGetLimit(&s.old, cudaLimitMaxL2FetchGranularity) == cudaSuccess &&
                      cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes) == cudaSuccess;
            cudaGetLastError();
        }
        active = true;
    }
    ~ScopedL2Fetch() {
        if (!active) return;
        std::lock_guard<std::mutex> lk(state().mu);
        State& s = state();
        if (--s.users == 0 && s.saved) {
            cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, s.old);
            cudaGetLastError();
        }
    }

  private:
    struct State {
        std::mutex mu;
        int users = 0;
        size_t old = 0;
        bool saved = false;
    };
    static State& state() {
        static State s;
        return s;
    }
};

// Launch shape of the walk kernels (fixed; every value yields the same
// results, only the speed depends on them):
//   WALK_MINB        resident 256-thread blocks per SM the walk kernels' register budget is sized for;
//   WALK_GRAB        32-walk chunks a warp takes per atomic;
//   WALK_REFILL_MIN  idle lanes a total-communicability warp waits for before it refills them;
//   L2_FETCH_BYTES   L2 fetch granularity the walk kernels run with (ScopedL2Fetch);
//   DIAG_CAP_LOG2    log2 of the slots of the largest hashed row Q_k of RandFunmDiag.
constexpr int WALK_MINB = 5;
constexpr int WALK_GRAB = 4;
constexpr int WALK_REFILL_MIN = 16;
constexpr int L2_FETCH_BYTES = 32;
constexpr int DIAG_CAP_LOG2 = 12;

// Global-timer window (ns) of a batch's last run: from its first kernel to its last.
void batch_window(const mcf_batch* b, uint64_t* begin_ns, uint64_t* end_ns);
// Outcome of query i of a batch's last run (MCF_OK or MCF_ERR_ACCURACY_BUDGET).
mcf_status batch_query_status(const mcf_batch* b, int i);

// Builds the graph's node_od / edge_od arrays on first use (binary, nnz < 2^32).
mcf_status ensure_edge_od(mcf_graph* g, cudaStream_t st);
mcf_status ensure_edge_key(mcf_graph* g, cudaStream_t st);
// Keeps freed stream-ordered scratch in the device's default pool.
void keep_pool_memory();

// A graph's device arrays come from the device's stream-ordered pool, which
// keeps freed memory (keep_pool_memory), so creating and destroying graphs of
// similar sizes reuses memory instead of mapping new pages every time.
inline cudaError_t graph_alloc(void** p, size_t bytes, cudaStream_t st = 0) {
    keep_pool_memory();
    return cudaMallocAsync(p, bytes, st);
}
template <class T>
inline cudaError_t graph_alloc(T** p, size_t bytes, cudaStream_t st = 0) {
    return graph_alloc(reinterpret_cast<void**>(p), bytes, st);
}
inline void graph_free(void* p, cudaStream_t st = 0) {
    if (p) cudaFreeAsync(p, st);
}

}  // namespace mcf
