// Internal declarations shared by the translation units of libmcf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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

// ---------------------------------------------------------------- helpers (host)
bool is_device_ptr(const void* p);
int num_sms();

// Exclusive scan of int64 values (in place allowed: out may equal in), n >= 0.
// Writes the total to *total_dev (device pointer) when non-null.  Deterministic.
mcf_status scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev, void* tmp, size_t tmp_bytes,
                    cudaStream_t st);
size_t scan_tmp_bytes(int64_t n);

// Float64 SpMV y = beta * (A x) (+ alpha * z if z), A the graph's matrix (values or binary).
mcf_status spmv_f64(const mcf_graph* g, const double* x, double* y, double beta, cudaStream_t st);

// Stream-ordered scratch allocation helpers.
struct Scratch {
    cudaStream_t st;
    void* ptrs[32];
    int n = 0;
    explicit Scratch(cudaStream_t s) : st(s) {}
    ~Scratch() {
        for (int i = 0; i < n; ++i) cudaFreeAsync(ptrs[i], st);
    }
    template <class T>
    mcf_status get(T** p, size_t count) {
        if (n >= 32) return fail(MCF_ERR_OOM, "too many scratch buffers");
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
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

}  // namespace mcf
