// Graph residency and preprocessing (the first step of the method's path):
// CSR upload and validation, per-row sums of Definition 1 (unscaled), Vose
// alias tables for weighted rows (Eq. definition1), the largest eigenvalue by
// power iteration for scale = 1/lambda_max, the Gershgorin bound
// (Section 4.5), and the library's shared device utilities (scan, SpMV).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "mcf_internal.cuh"

namespace mcf {

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
const char* get_error() { return g_last_error.c_str(); }

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// ------------------------------------------------------------------ scan
// Three-phase exclusive scan: per-block totals, a single-block scan of the
// totals, then per-block scans offset by the scanned totals.  The partition
// is fixed, so the result does not depend on timing.
// SCAN_THREADS, SCAN_ITEMS and SCAN_TILE are declared in mcf_internal.cuh.

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total.
__device__ int64_t block_excl_scan(int64_t v, int64_t* total) {
    __shared__ int64_t warp_tot[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan(v);
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t t = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
        t = warp_incl_scan(t);
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    int64_t base = wid ? warp_tot[wid - 1] : 0;
    *total = warp_tot[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return base + inc - v;
}

__global__ void scan_block_totals(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ tot) {
    MCF_KERNEL_ENTRY();
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) s += in[base + k];
    int64_t total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) tot[blockIdx.x] = total;
}

__global__ void scan_totals_single(int64_t* __restrict__ tot, int64_t nb, int64_t* __restrict__ total_out) {
    MCF_KERNEL_ENTRY();
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_THREADS) {
        int64_t i = b0 + threadIdx.x;
        int64_t v = i < nb ? tot[i] : 0;
        int64_t chunk;
        int64_t ex = block_excl_scan(v, &chunk);
        if (i < nb) tot[i] = carry + ex;
        carry += chunk;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void scan_apply(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                           const int64_t* __restrict__ tot) {
    MCF_KERNEL_ENTRY();
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t ex = block_excl_scan(s, &total) + tot[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
}

size_t scan_tmp_bytes(int64_t n) { return scan_tmp_bytes_for(n); }

mcf_status scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev, void* tmp, size_t tmp_bytes,
                    cudaStream_t st) {
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tmp_bytes < scan_tmp_bytes(n)) return fail(MCF_ERR_INVALID_ARG, "scan scratch too small");
    int64_t* tot = static_cast<int64_t*>(tmp);
    if (nb > 0) scan_block_totals<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, tot);
    scan_totals_single<<<1, SCAN_THREADS, 0, st>>>(tot, nb, total_dev);
    if (nb > 0) scan_apply<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, tot);
    MCF_CUDA_TRY(cudaGetLastError());
    return MCF_OK;
}

// ------------------------------------------------------------------ validation
enum : uint32_t {
    BAD_ROWPTR = 1u,
    BAD_COLUMN = 2u,
    BAD_ORDER = 4u,
    BAD_VALUE = 8u,
    BAD_SYMMETRY = 16u,
};

__device__ __forceinline__ unsigned long long pair_hash(uint32_t lo, uint32_t hi, uint32_t vbits) {
    unsigned long long z = ((unsigned long long)lo << 32 | hi) ^ ((unsigned long long)vbits * 0xD1B54A32D192ED03ull);
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Warp per row: checks order, range and finiteness; records loops, the
// diagonal (zeroed beforehand) and the maximum degree.  Symmetry: every
// off-diagonal entry (i, j) adds a 64-bit mix of the unordered pair and its
// value to sums[0] when i < j and to sums[1] when i > j; the matrix is
// symmetric exactly when the two multisets agree, which the equality of the
// wrap-around sums confirms up to a 2^-64 chance of a missed difference.
__global__ void validate_rows(int64_t n, int64_t nnz, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const float* __restrict__ val, uint32_t* __restrict__ bad,
                              unsigned long long* __restrict__ maxdeg, unsigned long long* __restrict__ loops,
                              double* __restrict__ diag, unsigned long long* __restrict__ sums) {
    MCF_KERNEL_ENTRY();
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long s_lo = 0, s_hi = 0, dmax = 0, nloops = 0;
    uint32_t flags = 0;
    for (int64_t i = warp; i < n; i += nwarps) {
        int64_t b = rp[i], e = rp[i + 1];
        if (b > e || b < 0 || e > nnz) {
            flags |= BAD_ROWPTR;
            continue;
        }
        dmax = max(dmax, (unsigned long long)(e - b));
        for (int64_t p = b + lane; p < e; p += 32) {
            int32_t j = col[p];
            if (j < 0 || j >= n) { flags |= BAD_COLUMN; continue; }
            if (p > b && col[p - 1] >= j) flags |= BAD_ORDER;
            float a = val ? val[p] : 1.0f;
            if (!isfinite(a)) flags |= BAD_VALUE;
            if (j == i) {
                ++nloops;
                diag[i] = (double)a;
                continue;
            }
            const uint32_t vb = val ? __float_as_uint(a) : 0u;
            if ((int64_t)j > i) s_lo += pair_hash((uint32_t)i, (uint32_t)j, vb);
            else s_hi += pair_hash((uint32_t)j, (uint32_t)i, vb);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        s_lo += __shfl_down_sync(0xffffffffu, s_lo, d);
        s_hi += __shfl_down_sync(0xffffffffu, s_hi, d);
        nloops += __shfl_down_sync(0xffffffffu, nloops, d);
        flags |= __shfl_down_sync(0xffffffffu, flags, d);
    }
    // one atomic per warp for each total (per-row atomics on one address serialise)
    if (lane == 0) {
        if (s_lo) atomicAdd(&sums[0], s_lo);
        if (s_hi) atomicAdd(&sums[1], s_hi);
        if (nloops) atomicAdd(loops, nloops);
        if (dmax) atomicMax(maxdeg, dmax);
        if (flags) atomicOr(bad, flags);
    }
}

// Thread per row, in CSR order (the same order as the oracle's definition):
// sum |a_ij|, sum a_ij^2, and Vose's alias table of t_ij = |a_ij| / sum_k |a_ik|
// with stack work lists filled in column order.  Every product and sum is
// rounded on its own (no contraction), so the tables are bit-reproducible.
__global__ void weighted_rows(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const float* __restrict__ val, double* __restrict__ row_abs,
                              double* __restrict__ row_sq, WEntry* __restrict__ went, double* __restrict__ s_buf,
                              int32_t* __restrict__ small_buf, int32_t* __restrict__ large_buf) {
    MCF_KERNEL_ENTRY();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t b = rp[i], e = rp[i + 1];
    int64_t d = e - b;
    double sa = 0.0, sq = 0.0;
    for (int64_t p = b; p < e; ++p) {
        double a = (double)val[p];
        sa = __dadd_rn(sa, fabs(a));
        sq = __dadd_rn(sq, __dmul_rn(a, a));
    }
    row_abs[i] = sa;
    row_sq[i] = sq;
    if (d == 0) return;
    double* s = s_buf + b;
    int32_t* sm = small_buf + b;
    int32_t* lg = large_buf + b;
    int64_t ns = 0, nl = 0;
    for (int64_t j = 0; j < d; ++j) {
        s[j] = __ddiv_rn(__dmul_rn((double)d, fabs((double)val[b + j])), sa);
        if (s[j] < 1.0) sm[ns++] = (int32_t)j;
        else lg[nl++] = (int32_t)j;
    }
    while (ns > 0 && nl > 0) {
        int32_t l = sm[--ns];
        int32_t gg = lg[--nl];
        went[b + l].prob = __double2float_rn(s[l]);
        went[b + l].alias = gg;
        s[gg] = __dadd_rn(__dadd_rn(s[gg], s[l]), -1.0);
        if (s[gg] < 1.0) sm[ns++] = gg;
        else lg[nl++] = gg;
    }
    while (nl > 0) { int32_t gg = lg[--nl]; went[b + gg].prob = 1.0f; went[b + gg].alias = gg; }
    while (ns > 0) { int32_t l = sm[--ns]; went[b + l].prob = 1.0f; went[b + l].alias = l; }
    for (int64_t j = 0; j < d; ++j) {
        went[b + j].col = col[b + j];
        went[b + j].val = val[b + j];
    }
}

// ------------------------------------------------------------------ SpMV and reductions
// A warp covers 32 consecutive rows (warp_row_sums).
__global__ void spmv_f64_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                const float* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                                double beta) {
    MCF_KERNEL_ENTRY();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
        const double s = warp_row_sums<32>(base, n, rp, col, val, x);
        const int64_t row = base + (threadIdx.x & 31);
        if (row < n) y[row] = beta * s;
    }
}

mcf_status spmv_f64(const mcf_graph* g, const double* x, double* y, double beta, cudaStream_t st) {
    if (g->n == 0) return MCF_OK;
    const int64_t blocks = std::min<int64_t>((g->n + 255) / 256, (int64_t)num_sms() * 16);
    spmv_f64_kernel<<<(unsigned)blocks, 256, 0, st>>>(g->n, g->row_ptr, g->col_idx, g->values, x, y, beta);
    MCF_CUDA_TRY(cudaGetLastError());
    return MCF_OK;
}

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 256;

// Deterministic two-level reductions: fixed grid, per-block partials, then one block.
__device__ double block_sum(double v) {
    __shared__ double part[RED_THREADS / 32];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < RED_THREADS / 32; ++w) s += part[w];
    __syncthreads();
    return s;
}

// part[b] = (x . y, (x + y) . (x + y)) over block b's grid-stride share
__global__ void power_partials(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                               double* __restrict__ part) {
    MCF_KERNEL_ENTRY();
    double d = 0.0, q = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double xi = x[i], yi = y[i];
        d += xi * yi;
        double z = xi + yi;
        q += z * z;
    }
    double sd = block_sum(d);
    double sq = block_sum(q);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = sd; part[2 * blockIdx.x + 1] = sq; }
}

__global__ void power_finish(const double* __restrict__ part, int nb, double* __restrict__ out) {
    MCF_KERNEL_ENTRY();
    double d = 0.0, q = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) { d += part[2 * b]; q += part[2 * b + 1]; }
    d = block_sum(d);
    q = block_sum(q);
    if (threadIdx.x == 0) { out[0] = d; out[1] = q; }
}

// x <- (x + y) / norm
__global__ void power_update(int64_t n, double* __restrict__ x, const double* __restrict__ y,
                             const double* __restrict__ stats) {
    MCF_KERNEL_ENTRY();
    double inv = 1.0 / sqrt(stats[1]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (x[i] + y[i]) * inv;
}

// y_i = sqrt(s_i) sum_j |a_ij| sqrt(s_j) x_j with s_i = sum_j |a_ij| (deg_i for
// a binary A): the product with S = D^1/2 |A| D^1/2, which is similar to the
// second-moment matrix D |A| of the walk weights (D = diag(s)).  Thread per row.
__global__ void moment_spmv(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const float* __restrict__ val, const double* __restrict__ row_abs,
                            const double* __restrict__ x, double* __restrict__ y) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            const int32_t j = col[p];
            const double sj = row_abs ? row_abs[j] : (double)(rp[j + 1] - rp[j]);
            acc += (val ? fabs((double)val[p]) : 1.0) * sqrt(sj) * x[j];
        }
        const double si = row_abs ? row_abs[i] : (double)(rp[i + 1] - rp[i]);
        y[i] = sqrt(si) * acc;
    }
}

// x <- (y + c x) / ||y + c x|| with c = stats[0] (the current Rayleigh quotient:
// a positive shift that keeps the Perron root dominant on bipartite graphs).
__global__ void moment_update(int64_t n, double* __restrict__ x, const double* __restrict__ y,
                              const double* __restrict__ stats, double* __restrict__ z) {
    MCF_KERNEL_ENTRY();
    const double c = stats[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = y[i] + c * x[i];
}

// dst = a * src
__global__ void scale_copy(int64_t n, const double* __restrict__ src, double a, double* __restrict__ dst) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = a * src[i];
}

__global__ void fill_f64(int64_t n, double* __restrict__ x, double v) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

__global__ void max_f64(int64_t n, const double* __restrict__ x, unsigned long long* __restrict__ out) {
    MCF_KERNEL_ENTRY();
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, x[i]);
    // non-negative doubles order like their bit patterns
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

}  // namespace mcf

using namespace mcf;

// ====================================================================== C ABI
uint64_t mcf::kernel_runs_graph() { return this_unit_kernel_runs(); }

extern "C" {

const char* mcf_last_error(void) { return get_error(); }
const char* mcf_version(void) { return "mcf 0.1 (sm_103a)"; }

// sum_j a_ji^2 of every column i, over the column-major copy in increasing
// row order, each product and sum rounded on its own.
__global__ void column_sq(int64_t n, const int64_t* __restrict__ cp, const float* __restrict__ cv,
                          double* __restrict__ out) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double sq = 0.0;
        for (int64_t q = cp[i]; q < cp[i + 1]; ++q) {
            const double a = (double)cv[q];
            sq = __dadd_rn(sq, __dmul_rn(a, a));
        }
        out[i] = sq;
    }
}

namespace {

// The column-major copy of a general A: a counting sort over the rows, done
// on the host (it visits the rows in order, so every column lists its rows
// in increasing order, deterministically), then copied to the device.
mcf_status build_columns(mcf_graph* g, const int64_t* row_ptr, const int32_t* col_idx, const float* values,
                         bool dev_in) {
    const int64_t n = g->n, nnz = g->nnz;
    std::vector<int64_t> h_rp;
    std::vector<int32_t> h_ci;
    std::vector<float> h_va;
    const int64_t* rp = row_ptr;
    const int32_t* ci = col_idx;
    const float* va = values;
    if (dev_in) {
        h_rp.resize((size_t)n + 1);
        h_ci.resize((size_t)std::max<int64_t>(nnz, 1));
        MCF_CUDA_TRY(cudaMemcpy(h_rp.data(), g->row_ptr, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
        if (nnz > 0)
            MCF_CUDA_TRY(cudaMemcpy(h_ci.data(), g->col_idx, (size_t)nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
        rp = h_rp.data();
        ci = h_ci.data();
        if (values) {
            h_va.resize((size_t)std::max<int64_t>(nnz, 1));
            if (nnz > 0)
                MCF_CUDA_TRY(cudaMemcpy(h_va.data(), g->values, (size_t)nnz * sizeof(float), cudaMemcpyDeviceToHost));
            va = h_va.data();
        }
    }
    std::vector<int64_t> cp((size_t)n + 1, 0);
    for (int64_t p = 0; p < nnz; ++p) ++cp[(size_t)ci[p] + 1];
    for (int64_t i = 0; i < n; ++i) cp[(size_t)i + 1] += cp[(size_t)i];
    std::vector<int64_t> cur(cp.begin(), cp.end() - 1);
    std::vector<int32_t> ri((size_t)std::max<int64_t>(nnz, 1));
    std::vector<float> cv(values ? (size_t)std::max<int64_t>(nnz, 1) : 0);
    for (int64_t r = 0; r < n; ++r)
        for (int64_t p = rp[r]; p < rp[r + 1]; ++p) {
            const int64_t q = cur[(size_t)ci[p]]++;
            ri[(size_t)q] = (int32_t)r;
            if (values) cv[(size_t)q] = va[p];
        }
    if (graph_alloc(&g->col_ptr, (size_t)(n + 1) * sizeof(int64_t)) != cudaSuccess ||
        graph_alloc(&g->row_idx, ri.size() * sizeof(int32_t)) != cudaSuccess ||
        (values && graph_alloc(&g->col_values, cv.size() * sizeof(float)) != cudaSuccess) ||
        (values && graph_alloc(&g->col_sq, (size_t)std::max<int64_t>(n, 1) * sizeof(double)) != cudaSuccess)) {
        cudaGetLastError();
        return fail(MCF_ERR_OOM, "device allocation of the column-major copy failed");
    }
    MCF_CUDA_TRY(cudaMemcpy(g->col_ptr, cp.data(), (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    MCF_CUDA_TRY(cudaMemcpy(g->row_idx, ri.data(), ri.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (values) {
        MCF_CUDA_TRY(cudaMemcpy(g->col_values, cv.data(), cv.size() * sizeof(float), cudaMemcpyHostToDevice));
        if (n > 0) column_sq<<<grid_for(n, 256), 256>>>(n, g->col_ptr, g->col_values, g->col_sq);
        MCF_CUDA_TRY(cudaGetLastError());
    }
    return MCF_OK;
}

}  // namespace

mcf_status mcf_create_graph(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const float* values,
                            uint32_t flags, mcf_graph_t* out) {
    set_error("");
    if (!out) return fail(MCF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || n > INT32_MAX) return fail(MCF_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    if (!row_ptr) return fail(MCF_ERR_INVALID_ARG, "row_ptr is NULL");
    const bool dev_in = (flags & MCF_GRAPH_DEVICE_PTRS) != 0;
    int64_t ends[2];
    if (dev_in) {
        MCF_CUDA_TRY(cudaMemcpy(&ends[0], row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost));
        MCF_CUDA_TRY(cudaMemcpy(&ends[1], row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    } else {
        ends[0] = row_ptr[0];
        ends[1] = row_ptr[n];
    }
    if (ends[0] != 0 || ends[1] < 0) return fail(MCF_ERR_INVALID_GRAPH, "row_ptr[0] must be 0 and row_ptr[n] >= 0");
    const int64_t nnz = ends[1];
    if (nnz > 0 && !col_idx) return fail(MCF_ERR_INVALID_ARG, "col_idx is NULL");
    mcf_graph* g = new (std::nothrow) mcf_graph();
    if (!g) return fail(MCF_ERR_OOM, "host allocation failed");
    cudaGetDevice(&g->device);
    g->n = n;
    g->nnz = nnz;
    g->weighted = values != nullptr;
    auto cleanup = [&](mcf_status s) {
        mcf_destroy_graph(g);
        return s;
    };
    const cudaMemcpyKind kind = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (graph_alloc(&g->row_ptr, (size_t)(n + 1) * sizeof(int64_t)) != cudaSuccess ||
        graph_alloc(&g->col_idx, (size_t)std::max<int64_t>(nnz, 1) * sizeof(int32_t)) != cudaSuccess ||
        graph_alloc(&g->diag, (size_t)std::max<int64_t>(n, 1) * sizeof(double)) != cudaSuccess) {
        // the first device call of a graph: tell a missing device or driver from a full one
        const cudaError_t e = cudaGetLastError();
        if (e != cudaErrorMemoryAllocation)
            return cleanup(fail(MCF_ERR_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e)));
        return cleanup(fail(MCF_ERR_OOM, "device allocation of the CSR failed"));
    }
    if (cudaMemcpy(g->row_ptr, row_ptr, (size_t)(n + 1) * sizeof(int64_t), kind) != cudaSuccess ||
        (nnz > 0 && cudaMemcpy(g->col_idx, col_idx, (size_t)nnz * sizeof(int32_t), kind) != cudaSuccess))
        return cleanup(fail(MCF_ERR_CUDA, std::string("CSR copy failed: ") + cudaGetErrorString(cudaGetLastError())));
    if (g->weighted) {
        if (graph_alloc(&g->values, (size_t)std::max<int64_t>(nnz, 1) * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return cleanup(fail(MCF_ERR_OOM, "device allocation of the values failed"));
        }
        if (nnz > 0 && cudaMemcpy(g->values, values, (size_t)nnz * sizeof(float), kind) != cudaSuccess)
            return cleanup(fail(MCF_ERR_CUDA, "values copy failed"));
    }
    // validation
    struct Flags { uint32_t bad; uint32_t pad; unsigned long long maxdeg; unsigned long long loops; unsigned long long sums[2]; };
    Flags* dflags = nullptr;
    if (graph_alloc(&dflags, sizeof(Flags)) != cudaSuccess) { cudaGetLastError(); return cleanup(fail(MCF_ERR_OOM, "alloc")); }
    cudaMemset(dflags, 0, sizeof(Flags));
    cudaMemset(g->diag, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(double));
    if (n > 0) {
        int blocks = (int)std::min<int64_t>((n + 7) / 8, (int64_t)num_sms() * 16);
        validate_rows<<<blocks, 256>>>(n, nnz, g->row_ptr, g->col_idx, g->values, &dflags->bad, &dflags->maxdeg,
                                       &dflags->loops, g->diag, dflags->sums);
    }
    Flags hf;
    cudaError_t e = cudaMemcpy(&hf, dflags, sizeof(Flags), cudaMemcpyDeviceToHost);
    graph_free(dflags);
    if (e != cudaSuccess) return cleanup(fail(MCF_ERR_CUDA, std::string("validation: ") + cudaGetErrorString(e)));
    const bool general = (flags & MCF_GRAPH_NONSYMMETRIC) != 0;
    if (!general && !(hf.bad & (BAD_ROWPTR | BAD_COLUMN)) && hf.sums[0] != hf.sums[1]) hf.bad |= BAD_SYMMETRY;
    if (hf.bad) {
        std::string why;
        if (hf.bad & BAD_ROWPTR) why += " row_ptr not non-decreasing within [0, nnz];";
        if (hf.bad & BAD_COLUMN) why += " column index out of range;";
        if (hf.bad & BAD_ORDER) why += " columns not strictly increasing within a row (unsorted or duplicate);";
        if (hf.bad & BAD_VALUE) why += " non-finite value;";
        if (hf.bad & BAD_SYMMETRY) why += " matrix not symmetric;";
        return cleanup(fail(MCF_ERR_INVALID_GRAPH, "invalid graph:" + why));
    }
    g->max_degree = (int64_t)hf.maxdeg;
    g->n_loops = (int64_t)hf.loops;
    g->gershgorin = (double)g->max_degree;
    if (g->weighted && n > 0) {
        double* s_buf = nullptr;
        int32_t *sm = nullptr, *lg = nullptr;
        size_t m = (size_t)std::max<int64_t>(nnz, 1);
        if (graph_alloc(&g->row_abs, (size_t)n * sizeof(double)) != cudaSuccess ||
            graph_alloc(&g->row_sq, (size_t)n * sizeof(double)) != cudaSuccess ||
            graph_alloc(&g->went, m * sizeof(WEntry)) != cudaSuccess || graph_alloc(&s_buf, m * sizeof(double)) != cudaSuccess ||
            graph_alloc(&sm, m * sizeof(int32_t)) != cudaSuccess || graph_alloc(&lg, m * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            graph_free(s_buf); graph_free(sm); graph_free(lg);
            return cleanup(fail(MCF_ERR_OOM, "device allocation of the alias tables failed"));
        }
        weighted_rows<<<(unsigned)((n + 127) / 128), 128>>>(n, g->row_ptr, g->col_idx, g->values, g->row_abs, g->row_sq,
                                                             g->went, s_buf, sm, lg);
        unsigned long long* dm = nullptr;
        graph_alloc(&dm, sizeof(unsigned long long));
        cudaMemset(dm, 0, sizeof(unsigned long long));
        max_f64<<<num_sms(), 256>>>(n, g->row_abs, dm);
        unsigned long long hm = 0;
        e = cudaMemcpy(&hm, dm, sizeof(hm), cudaMemcpyDeviceToHost);
        graph_free(dm); graph_free(s_buf); graph_free(sm); graph_free(lg);
        if (e != cudaSuccess) return cleanup(fail(MCF_ERR_CUDA, std::string("alias tables: ") + cudaGetErrorString(e)));
        double gm;
        memcpy(&gm, &hm, sizeof(gm));
        g->gershgorin = gm;
    }
    if (general) {
        g->symmetric = false;
        mcf_status rc = build_columns(g, row_ptr, col_idx, values, dev_in);
        if (rc != MCF_OK) return cleanup(rc);
    } else {
        g->col_ptr = g->row_ptr;
        g->row_idx = g->col_idx;
        g->col_values = g->values;
        g->col_sq = g->row_sq;
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cleanup(fail(MCF_ERR_CUDA, std::string("create_graph: ") + cudaGetErrorString(e)));
    *out = g;
    return MCF_OK;
}

mcf_status mcf_destroy_graph(mcf_graph_t g) {
    if (!g) return MCF_OK;
    cudaDeviceSynchronize();
    graph_free(g->row_ptr);
    graph_free(g->col_idx);
    graph_free(g->values);
    graph_free(g->row_abs);
    graph_free(g->row_sq);
    graph_free(g->diag);
    graph_free(g->went);
    graph_free(g->node_od);
    graph_free(g->edge_od);
    graph_free(g->edge_key);
    if (!g->symmetric) {
        graph_free(g->col_ptr);
        graph_free(g->row_idx);
        graph_free(g->col_values);
        graph_free(g->col_sq);
    }
    delete g;
    return MCF_OK;
}

mcf_status mcf_graph_info(mcf_graph_t g, int64_t* n, int64_t* nnz, int64_t* max_degree, int64_t* n_loops) {
    if (!g) return fail(MCF_ERR_INVALID_ARG, "graph is NULL");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (max_degree) *max_degree = g->max_degree;
    if (n_loops) *n_loops = g->n_loops;
    return MCF_OK;
}

mcf_status mcf_gershgorin(mcf_graph_t g, double* bound) {
    if (!g || !bound) return fail(MCF_ERR_INVALID_ARG, "NULL argument");
    *bound = g->gershgorin;
    return MCF_OK;
}

mcf_status mcf_spectral_radius(mcf_graph_t g, double tol, int32_t max_iter, double* lambda_max) {
    set_error("");
    if (!g || !lambda_max) return fail(MCF_ERR_INVALID_ARG, "NULL argument");
    if (!g->symmetric)
        return fail(MCF_ERR_UNSUPPORTED, "the power iteration needs a symmetric A; pass the scale explicitly");
    static std::mutex mu;   // one power iteration at a time (it caches its result on the graph)
    std::lock_guard<std::mutex> lk(mu);
    if (!(tol > 0.0) || max_iter < 1) return fail(MCF_ERR_INVALID_ARG, "tol must be > 0 and max_iter >= 1");
    if (g->n == 0 || g->nnz == 0) {
        *lambda_max = 0.0;
        g->lambda_max = 0.0;
        return MCF_OK;
    }
    cudaStream_t st = 0;
    double *x = nullptr, *y = nullptr, *part = nullptr, *hst = nullptr;
    const int64_t n = g->n;
    if (cudaMalloc(&x, n * sizeof(double)) != cudaSuccess || cudaMalloc(&y, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&part, (2 * RED_BLOCKS + 2) * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&hst, 2 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(x); cudaFree(y); cudaFree(part); cudaFreeHost(hst);
        return fail(MCF_ERR_OOM, "power iteration scratch");
    }
    mcf_status rc = MCF_OK;
    fill_f64<<<num_sms() * 4, 256, 0, st>>>(n, x, 1.0 / sqrt((double)n));
    double lam = 0.0, prev = 0.0;
    for (int it = 0; it < max_iter; ++it) {
        rc = spmv_f64(g, x, y, 1.0, st);
        if (rc != MCF_OK) break;
        power_partials<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, x, y, part);
        power_finish<<<1, RED_THREADS, 0, st>>>(part, RED_BLOCKS, part + 2 * RED_BLOCKS);
        power_update<<<num_sms() * 4, 256, 0, st>>>(n, x, y, part + 2 * RED_BLOCKS);
        if (cudaMemcpy(hst, part + 2 * RED_BLOCKS, 2 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = fail(MCF_ERR_CUDA, std::string("power iteration: ") + cudaGetErrorString(cudaGetLastError()));
            break;
        }
        lam = hst[0];   // Rayleigh quotient x^T A x with ||x|| = 1
        if (it > 0 && fabs(lam - prev) <= tol * fabs(lam)) break;
        prev = lam;
    }
    cudaFree(x); cudaFree(y); cudaFree(part); cudaFreeHost(hst);
    if (rc != MCF_OK) return rc;
    g->lambda_max = lam;
    *lambda_max = lam;
    return MCF_OK;
}

mcf_status mcf_second_moment_radius(mcf_graph_t g, double scale, double tol, int32_t max_iter, double* rho) {
    set_error("");
    if (!g || !rho) return fail(MCF_ERR_INVALID_ARG, "NULL argument");
    if (!g->symmetric)
        return fail(MCF_ERR_UNSUPPORTED, "the power iteration needs a symmetric A");
    if (!(tol > 0.0) || max_iter < 1 || !(scale >= 0.0) || !isfinite(scale))
        return fail(MCF_ERR_INVALID_ARG, "tol > 0, max_iter >= 1 and a finite scale >= 0 required");
    const double gam = scale == 0.0 ? 1.0 : scale;
    if (g->n == 0 || g->nnz == 0) {
        *rho = 0.0;
        return MCF_OK;
    }
    cudaStream_t st = 0;
    const int64_t n = g->n;
    double *x = nullptr, *y = nullptr, *z = nullptr, *part = nullptr, *hst = nullptr;
    if (cudaMalloc(&x, n * sizeof(double)) != cudaSuccess || cudaMalloc(&y, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&z, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&part, (2 * RED_BLOCKS + 4) * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&hst, 2 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(x); cudaFree(y); cudaFree(z); cudaFree(part); cudaFreeHost(hst);
        return fail(MCF_ERR_OOM, "power iteration scratch");
    }
    mcf_status rc = MCF_OK;
    const int grid = num_sms() * 4;
    fill_f64<<<grid, 256, 0, st>>>(n, x, 1.0 / sqrt((double)n));
    cudaMemsetAsync(part + 2 * RED_BLOCKS + 2, 0, 2 * sizeof(double), st);   // shift 0 in the first step
    double lam = 0.0, prev = 0.0;
    for (int it = 0; it < max_iter; ++it) {
        moment_spmv<<<grid, 256, 0, st>>>(n, g->row_ptr, g->col_idx, g->values, g->row_abs, x, y);
        // z = S x + c x; x . S x (the Rayleigh quotient, ||x|| = 1) and ||z||^2
        moment_update<<<grid, 256, 0, st>>>(n, x, y, part + 2 * RED_BLOCKS + 2, z);
        power_partials<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, x, y, part);
        power_finish<<<1, RED_THREADS, 0, st>>>(part, RED_BLOCKS, part + 2 * RED_BLOCKS);
        if (cudaMemcpy(hst, part + 2 * RED_BLOCKS, 2 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = fail(MCF_ERR_CUDA, std::string("power iteration: ") + cudaGetErrorString(cudaGetLastError()));
            break;
        }
        lam = hst[0];
        // next iterate: z / ||z||, shift = this Rayleigh quotient
        double zz = 0.0;
        power_partials<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, z, z, part);
        power_finish<<<1, RED_THREADS, 0, st>>>(part, RED_BLOCKS, part + 2 * RED_BLOCKS);
        if (cudaMemcpy(hst, part + 2 * RED_BLOCKS, 2 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = fail(MCF_ERR_CUDA, std::string("power iteration: ") + cudaGetErrorString(cudaGetLastError()));
            break;
        }
        zz = hst[0];
        if (!(zz > 0.0)) break;
        scale_copy<<<grid, 256, 0, st>>>(n, z, 1.0 / sqrt(zz), x);
        const double shift = lam;
        cudaMemcpyAsync(part + 2 * RED_BLOCKS + 2, &shift, sizeof(double), cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
        if (it > 0 && fabs(lam - prev) <= tol * fabs(lam)) break;
        prev = lam;
    }
    cudaFree(x); cudaFree(y); cudaFree(z); cudaFree(part); cudaFreeHost(hst);
    if (rc != MCF_OK) return rc;
    *rho = gam * gam * lam;
    return MCF_OK;
}

}  // extern "C"
