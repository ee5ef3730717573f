// Measurement helpers of libmcf (no counterpart in the paper): the random
// 8-byte gather rate of this GPU's memory, the ceiling a walk kernel that
// makes one random read per step is measured against, and the count of
// kernels the library has executed.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "mcf_internal.cuh"

namespace mcf {

// A 32-bit integer hash (xorshift-multiply finaliser) that spreads the read
// indices of thread t and read i uniformly over the array.
__device__ __forceinline__ uint32_t probe_mix(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Every thread makes `iters` reads of 8 bytes at independent uniform random
// positions of a[0 .. S), UNROLL of them in flight at a time, and folds the
// values into a sink so the reads cannot be dropped.
constexpr int PROBE_UNROLL = 16;
__global__ void __launch_bounds__(256) gather_probe_kernel(const uint2* __restrict__ a, uint64_t S, int iters,
                                                           uint32_t* __restrict__ sink) {
    MCF_KERNEL_ENTRY();
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int i = 0; i < iters; i += PROBE_UNROLL) {
        uint2 v[PROBE_UNROLL];
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) {
            const uint32_t h = probe_mix(t * 0x9E3779B1u + (uint32_t)(i + u) * 0x85EBCA6Bu);
            const uint64_t idx = ((uint64_t)h * S) >> 32;   // < S
            asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];"
                         : "=r"(v[u].x), "=r"(v[u].y)
                         : "l"(a + idx));
        }
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) acc ^= v[u].x + v[u].y;
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;   // practically never taken
}

}  // namespace mcf

using namespace mcf;

uint64_t mcf::kernel_runs_probe() { return this_unit_kernel_runs(); }

// The allocation counter of mcf_inject_allocation_failure: -1 = off, else the
// number of scratch allocations that still succeed before one fails.
static std::atomic<long long> g_fail_after{-1};

bool mcf::injected_allocation_failure() {
    long long v = g_fail_after.load(std::memory_order_relaxed);
    while (v >= 0) {
        if (g_fail_after.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return v == 0;
    }
    return false;
}

extern "C" {

mcf_status mcf_gather_probe(int64_t array_bytes, int64_t reads, void* stream, double* reads_per_s) {
    set_error("");
    if (!reads_per_s) return fail(MCF_ERR_INVALID_ARG, "reads_per_s is NULL");
    if (array_bytes < 8 || reads < 1) return fail(MCF_ERR_INVALID_ARG, "array_bytes >= 8 and reads >= 1 required");
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t S = (uint64_t)array_bytes / 8;
    if (S > 0xffffffffull) return fail(MCF_ERR_INVALID_ARG, "array_bytes must be below 32 GiB");
    const int threads = 256;
    const int grid = 8 * num_sms();   // 2048 threads per SM
    const int64_t per_thread = (reads + (int64_t)grid * threads - 1) / ((int64_t)grid * threads);
    const int iters = (int)std::max<int64_t>(PROBE_UNROLL, (per_thread + PROBE_UNROLL - 1) / PROBE_UNROLL * PROBE_UNROLL);
    uint2* a = nullptr;
    uint32_t* sink = nullptr;
    if (cudaMallocAsync((void**)&a, S * 8, st) != cudaSuccess || cudaMallocAsync((void**)&sink, 4, st) != cudaSuccess) {
        cudaGetLastError();
        if (a) cudaFreeAsync(a, st);
        return fail(MCF_ERR_OOM, "device allocation of the probe array failed");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    EventGuard guard{&e0, &e1};
    mcf_status rc = MCF_OK;
    float ms = 0.f;
    {
        ScopedL2Fetch fetch(L2_FETCH_BYTES);   // as the walk kernels run
        cudaMemsetAsync(a, 0x5a, S * 8, st);
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        gather_probe_kernel<<<grid, threads, 0, st>>>(a, S, iters, sink);   // warm-up
        cudaEventRecord(e0, st);
        gather_probe_kernel<<<grid, threads, 0, st>>>(a, S, iters, sink);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess)
            rc = fail(MCF_ERR_CUDA, "gather probe failed");
        else
            cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaFreeAsync(a, st);
    cudaFreeAsync(sink, st);
    if (rc != MCF_OK) return rc;
    MCF_CUDA_TRY(cudaStreamSynchronize(st));
    *reads_per_s = (double)grid * threads * iters / (ms * 1e-3);
    return MCF_OK;
}

mcf_status mcf_inject_allocation_failure(int64_t after) {
    set_error("");
    g_fail_after.store(after < 0 ? -1 : (long long)after);
    return MCF_OK;
}

mcf_status mcf_kernel_launches(uint64_t* count) {
    set_error("");
    if (!count) return fail(MCF_ERR_INVALID_ARG, "count is NULL");
    *count = kernel_runs_walk() + kernel_runs_batch() + kernel_runs_graph() + kernel_runs_probe();
    return MCF_OK;
}

}  // extern "C"
