// Device building blocks shared by the walk kernels of libmcf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <type_traits>

#include "mcf_internal.cuh"

namespace mcf {

// ====================================================================== RNG
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products by 0xD2511F53 and 0xCD9E8D57; between rounds the
// key is advanced by the Weyl constants 0x9E3779B9 and 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Random words of transition k of a walk (ids glo/ghi): a uniform row uses
// word k % 4 of block k / 4; a weighted row uses words 2(k % 2), 2(k % 2) + 1
// of block k / 2 (bucket and alias test).  u caches the current block and is
// refilled when k enters a new block, so consecutive transitions of a walk
// share one Philox4x32-10 evaluation.
template <bool WEIGHTED>
__device__ __forceinline__ void walk_words(uint4& u, int k, uint32_t glo, uint32_t ghi, uint32_t req, uint2 key,
                                           uint32_t& w0, uint32_t& w1) {
    if constexpr (!WEIGHTED) {
        if ((k & 3) == 0) u = philox4x32_10(make_uint4((uint32_t)(k >> 2), glo, ghi, req), key);
        const int s = k & 3;
        w0 = s == 0 ? u.x : (s == 1 ? u.y : (s == 2 ? u.z : u.w));
        w1 = 0u;
    } else {
        if ((k & 1) == 0) u = philox4x32_10(make_uint4((uint32_t)(k >> 1), glo, ghi, req), key);
        w0 = (k & 1) ? u.z : u.x;
        w1 = (k & 1) ? u.w : u.y;
    }
}

// ====================================================================== node records
// What one walk step reads about the state l it leaves: CSR offset, degree,
// r_l (the contracted row <R_l, v>, Section 3.4) and the weight multiplier
// sum_j |a'_lj| (Eq. weights: a/t = sign(a) * row sum).  One 16-byte (float)
// or 32-byte (double) load per step.
template <bool F64>
struct Rec;
template <>
struct __align__(16) Rec<false> {
    uint32_t off;
    uint32_t deg;
    float r;
    float mult;
};
template <>
struct __align__(16) Rec<true> {
    int64_t off;
    uint32_t deg;
    uint32_t pad;
    double r;
    double mult;
};

constexpr int RED_BLOCKS = 256;
constexpr int RED_THREADS = 256;
constexpr int WARP_CHUNK = 32;      // walks per chunk (one per lane)
constexpr int CHUNKS_PER_GRAB = 4;  // chunks a warp takes per atomic

enum Counter { C_NEXT = 0, C_STEPS = 1, C_WALKS = 2, C_FLAGS = 3, C_TOTAL = 4, C_STARTS = 5, N_COUNTERS = 8 };

__device__ __forceinline__ double block_sum_d(double v) {
    __shared__ double part[32];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
    __syncthreads();
    return s;
}

// L2 eviction-priority policies: node records are re-read by every walk that
// passes through a node and should stay in L2; column-index reads are spread
// uniformly over all nnz entries and should not displace them.
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ Rec<false> load_rec(const Rec<false>* p, uint64_t pol) {
    uint4 v;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "l"(pol));
    Rec<false> x;
    x.off = v.x;
    x.deg = v.y;
    x.r = __uint_as_float(v.z);
    x.mult = __uint_as_float(v.w);
    return x;
}
__device__ __forceinline__ Rec<true> load_rec(const Rec<true>* p, uint64_t) { return *p; }
__device__ __forceinline__ int32_t load_col(const int32_t* p, uint64_t pol) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// Compensated float32 accumulator: the pair (hi, lo) carries about 48 bits;
// each addition is Knuth's TwoSum followed by a renormalisation, so a walk's
// sum of at most MCF_MAX_COEFFS float32 terms is exact to a few units of
// 2^-48 relative, and no float64 instruction runs per step.
struct F2Acc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float t) {
        const float s = __fadd_rn(hi, t);
        const float bp = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(t, bp));
        const float l = __fadd_rn(lo, e);
        hi = __fadd_rn(s, l);
        lo = __fsub_rn(l, __fsub_rn(hi, s));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ uint2 load_od(const uint2* p, uint64_t pol) {
    uint2 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
        : "=r"(v.x), "=r"(v.y)
        : "l"(p), "l"(pol));
    return v;
}

// Per-warp buffer of finished walks (start node, walk sum).  Lanes that
// finish a walk in the same loop iteration append in lane order; when 32 or
// more results are waiting the whole warp flushes them together: each lane
// converts one result to float64, the warp sorts the 32 (node, value) pairs by
// node (bitonic network over shuffles), sums runs of equal nodes with a
// segmented scan, and the first lane of each run adds the run to acc[node].
// The float64 work of walk completion thus runs with full warps, and walks of
// one start node -- thousands of them on a small graph -- share one atomic.
__device__ __forceinline__ double walk_value(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ double walk_value(double v) { return v; }

__device__ __forceinline__ void warp_merge_add(uint32_t nd, double v, bool valid, int lane, double* __restrict__ acc) {
    const unsigned FULL = 0xffffffffu;
    uint32_t key = valid ? nd : 0xffffffffu;
    // bitonic sort of (key, v) across the 32 lanes, ascending keys
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint32_t ok = __shfl_xor_sync(FULL, key, stride);
            const double ov = __shfl_xor_sync(FULL, v, stride);
            const bool up = ((lane & size) == 0);
            const bool lower = (lane & stride) == 0;
            const bool take_min = (lower == up);
            const bool swap = take_min ? (ok < key) : (ok > key);
            if (swap) {
                key = ok;
                v = ov;
            }
        }
    }
    // runs of equal keys are now contiguous; run ids from the run heads
    const uint32_t prev = __shfl_up_sync(FULL, key, 1);
    const bool head = lane == 0 || prev != key;
    const unsigned heads = __ballot_sync(FULL, head);
    const int run = __popc(heads & ((2u << lane) - 1u));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double o = __shfl_down_sync(FULL, v, d);
        const int orun = __shfl_down_sync(FULL, run, d);
        if (lane + d < 32 && orun == run) v += o;
    }
    if (head && key != 0xffffffffu) atomicAdd(&acc[key], v);
}

// warp_merge_add that also adds the squares of the walk values to acc2[node]
// (the per-start second moments behind the standard-error estimate).
static __device__ __noinline__ void warp_merge_add2(uint32_t nd, double v, bool valid, int lane, double* __restrict__ acc,
                                             double* __restrict__ acc2) {
    const unsigned FULL = 0xffffffffu;
    uint32_t key = valid ? nd : 0xffffffffu;
    double v2 = v * v;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint32_t ok = __shfl_xor_sync(FULL, key, stride);
            const double ov = __shfl_xor_sync(FULL, v, stride);
            const double ov2 = __shfl_xor_sync(FULL, v2, stride);
            const bool up = ((lane & size) == 0);
            const bool lower = (lane & stride) == 0;
            const bool take_min = (lower == up);
            const bool swap = take_min ? (ok < key) : (ok > key);
            if (swap) {
                key = ok;
                v = ov;
                v2 = ov2;
            }
        }
    }
    const uint32_t prev = __shfl_up_sync(FULL, key, 1);
    const bool head = lane == 0 || prev != key;
    const unsigned heads = __ballot_sync(FULL, head);
    const int run = __popc(heads & ((2u << lane) - 1u));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double o = __shfl_down_sync(FULL, v, d);
        const double o2 = __shfl_down_sync(FULL, v2, d);
        const int orun = __shfl_down_sync(FULL, run, d);
        if (lane + d < 32 && orun == run) {
            v += o;
            v2 += o2;
        }
    }
    if (head && key != 0xffffffffu) {
        atomicAdd(&acc[key], v);
        atomicAdd(&acc2[key], v2);
    }
}

template <class T>
struct WalkResults {
    uint32_t node[64];
    T val[64];
    // acc2 (may be null, warp-uniform): also accumulate the squared values
    __device__ __forceinline__ void flush(int n, int lane, double* __restrict__ acc, double* __restrict__ acc2) {
        __syncwarp();
        for (int r = 0; r < n; r += 32) {
            const int e = r + lane;
            const bool valid = e < n;
            const uint32_t nd = valid ? node[e] : 0u;
            const double x = valid ? walk_value(val[e]) : 0.0;
            if (acc2) warp_merge_add2(nd, x, valid, lane, acc, acc2);
            else warp_merge_add(nd, x, valid, lane, acc);
        }
        __syncwarp();
    }
    // Appends the results of the lanes with done set; returns the new count.
    __device__ __forceinline__ int push(bool done, uint32_t nd, T v, int n, int lane, unsigned lt_mask,
                                        double* __restrict__ acc, double* __restrict__ acc2) {
        const unsigned dm = __ballot_sync(0xffffffffu, done);
        if (!dm) return n;
        if (done) {
            const int pos = n + __popc(dm & lt_mask);
            node[pos] = nd;
            val[pos] = v;
        }
        n += __popc(dm);
        if (n >= 32) {
            flush(n, lane, acc, acc2);
            n = 0;
        }
        return n;
    }
};

// ---------------------------------------------------------------- state transition
// SelectNextState (Section 3.1) for the state whose record is x: position
// within the row from the Philox block u; returns the next state and the
// signed multiplier sign(a_{l l'}) * sum_j |a'_lj|.
template <bool F64, bool WEIGHTED>
__device__ __forceinline__ uint32_t next_state(const Rec<F64>& x, uint32_t w0, uint32_t w1,
                                               const int32_t* __restrict__ col, const WEntry* __restrict__ went,
                                               typename std::conditional<F64, double, float>::type& mult) {
    const uint32_t b = __umulhi(w0, x.deg);
    mult = x.mult;
    if constexpr (!WEIGHTED) {
        return (uint32_t)__ldg(col + (int64_t)x.off + b);
    } else {
        const float xr = __fmul_rn(__uint2float_rn(w1 >> 8), 5.9604644775390625e-08f);
        WEntry e = went[(int64_t)x.off + b];
        if (!(xr < e.prob)) e = went[(int64_t)x.off + e.alias];
        if (e.val < 0.0f) mult = -mult;
        return (uint32_t)e.col;
    }
}

// ---------------------------------------------------------------- RandFunmDiag row Q_k
struct DiagTable {
    double* val;       // global, per CTA: n (dense) or cap (hash) entries
    int32_t* key;      // shared (hash): node of each slot, -1 when free
    int32_t* used;     // shared (hash): slots in use, in insertion order
    int32_t cap_log2;
    int32_t limit;
    int* count;        // shared (hash): number of slots in use
};

__device__ __forceinline__ uint32_t hash_slot(uint32_t x, int cap_log2) {
    return (x * 0x9E3779B1u) >> (32 - cap_log2);
}

// Slot of node l (inserting it if absent); -1 when the table is full.
template <bool DENSE>
__device__ __forceinline__ int q_slot(const DiagTable& t, uint32_t l) {
    if constexpr (DENSE) {
        return (int)l;
    } else {
        const uint32_t mask = (1u << t.cap_log2) - 1u;
        uint32_t h = hash_slot(l, t.cap_log2);
        for (uint32_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
            const int32_t k = t.key[h];
            if (k == (int32_t)l) return (int)h;
            if (k == -1) {
                if (*(volatile int*)t.count >= t.limit) return -1;
                const int32_t prev = atomicCAS(&t.key[h], -1, (int32_t)l);
                if (prev == -1) {
                    const int pos = atomicAdd(t.count, 1);
                    t.used[pos] = (int32_t)h;
                    return (int)h;
                }
                if (prev == (int32_t)l) return (int)h;
            }
        }
        return -1;
    }
}

template <bool DENSE>
__device__ __forceinline__ double q_get(const DiagTable& t, uint32_t l) {
    // row values are updated by L2 reductions: read them from L2, not L1
    if constexpr (DENSE) {
        return __ldcg(t.val + l);
    } else {
        const uint32_t mask = (1u << t.cap_log2) - 1u;
        uint32_t h = hash_slot(l, t.cap_log2);
        for (uint32_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
            const int32_t k = t.key[h];
            if (k == (int32_t)l) return __ldcg(t.val + h);
            if (k == -1) return 0.0;
        }
        return 0.0;
    }
}

// Runs walk g from column k0, recording the visits of steps >= from (from >= 1:
// the step-0 visit is added in bulk) and counting the transitions of steps
// >= count_from.  Returns -1 when the walk is complete, else the step whose
// visit could not be stored.
template <bool F64, bool WEIGHTED, bool DENSE>
__device__ int diag_walk(const DiagTable& t, uint32_t k0, int64_t g, int from, int count_from,
                         const Rec<F64>* __restrict__ rec,
                         const int32_t* __restrict__ col, const WEntry* __restrict__ went,
                         const typename std::conditional<F64, double, float>::type* zeta, int K, double wc,
                         float wc32, uint2 key, uint32_t req, uint32_t& steps, uint32_t& flags) {
    using real = typename std::conditional<F64, double, float>::type;
    uint32_t l = k0;
    real W = (real)1;
    uint4 u = make_uint4(0u, 0u, 0u, 0u);
    const uint32_t glo = (uint32_t)g, ghi = (uint32_t)((uint64_t)g >> 32);
    for (int k = 0; k <= K; ++k) {
        if constexpr (F64) {
            if (!(fabs(W) > wc)) break;
        } else {
            if (!(fabsf(W) > wc32)) break;   // same decision as (double)|W| > W_c
        }
        uint32_t w0, w1;
        walk_words<WEIGHTED>(u, k, glo, ghi, req, key, w0, w1);
        const Rec<F64> x = rec[l];
        if (k >= from) {
            const int h = q_slot<DENSE>(t, l);
            if (h < 0) return k;
            double term;
            if constexpr (F64) term = __dmul_rn(zeta[k + 2], W);
            else term = (double)__fmul_rn(zeta[k + 2], W);
            atomicAdd(&t.val[h], term);
        }
        if (k + 2 >= K || x.deg == 0) break;
        real mult;
        const uint32_t nl = next_state<F64, WEIGHTED>(x, w0, w1, col, went, mult);
        if constexpr (F64) W = __dmul_rn(W, mult);
        else W = __fmul_rn(W, mult);
        l = nl;
        if (k >= count_from) ++steps;
    }
    if constexpr (!F64) if (!isfinite(W)) flags |= 1u;
    return -1;
}

// The requested rows of each column for a RandFunmDiag node subset S:
// column k lists the nodes i in S with a_ik != 0 (row[ptr[k] .. ptr[k+1]))
// and, for a weighted A, the entries a_ik (val).  Built from the rows of the
// requested nodes, so the dot phase of a column costs sum over its listed
// rows instead of a pass over the whole column.
struct SubList {
    const int64_t* ptr;   // n + 1, or null: no subset (every row of column k)
    const int32_t* row;
    const float* val;     // null for a binary A
};

// MCF_ERR_INVALID_ARG unless every nodes_dev[t] (device memory) lies in [0, n);
// waits for the stream.
mcf_status check_nodes_on_device(const int64_t* nodes_dev, int64_t m, int64_t n, cudaStream_t st);

// ---------------------------------------------------------------- RandFunmDiag rows keyed by row offset
// Row Q_k of a symmetric binary graph keyed by the row offset of the visited
// node (every visited node has degree >= 1, and such nodes have distinct row
// offsets): keys in a shared-memory open-addressing table (linear probing),
// float64 values in a per-CTA region of global memory updated by L2
// reductions.  A one-hash bit filter beside the keys (8 bits per slot) holds
// a bit for every key present: the dot phase looks up many absent keys, and
// most of those end at the filter instead of walking a probe chain, which at
// the table's fill limit averages several slots.
constexpr uint32_t OD_EMPTY = 0xffffffffu;

struct OdTable {
    uint32_t* key;     // shared: row offset of the node in each slot, OD_EMPTY when free
    uint32_t* filt;    // shared: 2^cap_log2 / 4 words of filter bits
    double* val;       // global, per CTA
    int cap_log2;
    int limit;         // largest number of keys admitted
    int* count;        // shared
};

// Shared memory of a table of 2^cap_log2 slots: keys, then filter words.
__host__ __device__ constexpr size_t od_smem_bytes(int cap_log2) {
    return ((size_t)1 << cap_log2) * sizeof(uint32_t) + ((size_t)1 << cap_log2);
}

__device__ __forceinline__ uint32_t od_fbit(const OdTable& t, uint32_t key) {
    return (key * 0x2C1B3C6Du) >> (32 - (t.cap_log2 + 3));
}

__device__ __forceinline__ void od_mark(const OdTable& t, uint32_t key) {
    const uint32_t f = od_fbit(t, key);
    atomicOr(&t.filt[f >> 5], 1u << (f & 31u));
}

// Sets every key slot free and every filter bit to 0 (the table's first use).
__device__ __forceinline__ void od_init(const OdTable& t) {
    const int cap = 1 << t.cap_log2;
    for (int h = threadIdx.x; h < cap; h += blockDim.x) {
        t.key[h] = OD_EMPTY;
        __stcg(t.val + h, 0.0);
    }
    for (int w = threadIdx.x; w < cap / 4; w += blockDim.x) t.filt[w] = 0u;
}

// Slot of key, inserted if absent and the table holds fewer than limit keys
// (-1 otherwise).  claimed is set when this call took a new slot: the caller
// adds the claims of its warp to *count in one atomic (count then lags by at
// most one claim per thread, which the table's margin above limit absorbs).
__device__ __forceinline__ int od_insert(const OdTable& t, uint32_t key, bool& claimed) {
    const uint32_t mask = (1u << t.cap_log2) - 1u;
    uint32_t h = (key * 0x9E3779B1u) >> (32 - t.cap_log2);
    claimed = false;
    for (uint32_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
        const uint32_t k = t.key[h];
        if (k == key) return (int)h;
        if (k == OD_EMPTY) {
            if (*(volatile int*)t.count >= t.limit) return -1;
            const uint32_t prev = atomicCAS(&t.key[h], OD_EMPTY, key);
            if (prev == OD_EMPTY) {
                claimed = true;
                od_mark(t, key);
                return (int)h;
            }
            if (prev == key) return (int)h;
        }
    }
    return -1;
}

// Adds the claims of the calling lanes (those executing together) to *count.
__device__ __forceinline__ void od_count_claims(const OdTable& t, bool claimed) {
    const unsigned am = __activemask();
    const unsigned b = __ballot_sync(am, claimed);
    if (b && (threadIdx.x & 31) == __ffs(b) - 1) atomicAdd(t.count, __popc(b));
}

// Inserts key regardless of the fill limit (the table keeps room for the
// limit plus one in-flight insertion per thread plus this one): the bulk
// step-0 visit of a start, made while the other threads may start inserting.
__device__ __forceinline__ int od_insert_always(const OdTable& t, uint32_t key) {
    const uint32_t mask = (1u << t.cap_log2) - 1u;
    uint32_t h = (key * 0x9E3779B1u) >> (32 - t.cap_log2);
    for (uint32_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
        const uint32_t k = t.key[h];
        if (k == key) return (int)h;
        if (k == OD_EMPTY) {
            const uint32_t prev = atomicCAS(&t.key[h], OD_EMPTY, key);
            if (prev == OD_EMPTY) {
                atomicAdd(t.count, 1);
                od_mark(t, key);
                return (int)h;
            }
            if (prev == key) return (int)h;
        }
    }
    return -1;
}

__device__ __forceinline__ double od_get(const OdTable& t, uint32_t key) {
    const uint32_t f = od_fbit(t, key);
    if (!((t.filt[f >> 5] >> (f & 31u)) & 1u)) return 0.0;
    const uint32_t mask = (1u << t.cap_log2) - 1u;
    uint32_t h = (key * 0x9E3779B1u) >> (32 - t.cap_log2);
    for (uint32_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
        const uint32_t k = t.key[h];
        if (k == key) return __ldcg(t.val + h);
        if (k == OD_EMPTY) return 0.0;
    }
    return 0.0;
}

// d_i += a'_ik <Q_k, C'_i> / N_k for the rows i of column k (= row k), or the
// rows the subset lists for column k; the entries of row i name their
// neighbours' keys in edge_key (4 bytes per entry).  Warp per row.
__device__ __forceinline__ void od_apply(const OdTable& t, uint32_t k0, int64_t Nk, const int64_t* __restrict__ rp,
                                         const int32_t* __restrict__ col, const uint32_t* __restrict__ ekey,
                                         const SubList& sub, double gamma, double* __restrict__ dacc) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int64_t* lp = sub.ptr ? sub.ptr : rp;
    const int32_t* lrow = sub.ptr ? sub.row : col;
    const double scale = (gamma * gamma) / (double)Nk;
    const int cap = 1 << t.cap_log2;
    const int64_t long_row = 8 * (int64_t)cap + 32 * (int64_t)*t.count;
    for (int64_t p = lp[k0] + wid; p < lp[k0 + 1]; p += nwarp) {
        const int32_t i = lrow[p];
        const int64_t rb = rp[i], re = rp[i + 1];
        double dot = 0.0;
        if (re - rb > long_row) {
            // a row much longer than the table (a hub): look each key of the
            // table up in the row instead.  ekey is strictly increasing within
            // a row (row offsets of distinct neighbours, all of degree >= 1),
            // so a binary search finds it; the terms are the same as below.
            for (int h = lane; h < cap; h += 32) {
                const uint32_t key = t.key[h];
                if (key == OD_EMPTY) continue;
                int64_t lo = rb, hi = re;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (__ldg(&ekey[mid]) < key) lo = mid + 1;
                    else hi = mid;
                }
                if (lo < re && __ldg(&ekey[lo]) == key) {
                    const double qv = __ldcg(t.val + h);
                    if (__double_as_longlong(qv) != 0) dot += qv;
                }
            }
        } else {
            for (int64_t q = rb + lane; q < re; q += 32) {
                const double qv = od_get(t, __ldg(&ekey[q]));
                if (__double_as_longlong(qv) != 0) dot += qv;   // exact zeros change no sum
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, d);
        if (lane == 0) atomicAdd(&dacc[i], dot * scale);
    }
}

__device__ __forceinline__ void od_clear(const OdTable& t) {
    const int cap = 1 << t.cap_log2;
    for (int h = threadIdx.x; h < cap; h += blockDim.x) {
        if (t.key[h] != OD_EMPTY) {
            t.key[h] = OD_EMPTY;
            __stcg(t.val + h, 0.0);
        }
    }
    for (int w = threadIdx.x; w < cap / 4; w += blockDim.x) t.filt[w] = 0u;
}


// Builds the SubList of the node subset nodes_dev[0..m) (device indices, in
// range) of graph g on stream st; device memory comes from alloc.  Waits for
// the stream once (the number of pairs sizes the lists).
mcf_status build_subset_lists(const mcf_graph* g, const int64_t* nodes_dev, int64_t m, cudaStream_t st,
                              const std::function<mcf_status(void**, size_t)>& alloc, SubList* out);

// <Q_k, C'_i> / gamma summed over column i of A (rp/col/val: the
// column-major copy; for a symmetric A the row arrays themselves), reduced
// over the warp (every lane returns the sum).
template <bool DENSE>
__device__ __forceinline__ double diag_dot(const DiagTable& t, int32_t i, const int64_t* __restrict__ rp,
                                           const int32_t* __restrict__ col, const float* __restrict__ val) {
    const int lane = threadIdx.x & 31;
    // Q_k is sparse: most lookups find nothing, and adding an exact zero
    // changes no sum, so only nonzero entries reach the (narrow) float64
    // pipe; the test is on the bit pattern, an integer operation
    double dot = 0.0;
    if (val) {
        for (int64_t q = rp[i] + lane; q < rp[i + 1]; q += 32) {
            const double qv = q_get<DENSE>(t, (uint32_t)col[q]);
            if (__double_as_longlong(qv) != 0) dot += (double)val[q] * qv;
        }
    } else {
        for (int64_t q = rp[i] + lane; q < rp[i + 1]; q += 32) {
            const double qv = q_get<DENSE>(t, (uint32_t)col[q]);
            if (__double_as_longlong(qv) != 0) dot += qv;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, d);
    return dot;
}

// d_i += a'_ik <Q_k, C'_i> / N_k for the rows i of column k (warp per row):
// every row of the column (sub.ptr null; read from the column-major copy)
// or only the rows the subset lists for column k.
template <bool DENSE>
__device__ __forceinline__ void diag_apply(const DiagTable& t, uint32_t k0, int64_t Nk, const int64_t* __restrict__ rp,
                                           const int32_t* __restrict__ col, const float* __restrict__ val,
                                           const SubList& sub, double gamma, double* __restrict__ dacc) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int64_t* lp = sub.ptr ? sub.ptr : rp;
    const int32_t* lrow = sub.ptr ? sub.row : col;
    const float* lval = sub.ptr ? sub.val : val;
    for (int64_t p = lp[k0] + wid; p < lp[k0 + 1]; p += nwarp) {
        const int32_t i = lrow[p];
        const double dot = diag_dot<DENSE>(t, i, rp, col, val);
        if (lane == 0) {
            const double aik = gamma * (lval ? (double)lval[p] : 1.0);
            atomicAdd(&dacc[i], (aik * (gamma * dot)) / (double)Nk);
        }
    }
}

template <bool DENSE>
__device__ __forceinline__ void diag_clear(const DiagTable& t, int64_t n) {
    if constexpr (DENSE) {
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) __stcg(t.val + i, 0.0);
    } else {
        const int c = *t.count;
        for (int e = threadIdx.x; e < c; e += blockDim.x) {
            const int h = t.used[e];
            t.key[h] = -1;
            __stcg(t.val + h, 0.0);
        }
    }
}

}  // namespace mcf
