// The sampling path of the method: per-solve preparation of the Markov chain
// (Definition 1), walk allocation, the walk kernels of RandFunmAction
// (Algorithm 3) and RandFunmDiag (Section 3.3), and their epilogues.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <functional>
#include <type_traits>

#include "mcf_device.cuh"
#include "mcf_internal.cuh"

namespace mcf {

// r = A' v evaluated as gamma * sum_j (a_ij v_j), the sum in CSR order with
// every product and sum rounded on its own (thread per row); v == nullptr
// means v = 1, where a binary row gives gamma * deg exactly.
__global__ void r_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                         const float* __restrict__ val, const double* __restrict__ v, double gamma,
                         double* __restrict__ r) {
    MCF_KERNEL_ENTRY();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = rp[i], e = rp[i + 1];
    double s;
    if (!val && !v) {
        s = (double)(e - b);
    } else {
        s = 0.0;
        for (int64_t p = b; p < e; ++p) {
            const double a = val ? (double)val[p] : 1.0;
            const double x = v ? v[col[p]] : 1.0;
            s = __dadd_rn(s, __dmul_rn(a, x));
        }
    }
    r[i] = __dmul_rn(gamma, s);
}

// colnorm_i = ||C'_i||_2 (Eq. initial_prob) from the column-major copy (cp:
// column pointers, col_sq: sum_j a_ji^2, null for a binary A) and
// fixed-partition partial sums of it.
__global__ void colnorm_kernel(int64_t n, const int64_t* __restrict__ cp, const double* __restrict__ col_sq,
                               double gamma, double* __restrict__ colnorm, double* __restrict__ part) {
    MCF_KERNEL_ENTRY();
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double sq = col_sq ? col_sq[i] : (double)(cp[i + 1] - cp[i]);
        const double c = __dmul_rn(gamma, sqrt(sq));
        colnorm[i] = c;
        s += c;
    }
    s = block_sum_d(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void sum_partials(const double* __restrict__ part, int nb, double* __restrict__ out) {
    MCF_KERNEL_ENTRY();
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[b];
    s = block_sum_d(s);
    if (threadIdx.x == 0) *out = s;
}

// N_i of Definition 1: 0 for an empty column, walks_per_node when given, else
// max(1, llround(N_s * (||C_i|| / sum_k ||C_k||))).  flag_i marks the start
// nodes this solve walks from.
__global__ void alloc_kernel(int64_t n, const double* __restrict__ colnorm, const double* __restrict__ tot,
                             int64_t n_walks, int64_t wpn, const uint8_t* __restrict__ need, int64_t* __restrict__ nw,
                             int64_t* __restrict__ flag) {
    MCF_KERNEL_ENTRY();
    const double T = *tot;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double c = colnorm[i];
        int64_t w = 0;
        if (c > 0.0) {
            if (wpn > 0) w = wpn;
            else {
                const long long q = llround(__dmul_rn((double)n_walks, __ddiv_rn(c, T)));
                w = q < 1 ? 1 : (int64_t)q;
            }
        }
        nw[i] = w;
        flag[i] = (w > 0 && (!need || need[i])) ? 1 : 0;
    }
}

// Compacts the start nodes: starts[s] = i, soff[s] = first walk id of i.
__global__ void compact_starts(int64_t n, const int64_t* __restrict__ flag, const int64_t* __restrict__ spos,
                               const int64_t* __restrict__ woff, int32_t* __restrict__ starts,
                               int64_t* __restrict__ soff, const unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (flag[i]) {
            starts[spos[i]] = (int32_t)i;
            soff[spos[i]] = woff[i];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) soff[counters[C_STARTS]] = (int64_t)counters[C_TOTAL];
}

// chunk_s0[c] = index s of the start whose walk range holds walk 32c.
__global__ void chunk_table(const int64_t* __restrict__ soff, const unsigned long long* __restrict__ counters,
                            uint32_t* __restrict__ chunk_s0) {
    MCF_KERNEL_ENTRY();
    const int64_t S = (int64_t)counters[C_STARTS];
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c0 = (soff[s] + WARP_CHUNK - 1) / WARP_CHUNK;
        const int64_t c1 = (soff[s + 1] + WARP_CHUNK - 1) / WARP_CHUNK;
        for (int64_t c = c0; c < c1; ++c) chunk_s0[c] = (uint32_t)s;
    }
}

template <bool F64>
__global__ void build_records(int64_t n, const int64_t* __restrict__ rp, const double* __restrict__ row_abs,
                              double gamma, const double* __restrict__ r, Rec<F64>* __restrict__ rec) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rp[i];
        const int64_t d = rp[i + 1] - b;
        const double mult = __dmul_rn(gamma, row_abs ? row_abs[i] : (double)d);
        Rec<F64> x;
        if constexpr (F64) {
            x.off = b;
            x.deg = (uint32_t)d;
            x.pad = 0;
            x.r = r ? r[i] : 0.0;
            x.mult = mult;
        } else {
            x.off = (uint32_t)b;
            x.deg = (uint32_t)d;
            x.r = r ? __double2float_rn(r[i]) : 0.0f;
            x.mult = __double2float_rn(mult);
        }
        rec[i] = x;
    }
}

// ====================================================================== RandFunmAction walks
// Persistent kernel with per-lane refill.  A warp takes CHUNKS_PER_GRAB
// chunks of 32 consecutive walk ids per atomic; whenever lanes are idle they
// are handed the next walk ids of the chunk in lane order, so no lane waits
// for the longest walk of its warp.  The start node of a chunk's walks comes
// from a 5-step shuffle binary search over the chunk's 32 start boundaries.
// One loop iteration advances every active lane by one visit of
// Algorithm 3's while loop.  A lane keeps a running sum while its
// consecutive walks share a start node and adds it to acc[start] with one
// float64 atomic when the start changes.
template <bool F64, bool WEIGHTED>
__global__ void __launch_bounds__(256, WALK_MINB) walk_action_kernel(
    const Rec<F64>* __restrict__ rec, const int32_t* __restrict__ col, const WEntry* __restrict__ went,
    const int32_t* __restrict__ starts, const int64_t* __restrict__ soff, const int64_t* __restrict__ goff,
    const uint32_t* __restrict__ chunk_s0,
    const double* __restrict__ zeta_g, int K, double wc, float wc32, uint2 key, uint32_t req, int grab,
    double* __restrict__ acc, double* __restrict__ acc2, double* __restrict__ wvals,
    unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    using real = typename std::conditional<F64, double, float>::type;
    using rtype = typename std::conditional<F64, double, float2>::type;
    __shared__ real zeta[MCF_MAX_COEFFS];
    __shared__ WalkResults<rtype> rbuf[256 / 32];
    for (int k = threadIdx.x; k <= K; k += blockDim.x) zeta[k] = (real)zeta_g[k];
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    WalkResults<rtype>& rb = rbuf[threadIdx.x >> 5];
    int rb_n = 0;
    const int32_t n_chunks = (int32_t)(((int64_t)counters[C_TOTAL] + WARP_CHUNK - 1) / WARP_CHUNK);

    // warp-uniform pool of walk ids (chunk indices fit 32 bits: the host
    // bounds the walk count below 2^36)
    int32_t c = -1, c_end = -1;
    int p = 0, valid = 0;
    int32_t cs = 0;          // start index of walk 32c + lane
    bool exhausted = false;
    // lane state
    bool active = false;
    int64_t g = 0, gw = 0;   // walk id, and its index in the walked space
    uint32_t l = 0, node0 = 0;
    int k = 0;
    real W = (real)1;
    uint4 u = make_uint4(0u, 0u, 0u, 0u);
    F2Acc a32;
    double a64 = 0.0;
    uint32_t my_steps = 0, my_walks = 0, flags = 0;

    for (;;) {
        unsigned idle = __ballot_sync(FULL, !active);
        while (idle && !exhausted) {
            if (p >= valid) {
                ++c;
                if (c >= c_end) {
                    int32_t base = 0;
                    if (lane == 0) base = (int32_t)atomicAdd((unsigned int*)&counters[C_NEXT], (unsigned)grab);
                    base = __shfl_sync(FULL, base, 0);
                    c = base;
                    c_end = min(base + grab, n_chunks);
                }
                if (c >= n_chunks) {
                    exhausted = true;
                    break;
                }
                const int64_t S = (int64_t)counters[C_STARTS];
                const int64_t s0 = chunk_s0[c];
                const int64_t bnd = (s0 + 1 + lane <= S) ? soff[s0 + 1 + lane] : INT64_MAX;
                const int64_t gl = (int64_t)c * WARP_CHUNK + lane;
                int cnt = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int64_t bv = __shfl_sync(FULL, bnd, cnt + step - 1);
                    if (bv <= gl) cnt += step;
                }
                cs = (int32_t)(s0 + cnt);
                valid = (int)min((int64_t)WARP_CHUNK, (int64_t)counters[C_TOTAL] - (int64_t)c * WARP_CHUNK);
                p = 0;
            }
            const int avail = valid - p;
            const int rank = __popc(idle & lt_mask);
            const int src = min(p + rank, WARP_CHUNK - 1);
            const int32_t s_new = __shfl_sync(FULL, cs, src);
            if (((idle >> lane) & 1u) && rank < avail) {
                g = (int64_t)c * WARP_CHUNK + p + rank;
                gw = g;
                if (goff != soff) g = goff[s_new] + (g - soff[s_new]);   // node subset: full-run walk id
                node0 = (uint32_t)starts[s_new];
                l = node0;
                k = 0;
                W = (real)1;
                a32 = F2Acc();
                a64 = 0.0;
                active = true;
            }
            p += min(avail, __popc(idle));
            idle = __ballot_sync(FULL, !active);
        }
        if (!__any_sync(FULL, active)) break;
        bool done = false;
        if (active) {
            if constexpr (F64) done = !(fabs(W) > wc);
            else done = !(fabsf(W) > wc32);  // same decision as (double)|W| > W_c
            if (!done) {
                uint32_t w0, w1;
                walk_words<WEIGHTED>(u, k, (uint32_t)g, (uint32_t)((uint64_t)g >> 32), req, key, w0, w1);
                const Rec<F64> x = load_rec(rec + l, policy_evict_last());
                if constexpr (F64) a64 += __dmul_rn(__dmul_rn(zeta[k + 2], W), x.r);
                else a32.add(__fmul_rn(__fmul_rn(zeta[k + 2], W), x.r));
                if (k + 2 >= K || x.deg == 0) {
                    done = true;
                } else {
                    const uint32_t b = __umulhi(w0, x.deg);
                    real mult = x.mult;
                    uint32_t nl;
                    if constexpr (!WEIGHTED) {
                        nl = (uint32_t)load_col(col + (int64_t)x.off + b, policy_evict_first());
                    } else {
                        const float xr = __fmul_rn(__uint2float_rn(w1 >> 8), 5.9604644775390625e-08f);
                        WEntry e = went[(int64_t)x.off + b];
                        if (!(xr < e.prob)) e = went[(int64_t)x.off + e.alias];
                        if (e.val < 0.0f) mult = -mult;
                        nl = (uint32_t)e.col;
                    }
                    if constexpr (F64) W = __dmul_rn(W, mult);
                    else W = __fmul_rn(W, mult);
                    l = nl;
                    ++k;
                    ++my_steps;
                }
            }
            if (done) {
                if constexpr (!F64) if (!isfinite(W) || !isfinite(a32.hi)) flags |= 1u;
                ++my_walks;
                active = false;
                if (wvals) {   // deterministic mode: the walk's value goes to its slot
                    if constexpr (F64) wvals[gw] = a64;
                    else wvals[gw] = walk_value(make_float2(a32.hi, a32.lo));
                }
            }
        }
        if constexpr (F64) rb_n = rb.push(done && !wvals, node0, a64, rb_n, lane, lt_mask, acc, acc2);
        else rb_n = rb.push(done && !wvals, node0, make_float2(a32.hi, a32.lo), rb_n, lane, lt_mask, acc, acc2);
    }
    rb.flush(rb_n, lane, acc, acc2);
    unsigned long long ws = my_steps, ww = my_walks;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        ws += __shfl_down_sync(FULL, ws, d);
        ww += __shfl_down_sync(FULL, ww, d);
        flags |= __shfl_down_sync(FULL, flags, d);
    }
    if (lane == 0) {
        atomicAdd(&counters[C_STEPS], ws);
        atomicAdd(&counters[C_WALKS], ww);
        if (flags) atomicOr(&counters[C_FLAGS], (unsigned long long)flags);
    }
}

// ---------------------------------------------------------------- binary v = 1 path
// For total communicability and Katz on a binary matrix, r_l and the weight
// multiplier of a state are both gamma * deg_l, so a step needs only the
// {row offset, degree} of the state it moves to.  These come from edge_od
// (one random 8-byte read per step); rm[d] = float(gamma * d) is a per-solve
// table indexed by degree (small, cache-resident).
__global__ void build_node_od(int64_t n, const int64_t* __restrict__ rp, uint2* __restrict__ nod) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        nod[i] = make_uint2((uint32_t)rp[i], (uint32_t)(rp[i + 1] - rp[i]));
}

__global__ void build_edge_od(int64_t nnz, const int32_t* __restrict__ col, const uint2* __restrict__ nod,
                              uint2* __restrict__ eod) {
    MCF_KERNEL_ENTRY();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        eod[p] = nod[col[p]];
}

__global__ void degree_table(int64_t max_deg, double gamma, float* __restrict__ rm) {
    MCF_KERNEL_ENTRY();
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d <= max_deg; d += (int64_t)gridDim.x * blockDim.x)
        rm[d] = __double2float_rn(__dmul_rn(gamma, (double)d));
}

// The same walks (ids, Philox streams), float32 arithmetic and accumulation
// as walk_action_kernel<false, false> (so the same result up to float64
// summation order), with the per-step state reduced to {offset, degree} and
// a warp's idle lanes refilled refill_min or more at a time.  The next
// state's record is read only once the walk is known to go on (after the
// cutoff test): a read issued earlier would be wasted DRAM work at every
// walk's end, and the kernel is bound by the rate of random DRAM reads.
__global__ void __launch_bounds__(256, WALK_MINB) walk_tc_kernel(
    const uint2* __restrict__ nod, const uint2* __restrict__ eod, const float* __restrict__ rm,
    const int32_t* __restrict__ starts, const int64_t* __restrict__ soff, const int64_t* __restrict__ goff,
    const uint32_t* __restrict__ chunk_s0,
    const double* __restrict__ zeta_g, int K, float wc32, uint2 key, uint32_t req, int grab, int refill_min,
    double* __restrict__ acc, double* __restrict__ acc2, double* __restrict__ wvals,
    unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    __shared__ float zeta[MCF_MAX_COEFFS];
    __shared__ WalkResults<float2> rbuf[256 / 32];
    for (int k = threadIdx.x; k <= K; k += blockDim.x) zeta[k] = (float)zeta_g[k];
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    WalkResults<float2>& rb = rbuf[threadIdx.x >> 5];
    const int32_t n_chunks = (int32_t)(((int64_t)counters[C_TOTAL] + WARP_CHUNK - 1) / WARP_CHUNK);
    int32_t c = -1, c_end = -1;
    int p = 0, valid = 0, rb_n = 0;
    int32_t cs = 0;
    bool exhausted = false;
    bool active = false;
    int64_t g = 0, gw = 0;   // walk id, and its index in the walked space
    uint32_t node0 = 0, off = 0, deg = 0;
    int k = 0;
    float W = 1.f;
    uint4 u = make_uint4(0u, 0u, 0u, 0u);
    F2Acc a32;
    uint32_t my_steps = 0, my_walks = 0, flags = 0;
    for (;;) {
        unsigned idle = __ballot_sync(FULL, !active);
        // refill once at least refill_min lanes are idle (or all are): fewer
        // refill passes against a few idle lanes for a step or two
        if (idle != FULL && __popc(idle) < refill_min) idle = 0u;
        while (idle && !exhausted) {
            if (p >= valid) {
                ++c;
                if (c >= c_end) {
                    int32_t base = 0;
                    if (lane == 0) base = (int32_t)atomicAdd((unsigned int*)&counters[C_NEXT], (unsigned)grab);
                    base = __shfl_sync(FULL, base, 0);
                    c = base;
                    c_end = min(base + grab, n_chunks);
                }
                if (c >= n_chunks) {
                    exhausted = true;
                    break;
                }
                const int64_t S = (int64_t)counters[C_STARTS];
                const int64_t s0 = chunk_s0[c];
                const int64_t bnd = (s0 + 1 + lane <= S) ? soff[s0 + 1 + lane] : INT64_MAX;
                const int64_t gl = (int64_t)c * WARP_CHUNK + lane;
                int cnt = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int64_t bv = __shfl_sync(FULL, bnd, cnt + step - 1);
                    if (bv <= gl) cnt += step;
                }
                cs = (int32_t)(s0 + cnt);
                valid = (int)min((int64_t)WARP_CHUNK, (int64_t)counters[C_TOTAL] - (int64_t)c * WARP_CHUNK);
                p = 0;
            }
            const int avail = valid - p;
            const int rank = __popc(idle & lt_mask);
            const int src = min(p + rank, WARP_CHUNK - 1);
            const int32_t s_new = __shfl_sync(FULL, cs, src);
            if (((idle >> lane) & 1u) && rank < avail) {
                g = (int64_t)c * WARP_CHUNK + p + rank;
                gw = g;
                if (goff != soff) g = goff[s_new] + (g - soff[s_new]);   // node subset: full-run walk id
                node0 = (uint32_t)starts[s_new];
                const uint2 od = nod[node0];
                off = od.x;
                deg = od.y;
                k = 0;
                W = 1.f;
                a32 = F2Acc();
                active = true;
            }
            p += min(avail, __popc(idle));
            idle = __ballot_sync(FULL, !active);
        }
        if (!__any_sync(FULL, active)) break;
        bool done = false;
        if (active) {
            const bool last = k + 2 >= K || deg == 0;
            done = !(fabsf(W) > wc32);
            if (!done) {
                const float t = __ldg(rm + deg);
                a32.add(__fmul_rn(__fmul_rn(zeta[k + 2], W), t));
                if (last) {
                    done = true;
                } else {
                    uint32_t w0, w1;
                    walk_words<false>(u, k, (uint32_t)g, (uint32_t)((uint64_t)g >> 32), req, key, w0, w1);
                    const uint2 nx = load_od(eod + (int64_t)off + __umulhi(w0, deg), policy_evict_first());
                    W = __fmul_rn(W, t);
                    off = nx.x;
                    deg = nx.y;
                    ++k;
                    ++my_steps;
                }
            }
            if (done) {
                if (!isfinite(W) || !isfinite(a32.hi)) flags |= 1u;
                ++my_walks;
                active = false;
                if (wvals) wvals[gw] = walk_value(make_float2(a32.hi, a32.lo));   // deterministic mode
            }
        }
        rb_n = rb.push(done && !wvals, node0, make_float2(a32.hi, a32.lo), rb_n, lane, lt_mask, acc, acc2);
    }
    rb.flush(rb_n, lane, acc, acc2);
    unsigned long long ws = my_steps, ww = my_walks;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        ws += __shfl_down_sync(FULL, ws, d);
        ww += __shfl_down_sync(FULL, ww, d);
        flags |= __shfl_down_sync(FULL, flags, d);
    }
    if (lane == 0) {
        atomicAdd(&counters[C_STEPS], ws);
        atomicAdd(&counters[C_WALKS], ww);
        if (flags) atomicOr(&counters[C_FLAGS], (unsigned long long)flags);
    }
}

// q_i = acc_i / N_i (Eq. rand_funm_action_formula, the 1/N_i factor of W^(0)).
__global__ void finalize_q(int64_t n, double* __restrict__ acc, const int64_t* __restrict__ nw) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[i] = nw[i] > 0 ? acc[i] / (double)nw[i] : 0.0;
}

// y = zeta_0 v + zeta_1 r + A' q (Algorithm 3, last step): a CTA takes
// EPI_ROWS consecutive rows at a time (tile_row_sums).  Launched with
// EPI_ROWS threads.
__global__ void __launch_bounds__(EPI_ROWS) action_epilogue(int64_t n, const int64_t* __restrict__ rp,
                                                            const int32_t* __restrict__ col,
                                                            const float* __restrict__ val, double gamma, double z0,
                                                            double z1, const double* __restrict__ v,
                                                            const double* __restrict__ r,
                                                            const double* __restrict__ q, double* __restrict__ y) {
    MCF_KERNEL_ENTRY();
    __shared__ double prod[EPI_CHUNK];
    __shared__ int64_t off[EPI_ROWS + 1];
    for (int64_t r0 = (int64_t)blockIdx.x * EPI_ROWS; r0 < n; r0 += (int64_t)gridDim.x * EPI_ROWS) {
        const int nr = (int)min((int64_t)EPI_ROWS, n - r0);
        const double s = tile_row_sums(r0, nr, rp, col, val, q, prod, off);
        if ((int)threadIdx.x < nr) {
            const int64_t row = r0 + threadIdx.x;
            y[row] = z0 * (v ? v[row] : 1.0) + z1 * r[row] + gamma * s;
        }
        __syncthreads();   // off[] is rewritten for the next rows
    }
}

// Node subsets: the walked space holds only the needed starts' walks;
// cof[s] is where start s's walks begin in it (soff[s] keeps the full-run id).
__global__ void subset_walks(int64_t n, const int64_t* __restrict__ flag, const int64_t* __restrict__ nw,
                             int64_t* __restrict__ wmask) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        wmask[i] = flag[i] ? nw[i] : 0;
}

__global__ void subset_offsets(int64_t n, const int64_t* __restrict__ flag, const int64_t* __restrict__ spos,
                               const int64_t* __restrict__ cw, int64_t* __restrict__ cof,
                               const unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) cof[spos[i]] = cw[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) cof[counters[C_STARTS]] = (int64_t)counters[C_TOTAL];
}

// y_t = zeta_0 v_i + zeta_1 r_i + (A' q)_i for i = nodes[t].
__global__ void action_epilogue_nodes(int64_t m, const int64_t* __restrict__ nodes, const int64_t* __restrict__ rp,
                                      const int32_t* __restrict__ col, const float* __restrict__ val, double gamma,
                                      double z0, double z1, const double* __restrict__ v, const double* __restrict__ r,
                                      const double* __restrict__ q, double* __restrict__ y) {
    MCF_KERNEL_ENTRY();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 32; base < m; base += nwarps * 32) {
        const double s = warp_listed_row_sums<32>(base, m, nodes, rp, col, val, q);
        const int64_t t = base + lane;
        if (t < m) {
            const int64_t i = nodes[t];
            y[t] = z0 * (v ? v[i] : 1.0) + z1 * r[i] + gamma * s;
        }
    }
}

// Standard error of RandFunmAction (the estimator's variance, Section 3.5):
// y_j = ... + sum_i a'_ji q_i with q_i the mean of N_i independent walk sums,
// so Var(y_j) = sum_i a'_ji^2 Var(X_i) / N_i.  w_i = s_i^2 / N_i from the
// sample variance of column i's walk sums (q_i after finalize_q, sum of
// squares acc2_i); 0 when N_i < 2.
__global__ void se_node_var(int64_t n, const double* __restrict__ q, const double* __restrict__ acc2,
                            const int64_t* __restrict__ nw, double* __restrict__ w) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t N = nw[i];
        double x = 0.0;
        if (N >= 2) {
            const double ss = acc2[i] - (double)N * q[i] * q[i];
            x = fmax(ss, 0.0) / ((double)(N - 1) * (double)N);
        }
        w[i] = x;
    }
}

// max over the rows j = rows[t] (or t) of sqrt(sum_p (gamma a_jp)^2 w_{col p}) / |y_t|
// (warp per row), as the bits of a non-negative double, which order like the values.
__global__ void se_rows(int64_t m, const int64_t* __restrict__ rows, const int64_t* __restrict__ rp,
                        const int32_t* __restrict__ col, const float* __restrict__ val, double gamma,
                        const double* __restrict__ w, const double* __restrict__ y,
                        unsigned long long* __restrict__ out) {
    MCF_KERNEL_ENTRY();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double best = 0.0;
    for (int64_t t = warp; t < m; t += nwarps) {
        const int64_t j = rows ? rows[t] : t;
        double s = 0.0;
        for (int64_t p = rp[j] + lane; p < rp[j + 1]; p += 32) {
            const double a = val ? (double)val[p] : 1.0;
            s += a * a * w[col[p]];
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        const double yt = fabs(y[t]);
        if (yt > 0.0) best = fmax(best, gamma * sqrt(s) / yt);
    }
    if (lane == 0 && best > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(best));
}

// ====================================================================== RandFunmDiag walks
// One CTA per start column k at a time (taken from an atomic counter).  Its
// threads run the N_k walks (thread t runs walks t, t + blockDim, ...) and
// add zeta_{m+2} W^(m) into row Q_k.  Q_k's float64 values live in a
// per-CTA region of global memory and are updated with float64 reductions,
// which the L2 executes (GB300's SM float64 pipe is narrow, and shared-memory
// float64 atomics loop on it).  Small graphs index the region densely by
// node; larger ones use an open-addressing hash whose keys, and the list of
// slots in use, live in shared memory.  Every walk visits k at step 0 with
// weight 1, so those N_k visits are added once as N_k * zeta_2.  After the
// walks, d_i += a'_ik <Q_k, C'_i> / N_k for every neighbour i of k (warp per
// neighbour).  A hash that reaches its fill limit stops the inserting walk;
// once every thread has stopped or finished, the CTA applies and clears the
// partial row and the stopped walks resume from their first unrecorded visit
// (walks are deterministic in their Philox counters and Q_k enters d
// linearly).
template <bool F64, bool WEIGHTED, bool DENSE>
__global__ void __launch_bounds__(256) walk_diag_kernel(
    const Rec<F64>* __restrict__ rec, const int64_t* __restrict__ cp, const int32_t* __restrict__ ri,
    const float* __restrict__ cv, const int32_t* __restrict__ col, const WEntry* __restrict__ went,
    const int32_t* __restrict__ starts,
    const int64_t* __restrict__ woff, const int64_t* __restrict__ nw, SubList sub, double gamma,
    const double* __restrict__ zeta_g, int K, double wc, float wc32, uint2 key, uint32_t req, int64_t n, int cap_log2,
    double* __restrict__ qval, double* __restrict__ dacc, unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    using real = typename std::conditional<F64, double, float>::type;
    extern __shared__ int32_t smem_i[];
    __shared__ real zeta[MCF_MAX_COEFFS];
    __shared__ int64_t cur;
    __shared__ int count;
    for (int k = threadIdx.x; k <= K; k += blockDim.x) zeta[k] = (real)zeta_g[k];
    DiagTable t;
    const int64_t cap = DENSE ? n : ((int64_t)1 << cap_log2);
    t.val = qval + (int64_t)blockIdx.x * cap;
    t.key = smem_i;
    t.used = smem_i + (DENSE ? 0 : cap);
    t.cap_log2 = cap_log2;
    t.limit = DENSE ? 0 : (int)(cap - cap / 4 - (int64_t)blockDim.x);
    t.count = &count;
    for (int64_t i = threadIdx.x; i < cap; i += blockDim.x) {
        __stcg(t.val + i, 0.0);
        if (!DENSE) t.key[i] = -1;
    }
    if (threadIdx.x == 0) count = 0;
    const int64_t S = (int64_t)counters[C_STARTS];
    uint32_t steps = 0, walks = 0, flags = 0;
    // the step-0 visit (weight 1 at k): taken when 1 > W_c, as in the walks
    bool visit0;
    if constexpr (F64) visit0 = 1.0 > wc;
    else visit0 = 1.0f > wc32;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) cur = (int64_t)atomicAdd(&counters[C_NEXT], 1ull);
        __syncthreads();
        const int64_t s = cur;
        if (s >= S) break;
        const uint32_t k0 = (uint32_t)starts[s];
        const int64_t Nk = nw[k0];
        const int64_t g0 = woff[k0];
        if (threadIdx.x == 0 && visit0 && K >= 2) {
            double z2;
            if constexpr (F64) z2 = zeta[2];
            else z2 = (double)zeta[2];
            const int h = q_slot<DENSE>(t, k0);     // empty table: always succeeds
            atomicAdd(&t.val[h], (double)Nk * z2);
        }
        __syncthreads();
        int64_t w = threadIdx.x;
        int from = 1, cfrom = 0;
        walks += (uint32_t)(Nk > (int64_t)threadIdx.x ? (Nk - 1 - threadIdx.x) / blockDim.x + 1 : 0);
        for (;;) {
            bool stopped = false;
            while (w < Nk) {
                const int f = diag_walk<F64, WEIGHTED, DENSE>(t, k0, g0 + w, from, cfrom, rec, col, went, zeta, K, wc,
                                                              wc32, key, req, steps, flags);
                if (f >= 0) {
                    from = f;
                    cfrom = f;
                    stopped = true;
                    break;
                }
                w += blockDim.x;
                from = 1;
                cfrom = 0;
            }
            if (!__syncthreads_or(stopped)) break;
            // the table filled up: apply the partial row, clear it, resume
            __threadfence_block();
            diag_apply<DENSE>(t, k0, Nk, cp, ri, cv, sub, gamma, dacc);
            __syncthreads();
            diag_clear<DENSE>(t, n);
            __syncthreads();
            if (threadIdx.x == 0) count = 0;
            __syncthreads();
        }
        __threadfence_block();
        diag_apply<DENSE>(t, k0, Nk, cp, ri, cv, sub, gamma, dacc);
        __syncthreads();
        diag_clear<DENSE>(t, n);
        __syncthreads();
        if (threadIdx.x == 0) count = 0;
    }
    const int lane = threadIdx.x & 31;
    unsigned long long ws = steps, ww = walks;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        ws += __shfl_down_sync(0xffffffffu, ws, d);
        ww += __shfl_down_sync(0xffffffffu, ww, d);
        flags |= __shfl_down_sync(0xffffffffu, flags, d);
    }
    if (lane == 0) {
        atomicAdd(&counters[C_STEPS], ws);
        atomicAdd(&counters[C_WALKS], ww);
        if (flags) atomicOr(&counters[C_FLAGS], (unsigned long long)flags);
    }
}

// ---------------------------------------------------------------- RandFunmDiag, symmetric binary graphs
// The RandFunmDiag kernel for a symmetric binary A in float32 weights on a
// graph too large for a dense row Q_k.  A step reads the 8-byte record
// {row offset, degree} of the state it moves to (edge_od, as the
// total-communicability walks), and row Q_k is keyed by the row offset of the
// visited node instead of its id: every visited node has degree >= 1 (walks
// move along entries), and nodes of degree >= 1 have distinct row offsets.
// The keys live in a shared-memory open-addressing table (no slot list: a
// flush clears by scanning the table), the float64 values in a per-CTA
// region of global memory updated by L2 reductions.  A start costs three CTA
// barriers: after its walks, after its dot phase and after the clear (during
// which the next start is fetched).
//
// One CTA serves one start column k at a time.  Its lanes take the N_k walks
// from a shared counter and each lane starts the next walk as soon as its
// previous one ends (no lane waits for the longest walk of its warp).  A
// lane whose new key does not fit (the table holds its fill limit) keeps its
// walk in registers and pauses; once every lane of the CTA has paused or run
// out of walks, the CTA adds the partial row into d (the dot phase of
// Eq. rand_funm_formula_diag, which is linear in Q_k), clears the table and
// the paused walks go on from where they stopped.  The N_k step-0 visits
// (weight 1 at k) are added once as N_k * zeta_2.
//
// MINB is the launch-bounds occupancy hint: 0 (none) for the 64- and
// 128-thread launches, 3 for the 256-thread launch of long starts.  With a
// hint ptxas schedules the walk loop with about 60 registers instead of 47
// (four CTAs per SM instead of five), which measured 1441 against 1625 ms per
// solve at 2000 walks per start on the configuration model n = 2e6, while the
// 128-thread launch of 100 walks per start runs faster without it (97 against
// 116 ms).  The hint must keep the kernel within 64 registers: at 67 (a hint
// of 2 once the hub-row path of the dot phase was added) only three CTAs fit
// on an SM and the same solve took 1854 ms.

template <int MINB>
__global__ void __launch_bounds__(256, MINB) walk_diag_od_kernel(
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const uint2* __restrict__ nod,
    const uint2* __restrict__ eod, const uint32_t* __restrict__ ekey, const float* __restrict__ rm,
    const int32_t* __restrict__ starts,
    const int64_t* __restrict__ woff, const int64_t* __restrict__ nw, SubList sub, double gamma,
    const double* __restrict__ zeta_g, int K, float wc32, uint2 key, uint32_t req, int cap_log2,
    double* __restrict__ qval, double* __restrict__ dacc, unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    extern __shared__ uint32_t od_keys[];
    __shared__ float zeta[MCF_MAX_COEFFS];
    __shared__ int64_t cur;
    __shared__ int count;
    __shared__ unsigned long long next_walk;
    for (int k = threadIdx.x; k <= K; k += blockDim.x) zeta[k] = (float)zeta_g[k];
    OdTable t;
    const int cap = 1 << cap_log2;
    t.key = od_keys;
    t.filt = od_keys + cap;
    t.val = qval + (int64_t)blockIdx.x * cap;
    t.cap_log2 = cap_log2;
    t.limit = cap - cap / 4 - (int)blockDim.x;
    t.count = &count;
    od_init(t);
    if (threadIdx.x == 0) count = 0;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t S = (int64_t)counters[C_STARTS];
    const bool visit0 = 1.0f > wc32;   // the step-0 visit (weight 1 at k), as in the walks
    uint32_t steps = 0, walks = 0, flags = 0;
    if (threadIdx.x == 0) {
        cur = (int64_t)atomicAdd(&counters[C_NEXT], 1ull);
        next_walk = 0ull;
    }
    __syncthreads();
    for (;;) {
        const int64_t s = cur;
        if (s >= S) break;
        const uint32_t k0 = (uint32_t)starts[s];
        const int64_t Nk = nw[k0];
        const int64_t g0 = woff[k0];
        const uint2 od0 = nod[k0];
        if (threadIdx.x == 0 && visit0 && K >= 2) {
            // the N_k step-0 visits, into the cleared table while the walks begin
            const int h = od_insert_always(t, od0.x);
            atomicAdd(&t.val[h], (double)Nk * (double)zeta[2]);
        }
        // lane state
        bool active = false, paused = false, exhausted = false;
        int64_t g = 0;
        uint32_t off = 0, deg = 0;
        int k = 0;
        float W = 1.f;
        uint4 u = make_uint4(0u, 0u, 0u, 0u);
        for (;;) {
            for (;;) {
                // hand the next walks of this start to the idle lanes
                const unsigned idle = __ballot_sync(FULL, !active);
                if (idle && !exhausted) {
                    unsigned long long base = 0;
                    if (lane == __ffs(idle) - 1) base = atomicAdd(&next_walk, (unsigned long long)__popc(idle));
                    base = __shfl_sync(FULL, base, __ffs(idle) - 1);
                    if (base + __popc(idle) >= (unsigned long long)Nk) exhausted = true;
                    if (!active) {
                        const int64_t w = (int64_t)base + __popc(idle & lt_mask);
                        if (w < Nk) {
                            g = g0 + w;
                            off = od0.x;
                            deg = od0.y;
                            k = 0;
                            W = 1.f;
                            active = true;
                        }
                    }
                }
                const bool run = active && !paused;
                if (!__any_sync(FULL, run)) break;
                if (run) {
                    bool done = !(fabsf(W) > wc32);
                    if (!done && k >= 1) {
                        bool claimed;
                        const int h = od_insert(t, off, claimed);
                        od_count_claims(t, claimed);
                        if (h < 0) paused = true;
                        else atomicAdd(&t.val[h], (double)__fmul_rn(zeta[k + 2], W));
                    }
                    if (!done && !paused) {
                        if (k + 2 >= K || deg == 0) {
                            done = true;
                        } else {
                            uint32_t w0, w1;
                            walk_words<false>(u, k, (uint32_t)g, (uint32_t)((uint64_t)g >> 32), req, key, w0, w1);
                            const uint2 nx = load_od(eod + (int64_t)off + __umulhi(w0, deg), policy_evict_first());
                            W = __fmul_rn(W, __ldg(rm + deg));
                            off = nx.x;
                            deg = nx.y;
                            ++k;
                            ++steps;
                        }
                    }
                    if (done) {
                        if (!isfinite(W)) flags |= 1u;
                        ++walks;
                        active = false;
                    }
                }
            }
            // every lane has paused or run out of walks
            const bool any_paused = __syncthreads_or(paused);
            __threadfence_block();
            od_apply(t, k0, Nk, rp, col, ekey, sub, gamma, dacc);
            __syncthreads();
            od_clear(t);
            if (threadIdx.x == 0) {
                count = 0;
                if (!any_paused) {   // the start is done: take the next one
                    cur = (int64_t)atomicAdd(&counters[C_NEXT], 1ull);
                    next_walk = 0ull;
                }
            }
            __syncthreads();
            if (!any_paused) break;
            paused = false;   // the table is empty again: the paused walks go on
        }
    }
    unsigned long long ws = steps, ww = walks;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        ws += __shfl_down_sync(FULL, ws, d);
        ww += __shfl_down_sync(FULL, ww, d);
        flags |= __shfl_down_sync(FULL, flags, d);
    }
    if (lane == 0) {
        atomicAdd(&counters[C_STEPS], ws);
        atomicAdd(&counters[C_WALKS], ww);
        if (flags) atomicOr(&counters[C_FLAGS], (unsigned long long)flags);
    }
}

// Per-column lists of the requested rows of a RandFunmDiag node subset
// (SubList): first[i] = the first position t with nodes[t] = i claims node i
// (a node listed twice is counted once); cnt[k] = |{i in S : a_ik != 0}|; after
// the scan of cnt into ptr, fill places each pair (k, i) of a claimed node.
__global__ void sub_claim(int64_t m, const int64_t* __restrict__ nodes, long long* __restrict__ first) {
    MCF_KERNEL_ENTRY();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
        atomicCAS((unsigned long long*)&first[nodes[t]], ~0ull, (unsigned long long)t);
}

// sub_count, sub_fill and mark_nodes give one CTA to each requested node and
// let its threads share the node's row: a sampled hub (10^5 entries and more
// on R-MAT graphs) would otherwise hold one thread for its whole row.
__global__ void sub_count(int64_t m, const int64_t* __restrict__ nodes, const long long* __restrict__ first,
                          const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t* __restrict__ cnt) {
    MCF_KERNEL_ENTRY();
    for (int64_t t = blockIdx.x; t < m; t += gridDim.x) {
        const int64_t i = nodes[t];
        if (first[i] != t) continue;
        for (int64_t p = rp[i] + threadIdx.x; p < rp[i + 1]; p += blockDim.x)
            atomicAdd((unsigned long long*)&cnt[col[p]], 1ull);
    }
}

__global__ void sub_fill(int64_t m, const int64_t* __restrict__ nodes, const long long* __restrict__ first,
                         const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const float* __restrict__ val,
                         const int64_t* __restrict__ ptr, int64_t* __restrict__ fill, int32_t* __restrict__ row,
                         float* __restrict__ sval) {
    MCF_KERNEL_ENTRY();
    for (int64_t t = blockIdx.x; t < m; t += gridDim.x) {
        const int64_t i = nodes[t];
        if (first[i] != t) continue;
        for (int64_t p = rp[i] + threadIdx.x; p < rp[i + 1]; p += blockDim.x) {
            const int32_t k = col[p];
            const int64_t pos = ptr[k] + (int64_t)atomicAdd((unsigned long long*)&fill[k], 1ull);
            row[pos] = (int32_t)i;
            if (val) sval[pos] = val[p];
        }
    }
}

// need[j] = 1 for every column j adjacent to a requested node.
__global__ void mark_nodes(int64_t m, const int64_t* __restrict__ nodes, const int64_t* __restrict__ rp,
                           const int32_t* __restrict__ col, uint8_t* __restrict__ need) {
    MCF_KERNEL_ENTRY();
    for (int64_t t = blockIdx.x; t < m; t += gridDim.x) {
        const int64_t i = nodes[t];
        for (int64_t p = rp[i] + threadIdx.x; p < rp[i + 1]; p += blockDim.x) need[col[p]] = 1;
    }
}

__global__ void check_nodes(int64_t m, const int64_t* __restrict__ nodes, int64_t n,
                            unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
        if (nodes[t] < 0 || nodes[t] >= n) atomicOr(&counters[C_FLAGS], 2ull);
}

// d_t = zeta_0 + zeta_1 a'_ii + (sum_k a'_ik <Q_k, C'_i>) for i = nodes[t] (or t).
__global__ void diag_finish(int64_t m, const int64_t* __restrict__ nodes, const double* __restrict__ dacc,
                            const double* __restrict__ diag, double gamma, double z0, double z1, int K,
                            double* __restrict__ d) {
    MCF_KERNEL_ENTRY();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = nodes ? nodes[t] : t;
        double v = z0;
        if (K >= 1) v += z1 * (gamma * diag[i]);
        d[t] = v + dacc[i];
    }
}

// ====================================================================== host side
constexpr int64_t MAX_WALKS_PER_SOLVE = (int64_t)1 << 36;

static mcf_status check_params(const mcf_graph* g, const mcf_params* p) {
    if (!g) return fail(MCF_ERR_INVALID_ARG, "graph is NULL");
    if (!p) return fail(MCF_ERR_INVALID_ARG, "params is NULL");
    if (!p->coeffs || p->n_coeffs < 1 || p->n_coeffs > MCF_MAX_COEFFS)
        return fail(MCF_ERR_INVALID_ARG, "coeffs must hold 1.." + std::to_string(MCF_MAX_COEFFS) + " values");
    if (p->n_walks < 0 || p->walks_per_node < 0) return fail(MCF_ERR_INVALID_ARG, "walk counts must be >= 0");
    if (p->n_coeffs > 2 && p->n_walks == 0 && p->walks_per_node == 0)
        return fail(MCF_ERR_INVALID_ARG, "n_walks or walks_per_node must be > 0");
    if (!(p->w_cutoff >= 0.0)) return fail(MCF_ERR_INVALID_ARG, "w_cutoff must be >= 0");
    if (p->precision != MCF_F64 && p->precision != MCF_F32W_F64ACC)
        return fail(MCF_ERR_INVALID_ARG, "unknown precision");
    if (p->deterministic != 0 && p->deterministic != 1) return fail(MCF_ERR_INVALID_ARG, "deterministic is 0 or 1");
    if (p->error_estimate != 0 && p->error_estimate != 1) return fail(MCF_ERR_INVALID_ARG, "error_estimate is 0 or 1");
    if (!(p->scale >= 0.0) || !isfinite(p->scale)) return fail(MCF_ERR_INVALID_ARG, "scale must be finite and >= 0");
    for (int k = 0; k < p->n_coeffs; ++k)
        if (!isfinite(p->coeffs[k])) return fail(MCF_ERR_INVALID_ARG, "coefficients must be finite");
    if (p->precision == MCF_F32W_F64ACC && g->nnz >= ((int64_t)1 << 32))
        return fail(MCF_ERR_UNSUPPORTED, "float32 walk records need nnz < 2^32");
    // walk ids (and the chunk tables indexed by them) stay below 2^36:
    // compared without forming N_s + n or walks_per_node * n, which could overflow
    const int64_t n = g->n;
    const bool too_many = p->walks_per_node > 0 ? (n > 0 && p->walks_per_node > MAX_WALKS_PER_SOLVE / n)
                                                : p->n_walks > MAX_WALKS_PER_SOLVE - n;
    if (too_many) return fail(MCF_ERR_INVALID_ARG, "more than 2^36 walks per solve");
    return MCF_OK;
}

// Everything a solve prepares before its walks: r, the chain's allocation,
// the compacted start list and the per-node records.
struct Prep {
    double* r = nullptr;
    double* colnorm = nullptr;
    double* part = nullptr;
    int64_t* nw = nullptr;
    int64_t* flag = nullptr;
    int64_t* woff = nullptr;
    int64_t* spos = nullptr;
    int32_t* starts = nullptr;
    int64_t* soff = nullptr;   // first full-run walk id of each start (+ the total)
    int64_t* cof = nullptr;    // first walk of each start in the walked space (== soff unless a node subset)
    unsigned long long* counters = nullptr;
    void* rec = nullptr;
    double* zeta = nullptr;
    void* scan_tmp = nullptr;
    size_t scan_bytes = 0;
};

static mcf_status prepare(const mcf_graph* g, const mcf_params* p, double gamma, const double* v_dev,
                          const uint8_t* need, Scratch& sc, Prep& P, cudaStream_t st) {
    const int64_t n = g->n;
    const bool f64 = p->precision == MCF_F64;
    MCF_TRY(sc.get(&P.r, n));
    MCF_TRY(sc.get(&P.colnorm, n));
    MCF_TRY(sc.get(&P.part, RED_BLOCKS + 1));
    MCF_TRY(sc.get(&P.nw, n));
    MCF_TRY(sc.get(&P.flag, n));
    MCF_TRY(sc.get(&P.woff, n));
    MCF_TRY(sc.get(&P.spos, n));
    MCF_TRY(sc.get(&P.starts, n));
    MCF_TRY(sc.get(&P.soff, n + 1));
    P.cof = P.soff;
    MCF_TRY(sc.get(&P.counters, N_COUNTERS));
    MCF_TRY(sc.get(&P.zeta, MCF_MAX_COEFFS));
    P.scan_bytes = scan_tmp_bytes(n);
    MCF_TRY(sc.get((char**)&P.scan_tmp, P.scan_bytes));
    if (f64) MCF_TRY(sc.get((Rec<true>**)&P.rec, n));
    else MCF_TRY(sc.get((Rec<false>**)&P.rec, n));
    MCF_CUDA_TRY(cudaMemsetAsync(P.counters, 0, N_COUNTERS * sizeof(unsigned long long), st));
    MCF_CUDA_TRY(cudaMemcpyAsync(P.zeta, p->coeffs, p->n_coeffs * sizeof(double), cudaMemcpyHostToDevice, st));
    if (n == 0) return MCF_OK;
    r_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, g->row_ptr, g->col_idx, g->values, v_dev, gamma, P.r);
    colnorm_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, g->col_ptr, g->col_sq, gamma, P.colnorm, P.part);
    sum_partials<<<1, RED_THREADS, 0, st>>>(P.part, RED_BLOCKS, P.part + RED_BLOCKS);
    alloc_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, P.colnorm, P.part + RED_BLOCKS, p->n_walks, p->walks_per_node,
                                                   need, P.nw, P.flag);
    MCF_TRY(scan_i64(P.nw, P.woff, n, (int64_t*)&P.counters[C_TOTAL], P.scan_tmp, P.scan_bytes, st));
    MCF_TRY(scan_i64(P.flag, P.spos, n, (int64_t*)&P.counters[C_STARTS], P.scan_tmp, P.scan_bytes, st));
    compact_starts<<<grid_for(n, 256), 256, 0, st>>>(n, P.flag, P.spos, P.woff, P.starts, P.soff, P.counters);
    if (f64)
        build_records<true><<<grid_for(n, 256), 256, 0, st>>>(n, g->row_ptr, g->row_abs, gamma, P.r, (Rec<true>*)P.rec);
    else
        build_records<false><<<grid_for(n, 256), 256, 0, st>>>(n, g->row_ptr, g->row_abs, gamma, P.r,
                                                               (Rec<false>*)P.rec);
    MCF_CUDA_TRY(cudaGetLastError());
    return MCF_OK;
}

// Keeps freed stream-ordered scratch in the device's default pool instead of
// returning it to the driver at every synchronisation.
void keep_pool_memory() {
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[dev] = true;
}

static mcf_status finish_stats(mcf_stats* stats, const unsigned long long* counters, cudaEvent_t e0, cudaEvent_t e1,
                               cudaStream_t st) {
    if (!stats) return MCF_OK;
    unsigned long long h[N_COUNTERS];
    MCF_CUDA_TRY(cudaMemcpyAsync(h, counters, sizeof(h), cudaMemcpyDeviceToHost, st));
    MCF_CUDA_TRY(cudaStreamSynchronize(st));
    stats->walks = (int64_t)h[C_WALKS];
    stats->walk_steps = (int64_t)h[C_STEPS];
    stats->flags = (uint32_t)h[C_FLAGS];
    stats->max_rel_se = 0.0;
    stats->est_rel_err = 0.0;
    stats->replicas = 1;
    float ms = 0.f;
    if (e0 && e1) cudaEventElapsedTime(&ms, e0, e1);
    stats->kernel_ms = ms;
    return MCF_OK;
}

template <bool F64, bool WEIGHTED>
static void launch_action_walks(const mcf_graph* g, const Prep& P, uint32_t* chunk_s0, int K, double wc, uint2 key,
                                uint32_t req, double* acc, double* acc2, cudaStream_t st, double* wvals = nullptr) {
    auto kern = walk_action_kernel<F64, WEIGHTED>;
    const int grid = persistent_grid(kern, 256, 0);
    ScopedL2Fetch fetch(L2_FETCH_BYTES);
    kern<<<grid, 256, 0, st>>>((const Rec<F64>*)P.rec, g->col_idx, g->went, P.starts, P.cof, P.soff, chunk_s0, P.zeta,
                               K, wc, cutoff_f32(wc), key, req, WALK_GRAB, acc, acc2, wvals, P.counters);
}

// Builds the graph's node_od / edge_od arrays on first use (binary, nnz < 2^32).
// node_od (and the per-entry arrays below) are built once per graph;
// concurrent callers on other streams must not see the pointers before the
// arrays are complete, so each is published after a synchronisation.
static std::mutex g_records_mu;

static mcf_status ensure_node_od_locked(mcf_graph* g, cudaStream_t st) {
    if (g->node_od) return MCF_OK;
    uint2* nod = nullptr;
    if (graph_alloc(&nod, (size_t)std::max<int64_t>(g->n, 1) * sizeof(uint2), st) != cudaSuccess) {
        cudaGetLastError();
        return fail(MCF_ERR_OOM, "device allocation of the node records failed");
    }
    build_node_od<<<grid_for(g->n, 256), 256, 0, st>>>(g->n, g->row_ptr, nod);
    MCF_CUDA_TRY(cudaGetLastError());
    MCF_CUDA_TRY(cudaStreamSynchronize(st));
    g->node_od = nod;
    return MCF_OK;
}

mcf_status ensure_edge_od(mcf_graph* g, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_records_mu);
    if (g->edge_od) return MCF_OK;
    MCF_TRY(ensure_node_od_locked(g, st));
    uint2* eod = nullptr;
    if (graph_alloc(&eod, (size_t)std::max<int64_t>(g->nnz, 1) * sizeof(uint2), st) != cudaSuccess) {
        cudaGetLastError();
        return fail(MCF_ERR_OOM, "device allocation of the per-entry walk records failed");
    }
    build_edge_od<<<grid_for(g->nnz, 256), 256, 0, st>>>(g->nnz, g->col_idx, g->node_od, eod);
    MCF_CUDA_TRY(cudaGetLastError());
    MCF_CUDA_TRY(cudaStreamSynchronize(st));
    g->edge_od = eod;
    return MCF_OK;
}

__global__ void build_edge_key(int64_t nnz, const int32_t* __restrict__ col, const uint2* __restrict__ nod,
                               uint32_t* __restrict__ ekey) {
    MCF_KERNEL_ENTRY();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        ekey[p] = nod[col[p]].x;
}

mcf_status ensure_edge_key(mcf_graph* g, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_records_mu);
    if (g->edge_key) return MCF_OK;
    MCF_TRY(ensure_node_od_locked(g, st));
    uint32_t* ek = nullptr;
    if (graph_alloc(&ek, (size_t)std::max<int64_t>(g->nnz, 1) * sizeof(uint32_t), st) != cudaSuccess) {
        cudaGetLastError();
        return fail(MCF_ERR_OOM, "device allocation of the per-entry row keys failed");
    }
    build_edge_key<<<grid_for(g->nnz, 256), 256, 0, st>>>(g->nnz, g->col_idx, g->node_od, ek);
    MCF_CUDA_TRY(cudaGetLastError());
    MCF_CUDA_TRY(cudaStreamSynchronize(st));
    g->edge_key = ek;
    return MCF_OK;
}

static void launch_tc_walks(const mcf_graph* g, const Prep& P, const float* rm, uint32_t* chunk_s0, int K, double wc,
                            uint2 key, uint32_t req, double* acc, double* acc2, double* wvals, cudaStream_t st) {
    const int grid = persistent_grid(walk_tc_kernel, 256, 0);
    ScopedL2Fetch fetch(L2_FETCH_BYTES);
    walk_tc_kernel<<<grid, 256, 0, st>>>(g->node_od, g->edge_od, rm, P.starts, P.cof, P.soff, chunk_s0, P.zeta, K,
                                         cutoff_f32(wc), key, req, WALK_GRAB, WALK_REFILL_MIN, acc, acc2, wvals,
                                         P.counters);
}

// Deterministic mode: the sum (and sum of squares) of start s's walk values,
// read in walk order with a fixed assignment to lanes and a fixed shuffle
// tree (warp per start), so the same walks give bit-identical sums.
__global__ void det_walk_sums(const unsigned long long* __restrict__ counters, const int32_t* __restrict__ starts,
                              const int64_t* __restrict__ cof, const double* __restrict__ wvals,
                              double* __restrict__ acc, double* __restrict__ acc2) {
    MCF_KERNEL_ENTRY();
    const int lane = threadIdx.x & 31;
    const int64_t S = (int64_t)counters[C_STARTS];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp; s < S; s += nwarps) {
        double v = 0.0, v2 = 0.0;
        for (int64_t w = cof[s] + lane; w < cof[s + 1]; w += 32) {
            const double x = wvals[w];
            v += x;
            v2 += x * x;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, d);
            v2 += __shfl_xor_sync(0xffffffffu, v2, d);
        }
        if (lane == 0) {
            acc[starts[s]] = v;
            if (acc2) acc2[starts[s]] = v2;
        }
    }
}

static mcf_status solve_action(mcf_graph* g, const mcf_params* p, const double* v, double* y, mcf_stats* stats,
                               bool ones, const int64_t* nodes = nullptr, int64_t n_nodes = -1) {
    set_error("");
    MCF_TRY(check_params(g, p));
    if (!y) return fail(MCF_ERR_INVALID_ARG, "y is NULL");
    if (!ones && !v) return fail(MCF_ERR_INVALID_ARG, "v is NULL");
    if (nodes && n_nodes < 0) return fail(MCF_ERR_INVALID_ARG, "n_nodes must be >= 0");
    cudaStream_t st = (cudaStream_t)p->stream;
    const int64_t n = g->n;
    const double gamma = p->scale == 0.0 ? 1.0 : p->scale;
    const int K = p->n_coeffs - 1;
    const bool f64 = p->precision == MCF_F64;
    keep_pool_memory();
    Scratch sc(st);
    const double* v_dev = nullptr;
    if (!ones) {
        if (is_device_ptr(v)) v_dev = v;
        else {
            double* vd;
            MCF_TRY(sc.get(&vd, n));
            MCF_CUDA_TRY(cudaMemcpyAsync(vd, v, n * sizeof(double), cudaMemcpyHostToDevice, st));
            v_dev = vd;
        }
    }
    const int64_t m = nodes ? n_nodes : n;
    const bool y_on_dev = is_device_ptr(y);
    double* y_dev = y;
    if (!y_on_dev) MCF_TRY(sc.get(&y_dev, m));
    // a node subset walks only the columns adjacent to the requested nodes
    const int64_t* nodes_dev = nullptr;
    uint8_t* need = nullptr;
    if (nodes) {
        if (m == 0) return MCF_OK;
        if (is_device_ptr(nodes)) {
            unsigned long long* chk;
            MCF_TRY(sc.get(&chk, N_COUNTERS));
            MCF_CUDA_TRY(cudaMemsetAsync(chk, 0, N_COUNTERS * sizeof(unsigned long long), st));
            check_nodes<<<grid_for(m, 256), 256, 0, st>>>(m, nodes, n, chk);
            unsigned long long h = 0;
            MCF_CUDA_TRY(cudaMemcpyAsync(&h, &chk[C_FLAGS], sizeof(h), cudaMemcpyDeviceToHost, st));
            MCF_CUDA_TRY(cudaStreamSynchronize(st));
            if (h & 2ull) return fail(MCF_ERR_INVALID_ARG, "node index out of range");
            nodes_dev = nodes;
        } else {
            for (int64_t t = 0; t < m; ++t)
                if (nodes[t] < 0 || nodes[t] >= n) return fail(MCF_ERR_INVALID_ARG, "node index out of range");
            int64_t* nd;
            MCF_TRY(sc.get(&nd, m));
            MCF_CUDA_TRY(cudaMemcpyAsync(nd, nodes, m * sizeof(int64_t), cudaMemcpyHostToDevice, st));
            nodes_dev = nd;
        }
        MCF_TRY(sc.get(&need, n));
        MCF_CUDA_TRY(cudaMemsetAsync(need, 0, n, st));
        mark_nodes<<<grid_for(m * 256, 256), 256, 0, st>>>(m, nodes_dev, g->row_ptr, g->col_idx, need);
    }
    Prep P;
    MCF_TRY(prepare(g, p, gamma, v_dev, need, sc, P, st));
    P.cof = P.soff;
    if (nodes && n > 0) {
        int64_t *wmask, *cw, *cof;
        MCF_TRY(sc.get(&wmask, n));
        MCF_TRY(sc.get(&cw, n));
        MCF_TRY(sc.get(&cof, n + 1));
        subset_walks<<<grid_for(n, 256), 256, 0, st>>>(n, P.flag, P.nw, wmask);
        MCF_TRY(scan_i64(wmask, cw, n, (int64_t*)&P.counters[C_TOTAL], P.scan_tmp, P.scan_bytes, st));
        subset_offsets<<<grid_for(n, 256), 256, 0, st>>>(n, P.flag, P.spos, cw, cof, P.counters);
        P.cof = cof;
    }
    double* acc;
    MCF_TRY(sc.get(&acc, n));
    // per-start sums of squared walk values, for the standard error
    const bool want_se = stats && p->error_estimate;
    double* acc2 = nullptr;
    if (want_se && n > 0) {
        MCF_TRY(sc.get(&acc2, n));
        MCF_CUDA_TRY(cudaMemsetAsync(acc2, 0, n * sizeof(double), st));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    EventGuard event_guard{&e0, &e1};
    if (n > 0) {
        MCF_CUDA_TRY(cudaMemsetAsync(acc, 0, n * sizeof(double), st));
        if (K >= 2) {
            // walk ids are bounded by N_s + n (rounding) or walks_per_node * n,
            // below MAX_WALKS_PER_SOLVE (check_params)
            const int64_t max_walks = p->walks_per_node > 0 ? p->walks_per_node * n : p->n_walks + n;
            const int64_t max_chunks = max_walks / WARP_CHUNK + 2;
            uint32_t* chunk_s0;
            MCF_TRY(sc.get(&chunk_s0, max_chunks));
            chunk_table<<<grid_for(n, 256), 256, 0, st>>>(P.cof, P.counters, chunk_s0);
            if (stats) {
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                cudaEventRecord(e0, st);
            }
            const uint2 key = philox_key(p->seed);
            const bool tc_path = ones && !f64 && !g->weighted && g->nnz < ((int64_t)1 << 32);
            // deterministic mode: one float64 slot per walk, summed per start in walk order
            double* wvals = nullptr;
            if (p->deterministic) MCF_TRY(sc.get(&wvals, std::max<int64_t>(max_walks, 1)));
            if (tc_path) {
                MCF_TRY(ensure_edge_od(g, st));
                float* rm;
                MCF_TRY(sc.get(&rm, g->max_degree + 1));
                degree_table<<<grid_for(g->max_degree + 1, 256), 256, 0, st>>>(g->max_degree, gamma, rm);
                const uint32_t rq = p->request_id;
                const double wc = p->w_cutoff;
                launch_tc_walks(g, P, rm, chunk_s0, K, wc, key, rq, acc, acc2, wvals, st);
            } else if (f64 && g->weighted) {
                launch_action_walks<true, true>(g, P, chunk_s0, K, p->w_cutoff, key, p->request_id, acc, acc2, st, wvals);
            } else if (f64) {
                launch_action_walks<true, false>(g, P, chunk_s0, K, p->w_cutoff, key, p->request_id, acc, acc2, st,
                                                 wvals);
            } else if (g->weighted) {
                launch_action_walks<false, true>(g, P, chunk_s0, K, p->w_cutoff, key, p->request_id, acc, acc2, st,
                                                 wvals);
            } else {
                launch_action_walks<false, false>(g, P, chunk_s0, K, p->w_cutoff, key, p->request_id, acc, acc2, st,
                                                  wvals);
            }
            if (wvals)
                det_walk_sums<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(P.counters, P.starts, P.cof, wvals, acc,
                                                                               acc2);
            if (stats) cudaEventRecord(e1, st);
        }
        finalize_q<<<grid_for(n, 256), 256, 0, st>>>(n, acc, P.nw);
        const double z0 = p->coeffs[0], z1 = K >= 1 ? p->coeffs[1] : 0.0;
        if (nodes_dev)
            action_epilogue_nodes<<<grid_for(m, 256), 256, 0, st>>>(m, nodes_dev, g->row_ptr, g->col_idx, g->values,
                                                                    gamma, z0, z1, v_dev, P.r, acc, y_dev);
        else
            action_epilogue<<<grid_for(n, EPI_ROWS), EPI_ROWS, 0, st>>>(n, g->row_ptr, g->col_idx, g->values, gamma,
                                                                        z0, z1, v_dev, P.r, acc, y_dev);
        MCF_CUDA_TRY(cudaGetLastError());
    }
    unsigned long long* se_max = nullptr;
    if (want_se && n > 0) {
        double* w;
        MCF_TRY(sc.get(&w, n));
        MCF_TRY(sc.get(&se_max, 1));
        MCF_CUDA_TRY(cudaMemsetAsync(se_max, 0, sizeof(unsigned long long), st));
        se_node_var<<<grid_for(n, 256), 256, 0, st>>>(n, acc, acc2, P.nw, w);
        se_rows<<<grid_for(m * 32, 256), 256, 0, st>>>(m, nodes_dev, g->row_ptr, g->col_idx, g->values, gamma, w, y_dev,
                                                        se_max);
        MCF_CUDA_TRY(cudaGetLastError());
    }
    if (!y_on_dev && m > 0) MCF_CUDA_TRY(cudaMemcpyAsync(y, y_dev, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    unsigned long long se_bits = 0;
    if (se_max) MCF_CUDA_TRY(cudaMemcpyAsync(&se_bits, se_max, sizeof(se_bits), cudaMemcpyDeviceToHost, st));
    mcf_status rc = finish_stats(stats, P.counters, e0, e1, st);
    if (rc != MCF_OK) return rc;
    if (stats && se_max) {
        double v_se;
        memcpy(&v_se, &se_bits, sizeof(v_se));
        stats->max_rel_se = v_se;
    }
    if (!y_on_dev) MCF_CUDA_TRY(cudaStreamSynchronize(st));
    return MCF_OK;
}

constexpr int64_t DIAG_DENSE_MAX = 16384;   // dense row Q_k (global memory) up to this many nodes

// Launch shape of the diag kernel: threads per CTA follow the walks per start
// (64 .. 256) and the hash holds about four visits per walk of a start, at
// most 2^12 slots by default (keys and slot list: 32 KB of shared memory, so
// several CTAs share an SM and keep enough walks in flight); a start with
// more distinct visits flushes its partial row.
template <bool F64, bool WEIGHTED, bool DENSE>
static mcf_status launch_diag(const mcf_graph* g, const Prep& P, const SubList& sub, double gamma, int K, double wc,
                              uint2 key, uint32_t req, int64_t nk_hint, double* dacc, Scratch& sc, cudaStream_t st) {
    auto kern = walk_diag_kernel<F64, WEIGHTED, DENSE>;
    int threads = 256;
    if (nk_hint > 0 && nk_hint <= 64) threads = 64;
    else if (nk_hint > 0 && nk_hint <= 128) threads = 128;
    int cap_log2 = 0;
    size_t smem = 0;
    int64_t cap = g->n;
    if (!DENSE) {
        const int64_t want_slots = std::max<int64_t>(4 * std::max<int64_t>(nk_hint, 1) * 4, 4 * threads);
        cap_log2 = 10;
        while (cap_log2 < DIAG_CAP_LOG2 && ((int64_t)1 << cap_log2) < want_slots) ++cap_log2;
        cap = (int64_t)1 << cap_log2;
        smem = (size_t)cap * 2 * sizeof(int32_t);
    }
    MCF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 0)));
    const int grid = persistent_grid(kern, threads, smem);
    double* qval;
    MCF_TRY(sc.get(&qval, (size_t)grid * (size_t)std::max<int64_t>(cap, 1)));
    ScopedL2Fetch fetch(L2_FETCH_BYTES);
    kern<<<grid, threads, smem, st>>>((const Rec<F64>*)P.rec, g->col_ptr, g->row_idx, g->col_values, g->col_idx,
                                      g->went, P.starts, P.woff, P.nw, sub, gamma, P.zeta,
                                      K, wc, cutoff_f32(wc), key, req, g->n, cap_log2, qval, dacc, P.counters);
    MCF_CUDA_TRY(cudaGetLastError());
    return MCF_OK;
}

// Launch shape of walk_diag_od_kernel: threads per CTA follow the walks per
// start (64 .. 256); the key table holds about 16 visits per walk of a start,
// between 2^10 and 2^DIAG_OD_CAP_LOG2 slots (5 bytes each in shared memory:
// key and filter bits);
// a start with more distinct visits adds and clears its partial row on the way.
constexpr int DIAG_OD_CAP_LOG2 = 13;

static mcf_status launch_diag_od(mcf_graph* g, const Prep& P, const SubList& sub, double gamma, int K, double wc,
                                 uint2 key, uint32_t req, int64_t nk_hint, double* dacc, Scratch& sc, cudaStream_t st) {
    MCF_TRY(ensure_edge_od(g, st));
    MCF_TRY(ensure_edge_key(g, st));
    float* rm;
    MCF_TRY(sc.get(&rm, (size_t)g->max_degree + 1));
    degree_table<<<grid_for(g->max_degree + 1, 256), 256, 0, st>>>(g->max_degree, gamma, rm);
    int threads = 256;
    if (nk_hint > 0 && nk_hint <= 64) threads = 64;
    else if (nk_hint > 0 && nk_hint <= 128) threads = 128;
    const int64_t want_slots = std::max<int64_t>(16 * std::max<int64_t>(nk_hint, 1), 4 * threads);
    int cap_log2 = 10;
    while (cap_log2 < DIAG_OD_CAP_LOG2 && ((int64_t)1 << cap_log2) < want_slots) ++cap_log2;
    const size_t smem = od_smem_bytes(cap_log2);
    auto kern = threads == 256 ? walk_diag_od_kernel<3> : walk_diag_od_kernel<0>;   // <= 64 registers
    MCF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = persistent_grid(kern, threads, smem);
    double* qval;
    MCF_TRY(sc.get(&qval, (size_t)grid << cap_log2));
    ScopedL2Fetch fetch(L2_FETCH_BYTES);
    kern<<<grid, threads, smem, st>>>(g->row_ptr, g->col_idx, g->node_od, g->edge_od, g->edge_key, rm, P.starts, P.woff,
                                      P.nw, sub, gamma, P.zeta, K, cutoff_f32(wc), key, req, cap_log2, qval, dacc,
                                      P.counters);
    MCF_CUDA_TRY(cudaGetLastError());
    return MCF_OK;
}

mcf_status check_nodes_on_device(const int64_t* nodes_dev, int64_t m, int64_t n, cudaStream_t st) {
    if (m <= 0) return MCF_OK;
    unsigned long long* chk = nullptr;
    if (cudaMallocAsync((void**)&chk, N_COUNTERS * sizeof(unsigned long long), st) != cudaSuccess) {
        cudaGetLastError();
        return fail(MCF_ERR_OOM, "device allocation for the node check failed");
    }
    unsigned long long h = 0;
    cudaMemsetAsync(chk, 0, N_COUNTERS * sizeof(unsigned long long), st);
    check_nodes<<<grid_for(m, 256), 256, 0, st>>>(m, nodes_dev, n, chk);
    cudaMemcpyAsync(&h, &chk[C_FLAGS], sizeof(h), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(chk, st);
    MCF_CUDA_TRY(cudaStreamSynchronize(st));
    if (h & 2ull) return fail(MCF_ERR_INVALID_ARG, "node index out of range");
    return MCF_OK;
}

mcf_status build_subset_lists(const mcf_graph* g, const int64_t* nodes_dev, int64_t m, cudaStream_t st,
                              const std::function<mcf_status(void**, size_t)>& alloc, SubList* out) {
    const int64_t n = g->n;
    long long* first;
    int64_t *cnt, *ptr;
    void *stmp, *rowv, *svalv = nullptr;
    const size_t sbytes = scan_tmp_bytes(n);
    MCF_TRY(alloc((void**)&first, std::max<int64_t>(n, 1) * sizeof(long long)));
    MCF_TRY(alloc((void**)&cnt, std::max<int64_t>(n, 1) * sizeof(int64_t)));
    MCF_TRY(alloc((void**)&ptr, (n + 1) * sizeof(int64_t)));
    MCF_TRY(alloc(&stmp, sbytes));
    MCF_CUDA_TRY(cudaMemsetAsync(first, 0xff, n * sizeof(long long), st));
    MCF_CUDA_TRY(cudaMemsetAsync(cnt, 0, n * sizeof(int64_t), st));
    sub_claim<<<grid_for(m, 256), 256, 0, st>>>(m, nodes_dev, first);
    sub_count<<<grid_for(m * 256, 256), 256, 0, st>>>(m, nodes_dev, first, g->row_ptr, g->col_idx, cnt);
    MCF_TRY(scan_i64(cnt, ptr, n, ptr + n, stmp, sbytes, st));
    int64_t pairs = 0;
    MCF_CUDA_TRY(cudaMemcpyAsync(&pairs, ptr + n, sizeof(pairs), cudaMemcpyDeviceToHost, st));
    MCF_CUDA_TRY(cudaStreamSynchronize(st));
    MCF_TRY(alloc(&rowv, std::max<int64_t>(pairs, 1) * sizeof(int32_t)));
    if (g->values) MCF_TRY(alloc(&svalv, std::max<int64_t>(pairs, 1) * sizeof(float)));
    MCF_CUDA_TRY(cudaMemsetAsync(cnt, 0, n * sizeof(int64_t), st));
    sub_fill<<<grid_for(m * 256, 256), 256, 0, st>>>(m, nodes_dev, first, g->row_ptr, g->col_idx, g->values, ptr,
                                                     cnt, (int32_t*)rowv, (float*)svalv);
    MCF_CUDA_TRY(cudaGetLastError());
    *out = SubList{ptr, (const int32_t*)rowv, (const float*)svalv};
    return MCF_OK;
}

static mcf_status solve_diag(mcf_graph* g, const mcf_params* p, const int64_t* nodes, int64_t n_nodes, double* d,
                             mcf_stats* stats) {
    set_error("");
    MCF_TRY(check_params(g, p));
    if (p->deterministic)
        return fail(MCF_ERR_UNSUPPORTED, "the deterministic mode covers RandFunmAction solves only");
    if (!d) return fail(MCF_ERR_INVALID_ARG, "d is NULL");
    if (nodes && n_nodes < 0) return fail(MCF_ERR_INVALID_ARG, "n_nodes must be >= 0");
    cudaStream_t st = (cudaStream_t)p->stream;
    const int64_t n = g->n;
    const int64_t m = nodes ? n_nodes : n;
    const double gamma = p->scale == 0.0 ? 1.0 : p->scale;
    const int K = p->n_coeffs - 1;
    const bool f64 = p->precision == MCF_F64;
    keep_pool_memory();
    Scratch sc(st);
    const int64_t* nodes_dev = nullptr;
    uint8_t* need = nullptr;
    if (nodes && m > 0) {
        if (is_device_ptr(nodes)) nodes_dev = nodes;
        else {
            for (int64_t t = 0; t < m; ++t)
                if (nodes[t] < 0 || nodes[t] >= n) return fail(MCF_ERR_INVALID_ARG, "node index out of range");
            int64_t* nd;
            MCF_TRY(sc.get(&nd, m));
            MCF_CUDA_TRY(cudaMemcpyAsync(nd, nodes, m * sizeof(int64_t), cudaMemcpyHostToDevice, st));
            nodes_dev = nd;
        }
        MCF_TRY(sc.get(&need, n));
        MCF_CUDA_TRY(cudaMemsetAsync(need, 0, n, st));
    }
    const bool d_on_dev = is_device_ptr(d);
    double* d_dev = d;
    if (!d_on_dev) MCF_TRY(sc.get(&d_dev, m));
    if (nodes && m == 0) return MCF_OK;
    if (nodes_dev && is_device_ptr(nodes)) {
        // device-resident indices are checked on the device before use
        unsigned long long* chk;
        MCF_TRY(sc.get(&chk, N_COUNTERS));
        MCF_CUDA_TRY(cudaMemsetAsync(chk, 0, N_COUNTERS * sizeof(unsigned long long), st));
        check_nodes<<<grid_for(m, 256), 256, 0, st>>>(m, nodes_dev, n, chk);
        unsigned long long h = 0;
        MCF_CUDA_TRY(cudaMemcpyAsync(&h, &chk[C_FLAGS], sizeof(h), cudaMemcpyDeviceToHost, st));
        MCF_CUDA_TRY(cudaStreamSynchronize(st));
        if (h & 2ull) return fail(MCF_ERR_INVALID_ARG, "node index out of range");
    }
    SubList sub{nullptr, nullptr, nullptr};
    if (nodes_dev) {
        mark_nodes<<<grid_for(m * 256, 256), 256, 0, st>>>(m, nodes_dev, g->row_ptr, g->col_idx, need);
        // per-column lists of the requested rows (Section 3.3: only the
        // columns k with a_ik != 0 for a requested i, and of each only those i)
        MCF_TRY(build_subset_lists(g, nodes_dev, m, st, [&](void** q, size_t bytes) {
                    return sc.get((char**)q, bytes);
                }, &sub));
    }
    Prep P;
    MCF_TRY(prepare(g, p, gamma, nullptr, need, sc, P, st));
    double* dacc;
    MCF_TRY(sc.get(&dacc, n));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    EventGuard event_guard{&e0, &e1};
    if (n > 0) {
        MCF_CUDA_TRY(cudaMemsetAsync(dacc, 0, n * sizeof(double), st));
        if (K >= 2) {
            if (stats) {
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                cudaEventRecord(e0, st);
            }
            const uint2 key = philox_key(p->seed);
            const bool dense = n <= DIAG_DENSE_MAX;
            mcf_status rc;
            const int64_t nk_hint = p->walks_per_node > 0 ? p->walks_per_node : std::max<int64_t>(1, p->n_walks / std::max<int64_t>(n, 1));
#define MCF_DIAG(F, W, D) rc = launch_diag<F, W, D>(g, P, sub, gamma, K, p->w_cutoff, key, p->request_id, nk_hint, dacc, sc, st)
            if (!f64 && !g->weighted && g->symmetric && !dense && g->nnz < ((int64_t)1 << 32)) {
                // a symmetric binary graph too large for a dense row: one
                // 8-byte record per step, rows keyed by row offset
                rc = launch_diag_od(g, P, sub, gamma, K, p->w_cutoff, key, p->request_id, nk_hint, dacc, sc, st);
            } else if (f64) {
                if (g->weighted) { if (dense) MCF_DIAG(true, true, true); else MCF_DIAG(true, true, false); }
                else { if (dense) MCF_DIAG(true, false, true); else MCF_DIAG(true, false, false); }
            } else {
                if (g->weighted) { if (dense) MCF_DIAG(false, true, true); else MCF_DIAG(false, true, false); }
                else { if (dense) MCF_DIAG(false, false, true); else MCF_DIAG(false, false, false); }
            }
#undef MCF_DIAG
            if (rc != MCF_OK) return rc;
            if (stats) cudaEventRecord(e1, st);
        }
        const double z0 = p->coeffs[0], z1 = K >= 1 ? p->coeffs[1] : 0.0;
        diag_finish<<<grid_for(m, 256), 256, 0, st>>>(m, nodes_dev, dacc, g->diag, gamma, z0, z1, K, d_dev);
        MCF_CUDA_TRY(cudaGetLastError());
    }
    if (!d_on_dev && m > 0) MCF_CUDA_TRY(cudaMemcpyAsync(d, d_dev, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    mcf_status rc = finish_stats(stats, P.counters, e0, e1, st);
    if (rc != MCF_OK) return rc;
    if (!d_on_dev) MCF_CUDA_TRY(cudaStreamSynchronize(st));
    return MCF_OK;
}

// ====================================================================== RandFunm (Algorithm 2), dense F
// Row k0 of N_k0 * Q (Eq. rand_funm_Q before its 1/N_k0 factor) for every
// start column k0.  One CTA per start at a time (atomic counter); its threads
// run the N_k0 walks and add zeta_{m+2} W^(m) into the dense row with float64
// reductions executed by the L2.  The N_k0 step-0 visits are added once.
template <bool F64, bool WEIGHTED>
__global__ void __launch_bounds__(128) walk_full_kernel(
    const Rec<F64>* __restrict__ rec, const int32_t* __restrict__ col, const WEntry* __restrict__ went,
    const int32_t* __restrict__ starts, const int64_t* __restrict__ woff, const int64_t* __restrict__ nw,
    const double* __restrict__ zeta_g, int K, double wc, float wc32, uint2 key, uint32_t req, int64_t n,
    double* __restrict__ Q, unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    using real = typename std::conditional<F64, double, float>::type;
    __shared__ real zeta[MCF_MAX_COEFFS];
    __shared__ int64_t cur;
    for (int k = threadIdx.x; k <= K; k += blockDim.x) zeta[k] = (real)zeta_g[k];
    DiagTable t;
    t.key = nullptr;
    t.used = nullptr;
    t.cap_log2 = 0;
    t.limit = 0;
    t.count = nullptr;
    const int64_t S = (int64_t)counters[C_STARTS];
    uint32_t steps = 0, walks = 0, flags = 0;
    bool visit0;
    if constexpr (F64) visit0 = 1.0 > wc;
    else visit0 = 1.0f > wc32;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) cur = (int64_t)atomicAdd(&counters[C_NEXT], 1ull);
        __syncthreads();
        const int64_t s = cur;
        __syncthreads();   // every thread has read cur before it is reused
        if (s >= S) break;
        const uint32_t k0 = (uint32_t)starts[s];
        const int64_t Nk = nw[k0];
        const int64_t g0 = woff[k0];
        t.val = Q + (int64_t)k0 * n;
        if (threadIdx.x == 0 && visit0) {
            double z2;
            if constexpr (F64) z2 = zeta[2];
            else z2 = (double)zeta[2];
            atomicAdd(&t.val[k0], (double)Nk * z2);
        }
        walks += (uint32_t)(Nk > (int64_t)threadIdx.x ? (Nk - 1 - threadIdx.x) / blockDim.x + 1 : 0);
        for (int64_t w = threadIdx.x; w < Nk; w += blockDim.x)
            diag_walk<F64, WEIGHTED, true>(t, k0, g0 + w, 1, 0, rec, col, went, zeta, K, wc, wc32, key, req, steps,
                                           flags);
    }
    const int lane = threadIdx.x & 31;
    unsigned long long ws = steps, ww = walks;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        ws += __shfl_down_sync(0xffffffffu, ws, d);
        ww += __shfl_down_sync(0xffffffffu, ww, d);
        flags |= __shfl_down_sync(0xffffffffu, flags, d);
    }
    if (lane == 0) {
        atomicAdd(&counters[C_STEPS], ws);
        atomicAdd(&counters[C_WALKS], ww);
        if (flags) atomicOr(&counters[C_FLAGS], (unsigned long long)flags);
    }
}

// ce[p] = gamma a_p / N_{col p}: the entries of A' diag(1/N) that scale the
// rows of N Q (Eq. rand_funm_Q); 0 where column col p has no walks (its row
// of Q is zero).
__global__ void full_edge_coeffs(int64_t nnz, const int32_t* __restrict__ col, const float* __restrict__ val,
                                 const int64_t* __restrict__ nw, double gamma, double* __restrict__ ce) {
    MCF_KERNEL_ENTRY();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t Nm = nw[col[p]];
        ce[p] = Nm == 0 ? 0.0 : (gamma * (val ? (double)val[p] : 1.0)) / (double)Nm;
    }
}

// F = zeta_0 I + zeta_1 A' + A' Q A' (Algorithm 2, last step) one row i at a
// time: row i of A'Q is formed in shared memory from the rows of N Q of i's
// neighbours (each scaled by ce), then F_ij = zeta_0 [i == j] +
// sum_m (A'Q)_im a'_mj over column j of A' (the column-major copy), and
// finally zeta_1 a'_ij is added for the entries of row i.  Both products cost one
// float64 FMA per (i, j, entry): the kernel is bound by the float64 pipe, so
// no float64 division is left in its loops.  Each thread accumulates four
// columns j at once so that four row loads are in flight.
constexpr int FULL_THREADS = 1024;

// sum_{p in row} a_p x[col p] for the 32 rows base + lane (warp_row_sums with
// the binary case specialised: one float64 add per entry instead of a
// multiply and an add).
template <bool WEIGHTED>
__device__ __forceinline__ double full_row_sums(int64_t base, int64_t n, const int64_t* __restrict__ rp,
                                                const int32_t* __restrict__ col, const float* __restrict__ val,
                                                const double* __restrict__ x) {
    if constexpr (WEIGHTED) {
        return warp_row_sums<32>(base, n, rp, col, val, x);
    } else {
        const int lane = threadIdx.x & 31;
        const int64_t row = base + lane;
        int64_t b = 0, e = 0;
        if (row < n) {
            b = rp[row];
            e = rp[row + 1];
        }
        double s = 0.0;
        const bool is_short = e - b <= 32;
        if (is_short)
            for (int64_t p = b; p < e; ++p) s += x[col[p]];
        unsigned longs = __ballot_sync(0xffffffffu, !is_short);
        while (longs) {
            const int t = __ffs(longs) - 1;
            longs &= longs - 1;
            const int64_t lb = __shfl_sync(0xffffffffu, b, t);
            const int64_t le = __shfl_sync(0xffffffffu, e, t);
            double part = 0.0;
            for (int64_t p = lb + lane; p < le; p += 32) part += x[col[p]];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
            if (lane == t) s = part;
        }
        return s;
    }
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(FULL_THREADS) full_epilogue(
    int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const float* __restrict__ val,
    const int64_t* __restrict__ cp, const int32_t* __restrict__ ri, const float* __restrict__ cv,
    const double* __restrict__ Q, const double* __restrict__ ce, double gamma, double z0, double z1, int K,
    double* __restrict__ F) {
    MCF_KERNEL_ENTRY();
    extern __shared__ double aq[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int64_t B = blockDim.x;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t b = rp[i], e = rp[i + 1];
        for (int64_t j0 = threadIdx.x; j0 < n; j0 += 4 * B) {
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            if (K >= 2) {
                const bool h1 = j0 + B < n, h2 = j0 + 2 * B < n, h3 = j0 + 3 * B < n;
                for (int64_t p = b; p < e; ++p) {
                    const double c = ce[p];
                    const double* row = Q + (int64_t)col[p] * n + j0;
                    a0 = fma(c, __ldg(row), a0);
                    if (h1) a1 = fma(c, __ldg(row + B), a1);
                    if (h2) a2 = fma(c, __ldg(row + 2 * B), a2);
                    if (h3) a3 = fma(c, __ldg(row + 3 * B), a3);
                }
            }
            aq[j0] = a0;
            if (j0 + B < n) aq[j0 + B] = a1;
            if (j0 + 2 * B < n) aq[j0 + 2 * B] = a2;
            if (j0 + 3 * B < n) aq[j0 + 3 * B] = a3;
        }
        __syncthreads();
        double* Fi = F + i * n;
        for (int64_t base = (int64_t)wid * 32; base < n; base += (int64_t)nwarp * 32) {
            const double s = full_row_sums<WEIGHTED>(base, n, cp, ri, cv, aq);   // column j of A
            const int64_t j = base + lane;
            if (j < n) Fi[j] = (j == i ? z0 : 0.0) + gamma * s;
        }
        __syncthreads();
        if (K >= 1)
            for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x)
                atomicAdd(&Fi[col[p]], z1 * (gamma * (val ? (double)val[p] : 1.0)));
        __syncthreads();
    }
}

constexpr int64_t FULL_MAX_NODES = MCF_FULL_MAX_NODES;

static mcf_status solve_full(mcf_graph* g, const mcf_params* p, double* F, mcf_stats* stats) {
    set_error("");
    MCF_TRY(check_params(g, p));
    if (p->deterministic)
        return fail(MCF_ERR_UNSUPPORTED, "the deterministic mode covers RandFunmAction solves only");
    if (!F) return fail(MCF_ERR_INVALID_ARG, "F is NULL");
    const int64_t n = g->n;
    if (n > FULL_MAX_NODES)
        return fail(MCF_ERR_UNSUPPORTED, "the dense estimate needs n <= " + std::to_string(FULL_MAX_NODES));
    cudaStream_t st = (cudaStream_t)p->stream;
    const double gamma = p->scale == 0.0 ? 1.0 : p->scale;
    const int K = p->n_coeffs - 1;
    const bool f64 = p->precision == MCF_F64;
    keep_pool_memory();
    Scratch sc(st);
    const bool f_on_dev = is_device_ptr(F);
    double* F_dev = F;
    if (!f_on_dev) MCF_TRY(sc.get(&F_dev, (size_t)std::max<int64_t>(n * n, 1)));
    Prep P;
    MCF_TRY(prepare(g, p, gamma, nullptr, nullptr, sc, P, st));
    double* Q;
    MCF_TRY(sc.get(&Q, (size_t)std::max<int64_t>(n * n, 1)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    EventGuard event_guard{&e0, &e1};
    if (n > 0) {
        if (K >= 2) {
            MCF_CUDA_TRY(cudaMemsetAsync(Q, 0, (size_t)(n * n) * sizeof(double), st));
            if (stats) {
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                cudaEventRecord(e0, st);
            }
            const uint2 key = philox_key(p->seed);
            const float wc32 = cutoff_f32(p->w_cutoff);
#define MCF_FULL(F64_, W_)                                                                                           \
    do {                                                                                                             \
        auto kern = walk_full_kernel<F64_, W_>;                                                                      \
        const int grid = persistent_grid(kern, 128, 0);                                                              \
        kern<<<grid, 128, 0, st>>>((const Rec<F64_>*)P.rec, g->col_idx, g->went, P.starts, P.woff, P.nw, P.zeta, K, \
                                   p->w_cutoff, wc32, key, p->request_id, n, Q, P.counters);                         \
    } while (0)
            if (f64) {
                if (g->weighted) MCF_FULL(true, true);
                else MCF_FULL(true, false);
            } else {
                if (g->weighted) MCF_FULL(false, true);
                else MCF_FULL(false, false);
            }
#undef MCF_FULL
            MCF_CUDA_TRY(cudaGetLastError());
            if (stats) cudaEventRecord(e1, st);
        }
        double* ce;
        MCF_TRY(sc.get(&ce, (size_t)std::max<int64_t>(g->nnz, 1)));
        if (K >= 2 && g->nnz > 0)
            full_edge_coeffs<<<grid_for(g->nnz, 256), 256, 0, st>>>(g->nnz, g->col_idx, g->values, P.nw, gamma, ce);
        // two CTAs per SM (one works while the other waits at a barrier)
        // when two rows of A'Q fit in shared memory, else one larger CTA
        const size_t smem = (size_t)n * sizeof(double);
        const int threads = 2 * smem <= 200 * 1024 ? FULL_THREADS / 2 : FULL_THREADS;
        const double z0 = p->coeffs[0], z1 = K >= 1 ? p->coeffs[1] : 0.0;
        auto kern = g->weighted ? full_epilogue<true> : full_epilogue<false>;
        MCF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int grid = (int)std::min<int64_t>(n, persistent_grid(kern, threads, smem));
        kern<<<grid, threads, smem, st>>>(n, g->row_ptr, g->col_idx, g->values, g->col_ptr, g->row_idx,
                                          g->col_values, Q, ce, gamma, z0, z1, K, F_dev);
        MCF_CUDA_TRY(cudaGetLastError());
    }
    if (!f_on_dev && n > 0)
        MCF_CUDA_TRY(cudaMemcpyAsync(F, F_dev, (size_t)(n * n) * sizeof(double), cudaMemcpyDeviceToHost, st));
    mcf_status rc = finish_stats(stats, P.counters, e0, e1, st);
    if (rc != MCF_OK) return rc;
    if (!f_on_dev) MCF_CUDA_TRY(cudaStreamSynchronize(st));
    return MCF_OK;
}

// ====================================================================== classical Monte Carlo (Algorithm 1)
// y_t = (1/N) sum over N walks from row i = nodes[t] of sum_k zeta_k W^(k)
// v_{l_k}: every step samples one entry of the current row with probability
// |a_lj| / sum_j |a_lj| and multiplies W by sign(a_lj) sum_j |a'_lj| (the same
// chain as the row-sampling walks, Definition 1).  Walk ids are i * N + s.
// Walks are laid out t-major; every warp takes 32 consecutive walks, sums each
// walk in float64 (one FMA per visit) and adds the walks of one output with
// one atomic.
template <bool WEIGHTED>
__global__ void __launch_bounds__(256) mc_classic_kernel(
    int64_t m, const int64_t* __restrict__ nodes, int64_t N, const Rec<true>* __restrict__ rec,
    const int32_t* __restrict__ col, const WEntry* __restrict__ went, const double* __restrict__ v,
    const double* __restrict__ zeta_g, int K, double wc, uint2 key, uint32_t req, double* __restrict__ acc,
    unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    __shared__ double zeta[MCF_MAX_COEFFS];
    for (int k = threadIdx.x; k <= K; k += blockDim.x) zeta[k] = zeta_g[k];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long wc_bits = __double_as_longlong(wc);   // wc >= 0
    const int64_t total = m * N;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t steps = 0, walks = 0;
    for (int64_t base = warp0 * 32; base < total; base += nwarps * 32) {
        const int64_t w = base + lane;
        const bool valid = w < total;
        double sum = 0.0;
        uint32_t t = 0;
        if (valid) {
            t = (uint32_t)(w / N);
            const int64_t s = w - (int64_t)t * N;
            const int64_t i = nodes ? nodes[t] : (int64_t)t;
            const uint64_t g = (uint64_t)i * (uint64_t)N + (uint64_t)s;
            const uint32_t glo = (uint32_t)g, ghi = (uint32_t)(g >> 32);
            uint32_t l = (uint32_t)i;
            double W = 1.0;
            uint4 u = make_uint4(0u, 0u, 0u, 0u);
            ++walks;
            for (int k = 0;; ++k) {
                // |W| > W_c on the bit patterns (ordered like the values for
                // non-negative doubles), keeping the float64 pipe for the sums
                const long long wb = __double_as_longlong(W) & 0x7fffffffffffffffLL;
                if (!(wb > wc_bits && wb <= 0x7ff0000000000000LL)) break;
                if (v) sum = fma(zeta[k] * W, v[l], sum);
                else sum = fma(zeta[k], W, sum);
                if (k >= K) break;
                const Rec<true> x = rec[l];
                if (x.deg == 0) break;
                uint32_t w0, w1;
                walk_words<WEIGHTED>(u, k, glo, ghi, req, key, w0, w1);
                double mult;
                const uint32_t nl = next_state<true, WEIGHTED>(x, w0, w1, col, went, mult);
                W = __dmul_rn(W, mult);
                l = nl;
                ++steps;
            }
        }
        warp_merge_add(t, sum, valid, lane, acc);
    }
    unsigned long long ws = steps, ww = walks;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        ws += __shfl_down_sync(0xffffffffu, ws, d);
        ww += __shfl_down_sync(0xffffffffu, ww, d);
    }
    if (lane == 0) {
        atomicAdd(&counters[C_STEPS], ws);
        atomicAdd(&counters[C_WALKS], ww);
    }
}

__global__ void mc_classic_finish(int64_t m, const double* __restrict__ acc, int64_t N, double* __restrict__ y) {
    MCF_KERNEL_ENTRY();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
        y[t] = acc[t] / (double)N;
}

static mcf_status solve_mc_classic(mcf_graph* g, const mcf_params* p, const double* v, const int64_t* nodes,
                                   int64_t n_nodes, double* y, mcf_stats* stats) {
    set_error("");
    MCF_TRY(check_params(g, p));
    if (!y) return fail(MCF_ERR_INVALID_ARG, "y is NULL");
    if (p->deterministic)
        return fail(MCF_ERR_UNSUPPORTED, "the deterministic mode covers RandFunmAction solves only");
    if (p->precision != MCF_F64) return fail(MCF_ERR_UNSUPPORTED, "the classical method runs in float64 only");
    if (p->walks_per_node < 1) return fail(MCF_ERR_INVALID_ARG, "walks_per_node (walks per entry) must be >= 1");
    if (nodes && n_nodes < 0) return fail(MCF_ERR_INVALID_ARG, "n_nodes must be >= 0");
    cudaStream_t st = (cudaStream_t)p->stream;
    const int64_t n = g->n;
    const int64_t m = nodes ? n_nodes : n;
    const int64_t N = p->walks_per_node;
    if (m > 0xffffffffLL) return fail(MCF_ERR_UNSUPPORTED, "at most 2^32 - 1 entries per call");
    if (m > 0 && N > INT64_MAX / m) return fail(MCF_ERR_INVALID_ARG, "too many walks");
    const double gamma = p->scale == 0.0 ? 1.0 : p->scale;
    const int K = p->n_coeffs - 1;
    keep_pool_memory();
    Scratch sc(st);
    const int64_t* nodes_dev = nullptr;
    unsigned long long* counters;
    MCF_TRY(sc.get(&counters, N_COUNTERS));
    MCF_CUDA_TRY(cudaMemsetAsync(counters, 0, N_COUNTERS * sizeof(unsigned long long), st));
    if (nodes && m > 0) {
        if (is_device_ptr(nodes)) {
            nodes_dev = nodes;
            check_nodes<<<grid_for(m, 256), 256, 0, st>>>(m, nodes_dev, n, counters);
            unsigned long long h = 0;
            MCF_CUDA_TRY(cudaMemcpyAsync(&h, &counters[C_FLAGS], sizeof(h), cudaMemcpyDeviceToHost, st));
            MCF_CUDA_TRY(cudaStreamSynchronize(st));
            if (h & 2ull) return fail(MCF_ERR_INVALID_ARG, "node index out of range");
        } else {
            for (int64_t t = 0; t < m; ++t)
                if (nodes[t] < 0 || nodes[t] >= n) return fail(MCF_ERR_INVALID_ARG, "node index out of range");
            int64_t* nd;
            MCF_TRY(sc.get(&nd, m));
            MCF_CUDA_TRY(cudaMemcpyAsync(nd, nodes, m * sizeof(int64_t), cudaMemcpyHostToDevice, st));
            nodes_dev = nd;
        }
    }
    const double* v_dev = v;
    if (v && !is_device_ptr(v) && n > 0) {
        double* vd;
        MCF_TRY(sc.get(&vd, n));
        MCF_CUDA_TRY(cudaMemcpyAsync(vd, v, n * sizeof(double), cudaMemcpyHostToDevice, st));
        v_dev = vd;
    }
    const bool y_on_dev = is_device_ptr(y);
    double* y_dev = y;
    if (!y_on_dev) MCF_TRY(sc.get(&y_dev, std::max<int64_t>(m, 1)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    EventGuard event_guard{&e0, &e1};
    if (m > 0) {
        Rec<true>* rec;
        double *acc, *zeta;
        MCF_TRY(sc.get(&rec, n));
        MCF_TRY(sc.get(&acc, m));
        MCF_TRY(sc.get(&zeta, MCF_MAX_COEFFS));
        MCF_CUDA_TRY(cudaMemcpyAsync(zeta, p->coeffs, p->n_coeffs * sizeof(double), cudaMemcpyHostToDevice, st));
        MCF_CUDA_TRY(cudaMemsetAsync(acc, 0, m * sizeof(double), st));
        build_records<true><<<grid_for(n, 256), 256, 0, st>>>(n, g->row_ptr, g->row_abs, gamma, nullptr, rec);
        if (stats) {
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, st);
        }
        const uint2 key = philox_key(p->seed);
        if (g->weighted) {
            auto kern = mc_classic_kernel<true>;
            kern<<<persistent_grid(kern, 256, 0), 256, 0, st>>>(m, nodes_dev, N, rec, g->col_idx, g->went, v_dev,
                                                                zeta, K, p->w_cutoff, key, p->request_id, acc,
                                                                counters);
        } else {
            auto kern = mc_classic_kernel<false>;
            kern<<<persistent_grid(kern, 256, 0), 256, 0, st>>>(m, nodes_dev, N, rec, g->col_idx, g->went, v_dev,
                                                                zeta, K, p->w_cutoff, key, p->request_id, acc,
                                                                counters);
        }
        MCF_CUDA_TRY(cudaGetLastError());
        if (stats) cudaEventRecord(e1, st);
        mc_classic_finish<<<grid_for(m, 256), 256, 0, st>>>(m, acc, N, y_dev);
        MCF_CUDA_TRY(cudaGetLastError());
    }
    if (!y_on_dev && m > 0) MCF_CUDA_TRY(cudaMemcpyAsync(y, y_dev, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    mcf_status rc = finish_stats(stats, counters, e0, e1, st);
    if (rc != MCF_OK) return rc;
    if (!y_on_dev) MCF_CUDA_TRY(cudaStreamSynchronize(st));
    return MCF_OK;
}

// ====================================================================== allocation-free entry
// mcf_total_communicability_noalloc runs the same kernels as
// mcf_total_communicability, but every scratch buffer is carved from one
// file-scope device array of fixed size instead of being allocated, for
// callers that cannot allocate device memory.  Every GPU that loads the
// library holds this array until the process exits.
constexpr int64_t NOALLOC_MAX_NODES = MCF_NOALLOC_MAX_NODES;
constexpr int64_t NOALLOC_MAX_WALKS = MCF_NOALLOC_MAX_WALKS;

constexpr size_t na_align(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t NOALLOC_SCAN_BYTES = scan_tmp_bytes_for(NOALLOC_MAX_NODES);
// The carved layout, in the order solve_tc_noalloc takes it.
constexpr size_t NOALLOC_BYTES =
    na_align(8 * NOALLOC_MAX_NODES) * 7 +                      // r, colnorm, nw, flag, woff, spos, acc
    na_align(4 * NOALLOC_MAX_NODES) +                          // starts
    na_align(8 * (NOALLOC_MAX_NODES + 1)) +                    // soff
    na_align(sizeof(Rec<true>) * NOALLOC_MAX_NODES) +          // node records (largest variant)
    na_align(4 * (NOALLOC_MAX_WALKS / WARP_CHUNK + 2)) +       // chunk table
    na_align(NOALLOC_SCAN_BYTES) +                             // scan block totals
    na_align(8 * (RED_BLOCKS + 1)) + na_align(8 * N_COUNTERS) + na_align(8 * MCF_MAX_COEFFS) +
    na_align(8 * 4);                                           // partials, counters, coefficients, check flags
static_assert(sizeof(Rec<true>) >= sizeof(Rec<false>), "the record slot holds either variant");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (the host symbol is only a stand-in and must never be handed
// to a kernel).  The cached address belongs to the context it was taken in,
// so the library must not be used across a cudaDeviceReset.
static void* g_noalloc_base[64] = {};
static std::mutex g_noalloc_mu;

static mcf_status noalloc_base(void** out) {
    int dev = 0;
    MCF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(MCF_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(MCF_ERR_CUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
        g_noalloc_base[dev] = p;
    }
    *out = g_noalloc_base[dev];
    return MCF_OK;
}

struct Carve {
    char* p;
    template <class T>
    T* take(size_t count) {
        T* r = reinterpret_cast<T*>(p);
        p += na_align(count * sizeof(T));
        return r;
    }
};

// Memory-safety checks of a caller's device CSR (the walks index with these
// values): row_ptr[0] = 0, row_ptr[n] = nnz, rows non-decreasing inside
// [0, nnz], columns in [0, n) and strictly increasing within a row.
__global__ void noalloc_check_csr(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                                  const int32_t* __restrict__ col, unsigned long long* __restrict__ bad) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rp[i], e = rp[i + 1];
        if ((i == 0 && b != 0) || (i == n - 1 && e != nnz) || b < 0 || b > e || e > nnz) {
            atomicOr(bad, 1ull);
            continue;
        }
        for (int64_t p = b; p < e; ++p) {
            const int32_t j = col[p];
            if (j < 0 || j >= n || (p > b && col[p - 1] >= j)) {
                atomicOr(bad, 2ull);
                break;
            }
        }
    }
}

static mcf_status solve_tc_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                                   const mcf_params* p, double* y) {
    set_error("");
    if (!p) return fail(MCF_ERR_INVALID_ARG, "params is NULL");
    if (n < 0 || nnz < 0) return fail(MCF_ERR_INVALID_ARG, "n and nnz must be >= 0");
    if (n > NOALLOC_MAX_NODES)
        return fail(MCF_ERR_INVALID_ARG, "n = " + std::to_string(n) + " exceeds the allocation-free limit of " +
                                             std::to_string(NOALLOC_MAX_NODES) + " nodes");
    if (nnz >= ((int64_t)1 << 32)) return fail(MCF_ERR_INVALID_ARG, "nnz must be below 2^32");
    if (!p->coeffs || p->n_coeffs < 1 || p->n_coeffs > MCF_MAX_COEFFS)
        return fail(MCF_ERR_INVALID_ARG, "coeffs must hold 1.." + std::to_string(MCF_MAX_COEFFS) + " values");
    if (p->n_walks < 0 || p->walks_per_node < 0) return fail(MCF_ERR_INVALID_ARG, "walk counts must be >= 0");
    if (p->n_coeffs > 2 && p->n_walks == 0 && p->walks_per_node == 0)
        return fail(MCF_ERR_INVALID_ARG, "n_walks or walks_per_node must be > 0");
    // walk ids run up to N_s + n (rounding) or walks_per_node * n; compared
    // without forming the sums, which could overflow for huge requests
    const bool too_many = p->walks_per_node > 0 ? (n > 0 && p->walks_per_node > NOALLOC_MAX_WALKS / n)
                                                : p->n_walks > NOALLOC_MAX_WALKS - n;
    if (too_many)
        return fail(MCF_ERR_INVALID_ARG, "the walk count (N_s + n, or walks_per_node * n) exceeds the allocation-free "
                                         "limit of " + std::to_string(NOALLOC_MAX_WALKS) + " walks");
    if (!(p->w_cutoff >= 0.0)) return fail(MCF_ERR_INVALID_ARG, "w_cutoff must be >= 0");
    if (p->precision != MCF_F64 && p->precision != MCF_F32W_F64ACC)
        return fail(MCF_ERR_INVALID_ARG, "unknown precision");
    if (p->deterministic != 0) return fail(MCF_ERR_INVALID_ARG, "deterministic is reserved and must be 0");
    if (p->target_rel_err != 0.0)
        return fail(MCF_ERR_INVALID_ARG, "accuracy-targeted solves need scratch: target_rel_err must be 0 here");
    if (!(p->scale >= 0.0) || !isfinite(p->scale)) return fail(MCF_ERR_INVALID_ARG, "scale must be finite and >= 0");
    for (int k = 0; k < p->n_coeffs; ++k)
        if (!isfinite(p->coeffs[k])) return fail(MCF_ERR_INVALID_ARG, "coefficients must be finite");
    if (!row_ptr || !y || (nnz > 0 && !col_idx)) return fail(MCF_ERR_INVALID_ARG, "NULL array");
    if (!is_device_ptr(row_ptr) || (nnz > 0 && !is_device_ptr(col_idx)) || !is_device_ptr(y))
        return fail(MCF_ERR_INVALID_ARG, "row_ptr, col_idx and y must be device pointers");
    if (n == 0) return MCF_OK;
    void* base = nullptr;
    MCF_TRY(noalloc_base(&base));
    cudaStream_t st = (cudaStream_t)p->stream;
    const double gamma = p->scale == 0.0 ? 1.0 : p->scale;
    const int K = p->n_coeffs - 1;
    const bool f64 = p->precision == MCF_F64;
    Carve cv{static_cast<char*>(base)};
    Prep P;
    P.r = cv.take<double>(NOALLOC_MAX_NODES);
    P.colnorm = cv.take<double>(NOALLOC_MAX_NODES);
    P.nw = cv.take<int64_t>(NOALLOC_MAX_NODES);
    P.flag = cv.take<int64_t>(NOALLOC_MAX_NODES);
    P.woff = cv.take<int64_t>(NOALLOC_MAX_NODES);
    P.spos = cv.take<int64_t>(NOALLOC_MAX_NODES);
    double* acc = cv.take<double>(NOALLOC_MAX_NODES);
    P.starts = cv.take<int32_t>(NOALLOC_MAX_NODES);
    P.soff = cv.take<int64_t>(NOALLOC_MAX_NODES + 1);
    P.cof = P.soff;   // every start is walked: walk ids and walked space coincide
    P.rec = cv.take<Rec<true>>(NOALLOC_MAX_NODES);
    uint32_t* chunk_s0 = cv.take<uint32_t>(NOALLOC_MAX_WALKS / WARP_CHUNK + 2);
    P.scan_bytes = NOALLOC_SCAN_BYTES;
    P.scan_tmp = cv.take<char>(P.scan_bytes);
    P.part = cv.take<double>(RED_BLOCKS + 1);
    P.counters = cv.take<unsigned long long>(N_COUNTERS);
    P.zeta = cv.take<double>(MCF_MAX_COEFFS);
    unsigned long long* bad = cv.take<unsigned long long>(4);
    if ((size_t)(cv.p - static_cast<char*>(base)) > NOALLOC_BYTES)
        return fail(MCF_ERR_UNSUPPORTED, "internal: allocation-free scratch layout exceeds its array");
    // The array keeps the previous call's contents: clear what must start at zero.
    MCF_CUDA_TRY(cudaMemsetAsync(bad, 0, 4 * sizeof(unsigned long long), st));
    MCF_CUDA_TRY(cudaMemsetAsync(P.counters, 0, N_COUNTERS * sizeof(unsigned long long), st));
    MCF_CUDA_TRY(cudaMemsetAsync(acc, 0, n * sizeof(double), st));
    noalloc_check_csr<<<grid_for(n, 256), 256, 0, st>>>(n, nnz, row_ptr, col_idx, bad);
    unsigned long long hbad = 0;
    MCF_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st));
    MCF_CUDA_TRY(cudaStreamSynchronize(st));
    if (hbad) return fail(MCF_ERR_INVALID_GRAPH, "invalid CSR: row_ptr or column indices out of range or unsorted");
    MCF_CUDA_TRY(cudaMemcpyAsync(P.zeta, p->coeffs, p->n_coeffs * sizeof(double), cudaMemcpyHostToDevice, st));
    // the same kernel sequence as prepare() + solve_action(), binary matrix, v = 1
    r_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, row_ptr, col_idx, nullptr, nullptr, gamma, P.r);
    colnorm_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, row_ptr, nullptr, gamma, P.colnorm, P.part);
    sum_partials<<<1, RED_THREADS, 0, st>>>(P.part, RED_BLOCKS, P.part + RED_BLOCKS);
    alloc_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, P.colnorm, P.part + RED_BLOCKS, p->n_walks, p->walks_per_node,
                                                   nullptr, P.nw, P.flag);
    MCF_TRY(scan_i64(P.nw, P.woff, n, (int64_t*)&P.counters[C_TOTAL], P.scan_tmp, P.scan_bytes, st));
    MCF_TRY(scan_i64(P.flag, P.spos, n, (int64_t*)&P.counters[C_STARTS], P.scan_tmp, P.scan_bytes, st));
    compact_starts<<<grid_for(n, 256), 256, 0, st>>>(n, P.flag, P.spos, P.woff, P.starts, P.soff, P.counters);
    if (f64)
        build_records<true><<<grid_for(n, 256), 256, 0, st>>>(n, row_ptr, nullptr, gamma, P.r, (Rec<true>*)P.rec);
    else
        build_records<false><<<grid_for(n, 256), 256, 0, st>>>(n, row_ptr, nullptr, gamma, P.r, (Rec<false>*)P.rec);
    if (K >= 2) {
        chunk_table<<<grid_for(n, 256), 256, 0, st>>>(P.soff, P.counters, chunk_s0);
        mcf_graph view;
        view.n = n;
        view.nnz = nnz;
        view.row_ptr = const_cast<int64_t*>(row_ptr);
        view.col_idx = const_cast<int32_t*>(col_idx);
        const uint2 key = philox_key(p->seed);
        if (f64) launch_action_walks<true, false>(&view, P, chunk_s0, K, p->w_cutoff, key, p->request_id, acc, nullptr, st);
        else launch_action_walks<false, false>(&view, P, chunk_s0, K, p->w_cutoff, key, p->request_id, acc, nullptr, st);
    }
    finalize_q<<<grid_for(n, 256), 256, 0, st>>>(n, acc, P.nw);
    const double z0 = p->coeffs[0], z1 = K >= 1 ? p->coeffs[1] : 0.0;
    action_epilogue<<<grid_for(n, EPI_ROWS), EPI_ROWS, 0, st>>>(n, row_ptr, col_idx, nullptr, gamma, z0, z1, nullptr,
                                                                P.r, acc, y);
    MCF_CUDA_TRY(cudaGetLastError());
    return MCF_OK;
}

// ====================================================================== accuracy-targeted solves
// A solve with params.target_rel_err > 0 runs independent replicas of the
// plain solve (replica r: seed + r * 0x9E3779B97F4A7C15, so replica 0 is the
// plain solve) and returns their mean.  The replicas alternate between two
// halves H1, H2; est = max_i |mean_H1,i - mean_H2,i| / 2 / max_i |mean_i| has the
// spread of the relative l_inf error of the mean of all replicas (the two
// half-means differ by twice that error's standard deviation per entry), an
// estimate of the error in the standard-error sense of Section 3.5 that
// needs no variance formula, so it serves every query kind.  Starting from two
// replicas, the count grows to R (est / target)^2 x 1.25 (Theorem 1: the error
// falls like N^-1/2) until est <= target or the walk cap is reached.
__global__ void rep_add(int64_t m, const double* __restrict__ y, double* __restrict__ h) {
    MCF_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        h[i] += y[i];
}

// out = (H1 + H2) / (c1 + c2); mx[0] = max |H1/c1 - H2/c2| / 2, mx[1] = max |out|
// (as the bits of non-negative doubles, which order like the values).
__global__ void rep_finish(int64_t m, const double* __restrict__ h1, const double* __restrict__ h2, double c1,
                           double c2, double* __restrict__ out, unsigned long long* __restrict__ mx) {
    MCF_KERNEL_ENTRY();
    double d = 0.0, a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double mean = (h1[i] + h2[i]) / (c1 + c2);
        out[i] = mean;
        d = fmax(d, 0.5 * fabs(h1[i] / c1 - h2[i] / c2));
        a = fmax(a, fabs(mean));
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
        d = fmax(d, __shfl_xor_sync(0xffffffffu, d, k));
        a = fmax(a, __shfl_xor_sync(0xffffffffu, a, k));
    }
    if ((threadIdx.x & 31) == 0) {
        if (d > 0.0) atomicMax(&mx[0], (unsigned long long)__double_as_longlong(d));
        if (a > 0.0) atomicMax(&mx[1], (unsigned long long)__double_as_longlong(a));
    }
}

using SolveOnce = std::function<mcf_status(const mcf_params&, double*, mcf_stats*)>;
constexpr int64_t BUDGET_DEFAULT_MAX_WALKS = (int64_t)1 << 34;
constexpr int BUDGET_MAX_REPLICAS = 4096;

static mcf_status solve_budgeted(int64_t m, double* out, const mcf_params* p, mcf_stats* stats, const SolveOnce& one) {
    const double target = p->target_rel_err;
    const int64_t cap = p->max_walks > 0 ? p->max_walks : BUDGET_DEFAULT_MAX_WALKS;
    cudaStream_t st = (cudaStream_t)p->stream;
    keep_pool_memory();
    Scratch sc(st);
    double *yr, *h1, *h2, *mean;
    unsigned long long* mx;
    const int64_t mm = std::max<int64_t>(m, 1);
    MCF_TRY(sc.get(&yr, mm));
    MCF_TRY(sc.get(&h1, mm));
    MCF_TRY(sc.get(&h2, mm));
    MCF_TRY(sc.get(&mx, 2));
    const bool out_on_dev = is_device_ptr(out);
    if (out_on_dev) mean = out;
    else MCF_TRY(sc.get(&mean, mm));
    MCF_CUDA_TRY(cudaMemsetAsync(h1, 0, mm * sizeof(double), st));
    MCF_CUDA_TRY(cudaMemsetAsync(h2, 0, mm * sizeof(double), st));
    int R = 0;
    int64_t walks = 0, steps = 0, per_replica = 0;
    double kernel_ms = 0.0, est = INFINITY;
    uint32_t flags = 0;
    auto run_to = [&](int R_next) -> mcf_status {
        for (; R < R_next; ++R) {
            mcf_params q = *p;
            q.target_rel_err = 0.0;
            q.error_estimate = 0;
            q.seed = p->seed + (uint64_t)R * 0x9E3779B97F4A7C15ull;
            mcf_stats s1{};
            MCF_TRY(one(q, yr, &s1));
            if (m > 0) rep_add<<<grid_for(m, 256), 256, 0, st>>>(m, yr, (R & 1) ? h2 : h1);
            walks += s1.walks;
            steps += s1.walk_steps;
            kernel_ms += s1.kernel_ms;
            flags |= s1.flags;
            per_replica = std::max<int64_t>(per_replica, s1.walks);
        }
        const double c1 = (double)((R + 1) / 2), c2 = (double)(R / 2);
        MCF_CUDA_TRY(cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned long long), st));
        if (m > 0) rep_finish<<<grid_for(m, 256), 256, 0, st>>>(m, h1, h2, c1, c2, mean, mx);
        MCF_CUDA_TRY(cudaGetLastError());
        unsigned long long hm[2];
        MCF_CUDA_TRY(cudaMemcpyAsync(hm, mx, sizeof(hm), cudaMemcpyDeviceToHost, st));
        MCF_CUDA_TRY(cudaStreamSynchronize(st));
        double d, a;
        memcpy(&d, &hm[0], sizeof(d));
        memcpy(&a, &hm[1], sizeof(a));
        est = a > 0.0 ? d / a : 0.0;
        return MCF_OK;
    };
    MCF_TRY(run_to(2));
    while (est > target) {
        const int64_t by_cap = per_replica > 0 ? cap / per_replica : BUDGET_MAX_REPLICAS;
        const int R_cap = (int)std::min<int64_t>(BUDGET_MAX_REPLICAS, by_cap) & ~1;
        const double want = (double)R * (est / target) * (est / target) * 1.25;
        int R_next = (int)std::min<double>((double)R_cap, ceil(want));
        R_next = (R_next + 1) & ~1;
        if (R_next > R_cap) R_next = R_cap;
        if (R_next <= R) break;   // the walk cap is reached
        MCF_TRY(run_to(R_next));
    }
    if (!out_on_dev && m > 0) {
        MCF_CUDA_TRY(cudaMemcpyAsync(out, mean, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        MCF_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (stats) {
        stats->walks = walks;
        stats->walk_steps = steps;
        stats->kernel_ms = kernel_ms;
        stats->flags = flags;
        stats->max_rel_se = 0.0;
        stats->est_rel_err = est;
        stats->replicas = R;
    }
    if (est > target)
        return fail(MCF_ERR_ACCURACY_BUDGET, "estimated relative error " + std::to_string(est) + " above the target " +
                                                 std::to_string(target) + " at the walk cap (" + std::to_string(walks) +
                                                 " walks in " + std::to_string(R) + " replicas); the mean is returned");
    return MCF_OK;
}

static mcf_status check_budget(const mcf_params* p) {
    if (!p) return fail(MCF_ERR_INVALID_ARG, "params is NULL");
    if (!(p->target_rel_err >= 0.0) || !isfinite(p->target_rel_err))
        return fail(MCF_ERR_INVALID_ARG, "target_rel_err must be finite and >= 0");
    if (p->max_walks < 0) return fail(MCF_ERR_INVALID_ARG, "max_walks must be >= 0");
    return MCF_OK;
}

}  // namespace mcf

using namespace mcf;

uint64_t mcf::kernel_runs_walk() { return this_unit_kernel_runs(); }

extern "C" {

// The single-query entry points: with params->target_rel_err > 0 the solve
// runs as replicas until the estimated error meets the target.
static mcf_status action_entry(mcf_graph_t g, const mcf_params* params, const double* v, double* y, mcf_stats* stats,
                               bool ones, const int64_t* nodes, int64_t n_nodes) {
    set_error("");
    MCF_TRY(check_budget(params));
    if (params->target_rel_err == 0.0) return solve_action(g, params, v, y, stats, ones, nodes, n_nodes);
    MCF_TRY(check_params(g, params));
    if (!y) return fail(MCF_ERR_INVALID_ARG, "y is NULL");
    if (nodes && n_nodes < 0) return fail(MCF_ERR_INVALID_ARG, "n_nodes must be >= 0");
    const int64_t m = nodes ? n_nodes : g->n;
    return solve_budgeted(m, y, params, stats, [&](const mcf_params& q, double* yr, mcf_stats* s1) {
        return solve_action(g, &q, v, yr, s1, ones, nodes, n_nodes);
    });
}

mcf_status mcf_action(mcf_graph_t g, const mcf_params* params, const double* v, double* y, mcf_stats* stats) {
    return action_entry(g, params, v, y, stats, false, nullptr, -1);
}

mcf_status mcf_action_nodes(mcf_graph_t g, const mcf_params* params, const double* v, const int64_t* nodes,
                            int64_t n_nodes, double* y, mcf_stats* stats) {
    if (!nodes) return fail(MCF_ERR_INVALID_ARG, "nodes is NULL");
    return action_entry(g, params, v, y, stats, v == nullptr, nodes, n_nodes);
}

mcf_status mcf_total_communicability(mcf_graph_t g, const mcf_params* params, double* y, mcf_stats* stats) {
    return action_entry(g, params, nullptr, y, stats, true, nullptr, -1);
}

mcf_status mcf_subgraph_centrality(mcf_graph_t g, const mcf_params* params, const int64_t* nodes, int64_t n_nodes,
                                   double* d, mcf_stats* stats) {
    set_error("");
    MCF_TRY(check_budget(params));
    if (params->target_rel_err == 0.0) return solve_diag(g, params, nodes, n_nodes, d, stats);
    MCF_TRY(check_params(g, params));
    if (!d) return fail(MCF_ERR_INVALID_ARG, "d is NULL");
    if (nodes && n_nodes < 0) return fail(MCF_ERR_INVALID_ARG, "n_nodes must be >= 0");
    const int64_t m = nodes ? n_nodes : g->n;
    return solve_budgeted(m, d, params, stats, [&](const mcf_params& q, double* dr, mcf_stats* s1) {
        return solve_diag(g, &q, nodes, n_nodes, dr, s1);
    });
}

mcf_status mcf_katz(mcf_graph_t g, double gamma, int32_t K, const mcf_params* params, double* y, mcf_stats* stats) {
    set_error("");
    if (!g || !params) return fail(MCF_ERR_INVALID_ARG, "NULL argument");
    if (!(gamma > 0.0) || !isfinite(gamma)) return fail(MCF_ERR_INVALID_ARG, "gamma must be > 0");
    if (K < 0 || K + 1 > MCF_MAX_COEFFS) return fail(MCF_ERR_INVALID_ARG, "K out of range");
    if (K == 0) {
        if (g->lambda_max <= 0.0 && g->nnz > 0) {
            double lam;
            MCF_TRY(mcf_spectral_radius(g, 1e-10, 100000, &lam));
        }
        const double rho = gamma * g->lambda_max;
        if (!(rho < 1.0)) return fail(MCF_ERR_INVALID_ARG, "the Neumann series needs gamma * lambda_max < 1");
        if (rho <= 0.0) K = 2;
        else K = std::max(2, (int)ceil(log(1e-4 * (1.0 - rho)) / log(rho) - 1.0));
        if (K + 1 > MCF_MAX_COEFFS) return fail(MCF_ERR_INVALID_ARG, "rho too close to 1 for the coefficient limit");
    }
    double ones[MCF_MAX_COEFFS];
    for (int k = 0; k <= K; ++k) ones[k] = 1.0;
    mcf_params p = *params;
    p.coeffs = ones;
    p.n_coeffs = K + 1;
    p.scale = gamma;
    return action_entry(g, &p, nullptr, y, stats, true, nullptr, -1);
}

mcf_status mcf_funm_full(mcf_graph_t g, const mcf_params* params, double* F, mcf_stats* stats) {
    return solve_full(g, params, F, stats);
}

mcf_status mcf_mc_classic(mcf_graph_t g, const mcf_params* params, const double* v, const int64_t* nodes,
                          int64_t n_nodes, double* y, mcf_stats* stats) {
    return solve_mc_classic(g, params, v, nodes, n_nodes, y, stats);
}

mcf_status mcf_total_communicability_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                                             const mcf_params* params, double* y) {
    return solve_tc_noalloc(n, nnz, row_ptr, col_idx, params, y);
}

}  // extern "C"
