// Batched solves: many queries on many resident graphs in one pass.
//
// Total-communicability and Katz queries (RandFunmAction with v = 1,
// Algorithm 3) on binary graphs in MCF_F32W_F64ACC with fewer than
// B_FUSED_MAX_WALKS walks share ONE persistent walk launch; subgraph-centrality
// queries (RandFunmDiag, Section 3.3) on symmetric binary graphs in
// MCF_F32W_F64ACC share one diag launch.  Their preparation
// (Definition 1's allocation) and epilogues are segmented kernels over the
// concatenation of all their node sets.  Each query keeps its own walk ids
// (the exclusive prefix of N_i over its own nodes) and Philox streams, and the
// per-query reductions replicate the single-query kernels' order, so every
// result equals the single call's up to float64 summation order.  Other
// queries run one after another through the single-query entry points.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <new>
#include <vector>

#include "mcf_device.cuh"
#include "mcf_internal.cuh"

namespace mcf {

constexpr int B_RED_BLOCKS = 256;    // must equal the single-query colnorm grid
// A total-communicability or Katz query with this many walks fills the GPU on
// its own; it runs through the single-query kernel (whose per-step parameters
// are kernel arguments, measured about 12 % faster per step than the fused
// kernel's per-warp query slot), the smaller ones share the fused launch.
constexpr int64_t B_FUSED_MAX_WALKS = (int64_t)1 << 25;
constexpr int B_RED_THREADS = 256;
constexpr int B_CHUNK = 32;
enum { BC_NEXT = 0, BC_STEPS = 1, BC_WALKS = 2, BC_FLAGS = 3, BC_TOTAL = 4, BC_STARTS = 5, BC_STARTS_TC = 6,
       BC_CHUNKS = 7, BC_NEXT_SC = 8 /* .. 11: one per diag launch */, BC_N = 16 };

// Device descriptor of one fused query.
struct BQuery {
    int64_t node_off;   // first global node index of the query
    int64_t n;          // nodes of its graph
    int64_t walk_base;  // TC: first padded global walk id (device-filled)
    int64_t walk_end;   // TC: walk_base + walks of the query (device-filled)
    int64_t gw_base;    // exclusive prefix of N_i at node_off (device-filled)
    int64_t rm_off;     // offset of the degree table
    int64_t blk_off;    // first 32-entry output block
    int64_t n_out;      // outputs: n, or the size of the SC subset
    const int64_t* rp;
    const int32_t* col;
    const int64_t* cp;     // column-major copy of A (== rp/col for a symmetric A)
    const int32_t* ri;
    const uint2* nod;
    const uint2* eod;
    const uint32_t* ekey;  // SC: row offset of each entry's neighbour (keys of the rows Q_k)
    const double* diag;
    const int64_t* nodes;  // SC subset (device) or null
    const int64_t* sub_ptr;   // SC subset: per-column lists of the requested rows (SubList)
    const int32_t* sub_row;
    double* out;           // device output
    const double* zeta;    // K + 1 coefficients (device)
    const float* zf;       // the same, rounded to float32 (the walk kernels' precision)
    double gamma, z0, z1, wc;
    int64_t n_walks, wpn;
    uint2 key;
    uint32_t req;
    float wc32;
    int32_t K;
    int32_t kind;   // 0: TC/Katz, 1: SC
    int32_t subset; // SC: only the requested nodes
};

__device__ __forceinline__ int find_le(const int64_t* __restrict__ a, int m, int64_t x) {
    // largest q in [0, m) with a[q] <= x (a non-decreasing, a[0] <= x)
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ||C'_i|| and per-query partial sums with exactly the partition and order of
// the single-query colnorm kernel (block b of query q = blockIdx.x of that grid).
__global__ void bq_colnorm(const BQuery* __restrict__ desc, double* __restrict__ colnorm, double* __restrict__ part) {
    MCF_KERNEL_ENTRY();
    const BQuery& d = desc[blockIdx.y];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d.n; i += (int64_t)gridDim.x * blockDim.x) {
        const double c = __dmul_rn(d.gamma, sqrt((double)(d.cp[i + 1] - d.cp[i])));
        colnorm[d.node_off + i] = c;
        s += c;
    }
    s = block_sum_d(s);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

__global__ void bq_sum(const double* __restrict__ part, int nb, double* __restrict__ tot) {
    MCF_KERNEL_ENTRY();
    double s = 0.0;
    const double* p = part + (int64_t)blockIdx.x * nb;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += p[b];
    s = block_sum_d(s);
    if (threadIdx.x == 0) tot[blockIdx.x] = s;
}

__global__ void bq_alloc(const BQuery* __restrict__ desc, const int64_t* __restrict__ qoff, int Q, int64_t NT,
                         const double* __restrict__ colnorm, const double* __restrict__ tot,
                         const uint8_t* __restrict__ need, int64_t* __restrict__ nw, int64_t* __restrict__ flag) {
    MCF_KERNEL_ENTRY();
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < NT; u += (int64_t)gridDim.x * blockDim.x) {
        const int q = find_le(qoff, Q, u);
        const BQuery& d = desc[q];
        const double c = colnorm[u];
        int64_t w = 0;
        if (c > 0.0) {
            if (d.wpn > 0) w = d.wpn;
            else {
                const long long r = llround(__dmul_rn((double)d.n_walks, __ddiv_rn(c, tot[q])));
                w = r < 1 ? 1 : (int64_t)r;
            }
        }
        nw[u] = w;
        flag[u] = (w > 0 && (!d.subset || need[u])) ? 1 : 0;
    }
}

// Per-query walk bases: TC queries get consecutive walk ranges padded to
// whole 32-walk chunks, so no chunk mixes two queries.
__global__ void bq_bases(BQuery* __restrict__ desc, int Q, int Q_tc, int64_t NT, const int64_t* __restrict__ gw,
                         int64_t* __restrict__ wbase, unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int64_t total = (int64_t)counters[BC_TOTAL];
    int64_t base = 0;
    for (int q = 0; q < Q; ++q) {
        BQuery& d = desc[q];
        const int64_t first = d.node_off < NT ? gw[d.node_off] : total;
        const int64_t end = d.node_off + d.n;
        const int64_t next = end < NT ? gw[end] : total;
        d.gw_base = first;
        if (q < Q_tc) {
            d.walk_base = base;
            d.walk_end = base + (next - first);
            wbase[q] = base;
            base += (next - first + B_CHUNK - 1) / B_CHUNK * B_CHUNK;
        } else {
            d.walk_base = 0;
            d.walk_end = next - first;
        }
    }
    counters[BC_CHUNKS] = (unsigned long long)(base / B_CHUNK);
}

__global__ void bq_starts_tc(const int64_t* __restrict__ flag, const int64_t* __restrict__ spos, int64_t NT_tc,
                             unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    if (threadIdx.x == 0 && blockIdx.x == 0)
        counters[BC_STARTS_TC] = NT_tc > 0 ? (unsigned long long)(spos[NT_tc - 1] + flag[NT_tc - 1]) : 0ull;
}

__global__ void bq_compact(const BQuery* __restrict__ desc, const int64_t* __restrict__ qoff, int Q, int Q_tc,
                           int64_t NT, const int64_t* __restrict__ flag, const int64_t* __restrict__ spos,
                           const int64_t* __restrict__ gw, uint32_t* __restrict__ starts, int64_t* __restrict__ soff) {
    MCF_KERNEL_ENTRY();
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < NT; u += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[u]) continue;
        const int q = find_le(qoff, Q, u);
        const BQuery& d = desc[q];
        const int64_t local = gw[u] - d.gw_base;
        starts[spos[u]] = (uint32_t)u;
        soff[spos[u]] = q < Q_tc ? d.walk_base + local : local;
    }
}

__global__ void bq_chunks(const uint32_t* __restrict__ starts, const int64_t* __restrict__ soff,
                          const int64_t* __restrict__ nw, const unsigned long long* __restrict__ counters,
                          uint32_t* __restrict__ chunk_s0) {
    MCF_KERNEL_ENTRY();
    const int64_t S = (int64_t)counters[BC_STARTS_TC];
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c0 = (soff[s] + B_CHUNK - 1) / B_CHUNK;
        const int64_t c1 = (soff[s] + nw[starts[s]] + B_CHUNK - 1) / B_CHUNK;
        for (int64_t c = c0; c < c1; ++c) chunk_s0[c] = (uint32_t)s;
    }
}

// rm_q[d] = float(gamma_q * d): r_l and the weight multiplier of a state of degree d.
__global__ void bq_degree_tables(const BQuery* __restrict__ desc, const int64_t* __restrict__ rmoff, int Q,
                                 int64_t total, float* __restrict__ rm) {
    MCF_KERNEL_ENTRY();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int q = find_le(rmoff, Q, t);
        rm[t] = __double2float_rn(__dmul_rn(desc[q].gamma, (double)(t - rmoff[q])));
    }
}

__global__ void bq_mark(const BQuery* __restrict__ desc, int q0, int Q, uint8_t* __restrict__ need) {
    MCF_KERNEL_ENTRY();
    const BQuery& d = desc[q0 + blockIdx.y];
    if (!d.subset) return;
    // one CTA per requested node, its threads over the node's row
    for (int64_t t = blockIdx.x; t < d.n_out; t += gridDim.x) {
        const int64_t i = d.nodes[t];
        for (int64_t p = d.rp[i] + threadIdx.x; p < d.rp[i + 1]; p += blockDim.x) need[d.node_off + d.col[p]] = 1;
    }
}

// ---------------------------------------------------------------- TC / Katz walks
// The persistent kernel of walk_tc_kernel over the padded walk space of all
// TC queries.  A warp serves one query at a time: before it starts on a chunk
// of another query it lets its lanes finish their walks, then loads that
// query's parameters into its shared slot.
// The fields a walk step reads come first, in three 16-byte words that a
// step loads with three vector loads (StepParams); the rest serve refills.
struct __align__(16) WarpQuery {
    const uint2* eod;
    const float* rm;
    uint2 key;
    uint32_t req;
    float wc32;
    const float* zeta;   // float32 coefficients in global memory (L1-resident)
    int32_t K;
    int32_t pad;
    const uint2* nod;
    int64_t walk_base;
    int64_t walk_end;
    int64_t node_off;
};

struct StepParams {
    const uint2* eod;
    const float* rm;
    uint2 key;
    uint32_t req;
    float wc32;
    const float* zeta;
    int32_t K;
};

__device__ __forceinline__ StepParams step_params(const WarpQuery& w) {
    const uint4* v = reinterpret_cast<const uint4*>(&w);
    const uint4 a = v[0], b = v[1], c = v[2];
    StepParams p;
    p.eod = reinterpret_cast<const uint2*>(((uint64_t)a.y << 32) | a.x);
    p.rm = reinterpret_cast<const float*>(((uint64_t)a.w << 32) | a.z);
    p.key = make_uint2(b.x, b.y);
    p.req = b.z;
    p.wc32 = __uint_as_float(b.w);
    p.zeta = reinterpret_cast<const float*>(((uint64_t)c.y << 32) | c.x);
    p.K = (int32_t)c.z;
    return p;
}

template <int MINB>
__global__ void __launch_bounds__(256, MINB) bwalk_tc_kernel(
    const BQuery* __restrict__ desc, int Q_tc, const float* __restrict__ rm_all, const int64_t* __restrict__ rmoff,
    const uint32_t* __restrict__ starts, const int64_t* __restrict__ soff, const uint32_t* __restrict__ chunk_s0,
    const int64_t* __restrict__ wbase, int grab, double* __restrict__ acc, unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    double* const acc2 = nullptr;   // batches estimate no standard errors
    __shared__ WarpQuery wq[256 / 32];
    __shared__ WalkResults<float2> rbuf[256 / 32];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    WarpQuery& Wq = wq[threadIdx.x >> 5];
    WalkResults<float2>& rb = rbuf[threadIdx.x >> 5];
    const int32_t n_chunks = (int32_t)counters[BC_CHUNKS];
    const int64_t S = (int64_t)counters[BC_STARTS_TC];
    int32_t c = -1, c_end = -1, cn = -1;
    int qn = -1, cur_q = -1;
    bool have_next = false;
    int p = 0, valid = 0, rb_n = 0;
    int32_t cs = 0;
    bool exhausted = false, active = false;
    int64_t g = 0;
    uint32_t node0 = 0, off = 0, deg = 0;
    int k = 0;
    float W = 1.f;
    uint4 u = make_uint4(0u, 0u, 0u, 0u);
    F2Acc a32;
    uint32_t my_steps = 0, my_walks = 0, flags = 0;
    for (;;) {
        unsigned idle = __ballot_sync(FULL, !active);
        // refill once at least WALK_REFILL_MIN lanes are idle (or all are), as
        // the single-query kernel does: fewer refill passes for a few idle lanes
        if (idle != FULL && __popc(idle) < WALK_REFILL_MIN) idle = 0u;
        while (idle && !exhausted) {
            if (p >= valid) {
                if (!have_next) {
                    ++c;
                    if (c >= c_end) {
                        int32_t base = 0;
                        if (lane == 0) base = (int32_t)atomicAdd((unsigned int*)&counters[BC_NEXT], (unsigned)grab);
                        base = __shfl_sync(FULL, base, 0);
                        c = base;
                        c_end = min(base + grab, n_chunks);
                    }
                    if (c >= n_chunks) {
                        exhausted = true;
                        break;
                    }
                    cn = c;
                    qn = find_le(wbase, Q_tc, (int64_t)cn * B_CHUNK);
                    have_next = true;
                }
                if (qn != cur_q) {
                    if (__any_sync(FULL, active)) break;  // finish this query's walks first
                    const BQuery& d = desc[qn];
                    if (lane == 0) {
                        Wq.nod = d.nod;
                        Wq.eod = d.eod;
                        Wq.rm = rm_all + rmoff[qn];
                        Wq.walk_base = d.walk_base;
                        Wq.walk_end = d.walk_end;
                        Wq.node_off = d.node_off;
                        Wq.key = d.key;
                        Wq.req = d.req;
                        Wq.wc32 = d.wc32;
                        Wq.K = d.K;
                        Wq.zeta = d.zf;
                    }
                    __syncwarp();
                    cur_q = qn;
                }
                have_next = false;
                const int64_t s0 = chunk_s0[cn];
                const int64_t bnd = (s0 + 1 + lane < S) ? soff[s0 + 1 + lane] : INT64_MAX;
                const int64_t gl = (int64_t)cn * B_CHUNK + lane;
                int cnt = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int64_t bv = __shfl_sync(FULL, bnd, cnt + step - 1);
                    if (bv <= gl) cnt += step;
                }
                cs = (int32_t)(s0 + cnt);
                valid = (int)min((int64_t)B_CHUNK, Wq.walk_end - (int64_t)cn * B_CHUNK);
                p = 0;
                c = cn;
            }
            const int avail = valid - p;
            const int rank = __popc(idle & lt_mask);
            const int src = min(p + rank, B_CHUNK - 1);
            const int32_t s_new = __shfl_sync(FULL, cs, src);
            if (((idle >> lane) & 1u) && rank < avail) {
                g = (int64_t)c * B_CHUNK + p + rank - Wq.walk_base;   // the query's own walk id
                node0 = starts[s_new];
                const uint2 od = Wq.nod[node0 - Wq.node_off];
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
        if (!__any_sync(FULL, active)) {
            if (exhausted || !have_next) break;
            continue;   // drained: switch to the next query
        }
        bool done = false;
        if (active) {
            // The next state's record is read only once the walk is known to
            // go on (after the cutoff test): a read issued earlier is wasted
            // DRAM work at every walk's end, and the kernel is bound by the
            // rate of random DRAM reads.
            const StepParams P = step_params(Wq);
            const bool last = k + 2 >= P.K || deg == 0;
            done = !(fabsf(W) > P.wc32);
            if (!done) {
                const float t = __ldg(P.rm + deg);
                a32.add(__fmul_rn(__fmul_rn(__ldg(P.zeta + k + 2), W), t));
                if (last) {
                    done = true;
                } else {
                    uint32_t w0, w1;
                    walk_words<false>(u, k, (uint32_t)g, (uint32_t)((uint64_t)g >> 32), P.req, P.key, w0, w1);
                    const uint2 nx = load_od(P.eod + (int64_t)off + __umulhi(w0, deg), policy_evict_first());
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
            }
        }
        rb_n = rb.push(done, node0, make_float2(a32.hi, a32.lo), rb_n, lane, lt_mask, acc, acc2);
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
        atomicAdd(&counters[BC_STEPS], ws);
        atomicAdd(&counters[BC_WALKS], ww);
        if (flags) atomicOr(&counters[BC_FLAGS], (unsigned long long)flags);
    }
}

// ---------------------------------------------------------------- SC walks
// walk_diag_od_kernel over the start columns of the SC queries [q_lo, q_hi)
// (one launch per row-table size; cls picks the launch's start counter): a
// CTA takes one start at a time, reads its query's parameters into shared
// memory when the query changes and runs the start's walks with per-lane
// refill, recording visits in a row Q_k keyed by row offset (one random
// 8-byte record per step), then the dot phase over the requested rows and
// the clear.  Every SC query of a batch is on a symmetric binary graph.
struct CtaOdQuery {
    int64_t node_off;
    const int64_t* rp;
    const int32_t* col;
    const uint2* nod;
    const uint2* eod;
    const uint32_t* ekey;
    const float* rm;
    SubList sub;
    double* dacc;
    double gamma;
    uint2 key;
    uint32_t req;
    float wc32;
    int32_t K;
    float zeta[MCF_MAX_COEFFS];
};

// MINB: as for walk_diag_od_kernel (4 for the 256-thread launches, which
// ptxas then fits in 64 registers: four CTAs per SM; else 0).
template <int MINB>
__global__ void __launch_bounds__(256, MINB) bwalk_diag_kernel(
    const BQuery* __restrict__ desc, const int64_t* __restrict__ qoff, int Q, const uint32_t* __restrict__ starts,
    const int64_t* __restrict__ soff, const int64_t* __restrict__ nw, const float* __restrict__ rm_all,
    const int64_t* __restrict__ rmoff, int q_lo, int q_hi, int cls, int cap_log2, double* __restrict__ qval,
    double* __restrict__ acc, unsigned long long* __restrict__ counters) {
    MCF_KERNEL_ENTRY();
    extern __shared__ uint32_t od_keys[];
    __shared__ CtaOdQuery cq;
    __shared__ int64_t cur, cq_lo, cq_hi, s_lo, s_hi;
    __shared__ int count;
    __shared__ unsigned long long next_walk;
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
    uint32_t steps = 0, walks = 0, flags = 0;
    // Takes the next start (thread 0): its query's parameters are loaded into
    // shared memory only when the query changes (consecutive starts of a CTA
    // mostly belong to one query).
    auto next_start = [&]() {
        cur = s_lo + (int64_t)atomicAdd(&counters[BC_NEXT_SC + cls], 1ull);
        next_walk = 0ull;
        if (cur >= s_hi) return;
        const int64_t ug = (int64_t)starts[cur];
        if (ug >= cq_lo && ug < cq_hi) return;
        const int q = find_le(qoff, Q, ug);
        const BQuery& d = desc[q];
        cq.rp = d.rp;
        cq.col = d.col;
        cq.nod = d.nod;
        cq.eod = d.eod;
        cq.ekey = d.ekey;
        cq.rm = rm_all + rmoff[q];
        cq.sub = SubList{d.subset ? d.sub_ptr : nullptr, d.sub_row, nullptr};
        cq.dacc = acc + d.node_off;
        cq.node_off = d.node_off;
        cq.gamma = d.gamma;
        cq.key = d.key;
        cq.req = d.req;
        cq.wc32 = d.wc32;
        cq.K = d.K;
        for (int k = 0; k <= d.K; ++k) cq.zeta[k] = (float)d.zeta[k];
        cq_lo = qoff[q];
        cq_hi = qoff[q + 1];
    };
    if (threadIdx.x == 0) {
        // the starts of queries [q_lo, q_hi): starts[] holds the global
        // indices of all start columns in increasing order
        const int64_t S_tc = (int64_t)counters[BC_STARTS_TC];
        const int64_t S = (int64_t)counters[BC_STARTS];
        auto first_at = [&](int64_t node) {
            int64_t lo = S_tc, hi = S;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if ((int64_t)starts[mid] < node) lo = mid + 1;
                else hi = mid;
            }
            return lo;
        };
        s_lo = first_at(qoff[q_lo]);
        s_hi = first_at(qoff[q_hi]);
        cq_lo = cq_hi = -1;
        next_start();
    }
    __syncthreads();
    for (;;) {
        const int64_t s = cur;
        if (s >= s_hi) break;
        const uint32_t ug = starts[s];
        const uint32_t k0 = (uint32_t)(ug - cq.node_off);
        const int64_t Nk = nw[ug];
        const int64_t g0 = soff[s];
        const uint2 od0 = cq.nod[k0];
        const int K = cq.K;
        const float wc32 = cq.wc32;
        if (threadIdx.x == 0 && 1.0f > wc32 && K >= 2) {
            // the N_k step-0 visits, into the cleared table while the walks begin
            const int h = od_insert_always(t, od0.x);
            atomicAdd(&t.val[h], (double)Nk * (double)cq.zeta[2]);
        }
        bool active = false, paused = false, exhausted = false;
        int64_t g = 0;
        uint32_t off = 0, deg = 0;
        int k = 0;
        float W = 1.f;
        uint4 u = make_uint4(0u, 0u, 0u, 0u);
        for (;;) {
            for (;;) {
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
                        else atomicAdd(&t.val[h], (double)__fmul_rn(cq.zeta[k + 2], W));
                    }
                    if (!done && !paused) {
                        if (k + 2 >= K || deg == 0) {
                            done = true;
                        } else {
                            uint32_t w0, w1;
                            walk_words<false>(u, k, (uint32_t)g, (uint32_t)((uint64_t)g >> 32), cq.req, cq.key, w0,
                                              w1);
                            const uint2 nx = load_od(cq.eod + (int64_t)off + __umulhi(w0, deg), policy_evict_first());
                            W = __fmul_rn(W, __ldg(cq.rm + deg));
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
            const bool any_paused = __syncthreads_or(paused);
            __threadfence_block();
            od_apply(t, k0, Nk, cq.rp, cq.col, cq.ekey, cq.sub, cq.gamma, cq.dacc);
            __syncthreads();
            od_clear(t);
            if (threadIdx.x == 0) {
                count = 0;
                if (!any_paused) next_start();   // the start is done
            }
            __syncthreads();
            if (!any_paused) break;
            paused = false;   // the table is empty again: the paused walks go on
        }
    }
    unsigned long long ws = steps, ww = walks;
#pragma unroll
    for (int dd = 16; dd > 0; dd >>= 1) {
        ws += __shfl_down_sync(FULL, ws, dd);
        ww += __shfl_down_sync(FULL, ww, dd);
        flags |= __shfl_down_sync(FULL, flags, dd);
    }
    if (lane == 0) {
        atomicAdd(&counters[BC_STEPS], ws);
        atomicAdd(&counters[BC_WALKS], ww);
        if (flags) atomicOr(&counters[BC_FLAGS], (unsigned long long)flags);
    }
}

// Device time (the global nanosecond timer) when this kernel runs: one
// at the start and one at the end of a batch's device work bound the window
// in which that work ran.
__global__ void stamp_kernel(unsigned long long* __restrict__ slot) {
    MCF_KERNEL_ENTRY();
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    *slot = t;
}

// ---------------------------------------------------------------- epilogues
__global__ void bq_finalize(int64_t NT_tc, double* __restrict__ acc, const int64_t* __restrict__ nw) {
    MCF_KERNEL_ENTRY();
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < NT_tc; u += (int64_t)gridDim.x * blockDim.x)
        acc[u] = nw[u] > 0 ? acc[u] / (double)nw[u] : 0.0;
}

// One warp per 32-entry output block of any query: TC rows
// y_i = zeta_0 + zeta_1 gamma deg_i + gamma sum_j q_j, SC entries
// d = zeta_0 + zeta_1 gamma a_ii + sum_k a'_ik <Q_k, C'_i>.
// y = zeta_0 1 + zeta_1 r + A' q for the TC/Katz queries (global nodes
// [0, NT_tc)): a CTA takes EPI_ROWS consecutive global nodes at a time and
// sums the rows of each query they span with tile_row_sums.  Launched with
// EPI_ROWS threads.
__global__ void __launch_bounds__(EPI_ROWS) bq_epilogue_tc(const BQuery* __restrict__ desc,
                                                           const int64_t* __restrict__ qoff, int Q_tc, int64_t NT_tc,
                                                           const double* __restrict__ acc) {
    MCF_KERNEL_ENTRY();
    __shared__ double prod[EPI_CHUNK];
    __shared__ int64_t off[EPI_ROWS + 1];
    for (int64_t g0 = (int64_t)blockIdx.x * EPI_ROWS; g0 < NT_tc; g0 += (int64_t)gridDim.x * EPI_ROWS) {
        const int64_t g1 = min(g0 + (int64_t)EPI_ROWS, NT_tc);
        int q = find_le(qoff, Q_tc, g0);
        for (int64_t u = g0; u < g1;) {
            while (qoff[q + 1] <= u) ++q;   // queries of no nodes
            const BQuery& d = desc[q];
            const int64_t r0 = u - d.node_off;
            const int nr = (int)(min(g1, qoff[q + 1]) - u);
            const double s = tile_row_sums(r0, nr, d.rp, d.col, nullptr, acc + d.node_off, prod, off);
            if ((int)threadIdx.x < nr) {
                const int64_t row = r0 + threadIdx.x;
                const double r = __dmul_rn(d.gamma, (double)(off[threadIdx.x + 1] - off[threadIdx.x]));
                d.out[row] = d.z0 + d.z1 * r + d.gamma * s;
            }
            __syncthreads();   // off[] is rewritten for the next rows
            u += nr;
        }
    }
}

// The subgraph-centrality outputs of a batch, 32 per warp.
__global__ void bq_epilogue(const BQuery* __restrict__ desc, const int64_t* __restrict__ boff, int Q,
                            int64_t n_blocks, const double* __restrict__ acc) {
    MCF_KERNEL_ENTRY();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = warp; b < n_blocks; b += nwarps) {
        const int q = find_le(boff, Q, b);
        const BQuery& d = desc[q];
        const int64_t base = (b - d.blk_off) * 32;
        if (d.kind == 0) {
            continue;   // bq_epilogue_tc
        } else {
            const int64_t t = base + lane;
            if (t < d.n_out) {
                const int64_t i = d.nodes ? d.nodes[t] : t;
                double v = d.z0;
                if (d.K >= 1) v += d.z1 * (d.gamma * d.diag[i]);
                d.out[t] = v + acc[d.node_off + i];
            }
        }
    }
}

}  // namespace mcf

using namespace mcf;

uint64_t mcf::kernel_runs_batch() { return this_unit_kernel_runs(); }

// ====================================================================== host
struct BatchTuning {
    int minb = 5;
    int grab = 4;
};

static std::mutex g_tune_mu;
static std::map<std::string, BatchTuning> g_tune_cache;

constexpr int B_DIAG_CAP_LOG2 = 13;   // largest row table of the fused diag kernel
struct DiagShape {
    int cap_log2 = 10;
    int threads = 256;
    size_t smem = 0;
    int grid = 0;
};
static_assert(BC_NEXT_SC + (B_DIAG_CAP_LOG2 - 10) < BC_N, "a start counter per diag launch");
struct DiagClass {   // SC queries [q_lo, q_hi) of the fused list, one diag launch
    int q_lo = 0, q_hi = 0;
    DiagShape sh;
};

struct mcf_batch {
    std::vector<mcf_query> queries;
    std::vector<int> fused;       // query indices: TC/Katz first, then SC
    std::vector<int> single;      // queries run through the single-query path
    std::vector<std::vector<double>> coeffs;   // owned coefficient lists (Katz)
    std::vector<mcf_params> params;            // per query, with owned coefficients
    int Q = 0, Q_tc = 0;
    int64_t NT = 0, NT_tc = 0, rm_total = 0, n_blocks = 0, max_chunks = 0, sc_nodes = 0;
    std::vector<DiagClass> diag;   // SC queries grouped by row-table size (2^10 .. 2^13: at most 4)
    int tc_grid[4] = {0, 0, 0, 0};   // persistent grids of the walk kernel for 5, 6, 8 and 4 blocks per SM
    BatchTuning tune;
    std::vector<void*> bufs;
    // device arrays
    BQuery* desc = nullptr;
    int64_t *qoff = nullptr, *rmoff = nullptr, *boff = nullptr, *wbase = nullptr;
    double *colnorm = nullptr, *part = nullptr, *tot = nullptr, *acc = nullptr, *zeta = nullptr, *qval = nullptr;
    float* zf = nullptr;
    std::vector<float> zf_host;
    int64_t *nw = nullptr, *flag = nullptr, *gw = nullptr, *spos = nullptr, *soff = nullptr;
    uint32_t *starts = nullptr, *chunk_s0 = nullptr;
    float* rm = nullptr;
    uint8_t* need = nullptr;
    unsigned long long* counters = nullptr;
    void* scan_tmp = nullptr;
    size_t scan_bytes = 0;
    // outputs staged on the device for host destinations
    std::vector<mcf_status> qstatus;   // per query: MCF_OK, or MCF_ERR_ACCURACY_BUDGET from an accuracy-targeted query
    std::vector<std::pair<double*, double*>> out_copies;   // (device staging, host dst)
    std::vector<int64_t> out_sizes;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
    size_t bytes = 0;                         // device memory the plan holds
    cudaStream_t stream = nullptr;            // the planning stream (allocations and frees)
    unsigned long long* stamps = nullptr;     // device: global-timer ns at the start and end of the last run
    unsigned long long window[2] = {0, 0};    // host copy of the last run's stamps
};

// Plan buffers come from the device's stream-ordered pool (which keeps freed
// memory, keep_pool_memory) on the planning stream: a server planning a batch
// per request group then neither maps new pages nor synchronises the device.
template <class T>
static mcf_status balloc(mcf_batch* b, T** p, size_t count) {
    void* q = nullptr;
    keep_pool_memory();
    if (injected_allocation_failure()) return fail(MCF_ERR_OOM, "device allocation for the batch failed (injected)");
    if (cudaMallocAsync(&q, std::max<size_t>(count, 1) * sizeof(T), b->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(MCF_ERR_OOM, "device allocation for the batch failed");
    }
    b->bufs.push_back(q);
    b->bytes += std::max<size_t>(count, 1) * sizeof(T);
    *p = static_cast<T*>(q);
    return MCF_OK;
}

// Table size of the fused diag kernel for starts of about nk walks, as the
// single-query kernel sizes it: about 16 visits per walk, 2^10 .. 2^13 slots
// (5 bytes each in shared memory: key and filter bits), each CTA with a
// region of as many float64 values in global memory.  Threads per CTA follow
// from it (64 for 2^10, 128 for 2^11, 256 above): a CTA serves one start at a
// time, so lanes beyond its walks idle.  SC queries of a batch are grouped by this size, one launch per
// group, so that a query with long starts does not shrink every CTA's
// occupancy to its table.
static int diag_cap_log2(int64_t nk) {
    const int threads = nk <= 64 ? 64 : (nk <= 128 ? 128 : 256);
    const int64_t want_slots = std::max<int64_t>(16 * nk, 4 * threads);
    int c = 10;
    while (c < B_DIAG_CAP_LOG2 && ((int64_t)1 << c) < want_slots) ++c;
    return c;
}

static mcf_status diag_shape(int64_t nk, DiagShape* sh) {
    sh->cap_log2 = diag_cap_log2(nk);
    sh->threads = sh->cap_log2 == 10 ? 64 : (sh->cap_log2 == 11 ? 128 : 256);
    sh->smem = od_smem_bytes(sh->cap_log2);
    auto kern = sh->threads == 256 ? bwalk_diag_kernel<4> : bwalk_diag_kernel<0>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)od_smem_bytes(B_DIAG_CAP_LOG2)) !=
        cudaSuccess) {
        cudaGetLastError();
        return fail(MCF_ERR_CUDA, "diag kernel shared memory");
    }
    sh->grid = persistent_grid(kern, sh->threads, sh->smem);
    return MCF_OK;
}

// Walks per start of a subgraph-centrality query, the hint that sizes its
// CTAs and hashed rows.
static int64_t sc_walk_hint(const mcf_params& p, int64_t n) {
    return p.walks_per_node > 0 ? p.walks_per_node : std::max<int64_t>(1, p.n_walks / std::max<int64_t>(n, 1));
}

// Device memory a batch holding only query q allocates (mcf_batch_create's
// buffers for one fused query, or a bound on the single-query path's
// stream-ordered scratch for the other kinds); the request server admits by
// the sum of these over the requests in flight.
static int64_t query_footprint(const mcf_query& q, int64_t* out) {
    const mcf_graph* g = q.graph;
    const mcf_params& p = q.params;
    const int64_t n = g->n, nnz = g->nnz, md = g->max_degree;
    const int64_t walks = p.walks_per_node > 0 ? p.walks_per_node * n : p.n_walks + n;
    const bool binary32 = !g->weighted && p.precision == MCF_F32W_F64ACC && nnz < ((int64_t)1 << 32);
    const bool tc_kind = q.kind == MCF_QUERY_TOTAL_COMMUNICABILITY || q.kind == MCF_QUERY_KATZ;
    const bool sc_kind = q.kind == MCF_QUERY_SUBGRAPH_CENTRALITY;
    const int64_t tc_walks = p.walks_per_node > 0 ? p.walks_per_node * n : p.n_walks;
    const bool host_out = !is_device_ptr(q.out);
    const int64_t m = (sc_kind && q.nodes) ? q.n_nodes : n;
    // subset lists: claim, count and pointer arrays, their scan, one row index per pair
    const int64_t pairs = (sc_kind && q.nodes) ? std::min<int64_t>(nnz, m * md) : 0;
    const int64_t lists = (sc_kind && q.nodes) ? 24 * n + 8 + (int64_t)scan_tmp_bytes(n) + 4 * std::max<int64_t>(pairs, 1)
                                                     + (!is_device_ptr(q.nodes) ? 8 * m : 0)
                                               : 0;
    int64_t b = 16 + 4096;   // stamps, descriptor and offsets
    const bool plain = p.target_rel_err == 0.0 && p.deterministic == 0;
    if (plain && ((tc_kind && binary32 && tc_walks < B_FUSED_MAX_WALKS) || (sc_kind && binary32 && g->symmetric))) {
        b += 60 * n + 8 + 8 * B_RED_BLOCKS + 8 + BC_N * 8 + 12 * MCF_MAX_COEFFS + (int64_t)scan_tmp_bytes(n);
        b += 4 * (md + 1) + 4;   // degree table
        if (tc_kind) {
            b += 4 * (walks / B_CHUNK + 3);
        } else {
            DiagShape sh;
            if (diag_shape(sc_walk_hint(p, n), &sh) != MCF_OK) return -1;
            b += 1 * n + 8 + (int64_t)sh.grid * ((int64_t)1 << sh.cap_log2) * 8 + lists;
        }
        if (host_out) b += 8 * m;
    } else {
        // the single-query path: per-node preparation (about 130 bytes per
        // node with both precisions' records), chunk table, degree table,
        // outputs and inputs staged from the host, and for subgraph
        // centrality its accumulators and hashed or dense rows Q_k (at most
        // 4864 CTAs x 16384 float64 values)
        b += 200 * n + 4 * (walks / 32 + 3) + 4 * (md + 1) + (int64_t)scan_tmp_bytes(n) + 8 * MCF_MAX_COEFFS;
        if (sc_kind) b += 9 * n + lists + (int64_t)4864 * 16384 * 8;
        if (p.target_rel_err != 0.0) b += 32 * m + 16;   // replica output, two half sums, the mean
        if (p.deterministic) b += 8 * walks;               // one float64 slot per walk
    }
    *out = b;
    return b;
}

static mcf_status check_query(const mcf_query& q, int idx) {
    const std::string where = "query " + std::to_string(idx) + ": ";
    if (!q.graph) return fail(MCF_ERR_INVALID_ARG, where + "graph is NULL");
    if (!q.out) return fail(MCF_ERR_INVALID_ARG, where + "out is NULL");
    if (q.kind < 0 || q.kind > 3) return fail(MCF_ERR_INVALID_ARG, where + "unknown kind");
    const mcf_params& p = q.params;
    if (q.kind != MCF_QUERY_KATZ && (!p.coeffs || p.n_coeffs < 1 || p.n_coeffs > MCF_MAX_COEFFS))
        return fail(MCF_ERR_INVALID_ARG, where + "coeffs must hold 1.." + std::to_string(MCF_MAX_COEFFS) + " values");
    if (p.n_walks < 0 || p.walks_per_node < 0) return fail(MCF_ERR_INVALID_ARG, where + "walk counts must be >= 0");
    // as the single calls: fewer than 2^36 walks, compared without overflow
    const int64_t n = q.graph->n, lim = (int64_t)1 << 36;
    if (p.walks_per_node > 0 ? (n > 0 && p.walks_per_node > lim / n) : p.n_walks > lim - n)
        return fail(MCF_ERR_INVALID_ARG, where + "more than 2^36 walks per query");
    if (!(p.w_cutoff >= 0.0)) return fail(MCF_ERR_INVALID_ARG, where + "w_cutoff must be >= 0");
    if (!(p.target_rel_err >= 0.0) || !isfinite(p.target_rel_err) || p.max_walks < 0)
        return fail(MCF_ERR_INVALID_ARG, where + "target_rel_err must be finite and >= 0, max_walks >= 0");
    if (p.precision != MCF_F64 && p.precision != MCF_F32W_F64ACC)
        return fail(MCF_ERR_INVALID_ARG, where + "unknown precision");
    if (p.deterministic != 0 && p.deterministic != 1) return fail(MCF_ERR_INVALID_ARG, where + "deterministic is 0 or 1");
    if (q.kind == MCF_QUERY_ACTION && !q.v) return fail(MCF_ERR_INVALID_ARG, where + "v is NULL");
    if (q.kind == MCF_QUERY_SUBGRAPH_CENTRALITY && q.nodes && q.n_nodes < 0)
        return fail(MCF_ERR_INVALID_ARG, where + "n_nodes must be >= 0");
    return MCF_OK;
}

// The fused launch sequence (capturable: no allocation, no host synchronisation).
static mcf_status record(mcf_batch* b, cudaStream_t st) {
    MCF_CUDA_TRY(cudaMemsetAsync(b->counters, 0, BC_N * sizeof(unsigned long long), st));
    MCF_CUDA_TRY(cudaMemsetAsync(b->acc, 0, (size_t)std::max<int64_t>(b->NT, 1) * sizeof(double), st));
    if (b->sc_nodes > 0) {
        MCF_CUDA_TRY(cudaMemsetAsync(b->need, 0, (size_t)b->sc_nodes, st));
    }
    if (b->NT == 0) return MCF_OK;
    const int Q = b->Q;
    if (Q > b->Q_tc)
        bq_mark<<<dim3(1024, Q - b->Q_tc), 256, 0, st>>>(b->desc, b->Q_tc, Q, b->need - b->NT_tc);
    bq_colnorm<<<dim3(B_RED_BLOCKS, Q), B_RED_THREADS, 0, st>>>(b->desc, b->colnorm, b->part);
    bq_sum<<<Q, B_RED_THREADS, 0, st>>>(b->part, B_RED_BLOCKS, b->tot);
    bq_alloc<<<grid_for(b->NT, 256), 256, 0, st>>>(b->desc, b->qoff, Q, b->NT, b->colnorm, b->tot,
                                                   b->sc_nodes ? b->need - b->NT_tc : nullptr, b->nw, b->flag);
    MCF_TRY(scan_i64(b->nw, b->gw, b->NT, (int64_t*)&b->counters[BC_TOTAL], b->scan_tmp, b->scan_bytes, st));
    MCF_TRY(scan_i64(b->flag, b->spos, b->NT, (int64_t*)&b->counters[BC_STARTS], b->scan_tmp, b->scan_bytes, st));
    bq_bases<<<1, 32, 0, st>>>(b->desc, Q, b->Q_tc, b->NT, b->gw, b->wbase, b->counters);
    bq_starts_tc<<<1, 32, 0, st>>>(b->flag, b->spos, b->NT_tc, b->counters);
    bq_compact<<<grid_for(b->NT, 256), 256, 0, st>>>(b->desc, b->qoff, Q, b->Q_tc, b->NT, b->flag, b->spos, b->gw,
                                                     b->starts, b->soff);
    MCF_CUDA_TRY(cudaGetLastError());
    bq_degree_tables<<<grid_for(b->rm_total, 256), 256, 0, st>>>(b->desc, b->rmoff, Q, b->rm_total, b->rm);
    if (b->Q_tc > 0) {
        bq_chunks<<<grid_for(b->NT_tc, 256), 256, 0, st>>>(b->starts, b->soff, b->nw, b->counters, b->chunk_s0);
        auto launch = [&](auto kern, int grid) {
            kern<<<grid, 256, 0, st>>>(b->desc, b->Q_tc, b->rm, b->rmoff, b->starts, b->soff, b->chunk_s0, b->wbase,
                                       b->tune.grab, b->acc, b->counters);
        };
        if (b->tune.minb == 8) launch(bwalk_tc_kernel<8>, b->tc_grid[2]);
        else if (b->tune.minb == 6) launch(bwalk_tc_kernel<6>, b->tc_grid[1]);
        else if (b->tune.minb == 4) launch(bwalk_tc_kernel<4>, b->tc_grid[3]);
        else launch(bwalk_tc_kernel<5>, b->tc_grid[0]);
        MCF_CUDA_TRY(cudaGetLastError());
        bq_finalize<<<grid_for(b->NT_tc, 256), 256, 0, st>>>(b->NT_tc, b->acc, b->nw);
    }
    if (Q > b->Q_tc) {
        for (size_t c = 0; c < b->diag.size(); ++c) {
            const DiagClass& dc = b->diag[c];
            auto kern = dc.sh.threads == 256 ? bwalk_diag_kernel<4> : bwalk_diag_kernel<0>;
            kern<<<dc.sh.grid, dc.sh.threads, dc.sh.smem, st>>>(
                b->desc, b->qoff, Q, b->starts, b->soff, b->nw, b->rm, b->rmoff, dc.q_lo, dc.q_hi, (int)c,
                dc.sh.cap_log2, b->qval, b->acc, b->counters);
            MCF_CUDA_TRY(cudaGetLastError());
        }
    }
    if (b->NT_tc > 0) {
        bq_epilogue_tc<<<grid_for(b->NT_tc, EPI_ROWS), EPI_ROWS, 0, st>>>(b->desc, b->qoff, b->Q_tc, b->NT_tc, b->acc);
        MCF_CUDA_TRY(cudaGetLastError());
    }
    if (Q > b->Q_tc)
        bq_epilogue<<<grid_for(b->n_blocks * 32, 256), 256, 0, st>>>(b->desc, b->boff, Q, b->n_blocks, b->acc);
    MCF_CUDA_TRY(cudaGetLastError());
    return MCF_OK;
}

static std::string tune_key(const mcf_batch* b) {
    int64_t walks = 0;
    for (int i = 0; i < b->Q_tc; ++i) {
        const mcf_params& p = b->params[b->fused[i]];
        walks += p.walks_per_node > 0 ? p.walks_per_node * b->queries[b->fused[i]].graph->n : p.n_walks;
    }
    auto lg = [](int64_t x) { int r = 0; while (x > 1) { x >>= 1; ++r; } return r; };
    return "tc:w" + std::to_string(lg(walks)) + ":n" + std::to_string(lg(b->NT_tc)) + ":q" + std::to_string(lg(b->Q_tc));
}

static void load_tune_file() {
    static bool loaded = false;
    if (loaded) return;
    loaded = true;
    const char* path = getenv("MCF_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[256];
    int minb, grab;
    while (fscanf(f, "%255s %d %d", key, &minb, &grab) == 3) g_tune_cache[key] = BatchTuning{minb, grab};
    fclose(f);
}

static void save_tune_file() {
    const char* path = getenv("MCF_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "w");
    if (!f) return;
    for (auto& kv : g_tune_cache) fprintf(f, "%s %d %d\n", kv.first.c_str(), kv.second.minb, kv.second.grab);
    fclose(f);
}

// Times each candidate launch shape of the fused walk kernel on this batch
// (results are discarded; walks are deterministic) and keeps the fastest.
static mcf_status autotune(mcf_batch* b, cudaStream_t st) {
    if (b->Q_tc == 0) return MCF_OK;
    const std::string key = tune_key(b);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_tune_file();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->tune = it->second;
            return MCF_OK;
        }
    }
    const BatchTuning cands[] = {{4, 1}, {4, 4}, {5, 1}, {5, 4}, {6, 4}, {8, 4}};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    EventGuard event_guard{&e0, &e1};
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    BatchTuning pick = b->tune;
    ScopedL2Fetch fetch(L2_FETCH_BYTES);
    for (const BatchTuning& c : cands) {
        b->tune = c;
        MCF_TRY(record(b, st));   // warm
        cudaEventRecord(e0, st);
        MCF_TRY(record(b, st));
        cudaEventRecord(e1, st);
        MCF_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            pick = c;
        }
    }
    b->tune = pick;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = pick;
    save_tune_file();
    return MCF_OK;
}

mcf_status mcf::batch_query_status(const mcf_batch* b, int i) { return b->qstatus[i]; }

void mcf::batch_window(const mcf_batch* b, uint64_t* begin_ns, uint64_t* end_ns) {
    *begin_ns = b->window[0];
    *end_ns = b->window[1];
}

extern "C" {

mcf_status mcf_query_footprint(const mcf_query* q, size_t* bytes) {
    set_error("");
    if (!q || !bytes) return fail(MCF_ERR_INVALID_ARG, "NULL argument");
    MCF_TRY(check_query(*q, 0));
    int64_t b = 0;
    if (query_footprint(*q, &b) < 0) return MCF_ERR_CUDA;
    *bytes = (size_t)b;
    return MCF_OK;
}

mcf_status mcf_batch_device_bytes(mcf_batch_t b, size_t* bytes) {
    set_error("");
    if (!b || !bytes) return fail(MCF_ERR_INVALID_ARG, "NULL argument");
    *bytes = b->bytes;
    return MCF_OK;
}

mcf_status mcf_batch_destroy(mcf_batch_t b) {
    if (!b) return MCF_OK;
    // every run ends with a synchronisation of its stream, so no work of the
    // plan is pending; the buffers go back to the pool in stream order
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void* p : b->bufs) cudaFreeAsync(p, b->stream);
    cudaStreamSynchronize(b->stream);
    cudaGetLastError();
    delete b;
    return MCF_OK;
}

mcf_status mcf_batch_create(const mcf_query* queries, int32_t n_queries, uint32_t flags, void* stream,
                            mcf_batch_t* out) {
    set_error("");
    if (!out) return fail(MCF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!queries || n_queries <= 0) return fail(MCF_ERR_INVALID_ARG, "empty batch");
    for (int i = 0; i < n_queries; ++i) MCF_TRY(check_query(queries[i], i));
    cudaStream_t st = (cudaStream_t)stream;
    mcf_batch* b = new (std::nothrow) mcf_batch();
    if (!b) return fail(MCF_ERR_OOM, "host allocation failed");
    auto bail = [&](mcf_status s) {
        mcf_batch_destroy(b);
        return s;
    };
    cudaGetDevice(&b->device);
    b->stream = st;
    {
        mcf_status rs = balloc(b, &b->stamps, 2);
        if (rs != MCF_OK) return bail(rs);
    }
    b->queries.assign(queries, queries + n_queries);
    b->qstatus.assign(n_queries, MCF_OK);
    b->params.resize(n_queries);
    b->coeffs.resize(n_queries);
    std::vector<int> tc, sc;
    for (int i = 0; i < n_queries; ++i) {
        const mcf_query& q = b->queries[i];
        mcf_params p = q.params;
        if (q.kind == MCF_QUERY_KATZ) {
            if (!(q.katz_gamma > 0.0)) return bail(fail(MCF_ERR_INVALID_ARG, "query " + std::to_string(i) + ": katz_gamma must be > 0"));
            int K = q.katz_terms;
            if (K < 0 || K + 1 > MCF_MAX_COEFFS) return bail(fail(MCF_ERR_INVALID_ARG, "katz_terms out of range"));
            if (K == 0) {
                if (q.graph->lambda_max <= 0.0 && q.graph->nnz > 0) {
                    double lam;
                    mcf_status rc = mcf_spectral_radius(q.graph, 1e-10, 100000, &lam);
                    if (rc != MCF_OK) return bail(rc);
                }
                const double rho = q.katz_gamma * q.graph->lambda_max;
                if (!(rho < 1.0)) return bail(fail(MCF_ERR_INVALID_ARG, "Katz needs gamma * lambda_max < 1"));
                K = rho <= 0.0 ? 2 : std::max(2, (int)ceil(log(1e-4 * (1.0 - rho)) / log(rho) - 1.0));
                if (K + 1 > MCF_MAX_COEFFS) return bail(fail(MCF_ERR_INVALID_ARG, "rho too close to 1"));
            }
            b->coeffs[i].assign(K + 1, 1.0);
            p.scale = q.katz_gamma;
        } else {
            b->coeffs[i].assign(p.coeffs, p.coeffs + p.n_coeffs);
        }
        p.coeffs = b->coeffs[i].data();
        p.n_coeffs = (int32_t)b->coeffs[i].size();
        if (p.n_coeffs > 2 && p.n_walks == 0 && p.walks_per_node == 0)
            return bail(fail(MCF_ERR_INVALID_ARG, "query " + std::to_string(i) + ": n_walks or walks_per_node must be > 0"));
        b->params[i] = p;
        const bool binary32 = !q.graph->weighted && p.precision == MCF_F32W_F64ACC && q.graph->nnz < ((int64_t)1 << 32);
        const int64_t tc_walks = p.walks_per_node > 0 ? p.walks_per_node * q.graph->n : p.n_walks;
        // accuracy-targeted queries run as replicas, deterministic ones with per-walk
        // slots: both through the single-query path
        const bool plain = p.target_rel_err == 0.0 && p.deterministic == 0;
        if ((q.kind == MCF_QUERY_TOTAL_COMMUNICABILITY || q.kind == MCF_QUERY_KATZ) && binary32 && p.n_coeffs >= 3 &&
            tc_walks < B_FUSED_MAX_WALKS && plain)
            tc.push_back(i);
        else if (q.kind == MCF_QUERY_SUBGRAPH_CENTRALITY && binary32 && q.graph->symmetric && p.n_coeffs >= 3 && plain)
            sc.push_back(i);
        else
            b->single.push_back(i);
    }
    b->fused = tc;
    // SC queries grouped by row-table size (one diag launch per group)
    auto sc_cap = [&](int i) { return diag_cap_log2(sc_walk_hint(b->params[i], b->queries[i].graph->n)); };
    std::stable_sort(sc.begin(), sc.end(), [&](int x, int y) { return sc_cap(x) < sc_cap(y); });
    b->fused.insert(b->fused.end(), sc.begin(), sc.end());
    b->Q = (int)b->fused.size();
    b->Q_tc = (int)tc.size();
    if (b->Q > 0) {
        // ---- host-side layout
        std::vector<BQuery> d(b->Q);
        std::vector<int64_t> qoff(b->Q + 1), rmoff(b->Q + 1), boff(b->Q + 1);
        int64_t node = 0, rmt = 0, blocks = 0, max_chunks = 0;
        for (int f = 0; f < b->Q; ++f) {
            const int i = b->fused[f];
            const mcf_query& q = b->queries[i];
            const mcf_params& p = b->params[i];
            mcf_graph* g = q.graph;
            {
                mcf_status rc = ensure_edge_od(g, st);
                if (rc == MCF_OK && f >= b->Q_tc) rc = ensure_edge_key(g, st);
                if (rc != MCF_OK) return bail(rc);
            }
            BQuery& x = d[f];
            memset(&x, 0, sizeof(x));
            x.node_off = node;
            x.n = g->n;
            x.rp = g->row_ptr;
            x.col = g->col_idx;
            x.cp = g->col_ptr;
            x.ri = g->row_idx;
            x.nod = g->node_od;
            x.eod = g->edge_od;
            x.ekey = g->edge_key;
            x.diag = g->diag;
            x.gamma = p.scale == 0.0 ? 1.0 : p.scale;
            x.K = p.n_coeffs - 1;
            x.z0 = p.coeffs[0];
            x.z1 = x.K >= 1 ? p.coeffs[1] : 0.0;
            x.wc = p.w_cutoff;
            x.wc32 = cutoff_f32(p.w_cutoff);
            x.n_walks = p.n_walks;
            x.wpn = p.walks_per_node;
            x.key = philox_key(p.seed);
            x.req = p.request_id;
            x.kind = f < b->Q_tc ? 0 : 1;
            x.subset = (x.kind == 1 && q.nodes) ? 1 : 0;
            x.n_out = x.subset ? q.n_nodes : g->n;
            qoff[f] = node;
            boff[f] = blocks;
            x.blk_off = blocks;
            blocks += (x.n_out + 31) / 32;
            node += g->n;
            rmoff[f] = rmt;
            x.rm_off = rmt;
            rmt += g->max_degree + 1;
            if (f < b->Q_tc) {
                const int64_t mw = p.walks_per_node > 0 ? p.walks_per_node * g->n : p.n_walks + g->n;
                max_chunks += mw / B_CHUNK + 2;
            }
            if (f == b->Q_tc - 1) b->NT_tc = node;
        }
        if (b->Q_tc == 0) b->NT_tc = 0;
        qoff[b->Q] = node;
        rmoff[b->Q] = rmt;
        boff[b->Q] = blocks;
        b->NT = node;
        b->rm_total = rmt;
        b->n_blocks = blocks;
        b->max_chunks = max_chunks + 1;
        b->sc_nodes = b->NT - b->NT_tc;
        if (b->NT >= ((int64_t)1 << 32)) return bail(fail(MCF_ERR_INVALID_ARG, "a batch spans at most 2^32 nodes"));
        // diag launch shapes: one per run of SC queries with equal table size
        b->diag.clear();
        for (int f = b->Q_tc; f < b->Q;) {
            const int i = b->fused[f];
            const int c = diag_cap_log2(sc_walk_hint(b->params[i], b->queries[i].graph->n));
            DiagClass dc;
            dc.q_lo = f;
            while (f < b->Q &&
                   diag_cap_log2(sc_walk_hint(b->params[b->fused[f]], b->queries[b->fused[f]].graph->n)) == c)
                ++f;
            dc.q_hi = f;
            mcf_status rs = diag_shape(sc_walk_hint(b->params[i], b->queries[i].graph->n), &dc.sh);
            if (rs != MCF_OK) return bail(rs);
            b->diag.push_back(dc);
        }
        b->tc_grid[0] = persistent_grid(bwalk_tc_kernel<5>, 256, 0);
        b->tc_grid[1] = persistent_grid(bwalk_tc_kernel<6>, 256, 0);
        b->tc_grid[2] = persistent_grid(bwalk_tc_kernel<8>, 256, 0);
        b->tc_grid[3] = persistent_grid(bwalk_tc_kernel<4>, 256, 0);
        // ---- device buffers
        mcf_status rc = MCF_OK;
        auto A = [&](auto** p, size_t count) {
            if (rc == MCF_OK) rc = balloc(b, p, count);
        };
        A(&b->desc, b->Q);
        A(&b->qoff, b->Q + 1);
        A(&b->rmoff, b->Q + 1);
        A(&b->boff, b->Q + 1);
        A(&b->wbase, std::max(b->Q_tc, 1));
        A(&b->colnorm, b->NT);
        A(&b->part, (size_t)b->Q * B_RED_BLOCKS);
        A(&b->tot, b->Q);
        A(&b->nw, b->NT);
        A(&b->flag, b->NT);
        A(&b->gw, b->NT);
        A(&b->spos, b->NT);
        A(&b->starts, b->NT);
        A(&b->soff, b->NT + 1);
        A(&b->acc, b->NT);
        A(&b->counters, BC_N);
        A(&b->chunk_s0, b->max_chunks);
        A(&b->rm, b->rm_total);
        A(&b->zeta, (size_t)b->Q * MCF_MAX_COEFFS);
        A(&b->zf, (size_t)b->Q * MCF_MAX_COEFFS);
        A(&b->need, b->sc_nodes);
        b->scan_bytes = scan_tmp_bytes(b->NT);
        A((char**)&b->scan_tmp, b->scan_bytes);
        if (b->Q > b->Q_tc) {
            size_t qv = 0;   // the launches run one after another on the stream: one region serves all
            for (const DiagClass& dc : b->diag) qv = std::max(qv, (size_t)dc.sh.grid << dc.sh.cap_log2);
            A(&b->qval, qv);
        }
        if (rc != MCF_OK) return bail(rc);
        // coefficients, subsets and outputs
        for (int f = 0; f < b->Q; ++f) {
            const int i = b->fused[f];
            const mcf_query& q = b->queries[i];
            d[f].zeta = b->zeta + (size_t)f * MCF_MAX_COEFFS;
            d[f].zf = b->zf + (size_t)f * MCF_MAX_COEFFS;
            if (cudaMemcpyAsync((void*)d[f].zeta, b->coeffs[i].data(), b->coeffs[i].size() * sizeof(double),
                                cudaMemcpyHostToDevice, st) != cudaSuccess)
                return bail(fail(MCF_ERR_CUDA, "coefficient upload failed"));
            if (f == 0) b->zf_host.assign((size_t)b->Q * MCF_MAX_COEFFS, 0.f);
            for (size_t k = 0; k < b->coeffs[i].size(); ++k)
                b->zf_host[(size_t)f * MCF_MAX_COEFFS + k] = (float)b->coeffs[i][k];
            if (f == b->Q - 1 &&
                cudaMemcpyAsync(b->zf, b->zf_host.data(), b->zf_host.size() * sizeof(float), cudaMemcpyHostToDevice,
                                st) != cudaSuccess)
                return bail(fail(MCF_ERR_CUDA, "coefficient upload failed"));
            if (d[f].subset && d[f].n_out > 0) {
                for (int64_t t = 0; t < q.n_nodes && !is_device_ptr(q.nodes); ++t)
                    if (q.nodes[t] < 0 || q.nodes[t] >= q.graph->n)
                        return bail(fail(MCF_ERR_INVALID_ARG, "query " + std::to_string(i) + ": node out of range"));
                if (is_device_ptr(q.nodes)) {
                    if ((rc = check_nodes_on_device(q.nodes, q.n_nodes, q.graph->n, st)) != MCF_OK)
                        return bail(fail(rc, "query " + std::to_string(i) + ": " + get_error()));
                    d[f].nodes = q.nodes;
                } else {
                    int64_t* nd;
                    if ((rc = balloc(b, &nd, q.n_nodes)) != MCF_OK) return bail(rc);
                    cudaMemcpyAsync(nd, q.nodes, q.n_nodes * sizeof(int64_t), cudaMemcpyHostToDevice, st);
                    d[f].nodes = nd;
                }
                // per-column lists of the requested rows, built once: the
                // subset's indices are read when the batch is planned
                SubList sl{};
                rc = build_subset_lists(q.graph, d[f].nodes, q.n_nodes, st, [&](void** p, size_t bytes) {
                    return balloc(b, (char**)p, bytes);
                }, &sl);
                if (rc != MCF_OK) return bail(rc);
                d[f].sub_ptr = sl.ptr;
                d[f].sub_row = sl.row;
            }
            if (is_device_ptr(q.out)) {
                d[f].out = q.out;
            } else {
                double* so;
                if ((rc = balloc(b, &so, d[f].n_out)) != MCF_OK) return bail(rc);
                d[f].out = so;
                b->out_copies.push_back({so, q.out});
                b->out_sizes.push_back(d[f].n_out);
            }
        }
        if (cudaMemcpyAsync(b->desc, d.data(), b->Q * sizeof(BQuery), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(b->qoff, qoff.data(), (b->Q + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(b->rmoff, rmoff.data(), (b->Q + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(b->boff, boff.data(), (b->Q + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return bail(fail(MCF_ERR_CUDA, "descriptor upload failed"));
        if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(MCF_ERR_CUDA, "batch setup failed"));
        if (flags & MCF_BATCH_AUTOTUNE) {
            if ((rc = autotune(b, st)) != MCF_OK) return bail(rc);
        } else {
            b->tune.minb = WALK_MINB;
            b->tune.grab = WALK_GRAB;
        }
        if (flags & MCF_BATCH_CUDA_GRAPH) {
            cudaStream_t cs;
            if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
                return bail(fail(MCF_ERR_CUDA, "capture stream"));
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            mcf_status rr = e == cudaSuccess ? record(b, cs) : MCF_ERR_CUDA;
            cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
            cudaStreamDestroy(cs);
            if (e != cudaSuccess || rr != MCF_OK || e2 != cudaSuccess ||
                cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
                cudaGetLastError();
                return bail(fail(MCF_ERR_CUDA, "CUDA graph capture of the batch failed"));
            }
        }
    }
    *out = b;
    return MCF_OK;
}

mcf_status mcf_batch_run(mcf_batch_t b, void* stream, mcf_stats* stats) {
    set_error("");
    if (!b) return fail(MCF_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    EventGuard event_guard{&e0, &e1};
    if (stats) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
    }
    stamp_kernel<<<1, 1, 0, st>>>(b->stamps);
    if (b->Q > 0) {
        ScopedL2Fetch fetch(L2_FETCH_BYTES);
        if (b->exec) MCF_CUDA_TRY(cudaGraphLaunch(b->exec, st));
        else MCF_TRY(record(b, st));
    }
    if (stats) cudaEventRecord(e1, st);
    int64_t walks = 0, steps = 0;
    uint32_t fl = 0;
    for (size_t c = 0; c < b->out_copies.size(); ++c)
        MCF_CUDA_TRY(cudaMemcpyAsync(b->out_copies[c].second, b->out_copies[c].first, b->out_sizes[c] * sizeof(double),
                                     cudaMemcpyDeviceToHost, st));
    if (b->Q > 0 && stats) {
        unsigned long long h[BC_N];
        MCF_CUDA_TRY(cudaMemcpyAsync(h, b->counters, sizeof(h), cudaMemcpyDeviceToHost, st));
        MCF_CUDA_TRY(cudaStreamSynchronize(st));
        walks += (int64_t)h[BC_WALKS];
        steps += (int64_t)h[BC_STEPS];
        fl |= (uint32_t)h[BC_FLAGS];
    }
    float ms = 0.f;
    if (stats) {
        MCF_CUDA_TRY(cudaEventSynchronize(e1));
        cudaEventElapsedTime(&ms, e0, e1);
    }
    for (int i : b->single) {
        const mcf_query& q = b->queries[i];
        mcf_params p = b->params[i];
        p.stream = stream;
        mcf_stats s1{};
        mcf_status rc;
        switch (q.kind) {
            case MCF_QUERY_ACTION: rc = mcf_action(q.graph, &p, q.v, q.out, stats ? &s1 : nullptr); break;
            case MCF_QUERY_SUBGRAPH_CENTRALITY:
                rc = mcf_subgraph_centrality(q.graph, &p, q.nodes, q.n_nodes, q.out, stats ? &s1 : nullptr);
                break;
            default: rc = mcf_total_communicability(q.graph, &p, q.out, stats ? &s1 : nullptr); break;
        }
        b->qstatus[i] = rc;
        if (rc != MCF_OK && rc != MCF_ERR_ACCURACY_BUDGET) return rc;
        walks += s1.walks;
        steps += s1.walk_steps;
        ms += (float)s1.kernel_ms;
        fl |= s1.flags;
    }
    stamp_kernel<<<1, 1, 0, st>>>(b->stamps + 1);
    MCF_CUDA_TRY(cudaGetLastError());
    MCF_CUDA_TRY(cudaMemcpyAsync(b->window, b->stamps, sizeof(b->window), cudaMemcpyDeviceToHost, st));
    MCF_CUDA_TRY(cudaStreamSynchronize(st));
    if (stats) {
        stats->walks = walks;
        stats->walk_steps = steps;
        stats->kernel_ms = ms;
        stats->flags = fl;
        stats->max_rel_se = 0.0;
        stats->est_rel_err = 0.0;
        stats->replicas = 1;
    }
    for (mcf_status q : b->qstatus)
        if (q == MCF_ERR_ACCURACY_BUDGET)
            return fail(MCF_ERR_ACCURACY_BUDGET, "an accuracy-targeted query stopped at its walk cap; every result "
                                                 "is written");
    return MCF_OK;
}

}  // extern "C"
