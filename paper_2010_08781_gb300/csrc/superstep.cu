// Synchronous vertex-centric supersteps on sm_103a.
//
// One superstep s >= 1 (Section 4.2, Fig. 3) is:
//   exchange  deliver the messages broadcast in superstep s-1 into the one-slot
//             mailboxes (Section 4.3.3), in one of three modes (Section 4.3.2):
//               push-sparse  senders taken from compacted queues (the selection
//                            bypass of Section 4.3.1); the first message to
//                            reach a vertex appends it to the recipient queue
//               push-dense   senders taken from the broadcast bitmap
//               pull         every vertex folds its in-neighbours' broadcasts
//             Push combines with atomicMin (min apps) or atomicAdd (PageRank):
//             the lock-free combiners that Section 4.3.2 leaves as future work.
//   apply     compute() of every recipient (Figs. 9, 10) or of every vertex
//             (PageRank, Fig. 8): read and reset the mailbox, update the value,
//             decide whether to broadcast, vote to halt; plus the frontier
//             statistics of the superstep.
//   select    one warp: halt test (Section 4.2: every vertex halted and no
//             message in flight), frontier features, mode of the next exchange
//             (threshold rule or the learned MLP), per-superstep log.
// PageRank's pull mode fuses exchange and apply: the broadcast values are held
// in two buffers (read s-1, write s), so one kernel per superstep suffices.
//
// Broadcast bitmaps are double-buffered by superstep parity, as are the
// broadcaster queues.
//
// Scheduling uses static degree bins per edge direction: a vertex with degree
// <= t1 is handled by one lane inside a 32-vertex tile, t1 < degree < t2 by a
// whole warp, degree >= t2 in chunks of HCH edges by whole CTAs. Every kernel
// runs the CTA chunks first, then the warp vertices, then the tiles. Edge
// arrays are read as aligned 16-byte blocks, U blocks in flight per thread.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "internal.h"

namespace ipg {

constexpr int U = 4;  // 16-byte blocks loaded per thread before they are consumed

// ----------------------------------------------------------------- helpers
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) {
    const uint32_t s = a + b;
    return s < a ? INF : s;
}
__device__ __forceinline__ uint4 ld4(const uint32_t* p, uint32_t blk) {
    return __ldg(reinterpret_cast<const uint4*>(p) + blk);
}
__device__ __forceinline__ uint32_t qa(const uint4& q, int j) {
    return j == 0 ? q.x : (j == 1 ? q.y : (j == 2 ? q.z : q.w));
}
__device__ __forceinline__ bool bit_of(const uint32_t* bm, uint32_t v) {
    return (__ldg(bm + (v >> 5)) >> (v & 31u)) & 1u;
}
__device__ __forceinline__ uint32_t global_warp() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ uint32_t num_warps() { return (gridDim.x * blockDim.x) >> 5; }
__device__ __forceinline__ const uint32_t* bc_of(const Params& P, uint32_t s) { return (s & 1) ? P.bcast1 : P.bcast0; }
__device__ __forceinline__ uint32_t* bc_mut(const Params& P, uint32_t s) { return (s & 1) ? P.bcast1 : P.bcast0; }

// All 32 lanes call; lanes with pred append v to q (one atomic per warp).
__device__ __forceinline__ void warp_append(bool pred, uint32_t v, uint32_t* q, unsigned int* len) {
    const uint32_t m = __ballot_sync(FULL, pred);
    if (!m) return;
    const uint32_t leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane_id() == leader) base = atomicAdd(len, (unsigned int)__popc(m));
    base = __shfl_sync(FULL, base, leader);
    if (pred) q[base + __popc(m & lanemask_lt())] = v;
}

// All 32 lanes call; each lane appends its vertex's HCH-edge chunks {v, c}.
__device__ __forceinline__ void warp_append_chunks(uint32_t nch, uint32_t v, uint2* q, unsigned int* len) {
    uint32_t inc = nch;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane_id() >= (uint32_t)o) inc += y;
    }
    const uint32_t total = __shfl_sync(FULL, inc, 31);
    if (!total) return;
    uint32_t base = 0;
    if (lane_id() == 31) base = atomicAdd(len, total);
    base = __shfl_sync(FULL, base, 31) + inc - nch;
    for (uint32_t c = 0; c < nch; ++c) q[base + c] = make_uint2(v, c);
}

// Error-free transformation (Knuth's TwoSum): s + err == s_old + x exactly.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
    const float t = s + x;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (x - bp);
    s = t;
    c += err;
}

__device__ __forceinline__ void warp_two_sum(float& s, float& c) {
    for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_down_sync(FULL, s, o), oc = __shfl_down_sync(FULL, c, o);
        two_sum_acc(s, c, os);
        c += oc;
    }
}

struct Stats {
    unsigned int act, bc, maxd;
    unsigned long long msgs;
};

// Block-wide reduction of the superstep statistics, one atomic per field per CTA.
__device__ void flush_stats(Stats st, DevCtl* ctl) {
    __shared__ Stats sh[BLOCK / 32];
    for (int o = 16; o > 0; o >>= 1) {
        st.act += __shfl_down_sync(FULL, st.act, o);
        st.bc += __shfl_down_sync(FULL, st.bc, o);
        st.msgs += __shfl_down_sync(FULL, st.msgs, o);
        st.maxd = max(st.maxd, __shfl_down_sync(FULL, st.maxd, o));
    }
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0) sh[w] = st;
    __syncthreads();
    if (w == 0) {
        Stats t = lane_id() < blockDim.x / 32 ? sh[lane_id()] : Stats{0, 0, 0, 0};
        for (int o = 16; o > 0; o >>= 1) {
            t.act += __shfl_down_sync(FULL, t.act, o);
            t.bc += __shfl_down_sync(FULL, t.bc, o);
            t.msgs += __shfl_down_sync(FULL, t.msgs, o);
            t.maxd = max(t.maxd, __shfl_down_sync(FULL, t.maxd, o));
        }
        if (lane_id() == 0) {
            if (t.act) atomicAdd(&ctl->n_active, t.act);
            if (t.bc) atomicAdd(&ctl->n_bcast, t.bc);
            if (t.msgs) atomicAdd(&ctl->msgs, t.msgs);
            if (t.maxd) atomicMax(&ctl->max_deg, t.maxd);
        }
    }
}

// Appends a broadcaster to the queue of its degree bin (all 32 lanes call).
__device__ __forceinline__ void queue_broadcaster(const Params& P, int par, bool b, uint32_t v, uint32_t deg) {
    unsigned int* len = P.ctl->q_len[par];
    warp_append(b && deg <= P.t1, v, P.q[par][0], &len[0]);
    warp_append(b && deg > P.t1 && deg < P.t2, v, P.q[par][1], &len[1]);
    warp_append_chunks(b && deg >= P.t2 ? (deg + HCH - 1) / HCH : 0u, v, P.hq[par], &len[2]);
}

// =========================================================== superstep 0
// Hashmin (Fig. 9): value = id, every vertex broadcasts. SSSP (Fig. 10): the
// source takes 0 and broadcasts, every other vertex INF.
__global__ void k_init_min(Params P) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const bool hm = P.app == APP_HM;
    for (uint32_t v = tid; v < P.V; v += nth) {
        const uint32_t x = hm ? (P.orig ? P.orig[v] : v) : (v == P.source ? 0u : INF);
        P.value[v] = x;
        P.outbox[v] = x;  // every initial value below INF is broadcast
        P.mbox[v] = INF;
        if (P.last_send) P.last_send[v] = (x != INF && P.csr_off[v + 1] > P.csr_off[v]) ? 1u : 0u;
    }
    for (uint32_t w = tid; w < P.W; w += nth) {
        P.recv[w] = 0;
        uint32_t b = 0;
        if (hm) {
            const uint64_t lo = (uint64_t)w * 32;
            if (lo + 32 <= P.V)
                b = FULL;
            else if (lo < P.V)
                b = (1u << (P.V - lo)) - 1u;
        } else if (w == (P.source >> 5)) {
            b = 1u << (P.source & 31u);
        }
        P.bcast0[w] = b;
    }
    if (tid == 0) {
        DevCtl* c = P.ctl;
        c->superstep = 0;
        c->mode_used = 255;
        c->done = 0;
        c->err = 0;
        c->prev_bcast = 0;
        c->t_prev = globaltimer();
        c->n_active = P.V;
        c->rq_len = 0;
        for (int p = 0; p < 2; ++p)
            for (int k = 0; k < 3; ++k) c->q_len[p][k] = 0;
        if (hm) {
            c->n_bcast = P.V;
            c->msgs = P.E;
            c->max_deg = P.max_out_deg;
            c->q_valid = 0;
        } else {
            const uint32_t d = P.out_deg_src;
            c->n_bcast = 1;
            c->msgs = d;
            c->max_deg = d;
            if (d <= P.t1) {
                P.q[0][0][0] = P.source;
                c->q_len[0][0] = 1;
            } else if (d < P.t2) {
                P.q[0][1][0] = P.source;
                c->q_len[0][1] = 1;
            } else {
                const uint32_t nch = (d + HCH - 1) / HCH;
                for (uint32_t k = 0; k < nch; ++k) P.hq[0][k] = make_uint2(P.source, k);
                c->q_len[0][2] = nch;
            }
            c->q_valid = 1;
        }
    }
}

// PageRank superstep 0 (Fig. 8): value = 1/N, broadcast value / out-degree.
__global__ void k_pr_init(Params P) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const float r0 = 1.0f / (float)P.V;
    for (uint32_t v = tid; v < P.V; v += nth) {
        P.rank[v] = r0;
        P.contrib0[v] = P.T > 0 ? r0 * P.inv_outdeg[v] : 0.0f;
        P.mboxf[v] = 0.0f;
    }
    if (P.pb.on && tid == 0) P.pb.ctr[0] = P.pb.ctr[1] = 0;
    if (tid == 0) {
        DevCtl* c = P.ctl;
        c->superstep = 0;
        c->mode_used = 255;
        c->done = 0;
        c->err = 0;
        c->prev_bcast = 0;
        c->pr_stale = 0;
        c->pr_delta = 0.0;
        c->t_prev = globaltimer();
    }
}

// ============================================================ push (min apps)
template <int APP>
__device__ __forceinline__ uint32_t edge_msg(uint32_t val, const uint4& qw, int j) {
    if (APP == APP_HM) return val;
    return sat_add(val, qa(qw, j));
}

// One message into v's mailbox (min combiner) and v's recipient bit. With
// SPARSE, the first message to reach v appends v to the recipient queue; all
// 32 lanes must call.
template <bool SPARSE>
__device__ __forceinline__ void push_edge(const Params& P, bool live, uint32_t v, uint32_t msg) {
    bool first = false;
    if (live) {
        if (msg < __ldcg(P.mbox + v)) atomicMin(P.mbox + v, msg);
        const uint32_t bit = 1u << (v & 31u);
        uint32_t* rw = P.recv + (v >> 5);
        if (!(__ldcg(rw) & bit)) {
            if (SPARSE)
                first = !(atomicOr(rw, bit) & bit);
            else
                atomicOr(rw, bit);
        }
    }
    if (SPARSE) warp_append(first, v, P.rq, &P.ctl->rq_len);
}

// Pushes the edges [b, e) of one sender with value val. The thread at position
// pos of a group of `stride` threads takes 16-byte blocks pos, pos+stride, ...
// in `trips` iterations of U blocks; with SPARSE, trips must be equal over the warp.
template <int APP, bool SPARSE>
__device__ __forceinline__ void push_range(const Params& P, uint32_t val, uint32_t b, uint32_t e, uint32_t pos,
                                           uint32_t stride, uint32_t trips) {
    const uint32_t bs = b >> 2, be = (e + 3) >> 2;
    for (uint32_t t = 0; t < trips; ++t) {
        uint4 qc[U], qw[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t blk = bs + (t * U + u) * stride + pos;
            const bool ok = blk < be;
            qc[u] = ok ? ld4(P.csr_col, blk) : make_uint4(0, 0, 0, 0);
            qw[u] = (APP == APP_SSSP && P.csr_w && ok) ? ld4(P.csr_w, blk) : make_uint4(1, 1, 1, 1);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t blk = bs + (t * U + u) * stride + pos;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t ei = blk * 4 + j;
                const bool live = blk < be && ei >= b && ei < e;
                push_edge<SPARSE>(P, live, qa(qc[u], j), edge_msg<APP>(val, qw[u], j));
            }
        }
    }
}

__device__ __forceinline__ uint32_t trips_of(uint32_t b, uint32_t e, uint32_t stride) {
    const uint32_t nb = e > b ? ((e + 3) >> 2) - (b >> 2) : 0u;
    return (nb + stride * U - 1) / (stride * U);
}

template <int APP, bool SPARSE>
__global__ void __launch_bounds__(BLOCK) k_push(Params P) {
    const uint32_t sp = P.ctl->superstep - 1;  // deliver the broadcasts of superstep sp
    const int par = sp & 1;
    if (SPARSE) {
        // the bitmap of the superstep being computed is built by atomicOr in apply
        uint32_t* nb = bc_mut(P, sp + 1);
        for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < P.W; w += gridDim.x * blockDim.x) nb[w] = 0;
        // heavy senders: one CTA per HCH-edge chunk
        const uint32_t nh = P.ctl->q_len[par][2];
        for (uint32_t k = blockIdx.x; k < nh; k += gridDim.x) {
            const uint2 h = P.hq[par][k];
            const uint32_t u = h.x, e0 = P.csr_off[u + 1];
            const uint32_t b = P.csr_off[u] + h.y * HCH, e = min(e0, b + HCH);
            if (threadIdx.x == 0 && h.y == 0) P.outbox[u] = INF;  // the broadcast slot is consumed
            push_range<APP, SPARSE>(P, P.value[u], b, e, threadIdx.x, blockDim.x, trips_of(b, e, blockDim.x));
        }
        // medium senders: one warp each
        const uint32_t nm = P.ctl->q_len[par][1];
        const uint32_t* qm = P.q[par][1];
        for (uint32_t i = global_warp(); i < nm; i += num_warps()) {
            const uint32_t u = qm[i];
            const uint32_t b = P.csr_off[u], e = P.csr_off[u + 1];
            if (lane_id() == 0) P.outbox[u] = INF;
            push_range<APP, SPARSE>(P, P.value[u], b, e, lane_id(), 32, trips_of(b, e, 32));
        }
        // small senders: one lane each
        const uint32_t ns = P.ctl->q_len[par][0];
        const uint32_t* qs = P.q[par][0];
        for (uint32_t base = global_warp() * 32; base < ns; base += num_warps() * 32) {
            const uint32_t i = base + lane_id();
            uint32_t b = 0, e = 0, val = 0;
            if (i < ns) {
                const uint32_t u = qs[i];
                b = P.csr_off[u];
                e = P.csr_off[u + 1];
                val = P.value[u];
                P.outbox[u] = INF;
            }
            const uint32_t trips = __reduce_max_sync(FULL, trips_of(b, e, 1));
            push_range<APP, SPARSE>(P, val, b, e, 0, 1, trips);
        }
    } else {
        const uint32_t* bc = bc_of(P, sp);
        const Bins& B = P.bout;
        for (uint32_t k = blockIdx.x; k < B.n_hchunk; k += gridDim.x) {
            const uint4 ch = B.hchunk[k];
            if (bit_of(bc, ch.x))
                push_range<APP, SPARSE>(P, P.value[ch.x], ch.y, ch.z, threadIdx.x, blockDim.x,
                                        trips_of(ch.y, ch.z, blockDim.x));
        }
        for (uint32_t i = global_warp(); i < B.n_med; i += num_warps()) {
            const uint32_t u = B.med[i];
            if (bit_of(bc, u)) {
                const uint32_t b = P.csr_off[u], e = P.csr_off[u + 1];
                push_range<APP, SPARSE>(P, P.value[u], b, e, lane_id(), 32, trips_of(b, e, 32));
            }
        }
        const uint32_t tiles = (P.V + 31) / 32;
        for (uint32_t t = global_warp(); t < tiles; t += num_warps()) {
            const uint32_t word = __ldg(bc + t);
            if (!word) continue;
            const uint32_t u = t * 32 + lane_id();
            uint32_t b = 0, e = 0;
            if ((word >> lane_id()) & 1u) {
                b = P.csr_off[u];
                e = P.csr_off[u + 1];
                if (e - b > P.t1) e = b;  // the warp and CTA bins push these
            }
            if (e > b) push_range<APP, SPARSE>(P, P.value[u], b, e, 0, 1, trips_of(b, e, 1));
        }
    }
}

// Broadcast bitmap of the last completed superstep -> its binned broadcaster
// queues, unless the queues already hold it.
__global__ void __launch_bounds__(BLOCK) k_compact(Params P) {
    if (P.ctl->q_valid) return;
    const uint32_t sp = P.ctl->superstep - 1;
    const int par = sp & 1;
    const uint32_t* bc = bc_of(P, sp);
    const uint32_t tiles = (P.V + 31) / 32;
    for (uint32_t t = global_warp(); t < tiles; t += num_warps()) {
        const uint32_t word = __ldg(bc + t);
        if (!word) continue;
        const uint32_t u = t * 32 + lane_id();
        const bool act = (word >> lane_id()) & 1u;
        const uint32_t deg = act ? P.csr_off[u + 1] - P.csr_off[u] : 0;
        queue_broadcaster(P, par, act, u, deg);
    }
}

// ============================================================ pull (min apps)
// Folds the in-edges [b, e) into (m, any) reading the broadcast slots
// (outbox[u] = value of u if u broadcast in the last superstep, else INF):
// the thread at position pos of a group of `stride` threads takes blocks
// pos, pos+stride, ...
//
// EARLY (unit-weight SSSP, i.e. Fig. 10 exactly): under synchronous supersteps
// every vertex that broadcast in superstep s-1 holds the value s-1 (the
// broadcasters of superstep k are the vertices first reached in k), so every
// message into superstep s is s and the first broadcasting in-neighbour found
// decides both the combined message and whether the vertex is a recipient: the
// scan stops there (the direction-optimising pull). A group of 32 or more
// threads runs equal trip counts and stops as a whole warp.
template <int APP, bool EARLY = false>
__device__ __forceinline__ void pull_range(const Params& P, uint32_t b, uint32_t e, uint32_t pos, uint32_t stride,
                                           uint32_t& m, bool& any) {
    const uint32_t bs = b >> 2, be = (e + 3) >> 2;
    const uint32_t span = stride * U;
    const uint32_t trips = EARLY && be > bs ? (be - bs + span - 1) / span : 0u;
    uint32_t t = 0;
    for (uint32_t g0 = bs + pos; EARLY ? t < trips : g0 < be; g0 += span, ++t) {
        uint4 qr[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t blk = g0 + u * stride;
            qr[u] = blk < be ? ld4(P.csc_row, blk) : make_uint4(0, 0, 0, 0);
        }
        uint32_t x[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t blk = g0 + u * stride;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t ei = blk * 4 + j;
                x[u][j] = (blk < be && ei >= b && ei < e) ? __ldg(P.outbox + qa(qr[u], j)) : INF;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool h = (x[u][0] & x[u][1] & x[u][2] & x[u][3]) != INF;
            if (!h) continue;
            any = true;
            uint4 qw = make_uint4(1, 1, 1, 1);
            if (APP == APP_SSSP && P.csc_w) qw = ld4(P.csc_w, g0 + u * stride);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (x[u][j] != INF) m = min(m, edge_msg<APP>(x[u][j], qw, j));
        }
        if (EARLY && (stride >= 32 ? __any_sync(FULL, any) : any)) break;
    }
}

template <int APP, bool EARLY = false>
__global__ void __launch_bounds__(BLOCK) k_pull(Params P) {
    __shared__ uint32_t sm[BLOCK / 32];
    __shared__ uint32_t sa[BLOCK / 32];
    const Bins& B = P.bin;
    for (uint32_t k = blockIdx.x; k < B.n_hchunk; k += gridDim.x) {
        const uint4 ch = B.hchunk[k];
        uint32_t m = INF;
        bool any = false;
        pull_range<APP, EARLY>(P, ch.y, ch.z, threadIdx.x, blockDim.x, m, any);
        m = __reduce_min_sync(FULL, m);
        const uint32_t a = __any_sync(FULL, any);
        if (lane_id() == 0) {
            sm[threadIdx.x >> 5] = m;
            sa[threadIdx.x >> 5] = a;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t mm = INF, aa = 0;
            for (uint32_t w = 0; w < blockDim.x / 32; ++w) {
                mm = min(mm, sm[w]);
                aa |= sa[w];
            }
            if (aa) {
                atomicMin(P.mbox + ch.x, mm);
                atomicOr(P.recv + (ch.x >> 5), 1u << (ch.x & 31u));
            }
        }
        __syncthreads();
    }
    for (uint32_t i = global_warp(); i < B.n_med; i += num_warps()) {
        const uint32_t v = B.med[i];
        uint32_t m = INF;
        bool any = false;
        pull_range<APP, EARLY>(P, P.csc_off[v], P.csc_off[v + 1], lane_id(), 32, m, any);
        m = __reduce_min_sync(FULL, m);
        any = __any_sync(FULL, any);
        if (lane_id() == 0 && any) {
            P.mbox[v] = m;
            atomicOr(P.recv + (v >> 5), 1u << (v & 31u));
        }
    }
    const uint32_t tiles = (P.V + 31) / 32;
    for (uint32_t t = global_warp(); t < tiles; t += num_warps()) {
        const uint32_t v = t * 32 + lane_id();
        uint32_t m = INF;
        bool any = false;
        if (v < P.V) {
            const uint32_t b = P.csc_off[v], e = P.csc_off[v + 1];
            if (e - b <= P.t1) pull_range<APP, EARLY>(P, b, e, 0, 1, m, any);
        }
        if (any) P.mbox[v] = m;
        const uint32_t bits = __ballot_sync(FULL, any);
        if (lane_id() == 0 && bits) atomicOr(P.recv + t, bits);
    }
}

// ============================================================ apply (min apps)
// compute() of Figs. 9 and 10 for one recipient: m is the combined message.
__device__ __forceinline__ bool apply_vertex(const Params& P, uint32_t v, uint32_t& deg) {
    const uint32_t m = P.mbox[v];
    P.mbox[v] = INF;
    const uint32_t val = P.value[v];
    deg = 0;
    if (m < val) {
        P.value[v] = m;
        deg = P.csr_off[v + 1] - P.csr_off[v];
        if (P.last_send && deg) P.last_send[v] = P.ctl->superstep + 1;
        return true;  // broadcast the new value
    }
    return false;
}

// Recipients found in the recv bitmap (after pull or push-dense): one warp per
// 32-vertex word, AW words in flight per warp. Writes every word of this
// superstep's broadcast bitmap and every broadcast slot.
constexpr int AW = 4;
__global__ void __launch_bounds__(BLOCK) k_apply_bitmap(Params P) {
    Stats st{0, 0, 0, 0};
    uint32_t* bc = bc_mut(P, P.ctl->superstep);
    const uint32_t words = (P.V + 31) / 32;
    const uint32_t nw = num_warps(), lane = lane_id();
    for (uint32_t w0 = global_warp(); w0 < words; w0 += AW * nw) {
        uint32_t rw[AW], m[AW], val[AW];
#pragma unroll
        for (int k = 0; k < AW; ++k) {
            const uint32_t w = w0 + k * nw;
            rw[k] = w < words ? P.recv[w] : 0u;
        }
#pragma unroll
        for (int k = 0; k < AW; ++k) {
            const uint32_t v = (w0 + k * nw) * 32 + lane;
            const bool r = (rw[k] >> lane) & 1u;
            m[k] = r ? P.mbox[v] : INF;
            val[k] = r ? P.value[v] : 0u;
        }
        uint32_t deg[AW];
#pragma unroll
        for (int k = 0; k < AW; ++k) {
            const uint32_t w = w0 + k * nw;
            const uint32_t v = w * 32 + lane;
            const bool r = (rw[k] >> lane) & 1u;
            const bool b = m[k] < val[k];  // compute() of Figs. 9 / 10: improve and broadcast
            if (r) P.mbox[v] = INF;
            if (b) P.value[v] = m[k];
            if (w < words && v < P.V) P.outbox[v] = b ? m[k] : INF;
            deg[k] = b ? 1u : 0u;
        }
#pragma unroll
        for (int k = 0; k < AW; ++k) {
            const uint32_t w = w0 + k * nw;
            const uint32_t v = w * 32 + lane;
            const bool b = deg[k] != 0;
            deg[k] = b ? P.csr_off[v + 1] - P.csr_off[v] : 0u;
            if (P.last_send && deg[k]) P.last_send[v] = P.ctl->superstep + 1;
            const uint32_t bb = __ballot_sync(FULL, b);
            if (lane == 0 && w < words) {
                bc[w] = bb;
                if (rw[k]) P.recv[w] = 0;
                st.act += __popc(rw[k]);
            }
            st.bc += b;
            st.msgs += deg[k];
            st.maxd = max(st.maxd, deg[k]);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) P.ctl->q_valid = 0;
    flush_stats(st, P.ctl);
}

// Recipients taken from the recipient queue (after push-sparse); broadcasters
// go to this superstep's binned queues and (cleared) bitmap.
__global__ void __launch_bounds__(BLOCK) k_apply_queue(Params P) {
    Stats st{0, 0, 0, 0};
    const uint32_t s = P.ctl->superstep;
    const int par = s & 1;
    uint32_t* bc = bc_mut(P, s);
    const uint32_t n = P.ctl->rq_len;
    for (uint32_t base = global_warp() * 32; base < n; base += num_warps() * 32) {
        const uint32_t i = base + lane_id();
        const bool valid = i < n;
        uint32_t v = 0, deg = 0;
        bool b = false;
        if (valid) {
            v = P.rq[i];
            P.recv[v >> 5] = 0;  // every bit of this word belongs to a queued recipient
            b = apply_vertex(P, v, deg);
            if (b) {
                atomicOr(bc + (v >> 5), 1u << (v & 31u));
                P.outbox[v] = P.value[v];
            }
        }
        queue_broadcaster(P, par, b, v, deg);
        st.act += valid;
        st.bc += b;
        st.msgs += deg;
        st.maxd = max(st.maxd, deg);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) P.ctl->q_valid = 1;
    flush_stats(st, P.ctl);
}

// ================================================================ PageRank
// Compensated sum of cur[u] over the in-edges [b, e); thread pos of a group of
// `stride` threads takes blocks pos, pos+stride, ...
__device__ __forceinline__ void pr_gather(const uint32_t* row, const float* cur, uint32_t b, uint32_t e, uint32_t pos,
                                          uint32_t stride, float& s, float& c) {
    const uint32_t bs = b >> 2, be = (e + 3) >> 2;
    for (uint32_t g0 = bs + pos; g0 < be; g0 += stride * U) {
        uint4 qr[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t blk = g0 + u * stride;
            qr[u] = blk < be ? ld4(row, blk) : make_uint4(0, 0, 0, 0);
        }
        float x[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t blk = g0 + u * stride;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t ei = blk * 4 + j;
                x[u][j] = (blk < be && ei >= b && ei < e) ? __ldg(cur + qa(qr[u], j)) : 0.0f;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < 4; ++j) two_sum_acc(s, c, x[u][j]);
    }
}

// Fused exchange + compute for PageRank pull: sum of in-neighbours' broadcasts.
// A heavy vertex's chunks leave compensated partials; the CTA that completes
// the last chunk adds them in chunk order and finishes the vertex.
__global__ void __launch_bounds__(BLOCK) k_pr_pull(Params P) {
    __shared__ float ss[BLOCK / 32], sc[BLOCK / 32];
    const uint32_t s = P.ctl->superstep;  // the superstep being computed
    const float* cur = (s & 1) ? P.contrib0 : P.contrib1;
    float* nxt = (s & 1) ? P.contrib1 : P.contrib0;
    const Bins& B = P.bin;
    float dacc = 0.f;  // L1 rank change of the vertices this thread finishes (tolerance runs)
    for (uint32_t k = blockIdx.x; k < B.n_hchunk; k += gridDim.x) {
        const uint4 ch = B.hchunk[k];
        float a = 0.f, c = 0.f;
        pr_gather(P.csc_row, cur, ch.y, ch.z, threadIdx.x, blockDim.x, a, c);
        warp_two_sum(a, c);
        if (lane_id() == 0) {
            ss[threadIdx.x >> 5] = a;
            sc[threadIdx.x >> 5] = c;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float ta = ss[0], tc = sc[0];
            for (uint32_t w = 1; w < blockDim.x / 32; ++w) {
                two_sum_acc(ta, tc, ss[w]);
                tc += sc[w];
            }
            B.hpart[k] = make_float2(ta, tc);
            __threadfence();
            const uint2 hv = B.hvert[ch.w];
            if (atomicAdd(B.hcnt + ch.w, 1u) == hv.y - 1) {
                __threadfence();
                float fa = 0.f, fc = 0.f;
                for (uint32_t q = 0; q < hv.y; ++q) {
                    const float2 pq = __ldcg(B.hpart + hv.x + q);
                    two_sum_acc(fa, fc, pq.x);
                    fc += pq.y;
                }
                pr_finish(P, ch.x, fa + fc, s, nxt, dacc);
                B.hcnt[ch.w] = 0;
            }
        }
        __syncthreads();
    }
    for (uint32_t i = global_warp(); i < B.n_med; i += num_warps()) {
        const uint32_t v = B.med[i];
        float a = 0.f, c = 0.f;
        pr_gather(P.csc_row, cur, P.csc_off[v], P.csc_off[v + 1], lane_id(), 32, a, c);
        warp_two_sum(a, c);
        if (lane_id() == 0) pr_finish(P, v, a + c, s, nxt, dacc);
    }
    const uint32_t tiles = (P.V + 31) / 32;
    for (uint32_t t = global_warp(); t < tiles; t += num_warps()) {
        const uint32_t v = t * 32 + lane_id();
        if (v < P.V) {
            const uint32_t b = P.csc_off[v], e = P.csc_off[v + 1];
            if (e - b <= P.t1) {
                float a = 0.f, c = 0.f;
                pr_gather(P.csc_row, cur, b, e, 0, 1, a, c);
                pr_finish(P, v, a + c, s, nxt, dacc);
            }
        }
    }
    flush_delta(P, dacc);
}

// PageRank push: every vertex adds value/out-degree into its out-neighbours' mailboxes.
__device__ __forceinline__ void pr_scatter(const Params& P, float x, uint32_t b, uint32_t e, uint32_t pos,
                                           uint32_t stride) {
    const uint32_t bs = b >> 2, be = (e + 3) >> 2;
    for (uint32_t g0 = bs + pos; g0 < be; g0 += stride * U) {
        uint4 qc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t blk = g0 + u * stride;
            qc[u] = blk < be ? ld4(P.csr_col, blk) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t blk = g0 + u * stride;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t ei = blk * 4 + j;
                if (blk < be && ei >= b && ei < e) atomicAdd(P.mboxf + qa(qc[u], j), x);
            }
        }
    }
}

// After a blocked-pull superstep (which stores ranks only), the broadcasts of
// that superstep for the push and gather exchanges: rank / out-degree while it
// was < T. Nothing when the last superstep wrote them itself.
__global__ void __launch_bounds__(BLOCK) k_pr_contrib(Params P) {
    if (!P.ctl->pr_stale) return;
    const uint32_t sp = P.ctl->superstep - 1;
    float* cur = (sp & 1) ? P.contrib1 : P.contrib0;
    const bool sent = sp < P.T;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < P.V; v += gridDim.x * blockDim.x)
        cur[v] = sent ? P.rank[v] * P.inv_outdeg[v] : 0.0f;  // as pr_finish
}

// Clears the flag of k_pr_contrib once every CTA has read it.
__global__ void k_pr_contrib_done(Params P) { P.ctl->pr_stale = 0; }

__global__ void __launch_bounds__(BLOCK) k_pr_push(Params P) {
    const uint32_t sp = P.ctl->superstep - 1;  // deliver the broadcasts of superstep sp
    const float* cur = (sp & 1) ? P.contrib1 : P.contrib0;
    const Bins& B = P.bout;
    for (uint32_t k = blockIdx.x; k < B.n_hchunk; k += gridDim.x) {
        const uint4 ch = B.hchunk[k];
        pr_scatter(P, cur[ch.x], ch.y, ch.z, threadIdx.x, blockDim.x);
    }
    for (uint32_t i = global_warp(); i < B.n_med; i += num_warps()) {
        const uint32_t u = B.med[i];
        pr_scatter(P, cur[u], P.csr_off[u], P.csr_off[u + 1], lane_id(), 32);
    }
    const uint32_t tiles = (P.V + 31) / 32;
    for (uint32_t t = global_warp(); t < tiles; t += num_warps()) {
        const uint32_t u = t * 32 + lane_id();
        if (u < P.V) {
            const uint32_t b = P.csr_off[u], e = P.csr_off[u + 1];
            if (e - b <= P.t1) pr_scatter(P, cur[u], b, e, 0, 1);
        }
    }
}

__global__ void __launch_bounds__(BLOCK) k_pr_apply(Params P) {
    const uint32_t s = P.ctl->superstep;  // the superstep being computed
    float* nxt = (s & 1) ? P.contrib1 : P.contrib0;
    float dacc = 0.f;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < P.V; v += gridDim.x * blockDim.x) {
        const float sum = P.mboxf[v];
        P.mboxf[v] = 0.0f;
        pr_finish(P, v, sum, s, nxt, dacc);
    }
    flush_delta(P, dacc);
}

// ================================================================ selector
__device__ __forceinline__ float bf16f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// One warp: 8 -> 32 -> 32 -> 3 MLP, BF16 weights, FP32 accumulation.
__device__ int mlp_mode(const SelectorDev* S, const float* f) {
    const uint32_t j = lane_id();
    float xn[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) xn[i] = (f[i] - S->mu[i]) / S->sd[i];
    float h1 = S->b1[j];
#pragma unroll
    for (int i = 0; i < 8; ++i) h1 = fmaf(bf16f(S->W1[j * 8 + i]), xn[i], h1);
    h1 = fmaxf(h1, 0.f);
    float h2 = S->b2[j];
    for (int k = 0; k < 32; ++k) h2 = fmaf(bf16f(S->W2[j * 32 + k]), __shfl_sync(FULL, h1, k), h2);
    h2 = fmaxf(h2, 0.f);
    float z[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        float p = bf16f(S->W3[m * 32 + j]) * h2;
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(FULL, p, o);
        z[m] = p + S->b3[m];
    }
    int best = 0;
    if (z[1] > z[best]) best = 1;
    if (z[2] > z[best]) best = 2;
    return best;
}

// Restarts the clock of the "last superstep time" feature (label collection:
// only the final, kept trial of a superstep is timed into the feature).
__global__ void k_stamp(DevCtl* c) { c->t_prev = globaltimer(); }

__global__ void k_select(Params P) {
    DevCtl* c = P.ctl;
    const uint32_t s = c->superstep;
    uint32_t act, bc, maxd;
    unsigned long long msgs;
    if (P.app == APP_PR) {
        const bool b = s < P.T;
        act = P.V;
        bc = b ? P.V : 0;
        msgs = b ? P.E : 0;
        maxd = b ? P.max_out_deg : 0;
    } else {
        act = c->n_active;
        bc = c->n_bcast;
        msgs = c->msgs;
        maxd = c->max_deg;
    }
    const uint64_t now = globaltimer();
    const float dt = s == 0 ? 0.f : (float)(now - c->t_prev);
    float f[N_FEATURES];
    f[0] = log1pf((float)bc);
    f[1] = log1pf((float)msgs);
    f[2] = log1pf(bc ? (float)((double)msgs / bc) : 0.f);
    f[3] = log1pf((float)maxd);
    f[4] = (float)bc / (float)P.V;
    f[5] = log1pf(dt);
    f[6] = P.E ? (float)((double)msgs / (double)P.E) : 0.f;
    f[7] = logf(((float)bc + 1.f) / ((float)c->prev_bcast + 1.f));
    uint32_t done;
    const double pr_delta = P.app == APP_PR ? c->pr_delta : 0.0;
    if (P.app == APP_PR)  // T updates, or (PageRank to convergence) a superstep that changed the ranks
        done = (s >= P.T || (P.pr_tol > 0.f && s >= 1 && pr_delta < (double)P.pr_tol)) ? 1u : 0u;  // by < tol in L1
    else
        done = msgs == 0 ? 1u : 0u;
    if (!done && s + 1 >= P.max_supersteps) done = 2;
    int mode;
    switch (P.policy) {
        case IP_POLICY_FORCED: mode = P.forced_mode; break;
        case IP_POLICY_SEQUENCE: mode = P.seq[s % P.seq_len]; break;
        case IP_POLICY_MLP: mode = mlp_mode(P.sel, f); break;
        default:
            mode = f[6] < P.thr_sparse ? IP_MODE_PUSH_SPARSE : (f[6] >= P.thr_pull ? IP_MODE_PULL : IP_MODE_PUSH_DENSE);
    }
    if (P.app == APP_PR && mode == IP_MODE_PUSH_SPARSE) mode = IP_MODE_PUSH_DENSE;  // every vertex broadcasts
    __syncwarp();
    if (threadIdx.x == 0) {
        if (s < P.log_cap) {
            LogRec r;
            r.mode = c->mode_used;
            r.active = act;
            r.bcast = bc;
            r.max_deg = maxd;
            r.msgs = msgs;
            for (int i = 0; i < N_FEATURES; ++i) r.feat[i] = f[i];
            r.pr_delta = (float)pr_delta;
            P.log[s] = r;
        }
        c->mode = (unsigned)mode;
        c->done = done;
        c->prev_bcast = bc;
        c->t_prev = now;
        if (!done) {
            const uint32_t s1 = s + 1;
            c->superstep = s1;
            c->mode_used = (unsigned)mode;
            c->n_active = 0;
            c->n_bcast = 0;
            c->msgs = 0;
            c->max_deg = 0;
            c->rq_len = 0;
            c->pr_delta = 0.0;
            for (int k = 0; k < 3; ++k) c->q_len[s1 & 1][k] = 0;
        }
        if (P.use_graph) {
            cudaGraphSetConditional(P.h_switch, (unsigned)mode);
            cudaGraphSetConditional(P.h_while, done ? 0u : 1u);
        }
    }
}

// ================================================================ host side
namespace {

int grid_of(const ip_graph* g, const void* fn) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, BLOCK, 0) != cudaSuccess || occ < 1) {
        (void)cudaGetLastError();
        occ = 2;
    }
    return g->num_sms * occ;
}

enum { G_PR_PULL, G_PR_PUSH, G_PUSH_HM_S, G_PUSH_SSSP_S, G_PUSH_HM_D, G_PUSH_SSSP_D, G_PULL_HM, G_PULL_SSSP, G_MISC,
       G_PULL_BFS, G_COUNT };

// Grid sizes (resident CTAs per SM x SMs), queried once per handle, outside any capture.
void compute_grids(ip_graph* g) {
    if (g->grids_ready) return;
    const void* fns[G_COUNT] = {(const void*)k_pr_pull, (const void*)k_pr_push, (const void*)k_push<APP_HM, true>,
                                (const void*)k_push<APP_SSSP, true>, (const void*)k_push<APP_HM, false>,
                                (const void*)k_push<APP_SSSP, false>, (const void*)k_pull<APP_HM>,
                                (const void*)k_pull<APP_SSSP>, (const void*)k_apply_bitmap,
                                (const void*)k_pull<APP_SSSP, true>};
    for (int i = 0; i < G_COUNT; ++i) g->grid[i] = grid_of(g, fns[i]);
    g->grids_ready = true;
}

// Exchange + apply of one superstep in the given mode. With ev (4 events), the
// boundaries compaction | exchange | apply are recorded on st: ev[0] before the
// compaction, ev[1] before the exchange, ev[2] before the apply, ev[3] after it.
int launch_superstep(const ip_graph* g, const Params& P, int mode, cudaStream_t st, cudaEvent_t* ev = nullptr) {
    const int* G = g->grid;
    auto mark = [&](int i) {
        if (ev) cudaEventRecord(ev[i], st);
    };
    mark(0);
    if (P.app == APP_PR) {
        const bool blocked = mode == IP_MODE_PULL && P.pb.on;
        if (!blocked && P.pb.on) {  // the last superstep may have been a blocked pull: its broadcasts
            k_pr_contrib<<<G[G_MISC], BLOCK, 0, st>>>(P);
            k_pr_contrib_done<<<1, 1, 0, st>>>(P);
        }
        mark(1);
        if (mode == IP_MODE_PULL) {
            if (blocked) {
                const int r = pb_launch(g, P, st);
                if (r != IP_OK) return r;
            } else {
                k_pr_pull<<<G[G_PR_PULL], BLOCK, 0, st>>>(P);
            }
            mark(2);
        } else {
            k_pr_push<<<G[G_PR_PUSH], BLOCK, 0, st>>>(P);
            mark(2);
            k_pr_apply<<<G[G_MISC], BLOCK, 0, st>>>(P);
        }
        mark(3);
        return cuda_err(cudaGetLastError());
    }
    const bool hm = P.app == APP_HM;
    switch (mode) {
        case IP_MODE_PUSH_SPARSE:
            k_compact<<<G[G_MISC], BLOCK, 0, st>>>(P);
            mark(1);
            if (hm)
                k_push<APP_HM, true><<<G[G_PUSH_HM_S], BLOCK, 0, st>>>(P);
            else
                k_push<APP_SSSP, true><<<G[G_PUSH_SSSP_S], BLOCK, 0, st>>>(P);
            mark(2);
            k_apply_queue<<<G[G_MISC], BLOCK, 0, st>>>(P);
            break;
        case IP_MODE_PUSH_DENSE:
            mark(1);
            if (hm)
                k_push<APP_HM, false><<<G[G_PUSH_HM_D], BLOCK, 0, st>>>(P);
            else
                k_push<APP_SSSP, false><<<G[G_PUSH_SSSP_D], BLOCK, 0, st>>>(P);
            mark(2);
            k_apply_bitmap<<<G[G_MISC], BLOCK, 0, st>>>(P);
            break;
        default:
            mark(1);
            if (hm)
                k_pull<APP_HM><<<G[G_PULL_HM], BLOCK, 0, st>>>(P);
            else if (P.pull_early_exit)  // unit weights: the first broadcasting in-neighbour decides
                k_pull<APP_SSSP, true><<<G[G_PULL_BFS], BLOCK, 0, st>>>(P);
            else
                k_pull<APP_SSSP><<<G[G_PULL_SSSP], BLOCK, 0, st>>>(P);
            mark(2);
            k_apply_bitmap<<<G[G_MISC], BLOCK, 0, st>>>(P);
            break;
    }
    mark(3);
    return cuda_err(cudaGetLastError());
}

int launch_init(const ip_graph* g, const Params& P, cudaStream_t st) {
    const int gmisc = g->grid[G_MISC];
    if (P.app == APP_PR)
        k_pr_init<<<gmisc, BLOCK, 0, st>>>(P);
    else
        k_init_min<<<gmisc, BLOCK, 0, st>>>(P);
    k_select<<<1, 32, 0, st>>>(P);
    return cuda_err(cudaGetLastError());
}

#define CKR(x)                       \
    do {                             \
        int _r = (x);                \
        if (_r != IP_OK) return _r;  \
    } while (0)

int read_ctl(ip_graph* g, cudaStream_t st) {
    CKR(cuda_err(cudaMemcpyAsync(g->ctl_host, g->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st)));
    return cuda_err(cudaStreamSynchronize(st));
}

// Host-driven superstep loop; with profile, CUDA events time every kernel.
int host_loop(ip_graph* g, const Params& P, cudaStream_t st, bool profile, ip_run_stats_t* stats) {
    cudaEvent_t ev[5] = {};
    if (profile)
        for (int i = 0; i < 5; ++i) CKR(cuda_err(cudaEventCreate(&ev[i])));
    int r = launch_init(g, P, st);
    if (!r) r = read_ctl(g, st);
    while (!r && !g->ctl_host->done) {
        const uint32_t s1 = g->ctl_host->superstep;
        r = launch_superstep(g, P, (int)g->ctl_host->mode, st, profile ? ev : nullptr);
        if (r) break;
        k_select<<<1, 32, 0, st>>>(P);
        if (profile) cudaEventRecord(ev[4], st);
        r = cuda_err(cudaGetLastError());
        if (!r) r = read_ctl(g, st);
        if (!r && profile && stats && stats->kernel_ms && s1 < stats->capacity) {
            for (int k = 0; k < 4; ++k) {
                float ms = 0.f;
                r = cuda_err(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
                if (r) break;
                stats->kernel_ms[4 * s1 + k] = ms;
            }
        }
    }
    if (profile)
        for (int i = 0; i < 5; ++i) cudaEventDestroy(ev[i]);
    return r;
}

// Host loop that, before each exchange, times every mode from the same state:
// two rounds over the three modes, the round order rotated by superstep, the
// minimum per mode kept (so no mode is always the one that runs last, on the
// warmest cache). Every mode leaves the same values, broadcast slots, bitmaps
// and queue flags, so the state of whichever trial ran last is kept. Between
// trials the values, the broadcast slots and the control block are restored.
int label_loop(ip_graph* g, const Params& P, cudaStream_t st, ip_run_stats_t* stats) {
    if (!g->snap_value) CKR(alloc_dev(g, (void**)&g->snap_value, (size_t)g->V * 8));  // values + broadcast slots
    DevCtl snap_ctl;
    CKR(launch_init(g, P, st));
    CKR(read_ctl(g, st));
    constexpr int ROUNDS = 2;
    while (!g->ctl_host->done) {
        const uint32_t s1 = g->ctl_host->superstep;  // the superstep about to run
        snap_ctl = *g->ctl_host;
        if (P.app != APP_PR) {
            CKR(cuda_err(cudaMemcpyAsync(g->snap_value, g->value, (size_t)g->V * 4, cudaMemcpyDeviceToDevice, st)));
            CKR(cuda_err(cudaMemcpyAsync(g->snap_value + g->V, g->outbox, (size_t)g->V * 4, cudaMemcpyDeviceToDevice,
                                         st)));
        }
        float best[3] = {1e30f, 1e30f, 1e30f};
        for (int t = 0; t < 3 * ROUNDS; ++t) {
            const int m = (int)((t + s1) % 3);
            if (t > 0) {  // restore the pre-exchange state
                CKR(cuda_err(cudaMemcpyAsync(g->ctl, &snap_ctl, sizeof(DevCtl), cudaMemcpyHostToDevice, st)));
                if (P.app != APP_PR) {
                    CKR(cuda_err(
                        cudaMemcpyAsync(g->value, g->snap_value, (size_t)g->V * 4, cudaMemcpyDeviceToDevice, st)));
                    CKR(cuda_err(cudaMemcpyAsync(g->outbox, g->snap_value + g->V, (size_t)g->V * 4,
                                                 cudaMemcpyDeviceToDevice, st)));
                }
            }
            if (t == 3 * ROUNDS - 1) k_stamp<<<1, 1, 0, st>>>(g->ctl);
            CKR(cuda_err(cudaEventRecord(g->ev0, st)));
            CKR(launch_superstep(g, P, m, st));
            CKR(cuda_err(cudaEventRecord(g->ev1, st)));
            CKR(cuda_err(cudaStreamSynchronize(st)));
            float ms = 0.f;
            CKR(cuda_err(cudaEventElapsedTime(&ms, g->ev0, g->ev1)));
            best[m] = ms < best[m] ? ms : best[m];
        }
        if (stats && stats->mode_ms && s1 < stats->capacity)
            for (int m = 0; m < 3; ++m) stats->mode_ms[3 * s1 + m] = best[m];
        k_select<<<1, 32, 0, st>>>(P);
        CKR(cuda_err(cudaGetLastError()));
        CKR(read_ctl(g, st));
    }
    return IP_OK;
}

}  // namespace

void free_graph_exec(ip_graph* g) {
    for (ExecEntry& e : g->execs) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        if (e.graph) cudaGraphDestroy(e.graph);
    }
    g->execs.clear();
}

namespace {

// Adds a conditional node at the current capture position of st and makes it the
// new capture dependency. Returns its body graphs.
int add_conditional(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, unsigned size,
                    cudaGraph_t** bodies) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CKR(cuda_err(cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, nullptr, &ndeps)));
    if (cs != cudaStreamCaptureStatusActive) return IP_E_CUDA;
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = size;
    cudaGraphNode_t node;
    CKR(cuda_err(cudaGraphAddNode(&node, cg, deps, nullptr, ndeps, &np)));
    CKR(cuda_err(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies)));
    *bodies = np.conditional.phGraph_out;
    return IP_OK;
}

// Whole run as one graph: init, select, then while(continue){ switch(mode){...}; select }.
int build_graph(ip_graph* g, Params P, cudaGraphExec_t* exec_out, cudaGraph_t* graph_out) {
    cudaStream_t cap;
    CKR(cuda_err(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)));
    int r = IP_OK;
    cudaGraph_t graph = nullptr;
    do {
        r = cuda_err(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        if (r) break;
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg;
        r = cuda_err(cudaStreamGetCaptureInfo(cap, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
        if (!r) r = cuda_err(cudaGraphConditionalHandleCreate(&P.h_while, cg, 0, cudaGraphCondAssignDefault));
        if (!r) r = cuda_err(cudaGraphConditionalHandleCreate(&P.h_switch, cg, 0, cudaGraphCondAssignDefault));
        if (!r) r = launch_init(g, P, cap);
        cudaGraph_t* wbody = nullptr;
        if (!r) r = add_conditional(cap, P.h_while, cudaGraphCondTypeWhile, 1, &wbody);
        cudaGraph_t captured = nullptr;
        cudaError_t e = cudaStreamEndCapture(cap, &captured);
        if (!r) r = cuda_err(e);
        if (r) {
            if (captured) cudaGraphDestroy(captured);
            break;
        }
        graph = captured;
        // while body: switch node, then select
        r = cuda_err(
            cudaStreamBeginCaptureToGraph(cap, wbody[0], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        if (r) break;
        cudaGraph_t* sbody = nullptr;
        r = add_conditional(cap, P.h_switch, cudaGraphCondTypeSwitch, 3, &sbody);
        if (!r) {
            k_select<<<1, 32, 0, cap>>>(P);
            r = cuda_err(cudaGetLastError());
        }
        cudaGraph_t tmp = nullptr;
        e = cudaStreamEndCapture(cap, &tmp);
        if (!r) r = cuda_err(e);
        if (r) break;
        for (int m = 0; m < 3 && !r; ++m) {
            r = cuda_err(
                cudaStreamBeginCaptureToGraph(cap, sbody[m], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            if (r) break;
            r = launch_superstep(g, P, m, cap);
            e = cudaStreamEndCapture(cap, &tmp);
            if (!r) r = cuda_err(e);
        }
    } while (0);
    cudaGraphExec_t exec = nullptr;
    if (!r) r = cuda_err(cudaGraphInstantiate(&exec, graph, 0));
    cudaStreamDestroy(cap);
    if (r) {
        if (graph) cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        return r;
    }
    *exec_out = exec;
    *graph_out = graph;
    return IP_OK;
}

// The instantiated graph for these parameters: cached, least recently used evicted.
int graph_for(ip_graph* g, const Params& P, cudaGraphExec_t* exec) {
    Params key = P;
    key.h_while = key.h_switch = 0;
    ++g->use_clock;
    for (ExecEntry& e : g->execs)
        if (memcmp(e.key, &key, sizeof(Params)) == 0) {
            e.last_use = g->use_clock;
            *exec = e.exec;
            return IP_OK;
        }
    if (g->execs.size() >= 8) {
        size_t lru = 0;
        for (size_t i = 1; i < g->execs.size(); ++i)
            if (g->execs[i].last_use < g->execs[lru].last_use) lru = i;
        cudaGraphExecDestroy(g->execs[lru].exec);
        cudaGraphDestroy(g->execs[lru].graph);
        g->execs.erase(g->execs.begin() + lru);
    }
    ExecEntry e;
    memcpy(e.key, &key, sizeof(Params));
    CKR(build_graph(g, P, &e.exec, &e.graph));
    e.last_use = g->use_clock;
    g->execs.push_back(e);
    *exec = e.exec;
    return IP_OK;
}

}  // namespace

int run_app(ip_graph* g, int app, uint32_t max_supersteps, const ip_options_t* opt, ip_run_stats_t* stats) {
    ip_options_t o;
    if (opt)
        o = *opt;
    else
        ip_options_default(&o);
    cudaStream_t st = (cudaStream_t)o.stream;
    if (app == APP_SSSP && o.source >= g->V) return IP_E_RANGE;
    if (o.policy < IP_POLICY_AUTO || o.policy > IP_POLICY_SEQUENCE) return IP_E_INVAL;
    if (o.policy == IP_POLICY_FORCED && (o.forced_mode < 0 || o.forced_mode > 2)) return IP_E_INVAL;
    if (o.policy == IP_POLICY_SEQUENCE) {
        if (!o.mode_sequence || o.mode_sequence_len == 0 || o.mode_sequence_len > MAX_SEQ) return IP_E_INVAL;
        for (uint32_t i = 0; i < o.mode_sequence_len; ++i)
            if (o.mode_sequence[i] > 2) return IP_E_INVAL;
    }
    if (o.policy == IP_POLICY_MLP && !g->has_selector) return IP_E_STATE;
    if (app == APP_PR && !(o.damping >= 0.f && o.damping <= 1.f)) return IP_E_INVAL;
    if (o.pr_engine < IP_PR_ENGINE_AUTO || o.pr_engine > IP_PR_ENGINE_BLOCKED) return IP_E_INVAL;
    if (!(o.pr_tolerance >= 0.f && o.pr_tolerance <= 3.4e38f)) return IP_E_INVAL;  // also rejects NaN
    const uint32_t t1 = o.t1 ? o.t1 : DEFAULT_T1;
    const uint32_t t2 = o.t2 ? o.t2 : DEFAULT_T2;
    if (t1 >= t2) return IP_E_INVAL;
    CKR(ensure_bins(g, t1, t2, st));
    compute_grids(g);

    const uint32_t want_log = std::min<uint32_t>(max_supersteps, 1u << 16);
    if (g->log_cap < want_log) {
        if (g->log) {
            free_dev(g->log);
            g->device_bytes -= (size_t)g->log_cap * sizeof(LogRec);
        }
        g->log = nullptr;
        g->log_cap = 0;
        CKR(alloc_dev(g, (void**)&g->log, (size_t)want_log * sizeof(LogRec)));
        g->log_cap = want_log;
        free_graph_exec(g);
    }

    Params P;
    memset(&P, 0, sizeof(P));
    P.V = g->V;
    P.W = g->W;
    P.E = g->E;
    P.csr_off = g->csr_off;
    P.csr_col = g->csr_col;
    P.csr_w = g->csr_w;
    P.csc_off = g->csc_off;
    P.csc_row = g->csc_row;
    P.csc_w = g->csc_w;
    P.bout = g->cur->b[0];
    P.bin = g->cur->b[1];
    P.inv_outdeg = g->inv_outdeg;
    P.value = g->value;
    P.rank = g->rank;
    P.contrib0 = g->contrib[0];
    P.contrib1 = g->contrib[1];
    P.mbox = g->mbox;
    P.outbox = g->outbox;
    P.mboxf = g->mboxf;
    P.recv = g->recv;
    P.bcast0 = g->bcast[0];
    P.bcast1 = g->bcast[1];
    P.rq = g->rq;
    for (int p = 0; p < 2; ++p) {
        P.q[p][0] = g->q[p][0];
        P.q[p][1] = g->q[p][1];
        P.hq[p] = g->hq[p];
    }
    P.ctl = g->ctl;
    P.last_send = g->track_send;
    P.log = g->log;
    P.log_cap = g->log_cap;
    P.sel = g->sel;
    P.t1 = t1;
    P.t2 = t2;
    P.thr_sparse = o.thr_sparse;
    P.thr_pull = o.thr_pull;
    P.app = (uint32_t)app;
    P.T = o.pr_iterations;
    P.source = o.source;
    P.orig = g->old_of_new;
    if (app == APP_SSSP && g->new_of_old)  // the caller's source id -> internal id
        CKR(cuda_err(cudaMemcpyAsync(&P.source, g->new_of_old + o.source, 4, cudaMemcpyDeviceToHost, st)));
    P.max_supersteps = max_supersteps;
    P.damping = o.damping;
    P.pr_base = (float)((1.0 - (double)o.damping) / (double)g->V);
    P.pr_tol = app == APP_PR ? o.pr_tolerance : 0.f;
    P.pull_early_exit = (app == APP_SSSP && !g->csc_w && o.pull_early_exit) ? 1u : 0u;
    P.policy = o.policy == IP_POLICY_AUTO ? (g->has_selector ? IP_POLICY_MLP : IP_POLICY_THRESHOLD) : o.policy;
    P.forced_mode = o.forced_mode;
    P.seq_len = o.policy == IP_POLICY_SEQUENCE ? o.mode_sequence_len : 1;
    if (o.policy == IP_POLICY_SEQUENCE) memcpy(P.seq, o.mode_sequence, o.mode_sequence_len);
    P.max_out_deg = g->max_out_deg;
    if (app == APP_SSSP) {
        uint32_t two[2];
        CKR(cuda_err(cudaStreamSynchronize(st)));
        CKR(cuda_err(cudaMemcpyAsync(two, g->csr_off + P.source, 8, cudaMemcpyDeviceToHost, st)));
        CKR(cuda_err(cudaStreamSynchronize(st)));
        P.out_deg_src = two[1] - two[0];
    }
    const bool use_graph = o.use_graph && !o.collect_labels && !o.profile_kernels;
    P.use_graph = use_graph ? 1 : 0;
    if (app == APP_PR) {
        const bool blocked = o.pr_engine == IP_PR_ENGINE_BLOCKED ||
                             (o.pr_engine == IP_PR_ENGINE_AUTO && g->E >= PB_AUTO_EDGES && pb_supported(g));
        if (blocked) {
            const int r = pb_prepare(g, st, &P.pb);
            // AUTO keeps the gather engine where the layout does not fit (entries beyond 2^32)
            if (r != IP_OK && !(r == IP_E_RANGE && o.pr_engine == IP_PR_ENGINE_AUTO)) return r;
        }
    }

    if (stats && stats->mode_ms && stats->capacity) memset(stats->mode_ms, 0, sizeof(float) * 3 * stats->capacity);
    if (stats && stats->kernel_ms && stats->capacity)
        memset(stats->kernel_ms, 0, sizeof(float) * 4 * stats->capacity);
    CKR(cuda_err(cudaEventRecord(g->ev0, st)));
    int r;
    if (o.collect_labels) {
        r = label_loop(g, P, st, stats);
    } else if (use_graph) {
        // the graph bakes the kernel parameters: one instantiated graph per parameter set
        cudaGraphExec_t exec = nullptr;
        r = graph_for(g, P, &exec);
        if (!r) r = cuda_err(cudaGraphLaunch(exec, st));
    } else {
        r = host_loop(g, P, st, o.profile_kernels != 0, stats);
    }
    if (r) return r;
    CKR(cuda_err(cudaEventRecord(g->ev1, st)));
    CKR(cuda_err(cudaEventSynchronize(g->ev1)));
    float elapsed = 0.f;
    CKR(cuda_err(cudaEventElapsedTime(&elapsed, g->ev0, g->ev1)));
    CKR(read_ctl(g, st));
    const DevCtl& c = *g->ctl_host;
    const uint32_t supersteps = c.superstep + 1;
    g->last_app = app;
    if (c.err & 2u) return IP_E_TIMEOUT;  // a bounded wait of a kernel ran out
    if (c.err) return IP_E_DEVICE_ASSERT;
    if (stats) {
        stats->supersteps = supersteps;
        stats->halted = c.done == 1 ? 1 : 0;
        stats->elapsed_ms = elapsed;
        const uint32_t n = std::min(std::min(supersteps, stats->capacity), g->log_cap);
        if (n) {
            LogRec* h = (LogRec*)malloc(sizeof(LogRec) * n);
            if (!h) return IP_E_NOMEM;
            cudaError_t e = cudaMemcpy(h, g->log, sizeof(LogRec) * n, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                free(h);
                return cuda_err(e);
            }
            for (uint32_t i = 0; i < n; ++i) {
                if (stats->mode) stats->mode[i] = (uint8_t)h[i].mode;
                if (stats->active) stats->active[i] = h[i].active;
                if (stats->broadcasters) stats->broadcasters[i] = h[i].bcast;
                if (stats->messages) stats->messages[i] = h[i].msgs;
                if (stats->features)
                    for (int k = 0; k < N_FEATURES; ++k) stats->features[i * N_FEATURES + k] = h[i].feat[k];
                if (stats->pr_delta) stats->pr_delta[i] = h[i].pr_delta;
            }
            free(h);
        }
    }
    return c.done == 1 ? IP_OK : IP_E_MAXSTEPS;
}

}  // namespace ipg
