// The vertex-program engine: superstep 0, the three exchange modes and the apply
// step of Section 4.2 / Fig. 3, written once for any program of the shape in
// include/ipregel_program.cuh (Figs. 9 and 10: improve the value from the
// combined message, broadcast the new value, vote to halt).
//
//   exchange  deliver the broadcasts of superstep s-1 into the one-slot mailboxes
//             (Section 4.3.3) in one of three modes (Section 4.3.2):
//               push-sparse  senders from the binned broadcaster queues (the
//                            selection bypass of Section 4.3.1); the first message
//                            to reach a vertex appends it to the recipient queue
//               push-dense   senders from the broadcast bitmap
//               pull         every vertex folds its in-neighbours' broadcast slots
//             Push combines with the program combiner's atomic (a hardware atomic
//             where one exists, a compare-and-swap loop otherwise).
//   apply     compute() of every recipient: read and reset the mailbox, update the
//             value, broadcast or not, vote to halt; plus the superstep's frontier
//             statistics for the halt test and the mode selector.
//
// Scheduling uses the static degree bins of the graph (lane / warp / CTA chunk);
// edge arrays are read as aligned 16-byte blocks, U blocks in flight per thread.
// A program is registered with IPG_REGISTER_PROGRAM(PROG, app id); ip_run then
// dispatches on the id (PageRank keeps its own engine in superstep.cu).
#pragma once

#include <mutex>

#include "../../include/ipregel_program.cuh"
#include "kernel_util.cuh"

namespace ipg {

// Host-side entry points of one registered program.
struct ProgramOps {
    const char* name;
    bool uses_source;       // reads ip_options_t.source (range-checked, mapped when renumbered)
    bool float_values;      // values are FP32 (ip_get_values returns floats)
    int blocked_kind;       // the pull may run on the blocked layout (pb.cu): 0 no, PB_MIN_COPY (the
                            // codes are the broadcasts), PB_MIN_ADD_WEIGHT (broadcast + edge weight)
    int (*prepare)(const ip_graph* g);  // occupancy queries, before any stream capture
    int (*init)(const ip_graph* g, const Params& P, cudaStream_t st);
    // exchange + apply of one superstep in `mode`; with ev (4 events), the boundaries
    // compaction | exchange | apply are recorded: ev[0] before the compaction, ev[1]
    // before the exchange, ev[2] before the apply, ev[3] after it
    int (*superstep)(const ip_graph* g, const Params& P, int mode, cudaStream_t st, cudaEvent_t* ev);
};
constexpr int MAX_APPS = 8;
void register_program(int app, const ProgramOps* ops);  // superstep.cu
const ProgramOps* program_ops(int app);

namespace eng {

template <class PROG>
using Val = typename PROG::Value;
template <class PROG>
using Comb = typename PROG::Combiner;

template <class PROG>
__device__ __forceinline__ Val<PROG> val_of(uint32_t bits) {
    return ipregel::from_bits<Val<PROG>>(bits);
}
template <class PROG>
__device__ __forceinline__ uint32_t identity_bits() {
    return ipregel::to_bits(Comb<PROG>::identity());
}

// =========================================================== superstep 0
// Resets the control block (a separate launch, so that the statistics of the
// init kernel can be added by every CTA).
template <class PROG>
__global__ void k_ctl_init(Params P) {
    if (threadIdx.x != 0) return;
    DevCtl* c = P.ctl;
    c->superstep = 0;
    c->mode_used = 255;
    c->done = 0;
    c->err = 0;
    c->prev_bcast = 0;
    c->pr_delta = 0.0;
    c->n_pull = 0;
    c->t_prev = globaltimer();
    c->n_active = P.V;
    if (P.pb.on) P.pb.ctr[0] = P.pb.ctr[1] = 0;  // the blocked pull's task counters
    c->rq_len = 0;
    c->q_valid = 0;  // the first push-sparse exchange compacts the bitmap into queues
    for (int p = 0; p < 2; ++p)
        for (int k = 0; k < 3; ++k) c->q_len[p][k] = 0;
    if (PROG::kAllBroadcastAtStart) {
        c->n_bcast = P.V;
        c->msgs = P.E;
        c->max_deg = P.max_out_deg;
    } else {
        c->n_bcast = 0;
        c->msgs = 0;
        c->max_deg = 0;
    }
}

// compute() of superstep 0 for every vertex, one warp per 32-vertex bitmap word:
// the initial value, the broadcast slot (the value, or no-broadcast) and the
// broadcast bitmap; an empty mailbox.
template <class PROG>
__global__ void __launch_bounds__(BLOCK) k_init_prog(Params P) {
    Stats st{0, 0, 0, 0};
    const uint32_t lane = lane_id();
    const uint32_t ident = identity_bits<PROG>();
    for (uint32_t w = global_warp(); w < P.W; w += num_warps()) {
        const uint32_t v = w * 32 + lane;
        bool b = false;
        uint32_t deg = 0;
        if (v < P.V) {
            Val<PROG> x;
            b = PROG::init(v, P.orig ? P.orig[v] : v, P.source, x);
            P.value[v] = ipregel::to_bits(x);
            P.outbox[v] = b ? ipregel::to_bits(x) : ipregel::kNoBroadcastBits;
            P.mbox[v] = ident;
            if (b && (!PROG::kAllBroadcastAtStart || P.last_send)) deg = P.csr_off[v + 1] - P.csr_off[v];
            if (P.last_send) P.last_send[v] = (b && deg) ? 1u : 0u;
        }
        const uint32_t bits = __ballot_sync(FULL, b);
        if (lane == 0) {
            P.recv[w] = 0;
            P.bcast0[w] = bits;
        }
        if (!PROG::kAllBroadcastAtStart) {
            st.bc += b;
            st.msgs += deg;
            st.maxd = max(st.maxd, deg);
        }
    }
    if (!PROG::kAllBroadcastAtStart) flush_stats(st, P.ctl);
}

// ============================================================ push
// One message into v's mailbox (the program's combiner) and v's recipient bit.
// With SPARSE, the first message to reach v appends v to the recipient queue;
// all 32 lanes must call.
template <class PROG, bool SPARSE>
__device__ __forceinline__ void push_edge(const Params& P, bool live, uint32_t v, Val<PROG> msg) {
    using C = Comb<PROG>;
    bool first = false;
    if (live) {
        Val<PROG>* slot = reinterpret_cast<Val<PROG>*>(P.mbox) + v;
        if (ipregel::may_improve<C>(msg, val_of<PROG>(__ldcg(P.mbox + v)))) ipregel::combine_atomic<C>(slot, msg);
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
template <class PROG, bool SPARSE>
__device__ __forceinline__ void push_range(const Params& P, Val<PROG> val, uint32_t b, uint32_t e, uint32_t pos,
                                           uint32_t stride, uint32_t trips) {
    const uint32_t bs = b >> 2, be = (e + 3) >> 2;
    for (uint32_t t = 0; t < trips; ++t) {
        uint4 qc[U], qw[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t blk = bs + (t * U + u) * stride + pos;
            const bool ok = blk < be;
            qc[u] = ok ? ld4(P.csr_col, blk) : make_uint4(0, 0, 0, 0);
            qw[u] = (PROG::kWeighted && P.csr_w && ok) ? ld4(P.csr_w, blk) : make_uint4(1, 1, 1, 1);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t blk = bs + (t * U + u) * stride + pos;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t ei = blk * 4 + j;
                const bool live = blk < be && ei >= b && ei < e;
                push_edge<PROG, SPARSE>(P, live, qa(qc[u], j), PROG::message(val, qa(qw[u], j)));
            }
        }
    }
}

__device__ __forceinline__ uint32_t trips_of(uint32_t b, uint32_t e, uint32_t stride) {
    const uint32_t nb = e > b ? ((e + 3) >> 2) - (b >> 2) : 0u;
    return (nb + stride * U - 1) / (stride * U);
}

template <class PROG, bool SPARSE>
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
            if (threadIdx.x == 0 && h.y == 0) P.outbox[u] = ipregel::kNoBroadcastBits;  // the slot is consumed
            push_range<PROG, SPARSE>(P, val_of<PROG>(P.value[u]), b, e, threadIdx.x, blockDim.x,
                                     trips_of(b, e, blockDim.x));
        }
        // medium senders: one warp each (first the warps the heavy chunks leave idle)
        const uint32_t nm = P.ctl->q_len[par][1];
        const uint32_t* qm = P.q[par][1];
        const uint64_t hw = (uint64_t)min(nh, gridDim.x) * (blockDim.x / 32);
        for (uint32_t i = rotated_warp(hw); i < nm; i += num_warps()) {
            const uint32_t u = qm[i];
            const uint32_t b = P.csr_off[u], e = P.csr_off[u + 1];
            if (lane_id() == 0) P.outbox[u] = ipregel::kNoBroadcastBits;
            push_range<PROG, SPARSE>(P, val_of<PROG>(P.value[u]), b, e, lane_id(), 32, trips_of(b, e, 32));
        }
        // small senders: one lane each
        const uint32_t ns = P.ctl->q_len[par][0];
        const uint32_t* qs = P.q[par][0];
        for (uint32_t base = rotated_warp(hw + nm) * 32; base < ns; base += num_warps() * 32) {
            const uint32_t i = base + lane_id();
            uint32_t b = 0, e = 0, val = 0;
            if (i < ns) {
                const uint32_t u = qs[i];
                b = P.csr_off[u];
                e = P.csr_off[u + 1];
                val = P.value[u];
                P.outbox[u] = ipregel::kNoBroadcastBits;
            }
            const uint32_t trips = __reduce_max_sync(FULL, trips_of(b, e, 1));
            push_range<PROG, SPARSE>(P, val_of<PROG>(val), b, e, 0, 1, trips);
        }
    } else {
        const uint32_t* bc = bc_of(P, sp);
        const Bins& B = P.bout;
        for (uint32_t k = blockIdx.x; k < B.n_hchunk; k += gridDim.x) {
            const uint4 ch = B.hchunk[k];
            if (bit_of(bc, ch.x))
                push_range<PROG, SPARSE>(P, val_of<PROG>(P.value[ch.x]), ch.y, ch.z, threadIdx.x, blockDim.x,
                                         trips_of(ch.y, ch.z, blockDim.x));
        }
        const uint64_t hw = (uint64_t)min(B.n_hchunk, gridDim.x) * (blockDim.x / 32);
        for (uint32_t i = rotated_warp(hw); i < B.n_med; i += num_warps()) {
            const uint32_t u = B.med[i];
            if (bit_of(bc, u)) {
                const uint32_t b = P.csr_off[u], e = P.csr_off[u + 1];
                push_range<PROG, SPARSE>(P, val_of<PROG>(P.value[u]), b, e, lane_id(), 32, trips_of(b, e, 32));
            }
        }
        const uint32_t tiles = (P.V + 31) / 32;
        for (uint32_t t = rotated_warp(hw + B.n_med); t < tiles; t += num_warps()) {
            const uint32_t word = __ldg(bc + t);
            if (!word) continue;
            const uint32_t u = t * 32 + lane_id();
            uint32_t b = 0, e = 0;
            if ((word >> lane_id()) & 1u) {
                b = P.csr_off[u];
                e = P.csr_off[u + 1];
                if (e - b > P.t1) e = b;  // the warp and CTA bins push these
            }
            if (e > b) push_range<PROG, SPARSE>(P, val_of<PROG>(P.value[u]), b, e, 0, 1, trips_of(b, e, 1));
        }
    }
}

// Broadcast bitmap of the last completed superstep -> its binned broadcaster
// queues, unless the queues already hold it.
template <class PROG>
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

// ============================================================ pull
// Folds the in-edges [b, e) into (m, any) reading the broadcast slots
// (outbox[u] = value of u if u broadcast in the last superstep, else the
// no-broadcast pattern): the thread at position pos of a group of `stride`
// threads takes blocks pos, pos+stride, ...
//
// EARLY (a program with kEarlyExitUnweighted on a graph without weights, i.e.
// SSSP as in Fig. 10): under synchronous supersteps every vertex that broadcast
// in superstep s-1 holds the value s-1 (the broadcasters of superstep k are the
// vertices first reached in k), so every message into superstep s is the same
// and the first broadcasting in-neighbour found decides both the combined
// message and whether the vertex is a recipient: the scan stops there (the
// direction-optimising pull). A group of 32 or more threads runs equal trip
// counts and stops as a whole warp.
template <class PROG, bool EARLY>
__device__ __forceinline__ void pull_range(const Params& P, uint32_t b, uint32_t e, uint32_t pos, uint32_t stride,
                                           Val<PROG>& m, bool& any) {
    using C = Comb<PROG>;
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
                x[u][j] = (blk < be && ei >= b && ei < e) ? __ldg(P.outbox + qa(qr[u], j)) : ipregel::kNoBroadcastBits;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool h = (x[u][0] & x[u][1] & x[u][2] & x[u][3]) != ipregel::kNoBroadcastBits;
            if (!h) continue;
            any = true;
            uint4 qw = make_uint4(1, 1, 1, 1);
            if (PROG::kWeighted && P.csc_w) qw = ld4(P.csc_w, g0 + u * stride);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (x[u][j] != ipregel::kNoBroadcastBits) m = C::op(m, PROG::message(val_of<PROG>(x[u][j]), qa(qw, j)));
        }
        if (EARLY && (stride >= 32 ? __any_sync(FULL, any) : any)) break;
    }
}

template <class PROG, bool EARLY>
__global__ void __launch_bounds__(BLOCK) k_pull(Params P) {
    using C = Comb<PROG>;
    using T = Val<PROG>;
    __shared__ uint32_t sm[BLOCK / 32];
    __shared__ uint32_t sa[BLOCK / 32];
    const Bins& B = P.bin;
    T* mbox = reinterpret_cast<T*>(P.mbox);
    for (uint32_t k = blockIdx.x; k < B.n_hchunk; k += gridDim.x) {
        const uint4 ch = B.hchunk[k];
        T m = C::identity();
        bool any = false;
        pull_range<PROG, EARLY>(P, ch.y, ch.z, threadIdx.x, blockDim.x, m, any);
        m = ipregel::warp_combine<C>(m);
        const uint32_t a = __any_sync(FULL, any);
        if (lane_id() == 0) {
            sm[threadIdx.x >> 5] = ipregel::to_bits(m);
            sa[threadIdx.x >> 5] = a;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            T mm = C::identity();
            uint32_t aa = 0;
            for (uint32_t w = 0; w < blockDim.x / 32; ++w) {
                mm = C::op(mm, val_of<PROG>(sm[w]));
                aa |= sa[w];
            }
            if (aa) {  // the vertex's other chunks may be combined by other CTAs
                ipregel::combine_atomic<C>(mbox + ch.x, mm);
                atomicOr(P.recv + (ch.x >> 5), 1u << (ch.x & 31u));
            }
        }
        __syncthreads();
    }
    const uint64_t hw = (uint64_t)min(B.n_hchunk, gridDim.x) * (blockDim.x / 32);  // warps on heavy chunks
    for (uint32_t i = rotated_warp(hw); i < B.n_med; i += num_warps()) {
        const uint32_t v = B.med[i];
        T m = C::identity();
        bool any = false;
        pull_range<PROG, EARLY>(P, P.csc_off[v], P.csc_off[v + 1], lane_id(), 32, m, any);
        m = ipregel::warp_combine<C>(m);
        any = __any_sync(FULL, any);
        if (lane_id() == 0 && any) {
            mbox[v] = m;
            atomicOr(P.recv + (v >> 5), 1u << (v & 31u));
        }
    }
    const uint32_t tiles = (P.V + 31) / 32;
    for (uint32_t t = rotated_warp(hw + B.n_med); t < tiles; t += num_warps()) {
        const uint32_t v = t * 32 + lane_id();
        T m = C::identity();
        bool any = false;
        if (v < P.V) {
            const uint32_t b = P.csc_off[v], e = P.csc_off[v + 1];
            if (e - b <= P.t1) pull_range<PROG, EARLY>(P, b, e, 0, 1, m, any);
        }
        if (any) mbox[v] = m;
        const uint32_t bits = __ballot_sync(FULL, any);
        if (lane_id() == 0 && bits) atomicOr(P.recv + t, bits);
    }
}

// ============================================================ apply
// compute() of one recipient of the queue path: m is its combined message.
// Returns whether it broadcasts (then deg = its out-degree).
template <class PROG>
__device__ __forceinline__ bool apply_vertex(const Params& P, uint32_t v, uint32_t& deg) {
    const Val<PROG> m = val_of<PROG>(P.mbox[v]);
    P.mbox[v] = identity_bits<PROG>();
    Val<PROG> val = val_of<PROG>(P.value[v]);
    deg = 0;
    if (PROG::compute(val, m)) {
        P.value[v] = ipregel::to_bits(val);
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
template <class PROG>
__global__ void __launch_bounds__(BLOCK, 5) k_apply_bitmap(Params P) {  // 5 CTAs per SM, as before the programs
    Stats st{0, 0, 0, 0};
    uint32_t* bc = bc_mut(P, P.ctl->superstep);
    const uint32_t words = (P.V + 31) / 32;
    const uint32_t nw = num_warps(), lane = lane_id();
    const uint32_t ident = identity_bits<PROG>();
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
            m[k] = r ? P.mbox[v] : ident;
            val[k] = r ? P.value[v] : 0u;
        }
        uint32_t deg[AW];
#pragma unroll
        for (int k = 0; k < AW; ++k) {
            const uint32_t w = w0 + k * nw;
            const uint32_t v = w * 32 + lane;
            const bool r = (rw[k] >> lane) & 1u;
            Val<PROG> nv = val_of<PROG>(val[k]);
            const bool b = r && PROG::compute(nv, val_of<PROG>(m[k]));  // improve and broadcast
            if (r) P.mbox[v] = ident;
            if (b) P.value[v] = ipregel::to_bits(nv);
            if (w < words && v < P.V) P.outbox[v] = b ? ipregel::to_bits(nv) : ipregel::kNoBroadcastBits;
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
template <class PROG>
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
            b = apply_vertex<PROG>(P, v, deg);
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

}  // namespace eng

// ================================================================ host side
int cuda_err(cudaError_t e);

// Launch sizes and the host entry points of one program's kernels.
template <class PROG>
struct ProgramEngine {
    static constexpr bool kAddsWeight = ipregel::blocked_pull_adds_weight<PROG>::value;
    static_assert(!(PROG::kBlockedMinPull || kAddsWeight) ||
                      std::is_same<typename PROG::Combiner, ipregel::MinCombiner<uint32_t>>::value,
                  "the blocked pull folds uint32 broadcast slots with min");
    static_assert(!(PROG::kBlockedMinPull && kAddsWeight), "one kind of blocked pull per program");
    static constexpr int kBlockedKind = PROG::kBlockedMinPull ? PB_MIN_COPY : (kAddsWeight ? PB_MIN_ADD_WEIGHT : 0);
    enum { K_PUSH_S, K_PUSH_D, K_PULL, K_PULL_EARLY, K_MISC, K_COUNT };
    static int occ[K_COUNT];  // resident CTAs per SM of each kernel, queried once
    static std::once_flag once;

    static int prepare(const ip_graph*) {
        std::call_once(once, [] {
            const void* fns[K_COUNT] = {(const void*)eng::k_push<PROG, true>, (const void*)eng::k_push<PROG, false>,
                                        (const void*)eng::k_pull<PROG, false>, (const void*)eng::k_pull<PROG, true>,
                                        (const void*)eng::k_apply_bitmap<PROG>};
            for (int i = 0; i < K_COUNT; ++i) {
                int o = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fns[i], BLOCK, 0) != cudaSuccess || o < 1) {
                    (void)cudaGetLastError();
                    o = 2;
                }
                occ[i] = o;
            }
        });
        return IP_OK;
    }

    static int init(const ip_graph* g, const Params& P, cudaStream_t st) {
        eng::k_ctl_init<PROG><<<1, 32, 0, st>>>(P);
        eng::k_init_prog<PROG><<<g->num_sms * occ[K_MISC], BLOCK, 0, st>>>(P);
        return cuda_err(cudaGetLastError());
    }

    static int superstep(const ip_graph* g, const Params& P, int mode, cudaStream_t st, cudaEvent_t* ev) {
        const int n = g->num_sms;
        auto mark = [&](int i) {
            if (ev) cudaEventRecord(ev[i], st);
        };
        mark(0);
        switch (mode) {
            case IP_MODE_PUSH_SPARSE:
                eng::k_compact<PROG><<<n * occ[K_MISC], BLOCK, 0, st>>>(P);
                mark(1);
                eng::k_push<PROG, true><<<n * occ[K_PUSH_S], BLOCK, 0, st>>>(P);
                mark(2);
                eng::k_apply_queue<PROG><<<n * occ[K_MISC], BLOCK, 0, st>>>(P);
                break;
            case IP_MODE_PUSH_DENSE:
                mark(1);
                eng::k_push<PROG, false><<<n * occ[K_PUSH_D], BLOCK, 0, st>>>(P);
                mark(2);
                eng::k_apply_bitmap<PROG><<<n * occ[K_MISC], BLOCK, 0, st>>>(P);
                break;
            default:
                mark(1);
                if (kBlockedKind && P.pb.on) {
                    const int r = pb_min_launch(g, P, st, kBlockedKind);
                    if (r != IP_OK) return r;
                } else if (PROG::kEarlyExitUnweighted && P.pull_early_exit)
                    eng::k_pull<PROG, true><<<n * occ[K_PULL_EARLY], BLOCK, 0, st>>>(P);
                else
                    eng::k_pull<PROG, false><<<n * occ[K_PULL], BLOCK, 0, st>>>(P);
                mark(2);
                eng::k_apply_bitmap<PROG><<<n * occ[K_MISC], BLOCK, 0, st>>>(P);
                break;
        }
        mark(3);
        return cuda_err(cudaGetLastError());
    }

    static ProgramOps ops(const char* name) {
        ProgramOps o;
        o.name = name;
        o.uses_source = PROG::kUsesSource;
        o.float_values = std::is_floating_point<typename PROG::Value>::value;
        o.blocked_kind = kBlockedKind;
        o.prepare = &prepare;
        o.init = &init;
        o.superstep = &superstep;
        return o;
    }
};
template <class PROG>
int ProgramEngine<PROG>::occ[ProgramEngine<PROG>::K_COUNT] = {};
template <class PROG>
std::once_flag ProgramEngine<PROG>::once;

}  // namespace ipg

// Registers PROG as application APP_ID of ip_run (one line in a .cu file of the library).
#define IPG_REGISTER_PROGRAM(PROG, APP_ID)                                                          \
    namespace {                                                                                   \
    const ::ipg::ProgramOps ipg_ops_##PROG = ::ipg::ProgramEngine<PROG>::ops(#PROG);              \
    const bool ipg_registered_##PROG = (::ipg::register_program((APP_ID), &ipg_ops_##PROG), true); \
    }
