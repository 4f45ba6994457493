// Batched runs in one persistent launch: many SSSP sources on one graph, and
// many Hashmin instances (disjoint graphs concatenated block-diagonally).
//
// Each batch runs as one cooperative kernel that holds the whole superstep loop
// (Section 4.2, Fig. 3): superstep 0, then per superstep an exchange phase (pull,
// Section 4.3.2) and an apply phase (compute() of Figs. 9 / 10), separated by a
// grid-wide barrier. Every wait of the barrier is bounded by %globaltimer; a
// wait that runs out sets an error word and the kernel winds down, so a run can
// fail with IP_E_TIMEOUT but cannot hang. The cooperative launch is captured in
// a CUDA graph, so the host issues one graph launch per batch.
//
// Arrays that the kernel itself rewrites are read through L2 (ld.global.cg):
// the L1 cache is not coherent between the SMs of one running kernel.
//
// Multi-source SSSP keeps distances vertex-major, dist[v][source], in groups of
// 32 sources: one warp serves one vertex, lane k one source, so one read of an
// in-edge serves every source and each (in-edge, group) costs one 128-byte load.
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace ipg {
namespace {

constexpr int BB = 256;            // threads per CTA of the persistent kernels
constexpr uint32_t MS_CH = 128;    // in-edges per exchange task of the multi-source kernel
constexpr uint32_t NONE = 0xFFFFFFFFu;

struct GridBar {
    unsigned int count, gen, err, pad;
};

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t lane_of() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t gwarp() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ uint32_t nwarps() { return (gridDim.x * blockDim.x) >> 5; }
__device__ __forceinline__ uint32_t sat_add32(uint32_t a, uint32_t b) {
    const uint32_t s = a + b;
    return s < a ? INF : s;
}
__device__ __forceinline__ uint32_t ldcg(const uint32_t* p) { return __ldcg(p); }

// Grid-wide barrier of a cooperative launch. Waits are bounded by limit_ns; a
// block whose wait runs out sets err. Returns false once err is set, and every
// caller then leaves the kernel.
__device__ bool grid_sync(GridBar* b, uint64_t limit_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vg = &b->gen;
        volatile unsigned int* ve = &b->err;
        int good = *ve == 0;
        if (good) {
            const unsigned int g = *vg;
            __threadfence();
            if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
                atomicExch(&b->count, 0u);
                __threadfence();
                atomicAdd(&b->gen, 1u);
            } else {
                const uint64_t t0 = gtimer();
                while (*vg == g) {
                    if (*ve) break;
                    if (gtimer() - t0 > limit_ns) {
                        atomicOr(&b->err, 1u);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
            good = *ve == 0;
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ unsigned long long block_sum(unsigned long long x) {
    __shared__ unsigned long long sh[BB / 32];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(FULL, x, o);
    __syncthreads();
    if (lane_of() == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;  // valid in thread 0
}

// =================================================================== multi-source SSSP
struct MsParams {
    uint32_t V, G, K;
    const uint32_t* csr_off;
    const uint32_t* csc_off;
    const uint32_t* csc_row;
    const uint32_t* csc_w;
    const uint2* tasks;  // {vertex | 0x80000000 when the vertex has several tasks, first in-edge}
    uint32_t n_tasks;
    const uint32_t* sources;
    uint32_t* dist;  // [V][G][32]
    uint32_t* mbox;  // [V][G][32]
    uint32_t* mask0; // [V][GP]: sources whose value the vertex broadcast, even supersteps
    uint32_t* mask1; // odd supersteps
    uint32_t* rmask; // [V][GP]: sources for which the vertex received a message
    uint32_t* src_last;  // [K]: last superstep in which the source's run sent a message
    unsigned long long* msgs;  // [2] by superstep parity; [2] running total
    unsigned int* state;       // [0] supersteps run, [1] halted
    GridBar* bar;
    uint64_t limit_ns;
    uint32_t max_supersteps;
};

__device__ __forceinline__ size_t slot(uint32_t v, uint32_t G, uint32_t g) { return ((size_t)v * G + g) * 32u; }

// Mask words of one vertex, GP = G padded to 1, 2, 4 or 8 words (16-byte loads).
template <int GP>
__device__ __forceinline__ void load_masks(const uint32_t* base, uint32_t u, bool valid, uint32_t* mw) {
    if (!valid) {
#pragma unroll
        for (int g = 0; g < GP; ++g) mw[g] = 0;
        return;
    }
    const uint32_t* p = base + (size_t)u * GP;
    if (GP == 8) {
        const uint4 a = __ldcg(reinterpret_cast<const uint4*>(p)), b = __ldcg(reinterpret_cast<const uint4*>(p) + 1);
        mw[0] = a.x, mw[1] = a.y, mw[2] = a.z, mw[3] = a.w, mw[4] = b.x, mw[5] = b.y, mw[6] = b.z, mw[7] = b.w;
    } else if (GP == 4) {
        const uint4 a = __ldcg(reinterpret_cast<const uint4*>(p));
        mw[0] = a.x, mw[1] = a.y, mw[2] = a.z, mw[3] = a.w;
    } else if (GP == 2) {
        const uint2 a = __ldcg(reinterpret_cast<const uint2*>(p));
        mw[0] = a.x, mw[1] = a.y;
    } else {
        mw[0] = __ldcg(p);
    }
}

// Per-warp scratch of the exchange phase.
struct MsWarpSmem {
    uint4 pairs[32 * 8];  // active (in-edge, group): {source vertex u, weight, mask word, group}
    uint32_t cand[8 * 32];  // candidate minimum per (group, source lane)
};

// One exchange task: in-edges [b, e) of vertex v. Each batch of 32 in-edges is
// turned into a list of active (in-edge, group) pairs; each pair costs one
// 128-byte read of the sender's distances, eight pairs in flight at a time.
template <int G, int GP>
__device__ void ms_exchange_task(const MsParams& P, const uint32_t* prev, uint2 task, MsWarpSmem& S) {
    const uint32_t lane = lane_of();
    const uint32_t v = task.x & 0x7FFFFFFFu;
    const bool multi = task.x >> 31;
    const uint32_t b = task.y, e = min(b + MS_CH, P.csc_off[v + 1]);
#pragma unroll
    for (int g = 0; g < G; ++g) S.cand[g * 32 + lane] = INF;
    uint32_t rb[G];
#pragma unroll
    for (int g = 0; g < G; ++g) rb[g] = 0;
    for (uint32_t base = b; base < e; base += 32) {
        const uint32_t ei = base + lane;
        const bool valid = ei < e;
        const uint32_t u = valid ? P.csc_row[ei] : 0u;
        uint32_t mw[GP];
        load_masks<GP>(prev, u, valid, mw);
        uint32_t cnt = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) cnt += mw[g] != 0;
        uint32_t inc = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, inc, o);
            if (lane >= (uint32_t)o) inc += y;
        }
        const uint32_t total = __shfl_sync(FULL, inc, 31);
        if (!total) continue;  // no in-neighbour of this batch broadcast
        const uint32_t w = valid ? (P.csc_w ? P.csc_w[ei] : 1u) : 0u;
        uint32_t pos = inc - cnt;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            rb[g] |= __reduce_or_sync(FULL, mw[g]);
            if (mw[g]) S.pairs[pos++] = make_uint4(u, w, mw[g], (uint32_t)g);
        }
        __syncwarp();
        for (uint32_t p0 = 0; p0 < total; p0 += 8) {
            uint32_t x[8];
            uint4 pr[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const bool in = p0 + q < total;
                pr[q] = in ? S.pairs[p0 + q] : make_uint4(0, 0, 0, 0);
                const bool take = in && ((pr[q].z >> lane) & 1u);
                x[q] = take ? ldcg(P.dist + slot(pr[q].x, G, pr[q].w) + lane) : INF;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (x[q] != INF) {
                    uint32_t* c = &S.cand[pr[q].w * 32 + lane];
                    *c = min(*c, sat_add32(x[q], pr[q].y));
                }
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (!rb[g]) continue;
        const size_t idx = slot(v, G, g) + lane;
        const uint32_t ri = v * GP + g;
        const uint32_t cg = S.cand[g * 32 + lane];
        if (multi) {
            if ((rb[g] >> lane) & 1u) atomicMin(P.mbox + idx, cg);
            if (lane == 0) atomicOr(P.rmask + ri, rb[g]);
        } else {
            if ((rb[g] >> lane) & 1u) P.mbox[idx] = cg;
            if (lane == 0) P.rmask[ri] = rb[g];
        }
    }
    __syncwarp();
}

template <int G, int GP>
__device__ unsigned long long ms_apply_vertex(const MsParams& P, uint32_t* next, uint32_t v, uint32_t s) {
    const uint32_t lane = lane_of();
    const uint32_t ri0 = v * GP;
    // lane g < GP holds the recipient word of group g
    const uint32_t rwl = lane < (uint32_t)GP ? ldcg(P.rmask + ri0 + lane) : 0u;
    const uint32_t groups = __ballot_sync(FULL, rwl != 0);
    uint32_t bitsl = 0;  // lane g: the new broadcast word of group g
    unsigned long long sent = 0;
    if (groups) {
        const uint32_t deg = P.csr_off[v + 1] - P.csr_off[v];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (!((groups >> g) & 1u)) continue;
            const uint32_t rw = __shfl_sync(FULL, rwl, g);
            bool nb = false;
            if ((rw >> lane) & 1u) {
                const size_t idx = slot(v, G, g) + lane;
                const uint32_t m = ldcg(P.mbox + idx);
                P.mbox[idx] = INF;
                if (m < ldcg(P.dist + idx)) {  // compute() of Fig. 10: improve and broadcast
                    P.dist[idx] = m;
                    nb = true;
                }
            }
            const uint32_t bits = __ballot_sync(FULL, nb);
            if (lane == (uint32_t)g) bitsl = bits;
            if (bits && deg) {
                sent += (unsigned long long)__popc(bits) * deg;
                if (nb) P.src_last[g * 32 + lane] = s;
            }
        }
    }
    if (lane < (uint32_t)GP) {
        next[ri0 + lane] = bitsl;
        if (rwl) P.rmask[ri0 + lane] = 0;
    }
    return sent;
}

template <int G, int GP>
__global__ void __launch_bounds__(BB) k_msssp(MsParams P) {
    const uint32_t lane = lane_of(), gw = gwarp(), nw = nwarps();
    // superstep 0 (Fig. 10): each source takes 0 and broadcasts; every other value is INF
    for (uint32_t v = gw; v < P.V; v += nw) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t k = g * 32 + lane;
            const bool is_src = k < P.K && P.sources[k] == v;
            const size_t idx = slot(v, G, g) + lane;
            P.dist[idx] = is_src ? 0u : INF;
            P.mbox[idx] = INF;
            const uint32_t bits = __ballot_sync(FULL, is_src);
            if (lane == 0) {
                P.mask0[v * GP + g] = bits;
                P.rmask[v * GP + g] = 0;
            }
        }
        if (lane >= (uint32_t)G && lane < (uint32_t)GP) {  // padding words stay 0
            P.mask0[v * GP + lane] = 0;
            P.mask1[v * GP + lane] = 0;
            P.rmask[v * GP + lane] = 0;
        }
    }
    if (blockIdx.x == 0) {
        unsigned long long sent = 0;
        for (uint32_t k = threadIdx.x; k < P.K; k += blockDim.x) {
            const uint32_t sv = P.sources[k];
            const uint32_t d = P.csr_off[sv + 1] - P.csr_off[sv];
            sent += d;
            P.src_last[k] = d ? 0u : NONE;
        }
        const unsigned long long t = block_sum(sent);
        if (threadIdx.x == 0) {
            P.msgs[0] = t;
            P.msgs[2] = t;
            P.state[0] = 1;
            P.state[1] = 0;
            P.state[2] = P.state[3] = 0;  // task counters of the exchange phase, by parity
        }
    }
    if (!grid_sync(P.bar, P.limit_ns)) return;
    uint32_t s = 0;  // last completed superstep
    while (true) {
        const unsigned long long sent = *(volatile unsigned long long*)&P.msgs[s & 1];
        if (sent == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) P.state[1] = 1;
            break;
        }
        if (s + 1 >= P.max_supersteps) break;
        ++s;
        const uint32_t* prev = (s & 1) ? P.mask0 : P.mask1;
        uint32_t* next = (s & 1) ? P.mask1 : P.mask0;
        if (blockIdx.x == 0 && threadIdx.x == 0) P.msgs[s & 1] = 0;
        {  // tasks are claimed four at a time from a counter; the largest come first
            __shared__ MsWarpSmem smem[BB / 32];
            MsWarpSmem& S = smem[threadIdx.x >> 5];
            unsigned int* ctr = P.state + 2 + (s & 1);
            if (blockIdx.x == 0 && threadIdx.x == 0) P.state[2 + ((s + 1) & 1)] = 0;  // next superstep's counter
            while (true) {
                uint32_t t0 = 0;
                if (lane == 0) t0 = atomicAdd(ctr, 4u);
                t0 = __shfl_sync(FULL, t0, 0);
                if (t0 >= P.n_tasks) break;
                for (uint32_t t = t0; t < min(t0 + 4, P.n_tasks); ++t) ms_exchange_task<G, GP>(P, prev, P.tasks[t], S);
            }
        }
        if (!grid_sync(P.bar, P.limit_ns)) return;
        unsigned long long mine = 0;
        for (uint32_t v = gw; v < P.V; v += nw) mine += ms_apply_vertex<G, GP>(P, next, v, s);
        if (lane != 0) mine = 0;
        const unsigned long long t = block_sum(mine);
        if (threadIdx.x == 0 && t) {
            atomicAdd(&P.msgs[s & 1], t);
            atomicAdd(&P.msgs[2], t);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) P.state[0] = s + 1;
        if (!grid_sync(P.bar, P.limit_ns)) return;
    }
}

// dist[v][G][32] -> out[k][v] for k < K (source-major), 32x32 tiles through shared memory.
// On a renumbered graph v runs over the caller's ids and reads internal row nid[v].
__global__ void k_ms_transpose(const uint32_t* dist, uint32_t V, uint32_t G, uint32_t K, const uint32_t* nid,
                               uint32_t* out) {
    __shared__ uint32_t tile[32][33];
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const uint32_t vt = (V + 31) / 32;
    for (uint32_t t = blockIdx.x; t < vt * G; t += gridDim.x) {
        const uint32_t v0 = (t / G) * 32, g = t % G;
        for (uint32_t j = wib; j < 32; j += blockDim.x >> 5) {
            const uint32_t v = v0 + j;
            tile[j][lane] = v < V ? dist[slot(nid ? __ldg(nid + v) : v, G, g) + lane] : INF;
        }
        __syncthreads();
        for (uint32_t j = wib; j < 32; j += blockDim.x >> 5) {
            const uint32_t k = g * 32 + j, v = v0 + lane;
            if (k < K && v < V) out[(size_t)k * V + v] = tile[lane][j];
        }
        __syncthreads();
    }
}

// Caller's source ids -> internal ids, in place.
__global__ void k_map_ids(uint32_t* ids, uint32_t k, const uint32_t* nid) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) ids[i] = nid[ids[i]];
}

// =================================================================== multi-instance Hashmin
struct BhParams {
    uint32_t V, W;
    const uint32_t* csr_off;
    const uint32_t* csc_off;
    const uint32_t* csc_row;
    Bins bin;  // in-edge bins of the union graph
    uint32_t t1;
    uint32_t* label;
    uint32_t* outbox;  // label if broadcast in the last superstep, else INF
    uint32_t* mbox;
    uint32_t* recv;
    const uint32_t* inst_off;  // k+1 vertex offsets of the instances (caller's ids)
    const uint32_t* orig;      // renumbered graph: internal id -> caller's id, else null
    const uint32_t* nid;       // renumbered graph: caller's id -> internal id, else null
    uint32_t k;
    uint32_t* inst_last;       // [k]: last superstep in which the instance sent a message
    unsigned long long* msgs;
    unsigned int* state;
    GridBar* bar;
    uint64_t limit_ns;
    uint32_t max_supersteps;
};

__device__ __forceinline__ uint32_t instance_of(const BhParams& P, uint32_t v) {
    uint32_t lo = 0, hi = P.k;  // inst_off[lo] <= v < inst_off[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(P.inst_off + mid) <= v)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t caller_id(const BhParams& P, uint32_t v) { return P.orig ? __ldg(P.orig + v) : v; }

__device__ __forceinline__ void bh_fold(const BhParams& P, uint32_t b, uint32_t e, uint32_t pos, uint32_t stride,
                                        uint32_t& m, bool& any) {
    for (uint32_t ei = b + pos; ei < e; ei += stride) {
        const uint32_t x = ldcg(P.outbox + P.csc_row[ei]);
        if (x != INF) {
            any = true;
            m = min(m, x);
        }
    }
}

__global__ void __launch_bounds__(BB) k_bhashmin(BhParams P) {
    __shared__ uint32_t sm[BB / 32], sa[BB / 32];
    const uint32_t lane = lane_of(), gw = gwarp(), nw = nwarps();
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    // superstep 0 (Fig. 9): label = id, every vertex broadcasts
    unsigned long long sent0 = 0;
    for (uint32_t v = tid; v < P.V; v += nth) {
        const uint32_t id = caller_id(P, v);
        P.label[v] = id;
        P.outbox[v] = id;
        P.mbox[v] = INF;
        const uint32_t d = P.csr_off[v + 1] - P.csr_off[v];
        sent0 += d;
        if (d) P.inst_last[instance_of(P, id)] = 0;
    }
    for (uint32_t w = tid; w < P.W; w += nth) P.recv[w] = 0;
    const unsigned long long t0 = block_sum(sent0);
    if (threadIdx.x == 0) atomicAdd(&P.msgs[0], t0), atomicAdd(&P.msgs[2], t0);
    if (blockIdx.x == 0 && threadIdx.x == 0) P.state[0] = 1;
    if (!grid_sync(P.bar, P.limit_ns)) return;
    uint32_t s = 0;
    while (true) {
        const unsigned long long sent = *(volatile unsigned long long*)&P.msgs[s & 1];
        if (sent == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) P.state[1] = 1;
            break;
        }
        if (s + 1 >= P.max_supersteps) break;
        ++s;
        if (blockIdx.x == 0 && threadIdx.x == 0) P.msgs[s & 1] = 0;
        // ---- exchange (pull): heavy chunks per CTA, medium vertices per warp, small per lane
        for (uint32_t c = blockIdx.x; c < P.bin.n_hchunk; c += gridDim.x) {
            const uint4 ch = P.bin.hchunk[c];
            uint32_t m = INF;
            bool any = false;
            bh_fold(P, ch.y, ch.z, threadIdx.x, blockDim.x, m, any);
            m = __reduce_min_sync(FULL, m);
            const uint32_t a = __any_sync(FULL, any);
            if (lane == 0) {
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
        for (uint32_t i = gw; i < P.bin.n_med; i += nw) {
            const uint32_t v = P.bin.med[i];
            uint32_t m = INF;
            bool any = false;
            bh_fold(P, P.csc_off[v], P.csc_off[v + 1], lane, 32, m, any);
            m = __reduce_min_sync(FULL, m);
            any = __any_sync(FULL, any);
            if (lane == 0 && any) {
                P.mbox[v] = m;
                atomicOr(P.recv + (v >> 5), 1u << (v & 31u));
            }
        }
        const uint32_t tiles = (P.V + 31) / 32;
        for (uint32_t t = gw; t < tiles; t += nw) {
            const uint32_t v = t * 32 + lane;
            uint32_t m = INF;
            bool any = false;
            if (v < P.V) {
                const uint32_t b = P.csc_off[v], e = P.csc_off[v + 1];
                if (e - b <= P.t1) bh_fold(P, b, e, 0, 1, m, any);
            }
            if (any) P.mbox[v] = m;
            const uint32_t bits = __ballot_sync(FULL, any);
            if (lane == 0 && bits) atomicOr(P.recv + t, bits);
        }
        if (!grid_sync(P.bar, P.limit_ns)) return;
        // ---- apply: compute() of Fig. 9 for every recipient
        unsigned long long mine = 0;
        for (uint32_t t = gw; t < tiles; t += nw) {
            const uint32_t rw = ldcg(P.recv + t);
            const uint32_t v = t * 32 + lane;
            uint32_t out = INF;
            if ((rw >> lane) & 1u) {
                const uint32_t m = ldcg(P.mbox + v);
                P.mbox[v] = INF;
                if (m < ldcg(P.label + v)) {
                    P.label[v] = m;
                    out = m;
                    const uint32_t d = P.csr_off[v + 1] - P.csr_off[v];
                    mine += d;
                    if (d) P.inst_last[instance_of(P, caller_id(P, v))] = s;
                }
            }
            if (v < P.V) P.outbox[v] = out;
            if (lane == 0 && rw) P.recv[t] = 0;
        }
        const unsigned long long tot = block_sum(mine);
        if (threadIdx.x == 0 && tot) {
            atomicAdd(&P.msgs[s & 1], tot);
            atomicAdd(&P.msgs[2], tot);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) P.state[0] = s + 1;
        if (!grid_sync(P.bar, P.limit_ns)) return;
    }
}

// Union labels -> labels local to each instance, in the caller's numbering.
__global__ void k_bh_local(const BhParams P, uint32_t* out) {
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < P.V; u += gridDim.x * blockDim.x)
        out[u] = P.label[P.nid ? __ldg(P.nid + u) : u] - __ldg(P.inst_off + instance_of(P, u));
}

// Engine 0 helpers: per-instance maximum of the per-vertex last-send record
// (1 + superstep, 0 = never), and labels local to each instance.
__global__ void k_inst_max(const uint32_t* track, const uint32_t* off, uint32_t k, uint32_t* inst_last) {
    __shared__ uint32_t sh[BB / 32];
    for (uint32_t i = blockIdx.x; i < k; i += gridDim.x) {
        uint32_t m = 0;
        for (uint32_t v = off[i] + threadIdx.x; v < off[i + 1]; v += blockDim.x) m = max(m, track[v]);
        m = __reduce_max_sync(FULL, m);
        if (lane_of() == 0) sh[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = max(t, sh[w]);
            inst_last[i] = t;
        }
        __syncthreads();
    }
}

__global__ void k_local_labels(const uint32_t* label, uint32_t V, const uint32_t* off, uint32_t k, uint32_t* out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = k;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (off[mid] <= v)
                lo = mid;
            else
                hi = mid;
        }
        out[v] = label[v] - off[lo];
    }
}

// =================================================================== host state
struct BatchState {
    // multi-source SSSP
    uint32_t ms_G = 0;
    uint32_t* dist = nullptr;
    uint32_t* mbox = nullptr;
    uint32_t* masks = nullptr;  // mask0 | mask1 | rmask
    uint2* tasks = nullptr;
    uint32_t n_tasks = 0;
    size_t bytes = 0;
    // shared
    uint32_t* small = nullptr;  // sources / instance offsets / per-instance last superstep
    size_t small_cap = 0;
    unsigned long long* msgs = nullptr;  // [4]
    unsigned int* state = nullptr;       // [4]
    GridBar* bar = nullptr;
    uint32_t* out_tmp = nullptr;  // host-bound outputs staged on the device
    size_t out_cap = 0;
    uint32_t* track = nullptr;    // per-vertex last-send record (engine 0 Hashmin batches)
    cudaGraphExec_t exec = nullptr;
    unsigned char key[256] = {0};
    size_t key_len = 0;
};

#define CKB(x)                              \
    do {                                    \
        int _r = cuda_err(x);               \
        if (_r != IP_OK) return _r;         \
    } while (0)

BatchState* state_of(ip_graph* g) {
    if (!g->batch) g->batch = new BatchState();
    return (BatchState*)g->batch;
}

int ensure_small(ip_graph* g, BatchState* b, size_t words) {
    if (!b->msgs) {
        int r = alloc_dev(g, (void**)&b->msgs, 4 * sizeof(unsigned long long));
        if (!r) r = alloc_dev(g, (void**)&b->state, 4 * sizeof(unsigned int));
        if (!r) r = alloc_dev(g, (void**)&b->bar, sizeof(GridBar));
        if (r) return r;
    }
    if (b->small_cap < words) {
        if (b->small) free_dev(b->small);
        b->small = nullptr;
        b->small_cap = 0;
        int r = alloc_dev(g, (void**)&b->small, words * 4);
        if (r) return r;
        b->small_cap = words;
    }
    return IP_OK;
}

int ensure_out(ip_graph* g, BatchState* b, size_t words) {
    if (b->out_cap >= words) return IP_OK;
    if (b->out_tmp) free_dev(b->out_tmp);
    b->out_tmp = nullptr;
    b->out_cap = 0;
    int r = alloc_dev(g, (void**)&b->out_tmp, words * 4);
    if (!r) b->out_cap = words;
    return r;
}

void drop_exec(BatchState* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->key_len = 0;
}

// Captures one cooperative launch into a graph (cached on the parameters) and launches it.
template <class KP>
int launch_persistent(BatchState* b, const void* fn, const KP& params, int grid, cudaStream_t st) {
    const size_t kl = sizeof(KP) + sizeof(int) + sizeof(void*);
    unsigned char key[256];
    if (kl > sizeof(key)) return IP_E_INVAL;
    memcpy(key, &params, sizeof(KP));
    memcpy(key + sizeof(KP), &grid, sizeof(int));
    memcpy(key + sizeof(KP) + sizeof(int), &fn, sizeof(void*));
    if (!b->exec || b->key_len != kl || memcmp(b->key, key, kl) != 0) {
        drop_exec(b);
        cudaStream_t cap;
        CKB(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        int r = cuda_err(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        if (!r) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(grid);
            cfg.blockDim = dim3(BB);
            cfg.dynamicSmemBytes = 0;
            cfg.stream = cap;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            void* args[] = {(void*)&params};
            r = cuda_err(cudaLaunchKernelExC(&cfg, fn, args));
            cudaError_t e = cudaStreamEndCapture(cap, &graph);
            if (!r) r = cuda_err(e);
        }
        if (!r) r = cuda_err(cudaGraphInstantiate(&b->exec, graph, 0));
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (r) {
            b->exec = nullptr;
            (void)cudaGetLastError();
            return r;
        }
        memcpy(b->key, key, kl);
        b->key_len = kl;
    }
    return cuda_err(cudaGraphLaunch(b->exec, st));
}

uint32_t gpad(uint32_t G) { return G <= 1 ? 1u : (G <= 2 ? 2u : (G <= 4 ? 4u : 8u)); }

int coop_grid(ip_graph* g, const void* fn) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, BB, 0) != cudaSuccess || occ < 1) {
        (void)cudaGetLastError();
        return 0;
    }
    return occ * g->num_sms;
}

int finish_stats(ip_graph* g, BatchState* b, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, uint32_t max_supersteps,
                 ip_batch_stats_t* stats, int* halted_out) {
    unsigned int hstate[4];
    unsigned long long hmsgs[4];
    GridBar hb;
    CKB(cudaMemcpyAsync(hstate, b->state, sizeof(hstate), cudaMemcpyDeviceToHost, st));
    CKB(cudaMemcpyAsync(hmsgs, b->msgs, sizeof(hmsgs), cudaMemcpyDeviceToHost, st));
    CKB(cudaMemcpyAsync(&hb, b->bar, sizeof(hb), cudaMemcpyDeviceToHost, st));
    CKB(cudaStreamSynchronize(st));
    if (hb.err) return IP_E_TIMEOUT;
    *halted_out = hstate[1] != 0;
    if (stats) {
        stats->supersteps = hstate[0];
        stats->halted = hstate[1] != 0;
        stats->messages = hmsgs[2];
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        stats->elapsed_ms = ms;
    }
    (void)g;
    (void)max_supersteps;
    return IP_OK;
}

}  // namespace

void free_batch_state(ip_graph* g) {
    if (!g->batch) return;
    BatchState* b = (BatchState*)g->batch;
    drop_exec(b);
    void* bufs[] = {b->dist, b->mbox, b->masks, b->tasks, b->small, b->msgs, b->state, b->bar, b->out_tmp, b->track};
    for (void* p : bufs)
        if (p) free_dev(p);
    delete b;
    g->batch = nullptr;
}

}  // namespace ipg

using namespace ipg;

extern "C" {

int ip_run_batch_sssp(ip_graph_t* g, const uint32_t* sources, uint32_t k, uint32_t* dist_out, int out_is_device,
                      uint32_t max_supersteps, ip_batch_stats_t* stats, void* stream) {
    if (!g || !sources || !dist_out || k == 0 || max_supersteps == 0) return IP_E_INVAL;
    if (k > IP_BATCH_MAX_SOURCES) return IP_E_RANGE;
    if (g->V >= 0x80000000u) return IP_E_RANGE;
    for (uint32_t i = 0; i < k; ++i)
        if (sources[i] >= g->V) return IP_E_RANGE;
    cudaStream_t st = (cudaStream_t)stream;
    BatchState* b = state_of(g);
    const uint32_t G = (k + 31) / 32;
    int r;
    if ((r = ensure_in_rows(g, st))) return r;  // the exchange reads the in-edge rows
    if (b->ms_G != G) {  // per-vertex storage for G groups of 32 sources
        for (void* p : {(void*)b->dist, (void*)b->mbox, (void*)b->masks}) {
            if (p) free_dev(p);
        }
        g->device_bytes -= b->bytes;
        b->dist = b->mbox = b->masks = nullptr;
        b->bytes = 0;
        const size_t per = (size_t)g->V * G * 32 * 4;
        if ((r = alloc_dev(g, (void**)&b->dist, per))) return r;
        if ((r = alloc_dev(g, (void**)&b->mbox, per))) return r;
        if ((r = alloc_dev(g, (void**)&b->masks, (size_t)g->V * gpad(G) * 4 * 3))) return r;
        b->bytes = 2 * per + (size_t)g->V * gpad(G) * 12;
        b->ms_G = G;
        drop_exec(b);
    }
    if (!b->tasks) {  // exchange tasks: every vertex's in-edges in runs of MS_CH
        std::vector<uint32_t> off((size_t)g->V + 1);
        CKB(cudaMemcpyAsync(off.data(), g->csc_off, off.size() * 4, cudaMemcpyDeviceToHost, st));
        CKB(cudaStreamSynchronize(st));
        std::vector<uint2> tasks;
        for (uint32_t v = 0; v < g->V; ++v) {
            const uint32_t d = off[v + 1] - off[v];
            const uint32_t flag = d > MS_CH ? 0x80000000u : 0u;
            for (uint32_t c = 0; c < d; c += MS_CH) tasks.push_back(make_uint2(v | flag, off[v] + c));
        }
        // largest tasks first (they are claimed in list order)
        auto len = [&](const uint2& t) {
            const uint32_t v = t.x & 0x7FFFFFFFu;
            return std::min(MS_CH, off[v + 1] - t.y);
        };
        std::stable_sort(tasks.begin(), tasks.end(), [&](const uint2& a, const uint2& b) { return len(a) > len(b); });
        if ((r = alloc_dev(g, (void**)&b->tasks, std::max<size_t>(tasks.size(), 1) * sizeof(uint2)))) return r;
        if (!tasks.empty())
            CKB(cudaMemcpyAsync(b->tasks, tasks.data(), tasks.size() * sizeof(uint2), cudaMemcpyHostToDevice, st));
        b->n_tasks = (uint32_t)tasks.size();
    }
    if ((r = ensure_small(g, b, 2 * (size_t)G * 32))) return r;
    CKB(cudaMemcpyAsync(b->small, sources, (size_t)k * 4, cudaMemcpyHostToDevice, st));
    if (g->new_of_old) {
        k_map_ids<<<(k + 255) / 256, 256, 0, st>>>(b->small, k, g->new_of_old);
        CKB(cudaGetLastError());
    }
    CKB(cudaMemsetAsync(b->msgs, 0, 4 * sizeof(unsigned long long), st));
    CKB(cudaMemsetAsync(b->bar, 0, sizeof(GridBar), st));

    MsParams P;
    memset(&P, 0, sizeof(P));
    P.V = g->V;
    P.G = G;
    P.K = k;
    P.csr_off = g->csr_off;
    P.csc_off = g->csc_off;
    P.csc_row = g->csc_row;
    P.csc_w = g->csc_w;
    P.tasks = b->tasks;
    P.n_tasks = b->n_tasks;
    P.sources = b->small;
    P.dist = b->dist;
    P.mbox = b->mbox;
    P.mask0 = b->masks;
    P.mask1 = b->masks + (size_t)g->V * gpad(G);
    P.rmask = b->masks + 2 * (size_t)g->V * gpad(G);
    P.src_last = b->small + (size_t)G * 32;
    P.msgs = b->msgs;
    P.state = b->state;
    P.bar = b->bar;
    P.limit_ns = stats && stats->barrier_timeout_ns ? stats->barrier_timeout_ns : 2000000000ull;
    P.max_supersteps = max_supersteps;
    const void* fns[8] = {(const void*)k_msssp<1, 1>, (const void*)k_msssp<2, 2>, (const void*)k_msssp<3, 4>,
                          (const void*)k_msssp<4, 4>, (const void*)k_msssp<5, 8>, (const void*)k_msssp<6, 8>,
                          (const void*)k_msssp<7, 8>, (const void*)k_msssp<8, 8>};
    const void* fn = fns[G - 1];
    const int grid = coop_grid(g, fn);
    if (grid <= 0) return IP_E_CUDA;
    CKB(cudaEventRecord(g->ev0, st));
    if ((r = launch_persistent(b, fn, P, grid, st))) return r;
    CKB(cudaEventRecord(g->ev1, st));
    int halted = 0;
    if ((r = finish_stats(g, b, st, g->ev0, g->ev1, max_supersteps, stats, &halted))) return r;
    // outputs: source-major distances, per-source supersteps
    uint32_t* out = dist_out;
    if (!out_is_device) {
        if ((r = ensure_out(g, b, (size_t)k * g->V))) return r;
        out = b->out_tmp;
    }
    const uint32_t tiles = ((g->V + 31) / 32) * G;
    k_ms_transpose<<<std::min<uint32_t>(tiles, (uint32_t)g->num_sms * 8), 256, 0, st>>>(b->dist, g->V, G, k, g->new_of_old, out);
    CKB(cudaGetLastError());
    if (!out_is_device)
        CKB(cudaMemcpyAsync(dist_out, out, (size_t)k * g->V * 4, cudaMemcpyDeviceToHost, st));
    if (stats && stats->instance_supersteps) {
        std::vector<uint32_t> last(k);
        CKB(cudaMemcpyAsync(last.data(), P.src_last, (size_t)k * 4, cudaMemcpyDeviceToHost, st));
        CKB(cudaStreamSynchronize(st));
        for (uint32_t i = 0; i < k; ++i) stats->instance_supersteps[i] = last[i] == NONE ? 1u : last[i] + 2u;
    }
    CKB(cudaStreamSynchronize(st));
    return halted ? IP_OK : IP_E_MAXSTEPS;
}

int ip_run_batch_hashmin(ip_graph_t* g, const uint32_t* instance_offsets, uint32_t k, uint32_t* labels_out,
                         int out_is_device, uint32_t max_supersteps, ip_batch_stats_t* stats, void* stream) {
    if (!g || !instance_offsets || !labels_out || k == 0 || max_supersteps == 0) return IP_E_INVAL;
    if (instance_offsets[0] != 0 || instance_offsets[k] != g->V) return IP_E_INVAL;
    for (uint32_t i = 0; i < k; ++i)
        if (instance_offsets[i + 1] < instance_offsets[i]) return IP_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    BatchState* b = state_of(g);
    int r;
    if ((r = ensure_bins(g, g->cur ? g->cur->t1 : DEFAULT_T1, g->cur ? g->cur->t2 : DEFAULT_T2, st))) return r;
    if ((r = ensure_in_rows(g, st))) return r;  // both engines pull over the in-edge rows
    if ((r = ensure_small(g, b, 2 * (size_t)k + 1))) return r;
    if (!stats || stats->engine == 0) {
        // the union runs through ip_run's device-driven superstep graph, recording last sends
        if (!b->track && (r = alloc_dev(g, (void**)&b->track, (size_t)g->V * 4))) return r;
        CKB(cudaMemcpyAsync(b->small, instance_offsets, ((size_t)k + 1) * 4, cudaMemcpyHostToDevice, st));
        ip_options_t o;
        ip_options_default(&o);
        o.stream = stream;
        const uint32_t cap = std::min<uint32_t>(max_supersteps, 1u << 16);
        std::vector<uint64_t> msgs(cap);
        ip_run_stats_t rs;
        memset(&rs, 0, sizeof(rs));
        rs.capacity = cap;
        rs.messages = msgs.data();
        g->track_send = b->track;
        r = run_app(g, APP_HM, max_supersteps, &o, &rs);
        g->track_send = nullptr;
        if (r != IP_OK && r != IP_E_MAXSTEPS) return r;
        uint32_t* inst_last = b->small + k + 1;
        const uint32_t* label = g->value;
        const uint32_t* track = b->track;
        if (g->new_of_old) {  // per-vertex records back to the caller's numbering
            int r2;  // r keeps the run's own status
            if (!g->snap_value && (r2 = alloc_dev(g, (void**)&g->snap_value, (size_t)g->V * 8))) return r2;
            if ((r2 = unpermute(g, g->value, g->snap_value, st))) return r2;
            if ((r2 = unpermute(g, b->track, g->snap_value + g->V, st))) return r2;
            label = g->snap_value;
            track = g->snap_value + g->V;
        }
        k_inst_max<<<std::min<uint32_t>(k, (uint32_t)g->num_sms * 8), BB, 0, st>>>(track, b->small, k, inst_last);
        uint32_t* out = labels_out;
        if (!out_is_device) {
            int r2 = ensure_out(g, b, g->V);
            if (r2) return r2;
            out = b->out_tmp;
        }
        k_local_labels<<<g->num_sms * 8, 256, 0, st>>>(label, g->V, b->small, k, out);
        CKB(cudaGetLastError());
        if (!out_is_device) CKB(cudaMemcpyAsync(labels_out, out, (size_t)g->V * 4, cudaMemcpyDeviceToHost, st));
        if (stats) {
            stats->supersteps = rs.supersteps;
            stats->halted = rs.halted;
            stats->elapsed_ms = rs.elapsed_ms;
            uint64_t tot = 0;
            for (uint32_t i = 0; i < std::min(rs.supersteps, cap); ++i) tot += msgs[i];
            stats->messages = tot;
            if (stats->instance_supersteps) {
                std::vector<uint32_t> last(k);
                CKB(cudaMemcpyAsync(last.data(), inst_last, (size_t)k * 4, cudaMemcpyDeviceToHost, st));
                CKB(cudaStreamSynchronize(st));
                for (uint32_t i = 0; i < k; ++i) stats->instance_supersteps[i] = last[i] == 0 ? 1u : last[i] + 1u;
            }
        }
        CKB(cudaStreamSynchronize(st));
        g->last_app = -1;
        return r;
    }
    CKB(cudaMemcpyAsync(b->small, instance_offsets, ((size_t)k + 1) * 4, cudaMemcpyHostToDevice, st));
    CKB(cudaMemsetAsync(b->small + k + 1, 0xFF, (size_t)k * 4, st));
    CKB(cudaMemsetAsync(b->msgs, 0, 4 * sizeof(unsigned long long), st));
    CKB(cudaMemsetAsync(b->bar, 0, sizeof(GridBar), st));
    BhParams P;
    memset(&P, 0, sizeof(P));
    P.V = g->V;
    P.W = g->W;
    P.csr_off = g->csr_off;
    P.csc_off = g->csc_off;
    P.csc_row = g->csc_row;
    P.bin = g->cur->b[1];
    P.t1 = g->cur->t1;
    P.label = g->value;
    P.outbox = g->outbox;
    P.mbox = g->mbox;
    P.recv = g->recv;
    P.inst_off = b->small;
    P.orig = g->old_of_new;
    P.nid = g->new_of_old;
    P.k = k;
    P.inst_last = b->small + k + 1;
    P.msgs = b->msgs;
    P.state = b->state;
    P.bar = b->bar;
    P.limit_ns = stats && stats->barrier_timeout_ns ? stats->barrier_timeout_ns : 2000000000ull;
    P.max_supersteps = max_supersteps;
    const void* fn = (const void*)k_bhashmin;
    const int grid = coop_grid(g, fn);
    if (grid <= 0) return IP_E_CUDA;
    CKB(cudaEventRecord(g->ev0, st));
    if ((r = launch_persistent(b, fn, P, grid, st))) return r;
    CKB(cudaEventRecord(g->ev1, st));
    int halted = 0;
    if ((r = finish_stats(g, b, st, g->ev0, g->ev1, max_supersteps, stats, &halted))) return r;
    uint32_t* out = labels_out;
    if (!out_is_device) {
        if ((r = ensure_out(g, b, g->V))) return r;
        out = b->out_tmp;
    }
    k_bh_local<<<g->num_sms * 8, 256, 0, st>>>(P, out);
    CKB(cudaGetLastError());
    if (!out_is_device) CKB(cudaMemcpyAsync(labels_out, out, (size_t)g->V * 4, cudaMemcpyDeviceToHost, st));
    if (stats && stats->instance_supersteps) {
        std::vector<uint32_t> last(k);
        CKB(cudaMemcpyAsync(last.data(), P.inst_last, (size_t)k * 4, cudaMemcpyDeviceToHost, st));
        CKB(cudaStreamSynchronize(st));
        for (uint32_t i = 0; i < k; ++i) stats->instance_supersteps[i] = last[i] == NONE ? 1u : last[i] + 2u;
    }
    CKB(cudaStreamSynchronize(st));
    g->last_app = -1;  // the handle's value array now holds union labels, not a run of ip_run
    return halted ? IP_OK : IP_E_MAXSTEPS;
}

}  // extern "C"
