// Device helpers shared by the superstep kernels of every translation unit:
// lane arithmetic, aligned 16-byte edge loads, broadcast bitmaps by superstep
// parity, warp-aggregated queue appends, compensated FP32 sums, and the block
// reduction of the per-superstep frontier statistics.
#pragma once

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
// The first index of this warp in a grid-stride loop over a work list that comes
// after `skip` warps' worth of earlier lists (the heavy vertices' CTAs, the medium
// vertices): the warps those lists keep busy take this one last, so that on small
// graphs the lists run side by side instead of one after another. A rotation of
// the warps, so every item is still taken exactly once.
__device__ __forceinline__ uint32_t rotated_warp(uint64_t skip) {
    const uint32_t nw = num_warps();
    return (uint32_t)((global_warp() + nw - (uint32_t)(skip % nw)) % nw);
}
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
static __device__ void flush_stats(Stats st, DevCtl* ctl) {
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

}  // namespace ipg
