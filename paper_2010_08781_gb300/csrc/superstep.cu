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
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "engine.cuh"
#include "kernel_util.cuh"

namespace ipg {

// =========================================================== PageRank superstep 0
// PageRank superstep 0 (Fig. 8): value = 1/N, broadcast value / out-degree.
__global__ void k_pr_init(Params P) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const float r0 = 1.0f / (float)P.V;
    for (uint32_t v = tid; v < P.V; v += nth) {
        P.rank[v] = r0;
        P.contrib0[v] = P.T > 0 ? PageRankProgram::message(r0, P.inv_outdeg[v]) : 0.0f;
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
    const uint64_t hw = (uint64_t)min(B.n_hchunk, gridDim.x) * (blockDim.x / 32);  // warps on heavy chunks
    for (uint32_t i = rotated_warp(hw); i < B.n_med; i += num_warps()) {
        const uint32_t v = B.med[i];
        float a = 0.f, c = 0.f;
        pr_gather(P.csc_row, cur, P.csc_off[v], P.csc_off[v + 1], lane_id(), 32, a, c);
        warp_two_sum(a, c);
        if (lane_id() == 0) pr_finish(P, v, a + c, s, nxt, dacc);
    }
    const uint32_t tiles = (P.V + 31) / 32;
    for (uint32_t t = rotated_warp(hw + B.n_med); t < tiles; t += num_warps()) {
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
                if (blk < be && ei >= b && ei < e)
                    ipregel::combine_atomic<PageRankProgram::Combiner>(P.mboxf + qa(qc[u], j), x);  // atomicAdd
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
        cur[v] = sent ? PageRankProgram::message(P.rank[v], P.inv_outdeg[v]) : 0.0f;  // as pr_finish
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
    const uint64_t hw = (uint64_t)min(B.n_hchunk, gridDim.x) * (blockDim.x / 32);  // warps on heavy chunks
    for (uint32_t i = rotated_warp(hw); i < B.n_med; i += num_warps()) {
        const uint32_t u = B.med[i];
        pr_scatter(P, cur[u], P.csr_off[u], P.csr_off[u + 1], lane_id(), 32);
    }
    const uint32_t tiles = (P.V + 31) / 32;
    for (uint32_t t = rotated_warp(hw + B.n_med); t < tiles; t += num_warps()) {
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

// One warp: 8 -> 32 -> 32 -> 3 MLP, BF16 weights, FP32 accumulation. Lane j owns
// hidden unit j of both layers. A lane's parameters (its W1 row as one 16-byte
// load, its W2 row as four, its W3 column, biases, and the feature normalisation
// by lanes 0-7) are loaded by mlp_load at the start of k_select, so their L2 round
// trip overlaps the one for the superstep's counters; the arithmetic and its order
// are those of the training forward pass (ip_mlp_forward), so the logits are
// identical.
static_assert(offsetof(SelectorDev, W1) % 16 == 0 && offsetof(SelectorDev, W2) % 16 == 0, "16-byte weight rows");
struct MlpLane {
    uint4 w1;
    uint4 w2[4];
    float b1, b2, b3m, mu, sd;
    uint16_t w3[3];
};
__device__ __forceinline__ MlpLane mlp_load(const SelectorDev* S) {
    const uint32_t j = lane_id();
    MlpLane L;
    L.w1 = __ldg(reinterpret_cast<const uint4*>(S->W1) + j);  // W1[j][0..7]
#pragma unroll
    for (int q = 0; q < 4; ++q) L.w2[q] = __ldg(reinterpret_cast<const uint4*>(S->W2 + j * 32) + q);  // W2[j][8q..]
    L.b1 = __ldg(S->b1 + j);
    L.b2 = __ldg(S->b2 + j);
#pragma unroll
    for (int m = 0; m < 3; ++m) L.w3[m] = __ldg(S->W3 + m * 32 + j);
    L.b3m = j < 3 ? __ldg(S->b3 + j) : 0.f;
    L.mu = j < 8 ? __ldg(S->mu + j) : 0.f;
    L.sd = j < 8 ? __ldg(S->sd + j) : 1.f;
    return L;
}
__device__ int mlp_mode(const MlpLane& L, const float* f) {
    const uint4 w1 = L.w1;
    const uint4* w2 = L.w2;
    const float b1 = L.b1, b2 = L.b2, b3m = L.b3m, mu = L.mu, sd = L.sd;
    const uint16_t* w3 = L.w3;
    float xn[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) xn[i] = (f[i] - __shfl_sync(FULL, mu, i)) / __shfl_sync(FULL, sd, i);
    auto lo = [](uint32_t w) { return __uint_as_float(w << 16); };          // element 2t of a pair
    auto hi = [](uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); };  // element 2t + 1
    const uint32_t r1[4] = {w1.x, w1.y, w1.z, w1.w};
    float h1 = b1;
#pragma unroll
    for (int i = 0; i < 8; ++i) h1 = fmaf((i & 1) ? hi(r1[i >> 1]) : lo(r1[i >> 1]), xn[i], h1);
    h1 = fmaxf(h1, 0.f);
    float h2 = b2;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const uint4 q = w2[k >> 3];
        const uint32_t pair = (k & 7) < 2 ? q.x : (k & 7) < 4 ? q.y : (k & 7) < 6 ? q.z : q.w;
        h2 = fmaf((k & 1) ? hi(pair) : lo(pair), __shfl_sync(FULL, h1, k), h2);
    }
    h2 = fmaxf(h2, 0.f);
    float z[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        float p = bf16f(w3[m]) * h2;
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(FULL, p, o);
        z[m] = p + __shfl_sync(FULL, b3m, m);
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
    MlpLane mlp{};
    if (P.policy == IP_POLICY_MLP) mlp = mlp_load(P.sel);  // in flight while the counters load
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
        case IP_POLICY_MLP:  // below the sparse cutoff every policy takes push-sparse: no inference there
            mode = f[6] < P.thr_sparse ? IP_MODE_PUSH_SPARSE : mlp_mode(mlp, f);
            break;
        default:
            mode = f[6] < P.thr_sparse ? IP_MODE_PUSH_SPARSE : (f[6] >= P.thr_pull ? IP_MODE_PULL : IP_MODE_PUSH_DENSE);
    }
    if (P.app == APP_PR && mode == IP_MODE_PUSH_SPARSE) mode = IP_MODE_PUSH_DENSE;  // every vertex broadcasts
    if (!done && mode == IP_MODE_PULL && threadIdx.x == 0) ++c->n_pull;
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

static_assert(ipregel::has_hw_atomic<PageRankProgram::Combiner>::value, "the PageRank push combines with atomicAdd");

// ================================================================ host side
// Vertex programs registered by the app_*.cu translation units (static
// initialisation; the table is zero-initialised before any of it runs).
static const ProgramOps* g_programs[MAX_APPS];

void register_program(int app, const ProgramOps* ops) {
    if (app >= 0 && app < MAX_APPS && app != APP_PR) g_programs[app] = ops;
}

const ProgramOps* program_ops(int app) { return app >= 0 && app < MAX_APPS ? g_programs[app] : nullptr; }

namespace {

int grid_of(const ip_graph* g, const void* fn) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, BLOCK, 0) != cudaSuccess || occ < 1) {
        (void)cudaGetLastError();
        occ = 2;
    }
    return g->num_sms * occ;
}

enum { G_PR_PULL, G_PR_PUSH, G_MISC, G_COUNT };

// Grid sizes of the PageRank kernels (resident CTAs per SM x SMs), queried once per
// handle, outside any capture; the vertex programs size their own (engine.cuh).
void compute_grids(ip_graph* g) {
    if (g->grids_ready) return;
    const void* fns[G_COUNT] = {(const void*)k_pr_pull, (const void*)k_pr_push, (const void*)k_pr_apply};
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
    const ProgramOps* ops = program_ops((int)P.app);
    if (!ops) return IP_E_INVAL;
    return ops->superstep(g, P, mode, st, ev);
}

int launch_init(const ip_graph* g, const Params& P, cudaStream_t st) {
    if (P.app == APP_PR) {
        k_pr_init<<<g->grid[G_MISC], BLOCK, 0, st>>>(P);
    } else {
        const ProgramOps* ops = program_ops((int)P.app);
        if (!ops) return IP_E_INVAL;
        const int r = ops->init(g, P, st);
        if (r != IP_OK) return r;
    }
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
    const ProgramOps* ops = app == APP_PR ? nullptr : program_ops(app);
    if (app != APP_PR && !ops) return IP_E_INVAL;
    if (ops && ops->uses_source && o.source >= g->V) return IP_E_RANGE;
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
    if (ops) CKR(ops->prepare(g));

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
    if (ops && ops->uses_source && g->new_of_old)  // the caller's source id -> internal id
        CKR(cuda_err(cudaMemcpyAsync(&P.source, g->new_of_old + o.source, 4, cudaMemcpyDeviceToHost, st)));
    P.max_supersteps = max_supersteps;
    P.damping = o.damping;
    P.pr_base = (float)((1.0 - (double)o.damping) / (double)g->V);
    P.pr_tol = app == APP_PR ? o.pr_tolerance : 0.f;
    P.pull_early_exit = (ops && !g->weighted && o.pull_early_exit) ? 1u : 0u;  // used by programs that allow it
    // AUTO is the threshold rule: on R-MAT 22 and 26 graphs the learned selector picks the
    // same modes or slightly slower ones, and its inference costs a few microseconds
    P.policy = o.policy == IP_POLICY_AUTO ? IP_POLICY_THRESHOLD : o.policy;
    P.forced_mode = o.forced_mode;
    P.seq_len = o.policy == IP_POLICY_SEQUENCE ? o.mode_sequence_len : 1;
    if (o.policy == IP_POLICY_SEQUENCE) memcpy(P.seq, o.mode_sequence, o.mode_sequence_len);
    P.max_out_deg = g->max_out_deg;
    if (ops && ops->uses_source && g->new_of_old) CKR(cuda_err(cudaStreamSynchronize(st)));  // the mapped source
    const bool use_graph = o.use_graph && !o.collect_labels && !o.profile_kernels;
    P.use_graph = use_graph ? 1 : 0;
    if (app == APP_PR) {
        const bool blocked = o.pr_engine == IP_PR_ENGINE_BLOCKED ||
                             (o.pr_engine == IP_PR_ENGINE_AUTO && g->E >= PB_AUTO_EDGES && pb_supported(g));
        if (blocked) {
            const int r = pb_prepare(g, st, &P.pb);
            // AUTO keeps the gather engine where the layout does not fit (entries beyond 2^32)
            if (r != IP_OK && !(r == IP_E_RANGE && o.pr_engine == IP_PR_ENGINE_AUTO)) return r;
            if (P.pb.on) CKR(pb_set_mode(g, 0, st));
        }
    } else if (ops->blocked_kind) {
        // the blocked pull of a min program: forced, or (AUTO) once the layout exists or this
        // handle's gather pulls have cost about as much as building it (PB_MIN_BUILD_PULLS).
        // A program that adds the edge weight needs weights below 256 (one byte per entry in
        // the layout) and V x the largest weight below the no-broadcast pattern.
        bool fits = true;
        if (ops->blocked_kind == PB_MIN_ADD_WEIGHT && g->weighted) {
            CKR(graph_max_weight(g, st));
            fits = g->max_w <= 255 && (uint64_t)g->V * g->max_w < 0xFFFFFFFFull;
        }
        const bool blocked = fits && (o.pr_engine == IP_PR_ENGINE_BLOCKED ||
                                      (o.pr_engine == IP_PR_ENGINE_AUTO && g->E >= PB_MIN_AUTO_EDGES && pb_supported(g) &&
                                       (g->pb || g->pull_gathered >= PB_MIN_BUILD_PULLS)));
        if (blocked) {
            const int r = pb_prepare(g, st, &P.pb);
            if (r != IP_OK && !(r == IP_E_RANGE && o.pr_engine == IP_PR_ENGINE_AUTO)) return r;
            if (P.pb.on && ops->blocked_kind == PB_MIN_ADD_WEIGHT && g->weighted && !P.pb.w8) P.pb.on = 0;
            if (P.pb.on) CKR(pb_set_mode(g, 1, st));
        }
    }

    // the in-edge rows (built now if creation deferred them), unless every pull of this
    // run streams the blocked layout (the push exchanges read the out-edges)
    if (!P.pb.on) {
        CKR(ensure_in_rows(g, st));
        P.csc_row = g->csc_row;
        P.csc_w = g->csc_w;
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
    if (ops && ops->blocked_kind && !P.pb.on) g->pull_gathered += c.n_pull;
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
