// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ipregel.h"
#include "../../include/ipregel_program.cuh"

namespace ipg {

constexpr uint32_t INF = 0xFFFFFFFFu;
constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr int APP_PR = IP_PAGERANK, APP_HM = IP_HASHMIN, APP_SSSP = IP_SSSP;
constexpr int N_FEATURES = 8;
constexpr uint32_t MAX_SEQ = 64;
constexpr int BLOCK = 256;  // threads per CTA for every superstep kernel
constexpr uint32_t DEFAULT_T1 = 16;
constexpr uint32_t DEFAULT_T2 = 1024;
constexpr uint32_t HCH = 4096;  // edges per heavy-vertex chunk (one CTA pass: 256 threads x 4 blocks x 4)

// Device control block: the counters the kernels of one superstep fill, and the
// decision the selector kernel takes after it. Lives in device memory; the host
// reads it back only in the host-driven loop.
struct DevCtl {
    // statistics of the superstep being completed (filled by init / apply kernels)
    unsigned int n_active;  // vertices that ran compute()
    unsigned int n_bcast;   // vertices that broadcast
    unsigned long long msgs;  // messages sent = sum of out-degrees of broadcasters
    unsigned int max_deg;   // largest out-degree among broadcasters
    unsigned int rq_len;    // recipient queue length (push-sparse)
    unsigned int q_len[2][3];  // broadcaster queue lengths [superstep parity][small, medium, heavy]
    unsigned int q_valid;   // the queues of the last completed superstep hold exactly its bcast bitmap
    // decision state (owned by the selector kernel)
    unsigned int superstep; // superstep being computed; at selector time, the one just completed
    unsigned int mode;      // mode of the next exchange
    unsigned int mode_used; // mode of the exchange that delivered into `superstep`
    unsigned int done;      // 0 running, 1 halted, 2 superstep cap reached
    unsigned int err;       // device-side error bits
    unsigned int prev_bcast;
    unsigned int pr_stale;  // PageRank: the broadcasts of the last superstep were not written (blocked pull)
    unsigned long long t_prev;  // %globaltimer at the previous selector call
    double pr_delta;        // PageRank with a tolerance: sum over vertices of |rank change| this superstep
    unsigned int n_pull;    // pull exchanges of this run (the blocked min pull is built once they add up)
};

// One record per superstep, written by the selector kernel.
struct LogRec {
    unsigned int mode;
    unsigned int active;
    unsigned int bcast;
    unsigned int max_deg;
    unsigned long long msgs;
    float feat[N_FEATURES];
    float pr_delta;  // PageRank: L1 rank change of the superstep (tolerance runs; 0 otherwise)
};

// Learned selector parameters on the device (layout of IP_SELECTOR_BYTES).
struct SelectorDev {
    float mu[8], sd[8];
    uint16_t W1[32 * 8], W2[32 * 32], W3[3 * 32];
    float b1[32], b2[32], b3[3];
};
static_assert(sizeof(SelectorDev) == IP_SELECTOR_BYTES, "selector layout");

// Static degree bins of one edge direction (CSR out-edges or CSC in-edges).
// small: deg <= t1 (handled lane-per-vertex inside 32-vertex tiles);
// med:   t1 < deg < t2 (warp per vertex);
// heavy: deg >= t2, split into chunks of at most HCH edges (CTA per chunk).
struct Bins {
    const uint32_t* med;
    uint32_t n_med;
    uint32_t n_hchunk;
    const uint4* hchunk;  // {vertex, first edge, end edge, heavy-vertex index}
    const uint2* hvert;   // per heavy vertex: {first chunk, chunk count}
    uint32_t n_hvert;
    uint32_t* hcnt;       // per heavy vertex: chunk arrival counter (PageRank finish), kept at 0 between launches
    float2* hpart;        // per chunk: compensated partial sum (PageRank)
};

// Blocked PageRank pull (pb.cu): the edges are stored once more, grouped by
// source chunk and, inside a chunk, by destination bin. Phase 1 streams every
// chunk and writes its sources' broadcasts next to the entries; phase 2
// accumulates every bin in shared memory. Device pointers of that layout.
constexpr uint32_t PB_BIN_V = 24576;  // most destinations per bin (one 32-bit accumulator word each in shared memory)
constexpr uint64_t PB_AUTO_EDGES = 1ull << 24;  // IP_PR_ENGINE_AUTO picks the blocked pull from this many edges
// ... and for min programs from this many: at R-MAT 20 (31M edges) their gather pull was
// 7-15% faster, at R-MAT 21 (64M) even, at R-MAT 22-23 (128-259M) 8-18% slower
constexpr uint64_t PB_MIN_AUTO_EDGES = 1ull << 26;
// A min program's AUTO pull switches to the blocked layout once the handle has run this
// many pull exchanges with the gather kernel (two Hashmin runs on R-MAT graphs): a handle
// that is run again and again then pays the build once (at R-MAT 26 it costs about as
// much as ten gather exchanges, and every later exchange is 1.6x faster), while a
// handle run once or twice never builds it
constexpr uint64_t PB_MIN_BUILD_PULLS = 6;
struct PbDev {
    uint32_t on;             // 1: PageRank pull runs on this layout
    uint32_t n_chunks, n_tasks;
    const uint4* chunk;      // [n_chunks] {first source, sources, first run, end run}
    const uint4* runs;       // {chunk-major first entry, bin-major first entry, length padded to 4, 0},
                             // by chunk then bin
    const uint16_t* src;     // chunk-major: source minus the first source of its chunk (padding: source count)
    const uint16_t* dst;     // [entries] bin-major: destination minus the first vertex of its bin (padding 0)
    uint32_t* code;          // [entries] bin-major: the source's broadcast as a fixed-point code (padding 0)
    const uint8_t* w8;       // chunk-major: the entry's edge weight (graphs whose weights are below 256;
                             // null otherwise), for the pull of PB_MIN_ADD_WEIGHT programs
    unsigned long long* big; // [V] fixed-point broadcasts of 2^31 units or more (code = 2^31 | source)
    const uint4* tasks;      // per bin {first vertex, vertices, first entry, end entry}, in bin order
    uint32_t* hi;            // [V] high words of the fixed-point sums, zero between launches
    uint32_t* ctr;           // [2] task counters of phase 1 and phase 2
    int32_t shift;           // S: a contribution v is added as round(v * 2^S)
    float inv_scale;         // 2^-S
};

// Everything a superstep kernel needs, passed by value.
struct Params {
    uint32_t V;
    uint32_t W;      // bitmap words, padded to a multiple of 32
    uint64_t E;
    const uint32_t* csr_off;
    const uint32_t* csr_col;
    const uint32_t* csr_w;
    const uint32_t* csc_off;
    const uint32_t* csc_row;
    const uint32_t* csc_w;
    Bins bout, bin;  // degree bins of the CSR and of the CSC
    const float* inv_outdeg;
    uint32_t* value;
    float* rank;
    float* contrib0;
    float* contrib1;
    uint32_t* mbox;
    uint32_t* outbox;  // broadcast slot: the value of a vertex that broadcast in the last superstep, else INF
    float* mboxf;
    uint32_t* recv;
    uint32_t* bcast0;  // broadcast bitmap of even supersteps
    uint32_t* bcast1;  // broadcast bitmap of odd supersteps
    uint32_t* rq;
    uint32_t* q[2][2];  // broadcaster queues [parity][small, medium]
    uint2* hq[2];       // heavy broadcaster chunks [parity]: {vertex, chunk index}
    DevCtl* ctl;
    uint32_t* last_send;  // optional [V]: 1 + last superstep in which the vertex sent a message (0 = never)
    LogRec* log;
    uint32_t log_cap;
    const SelectorDev* sel;
    uint32_t t1, t2;
    float thr_sparse, thr_pull;
    uint32_t app, T, source, max_supersteps;
    float damping, pr_base;  // pr_base = (1-d)/N rounded to float
    float pr_tol;            // PageRank to convergence: halt once the L1 rank change is below this (0: off)
    uint32_t pull_early_exit;  // unit-weight SSSP: pull stops at the first broadcasting in-neighbour
    int32_t policy, forced_mode;
    uint32_t seq_len;
    uint8_t seq[MAX_SEQ];
    uint32_t max_out_deg;
    uint32_t out_deg_src;
    int32_t use_graph;
    cudaGraphConditionalHandle h_while, h_switch;
    PbDev pb;
    const uint32_t* orig;  // renumbered graph: internal id -> caller's id (Hashmin labels are caller ids), else null
};

// PageRank (Fig. 8) in the terms of the vertex-program interface: a sum combiner
// (FP32, atomicAdd in the push exchange), compute() forming the rank from the
// combined sum, and the broadcast rank / out-degree. Every vertex is active for T
// supersteps, so PageRank runs in its own engines (the CSC gather and the blocked
// pull below, the push in superstep.cu), which all take these three pieces.
struct PageRankProgram {
    using Combiner = ipregel::SumCombiner<float>;
    using Value = float;
    // (1-d)/N + d * sum, with base = (1-d)/N rounded to FP32
    __device__ static float compute(float damping, float base, float sum) { return fmaf(damping, sum, base); }
    // the message of a vertex that broadcasts: rank / out-degree (0 for a vertex without out-edges)
    __device__ static float message(float rank, float inv_outdeg) { return rank * inv_outdeg; }
};

// PageRank compute() of superstep s (Fig. 8): rank from the sum of the received
// broadcasts, then broadcast rank / out-degree while s < T. With a tolerance, the
// rank's change is added to the calling thread's L1 partial dacc.
__device__ __forceinline__ void pr_finish(const Params& P, uint32_t v, float sum, uint32_t s, float* nxt,
                                          float& dacc) {
    const float r = PageRankProgram::compute(P.damping, P.pr_base, sum);
    if (P.pr_tol > 0.f) dacc += fabsf(r - P.rank[v]);
    P.rank[v] = r;
    nxt[v] = s < P.T ? PageRankProgram::message(r, P.inv_outdeg[v]) : 0.0f;
}

// Adds the calling warp's L1 partials to the superstep's rank change (all 32 lanes
// call; nothing when no tolerance is set).
__device__ __forceinline__ void flush_delta(const Params& P, float dacc) {
    if (!(P.pr_tol > 0.f)) return;
    for (int o = 16; o > 0; o >>= 1) dacc += __shfl_down_sync(0xFFFFFFFFu, dacc, o);
    if ((threadIdx.x & 31u) == 0 && dacc != 0.f) atomicAdd(&P.ctl->pr_delta, (double)dacc);
}

// Degree bins of both directions for one (t1, t2) pair, with their device buffers.
struct BinSet {
    uint32_t t1 = 0, t2 = 0;
    Bins b[2] = {};  // [0] CSR, [1] CSC
    void* mem[2][5] = {};
    size_t bytes[2][5] = {};
    uint64_t last_use = 0;
};

// One instantiated superstep graph, keyed by the kernel parameters it bakes in.
struct ExecEntry {
    unsigned char key[sizeof(Params)];
    cudaGraphExec_t exec;
    cudaGraph_t graph;
    uint64_t last_use;
};

}  // namespace ipg

struct ip_graph {
    int device = 0;
    int num_sms = 0;
    uint32_t V = 0;
    uint64_t E = 0;
    uint32_t W = 0;
    uint32_t* csr_off = nullptr;
    uint32_t* csr_col = nullptr;
    uint32_t* csr_w = nullptr;
    uint32_t* csc_off = nullptr;
    uint32_t* csc_row = nullptr;
    uint32_t* csc_w = nullptr;
    bool csc_alias = false;
    bool csc_rows_pending = false;  // csc_off built, csc_row / csc_w not yet (directed graphs)
    bool weighted = false;
    bool max_w_known = false;  // max_w holds the largest edge weight (graph_max_weight)
    uint32_t max_w = 0;
    uint32_t max_out_deg = 0, max_in_deg = 0;
    float* inv_outdeg = nullptr;
    std::vector<ipg::BinSet*> binsets;  // degree bins cached by (t1, t2), at most 4
    ipg::BinSet* cur = nullptr;          // the set of the current run
    // run state
    uint32_t* value = nullptr;
    float* rank = nullptr;
    float* contrib[2] = {nullptr, nullptr};
    uint32_t* mbox = nullptr;
    uint32_t* outbox = nullptr;
    float* mboxf = nullptr;
    uint32_t* recv = nullptr;
    uint32_t* bcast[2] = {nullptr, nullptr};
    uint32_t* rq = nullptr;
    uint32_t* q[2][2] = {};
    uint2* hq[2] = {nullptr, nullptr};  // capacity: heavy chunks of the CSR (allocated with the bins)
    uint32_t hq_cap = 0;
    ipg::DevCtl* ctl = nullptr;
    ipg::DevCtl* ctl_host = nullptr;  // pinned mirror
    ipg::LogRec* log = nullptr;
    uint32_t log_cap = 0;
    ipg::SelectorDev* sel = nullptr;
    bool has_selector = false;
    int last_app = -1;
    uint64_t device_bytes = 0;
    // scratch used by label collection (snapshots)
    uint32_t* snap_value = nullptr;

    // instantiated superstep graphs of recent runs, at most 8
    std::vector<ipg::ExecEntry> execs;
    uint64_t use_clock = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int grid[16] = {0};
    bool grids_ready = false;
    void* batch = nullptr;        // state of the batched runs (batch.cu)
    uint32_t* track_send = nullptr;  // when set, runs record per-vertex last sends here (batched Hashmin)
    void* pb = nullptr;              // blocked PageRank pull layout (pb.cu), built on first use
    uint32_t* bin_cnt = nullptr;     // [3] device counters of the degree-bin builder
    uint32_t* new_of_old = nullptr;  // renumbered graph (ip_graph_relabel): caller's id -> internal id
    uint32_t* old_of_new = nullptr;  // internal id -> caller's id
    uint64_t pull_gathered = 0;      // pull exchanges of min programs run by the gather kernel on this handle
};

namespace ipg {
// graph.cu
int alloc_dev(ip_graph* g, void** p, size_t bytes);
void free_dev(void* p);
int ensure_bins(ip_graph* g, uint32_t t1, uint32_t t2, cudaStream_t st);
int ensure_in_rows(ip_graph* g, cudaStream_t st);  // the transposed rows, if creation deferred them
int exclusive_scan(ip_graph* g, uint32_t* data, uint64_t n, cudaStream_t st);  // in place, n uint32
int cuda_err(cudaError_t e);
// batch.cu
void free_batch_state(ip_graph* g);
// pb.cu
int pb_prepare(ip_graph* g, cudaStream_t st, PbDev* out);
int pb_launch(const ip_graph* g, const Params& P, cudaStream_t st);
// Blocked pull of a min program: kind PB_MIN_COPY (the codes are the broadcast slots) or
// PB_MIN_ADD_WEIGHT (broadcast + the entry's weight, 1 on unweighted graphs).
enum { PB_MIN_COPY = 1, PB_MIN_ADD_WEIGHT = 2 };
int pb_min_launch(const ip_graph* g, const Params& P, cudaStream_t st, int kind);
// Largest edge weight of a weighted graph, computed once (g->max_w).
int graph_max_weight(ip_graph* g, cudaStream_t st);
int pb_set_mode(ip_graph* g, int min_mode, cudaStream_t st);  // neutral tail codes: 0 PageRank, 1 min programs
bool pb_supported(const ip_graph* g);
void pb_free(ip_graph* g);
size_t pb_bytes(const ip_graph* g);  // device bytes of the blocked layout (0 if not built)
int unpermute(const ip_graph* g, const uint32_t* in, uint32_t* out, cudaStream_t st);
// superstep.cu
struct ProgramOps;
const ProgramOps* program_ops(int app);  // the vertex program registered as app, or null
int run_app(ip_graph* g, int app, uint32_t max_supersteps, const ip_options_t* opt, ip_run_stats_t* stats);
void free_graph_exec(ip_graph* g);
}  // namespace ipg
