/*
 * ipregel.h — C ABI of the GB300 (sm_103a) synchronous vertex-centric superstep
 * library (libipregel_gb300.so).
 *
 * The library runs the superstep model of the iPregel paper (Capelli et al.,
 * "iPregel: Vertex-centric programmability vs memory efficiency and
 * performance, why choose?", Parallel Computing 2019): Section 4.2 and Fig. 3
 * (bulk-synchronous supersteps: compute, communicate, synchronise), with the
 * optimisations of Section 4.3 (selection bypass, push or pull message
 * exchange, combined one-slot mailboxes) for its three applications:
 * PageRank (Fig. 8, sum combiner), Hashmin connected components (Fig. 9, min
 * combiner) and single-source shortest paths (Fig. 10, min combiner, here with
 * per-edge uint32 weights).
 *
 * Conventions shared by every entry point:
 *  - Every function returns int: IP_OK (0) or a negative IP_E_* code. No C++
 *    exception crosses this boundary.
 *  - Vertex IDs are uint32 in [0, n_vertices); edge offsets are uint32, so a
 *    graph holds at most 2^32 - 1 directed edges.
 *  - An ip_graph_t owns all device memory it uses. Caller buffers are only read
 *    (or written, for outputs) during the call and never retained.
 *  - `stream` arguments are cudaStream_t values passed as void*; NULL means the
 *    legacy default stream. Calls that return results synchronise that stream
 *    before returning.
 *  - Handles are not thread safe: one thread at a time per handle.
 */
#ifndef IPREGEL_H
#define IPREGEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define IP_OK 0
#define IP_E_INVAL (-1)         /* malformed argument or graph (offsets, sizes, NULL) */
#define IP_E_RANGE (-2)         /* a vertex ID, size or count out of range */
#define IP_E_NOMEM (-3)         /* a device allocation failed */
#define IP_E_CUDA (-4)          /* a CUDA runtime call failed */
#define IP_E_TIMEOUT (-5)       /* a bounded device-side wait gave up */
#define IP_E_MAXSTEPS (-6)      /* the superstep cap stopped the run before global halt;
                                   the values hold the state after the last superstep run */
#define IP_E_DEVICE_ASSERT (-7) /* a device-side check recorded an error */
#define IP_E_STATE (-8)         /* the call is not valid in the handle's current state */

/* ------------------------------------------------------------ enumerations */
typedef enum {
    IP_PAGERANK = 0, /* Fig. 8 (constant (1-d)/N as in Fig. 12); FP32 ranks */
    IP_HASHMIN = 1,  /* Fig. 9; uint32 labels */
    IP_SSSP = 2,     /* Fig. 10 with message value(u) + w(u,v); uint32 distances,
                        unreachable = 0xFFFFFFFF */
    IP_RELIABILITY = 3 /* not in the paper: most reliable path from ip_options_t.source, written
                          against the vertex-program interface (include/ipregel_program.cuh);
                          edge survival probability w(u,v) / 256 (1/256 without weights);
                          FP32 value = the largest product of probabilities over the paths
                          from the source, products taken along the path from the source
                          (max combiner, CAS-combined); 0 where unreachable */
} ip_app_t;

/* How the messages broadcast in superstep s reach their recipients in s+1
 * (Section 4.3.2): pushed along out-edges by the senders, from a compacted
 * queue of senders (PUSH_SPARSE, the selection bypass of Section 4.3.1) or by
 * scanning a sender bitmap over all vertices (PUSH_DENSE); or pulled by every
 * vertex from its in-neighbours' broadcast values (PULL). The vertex values
 * after every superstep do not depend on the mode. */
typedef enum { IP_MODE_PUSH_SPARSE = 0, IP_MODE_PUSH_DENSE = 1, IP_MODE_PULL = 2 } ip_mode_t;

typedef enum {
    IP_POLICY_AUTO = 0,      /* the threshold rule (the learned selector is IP_POLICY_MLP: it gains
                                on some graph shapes and loses 0.2-1.7% on R-MAT 22 and 26) */
    IP_POLICY_THRESHOLD = 1, /* fixed rule on the frontier's out-edge fraction (see ip_options_t) */
    IP_POLICY_MLP = 2,       /* the learned selector; IP_E_STATE if none is loaded. A superstep whose
                                frontier sends fewer than thr_sparse * E messages takes PUSH_SPARSE
                                without running the network (the threshold rule's sparse region) */
    IP_POLICY_FORCED = 3,    /* always forced_mode */
    IP_POLICY_SEQUENCE = 4   /* exchange into superstep s uses mode_sequence[(s-1) % len] */
} ip_policy_t;

/* How a PULL exchange runs, for PageRank and for the vertex programs that allow
 * the blocked layout (Hashmin; SSSP on graphs whose weights are below 256 and
 * whose vertex count times the largest weight is below 2^32 - 1, unweighted
 * graphs included; the others always GATHER). Both engines compute the same
 * combined messages; they differ in how the in-neighbours' broadcasts reach the
 * destination. */
typedef enum {
    IP_PR_ENGINE_AUTO = 0,    /* PageRank: BLOCKED on graphs of at least 2^24 edges that it supports,
                                 else GATHER. Hashmin and SSSP: GATHER until the handle has run 6
                                 gather pulls of either (a handle that is run again and again),
                                 BLOCKED from then on (or whenever the layout already exists) on
                                 graphs of at least 2^26 edges */
    IP_PR_ENGINE_GATHER = 1,  /* every in-edge of the CSC reads its source's broadcast */
    IP_PR_ENGINE_BLOCKED = 2  /* two streaming passes over a second edge layout built on first use
                                 (8 bytes per edge, 9 on weighted graphs whose weights are below
                                 256): the sources' broadcasts are written out per
                                 edge, grouped by destination bin, and every bin is summed in shared
                                 memory in 64-bit fixed point; IP_E_RANGE on graphs of more than
                                 339,738,624 vertices */
} ip_pr_engine_t;

typedef struct ip_graph ip_graph_t;

/* Options of one run. Fill with ip_options_default() and override fields. */
typedef struct {
    float damping;                /* PageRank damping d (default 0.85) */
    uint32_t pr_iterations;       /* PageRank T: broadcasts while superstep < T (default 30) */
    uint32_t source;              /* SSSP source vertex (default 0) */
    int32_t policy;               /* ip_policy_t (default IP_POLICY_AUTO) */
    int32_t forced_mode;          /* ip_mode_t for IP_POLICY_FORCED */
    const uint8_t* mode_sequence; /* host array of ip_mode_t for IP_POLICY_SEQUENCE */
    uint32_t mode_sequence_len;   /* 1..64 */
    uint32_t t1;                  /* degree cutoff: deg <= t1 is handled by one lane (0 = default) */
    uint32_t t2;                  /* degree cutoff: deg >= t2 is handled by a whole CTA (0 = default);
                                     between the two a warp handles the vertex */
    float thr_sparse;             /* threshold rule: f = out-edges of senders / E; f < thr_sparse
                                     -> PUSH_SPARSE, f >= thr_pull -> PULL, else PUSH_DENSE */
    float thr_pull;
    int32_t use_graph;            /* 1 (default): the whole run is one CUDA graph whose superstep
                                     loop runs on the device (conditional while/switch nodes);
                                     0: the host drives the loop, one 4-byte readback per superstep */
    int32_t collect_labels;       /* 1: also time all three modes in every superstep (host loop);
                                     fills ip_run_stats_t.mode_ms. Values are unchanged. */
    int32_t profile_kernels;      /* 1: host loop with CUDA events around every kernel; fills
                                     ip_run_stats_t.kernel_ms. Values are unchanged. */
    void* stream;                 /* cudaStream_t */
    int32_t pr_engine;            /* ip_pr_engine_t: the PULL engine of PageRank, Hashmin and SSSP
                                     (default IP_PR_ENGINE_AUTO) */
    float pr_tolerance;           /* PageRank to convergence (the paper's Section 6.1 notes that a
                                     real PageRank runs until convergence): > 0 ends the run after
                                     the first superstep s >= 1 whose L1 rank change
                                     sum_v |rank_s(v) - rank_(s-1)(v)| is below it (summed in FP32
                                     per thread, FP64 across threads); T still caps the run.
                                     0 (default): T updates exactly. */
    int32_t pull_early_exit;      /* unit-weight SSSP (no weights given: Fig. 10 exactly), PULL mode:
                                     1 (default) stops scanning a vertex's in-edges at the first one
                                     whose source broadcast in the last superstep — all of them
                                     carry the same distance under synchronous supersteps, so the
                                     result is the same; 0 scans every in-edge. Ignored otherwise. */
} ip_options_t;

/* Per-run statistics. The caller owns the arrays; `capacity` is their length in
 * supersteps (entries for supersteps >= capacity are dropped). Any array
 * pointer may be NULL. */
typedef struct {
    uint32_t supersteps;   /* supersteps executed, superstep 0 included */
    int32_t halted;        /* 1: global halt; 0: the cap stopped the run */
    uint32_t capacity;
    uint8_t* mode;         /* [s]: mode that delivered the messages read in superstep s
                              (255 for superstep 0) */
    uint32_t* active;      /* [s]: vertices that ran compute() in superstep s */
    uint32_t* broadcasters;/* [s]: vertices that broadcast in superstep s */
    uint64_t* messages;    /* [s]: messages sent in superstep s */
    float* features;       /* [8*s + i]: selector input computed after superstep s */
    float* mode_ms;        /* [3*s + m]: milliseconds of mode m delivering into superstep s
                              (collect_labels only; 0 otherwise) */
    float* kernel_ms;      /* [4*s + k]: milliseconds of the kernels that computed superstep s:
                              k = 0 queue compaction, 1 exchange, 2 apply, 3 selector
                              (profile_kernels only; 0 for kernels that did not run) */
    float elapsed_ms;      /* device time of the whole run (init to halt) */
    float* pr_delta;       /* [s]: PageRank with pr_tolerance > 0: L1 rank change of superstep s
                              (0 for superstep 0 and for runs without a tolerance) */
} ip_run_stats_t;

/* Graph facts for callers and tests. */
typedef struct {
    uint32_t n_vertices;
    uint64_t n_edges;
    uint32_t max_out_degree;
    uint32_t max_in_degree;
    uint32_t csc_is_csr;      /* 1 when the in-edge arrays alias the out-edge arrays */
    uint32_t weighted;
    uint32_t num_sms;         /* SMs of the device the graph lives on */
    uint64_t device_bytes;    /* device memory held by the handle, the sum of the parts below */
    /* Where those bytes go (the analogue of the paper's memory-footprint study,
     * Section 7.2 and Table 3; the combined one-slot mailbox of Section 4.3.3 is
     * one 4-byte word per vertex): */
    uint64_t bytes_graph;         /* CSR and CSC offsets, indices and weights (the CSC shares
                                     the CSR's arrays for a symmetric graph; a CSC built on
                                     the device holds its offsets only until a run reads
                                     its rows) */
    uint64_t bytes_vertex_state;  /* per-vertex values, ranks, broadcast slots, mailboxes,
                                     out-degree reciprocals, bitmaps and frontier queues */
    uint64_t bytes_degree_bins;   /* degree-binned schedules of both edge directions (every
                                     cached cutoff pair) */
    uint64_t bytes_blocked_layout;/* the blocked PageRank pull's second edge layout (0 until a
                                     run builds it) */
    uint64_t bytes_renumbering;   /* the two vertex maps of ip_graph_relabel */
    uint64_t bytes_other;         /* batched-run state, run logs, selector, control block */
} ip_graph_info_t;

/* ------------------------------------------------------------ entry points */

/* Sets every field of *opt to its default. */
void ip_options_default(ip_options_t* opt);

/* Creates a graph on the current CUDA device (Section 4.2: the vertex array and
 * the adjacency array of the paper become a CSR (out-edges) and a CSC (in-edges)
 * store).
 *   n_vertices   >= 1.
 *   n_edges      number of directed edges, < 2^32.
 *   csr_offsets  n_vertices+1 offsets (offsets[0] = 0, non-decreasing,
 *                offsets[n] = n_edges); csr_cols n_edges destination IDs.
 *   csr_weights  n_edges weights in CSR order, or NULL (unweighted: every
 *                edge weighs 1 for SSSP).
 *   csc_offsets / csc_rows / csc_weights  the in-edge (transposed) arrays in the
 *                same form; NULL csc_offsets means "build the transpose on the
 *                device": its offsets at creation, its rows and weights at the
 *                first run that reads them (a pull on the gather engine, a batched
 *                run; a run that cannot allocate them returns IP_E_NOMEM and leaves
 *                the graph as it was; runs that pull on the blocked engine never
 *                need them); csc_offsets == csr_offsets and csc_rows == csr_cols
 *                declares a symmetric graph and shares the arrays. csc_weights
 *                is required when csc arrays and csr_weights are both given.
 *   flags        IP_CREATE_DEVICE_PTRS: all arrays are device memory (else all are
 *                host memory; 0 and 1 keep their old meaning); IP_CREATE_RELABEL:
 *                renumber the vertices by degree class as part of creation, exactly as
 *                ip_graph_create followed by ip_graph_relabel, except that the in-edges
 *                and degree bins are built once, for the renumbered graph. Other bits:
 *                IP_E_INVAL.
 * Host arrays are validated on the host (IP_E_INVAL / IP_E_RANGE); device
 * arrays by a device check (same codes). The library copies every array.
 * A CSC that is not the transpose of the CSR is not detected: pull mode then
 * computes on the CSC's edges. */
#define IP_CREATE_DEVICE_PTRS 1
#define IP_CREATE_RELABEL 2
int ip_graph_create(ip_graph_t** out, uint32_t n_vertices, uint64_t n_edges, const uint32_t* csr_offsets,
                    const uint32_t* csr_cols, const uint32_t* csr_weights, const uint32_t* csc_offsets,
                    const uint32_t* csc_rows, const uint32_t* csc_weights, int flags, void* stream);

/* Releases the graph store and the run state of the handle (the vertex and
 * edge arrays of Section 4.2, the mailboxes of Section 4.3.3 and everything the
 * library built for them). Synchronises the graph's device once; the buffers go
 * to the library's device-buffer cache (ip_release_cached_memory). NULL is
 * ignored; the handle must not be used afterwards. */
void ip_graph_destroy(ip_graph_t* g);

/* Facts of the graph and of the device memory its handle holds (struct above).
 * IP_E_INVAL for a NULL argument. */
int ip_graph_info(const ip_graph_t* g, ip_graph_info_t* info);

/* Renumbers the graph's vertices inside the handle by decreasing out-degree
 * class (class = floor(log2 out-degree), vertices without out-edges last; the
 * original order is kept inside a class), on the device. The paper keeps the
 * caller's numbering (Section 4.2); the renumbering only changes where a vertex's
 * state sits in memory, so that the high-degree vertices the pull exchanges gather
 * from share cache lines. It is invisible through the ABI: sources, instance
 * offsets, Hashmin labels (smallest CALLER id of the component), distances and
 * ranks stay in the caller's numbering, and every result is the one of the graph
 * as given. Costs: two n_vertices uint32 maps, one more copy of the edges while it
 * runs, and a gather on every ip_get_values. Every cached state of the handle
 * (degree bins, run graphs, blocked-engine layout, batched-run state) is rebuilt;
 * the values of a previous run are dropped (IP_E_STATE until the next run).
 * A second call is a no-op. Returns IP_E_NOMEM (the handle is then unusable and
 * must only be destroyed) or IP_E_CUDA on failure. Synchronises the device (the
 * buffers of the old numbering go back to the library's cache). */
int ip_graph_relabel(ip_graph_t* g, void* stream);

/* Runs one application to global halt (Section 4.2: the run ends when every
 * vertex has voted to halt and no message is in flight) or until
 * max_supersteps supersteps (superstep 0 included) have run, whichever comes
 * first; returns IP_E_MAXSTEPS in the second case. PageRank halts after
 * superstep T = opt->pr_iterations (T+1 supersteps). opt may be NULL
 * (defaults). stats may be NULL. The values stay on the device until
 * ip_get_values or the next run. */
int ip_run(ip_graph_t* g, ip_app_t app, uint32_t max_supersteps, const ip_options_t* opt,
           ip_run_stats_t* stats);

/* Copies the result of the last run: the vertex values once the run has ended
 * (Section 4.2: global halt, when every vertex has voted to halt and no message
 * is in flight; or the superstep cap): n_vertices FP32 ranks (PageRank, Fig. 8)
 * or uint32 labels (Hashmin, Fig. 9) / distances (SSSP, Fig. 10), indexed by the
 * caller's vertex ids. dst is host memory (dst_is_device = 0) or device memory
 * (1) the caller owns; dst_bytes must be >= 4 * n_vertices (IP_E_RANGE).
 * Synchronises the stream. IP_E_STATE if nothing has run yet, or after a batched
 * Hashmin run (which uses the value array as scratch). */
int ip_get_values(ip_graph_t* g, void* dst, size_t dst_bytes, int dst_is_device, void* stream);

/* Loads the learned mode selector (a trained 8-32-32-3 MLP) into the handle.
 * blob layout (little endian, IP_SELECTOR_BYTES bytes):
 *   float  mu[8], sd[8]          feature normalisation
 *   bf16   W1[32][8], W2[32][32], W3[3][32]   (row-major, output-major)
 *   float  b1[32], b2[32], b3[3]
 * bytes must equal IP_SELECTOR_BYTES. */
#define IP_SELECTOR_BYTES (16 * 4 + (32 * 8 + 32 * 32 + 3 * 32) * 2 + (32 + 32 + 3) * 4)
int ip_set_selector(ip_graph_t* g, const void* blob, size_t bytes);

/* ---------------------------------------------------------- batched runs
 * Many independent runs in one persistent launch (not in the paper, whose runs
 * are one at a time): one cooperative kernel holds the whole superstep loop
 * (Section 4.2), its phases separated by a grid-wide barrier whose every wait is
 * bounded (IP_E_TIMEOUT when a wait runs out; the kernel then exits), launched
 * through a CUDA graph. Each run keeps the synchronous semantics of ip_run. */
#define IP_BATCH_MAX_SOURCES 256
typedef struct {
    uint32_t supersteps;            /* supersteps of the batch (its longest run), superstep 0 included */
    int32_t halted;                 /* 1: every run halted; 0: the superstep cap stopped the batch */
    uint64_t messages;              /* messages sent, all runs */
    uint32_t* instance_supersteps;  /* caller array of k entries, or NULL: supersteps each run
                                       takes on its own (as ip_run would report) */
    float elapsed_ms;               /* device time of the persistent launch */
    uint64_t barrier_timeout_ns;    /* input: bound of every barrier wait; 0 = 2 seconds */
    int32_t engine;                 /* input, Hashmin batches: 0 = the device-driven superstep graph
                                       of ip_run (all exchange modes, default), 1 = the persistent
                                       cooperative pull kernel */
} ip_batch_stats_t;

/* SSSP (Fig. 10, weighted) from k sources at once on one graph: distances are held
 * per vertex for all sources, so one read of an in-edge serves every source.
 *   sources   k host uint32 vertex IDs, 1 <= k <= IP_BATCH_MAX_SOURCES.
 *   dist_out  k x n_vertices uint32, source-major (dist_out[i*n + v]), host or device
 *             memory per out_is_device; INF = 0xFFFFFFFF for unreachable vertices.
 * Returns IP_OK, IP_E_MAXSTEPS, IP_E_TIMEOUT, IP_E_RANGE (k or a source out of range). */
int ip_run_batch_sssp(ip_graph_t* g, const uint32_t* sources, uint32_t k, uint32_t* dist_out, int out_is_device,
                      uint32_t max_supersteps, ip_batch_stats_t* stats, void* stream);

/* Hashmin (Fig. 9) on k independent graphs held as one block-diagonal graph g,
 * in one launch (engine 0: one CUDA-graph launch whose superstep loop runs on the
 * device; engine 1: one persistent cooperative kernel):
 * instance i owns vertices [instance_offsets[i], instance_offsets[i+1]) and no edge
 * crosses instances (not checked).
 *   instance_offsets  k+1 host uint32, from 0 to n_vertices, non-decreasing.
 *   labels_out        n_vertices uint32, label of each vertex as an ID local to its
 *                     instance (host or device memory per out_is_device).
 * The handle's value array is used as scratch: ip_get_values returns IP_E_STATE after. */
int ip_run_batch_hashmin(ip_graph_t* g, const uint32_t* instance_offsets, uint32_t k, uint32_t* labels_out,
                         int out_is_device, uint32_t max_supersteps, ip_batch_stats_t* stats, void* stream);

/* ---------------------------------------------------------- selector training
 * Kernels that train the learned mode selector (not in the paper: the paper
 * chooses push or pull with a compile flag, Section 4.3.2). The network is the
 * 8-32-32-3 MLP loaded by ip_set_selector:
 *   xn = (x - mu)/sd, h1 = relu(W1 xn + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3,
 * loss = sum_i w_i (logsumexp(z_i) - z_i[y_i]) / weight_total.
 * params: IP_MLP_PARAMS FP32 masters in the order W1[32][8], b1[32], W2[32][32],
 * b2[32], W3[3][32], b3[3] (row-major, output-major); the weights are rounded to
 * BF16 (nearest even) inside every pass, accumulation is FP32, and gradients
 * flow to the FP32 masters. mu_sd: mu[8] then sd[8]. X: n x 8 features, y: n
 * labels in {0,1,2}, w: n sample weights. All pointers are DEVICE memory; the
 * caller owns every buffer, including the workspace of the backward pass
 * (ip_mlp_workspace_bytes() bytes). Gradients are summed in a fixed order:
 * repeated calls give identical results. */
#define IP_MLP_PARAMS (32 * 8 + 32 + 32 * 32 + 32 + 3 * 32 + 3)
size_t ip_mlp_workspace_bytes(void);
/* logits: n x 3 FP32 outputs. */
int ip_mlp_forward(const float* params, const float* mu_sd, const float* X, uint32_t n, float* logits, void* stream);
/* grad: IP_MLP_PARAMS FP32 outputs; loss: one FP32 output (may be NULL). */
int ip_mlp_backward(const float* params, const float* mu_sd, const float* X, const int32_t* y, const float* w,
                    uint32_t n, float weight_total, float* grad, float* loss, void* workspace,
                    size_t workspace_bytes, void* stream);
/* One Adam step on `count` parameters (step >= 1; bias-corrected). */
int ip_mlp_adam(float* params, const float* grad, float* m, float* v, uint32_t count, float lr, float beta1,
                float beta2, float eps, uint32_t step, void* stream);
/* Writes the IP_SELECTOR_BYTES selector blob (device memory) from the FP32 masters. */
int ip_mlp_pack(const float* params, const float* mu_sd, void* blob, void* stream);

/* Hashmin connected components without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory, for example code running inside another
 * framework's memory pool or under a fixed memory budget. It computes exactly
 * what ip_run(IP_HASHMIN) computes (same labels, same superstep count), keeping
 * all of its temporary state in one fixed array inside the library image
 * (about 4.4 MiB per device that loads the library, held until exit).
 *   n_vertices     1 .. IP_NOALLOC_MAX_VERTICES; larger graphs give IP_E_RANGE.
 *   csr_offsets / csr_cols   the out-edge CSR, DEVICE memory, not modified.
 *   labels         n_vertices uint32 outputs, DEVICE memory.
 *   supersteps_out host pointer or NULL: supersteps run, superstep 0 included.
 * Returns IP_OK at global halt, IP_E_MAXSTEPS at the cap. The input is checked
 * on the device: offsets that do not start at 0, decrease, or do not end at
 * n_edges give IP_E_INVAL before any edge is read; an edge whose destination is
 * not below n_vertices is skipped and the call returns IP_E_RANGE (labels are
 * then unspecified). The first call on a device looks up the array's device address;
 * make that first call before any stream capture. All calls on a device share
 * the array: calls that overlap on the GPU race and give wrong results. */
#define IP_NOALLOC_MAX_VERTICES (1u << 20)
int ip_hashmin_noalloc(uint32_t n_vertices, uint64_t n_edges, const uint32_t* csr_offsets, const uint32_t* csr_cols,
                       uint32_t* labels, uint32_t max_supersteps, uint32_t* supersteps_out, void* stream);

/* Device memory. A graph's device buffers come from a process-wide cache kept by
 * the library: ip_graph_destroy synchronises the graph's device and returns the
 * buffers to the cache (at most a quarter of the device's memory, up to 64 GiB,
 * stay cached), and an allocation of the same size on the same device reuses one,
 * so building graphs of the same shape again and again allocates once. An allocation that fails releases the cache of its
 * device and retries. The paper has no counterpart (its graphs are built once).
 * ip_release_cached_memory frees every cached buffer on every device and returns
 * IP_OK; the cache is guarded by a lock, so any thread may call it. */
int ip_release_cached_memory(void);

/* Human-readable text for an IP_* code (static storage). */
const char* ip_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* IPREGEL_H */
