/*
 * CPU ORACLE — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, single-threaded, synchronous Pregel engine and the three
 * applications of the iPregel paper, written for obvious correctness and not
 * for speed. Only the test suite, the smoke check and the benchmark's CPU
 * baseline use it; the GPU library never links, loads or calls it, and it
 * shares no code with the GPU library.
 *
 * Model (Section 4.2, Fig. 3 of the paper): execution proceeds in supersteps.
 * In a superstep every active vertex runs compute(); messages it sends become
 * visible to their recipients only in the next superstep; a global
 * synchronisation ends the superstep.
 *
 * Vertex selection (Section 4.3.1): a vertex runs in superstep s when
 *   (1) s is the first superstep, or
 *   (2) it has not voted to halt, or
 *   (3) it received a message during superstep s-1 (which also re-activates it).
 * The run ends once every vertex has halted and no message is in flight.
 *
 * Mailboxes (Section 4.3.3): one slot per vertex; a second message for the
 * same slot is folded in with the application's combine function as it
 * arrives. Two mailbox buffers separate the messages being read (sent in s-1)
 * from those being written (sent in s).
 *
 * Applications:
 *   PageRank   Fig. 8, with the constant term (1-d)/N of the Pregel version
 *              in Fig. 12; sum combiner; broadcasts value/out-degree while the
 *              superstep is below T, then votes to halt.
 *   Hashmin    Fig. 9; min combiner; always votes to halt.
 *   SSSP       Fig. 10, generalised to per-edge weights: the message along
 *              edge (u,v) is value(u) + w(u,v), saturating at INF
 *              (0xFFFFFFFF). With no weights every edge weighs 1, which is
 *              exactly Fig. 10.
 *   Reliability  (not in the paper; the library's example of an application
 *              added through its vertex-program interface) the most reliable
 *              path from a source: edge survival probability p = w(u,v)/256
 *              (1/256 without weights), FP32 value, message value(u) * p
 *              rounded to FP32, max combiner; written in the shape of Fig. 10
 *              with the comparison reversed.
 * A vertex with out-degree 0 broadcasts to nobody, so PageRank mass at
 * dangling vertices is dropped, as in the Pregel version (Fig. 12).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_INF 0xFFFFFFFFu

typedef struct {
    uint32_t supersteps; /* supersteps executed, superstep 0 included */
    int32_t halted;      /* 1: global halt reached; 0: the superstep cap stopped the run */
    uint32_t cap;        /* length of the arrays below (0 = do not record) */
    uint32_t* active;    /* per superstep: vertices that ran compute() */
    uint32_t* broadcasters; /* per superstep: vertices that called broadcast() */
    uint64_t* messages;  /* per superstep: messages sent */
    double* delta;       /* per superstep (PageRank, may be NULL): sum over vertices of
                            |rank after the superstep - rank before it| (0 for superstep 0) */
} oracle_stats;

/* ------------------------------------------------------------------ graph */
typedef struct {
    uint32_t n;
    const uint32_t* row_ptr; /* CSR out-edges */
    const uint32_t* col;
    const uint32_t* w; /* per-edge weights in CSR order, or NULL (all 1) */
} graph;

/* ---------------------------------------------------------- vertex record */
typedef struct {
    uint32_t id;
    uint32_t out_neighbour_count;
    int halted;
    double value_f; /* PageRank value */
    uint32_t value; /* Hashmin / SSSP value */
    float value_r;  /* Reliability value */
} vertex;

/* ------------------------------------------------------- engine contexts */
typedef struct engine engine;
typedef void (*compute_fn)(engine*, vertex*);

struct engine {
    graph g;
    vertex* vertices;
    uint32_t superstep;
    /* one-slot mailboxes: [0] read this superstep, [1] written this superstep */
    uint8_t* has_msg[2];
    double* box_f[2];
    uint32_t* box_u[2];
    float* box_r[2];
    int combiner; /* COMBINE_MIN_U32, COMBINE_SUM_F64 (PageRank) or COMBINE_MAX_F32 (Reliability) */
    uint8_t* consumed; /* the current message of a vertex was already read */
    /* per-superstep counters */
    uint32_t broadcasters;
    uint64_t messages;
    /* application parameters */
    double damping;
    uint32_t T;
    uint32_t source;
    /* PageRank to convergence: the run ends after the first superstep s >= 1 whose
     * L1 change (delta) is below tolerance; 0 disables the test */
    double tolerance;
    double delta;
};

enum { COMBINE_MIN_U32 = 0, COMBINE_SUM_F64 = 1, COMBINE_MAX_F32 = 2 };

/* Fig. 5: the min combiner. */
static void combine_min(uint32_t* old, uint32_t new_msg) {
    if (*old > new_msg) *old = new_msg;
}
/* Fig. 8: the sum combiner. */
static void combine_sum(double* old, double new_msg) { *old += new_msg; }
/* The max combiner over FP32 (Reliability). */
static void combine_max_f32(float* old, float new_msg) {
    if (new_msg > *old) *old = new_msg;
}

/* Delivery of one message into the recipient's next-superstep mailbox. */
static void deliver_u(engine* e, uint32_t dst, uint32_t msg) {
    if (!e->has_msg[1][dst]) {
        e->has_msg[1][dst] = 1;
        e->box_u[1][dst] = msg;
    } else {
        combine_min(&e->box_u[1][dst], msg);
    }
    e->messages++;
}
static void deliver_r(engine* e, uint32_t dst, float msg) {
    if (!e->has_msg[1][dst]) {
        e->has_msg[1][dst] = 1;
        e->box_r[1][dst] = msg;
    } else {
        combine_max_f32(&e->box_r[1][dst], msg);
    }
    e->messages++;
}
static void deliver_f(engine* e, uint32_t dst, double msg) {
    if (!e->has_msg[1][dst]) {
        e->has_msg[1][dst] = 1;
        e->box_f[1][dst] = msg;
    } else {
        combine_sum(&e->box_f[1][dst], msg);
    }
    e->messages++;
}

/* Runtime functions of Fig. 2. */
static uint32_t get_superstep(engine* e) { return e->superstep; }

static int get_next_message_u(engine* e, vertex* me, uint32_t* msg) {
    if (!e->has_msg[0][me->id] || e->consumed[me->id]) return 0;
    e->consumed[me->id] = 1;
    *msg = e->box_u[0][me->id];
    return 1;
}
static int get_next_message_r(engine* e, vertex* me, float* msg) {
    if (!e->has_msg[0][me->id] || e->consumed[me->id]) return 0;
    e->consumed[me->id] = 1;
    *msg = e->box_r[0][me->id];
    return 1;
}
static int get_next_message_f(engine* e, vertex* me, double* msg) {
    if (!e->has_msg[0][me->id] || e->consumed[me->id]) return 0;
    e->consumed[me->id] = 1;
    *msg = e->box_f[0][me->id];
    return 1;
}

/* broadcast: send msg to every out-neighbour. */
static void broadcast_f(engine* e, vertex* me, double msg) {
    e->broadcasters++;
    for (uint32_t k = e->g.row_ptr[me->id]; k < e->g.row_ptr[me->id + 1]; ++k) deliver_f(e, e->g.col[k], msg);
}
static void broadcast_u(engine* e, vertex* me, uint32_t msg) {
    e->broadcasters++;
    for (uint32_t k = e->g.row_ptr[me->id]; k < e->g.row_ptr[me->id + 1]; ++k) deliver_u(e, e->g.col[k], msg);
}
/* Weighted broadcast for SSSP: the message along edge k is base + w[k]
 * (w = 1 when the graph is unweighted), saturating at INF. */
static void broadcast_plus_weight(engine* e, vertex* me, uint32_t base) {
    e->broadcasters++;
    for (uint32_t k = e->g.row_ptr[me->id]; k < e->g.row_ptr[me->id + 1]; ++k) {
        uint64_t m = (uint64_t)base + (e->g.w ? e->g.w[k] : 1u);
        deliver_u(e, e->g.col[k], m >= ORACLE_INF ? ORACLE_INF : (uint32_t)m);
    }
}
/* Broadcast for Reliability: the message along edge k is base * p(k) in FP32,
 * p(k) = w[k] / 256 (w = 1 when the graph is unweighted; w * 2^-8 is exact). */
static void broadcast_times_probability(engine* e, vertex* me, float base) {
    e->broadcasters++;
    for (uint32_t k = e->g.row_ptr[me->id]; k < e->g.row_ptr[me->id + 1]; ++k) {
        const float p = (float)(e->g.w ? e->g.w[k] : 1u) * 0.00390625f;
        const float m = base * p;
        deliver_r(e, e->g.col[k], m);
    }
}
static void vote_to_halt(vertex* me) { me->halted = 1; }

/* ------------------------------------------------------- the three apps */
/* PageRank, Fig. 8 (ratio = (1-d)/N as in Fig. 12). */
static void compute_pagerank(engine* e, vertex* me) {
    const double N = (double)e->g.n;
    if (get_superstep(e) == 0) {
        me->value_f = 1.0 / N;
    } else {
        double sum = 0.0, msg;
        while (get_next_message_f(e, me, &msg)) sum += msg;
        const double old_value = me->value_f;
        me->value_f = (1.0 - e->damping) / N + e->damping * sum;
        e->delta += fabs(me->value_f - old_value);
    }
    if (get_superstep(e) < e->T) {
        if (me->out_neighbour_count > 0)
            broadcast_f(e, me, me->value_f / (double)me->out_neighbour_count);
        else
            e->broadcasters++; /* a broadcast to no neighbour sends nothing */
    } else {
        vote_to_halt(me);
    }
}

/* Hashmin connected components, Fig. 9. */
static void compute_hashmin(engine* e, vertex* me) {
    if (get_superstep(e) == 0) {
        me->value = me->id;
        broadcast_u(e, me, me->value);
    } else {
        uint32_t old_value = me->value, msg;
        while (get_next_message_u(e, me, &msg)) me->value = msg < me->value ? msg : me->value;
        if (me->value < old_value) broadcast_u(e, me, me->value);
    }
    vote_to_halt(me);
}

/* SSSP, Fig. 10 with per-edge weights. */
static void compute_sssp(engine* e, vertex* me) {
    if (get_superstep(e) == 0) {
        if (me->id == e->source) {
            me->value = 0;
            broadcast_plus_weight(e, me, me->value);
        } else {
            me->value = ORACLE_INF;
        }
    } else {
        uint32_t mindist = ORACLE_INF, msg;
        while (get_next_message_u(e, me, &msg)) mindist = msg < mindist ? msg : mindist;
        if (mindist < me->value) {
            me->value = mindist;
            broadcast_plus_weight(e, me, me->value);
        }
    }
    vote_to_halt(me);
}

/* Reliability: the source is certain and broadcasts; a larger combined
 * probability replaces the value and is broadcast. */
static void compute_reliability(engine* e, vertex* me) {
    if (get_superstep(e) == 0) {
        if (me->id == e->source) {
            me->value_r = 1.0f;
            broadcast_times_probability(e, me, me->value_r);
        } else {
            me->value_r = 0.0f;
        }
    } else {
        float best = 0.0f, msg;
        int got = 0;
        while (get_next_message_r(e, me, &msg)) {
            best = (!got || msg > best) ? msg : best;
            got = 1;
        }
        if (got && best > me->value_r) {
            me->value_r = best;
            broadcast_times_probability(e, me, me->value_r);
        }
    }
    vote_to_halt(me);
}

/* ---------------------------------------------------- superstep driver */
static int run(engine* e, compute_fn compute, uint32_t max_supersteps, oracle_stats* st) {
    const uint32_t n = e->g.n;
    int halted_globally = 0;
    uint32_t s;
    for (s = 0; s < max_supersteps; ++s) {
        e->superstep = s;
        e->broadcasters = 0;
        e->messages = 0;
        e->delta = 0.0;
        uint32_t active = 0;
        memset(e->consumed, 0, n);
        for (uint32_t v = 0; v < n; ++v) {
            vertex* me = &e->vertices[v];
            int selected = (s == 0) || !me->halted || e->has_msg[0][v];
            if (!selected) continue;
            me->halted = 0; /* a message re-activates a halted vertex */
            active++;
            compute(e, me);
        }
        if (st && s < st->cap) {
            st->active[s] = active;
            st->broadcasters[s] = e->broadcasters;
            st->messages[s] = e->messages;
            if (st->delta) st->delta[s] = e->delta;
        }
        /* convergence (PageRank with a tolerance): after the global synchronisation
         * of superstep s >= 1 the run ends when the ranks moved by less than the
         * tolerance in total; the broadcasts of s are never read */
        if (e->tolerance > 0.0 && s >= 1 && e->delta < e->tolerance) {
            halted_globally = 1;
            ++s;
            break;
        }
        /* global synchronisation: messages sent in s become readable in s+1 */
        uint8_t* th = e->has_msg[0];
        e->has_msg[0] = e->has_msg[1];
        e->has_msg[1] = th;
        memset(e->has_msg[1], 0, n);
        if (e->combiner == COMBINE_SUM_F64) {
            double* tf = e->box_f[0];
            e->box_f[0] = e->box_f[1];
            e->box_f[1] = tf;
        } else if (e->combiner == COMBINE_MAX_F32) {
            float* tr = e->box_r[0];
            e->box_r[0] = e->box_r[1];
            e->box_r[1] = tr;
        } else {
            uint32_t* tu = e->box_u[0];
            e->box_u[0] = e->box_u[1];
            e->box_u[1] = tu;
        }
        int all_halted = 1, in_flight = 0;
        for (uint32_t v = 0; v < n; ++v) {
            if (!e->vertices[v].halted) all_halted = 0;
            if (e->has_msg[0][v]) in_flight = 1;
        }
        if (all_halted && !in_flight) {
            halted_globally = 1;
            ++s;
            break;
        }
    }
    if (st) {
        st->supersteps = s;
        st->halted = halted_globally;
    }
    return halted_globally;
}

static int setup(engine* e, uint32_t n, const uint32_t* row_ptr, const uint32_t* col, const uint32_t* w,
                 int combiner) {
    memset(e, 0, sizeof(*e));
    e->g.n = n;
    e->g.row_ptr = row_ptr;
    e->g.col = col;
    e->g.w = w;
    e->combiner = combiner;
    size_t nn = n ? n : 1;
    e->vertices = (vertex*)calloc(nn, sizeof(vertex));
    e->consumed = (uint8_t*)calloc(nn, 1);
    for (int b = 0; b < 2; ++b) {
        e->has_msg[b] = (uint8_t*)calloc(nn, 1);
        if (combiner == COMBINE_SUM_F64)
            e->box_f[b] = (double*)calloc(nn, sizeof(double));
        else if (combiner == COMBINE_MAX_F32)
            e->box_r[b] = (float*)calloc(nn, sizeof(float));
        else
            e->box_u[b] = (uint32_t*)calloc(nn, sizeof(uint32_t));
    }
    if (!e->vertices || !e->consumed || !e->has_msg[0] || !e->has_msg[1]) return -1;
    for (uint32_t v = 0; v < n; ++v) {
        e->vertices[v].id = v;
        e->vertices[v].out_neighbour_count = row_ptr[v + 1] - row_ptr[v];
    }
    return 0;
}

static void teardown(engine* e) {
    free(e->vertices);
    free(e->consumed);
    for (int b = 0; b < 2; ++b) {
        free(e->has_msg[b]);
        free(e->box_f[b]);
        free(e->box_u[b]);
        free(e->box_r[b]);
    }
}

/* Public entry points. Return 1 on global halt, 0 when the cap stopped the
 * run, -1 on allocation failure. */
int oracle_pagerank(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, uint32_t T, double damping,
                    double tolerance, uint32_t max_supersteps, double* value_out, oracle_stats* st) {
    engine e;
    if (setup(&e, n, row_ptr, col, NULL, COMBINE_SUM_F64)) return -1;
    e.T = T;
    e.damping = damping;
    e.tolerance = tolerance;
    int r = run(&e, compute_pagerank, max_supersteps, st);
    for (uint32_t v = 0; v < n; ++v) value_out[v] = e.vertices[v].value_f;
    teardown(&e);
    return r;
}

int oracle_hashmin(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, uint32_t max_supersteps,
                   uint32_t* value_out, oracle_stats* st) {
    engine e;
    if (setup(&e, n, row_ptr, col, NULL, COMBINE_MIN_U32)) return -1;
    int r = run(&e, compute_hashmin, max_supersteps, st);
    for (uint32_t v = 0; v < n; ++v) value_out[v] = e.vertices[v].value;
    teardown(&e);
    return r;
}

int oracle_sssp(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, const uint32_t* w, uint32_t source,
                uint32_t max_supersteps, uint32_t* value_out, oracle_stats* st) {
    engine e;
    if (setup(&e, n, row_ptr, col, w, COMBINE_MIN_U32)) return -1;
    e.source = source;
    int r = run(&e, compute_sssp, max_supersteps, st);
    for (uint32_t v = 0; v < n; ++v) value_out[v] = e.vertices[v].value;
    teardown(&e);
    return r;
}

/* One superstep s >= 1 of PageRank (Fig. 8 with the constant of Fig. 12) for the
 * vertices [v_begin, v_end), written from the receiving side: in superstep s-1
 * every in-neighbour u of v broadcast prev_rank[u] / out_degree[u] (u has at
 * least one out-edge, the one to v), the sum combiner added those messages, and
 * compute() takes (1-d)/N + d * sum. in_ptr / in_src are the in-edge arrays.
 * out[v - v_begin] receives the new rank. Independent vertices: any split of the
 * range gives the same values. Used to check one superstep of a graph too large
 * for a whole oracle run, and to time bounded samples of a run. */
void oracle_pagerank_superstep(uint32_t n, const uint32_t* in_ptr, const uint32_t* in_src,
                               const uint32_t* out_degree, const double* prev_rank, double damping,
                               uint32_t v_begin, uint32_t v_end, double* out) {
    const double base = (1.0 - damping) / (double)n;
    for (uint32_t v = v_begin; v < v_end; ++v) {
        double sum = 0.0;
        for (uint32_t k = in_ptr[v]; k < in_ptr[v + 1]; ++k) {
            const uint32_t u = in_src[k];
            sum += prev_rank[u] / (double)out_degree[u];
        }
        out[v - v_begin] = base + damping * sum;
    }
}

int oracle_reliability(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, const uint32_t* w, uint32_t source,
                       uint32_t max_supersteps, float* value_out, oracle_stats* st) {
    engine e;
    if (setup(&e, n, row_ptr, col, w, COMBINE_MAX_F32)) return -1;
    e.source = source;
    int r = run(&e, compute_reliability, max_supersteps, st);
    for (uint32_t v = 0; v < n; ++v) value_out[v] = e.vertices[v].value_r;
    teardown(&e);
    return r;
}

/* One superstep s >= 1 of Hashmin (Fig. 9) for the vertices [v_begin, v_end),
 * written from the receiving side: the in-neighbours u of v with bcast[u] != 0
 * broadcast prev_label[u] in superstep s-1, the min combiner folded them, and
 * compute() keeps the smaller of the vertex's label and that minimum.
 * out_label[v - v_begin] receives the new label; out_recv[v - v_begin] (may be
 * NULL) whether v received a message (and so ran compute()). Used to time a
 * bounded sample of a Hashmin run and to check single supersteps. */
void oracle_hashmin_superstep(uint32_t n, const uint32_t* in_ptr, const uint32_t* in_src, const uint32_t* prev_label,
                              const uint8_t* bcast, uint32_t v_begin, uint32_t v_end, uint32_t* out_label,
                              uint8_t* out_recv) {
    (void)n;
    for (uint32_t v = v_begin; v < v_end; ++v) {
        uint32_t m = ORACLE_INF;
        int got = 0;
        for (uint32_t k = in_ptr[v]; k < in_ptr[v + 1]; ++k) {
            const uint32_t u = in_src[k];
            if (!bcast[u]) continue;
            got = 1;
            if (prev_label[u] < m) m = prev_label[u];
        }
        out_label[v - v_begin] = (got && m < prev_label[v]) ? m : prev_label[v];
        if (out_recv) out_recv[v - v_begin] = (uint8_t)got;
    }
}
