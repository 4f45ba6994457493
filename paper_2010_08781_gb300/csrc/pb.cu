// Blocked PageRank pull.
//
// The PULL exchange of PageRank (Section 4.3: every vertex combines the
// broadcasts of its in-neighbours with the sum combiner, Fig. 8) reads one
// broadcast per in-edge at a random address. On this GPU a random 4-byte load
// costs one L1 pass of its own, about one per SM clock even when the line is in
// L2, so a CSC gather cannot go faster than that however the work is scheduled.
// This engine moves every random access into shared memory, after the
// propagation-blocking idea (Beamer, Asanovic and Patterson, IPDPS 2017):
//
//   layout (built once per graph): the out-edges are cut into chunks of
//   consecutive sources (at most PB_MAXS sources, about E / 4096 out-edges,
//   clamped to [PB_CHUNK_MIN, PB_CHUNK_MAX]: longer chunks give longer runs), the
//   vertices into bins of consecutive destinations (at most PB_BIN_V vertices and
//   about E / (4 x phase-2 CTAs) in-edges, so that every bin is a balanced task).
//   A run is the edges of one chunk into one bin, padded to a multiple of 4
//   entries (padding adds 0). Every entry is stored twice: its source relative
//   to the chunk (u16) in chunk-major order (chunk, then bin), its destination
//   relative to the bin (u16) and its code in bin-major order (bin, then chunk).
//   A run is contiguous in both orders.
//   phase 1 (k_pb_scatter): a CTA stages its chunk's broadcasts in shared
//   memory as fixed-point codes, then copies every run: sources read in order,
//   codes written to the run's place in its bin. Chunks go in index order, so
//   the runs of neighbouring chunks (neighbours in every bin) are written close
//   in time and their shared sectors meet in L2.
//   phase 2 (k_pb_accumulate): a CTA owns one bin, streams its codes and
//   destinations through asynchronous copies into shared memory and adds every
//   code into a shared-memory accumulator of its destination, then runs
//   compute() (pr_finish) for the bin's vertices.
//
// The accumulators are 64-bit fixed point (2^-S units: the low 32-bit word in
// shared memory, the high word in global memory, an explicit carry between
// them), so the sums are exact integer sums: independent of the order of the
// additions, and deterministic. S = min(62, 29 + ceil(log2 V)) keeps the total
// below 2^64 (ranks sum to at most 1) and the rounding of one contribution below
// 2^-(S+1), under 1e-8 of the smallest rank (1-d)/V; a typical contribution
// rank / out-degree ~ 1 / (V deg) stays below 2^31 units, the size of a code.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"

namespace ipg {
namespace {

constexpr uint32_t PB_MAXS = 16384;      // sources per chunk: their codes fit 64 KB of shared memory
constexpr uint32_t PB_CHUNK_MIN = 65536, PB_CHUNK_MAX = 262144;  // target out-edges per chunk
constexpr uint32_t PB_MAX_BINS = 16384;  // bins a chunk histograms in shared memory
constexpr uint32_t PB_MAX_V = 13824u * PB_BIN_V;  // vertex-capped bins plus entry-capped ones fit PB_MAX_BINS
constexpr int PB1_THREADS = 512, PBB_THREADS = 512;
// k_pb_place: one CTA of 1024 threads per SM (its shared memory is padded to
// PBP_MIN_SMEM): each CTA writes its chunk's runs, spread over about 0.5 MB, as
// its edges come; with 152 chunks in flight those writes stay in L2 until their
// sectors are complete instead of leaving it half written and being read back.
constexpr int PBP_THREADS = 1024;
constexpr size_t PBP_MIN_SMEM = 120 * 1024;
// phase 1: groups of 4 entries per lane in flight (PageRank's scatter / the min programs')
constexpr int PB1_LOADS_PR = 6, PB1_LOADS_MIN = 4;
constexpr int PB_BATCH = 8;          // per-vertex loops (staging, compute()): loads in flight per thread
constexpr int PB2_CONSUMERS = 24;    // phase 2: consumer warps (plus one producer warp)
constexpr int PB_GROUPS = 2;        // phase 2: groups of 4 entries per consumer thread and stage
constexpr uint32_t PB_TILE = 4 * PB_GROUPS * 32 * PB2_CONSUMERS;  // entries per stage (6144)
constexpr int PB_STAGES = 3;         // phase 2: stages of the bulk-copy ring (108 KB)
constexpr size_t PB1_SMEM = (PB_MAXS + 1) * sizeof(uint32_t);
// k_pb_scatter's dynamic shared memory, padded so that two CTAs share an SM: at R-MAT 26
// two chunks in flight per SM took 68.05 ms for T = 30 against 69.78 ms with three
// (and 76.2 ms with one); the depth of loads in flight mattered less (4-12 groups within 0.7%)
constexpr size_t PB1_SMEM_PR = 80 * 1024;
// k_pbm_scatter's: three CTAs per SM measured best; 6 groups of loads in flight instead of
// 4 made R-MAT 22's pulls 1-3% faster but Hashmin at R-MAT 26 2-3% slower (kept at 4)
constexpr size_t PB1_SMEM_MIN = PB1_SMEM;
constexpr size_t PB2_SMEM = PB_BIN_V * sizeof(uint32_t) + (size_t)PB_STAGES * PB_TILE * (4 + 2) +
                            PB_STAGES * (32 + 16);

// v * 2^S as a 64-bit integer (xl, xh), rounded half up, from the bits of v
// (0 <= v < 2, S <= 62: the product stays below 2^63). Integer arithmetic only:
// a float-to-u64 conversion would run on this GPU's narrow FP64 pipe.
__device__ __forceinline__ void pb_fixed(float v, int S, uint32_t& xl, uint32_t& xh) {
    const uint32_t b = __float_as_uint(v);
    const uint32_t e = b >> 23;
    const uint32_t m = e ? (b & 0x7FFFFFu) | 0x800000u : b;  // v = m * 2^(max(e,1) - 150)
    const int sh = (int)(e ? e : 1u) - 150 + S;
    if (sh >= 0) {
        xl = sh < 32 ? m << sh : 0u;
        xh = sh == 0 ? 0u : (sh < 32 ? m >> (32 - sh) : m << (sh - 32));
    } else {
        const int r = -sh;
        xl = r > 25 ? 0u : (m + (1u << (r - 1))) >> r;
        xh = 0u;
    }
}

// ---------------------------------------------------------------- phase 1
// Copies the codes of one staged chunk (scode[i]: the code of source s0 + i,
// scode[ns]: the code of the padding entries) into every run of the chunk at the
// run's place in its bin. A warp takes windows of 32 consecutive runs (lengths
// padded to 4 entries); their sources are one contiguous chunk-major range, so
// lane k of a step reads the 4 entries a0 + 4k.. and finds their run (for the
// bin-major place) by a search over the window. Windows are claimed one by one
// through *next_win (shared, 0 at the start): their sizes vary.
// KIND: PB_COPY_CODES writes the staged codes; PB_ADD_W8 / PB_ADD_ONE (min programs
// whose message adds the edge weight) write broadcast + the entry's weight (w8, one
// byte per entry, chunk-major) / + 1, and the no-broadcast pattern for silent sources.
enum { PB_COPY_CODES = 0, PB_ADD_W8 = 1, PB_ADD_ONE = 2 };
__device__ __forceinline__ uint32_t pb_add_w(uint32_t x, uint32_t w) {
    return x == ipregel::kNoBroadcastBits ? x : x + w;  // below the pattern: V x max weight < 2^32 - 1
}
template <int KIND, int PB1_LOADS>
__device__ __forceinline__ void pb_copy_runs(const PbDev& B, const uint4& ch, const uint32_t* scode, uint32_t lane,
                                             uint32_t* next_win) {
    const uint32_t nwin = (ch.w - ch.z + 31) / 32;
    for (;;) {
        uint32_t wi = 0;
        if (lane == 0) wi = atomicAdd(next_win, 1u);
        wi = __shfl_sync(FULL, wi, 0);
        if (wi >= nwin) break;
        const uint32_t r = ch.z + 32 * wi + lane;
        const uint4 run = r < ch.w ? __ldcs(B.runs + r) : make_uint4(0, 0, 0, 0);
        const uint32_t a0 = __shfl_sync(FULL, run.x, 0);
        uint32_t inc = run.z >> 2;  // inclusive prefix of the runs' groups of 4
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, inc, o);
            if (lane >= (uint32_t)o) inc += y;
        }
        const uint32_t total = __shfl_sync(FULL, inc, 31);
        const uint32_t delta = run.y - run.x;  // bin-major minus chunk-major place (mod 2^32)
        for (uint32_t k0 = 0; k0 < total; k0 += 32u * PB1_LOADS) {
            uint2 sv[PB1_LOADS];
            uint32_t out[PB1_LOADS], wq[PB1_LOADS];
#pragma unroll
            for (int u = 0; u < PB1_LOADS; ++u) {
                const uint32_t k = k0 + 32u * u + lane;
                uint32_t j = 0;  // run of group k: the runs that end at or before it
#pragma unroll
                for (uint32_t st = 16; st; st >>= 1) {
                    const uint32_t y = __shfl_sync(FULL, inc, j + st - 1);
                    if (y <= k) j += st;
                }
                out[u] = __shfl_sync(FULL, delta, j) + a0 + 4 * k;
                sv[u] = k < total ? __ldcs(reinterpret_cast<const uint2*>(B.src + a0 + 4 * k)) : make_uint2(0, 0);
                if (KIND == PB_ADD_W8)  // the 4 entries' weights: one aligned word (groups of 4 start at 4i)
                    wq[u] = k < total ? __ldcs(reinterpret_cast<const unsigned int*>(B.w8 + a0 + 4 * k)) : 0u;
            }
#pragma unroll
            for (int u = 0; u < PB1_LOADS; ++u)
                if (k0 + 32u * u + lane < total) {
                    uint4 c = make_uint4(scode[sv[u].x & 0xFFFF], scode[sv[u].x >> 16], scode[sv[u].y & 0xFFFF],
                                         scode[sv[u].y >> 16]);
                    if (KIND == PB_ADD_W8) {
                        c = make_uint4(pb_add_w(c.x, wq[u] & 0xFF), pb_add_w(c.y, (wq[u] >> 8) & 0xFF),
                                       pb_add_w(c.z, (wq[u] >> 16) & 0xFF), pb_add_w(c.w, wq[u] >> 24));
                    } else if (KIND == PB_ADD_ONE) {
                        c = make_uint4(pb_add_w(c.x, 1u), pb_add_w(c.y, 1u), pb_add_w(c.z, 1u), pb_add_w(c.w, 1u));
                    }
                    *reinterpret_cast<uint4*>(B.code + out[u]) = c;
                }
        }
    }
}

// Staging turns every source's broadcast into its 32-bit code once: the
// fixed-point value itself below 2^31, else 2^31 | source with the 64-bit value
// in big[source]. Then every warp copies whole runs, lane by lane.
__global__ void __launch_bounds__(PB1_THREADS) k_pb_scatter(Params P) {
    extern __shared__ uint32_t scode[];
    __shared__ uint32_t task, next_win;
    const PbDev& B = P.pb;
    const uint32_t s = P.ctl->superstep;  // the superstep being computed
    const bool sent = s - 1 < P.T;        // superstep s-1 broadcast rank / out-degree (Fig. 8)
    const uint32_t lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) B.ctr[1] = 0;  // phase 2 of this superstep claims from 0
    for (;;) {
        if (threadIdx.x == 0) task = atomicAdd(B.ctr, 1u);
        __syncthreads();
        const uint32_t c = task;
        if (c >= B.n_chunks) break;
        const uint4 ch = B.chunk[c];  // {first source, sources, first run, end run}
        const uint32_t s0 = ch.x, ns = ch.y;
        // the broadcast of superstep s-1 is its rank / out-degree, formed here from
        // the rank (the accumulate launch stores only ranks: compute() of a bin then
        // reads no global memory)
        for (uint32_t i0 = threadIdx.x; i0 < ns; i0 += PB_BATCH * blockDim.x) {  // PB_BATCH loads in flight
            float x[PB_BATCH], iod[PB_BATCH];
#pragma unroll
            for (int u = 0; u < PB_BATCH; ++u) {
                const uint32_t i = i0 + u * blockDim.x;
                x[u] = i < ns ? P.rank[s0 + i] : 0.0f;
                iod[u] = i < ns ? __ldg(P.inv_outdeg + s0 + i) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < PB_BATCH; ++u) x[u] = sent ? PageRankProgram::message(x[u], iod[u]) : 0.0f;
#pragma unroll
            for (int u = 0; u < PB_BATCH; ++u) {
                const uint32_t i = i0 + u * blockDim.x;
                if (i < ns) {
                    uint32_t xl, xh;
                    pb_fixed(x[u], B.shift, xl, xh);
                    uint32_t code = xl;
                    if (xh || xl >= 0x80000000u) {
                        code = 0x80000000u | (s0 + i);
                        B.big[s0 + i] = ((unsigned long long)xh << 32) | xl;
                    }
                    scode[i] = code;
                }
            }
        }
        if (threadIdx.x == 0) {
            scode[ns] = 0u;  // source of the padding entries
            next_win = 0;
        }
        __syncthreads();
        pb_copy_runs<PB_COPY_CODES, PB1_LOADS_PR>(B, ch, scode, lane, &next_win);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- phase 2
// The low words of the sums live in shared memory, the high words in global
// memory (hi = B.hi + first vertex of the bin); the high words take the rare
// carries and the high halves of big contributions.
__device__ __forceinline__ void pb_add_big(const PbDev& B, uint32_t* lo, uint32_t* hi, uint32_t d, uint32_t code) {
    const unsigned long long x = __ldcg(B.big + (code & 0x7FFFFFFFu));
    const uint32_t xl = (uint32_t)x;
    uint32_t xh = (uint32_t)(x >> 32);
    const uint32_t old = atomicAdd(lo + d, xl);
    xh += old + xl < old ? 1u : 0u;
    if (xh) atomicAdd(hi + d, xh);
}

// Fixed-point sum (hi:lo units of 2^-S) as a float: both halves convert exactly
// or with one rounding, the fma rounds once more; scaling by 2^-S is exact.
__device__ __forceinline__ float pb_value(uint32_t hi, uint32_t lo, float inv_scale) {
    return fmaf(__uint2float_rn(hi), 4294967296.0f, __uint2float_rn(lo)) * inv_scale;
}

// ---- mbarrier / bulk-copy helpers (shared-memory addresses are 32-bit)
__device__ __forceinline__ uint32_t pb_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void pb_mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void pb_mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void pb_mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void pb_bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ uint64_t pb_clock_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of the given parity; false after PB_WAIT_NS without it.
constexpr uint64_t PB_WAIT_NS = 2000000000ull;
__device__ __forceinline__ bool pb_mbar_wait(uint32_t bar, uint32_t parity) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255u) == 0) {
            const uint64_t now = pb_clock_ns();
            if (it == 0)
                t0 = now;
            else if (now - t0 > PB_WAIT_NS)
                return false;
        }
    }
}

// compute() of the bin's vertices first, first + stride, ... < nv (vertex v0 + v):
// the sum is hi:lo in 2^-S units, the high word read only where touched marks
// one (carries and big contributions set it). Clears the vertex's high word and
// low word for the next bin. Stores the rank only: the broadcast rank / out-degree
// is formed by the next scatter (or by k_pr_contrib before a push or gather
// superstep), so this loop reads no global memory on the common path.
__device__ __forceinline__ void pb_finish(const Params& P, uint32_t* hi, uint32_t* lo, const uint32_t* touched,
                                          uint32_t v0, uint32_t nv, uint32_t first, uint32_t stride,
                                          float inv_scale, float& dacc) {
    for (uint32_t v = first; v < nv; v += stride) {
        uint32_t h = 0;
        if ((touched[v >> 5] >> (v & 31)) & 1u) {
            h = __ldcg(hi + v);
            if (h) hi[v] = 0;
        }
        const float r = PageRankProgram::compute(P.damping, P.pr_base, pb_value(h, lo[v], inv_scale));
        if (P.pr_tol > 0.f) dacc += fabsf(r - P.rank[v0 + v]);  // tolerance runs only
        P.rank[v0 + v] = r;
        lo[v] = 0;
    }
}

// Barrier of the consumer warps on an mbarrier of count PB2_CONSUMERS: lane 0
// of every warp arrives after __syncwarp (ordering its warp's memory operations
// before the release) and waits, bounded, for the given phase.
__device__ __forceinline__ bool pb_consumer_sync(uint32_t bar, uint32_t parity, uint32_t lane) {
    __syncwarp();
    bool ok = true;
    if (lane == 0) {
        pb_mbar_arrive(bar);
        ok = pb_mbar_wait(bar, parity);
    }
    return __shfl_sync(FULL, ok ? 1u : 0u, 0) != 0;
}

// Phase 2's producer (lane 0 of warp 0): claims bins in order (B.ctr[1]) and
// streams each bin's codes and destinations in tiles of PB_TILE entries with bulk
// copies into the PB_STAGES-stage ring (full/empty mbarriers); meta[2 st] =
// {first vertex, vertices, tile, tiles} (first vertex INF: no more bins),
// meta[2 st + 1].x = entries of the tile. On a timeout it records error bit 2 and
// waits (bounded) for its copies still in flight.
__device__ __forceinline__ void pb_produce(const Params& P, uint32_t* ring_code, uint16_t* ring_dst, uint4* meta,
                                           uint32_t full0, uint32_t empty0) {
    const PbDev& B = P.pb;
    uint32_t k = 0;
    bool ok = true;
    for (bool more = true; more && ok;) {
        const uint32_t t = atomicAdd(B.ctr + 1, 1u);
        more = t < B.n_tasks;
        const uint4 tk = more ? B.tasks[t] : make_uint4(0, 0, 0, 0);
        const uint32_t n = tk.w - tk.z;
        const uint32_t ntiles = more ? max(1u, (n + PB_TILE - 1) / PB_TILE) : 1u;
        for (uint32_t j = 0; j < ntiles; ++j, ++k) {
            const uint32_t st = k % PB_STAGES, r = k / PB_STAGES;
            if (r >= 1 && !pb_mbar_wait(empty0 + 8 * st, (r - 1) & 1)) {
                ok = false;
                break;
            }
            const uint32_t cnt = more ? min(PB_TILE, n - j * PB_TILE) : 0u;
            meta[2 * st] = make_uint4(more ? tk.x : INF, tk.y, j, ntiles);  // {first vertex, vertices, tile, tiles}
            meta[2 * st + 1] = make_uint4(cnt, 0, 0, 0);
            if (cnt) {
                pb_mbar_arrive_tx(full0 + 8 * st, cnt * 6u);
                pb_bulk_load(pb_smem(ring_code + st * PB_TILE), B.code + tk.z + j * PB_TILE, cnt * 4u, full0 + 8 * st);
                pb_bulk_load(pb_smem(ring_dst + st * PB_TILE), B.dst + tk.z + j * PB_TILE, cnt * 2u, full0 + 8 * st);
            } else {
                pb_mbar_arrive(full0 + 8 * st);
            }
        }
    }
    if (!ok) {  // record the timeout, then wait (bounded) for the copies still in flight
        atomicOr(&P.ctl->err, 2u);
        for (uint32_t q = k > PB_STAGES ? k - PB_STAGES : 0; q < k; ++q)
            (void)pb_mbar_wait(full0 + 8 * (q % PB_STAGES), (q / PB_STAGES) & 1);
    }
}

// Phase 2. Warp 0 is the producer: one thread claims bins and streams each
// bin's codes and destinations in tiles of PB_TILE entries with bulk copies
// into a ring of PB_STAGES shared-memory stages (full/empty mbarriers). The
// PB2_CONSUMERS other warps take the tiles in order: thread c adds the groups of
// 4 entries c, c + 512, ... of a tile (codes below 2^31 branch free; carries into the high words
// and big contributions in a warp-uniform slow path), and after a bin's last
// tile they run compute() for its vertices. Every wait (stages, and the
// consumers' own barriers, which are mbarriers too) is bounded: on timeout a
// thread records bit 2 in ctl->err (IP_E_TIMEOUT) and stops; the producer then
// waits, bounded, for its copies in flight.
__global__ void __launch_bounds__(32 * (PB2_CONSUMERS + 1), 1) k_pb_accumulate(Params P) {
    extern __shared__ __align__(128) uint32_t acc_lo[];                         // [PB_BIN_V]
    uint32_t* ring_code = acc_lo + PB_BIN_V;                                    // [PB_STAGES][PB_TILE]
    uint16_t* ring_dst = reinterpret_cast<uint16_t*>(ring_code + PB_STAGES * PB_TILE);  // [PB_STAGES][PB_TILE]
    uint4* meta = reinterpret_cast<uint4*>(ring_dst + PB_STAGES * PB_TILE);     // [PB_STAGES][2]
    uint64_t* bars = reinterpret_cast<uint64_t*>(meta + 2 * PB_STAGES);         // full[PB_STAGES], empty[PB_STAGES]
    __shared__ __align__(8) uint64_t cbar[2];                                  // consumer barriers
    // vertices of a bin whose high word was written, by bin parity: the bitmap of
    // bin k is cleared after its compute() while bin k+1 marks the other one
    __shared__ uint32_t touched2[2][PB_BIN_V / 32];
    const PbDev& B = P.pb;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t full0 = pb_smem(bars), empty0 = pb_smem(bars + PB_STAGES);
    if (threadIdx.x == 0) {
        for (int i = 0; i < PB_STAGES; ++i) {
            pb_mbar_init(full0 + 8 * i, 1);
            pb_mbar_init(empty0 + 8 * i, PB2_CONSUMERS);
        }
        pb_mbar_init(pb_smem(cbar), PB2_CONSUMERS);
        pb_mbar_init(pb_smem(cbar + 1), PB2_CONSUMERS);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        if (blockIdx.x == 0) {
            B.ctr[0] = 0;          // phase 1 of the next superstep claims from 0
            P.ctl->pr_stale = 1;   // this superstep's broadcasts are not written (see k_pr_contrib)
        }
    }
    for (uint32_t i = threadIdx.x; i < PB_BIN_V; i += blockDim.x) acc_lo[i] = 0;
    for (uint32_t i = threadIdx.x; i < 2 * (PB_BIN_V / 32); i += blockDim.x) touched2[i / (PB_BIN_V / 32)][i % (PB_BIN_V / 32)] = 0;
    __syncthreads();

    if (warp == 0) {  // ------------------------------------------------ producer
        if (lane == 0) pb_produce(P, ring_code, ring_dst, meta, full0, empty0);
        return;
    }

    // --------------------------------------------------------------- consumers
    const uint32_t c = threadIdx.x - 32;  // 0 .. 32 * PB2_CONSUMERS - 1
    const float inv_scale = B.inv_scale;
    const uint32_t cb0 = pb_smem(cbar), cb1 = pb_smem(cbar + 1);
    uint32_t bins_done = 0;
    float dacc = 0.f;  // L1 rank change of the vertices this thread finishes (tolerance runs)
    for (uint32_t k = 0;; ++k) {
        const uint32_t st = k % PB_STAGES, r = k / PB_STAGES;
        if (!pb_mbar_wait(full0 + 8 * st, r & 1)) {
            atomicOr(&P.ctl->err, 2u);
            break;
        }
        const uint4 m = meta[2 * st];  // {first vertex, vertices, tile, tiles}
        const uint32_t cnt = meta[2 * st + 1].x;
        if (m.x == INF) break;
        uint32_t* hi = B.hi + m.x;
#pragma unroll
        for (int gq = 0; gq < PB_GROUPS; ++gq) {
            const uint32_t i = 4 * (c + gq * 32 * PB2_CONSUMERS);
            uint32_t flags = 0;  // bit q: carry or big in entry i + q
            uint4 cv = make_uint4(0, 0, 0, 0);
            uint2 dv = make_uint2(0, 0);
            if (i < cnt) {
                cv = *reinterpret_cast<const uint4*>(ring_code + st * PB_TILE + i);
                dv = *reinterpret_cast<const uint2*>(ring_dst + st * PB_TILE + i);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t code = q == 0 ? cv.x : q == 1 ? cv.y : q == 2 ? cv.z : cv.w;
                    const uint32_t d = ((q < 2 ? dv.x : dv.y) >> (16 * (q & 1))) & 0xFFFFu;
                    const uint32_t big = code >> 31;
                    const uint32_t v = big ? 0u : code;
                    const uint32_t old = atomicAdd(acc_lo + d, v);
                    flags |= ((old + v < old ? 1u : 0u) | big) << q;
                }
            }
            if (__any_sync(FULL, flags)) {
                for (int q = 0; q < 4; ++q)
                    if ((flags >> q) & 1u) {
                        const uint32_t code = q == 0 ? cv.x : q == 1 ? cv.y : q == 2 ? cv.z : cv.w;
                        const uint32_t d = ((q < 2 ? dv.x : dv.y) >> (16 * (q & 1))) & 0xFFFFu;
                        atomicOr(touched2[bins_done & 1] + (d >> 5), 1u << (d & 31));
                        if (code >> 31)
                            pb_add_big(B, acc_lo, hi, d, code);
                        else  // the carry of the common path (a big entry added 0 there and cannot carry)
                            atomicAdd(hi + d, 1u);
                    }
            }
        }
        __syncwarp();
        if (lane == 0) pb_mbar_arrive(empty0 + 8 * st);
        if (m.z + 1 == m.w) {  // the bin's last tile: every code is in
            // the barrier also orders the high-word atomics before the reads below
            bool ok = pb_consumer_sync(cb0, bins_done & 1, lane);
            uint32_t* touched = touched2[bins_done & 1];
            pb_finish(P, hi, acc_lo, touched, m.x, m.y, c, 32 * PB2_CONSUMERS, inv_scale, dacc);
            ok = pb_consumer_sync(cb1, bins_done & 1, lane) && ok;
            // bin k+1 marks the other bitmap; this one is clear before bin k+2 starts
            for (uint32_t i = c; i < PB_BIN_V / 32; i += 32 * PB2_CONSUMERS) touched[i] = 0;
            ++bins_done;
            if (!ok) {
                if (lane == 0) atomicOr(&P.ctl->err, 2u);
                break;
            }
        }
    }
    flush_delta(P, dacc);  // every consumer warp leaves the loop whole (warp-uniform breaks)
}

// ---------------------------------------------------------------- min programs
// The same layout and the same two phases for a vertex program whose combiner is
// the uint32 minimum and whose message is the sender's value itself (Hashmin,
// Fig. 9; KIND PB_COPY_CODES) or the value plus the edge's weight (SSSP, Fig. 10;
// PB_ADD_W8 with the entry's weight byte, PB_ADD_ONE on unweighted graphs): the codes
// are the messages of the broadcasting senders (the no-broadcast pattern for a vertex
// that did not broadcast, which also fills the padding entries and the bin tails,
// so they change nothing), and a bin folds its codes with a shared-memory atomicMin
// per destination. A destination whose minimum is a message is a recipient (no
// message of such a program equals the pattern): its mailbox gets the minimum and
// its recipient bit is set, and the apply kernel runs compute() as after any pull.
template <int KIND>
__global__ void __launch_bounds__(PB1_THREADS) k_pbm_scatter(Params P) {
    extern __shared__ uint32_t scode[];
    __shared__ uint32_t task, next_win;
    const PbDev& B = P.pb;
    const uint32_t lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) B.ctr[1] = 0;  // phase 2 of this superstep claims from 0
    for (;;) {
        if (threadIdx.x == 0) task = atomicAdd(B.ctr, 1u);
        __syncthreads();
        const uint32_t c = task;
        if (c >= B.n_chunks) break;
        const uint4 ch = B.chunk[c];  // {first source, sources, first run, end run}
        const uint32_t s0 = ch.x, ns = ch.y;
        for (uint32_t i0 = threadIdx.x; i0 < ns; i0 += PB_BATCH * blockDim.x) {  // PB_BATCH loads in flight
            uint32_t x[PB_BATCH];
#pragma unroll
            for (int u = 0; u < PB_BATCH; ++u) {
                const uint32_t i = i0 + u * blockDim.x;
                x[u] = i < ns ? P.outbox[s0 + i] : 0u;
            }
#pragma unroll
            for (int u = 0; u < PB_BATCH; ++u) {
                const uint32_t i = i0 + u * blockDim.x;
                if (i < ns) scode[i] = x[u];
            }
        }
        if (threadIdx.x == 0) {
            scode[ns] = ipregel::kNoBroadcastBits;  // source of the padding entries
            next_win = 0;
        }
        __syncthreads();
        pb_copy_runs<KIND, PB1_LOADS_MIN>(B, ch, scode, lane, &next_win);
        __syncthreads();
    }
}

// compute() input of the bin's vertices first, first + stride, ... < nv (vertex v0 +
// v): every lane of a warp takes consecutive vertices, so the warp's recipient bits
// are one ballot (shifted into the one or two bitmap words it overlaps). Resets the
// accumulators for the next bin.
__device__ __forceinline__ void pbm_finish(const Params& P, uint32_t* acc, uint32_t v0, uint32_t nv, uint32_t first,
                                           uint32_t stride, uint32_t lane) {
    for (uint32_t base = first - lane; base < nv; base += stride) {
        const uint32_t v = base + lane;
        const bool in = v < nv;
        const uint32_t m = in ? acc[v] : ipregel::kNoBroadcastBits;
        if (in) acc[v] = ipregel::kNoBroadcastBits;
        const bool r = m != ipregel::kNoBroadcastBits;
        if (r) P.mbox[v0 + v] = m;
        const uint32_t bits = __ballot_sync(FULL, r);
        if (lane == 0 && bits) {
            const uint32_t gv = v0 + base, w = gv >> 5, sh = gv & 31u;
            atomicOr(P.recv + w, bits << sh);
            if (sh && (bits >> (32 - sh))) atomicOr(P.recv + w + 1, bits >> (32 - sh));
        }
    }
}

__global__ void __launch_bounds__(32 * (PB2_CONSUMERS + 1), 1) k_pbm_accumulate(Params P) {
    extern __shared__ __align__(128) uint32_t acc[];                              // [PB_BIN_V]
    uint32_t* ring_code = acc + PB_BIN_V;                                          // [PB_STAGES][PB_TILE]
    uint16_t* ring_dst = reinterpret_cast<uint16_t*>(ring_code + PB_STAGES * PB_TILE);  // [PB_STAGES][PB_TILE]
    uint4* meta = reinterpret_cast<uint4*>(ring_dst + PB_STAGES * PB_TILE);     // [PB_STAGES][2]
    uint64_t* bars = reinterpret_cast<uint64_t*>(meta + 2 * PB_STAGES);         // full[PB_STAGES], empty[PB_STAGES]
    __shared__ __align__(8) uint64_t cbar[2];                                  // consumer barriers
    const PbDev& B = P.pb;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t full0 = pb_smem(bars), empty0 = pb_smem(bars + PB_STAGES);
    if (threadIdx.x == 0) {
        for (int i = 0; i < PB_STAGES; ++i) {
            pb_mbar_init(full0 + 8 * i, 1);
            pb_mbar_init(empty0 + 8 * i, PB2_CONSUMERS);
        }
        pb_mbar_init(pb_smem(cbar), PB2_CONSUMERS);
        pb_mbar_init(pb_smem(cbar + 1), PB2_CONSUMERS);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        if (blockIdx.x == 0) B.ctr[0] = 0;  // phase 1 of the next superstep claims from 0
    }
    for (uint32_t i = threadIdx.x; i < PB_BIN_V; i += blockDim.x) acc[i] = ipregel::kNoBroadcastBits;
    __syncthreads();
    if (warp == 0) {  // producer
        if (lane == 0) pb_produce(P, ring_code, ring_dst, meta, full0, empty0);
        return;
    }
    const uint32_t c = threadIdx.x - 32;  // 0 .. 32 * PB2_CONSUMERS - 1
    const uint32_t cb0 = pb_smem(cbar), cb1 = pb_smem(cbar + 1);
    uint32_t bins_done = 0;
    for (uint32_t k = 0;; ++k) {
        const uint32_t st = k % PB_STAGES, r = k / PB_STAGES;
        if (!pb_mbar_wait(full0 + 8 * st, r & 1)) {
            atomicOr(&P.ctl->err, 2u);
            break;
        }
        const uint4 m = meta[2 * st];  // {first vertex, vertices, tile, tiles}
        const uint32_t cnt = meta[2 * st + 1].x;
        if (m.x == INF) break;
#pragma unroll
        for (int gq = 0; gq < PB_GROUPS; ++gq) {
            const uint32_t i = 4 * (c + gq * 32 * PB2_CONSUMERS);
            if (i < cnt) {
                const uint4 cv = *reinterpret_cast<const uint4*>(ring_code + st * PB_TILE + i);
                const uint2 dv = *reinterpret_cast<const uint2*>(ring_dst + st * PB_TILE + i);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t code = q == 0 ? cv.x : q == 1 ? cv.y : q == 2 ? cv.z : cv.w;
                    const uint32_t d = ((q < 2 ? dv.x : dv.y) >> (16 * (q & 1))) & 0xFFFFu;
                    if (code != ipregel::kNoBroadcastBits) atomicMin(acc + d, code);
                }
            }
        }
        __syncwarp();
        if (lane == 0) pb_mbar_arrive(empty0 + 8 * st);
        if (m.z + 1 == m.w) {  // the bin's last tile: every code is in
            bool ok = pb_consumer_sync(cb0, bins_done & 1, lane);
            pbm_finish(P, acc, m.x, m.y, c, 32 * PB2_CONSUMERS, lane);
            ok = pb_consumer_sync(cb1, bins_done & 1, lane) && ok;
            ++bins_done;
            if (!ok) {
                if (lane == 0) atomicOr(&P.ctl->err, 2u);
                break;
            }
        }
    }
}

// Sets the codes of the bin tails (the entries between a bin's last run and the
// next bin, which no scatter writes) to the neutral code of an engine: 0 for the
// PageRank sums, the no-broadcast pattern for the min programs.
__global__ void k_pb_tails(uint32_t* code, const uint2* tails, uint32_t nb, uint32_t value) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nb; q += gridDim.x * blockDim.x)
        for (uint32_t e = tails[q].x; e < tails[q].y; ++e) code[e] = value;
}

// At build: the bin tails hold code 0 and destination 0 (every other entry belongs to a
// run: the placement writes its destination, every scatter its code).
__global__ void k_pb_tails_init(uint32_t* code, uint16_t* dst, const uint2* tails, uint32_t nb) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nb; q += gridDim.x * blockDim.x)
        for (uint32_t e = tails[q].x; e < tails[q].y; ++e) {
            code[e] = 0u;
            dst[e] = 0;
        }
}

// ---------------------------------------------------------------- layout build
// Bin of a destination without a per-vertex table: tab[b] is the bin of vertex
// min(b << sh, V - 1) (at most PB_TAB + 1 entries, in shared memory), so the bin of v
// lies in [tab[v >> sh], tab[(v >> sh) + 1]]; a binary search over the bin starts
// (global, L1-resident) narrows that range, which holds one or two bins except where
// the bins are narrow (the high in-degree vertices).
constexpr uint32_t PB_TAB = 4096;
__device__ __forceinline__ uint32_t pb_bin_of(uint32_t v, const uint32_t* tab, uint32_t sh,
                                              const uint32_t* __restrict__ bstart) {
    const uint32_t b = v >> sh;
    uint32_t lo = tab[b], hi = tab[b + 1];
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (__ldg(bstart + mid) <= v)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void k_pb_tab(const uint32_t* __restrict__ bstart, uint32_t nb, uint32_t V, uint32_t sh, uint32_t ntab,
                         uint32_t* tab) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= ntab; i += gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)min((uint64_t)i << sh, (uint64_t)V - 1);
        uint32_t lo = 0, hi = nb - 1;  // the last bin whose start is <= x
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (bstart[mid] <= x)
                lo = mid;
            else
                hi = mid - 1;
        }
        tab[i] = lo;
    }
}

__device__ __forceinline__ void pb_load_tab(const uint32_t* __restrict__ g_tab, uint32_t ntab, uint32_t* tab) {
    for (uint32_t i = threadIdx.x; i <= ntab; i += blockDim.x) tab[i] = g_tab[i];
}

__device__ __forceinline__ uint32_t pad4(uint32_t n) { return (n + 3) & ~3u; }

// Per chunk: its entries per bin (row c of the chunk x bin matrix of run lengths),
// its number of runs and its padded entry count.
__global__ void __launch_bounds__(PBB_THREADS) k_pb_count(const uint32_t* __restrict__ csr_off,
                                                          const uint32_t* __restrict__ col,
                                                          const uint4* __restrict__ cs,
                                                          const uint32_t* __restrict__ g_tab, uint32_t sh,
                                                          uint32_t ntab, const uint32_t* __restrict__ bstart,
                                                          uint32_t nb, uint32_t* M, uint32_t* chunk_runs,
                                                          uint32_t* chunk_len) {
    extern __shared__ uint32_t sm[];
    uint32_t* hist = sm;       // [nb]
    uint32_t* tab = sm + nb;   // [ntab + 1]
    const uint32_t c = blockIdx.x;
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
    pb_load_tab(g_tab, ntab, tab);
    __syncthreads();
    const uint32_t e0 = csr_off[cs[c].x], e1 = csr_off[cs[c].x + cs[c].y];
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) atomicAdd(hist + pb_bin_of(col[e], tab, sh, bstart), 1u);
    __syncthreads();
    uint32_t runs = 0, len = 0;
    for (uint32_t q = threadIdx.x; q < nb; q += blockDim.x) {
        const uint32_t n = hist[q];
        M[(size_t)c * nb + q] = n;
        runs += n ? 1u : 0u;
        len += pad4(n);
    }
    for (int o = 16; o; o >>= 1) {
        runs += __shfl_xor_sync(FULL, runs, o);
        len += __shfl_xor_sync(FULL, len, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(chunk_runs + c, runs);
        atomicAdd(chunk_len + c, len);
    }
}

// Per bin: exclusive scan of its column of padded run lengths over the chunks (the
// place of every run inside its bin, into O), and the bin's padded total.
__global__ void k_pb_colscan(const uint32_t* __restrict__ M, uint32_t* O, uint32_t nC, uint32_t nb, uint32_t* total) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb) return;
    uint32_t run = 0;
    for (uint32_t c = 0; c < nC; ++c) {
        const uint32_t t = pad4(M[(size_t)c * nb + q]);
        O[(size_t)c * nb + q] = run;
        run += t;
    }
    total[q] = run;
}

constexpr uint32_t PB_PIECE = 1024;  // out-edges per warp task of k_pb_place
constexpr int PB_PU = 4;             // k_pb_place: out-edges per lane in flight

// Per chunk: the run records (padded to 4 entries, the padding reads source `ns`
// whose code is the neutral one), then every out-edge into its run in both orders.
// The out-edges are taken by warps in pieces of PB_PIECE; a warp keeps the offsets
// of 32 consecutive sources in registers and finds each lane's source by a 5-step
// shuffle search (the sources' edge ranges are sorted), sliding the window forward
// as the piece advances.
__global__ void __launch_bounds__(PBP_THREADS, 1) k_pb_place(const uint32_t* __restrict__ csr_off,
                                                          const uint32_t* __restrict__ col,
                                                          const uint4* __restrict__ cs,
                                                          const uint32_t* __restrict__ abase,
                                                          const uint32_t* __restrict__ g_tab, uint32_t sh,
                                                          uint32_t ntab, const uint32_t* __restrict__ bstart,
                                                          const uint32_t* __restrict__ bbase, uint32_t nb,
                                                          const uint32_t* __restrict__ M,
                                                          const uint32_t* __restrict__ O, uint4* runs,
                                                          uint16_t* src, uint16_t* dst,
                                                          const uint32_t* __restrict__ wsrc, uint8_t* w8) {
    extern __shared__ uint32_t sm[];
    uint32_t* cnt = sm;            // [nb]: entries per bin, then the run's offset inside the chunk
    uint32_t* cur = sm + nb;       // [nb]: placement cursor
    uint32_t* rb = sm + 2 * nb;    // [nb]: the run's bin-major start
    uint32_t* tab = sm + 3 * nb;   // [ntab + 1]
    __shared__ uint32_t wsum[PBP_THREADS / 32], wnz[PBP_THREADS / 32];
    const uint4 ch = cs[blockIdx.x];
    const uint32_t s0 = ch.x, ns = ch.y, a_c = abase[blockIdx.x];
    const uint32_t* Mc = M + (size_t)blockIdx.x * nb;
    const uint32_t* Oc = O + (size_t)blockIdx.x * nb;
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
        cnt[i] = Mc[i];
        cur[i] = 0;
        rb[i] = bbase[i] + Oc[i];
    }
    pb_load_tab(g_tab, ntab, tab);
    __syncthreads();
    // exclusive scans of the padded counts and of the non-empty bins: thread t owns bins [b0, b1)
    const uint32_t per = (nb + blockDim.x - 1) / blockDim.x;
    const uint32_t b0 = min(nb, threadIdx.x * per), b1 = min(nb, b0 + per);
    uint32_t mine = 0, mnz = 0;
    for (uint32_t q = b0; q < b1; ++q) {
        mine += pad4(cnt[q]);
        mnz += cnt[q] ? 1u : 0u;
    }
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = mine, inz = mnz;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, inc, o), z = __shfl_up_sync(FULL, inz, o);
        if (lane >= (uint32_t)o) {
            inc += y;
            inz += z;
        }
    }
    if (lane == 31) {
        wsum[w] = inc;
        wnz[w] = inz;
    }
    __syncthreads();
    uint32_t off = inc - mine, rk = inz - mnz;
    for (uint32_t k = 0; k < w; ++k) {
        off += wsum[k];
        rk += wnz[k];
    }
    for (uint32_t q = b0; q < b1; ++q) {
        const uint32_t n = cnt[q], n4 = pad4(n);
        if (n) {
            runs[ch.z + rk++] = make_uint4(a_c + off, rb[q], n4, 0u);
            for (uint32_t k = n; k < n4; ++k) {
                src[a_c + off + k] = (uint16_t)ns;
                dst[rb[q] + k] = 0;
                if (w8) w8[a_c + off + k] = 0;
            }
        }
        cnt[q] = off;
        off += n4;
    }
    __syncthreads();
    const uint32_t* offs = csr_off + s0;  // the chunk's offsets, ns + 1 of them
    const uint32_t e0 = offs[0], e1 = offs[ns];
    const uint32_t n_pieces = (e1 - e0 + PB_PIECE - 1) / PB_PIECE;
    for (uint32_t piece = w; piece < n_pieces; piece += blockDim.x / 32) {
        const uint32_t p0 = e0 + piece * PB_PIECE, p1 = min(e1, p0 + PB_PIECE);
        // the window starts at the source of p0: the last s with offs[s] <= p0
        uint32_t lo = 0, hi = ns - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (offs[mid] <= p0)
                lo = mid;
            else
                hi = mid - 1;
        }
        for (uint32_t ws = lo;; ws += 32) {                   // windows of 32 sources
            const uint32_t a = offs[min(ws + lane, ns)];      // lane i: first edge of source ws + i
            const uint32_t wend = offs[min(ws + 32, ns)];     // first edge after the window
            const uint32_t whi = min(p1, wend);
            const uint32_t wlo = max(p0, __shfl_sync(FULL, a, 0));
            for (uint32_t base = wlo; base < whi; base += 32 * PB_PU) {  // PB_PU edges per lane in flight
                uint32_t e[PB_PU], jv[PB_PU], v[PB_PU], q[PB_PU], b[PB_PU];
#pragma unroll
                for (int u = 0; u < PB_PU; ++u) {
                    e[u] = base + 32 * u + lane;
                    uint32_t jj = 0;  // the last lane jj with a_jj <= e
#pragma unroll
                    for (uint32_t k = 16; k; k >>= 1) {
                        const uint32_t aj = __shfl_sync(FULL, a, jj + k);
                        if (aj <= e[u]) jj += k;
                    }
                    jv[u] = jj;
                }
#pragma unroll
                for (int u = 0; u < PB_PU; ++u) v[u] = e[u] < whi ? col[e[u]] : 0u;
#pragma unroll
                for (int u = 0; u < PB_PU; ++u) q[u] = e[u] < whi ? pb_bin_of(v[u], tab, sh, bstart) : 0u;
#pragma unroll
                for (int u = 0; u < PB_PU; ++u) b[u] = e[u] < whi ? __ldg(bstart + q[u]) : 0u;
#pragma unroll
                for (int u = 0; u < PB_PU; ++u)
                    if (e[u] < whi) {
                        const uint32_t k = atomicAdd(cur + q[u], 1u);
                        src[a_c + cnt[q[u]] + k] = (uint16_t)(ws + jv[u]);
                        dst[rb[q[u]] + k] = (uint16_t)(v[u] - b[u]);
                        if (w8) w8[a_c + cnt[q[u]] + k] = (uint8_t)wsrc[e[u]];
                    }
            }
            if (wend >= p1) break;
        }
    }
}

// Cuts of a vertex range into consecutive groups (chunks of sources over the CSR
// offsets, bins of destinations over the CSC offsets), greedily: a group grows while
// it has fewer than max_n vertices and at most per_e edges (a vertex with more edges
// than that is a group of its own). The greedy pass is sequential, but where a group
// that starts at u ends depends on u alone: k_pb_next finds that end for every u in
// parallel (a binary search, the offsets being sorted). The chain of ends from vertex 0
// is then followed PB_JUMP groups at a time: k_pb_jump gives every u the start of the
// group PB_JUMP groups later, one thread walks those jumps from vertex 0 (one dependent
// load per PB_JUMP groups instead of per group: each costs a trip to DRAM), and
// k_pb_fill expands every jump into its PB_JUMP group starts in parallel.
__global__ void k_pb_next(const uint32_t* __restrict__ off, uint32_t n, uint32_t per_e, uint32_t max_n,
                          uint32_t* nxt) {
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const uint64_t lim = (uint64_t)off[u] + per_e;
        const uint64_t end = (uint64_t)u + max_n;
        const uint32_t cap = end < n ? (uint32_t)end : n;
        // the group [u, j) ends at the smallest j in [u + 1, cap] with j == cap or off[j + 1] > lim
        uint32_t lo = u + 1, hi = cap;  // answer in [lo, hi]
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo) / 2;
            if ((uint64_t)off[mid + 1] > lim)
                hi = mid;
            else
                lo = mid + 1;
        }
        nxt[u] = lo;
    }
}

constexpr uint32_t PB_JUMP = 16;

__global__ void k_pb_jump(const uint32_t* __restrict__ nxt, uint32_t n, uint32_t* jk) {
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        uint32_t v = u;
        for (uint32_t i = 0; i < PB_JUMP && v < n; ++i) v = nxt[v];
        jk[u] = v;
    }
}

// One thread: every PB_JUMP-th group start from vertex 0, at most acap of them
// (*n_anchors = acap + 1 if the chain goes on). *count starts as "did not end".
__global__ void k_pb_anchors(const uint32_t* __restrict__ jk, uint32_t n, uint32_t acap, uint32_t cap,
                             uint32_t* anchors, uint32_t* n_anchors, uint32_t* count) {
    uint32_t u = 0, k = 0;
    while (u < n && k < acap) {
        anchors[k++] = u;
        u = jk[u];
    }
    *n_anchors = u < n ? acap + 1 : k;
    *count = cap + 1;
}

// Anchor i's PB_JUMP group starts {first vertex, its first edge} at places i * PB_JUMP
// on; the walk of the last anchor reaches n and writes the number of groups.
__global__ void k_pb_fill(const uint32_t* __restrict__ nxt, const uint32_t* __restrict__ off, uint32_t n,
                          const uint32_t* __restrict__ anchors, const uint32_t* __restrict__ n_anchors,
                          uint32_t acap, uint32_t cap, uint2* starts, uint32_t* count) {
    const uint32_t na = min(*n_anchors, acap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x) {
        uint32_t u = anchors[i];
        uint64_t k = (uint64_t)i * PB_JUMP;
        for (uint32_t j = 0; j < PB_JUMP && u < n; ++j, ++k) {
            if (k < cap) starts[k] = make_uint2(u, off[u]);
            u = nxt[u];
        }
        if (u >= n) *count = k <= (uint64_t)cap ? (uint32_t)k : cap + 1;
    }
}

// Host-side owner of the layout's device buffers.
struct PbLayout {
    PbDev d;
    std::vector<std::pair<void*, size_t>> bufs;
    int grid1 = 0, grid2 = 0, grid1m = 0;
    uint2* tails = nullptr;  // [n_tasks] bin tails {first entry, end entry}
    int tail_mode = 0;       // 0: tail codes 0 (PageRank), 1: no-broadcast pattern (min programs)
};

template <class T>
int pb_alloc(ip_graph* g, PbLayout* L, T** p, size_t count) {
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    const int r = alloc_dev(g, (void**)p, bytes);
    if (r == IP_OK) L->bufs.push_back({(void*)*p, bytes});
    return r;
}

void pb_release(ip_graph* g, PbLayout* L) {
    for (auto& b : L->bufs) {
        free_dev(b.first);
        g->device_bytes -= b.second;
    }
    delete L;
}

// A temporary device buffer of the build, freed on every exit.
struct TmpBuf {
    ip_graph* g;
    void* p = nullptr;
    size_t bytes = 0;
    ~TmpBuf() {
        if (p) {
            free_dev(p);
            g->device_bytes -= bytes;
        }
    }
    template <class T>
    int alloc(T** out, size_t count) {
        bytes = std::max<size_t>(count, 1) * sizeof(T);
        const int r = alloc_dev(g, &p, bytes);
        if (r != IP_OK) bytes = 0;
        *out = (T*)p;
        return r;
    }
};

// The greedy group starts for the offsets off (device, n + 1 entries), read back as
// {first vertex, its first edge} pairs in vertex order. A group that ends by the
// vertex cap has max_n vertices; two groups in a row that end by the edge cap hold
// more than per_e edges together: so there are at most n / max_n + 2 E / per_e + 2.
int pb_cuts(ip_graph* g, const uint32_t* off, uint32_t n, uint64_t per_e, uint32_t max_n, cudaStream_t st,
            std::vector<uint2>* out) {
    const uint32_t pe = (uint32_t)std::min<uint64_t>(per_e, 0xFFFFFFFFull);
    const uint64_t bound = (uint64_t)n / max_n + 2 * g->E / pe + 16;
    const uint32_t cap = (uint32_t)std::min<uint64_t>(bound, n);
    const uint32_t acap = cap / PB_JUMP + 2;
    uint32_t *nxt = nullptr, *count = nullptr, *jk = nullptr, *anchors = nullptr;
    uint2* starts = nullptr;
    int r = alloc_dev(g, (void**)&nxt, (size_t)n * sizeof(uint32_t));
    if (!r) r = alloc_dev(g, (void**)&jk, (size_t)n * sizeof(uint32_t));
    if (!r) r = alloc_dev(g, (void**)&count, 2 * sizeof(uint32_t));
    if (!r) r = alloc_dev(g, (void**)&anchors, (size_t)acap * sizeof(uint32_t));
    if (!r) r = alloc_dev(g, (void**)&starts, std::max<size_t>(cap, 1) * sizeof(uint2));
    if (!r) {
        const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)g->num_sms * 8, ((uint64_t)n + 255) / 256));
        k_pb_next<<<grid, 256, 0, st>>>(off, n, pe, max_n, nxt);
        k_pb_jump<<<grid, 256, 0, st>>>(nxt, n, jk);
        k_pb_anchors<<<1, 1, 0, st>>>(jk, n, acap, cap, anchors, count + 1, count);
        k_pb_fill<<<(acap + 255) / 256, 256, 0, st>>>(nxt, off, n, anchors, count + 1, acap, cap, starts, count);
        r = cuda_err(cudaGetLastError());
    }
    uint32_t total = 0;
    if (!r) r = cuda_err(cudaMemcpyAsync(&total, count, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    if (!r) r = cuda_err(cudaStreamSynchronize(st));
    if (!r && total > cap) r = IP_E_RANGE;  // cannot happen (see the bound above)
    if (!r) {
        out->resize(total);
        r = cuda_err(cudaMemcpyAsync(out->data(), starts, sizeof(uint2) * total, cudaMemcpyDeviceToHost, st));
    }
    if (!r) r = cuda_err(cudaStreamSynchronize(st));
    for (void* p : {(void*)nxt, (void*)jk, (void*)count, (void*)anchors, (void*)starts}) free_dev(p);
    g->device_bytes -= (nxt ? (size_t)n * sizeof(uint32_t) : 0) + (jk ? (size_t)n * sizeof(uint32_t) : 0) +
                       (count ? 2 * sizeof(uint32_t) : 0) + (anchors ? (size_t)acap * sizeof(uint32_t) : 0) +
                       (starts ? std::max<size_t>(cap, 1) * sizeof(uint2) : 0);
    return r;
}

int occupancy_grid(const ip_graph* g, const void* fn, int threads, size_t smem) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess || occ < 1) {
        (void)cudaGetLastError();
        occ = 1;
    }
    return g->num_sms * occ;
}

#define PBK(x)                \
    do {                      \
        int _r = (x);         \
        if (_r != IP_OK) {    \
            pb_release(g, L); \
            return _r;        \
        }                     \
    } while (0)

int build(ip_graph* g, cudaStream_t st, PbLayout** out) {
    const uint32_t V = g->V;
    PbLayout* L = new PbLayout();
    memset(&L->d, 0, sizeof(L->d));
    PbDev& d = L->d;
    PBK(cuda_err(cudaFuncSetAttribute(k_pb_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PB1_SMEM_PR)));
    PBK(cuda_err(cudaFuncSetAttribute(k_pb_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PB2_SMEM)));
    PBK(cuda_err(cudaFuncSetAttribute(k_pbm_scatter<PB_COPY_CODES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)PB1_SMEM_MIN)));
    PBK(cuda_err(cudaFuncSetAttribute(k_pbm_scatter<PB_ADD_W8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)PB1_SMEM_MIN)));
    PBK(cuda_err(cudaFuncSetAttribute(k_pbm_scatter<PB_ADD_ONE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)PB1_SMEM_MIN)));
    PBK(cuda_err(cudaFuncSetAttribute(k_pbm_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PB2_SMEM)));
    L->grid1 = occupancy_grid(g, (const void*)k_pb_scatter, PB1_THREADS, PB1_SMEM_PR);
    L->grid1m = occupancy_grid(g, (const void*)k_pbm_scatter<PB_ADD_W8>, PB1_THREADS, PB1_SMEM_MIN);
    L->grid2 = g->num_sms;  // one producer/consumer CTA per SM

    // chunks of consecutive sources, cut greedily on the device (pb_cuts) by edge count
    // and by source count; chunks of sources without out-edges are skipped
    std::vector<uint2> cut;
    const uint64_t chunk_e = std::min<uint64_t>(PB_CHUNK_MAX, std::max<uint64_t>(PB_CHUNK_MIN, g->E >> 12));
    PBK(pb_cuts(g, g->csr_off, V, chunk_e, PB_MAXS, st, &cut));
    std::vector<uint2> chunks;
    for (size_t i = 0; i < cut.size(); ++i) {
        const uint32_t first = cut[i].x, next = i + 1 < cut.size() ? cut[i + 1].x : V;
        const uint64_t e1 = i + 1 < cut.size() ? cut[i + 1].y : g->E;
        if (e1 != cut[i].y) chunks.push_back(make_uint2(first, next - first));
    }
    const uint32_t nC = (uint32_t)chunks.size();
    // bins of consecutive destinations, cut by vertex count and by in-edge count
    const uint64_t bin_e = std::max<uint64_t>(16384, (g->E + 4ull * L->grid2 - 1) / (4ull * L->grid2));
    PBK(pb_cuts(g, g->csc_off, V, bin_e, PB_BIN_V, st, &cut));
    std::vector<uint32_t> bstart;
    bstart.reserve(cut.size() + 1);
    for (const uint2& c : cut) bstart.push_back(c.x);
    bstart.push_back(V);
    const uint32_t nb = (uint32_t)bstart.size() - 1;
    if (nb > PB_MAX_BINS) PBK(IP_E_RANGE);

    uint4* d_cs;
    uint32_t* d_bstart;
    PBK(pb_alloc(g, L, &d_cs, nC));
    // the bin lookup table: ntab + 1 entries, vertex blocks of 2^sh
    uint32_t sh = 0;
    while (((V - 1) >> sh) + 1 > PB_TAB) ++sh;
    const uint32_t ntab = ((V - 1) >> sh) + 1;
    TmpBuf t_tab{g}, t_bstart{g}, t_M{g}, t_O{g}, t_chunk_runs{g}, t_chunk_len{g}, t_total{g}, t_bbase{g}, t_abase{g};
    uint32_t *d_tab, *d_M, *d_O, *d_chunk_runs, *d_chunk_len, *d_total, *d_bbase, *d_abase;
    PBK(t_tab.alloc(&d_tab, ntab + 1));
    PBK(t_bstart.alloc(&d_bstart, nb + 1));
    PBK(t_M.alloc(&d_M, (size_t)nC * nb));
    PBK(t_O.alloc(&d_O, (size_t)nC * nb));
    PBK(t_chunk_runs.alloc(&d_chunk_runs, nC));
    PBK(t_chunk_len.alloc(&d_chunk_len, nC));
    PBK(t_abase.alloc(&d_abase, nC));
    PBK(t_total.alloc(&d_total, nb));
    PBK(t_bbase.alloc(&d_bbase, nb + 1));
    std::vector<uint4> cinfo(nC);
    for (uint32_t c = 0; c < nC; ++c) cinfo[c] = make_uint4(chunks[c].x, chunks[c].y, 0, 0);
    if (nC) PBK(cuda_err(cudaMemcpyAsync(d_cs, cinfo.data(), sizeof(uint4) * nC, cudaMemcpyHostToDevice, st)));
    PBK(cuda_err(cudaMemcpyAsync(d_bstart, bstart.data(), sizeof(uint32_t) * (nb + 1), cudaMemcpyHostToDevice, st)));
    PBK(cuda_err(cudaMemsetAsync(d_chunk_runs, 0, sizeof(uint32_t) * std::max<uint32_t>(nC, 1), st)));
    PBK(cuda_err(cudaMemsetAsync(d_chunk_len, 0, sizeof(uint32_t) * std::max<uint32_t>(nC, 1), st)));
    k_pb_tab<<<(ntab + 256) / 256, 256, 0, st>>>(d_bstart, nb, V, sh, ntab, d_tab);
    const size_t smem_count = sizeof(uint32_t) * (nb + ntab + 1);
    const size_t smem_place = std::max(PBP_MIN_SMEM, sizeof(uint32_t) * (3 * nb + ntab + 1));
    PBK(cuda_err(cudaFuncSetAttribute(k_pb_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_count)));
    PBK(cuda_err(cudaFuncSetAttribute(k_pb_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_place)));
    if (nC) {
        k_pb_count<<<nC, PBB_THREADS, smem_count, st>>>(g->csr_off, g->csr_col, d_cs, d_tab, sh, ntab, d_bstart,
                                                        nb, d_M, d_chunk_runs, d_chunk_len);
        k_pb_colscan<<<(nb + 255) / 256, 256, 0, st>>>(d_M, d_O, nC, nb, d_total);
    } else {
        PBK(cuda_err(cudaMemsetAsync(d_total, 0, sizeof(uint32_t) * nb, st)));
    }
    PBK(cuda_err(cudaGetLastError()));
    std::vector<uint32_t> total(nb), chunk_runs(nC), chunk_len(nC), abase(nC);
    PBK(cuda_err(cudaMemcpyAsync(total.data(), d_total, sizeof(uint32_t) * nb, cudaMemcpyDeviceToHost, st)));
    if (nC) {
        PBK(cuda_err(cudaMemcpyAsync(chunk_runs.data(), d_chunk_runs, sizeof(uint32_t) * nC, cudaMemcpyDeviceToHost, st)));
        PBK(cuda_err(cudaMemcpyAsync(chunk_len.data(), d_chunk_len, sizeof(uint32_t) * nC, cudaMemcpyDeviceToHost, st)));
    }
    PBK(cuda_err(cudaStreamSynchronize(st)));
    // bin-major places of the bins (padded to 8 entries) and run records per chunk
    std::vector<uint32_t> bbase(nb + 1, 0);
    uint64_t acc = 0;
    for (uint32_t q = 0; q < nb; ++q) {
        bbase[q] = (uint32_t)acc;
        acc += (total[q] + 7ull) & ~7ull;
        if (acc >= 0xFFFFFFF0ull) PBK(IP_E_RANGE);  // entries must be indexable by uint32
    }
    bbase[nb] = (uint32_t)acc;
    const uint64_t P_total = acc;
    uint64_t R = 0, A = 0;
    for (uint32_t c = 0; c < nC; ++c) {
        cinfo[c].z = (uint32_t)R;
        R += chunk_runs[c];
        cinfo[c].w = (uint32_t)R;
        abase[c] = (uint32_t)A;
        A += chunk_len[c];
    }
    if (A >= 0xFFFFFFF0ull) PBK(IP_E_RANGE);
    if (nC) PBK(cuda_err(cudaMemcpyAsync(d_abase, abase.data(), sizeof(uint32_t) * nC, cudaMemcpyHostToDevice, st)));
    if (nC) PBK(cuda_err(cudaMemcpyAsync(d_cs, cinfo.data(), sizeof(uint4) * nC, cudaMemcpyHostToDevice, st)));
    PBK(cuda_err(cudaMemcpyAsync(d_bbase, bbase.data(), sizeof(uint32_t) * (nb + 1), cudaMemcpyHostToDevice, st)));
    uint4* d_runs;
    uint32_t *d_code, *d_hi;
    uint16_t *d_src, *d_dst;
    unsigned long long* d_big;
    PBK(pb_alloc(g, L, &d_runs, R));
    PBK(pb_alloc(g, L, &d_src, A));
    // the edge weights beside the sources, one byte each, where they all fit one
    uint8_t* d_w8 = nullptr;
    if (g->weighted) {
        PBK(graph_max_weight(g, st));
        if (g->max_w <= 255) PBK(pb_alloc(g, L, &d_w8, A));
    }
    PBK(pb_alloc(g, L, &d_dst, P_total));
    PBK(pb_alloc(g, L, &d_code, P_total));
    PBK(pb_alloc(g, L, &d_big, V));
    PBK(pb_alloc(g, L, &d_hi, V));
    PBK(cuda_err(cudaMemsetAsync(d_hi, 0, sizeof(uint32_t) * V, st)));
    // phase-2 tasks, one per bin, in bin order; the tail of every bin (entries after its
    // runs, never written by the placement or a scatter) starts as code 0, destination 0
    std::vector<uint4> tasks(nb);
    std::vector<uint2> tails(nb);
    for (uint32_t q = 0; q < nb; ++q) {
        tasks[q] = make_uint4(bstart[q], bstart[q + 1] - bstart[q], bbase[q], bbase[q + 1]);
        tails[q] = make_uint2(bbase[q] + total[q], bbase[q + 1]);
    }
    PBK(pb_alloc(g, L, &L->tails, nb));
    PBK(cuda_err(cudaMemcpyAsync(L->tails, tails.data(), sizeof(uint2) * nb, cudaMemcpyHostToDevice, st)));
    k_pb_tails_init<<<std::max<uint32_t>(1, (nb + 255) / 256), 256, 0, st>>>(d_code, d_dst, L->tails, nb);
    if (nC)
        k_pb_place<<<nC, PBP_THREADS, smem_place, st>>>(g->csr_off, g->csr_col, d_cs, d_abase, d_tab, sh, ntab,
                                                        d_bstart, d_bbase, nb, d_M, d_O, d_runs, d_src, d_dst,
                                                        g->csr_w, d_w8);
    PBK(cuda_err(cudaGetLastError()));

    uint4* d_tasks;
    uint32_t* d_ctr;
    PBK(pb_alloc(g, L, &d_tasks, nb));
    PBK(pb_alloc(g, L, &d_ctr, 2));
    PBK(cuda_err(cudaMemcpyAsync(d_tasks, tasks.data(), sizeof(uint4) * nb, cudaMemcpyHostToDevice, st)));
    PBK(cuda_err(cudaMemsetAsync(d_ctr, 0, sizeof(uint32_t) * 2, st)));
    PBK(cuda_err(cudaStreamSynchronize(st)));

    d.n_chunks = nC;
    d.n_tasks = nb;
    d.chunk = d_cs;
    d.runs = d_runs;
    d.src = d_src;
    d.w8 = d_w8;
    d.dst = d_dst;
    d.code = d_code;
    d.big = d_big;
    d.tasks = d_tasks;
    d.hi = d_hi;
    d.ctr = d_ctr;
    int lg = 0;
    while (lg < 32 && (1ull << lg) < V) ++lg;
    const int S = std::min(62, 29 + lg);
    d.shift = S;
    d.inv_scale = ldexpf(1.0f, -S);
    d.on = 1;
    *out = L;
    return IP_OK;
}

}  // namespace

bool pb_supported(const ip_graph* g) { return g->V > 0 && g->E > 0 && g->V <= PB_MAX_V; }

int pb_prepare(ip_graph* g, cudaStream_t st, PbDev* out) {
    if (!pb_supported(g)) return IP_E_RANGE;
    if (!g->pb) {
        PbLayout* L = nullptr;
        const int r = build(g, st, &L);
        if (r != IP_OK) return r;
        g->pb = L;
    }
    *out = static_cast<PbLayout*>(g->pb)->d;
    return IP_OK;
}

int pb_launch(const ip_graph* g, const Params& P, cudaStream_t st) {
    const PbLayout* L = static_cast<const PbLayout*>(g->pb);
    k_pb_scatter<<<L->grid1, PB1_THREADS, PB1_SMEM_PR, st>>>(P);
    k_pb_accumulate<<<L->grid2, 32 * (PB2_CONSUMERS + 1), PB2_SMEM, st>>>(P);
    return cuda_err(cudaGetLastError());
}

int pb_min_launch(const ip_graph* g, const Params& P, cudaStream_t st, int kind) {
    const PbLayout* L = static_cast<const PbLayout*>(g->pb);
    if (kind == PB_MIN_COPY)
        k_pbm_scatter<PB_COPY_CODES><<<L->grid1m, PB1_THREADS, PB1_SMEM_MIN, st>>>(P);
    else if (g->weighted)  // run_app checked that the layout holds the weights
        k_pbm_scatter<PB_ADD_W8><<<L->grid1m, PB1_THREADS, PB1_SMEM_MIN, st>>>(P);
    else
        k_pbm_scatter<PB_ADD_ONE><<<L->grid1m, PB1_THREADS, PB1_SMEM_MIN, st>>>(P);
    k_pbm_accumulate<<<L->grid2, 32 * (PB2_CONSUMERS + 1), PB2_SMEM, st>>>(P);
    return cuda_err(cudaGetLastError());
}

int pb_set_mode(ip_graph* g, int min_mode, cudaStream_t st) {
    PbLayout* L = static_cast<PbLayout*>(g->pb);
    if (!L || L->tail_mode == min_mode) return IP_OK;
    const uint32_t nb = L->d.n_tasks;
    k_pb_tails<<<std::max<uint32_t>(1, (nb + 255) / 256), 256, 0, st>>>(L->d.code, L->tails, nb,
                                                                         min_mode ? ipregel::kNoBroadcastBits : 0u);
    const int r = cuda_err(cudaGetLastError());
    if (r == IP_OK) L->tail_mode = min_mode;
    return r;
}

size_t pb_bytes(const ip_graph* g) {
    size_t b = 0;
    if (g->pb)
        for (const auto& x : static_cast<const PbLayout*>(g->pb)->bufs) b += x.second;
    return b;
}

void pb_free(ip_graph* g) {
    if (g->pb) pb_release(g, static_cast<PbLayout*>(g->pb));
    g->pb = nullptr;
}

}  // namespace ipg
