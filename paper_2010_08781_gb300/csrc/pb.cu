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
//   consecutive sources (at most PB_MAXS sources, about PB_CHUNK_E edges), the
//   vertices into bins of consecutive destinations (at most PB_BIN_V vertices and
//   about E / (4 x phase-2 CTAs) in-edges, so that every bin is a balanced task).
//   Inside a chunk the entries are grouped by bin; entry i stores its source
//   relative to the chunk (u16) and its destination relative to the bin (u16).
//   A run is the entries of one chunk into one bin, padded to whole units of 8
//   entries whose broadcast is 0; every bin lists the units of its runs.
//   phase 1 (k_pb_scatter): a CTA stages its chunk's broadcasts in shared
//   memory, as fixed-point codes, and writes code[i] = code of src[i], streaming.
//   phase 2 (k_pb_accumulate): a CTA owns one bin, reads that bin's units and
//   adds every code into a shared-memory accumulator of its destination, then
//   runs compute() (pr_finish) for the bin's vertices.
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
constexpr uint32_t PB_CHUNK_E = 131072;  // target out-edges per chunk
constexpr uint32_t PB_MAX_BINS = 16384;  // bins a chunk histograms in shared memory
constexpr uint32_t PB_MAX_V = 13824u * PB_BIN_V;  // vertex-capped bins plus entry-capped ones fit PB_MAX_BINS
constexpr int PB1_THREADS = 512, PB2_THREADS = 512, PBB_THREADS = 512;
constexpr int PB1_LOADS = 4;  // phase 1: 16-byte loads per thread in flight
constexpr int PB_U = 4;       // phase 2: groups of 64 entries (2 per lane) per claim of 32 units
constexpr size_t PB1_SMEM = (PB_MAXS + 1) * sizeof(uint32_t);
constexpr size_t PB2_SMEM = PB_BIN_V * sizeof(uint32_t);

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
// Staging turns every source's broadcast into its 32-bit code once: the
// fixed-point value itself below 2^31, else 2^31 | source with the 64-bit value
// in big[source]. The entries then only copy codes.
__global__ void __launch_bounds__(PB1_THREADS) k_pb_scatter(Params P) {
    extern __shared__ uint32_t scode[];
    __shared__ uint32_t task;
    const PbDev& B = P.pb;
    const uint32_t s = P.ctl->superstep;  // the superstep being computed
    const float* cur = (s & 1) ? P.contrib0 : P.contrib1;
    if (blockIdx.x == 0 && threadIdx.x == 0) B.ctr[1] = 0;  // phase 2 of this superstep claims from 0
    for (;;) {
        if (threadIdx.x == 0) task = atomicAdd(B.ctr, 1u);
        __syncthreads();
        const uint32_t t = task;
        if (t >= B.n_chunks) break;
        const uint32_t c = B.corder[t];
        const uint32_t s0 = B.chunk[c].x, ns = B.chunk[c].y;
        for (uint32_t i = threadIdx.x; i < ns; i += blockDim.x) {
            uint32_t xl, xh;
            pb_fixed(cur[s0 + i], B.shift, xl, xh);
            uint32_t code = xl;
            if (xh || xl >= 0x80000000u) {
                code = 0x80000000u | (s0 + i);
                B.big[s0 + i] = ((unsigned long long)xh << 32) | xl;
            }
            scode[i] = code;
        }
        if (threadIdx.x == 0) scode[ns] = 0u;  // source of the padding entries
        __syncthreads();
        const uint32_t p8 = B.pbase[c] >> 3, n8 = (B.pbase[c + 1] >> 3) - p8;
        const uint4* src8 = reinterpret_cast<const uint4*>(B.src) + p8;
        uint4* code4 = reinterpret_cast<uint4*>(B.code) + 2 * (size_t)p8;
        for (uint32_t j0 = threadIdx.x; j0 < n8; j0 += PB1_LOADS * blockDim.x) {
            uint4 a[PB1_LOADS];
#pragma unroll
            for (int k = 0; k < PB1_LOADS; ++k) {
                const uint32_t j = j0 + k * blockDim.x;
                a[k] = j < n8 ? __ldcs(src8 + j) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int k = 0; k < PB1_LOADS; ++k) {
                const uint32_t j = j0 + k * blockDim.x;
                if (j < n8) {
                    code4[2 * j] = make_uint4(scode[a[k].x & 0xFFFF], scode[a[k].x >> 16], scode[a[k].y & 0xFFFF],
                                              scode[a[k].y >> 16]);
                    code4[2 * j + 1] = make_uint4(scode[a[k].z & 0xFFFF], scode[a[k].z >> 16],
                                                  scode[a[k].w & 0xFFFF], scode[a[k].w >> 16]);
                }
            }
        }
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

// One claim of a warp: 32 units (256 entries); lane l holds the index of unit
// l. In group g lane l takes entries 2(l % 4) and 2(l % 4) + 1 of unit
// 8g + l / 4, so the four lanes of a unit read one aligned 32-byte sector of
// codes.
struct PbClaim {
    uint2 c[PB_U];
    uint32_t d[PB_U];
};

__device__ __forceinline__ void pb_load(const PbDev& B, uint32_t u, uint32_t my, uint32_t ue, uint32_t lane,
                                        PbClaim& x) {
#pragma unroll
    for (int g = 0; g < PB_U; ++g) {
        const uint32_t k = 8 * g + (lane >> 2);
        const uint32_t unit = __shfl_sync(FULL, my, k);
        const bool ok = u + k < ue;
        const uint32_t pos = unit * 8 + 2 * (lane & 3);
        x.c[g] = ok ? __ldcs(reinterpret_cast<const uint2*>(B.code + pos)) : make_uint2(0, 0);
        x.d[g] = ok ? __ldcs(reinterpret_cast<const uint32_t*>(B.dst + pos)) : 0u;
    }
}

// Adds one claim: branch free for codes below 2^31 (their own value); carries
// into the high words and big contributions take a warp-uniform slow path that
// reads the flagged entries again.
__device__ __forceinline__ void pb_accumulate_claim(const PbDev& B, uint32_t* acc_lo, uint32_t* hi,
                                                    const PbClaim& x, uint32_t my, uint32_t lane) {
    uint32_t carry = 0, bigs = 0;
#pragma unroll
    for (int g = 0; g < PB_U; ++g) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t code = h ? x.c[g].y : x.c[g].x;
            const uint32_t big = code >> 31;
            const uint32_t v = big ? 0u : code;
            const uint32_t old = atomicAdd(acc_lo + ((x.d[g] >> (16 * h)) & 0xFFFFu), v);
            carry |= (old + v < old ? 1u : 0u) << (2 * g + h);
            bigs |= big << (2 * g + h);
        }
    }
    if (__any_sync(FULL, carry | bigs)) {
        for (int g = 0; g < PB_U; ++g) {
            const uint32_t unit = __shfl_sync(FULL, my, 8 * g + (lane >> 2));
            const uint32_t pos = unit * 8 + 2 * (lane & 3);
            for (int h = 0; h < 2; ++h) {
                const uint32_t bit = 2 * g + h;
                if (((carry | bigs) >> bit) & 1u) {
                    const uint32_t d = B.dst[pos + h];
                    if ((carry >> bit) & 1u) atomicAdd(hi + d, 1u);
                    if ((bigs >> bit) & 1u) pb_add_big(B, acc_lo, hi, d, B.code[pos + h]);
                }
            }
        }
    }
}

// Warps claim 32 units at a time from the bin's unit list. Software pipeline:
// the unit indices of claim n+2 and the codes of claim n+1 are in flight while
// claim n is added.
__global__ void __launch_bounds__(PB2_THREADS, 2) k_pb_accumulate(Params P) {
    extern __shared__ uint32_t acc_lo[];
    __shared__ uint32_t task, next_unit;
    const PbDev& B = P.pb;
    const uint32_t s = P.ctl->superstep;
    float* nxt = (s & 1) ? P.contrib1 : P.contrib0;
    const uint32_t lane = threadIdx.x & 31;
    const float inv_scale = B.inv_scale;
    if (blockIdx.x == 0 && threadIdx.x == 0) B.ctr[0] = 0;  // phase 1 of the next superstep claims from 0
    for (;;) {
        if (threadIdx.x == 0) task = atomicAdd(B.ctr + 1, 1u);
        __syncthreads();
        const uint32_t t = task;
        if (t >= B.n_tasks) break;
        const uint4 tk = B.tasks[t];  // {first vertex, vertices, first unit, end unit}
        const uint32_t v0 = tk.x, nv = tk.y, ue = tk.w;
        uint32_t* hi = B.hi + v0;
        for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) acc_lo[i] = 0;
        if (threadIdx.x == 0) next_unit = tk.z;
        __syncthreads();
        auto claim = [&](uint32_t& u, uint32_t& my) {
            uint32_t c = 0;
            if (lane == 0) c = atomicAdd(&next_unit, 32u);
            u = __shfl_sync(FULL, c, 0);
            my = u + lane < ue ? __ldcs(B.units + u + lane) : 0u;
        };
        uint32_t u0, my0, u1, my1;
        claim(u0, my0);
        claim(u1, my1);
        PbClaim x0, x1;
        if (u0 < ue) pb_load(B, u0, my0, ue, lane, x0);
        while (u0 < ue) {
            uint32_t u2, my2;
            claim(u2, my2);
            if (u1 < ue) pb_load(B, u1, my1, ue, lane, x1);
            pb_accumulate_claim(B, acc_lo, hi, x0, my0, lane);
            u0 = u1;
            my0 = my1;
            x0 = x1;
            u1 = u2;
            my1 = my2;
        }
        __syncthreads();  // also orders this CTA's high-word atomics before the reads below
        for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) {
            const uint32_t h = __ldcg(hi + i);
            if (h) hi[i] = 0;
            pr_finish(P, v0 + i, pb_value(h, acc_lo[i], inv_scale), s, nxt);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- layout build
__global__ void k_pb_binof(const uint32_t* __restrict__ bstart, uint32_t* binof) {
    const uint32_t q = blockIdx.x;
    for (uint32_t v = bstart[q] + threadIdx.x; v < bstart[q + 1]; v += blockDim.x) binof[v] = q;
}

// Entries per bin of one chunk, in shared memory.
__device__ __forceinline__ void pb_hist(const uint32_t* __restrict__ col, const uint32_t* __restrict__ binof,
                                        uint32_t e0, uint32_t e1, uint32_t nb, uint32_t* hist) {
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) atomicAdd(hist + binof[col[e]], 1u);
    __syncthreads();
}

__device__ __forceinline__ uint32_t pad8(uint32_t n) { return (n + 7) & ~7u; }

// Per chunk: units (8 entries, runs padded to whole units) per bin, and the
// chunk's unit count.
__global__ void __launch_bounds__(PBB_THREADS) k_pb_count(const uint32_t* __restrict__ csr_off,
                                                          const uint32_t* __restrict__ col,
                                                          const uint2* __restrict__ cs,
                                                          const uint32_t* __restrict__ binof, uint32_t nb,
                                                          uint32_t* unit_count, uint32_t* chunk_units) {
    extern __shared__ uint32_t hist[];
    const uint32_t c = blockIdx.x;
    pb_hist(col, binof, csr_off[cs[c].x], csr_off[cs[c].x + cs[c].y], nb, hist);
    uint32_t mine = 0;
    for (uint32_t q = threadIdx.x; q < nb; q += blockDim.x) {
        const uint32_t n = pad8(hist[q]) >> 3;
        if (n) atomicAdd(unit_count + q, n);
        mine += n;
    }
    for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(FULL, mine, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(chunk_units + c, mine);
}

// Per chunk: place every out-edge into its bin's run, pad the run to whole units
// with entries of source `ns` (whose staged code is 0), and list the units.
__global__ void __launch_bounds__(PBB_THREADS) k_pb_place(const uint32_t* __restrict__ csr_off,
                                                          const uint32_t* __restrict__ col,
                                                          const uint2* __restrict__ cs,
                                                          const uint32_t* __restrict__ pbase,
                                                          const uint32_t* __restrict__ binof,
                                                          const uint32_t* __restrict__ bstart, uint32_t nb,
                                                          const uint32_t* __restrict__ unit_off, uint32_t* unit_cur,
                                                          uint32_t* units, uint16_t* src, uint16_t* dst) {
    extern __shared__ uint32_t sm[];
    uint32_t* cnt = sm;        // [nb]: entries per bin, then the placement cursor
    uint32_t* offs = sm + nb;  // [ns + 1]: the chunk's CSR offsets
    __shared__ uint32_t wsum[PBB_THREADS / 32];
    const uint32_t c = blockIdx.x, s0 = cs[c].x, ns = cs[c].y, p0 = pbase[c];
    for (uint32_t i = threadIdx.x; i <= ns; i += blockDim.x) offs[i] = csr_off[s0 + i];
    pb_hist(col, binof, csr_off[s0], csr_off[s0 + ns], nb, cnt);
    const uint32_t e0 = offs[0], e1 = offs[ns];
    // exclusive scan of the padded counts: thread t owns bins [b0, b1)
    const uint32_t per = (nb + blockDim.x - 1) / blockDim.x;
    const uint32_t b0 = min(nb, threadIdx.x * per), b1 = min(nb, b0 + per);
    uint32_t mine = 0;
    for (uint32_t q = b0; q < b1; ++q) mine += pad8(cnt[q]);
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= (uint32_t)o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t run = inc - mine;
    for (uint32_t k = 0; k < w; ++k) run += wsum[k];
    for (uint32_t q = b0; q < b1; ++q) {
        const uint32_t n = cnt[q], n8 = pad8(n);
        if (n) {
            const uint32_t nu = n8 >> 3;
            const uint32_t slot = unit_off[q] + atomicAdd(unit_cur + q, nu);
            const uint32_t first = (p0 + run) >> 3;
            for (uint32_t k = 0; k < nu; ++k) units[slot + k] = first + k;
            for (uint32_t k = n; k < n8; ++k) {
                src[p0 + run + k] = (uint16_t)ns;
                dst[p0 + run + k] = 0;
            }
        }
        cnt[q] = run;
        run += n8;
    }
    __syncthreads();
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const uint32_t v = col[e], q = binof[v];
        uint32_t lo = 0, hi = ns;  // offs[lo] <= e < offs[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (offs[mid] <= e)
                lo = mid;
            else
                hi = mid;
        }
        const uint32_t pos = p0 + atomicAdd(cnt + q, 1u);
        src[pos] = (uint16_t)lo;
        dst[pos] = (uint16_t)(v - bstart[q]);
    }
}

// Host-side owner of the layout's device buffers.
struct PbLayout {
    PbDev d;
    std::vector<std::pair<void*, size_t>> bufs;
    int grid1 = 0, grid2 = 0;
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
        cudaFree(b.first);
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
            cudaFree(p);
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
    PBK(cuda_err(cudaFuncSetAttribute(k_pb_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PB1_SMEM)));
    PBK(cuda_err(cudaFuncSetAttribute(k_pb_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PB2_SMEM)));
    L->grid1 = occupancy_grid(g, (const void*)k_pb_scatter, PB1_THREADS, PB1_SMEM);
    L->grid2 = occupancy_grid(g, (const void*)k_pb_accumulate, PB2_THREADS, PB2_SMEM);

    // chunks of consecutive sources, cut by edge count and by source count; runs of
    // sources without out-edges that would form a chunk of their own are skipped
    std::vector<uint32_t> off(V + 1);
    PBK(cuda_err(cudaMemcpyAsync(off.data(), g->csr_off, sizeof(uint32_t) * (V + 1), cudaMemcpyDeviceToHost, st)));
    PBK(cuda_err(cudaStreamSynchronize(st)));
    std::vector<uint2> chunks;
    for (uint32_t u = 0; u < V;) {
        const uint32_t first = u, e0 = off[u];
        ++u;
        while (u < V && u - first < PB_MAXS && off[u + 1] - e0 <= PB_CHUNK_E) ++u;
        if (off[u] != e0) chunks.push_back(make_uint2(first, u - first));
    }
    const uint32_t nC = (uint32_t)chunks.size();
    // bins of consecutive destinations, cut by vertex count and by in-edge count
    PBK(cuda_err(cudaMemcpyAsync(off.data(), g->csc_off, sizeof(uint32_t) * (V + 1), cudaMemcpyDeviceToHost, st)));
    PBK(cuda_err(cudaStreamSynchronize(st)));
    const uint64_t bin_e = std::max<uint64_t>(16384, (g->E + 4ull * L->grid2 - 1) / (4ull * L->grid2));
    std::vector<uint32_t> bstart{0};
    for (uint32_t v = 0; v < V;) {
        const uint32_t first = v, e0 = off[v];
        ++v;
        while (v < V && v - first < PB_BIN_V && off[v + 1] - e0 <= bin_e) ++v;
        bstart.push_back(v);
    }
    const uint32_t nb = (uint32_t)bstart.size() - 1;
    if (nb > PB_MAX_BINS) PBK(IP_E_RANGE);
    off.clear();
    off.shrink_to_fit();

    uint2* d_cs;
    uint32_t *d_pbase, *d_unit_count, *d_corder, *d_chunk_units;
    PBK(pb_alloc(g, L, &d_cs, nC));
    PBK(pb_alloc(g, L, &d_pbase, nC + 1));
    PBK(pb_alloc(g, L, &d_corder, nC));
    PBK(pb_alloc(g, L, &d_chunk_units, nC));
    PBK(pb_alloc(g, L, &d_unit_count, nb));
    TmpBuf t_binof{g}, t_bstart{g}, t_unit_cur{g}, t_unit_off{g};
    uint32_t *d_binof, *d_bstart, *d_unit_cur, *d_unit_off;
    PBK(t_binof.alloc(&d_binof, V));
    PBK(t_bstart.alloc(&d_bstart, nb + 1));
    PBK(t_unit_cur.alloc(&d_unit_cur, nb));
    PBK(t_unit_off.alloc(&d_unit_off, nb + 1));
    if (nC) PBK(cuda_err(cudaMemcpyAsync(d_cs, chunks.data(), sizeof(uint2) * nC, cudaMemcpyHostToDevice, st)));
    PBK(cuda_err(cudaMemcpyAsync(d_bstart, bstart.data(), sizeof(uint32_t) * (nb + 1), cudaMemcpyHostToDevice, st)));
    PBK(cuda_err(cudaMemsetAsync(d_unit_count, 0, sizeof(uint32_t) * nb, st)));
    PBK(cuda_err(cudaMemsetAsync(d_unit_cur, 0, sizeof(uint32_t) * nb, st)));
    PBK(cuda_err(cudaMemsetAsync(d_chunk_units, 0, sizeof(uint32_t) * std::max<uint32_t>(nC, 1), st)));
    k_pb_binof<<<nb, 256, 0, st>>>(d_bstart, d_binof);
    const size_t smem_count = sizeof(uint32_t) * nb;
    const size_t smem_place = sizeof(uint32_t) * (nb + PB_MAXS + 1);
    PBK(cuda_err(cudaFuncSetAttribute(k_pb_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_count)));
    PBK(cuda_err(cudaFuncSetAttribute(k_pb_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_place)));
    if (nC)
        k_pb_count<<<nC, PBB_THREADS, smem_count, st>>>(g->csr_off, g->csr_col, d_cs, d_binof, nb, d_unit_count,
                                                        d_chunk_units);
    PBK(cuda_err(cudaGetLastError()));
    std::vector<uint32_t> unit_off(nb + 1, 0), chunk_units(nC);
    PBK(cuda_err(cudaMemcpyAsync(unit_off.data() + 1, d_unit_count, sizeof(uint32_t) * nb, cudaMemcpyDeviceToHost, st)));
    if (nC)
        PBK(cuda_err(cudaMemcpyAsync(chunk_units.data(), d_chunk_units, sizeof(uint32_t) * nC, cudaMemcpyDeviceToHost, st)));
    PBK(cuda_err(cudaStreamSynchronize(st)));
    uint64_t total_units = 0;
    for (uint32_t q = 0; q < nb; ++q) {
        total_units += unit_off[q + 1];
        if (total_units >= (1ull << 29)) PBK(IP_E_RANGE);  // entries must be indexable by uint32
        unit_off[q + 1] = (uint32_t)total_units;
    }
    std::vector<uint32_t> pbase(nC + 1, 0);
    for (uint32_t c = 0; c < nC; ++c) pbase[c + 1] = pbase[c] + 8 * chunk_units[c];
    const uint64_t P_total = (uint64_t)pbase[nC];
    PBK(cuda_err(cudaMemcpyAsync(d_unit_off, unit_off.data(), sizeof(uint32_t) * (nb + 1), cudaMemcpyHostToDevice, st)));
    PBK(cuda_err(cudaMemcpyAsync(d_pbase, pbase.data(), sizeof(uint32_t) * (nC + 1), cudaMemcpyHostToDevice, st)));
    uint32_t *d_units, *d_code, *d_hi;
    uint16_t *d_src, *d_dst;
    unsigned long long* d_big;
    PBK(pb_alloc(g, L, &d_units, total_units));
    PBK(pb_alloc(g, L, &d_src, P_total));
    PBK(pb_alloc(g, L, &d_dst, P_total));
    PBK(pb_alloc(g, L, &d_code, P_total));
    PBK(pb_alloc(g, L, &d_big, V));
    PBK(pb_alloc(g, L, &d_hi, V));
    PBK(cuda_err(cudaMemsetAsync(d_hi, 0, sizeof(uint32_t) * V, st)));
    if (nC)
        k_pb_place<<<nC, PBB_THREADS, smem_place, st>>>(g->csr_off, g->csr_col, d_cs, d_pbase, d_binof, d_bstart, nb,
                                                        d_unit_off, d_unit_cur, d_units, d_src, d_dst);
    PBK(cuda_err(cudaGetLastError()));

    // phase-2 tasks, one per bin, in bin order: neighbouring bins run at the same
    // time, so the sectors their runs share at chunk-region boundaries are read
    // from DRAM once. Phase-1 chunks, largest first.
    std::vector<uint4> tasks(nb);
    for (uint32_t q = 0; q < nb; ++q)
        tasks[q] = make_uint4(bstart[q], bstart[q + 1] - bstart[q], unit_off[q], unit_off[q + 1]);
    std::vector<uint32_t> corder(nC);
    std::iota(corder.begin(), corder.end(), 0u);
    std::stable_sort(corder.begin(), corder.end(),
                     [&](uint32_t a, uint32_t b) { return chunk_units[a] > chunk_units[b]; });
    uint4* d_tasks;
    uint32_t* d_ctr;
    PBK(pb_alloc(g, L, &d_tasks, nb));
    PBK(pb_alloc(g, L, &d_ctr, 2));
    PBK(cuda_err(cudaMemcpyAsync(d_tasks, tasks.data(), sizeof(uint4) * nb, cudaMemcpyHostToDevice, st)));
    if (nC) PBK(cuda_err(cudaMemcpyAsync(d_corder, corder.data(), sizeof(uint32_t) * nC, cudaMemcpyHostToDevice, st)));
    PBK(cuda_err(cudaMemsetAsync(d_ctr, 0, sizeof(uint32_t) * 2, st)));
    PBK(cuda_err(cudaStreamSynchronize(st)));

    d.n_chunks = nC;
    d.n_tasks = nb;
    d.chunk = d_cs;
    d.pbase = d_pbase;
    d.corder = d_corder;
    d.src = d_src;
    d.dst = d_dst;
    d.code = d_code;
    d.big = d_big;
    d.units = d_units;
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
    k_pb_scatter<<<L->grid1, PB1_THREADS, PB1_SMEM, st>>>(P);
    k_pb_accumulate<<<L->grid2, PB2_THREADS, PB2_SMEM, st>>>(P);
    return cuda_err(cudaGetLastError());
}

void pb_free(ip_graph* g) {
    if (g->pb) pb_release(g, static_cast<PbLayout*>(g->pb));
    g->pb = nullptr;
}

}  // namespace ipg
