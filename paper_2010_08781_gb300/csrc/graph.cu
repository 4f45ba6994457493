// Graph store: creation (validation, upload, device-side transposition),
// vertex renumbering by degree class, degree bins, value readback, selector
// upload, the process-wide device-buffer cache and the small ABI helpers.
//
// The paper keeps one global vertex array and one global adjacency array
// shared by all threads (Section 4.2). Here the adjacency is held twice on the
// device: CSR (out-edges, used by push) and CSC (in-edges, used by pull,
// Section 4.3.2), with uint32 IDs and offsets. Edge arrays are padded to a
// multiple of four entries plus four, so kernels can read any aligned 16-byte
// block that overlaps a vertex's edge range.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace ipg {

int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return IP_OK;
    if (e == cudaErrorMemoryAllocation) return IP_E_NOMEM;
    return IP_E_CUDA;
}

#define CK(x)                              \
    do {                                   \
        int _r = cuda_err(x);              \
        if (_r != IP_OK) return _r;        \
    } while (0)

// Process-wide cache of the library's device buffers, by device and exact size.
// ip_graph_destroy returns a graph's buffers here (after one device
// synchronisation) instead of freeing them, and the next allocation of the same
// size on the same device takes one back: a caller that builds graphs of the same
// shape again and again pays cudaMalloc / cudaFree (which synchronises) once. At
// most dev_cache_cap() bytes stay cached (a quarter of the device's memory, at most
// 64 GiB: two billion-edge graphs); an allocation that fails first releases the
// cache of its device; ip_release_cached_memory() releases everything.
namespace {
size_t dev_cache_cap() {
    static const size_t cap = [] {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            (void)cudaGetLastError();
            return (size_t)32 << 30;
        }
        return std::min<size_t>((size_t)64 << 30, total_b / 4);
    }();
    return cap;
}
struct DeviceCache {
    std::mutex m;
    std::unordered_map<void*, std::pair<int, size_t>> live;   // buffers handed out: device, size
    std::multimap<std::pair<int, size_t>, void*> cached;      // returned buffers, by (device, size)
    size_t cached_bytes = 0;
};
DeviceCache& dcache() {
    static DeviceCache* c = new DeviceCache();  // never destroyed: no ordering problem at process exit
    return *c;
}

// Frees the cached buffers of one device (dev < 0: of every device). Caller holds the lock.
void dcache_trim_locked(DeviceCache& C, int dev) {
    int cur = -1;
    (void)cudaGetDevice(&cur);
    for (auto it = C.cached.begin(); it != C.cached.end();) {
        if (dev >= 0 && it->first.first != dev) {
            ++it;
            continue;
        }
        (void)cudaSetDevice(it->first.first);
        cudaFree(it->second);
        C.cached_bytes -= it->first.second;
        it = C.cached.erase(it);
    }
    if (cur >= 0) (void)cudaSetDevice(cur);
}

// Hands a library buffer back to the cache (the device has been synchronised).
void dcache_release(void* p) {
    if (!p) return;
    DeviceCache& C = dcache();
    std::lock_guard<std::mutex> l(C.m);
    auto it = C.live.find(p);
    if (it == C.live.end()) {
        cudaFree(p);
        return;
    }
    const std::pair<int, size_t> key = it->second;
    C.live.erase(it);
    if (C.cached_bytes + key.second <= dev_cache_cap()) {
        C.cached.insert({key, p});
        C.cached_bytes += key.second;
    } else {
        cudaFree(p);
    }
}
}  // namespace

int alloc_dev(ip_graph* g, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    DeviceCache& C = dcache();
    std::lock_guard<std::mutex> l(C.m);
    auto it = C.cached.find({g->device, bytes});
    if (it != C.cached.end()) {
        *p = it->second;
        C.cached.erase(it);
        C.cached_bytes -= bytes;
    } else {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaErrorMemoryAllocation && C.cached_bytes) {
            (void)cudaGetLastError();
            dcache_trim_locked(C, g->device);
            e = cudaMalloc(p, bytes);
        }
        if (e != cudaSuccess) {
            *p = nullptr;
            (void)cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? IP_E_NOMEM : IP_E_CUDA;
        }
    }
    C.live[*p] = {g->device, bytes};
    g->device_bytes += bytes;
    return IP_OK;
}

// While set on a thread, free_dev hands buffers to the cache instead of freeing
// them: the caller has synchronised the device, so no launch still reads them.
static thread_local bool t_device_idle = false;
struct DeviceIdleScope {
    DeviceIdleScope() { t_device_idle = true; }
    ~DeviceIdleScope() { t_device_idle = false; }
};

// Frees a library buffer now (mid-run frees: bin sets, regrown logs, build temporaries).
void free_dev(void* p) {
    if (!p) return;
    if (t_device_idle) {
        dcache_release(p);
        return;
    }
    DeviceCache& C = dcache();
    {
        std::lock_guard<std::mutex> l(C.m);
        C.live.erase(p);
    }
    cudaFree(p);
}

static size_t edge_alloc_count(uint64_t E) { return (size_t)(((E + 3) & ~3ull) + 4); }

// ------------------------------------------------------------------ kernels
__global__ void k_validate_offsets(const uint32_t* off, uint32_t n, uint64_t E, unsigned int* err) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (off[i + 1] < off[i]) atomicOr(err, 1u);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (off[0] != 0 || (uint64_t)off[n] != E) atomicOr(err, 1u);
    }
}

__global__ void k_validate_ids(const uint32_t* ids, uint64_t E, uint32_t n, unsigned int* err) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < E; i += (uint64_t)gridDim.x * blockDim.x)
        if (ids[i] >= n) atomicOr(err, 2u);
}

__global__ void k_degrees(const uint32_t* off, uint32_t n, float* inv_outdeg, unsigned int* max_deg) {
    unsigned int mx = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t d = off[v + 1] - off[v];
        if (inv_outdeg) inv_outdeg[v] = d ? 1.0f / (float)d : 0.0f;
        mx = max(mx, d);
    }
    mx = __reduce_max_sync(FULL, mx);
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(max_deg, mx);
}

// In-degrees: one reduction per edge into its destination's counter. The counters of
// the first CI_HOT vertices are kept per CTA in shared memory and added once at the
// end: after the renumbering by degree class those are the high-degree vertices,
// whose global counters share a few L2 lines that every SM's reductions would queue
// on. Edges are read 4 at a time (col is 16-byte aligned; the last E % 4 singly).
constexpr uint32_t CI_HOT = 8192;
constexpr int CI_THREADS = 512;
__global__ void __launch_bounds__(CI_THREADS) k_count_in(const uint32_t* __restrict__ col, uint64_t E, uint32_t n,
                                                         uint32_t* cnt) {
    __shared__ uint32_t hot[CI_HOT];
    const uint32_t H = min(n, CI_HOT);
    for (uint32_t i = threadIdx.x; i < H; i += blockDim.x) hot[i] = 0;
    __syncthreads();
    auto add = [&](uint32_t v) {
        if (v < H)
            atomicAdd(hot + v, 1u);
        else
            atomicAdd(cnt + v, 1u);
    };
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t E4 = E / 4;
    const uint4* c4 = reinterpret_cast<const uint4*>(col);
    for (uint64_t i = tid; i < E4; i += stride) {
        const uint4 v = c4[i];
        add(v.x);
        add(v.y);
        add(v.z);
        add(v.w);
    }
    for (uint64_t i = E4 * 4 + tid; i < E; i += stride) add(col[i]);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < H; i += blockDim.x)
        if (hot[i]) atomicAdd(cnt + i, hot[i]);
}

// Exclusive scan of n uint32 values in place, one CTA of 1024 threads per
// chunk of 4096; per-chunk totals written to sums.
__global__ void k_scan_chunks(uint32_t* data, uint64_t n, uint32_t* sums) {
    __shared__ uint32_t warp_tot[32];
    const uint64_t base = (uint64_t)blockIdx.x * 4096 + threadIdx.x * 4;
    uint32_t x[4];
    uint32_t t = 0;
    for (int j = 0; j < 4; ++j) {
        x[j] = base + j < n ? data[base + j] : 0u;
        t += x[j];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = t;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = warp_tot[lane];
        uint32_t wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += y;
        }
        warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
        if (lane == 31 && sums) sums[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run = warp_tot[wid] + inc - t;
    for (int j = 0; j < 4; ++j) {
        if (base + j < n) data[base + j] = run;
        run += x[j];
    }
}

__global__ void k_add_chunk_offsets(uint32_t* data, uint64_t n, const uint32_t* offs) {
    const uint64_t base = (uint64_t)blockIdx.x * 4096;
    const uint32_t add = offs[blockIdx.x];
    for (uint32_t j = threadIdx.x; j < 4096; j += blockDim.x)
        if (base + j < n) data[base + j] += add;
}

int exclusive_scan(ip_graph* g, uint32_t* data, uint64_t n, cudaStream_t st) {
    uint64_t chunks = (n + 4095) / 4096;
    if (chunks <= 1) {
        k_scan_chunks<<<1, 1024, 0, st>>>(data, n, nullptr);
        return cuda_err(cudaGetLastError());
    }
    uint32_t* sums = nullptr;
    int r = alloc_dev(g, (void**)&sums, chunks * sizeof(uint32_t));
    if (r) return r;
    g->device_bytes -= chunks * sizeof(uint32_t);
    k_scan_chunks<<<(unsigned)chunks, 1024, 0, st>>>(data, n, sums);
    r = cuda_err(cudaGetLastError());
    if (!r) r = exclusive_scan(g, sums, chunks, st);
    if (!r) {
        k_add_chunk_offsets<<<(unsigned)chunks, 1024, 0, st>>>(data, n, sums);
        r = cuda_err(cudaGetLastError());
    }
    cudaStreamSynchronize(st);
    free_dev(sums);
    return r;
}

// Edge chunks for the warp-per-chunk edge kernels (transposition, renumbering copy).
constexpr uint32_t RL_CH = 1024;
constexpr uint32_t RL_UNROLL = 4;

// chunk_src[c] = the source of edge position c * RL_CH (largest s with off[s] <= c * RL_CH).
__global__ void k_rl_chunk_src(const uint32_t* __restrict__ off_new, uint32_t n, uint32_t n_chunks,
                               uint32_t* chunk_src) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n_chunks; c += gridDim.x * blockDim.x) {
        const uint64_t p = (uint64_t)c * RL_CH;
        uint32_t lo = 0, hi = n;  // off_new[lo] <= p; the answer is below hi
        while (hi - lo > 1) {
            const uint32_t mid = lo + (hi - lo) / 2;
            if (off_new[mid] <= p)
                lo = mid;
            else
                hi = mid;
        }
        chunk_src[c] = lo;
    }
}

// Transposition scatter: edge e = (u, v) goes to a free slot of v's in-list
// (slot order inside an in-list follows atomic arrival order). One warp per chunk
// of RL_CH consecutive edges: the chunk's first source comes from chunk_src, the
// warp keeps the first edges of 32 consecutive sources in registers and finds each
// lane's source by a 5-step shuffle search (a source owns edge e when it is the
// last one starting at or before e), so no edge searches the whole offset array.
__global__ void k_scatter_in(const uint32_t* __restrict__ csr_off, const uint32_t* __restrict__ chunk_src,
                             const uint32_t* __restrict__ col, const uint32_t* __restrict__ w, uint32_t n,
                             uint64_t E, uint32_t n_chunks, uint32_t* cursor, uint32_t* __restrict__ row,
                             uint32_t* __restrict__ wt) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += nw) {
        const uint64_t p0 = (uint64_t)c * RL_CH;
        const uint64_t p1 = p0 + RL_CH < E ? p0 + RL_CH : E;
        for (uint64_t s = chunk_src[c];; s += 32) {  // windows of 32 sources
            const uint64_t sl = s + lane;
            const uint32_t wo = sl < n ? csr_off[sl] : (uint32_t)E;  // the lane's source: its first edge
            const uint64_t wend = s + 32 <= n ? (uint64_t)csr_off[s + 32] : E;
            const uint64_t w0 = __shfl_sync(FULL, wo, 0);
            const uint64_t lo = p0 > w0 ? p0 : w0, hi = p1 < wend ? p1 : wend;
            for (uint64_t base = lo; base < hi; base += 32 * RL_UNROLL) {
                uint32_t e[RL_UNROLL], u[RL_UNROLL], v[RL_UNROLL], wv[RL_UNROLL];
#pragma unroll
                for (uint32_t k = 0; k < RL_UNROLL; ++k) {
                    const uint64_t ee = base + 32 * k + lane;
                    e[k] = ee < hi ? (uint32_t)ee : 0xFFFFFFFFu;
                    uint32_t i = 0;  // largest i with wo(i) <= e
#pragma unroll
                    for (uint32_t step = 16; step; step >>= 1)
                        if (__shfl_sync(FULL, wo, i + step) <= e[k]) i += step;
                    u[k] = (uint32_t)(s + i);
                }
#pragma unroll
                for (uint32_t k = 0; k < RL_UNROLL; ++k) {
                    v[k] = e[k] != 0xFFFFFFFFu ? col[e[k]] : 0u;
                    wv[k] = (w && e[k] != 0xFFFFFFFFu) ? w[e[k]] : 0u;
                }
#pragma unroll
                for (uint32_t k = 0; k < RL_UNROLL; ++k)
                    if (e[k] != 0xFFFFFFFFu) {
                        const uint32_t pos = atomicAdd(&cursor[v[k]], 1u);
                        row[pos] = u[k];
                        if (w) wt[pos] = wv[k];
                    }
            }
            if (wend >= p1) break;
        }
    }
}

// ------------------------------------------------------------------ helpers
static int grid_for(const ip_graph* g, uint64_t work) {
    uint64_t b = (work + 255) / 256;
    uint64_t cap = (uint64_t)g->num_sms * 16;
    if (b > cap) b = cap;
    return (int)(b ? b : 1);
}

static void free_binset(ip_graph* g, BinSet* S) {
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i < 5; ++i)
            if (S->mem[k][i]) {
                free_dev(S->mem[k][i]);
                g->device_bytes -= S->bytes[k][i];
            }
    delete S;
}

static int bin_alloc(ip_graph* g, BinSet* S, int k, int i, size_t bytes) {
    bytes = bytes ? bytes : 16;
    int r = alloc_dev(g, &S->mem[k][i], bytes);
    if (!r) S->bytes[k][i] = bytes;
    return r;
}

// Degree bins on the device. Counting pass: medium vertices (t1 < deg < t2), heavy
// vertices (deg >= t2) and their chunks of at most HCH edges, warp-aggregated.
__global__ void k_bin_count(const uint32_t* __restrict__ off, uint32_t n, uint32_t t1, uint32_t t2, uint32_t* cnt) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t wbase = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u, wstride = gridDim.x * blockDim.x;
    uint32_t med = 0, hv = 0, ch = 0;
    for (uint32_t v0 = wbase; v0 < n; v0 += wstride) {  // the same trip count for the 32 lanes of a warp
        const uint32_t v = v0 + lane;
        const uint32_t d = v < n ? off[v + 1] - off[v] : 0u;
        med += (d > t1 && d < t2) ? 1u : 0u;
        if (d >= t2) {
            ++hv;
            ch += (d + HCH - 1) / HCH;
        }
    }
    for (int o = 16; o; o >>= 1) {
        med += __shfl_xor_sync(0xFFFFFFFFu, med, o);
        hv += __shfl_xor_sync(0xFFFFFFFFu, hv, o);
        ch += __shfl_xor_sync(0xFFFFFFFFu, ch, o);
    }
    if (lane == 0) {
        if (med) atomicAdd(cnt, med);
        if (hv) atomicAdd(cnt + 1, hv);
        if (ch) atomicAdd(cnt + 2, ch);
    }
}

// Filling pass (cnt = cursors from 0): the medium list, and per heavy vertex its
// table entry {first chunk, chunks} and its chunks {vertex, first edge, end edge,
// heavy-vertex index} in edge order (the PageRank finish sums partials in that order).
__global__ void k_bin_fill(const uint32_t* __restrict__ off, uint32_t n, uint32_t t1, uint32_t t2, uint32_t* cnt,
                           uint32_t* med, uint4* chunks, uint2* hvert) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t wbase = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u, wstride = gridDim.x * blockDim.x;
    for (uint32_t v0 = wbase; v0 < n; v0 += wstride) {
        const uint32_t v = v0 + lane;
        const uint32_t b = v < n ? off[v] : 0u, e = v < n ? off[v + 1] : 0u, d = e - b;
        const bool is_med = d > t1 && d < t2;
        const uint32_t mask = __ballot_sync(0xFFFFFFFFu, is_med);
        uint32_t base = 0;
        if (lane == 0 && mask) base = atomicAdd(cnt, (uint32_t)__popc(mask));
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (is_med) med[base + __popc(mask & ((1u << lane) - 1u))] = v;
        if (d >= t2) {
            const uint32_t nch = (d + HCH - 1) / HCH;
            const uint32_t hi = atomicAdd(cnt + 1, 1u), c0 = atomicAdd(cnt + 2, nch);
            hvert[hi] = make_uint2(c0, nch);
            for (uint32_t c = 0; c < nch; ++c) {
                const uint32_t cb = b + c * HCH;
                chunks[c0 + c] = make_uint4(v, cb, (e - cb) > HCH ? cb + HCH : e, hi);
            }
        }
    }
}

// Static degree bins of one direction, built on the device from the offsets;
// the host reads back only the three list sizes.
static int build_bins(ip_graph* g, BinSet* S, int k, const uint32_t* dev_off, cudaStream_t st) {
    const uint32_t n = g->V, t1 = S->t1, t2 = S->t2;
    uint32_t* cnt = g->bin_cnt;  // [3], device
    CK(cudaMemsetAsync(cnt, 0, 3 * sizeof(uint32_t), st));
    const int grid = std::max(1, std::min(g->num_sms * 8, (int)(((uint64_t)n + 255) / 256)));
    k_bin_count<<<grid, 256, 0, st>>>(dev_off, n, t1, t2, cnt);
    CK(cudaGetLastError());
    uint32_t h[3];
    CK(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    Bins& B = S->b[k];
    void** mem = S->mem[k];
    int r;
    const size_t sz[5] = {(size_t)h[0] * 4, (size_t)h[2] * 16, (size_t)h[1] * 8, (size_t)h[1] * 4, (size_t)h[2] * 8};
    for (int i = 0; i < 5; ++i)
        if ((r = bin_alloc(g, S, k, i, sz[i]))) return r;
    CK(cudaMemsetAsync(cnt, 0, 3 * sizeof(uint32_t), st));
    k_bin_fill<<<grid, 256, 0, st>>>(dev_off, n, t1, t2, cnt, (uint32_t*)mem[0], (uint4*)mem[1], (uint2*)mem[2]);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(mem[3], 0, sz[3] ? sz[3] : 16, st));
    B.med = (const uint32_t*)mem[0];
    B.n_med = h[0];
    B.hchunk = (const uint4*)mem[1];
    B.n_hchunk = h[2];
    B.hvert = (const uint2*)mem[2];
    B.n_hvert = h[1];
    B.hcnt = (uint32_t*)mem[3];
    B.hpart = (float2*)mem[4];
    return IP_OK;
}

// Selects (building if needed) the degree bins for (t1, t2) as g->cur.
int ensure_bins(ip_graph* g, uint32_t t1, uint32_t t2, cudaStream_t st) {
    ++g->use_clock;
    for (BinSet* S : g->binsets)
        if (S->t1 == t1 && S->t2 == t2) {
            S->last_use = g->use_clock;
            g->cur = S;
            return IP_OK;
        }
    if (g->binsets.size() >= 4) {  // evict the least recently used set (and the graphs that bake it in)
        size_t lru = 0;
        for (size_t i = 1; i < g->binsets.size(); ++i)
            if (g->binsets[i]->last_use < g->binsets[lru]->last_use) lru = i;
        free_graph_exec(g);
        if (g->cur == g->binsets[lru]) g->cur = nullptr;
        free_binset(g, g->binsets[lru]);
        g->binsets.erase(g->binsets.begin() + lru);
    }
    BinSet* S = new (std::nothrow) BinSet();
    if (!S) return IP_E_NOMEM;
    S->t1 = t1;
    S->t2 = t2;
    int r = build_bins(g, S, 0, g->csr_off, st);
    if (!r) {
        if (g->csc_alias) {
            // share the CSR bins except the PageRank finish state, which must be private
            S->b[1] = S->b[0];
            r = bin_alloc(g, S, 1, 3, S->b[0].n_hvert * 4 + 16);
            if (!r) r = bin_alloc(g, S, 1, 4, S->b[0].n_hchunk * 8 + 16);
            if (!r) r = cuda_err(cudaMemsetAsync(S->mem[1][3], 0, S->b[0].n_hvert * 4 + 16, st));
            S->b[1].hcnt = (uint32_t*)S->mem[1][3];
            S->b[1].hpart = (float2*)S->mem[1][4];
        } else {
            r = build_bins(g, S, 1, g->csc_off, st);
        }
    }
    if (!r && S->b[0].n_hchunk > g->hq_cap) {  // heavy broadcaster queues hold every heavy CSR chunk once
        free_graph_exec(g);
        for (int p = 0; p < 2; ++p)
            if (g->hq[p]) {
                free_dev(g->hq[p]);
                g->device_bytes -= (size_t)(g->hq_cap + 1) * sizeof(uint2);
                g->hq[p] = nullptr;
            }
        g->hq_cap = S->b[0].n_hchunk;
        for (int p = 0; p < 2 && !r; ++p) r = alloc_dev(g, (void**)&g->hq[p], (size_t)(g->hq_cap + 1) * sizeof(uint2));
    }
    if (r) {
        free_binset(g, S);
        return r;
    }
    S->last_use = g->use_clock;
    g->binsets.push_back(S);
    g->cur = S;
    return IP_OK;
}

// Checks offsets and ids on the device (the ids already checked when ids_checked: the
// upload kernel checked them on the way). The error word is zero on entry (cleared at
// creation and after every check) and holds what the uploads recorded.
static int validate_device(ip_graph* g, const uint32_t* off, const uint32_t* ids, cudaStream_t st,
                           bool ids_checked = false) {
    unsigned int* err = &g->ctl->err;
    k_validate_offsets<<<grid_for(g, g->V), 256, 0, st>>>(off, g->V, g->E, err);
    CK(cudaGetLastError());
    if (!ids_checked) {
        k_validate_ids<<<grid_for(g, g->E), 256, 0, st>>>(ids, g->E, g->V, err);
        CK(cudaGetLastError());
    }
    unsigned int h = 0;
    CK(cudaMemcpyAsync(&h, err, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemsetAsync(err, 0, sizeof(unsigned int), st));
    if (h & 1u) return IP_E_INVAL;
    if (h & 2u) return IP_E_RANGE;
    return IP_OK;
}

// Host-to-device upload by the SMs: the device reads the caller's page-locked host
// array directly (page-locked memory is mapped into the unified address space) with
// 16-byte loads over the host link, writes the device copy and, with limit > 0,
// checks every word against it on the way (vertex ids < n: bit 2 of *err, as
// k_validate_ids). On this system a DMA copy of the same multi-GB array ran between
// 110 and 211 GB/s from one call to the next, this kernel at a steady 211 GB/s.
__global__ void __launch_bounds__(512) k_upload_words(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                                                      uint64_t count, uint32_t limit, unsigned int* err) {
    const uint64_t n16 = count / 4;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, nth = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (uint64_t i = tid; i < n16; i += nth) {
        const uint4 v = s4[i];
        d4[i] = v;
        if (limit) bad |= (v.x >= limit) | (v.y >= limit) | (v.z >= limit) | (v.w >= limit);
    }
    for (uint64_t i = n16 * 4 + tid; i < count; i += nth) {  // the last 0-3 words
        const uint32_t v = src[i];
        dst[i] = v;
        if (limit) bad |= v >= limit;
    }
    if (bad) atomicOr(err, 2u);
}

// The device address of a page-locked host array the device can read at 16-byte
// alignment, or null (pageable memory, device memory, or misaligned).
static const uint32_t* mapped_host(const uint32_t* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    if (reinterpret_cast<uintptr_t>(a.devicePointer) & 15u) return nullptr;
    return static_cast<const uint32_t*>(a.devicePointer);
}

// Allocates alloc_count words for count words of src (host or device memory) and copies
// them; page-locked host arrays go through k_upload_words, which checks ids against
// id_limit (> 0) on the way and then sets *ids_checked.
static int upload(ip_graph* g, uint32_t** dst, const uint32_t* src, size_t count, size_t alloc_count, int device_ptrs,
                  cudaStream_t st, uint32_t id_limit = 0, bool* ids_checked = nullptr) {
    int r = alloc_dev(g, (void**)dst, alloc_count * sizeof(uint32_t));
    if (r) return r;
    if (alloc_count > count) CK(cudaMemsetAsync(*dst + count, 0, (alloc_count - count) * sizeof(uint32_t), st));
    if (!count) return IP_OK;
    const uint32_t* dsrc = device_ptrs ? nullptr : mapped_host(src);
    if (dsrc) {
        const uint64_t work = (count + 3) / 4;
        const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)g->num_sms * 8, (work + 511) / 512));
        k_upload_words<<<grid, 512, 0, st>>>(dsrc, *dst, count, id_limit, &g->ctl->err);
        CK(cudaGetLastError());
        if (ids_checked) *ids_checked = id_limit != 0;
    } else {
        CK(cudaMemcpyAsync(*dst, src, count * sizeof(uint32_t),
                           device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    }
    return IP_OK;
}

// The CSC of g's CSR, transposed on the device (count, scan, scatter; the order of a
// vertex's in-edges is unspecified), in two parts. Its offsets (in-degrees counted
// and scanned) are built with the graph: the degree bins, the blocked layout's bin
// cuts and the maximum in-degree read them. Its rows (and weights) are built by the
// first run that reads them (ensure_in_rows): a pull on the gather engine or a
// batched run. The blocked pull streams its own layout, so a graph that only pulls on
// it never holds the rows.
static int build_in_offsets(ip_graph* g, cudaStream_t st) {
    const uint32_t n = g->V;
    const uint64_t E = g->E;
    int r;
    if ((r = alloc_dev(g, (void**)&g->csc_off, ((size_t)n + 1) * sizeof(uint32_t)))) return r;
    CK(cudaMemsetAsync(g->csc_off, 0, ((size_t)n + 1) * sizeof(uint32_t), st));
    if (E) {
        k_count_in<<<g->num_sms * (2048 / CI_THREADS), CI_THREADS, 0, st>>>(g->csr_col, E, n, g->csc_off);
        CK(cudaGetLastError());
    }
    if ((r = exclusive_scan(g, g->csc_off, (uint64_t)n + 1, st))) return r;
    g->csc_rows_pending = true;
    return IP_OK;
}

// Places every out-edge (u, v) at the next free slot of v's in-edge row. On an
// allocation failure nothing is kept: the rows stay pending.
static int build_in_rows(ip_graph* g, cudaStream_t st) {
    const uint32_t n = g->V;
    const uint64_t E = g->E;
    const size_t ea = edge_alloc_count(E);
    const uint32_t n_chunks = (uint32_t)((E + RL_CH - 1) / RL_CH);
    const size_t tmp_bytes = (size_t)n * sizeof(uint32_t) + std::max<size_t>(n_chunks, 1) * sizeof(uint32_t);
    uint32_t *row = nullptr, *w = nullptr, *cursor = nullptr, *chunk_src = nullptr;
    int r = alloc_dev(g, (void**)&row, ea * sizeof(uint32_t));
    if (!r && g->csr_w) r = alloc_dev(g, (void**)&w, ea * sizeof(uint32_t));
    if (!r) r = alloc_dev(g, (void**)&cursor, (size_t)n * sizeof(uint32_t));
    if (!r) r = alloc_dev(g, (void**)&chunk_src, std::max<size_t>(n_chunks, 1) * sizeof(uint32_t));
    if (r) {
        size_t held = 0;
        if (row) held += ea * sizeof(uint32_t);
        if (w) held += ea * sizeof(uint32_t);
        if (cursor) held += (size_t)n * sizeof(uint32_t);
        free_dev(row);
        free_dev(w);
        free_dev(cursor);
        g->device_bytes -= held;
        return r;
    }
    g->device_bytes -= tmp_bytes;  // the cursor and chunk sources are freed below
    g->csc_row = row;              // the handle's destroy frees them from here on
    g->csc_w = w;
    CK(cudaMemsetAsync(row + E, 0, (ea - E) * sizeof(uint32_t), st));  // the padding after the last edge
    if (w) CK(cudaMemsetAsync(w + E, 0, (ea - E) * sizeof(uint32_t), st));
    CK(cudaMemcpyAsync(cursor, g->csc_off, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    if (E) {
        k_rl_chunk_src<<<grid_for(g, n_chunks), 256, 0, st>>>(g->csr_off, n, n_chunks, chunk_src);
        k_scatter_in<<<grid_for(g, (uint64_t)n_chunks * 32), 256, 0, st>>>(g->csr_off, chunk_src, g->csr_col, g->csr_w,
                                                                           n, E, n_chunks, cursor, row, w);
    }
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(st);
    free_dev(cursor);
    free_dev(chunk_src);
    g->csc_rows_pending = false;
    CK(e1);
    CK(e2);
    return IP_OK;
}

int ensure_in_rows(ip_graph* g, cudaStream_t st) { return g->csc_rows_pending ? build_in_rows(g, st) : IP_OK; }

__global__ void k_max_words(const uint32_t* __restrict__ a, uint64_t n, unsigned int* out) {
    uint32_t m = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, a[i]);
    m = __reduce_max_sync(FULL, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

int graph_max_weight(ip_graph* g, cudaStream_t st) {
    if (!g->weighted || g->max_w_known) return IP_OK;
    unsigned int* mx = nullptr;
    int r = alloc_dev(g, (void**)&mx, sizeof(unsigned int));
    if (r) return r;
    uint32_t h = 0;
    r = cuda_err(cudaMemsetAsync(mx, 0, sizeof(unsigned int), st));
    if (!r && g->E) {
        k_max_words<<<grid_for(g, g->E), 256, 0, st>>>(g->csr_w, g->E, mx);
        r = cuda_err(cudaGetLastError());
    }
    if (!r) r = cuda_err(cudaMemcpyAsync(&h, mx, sizeof(h), cudaMemcpyDeviceToHost, st));
    if (!r) r = cuda_err(cudaStreamSynchronize(st));
    free_dev(mx);
    g->device_bytes -= sizeof(unsigned int);
    if (r) return r;
    g->max_w = h;
    g->max_w_known = true;
    return IP_OK;
}

static int relabel(ip_graph* g, cudaStream_t st, const uint32_t* hcol = nullptr, const uint32_t* hw = nullptr);

static int create(ip_graph* g, uint32_t n, uint64_t E, const uint32_t* csr_off, const uint32_t* csr_col,
                  const uint32_t* csr_w, const uint32_t* csc_off, const uint32_t* csc_row, const uint32_t* csc_w,
                  int flags, cudaStream_t st) {
    const int device_ptrs = (flags & IP_CREATE_DEVICE_PTRS) ? 1 : 0;
    // renumbering as part of creation: the in-edges and degree bins are built once, for
    // the renumbered graph (a CSC given by the caller is still copied and then rebuilt)
    const bool renumber = (flags & IP_CREATE_RELABEL) != 0;
    CK(cudaGetDevice(&g->device));
    CK(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device));
    g->V = n;
    g->E = E;
    g->W = ((n + 31) / 32 + 31) & ~31u;
    g->weighted = csr_w != nullptr;
    int r;
    // control block first: validation uses its error word
    if ((r = alloc_dev(g, (void**)&g->ctl, sizeof(DevCtl)))) return r;
    if ((r = alloc_dev(g, (void**)&g->bin_cnt, 4 * sizeof(uint32_t)))) return r;
    CK(cudaMemsetAsync(g->ctl, 0, sizeof(DevCtl), st));
    CK(cudaMallocHost((void**)&g->ctl_host, sizeof(DevCtl)));

    const bool alias = csc_off != nullptr && csc_off == csr_off && csc_row == csr_col;
    const size_t ea = edge_alloc_count(E);
    // Renumbered from page-locked host arrays (and no separate CSC to copy): the
    // renumbering reads the edges from the host itself (k_rl_host_edges), so they are
    // not first uploaded in the caller's numbering.
    const uint32_t* hcol = nullptr;
    const uint32_t* hw = nullptr;
    if (renumber && !device_ptrs && E && (alias || !csc_off)) {
        hcol = mapped_host(csr_col);
        hw = csr_w ? mapped_host(csr_w) : nullptr;
        if (csr_w && !hw) hcol = nullptr;
    }
    if ((r = upload(g, &g->csr_off, csr_off, (size_t)n + 1, (size_t)n + 1, device_ptrs, st))) return r;
    bool ids_checked = false;
    if (hcol) {
        ids_checked = true;  // by k_rl_host_edges
    } else {
        if ((r = upload(g, &g->csr_col, csr_col, E, ea, device_ptrs, st, n, &ids_checked))) return r;
        if (csr_w && (r = upload(g, &g->csr_w, csr_w, E, ea, device_ptrs, st))) return r;
    }
    // validated on the device whether the caller's arrays were host or device memory
    if ((r = validate_device(g, g->csr_off, g->csr_col, st, ids_checked))) return r;
    if (alias) {
        g->csc_alias = true;
        g->csc_off = g->csr_off;
        g->csc_row = g->csr_col;
        g->csc_w = g->csr_w;
    } else if (csc_off) {
        if ((r = upload(g, &g->csc_off, csc_off, (size_t)n + 1, (size_t)n + 1, device_ptrs, st))) return r;
        ids_checked = false;
        if ((r = upload(g, &g->csc_row, csc_row, E, ea, device_ptrs, st, n, &ids_checked))) return r;
        if (csc_w && (r = upload(g, &g->csc_w, csc_w, E, ea, device_ptrs, st))) return r;
        if ((r = validate_device(g, g->csc_off, g->csc_row, st, ids_checked))) return r;
    } else if (!renumber && (r = build_in_offsets(g, st))) {
        return r;
    }
    if (csr_w && csc_off && !alias && !g->csc_w) return IP_E_INVAL;

    // per-vertex arrays
    const size_t nv = (size_t)n;
    if ((r = alloc_dev(g, (void**)&g->inv_outdeg, nv * 4))) return r;
    if ((r = alloc_dev(g, (void**)&g->value, nv * 4))) return r;
    if ((r = alloc_dev(g, (void**)&g->rank, nv * 4))) return r;
    if ((r = alloc_dev(g, (void**)&g->contrib[0], nv * 4))) return r;
    if ((r = alloc_dev(g, (void**)&g->contrib[1], nv * 4))) return r;
    if ((r = alloc_dev(g, (void**)&g->mbox, nv * 4))) return r;
    if ((r = alloc_dev(g, (void**)&g->outbox, nv * 4))) return r;
    if ((r = alloc_dev(g, (void**)&g->mboxf, nv * 4))) return r;
    if ((r = alloc_dev(g, (void**)&g->recv, (size_t)g->W * 4))) return r;
    if ((r = alloc_dev(g, (void**)&g->rq, nv * 4))) return r;
    for (int k = 0; k < 2; ++k) {
        if ((r = alloc_dev(g, (void**)&g->bcast[k], (size_t)g->W * 4))) return r;
        CK(cudaMemsetAsync(g->bcast[k], 0, (size_t)g->W * 4, st));
        for (int b = 0; b < 2; ++b)
            if ((r = alloc_dev(g, (void**)&g->q[k][b], nv * 4))) return r;
    }
    if ((r = alloc_dev(g, (void**)&g->sel, sizeof(SelectorDev)))) return r;
    CK(cudaMemsetAsync(g->recv, 0, (size_t)g->W * 4, st));

    unsigned int* mx = &g->ctl->err;
    CK(cudaMemsetAsync(mx, 0, 4, st));
    k_degrees<<<grid_for(g, n), 256, 0, st>>>(g->csr_off, n, g->inv_outdeg, mx);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&g->max_out_deg, mx, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemsetAsync(mx, 0, 4, st));
    if ((r = alloc_dev(g, (void**)&g->hq[0], sizeof(uint2)))) return r;
    if ((r = alloc_dev(g, (void**)&g->hq[1], sizeof(uint2)))) return r;
    g->hq_cap = 0;
    CK(cudaEventCreate(&g->ev0));
    CK(cudaEventCreate(&g->ev1));
    if (renumber) {
        if ((r = relabel(g, st, hcol, hw))) return r;  // transposes (directed) and builds the bins
    } else {
        if ((r = ensure_bins(g, DEFAULT_T1, DEFAULT_T2, st))) return r;
    }
    k_degrees<<<grid_for(g, n), 256, 0, st>>>(g->csc_off, n, nullptr, mx);  // max in-degree
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&g->max_in_deg, mx, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemsetAsync(mx, 0, 4, st));
    CK(cudaStreamSynchronize(st));
    return IP_OK;
}

// ------------------------------------------------------------ vertex renumbering
// Vertices are renumbered by decreasing out-degree class (class = leading zeros of
// the degree, degree 0 last), keeping the original order inside a class (a stable
// counting sort): the sources of the high-degree vertices then share cache lines,
// so the gathers of the pull exchanges hit L1/L2 more often. The caller's numbering
// stays the interface: values, sources and instance offsets are mapped at the edge.
constexpr uint32_t RL_KEYS = 33;
__device__ __forceinline__ uint32_t rl_key(uint32_t d) { return d ? (uint32_t)__clz(d) : 32u; }

// Per block of consecutive vertices [b*R, (b+1)*R): counts per key.
__global__ void k_rl_hist(const uint32_t* __restrict__ off, uint32_t n, uint32_t R, uint32_t* hist) {
    __shared__ uint32_t h[RL_KEYS];
    for (uint32_t i = threadIdx.x; i < RL_KEYS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint64_t v0 = (uint64_t)blockIdx.x * R, v1 = v0 + R < n ? v0 + R : n;
    for (uint64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) atomicAdd(h + rl_key(off[v + 1] - off[v]), 1u);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < RL_KEYS; i += blockDim.x) hist[(size_t)blockIdx.x * RL_KEYS + i] = h[i];
}

// One warp per block of vertices, in order: new number = the key's first place
// for this block (pos) + the rank among the block's earlier vertices of that key.
__global__ void k_rl_place(const uint32_t* __restrict__ off, uint32_t n, uint32_t R, const uint32_t* __restrict__ pos,
                           uint32_t* new_of_old, uint32_t* old_of_new, uint32_t* deg_new, uint32_t* start_old) {
    __shared__ uint32_t cur[RL_KEYS];
    const uint32_t lane = threadIdx.x;
    for (uint32_t i = lane; i < RL_KEYS; i += 32) cur[i] = pos[(size_t)blockIdx.x * RL_KEYS + i];
    __syncwarp();
    const uint64_t v0 = (uint64_t)blockIdx.x * R, v1 = v0 + R < n ? v0 + R : n;
    for (uint64_t b = v0; b < v1; b += 32) {  // the same trip count for the 32 lanes
        const uint64_t v = b + lane;
        const bool ok = v < v1;
        const uint32_t d = ok ? off[v + 1] - off[v] : 0u;
        const uint32_t key = ok ? rl_key(d) : RL_KEYS;
        const uint32_t same = __match_any_sync(0xFFFFFFFFu, key);
        const uint32_t leader = __ffs(same) - 1;
        uint32_t base = 0;
        if (lane == leader && ok) base = cur[key];
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (ok) {
            const uint32_t p = base + __popc(same & ((1u << lane) - 1u));
            new_of_old[v] = p;
            old_of_new[p] = (uint32_t)v;
            deg_new[p] = d;
            start_old[p] = off[v];
        }
        __syncwarp();
        if (lane == leader && ok) cur[key] += __popc(same);
        __syncwarp();
    }
}

// The renumbered CSR, cut into chunks of RL_CH consecutive NEW edge positions, one
// warp per chunk: the chunk's first source comes from k_rl_chunk_src, the warp holds
// the first new and old edge positions of 32 consecutive sources in registers, and
// each lane finds the source of its edge by a binary search over them (shuffles).
// Writes are coalesced whatever the degrees; the targets are renumbered on the way.
__global__ void k_rl_edges(const uint32_t* __restrict__ off_new, const uint32_t* __restrict__ start_old,
                           const uint32_t* __restrict__ chunk_src, const uint32_t* __restrict__ col,
                           const uint32_t* __restrict__ w, const uint32_t* __restrict__ new_of_old, uint32_t n,
                           uint64_t E, uint32_t n_chunks, uint32_t* __restrict__ col_new, uint32_t* __restrict__ w_new) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += nw) {
        const uint64_t p0 = (uint64_t)c * RL_CH;
        const uint64_t p1 = p0 + RL_CH < E ? p0 + RL_CH : E;
        for (uint64_t s = chunk_src[c];; s += 32) {  // windows of 32 sources
            const uint64_t sl = s + lane;
            const uint32_t wo = sl < n ? off_new[sl] : (uint32_t)E;  // the lane's source: first new position
            const uint32_t ws = sl < n ? start_old[sl] : 0u;         // and first old position
            const uint64_t wend = s + 32 <= n ? (uint64_t)off_new[s + 32] : E;
            const uint64_t w0 = __shfl_sync(FULL, wo, 0);
            const uint64_t lo = p0 > w0 ? p0 : w0, hi = p1 < wend ? p1 : wend;
            for (uint64_t base = lo; base < hi; base += 32 * RL_UNROLL) {
                uint32_t q[RL_UNROLL], pos[RL_UNROLL], cv[RL_UNROLL], wv[RL_UNROLL];
#pragma unroll
                for (uint32_t u = 0; u < RL_UNROLL; ++u) {
                    const uint64_t qq = base + 32 * u + lane;
                    q[u] = qq < hi ? (uint32_t)qq : 0xFFFFFFFFu;
                    uint32_t i = 0;  // largest i with wo(i) <= q
#pragma unroll
                    for (uint32_t step = 16; step; step >>= 1)
                        if (__shfl_sync(FULL, wo, i + step) <= q[u]) i += step;
                    pos[u] = __shfl_sync(FULL, ws, i) + (q[u] - __shfl_sync(FULL, wo, i));
                }
#pragma unroll
                for (uint32_t u = 0; u < RL_UNROLL; ++u) {
                    cv[u] = q[u] != 0xFFFFFFFFu ? col[pos[u]] : 0u;
                    wv[u] = (w && q[u] != 0xFFFFFFFFu) ? w[pos[u]] : 0u;
                }
#pragma unroll
                for (uint32_t u = 0; u < RL_UNROLL; ++u)
                    if (q[u] != 0xFFFFFFFFu) {
                        col_new[q[u]] = new_of_old[cv[u]];
                        if (w) w_new[q[u]] = wv[u];
                    }
            }
            if (wend >= p1) break;
        }
    }
}

// The renumbered CSR read straight from the caller's page-locked host arrays (mapped
// into the device's address space), for creation with renumbering: the edges cross
// the host link once and are never stored in the caller's numbering. Warps take
// chunks of RL_CH old edge positions and read them in order (coalesced), check every
// id (< n; otherwise bit 2 of *err, as k_validate_ids, and the edge is written as 0)
// and write each edge at its new position with its new id. A warp keeps the first old
// and new positions of 32 consecutive old sources in registers and finds each lane's
// source by a 5-step shuffle search. With cnt (a directed graph), the in-degrees of
// the new ids are counted on the way, as k_count_in does (the first CI_HOT vertices'
// counters in dynamic shared memory, CI_HOT words), while the link is the bound.
__global__ void __launch_bounds__(256) k_rl_host_edges(const uint32_t* __restrict__ off_old,
                                                       const uint32_t* __restrict__ off_new,
                                                       const uint32_t* __restrict__ new_of_old,
                                                       const uint32_t* __restrict__ chunk_src,
                                                       const uint32_t* __restrict__ hcol,
                                                       const uint32_t* __restrict__ hw, uint32_t n, uint64_t E,
                                                       uint32_t n_chunks, uint32_t* __restrict__ col_new,
                                                       uint32_t* __restrict__ w_new, uint32_t* cnt,
                                                       unsigned int* err) {
    extern __shared__ uint32_t hot[];
    const uint32_t H = cnt ? min(n, CI_HOT) : 0u;
    for (uint32_t i = threadIdx.x; i < H; i += blockDim.x) hot[i] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    bool bad = false;
    for (uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += nw) {
        const uint64_t p0 = (uint64_t)c * RL_CH;
        const uint64_t p1 = p0 + RL_CH < E ? p0 + RL_CH : E;
        for (uint64_t s = chunk_src[c];; s += 32) {  // windows of 32 old sources
            const uint64_t sl = s + lane;
            const uint32_t wo = sl < n ? off_old[sl] : (uint32_t)E;          // the lane's source: first old position
            const uint32_t wn = sl < n ? off_new[new_of_old[sl]] : 0u;       // and first new position
            const uint64_t wend = s + 32 <= n ? (uint64_t)off_old[s + 32] : E;
            const uint64_t w0 = __shfl_sync(FULL, wo, 0);
            const uint64_t lo = p0 > w0 ? p0 : w0, hi = p1 < wend ? p1 : wend;
            for (uint64_t base = lo; base < hi; base += 32 * RL_UNROLL) {
                uint32_t q[RL_UNROLL], pos[RL_UNROLL], cv[RL_UNROLL], wv[RL_UNROLL];
#pragma unroll
                for (uint32_t u = 0; u < RL_UNROLL; ++u) {
                    const uint64_t qq = base + 32 * u + lane;
                    q[u] = qq < hi ? (uint32_t)qq : 0xFFFFFFFFu;
                    uint32_t i = 0;  // largest i with wo(i) <= q
#pragma unroll
                    for (uint32_t step = 16; step; step >>= 1)
                        if (__shfl_sync(FULL, wo, i + step) <= q[u]) i += step;
                    pos[u] = __shfl_sync(FULL, wn, i) + (q[u] - __shfl_sync(FULL, wo, i));
                }
#pragma unroll
                for (uint32_t u = 0; u < RL_UNROLL; ++u) {
                    cv[u] = q[u] != 0xFFFFFFFFu ? hcol[q[u]] : 0u;
                    wv[u] = (hw && q[u] != 0xFFFFFFFFu) ? hw[q[u]] : 0u;
                }
#pragma unroll
                for (uint32_t u = 0; u < RL_UNROLL; ++u)
                    if (q[u] != 0xFFFFFFFFu) {
                        const bool ok = cv[u] < n;
                        bad |= !ok;
                        const uint32_t v = ok ? new_of_old[cv[u]] : 0u;
                        col_new[pos[u]] = v;
                        if (hw) w_new[pos[u]] = wv[u];
                        if (cnt && ok) {
                            if (v < H)
                                atomicAdd(hot + v, 1u);
                            else
                                atomicAdd(cnt + v, 1u);
                        }
                    }
            }
            if (wend >= p1) break;
        }
    }
    if (bad) atomicOr(err, 2u);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < H; i += blockDim.x)
        if (hot[i]) atomicAdd(cnt + i, hot[i]);
}

// out[old] = in[new_of_old[old]] (a per-vertex array back to the caller's numbering).
__global__ void k_rl_unpermute(const uint32_t* __restrict__ in, const uint32_t* __restrict__ new_of_old, uint32_t n,
                               uint32_t* out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        out[v] = in[new_of_old[v]];
}

int unpermute(const ip_graph* g, const uint32_t* in, uint32_t* out, cudaStream_t st) {
    k_rl_unpermute<<<grid_for(g, g->V), 256, 0, st>>>(in, g->new_of_old, g->V, out);
    return cuda_err(cudaGetLastError());
}

// hcol / hw: the caller's page-locked CSR columns and weights (device-visible
// addresses) when creation reads them here instead of uploading them first.
static int relabel(ip_graph* g, cudaStream_t st, const uint32_t* hcol, const uint32_t* hw) {
    if (g->new_of_old) return IP_OK;
    const uint32_t n = g->V;
    const uint64_t E = g->E;
    const size_t ea = edge_alloc_count(E);
    int r;
    const uint32_t nblk =
        (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)g->num_sms * 16, ((uint64_t)n + 255) / 256));
    const uint32_t R = (uint32_t)(((uint64_t)n + nblk - 1) / nblk);
    const uint32_t n_chunks = (uint32_t)((E + RL_CH - 1) / RL_CH);
    uint32_t *hist = nullptr, *pos = nullptr, *off_new = nullptr, *col_new = nullptr, *w_new = nullptr;
    uint32_t *start_old = nullptr, *chunk_src = nullptr;
    if ((r = alloc_dev(g, (void**)&g->new_of_old, (size_t)n * 4))) return r;
    if ((r = alloc_dev(g, (void**)&g->old_of_new, (size_t)n * 4))) return r;
    if ((r = alloc_dev(g, (void**)&hist, (size_t)nblk * RL_KEYS * 4))) return r;
    if ((r = alloc_dev(g, (void**)&pos, (size_t)nblk * RL_KEYS * 4))) return r;
    if ((r = alloc_dev(g, (void**)&off_new, ((size_t)n + 1) * 4))) return r;
    if ((r = alloc_dev(g, (void**)&start_old, (size_t)n * 4))) return r;
    if ((r = alloc_dev(g, (void**)&chunk_src, (size_t)n_chunks * 4))) return r;
    if ((r = alloc_dev(g, (void**)&col_new, ea * 4))) return r;
    CK(cudaMemsetAsync(col_new + E, 0, (ea - E) * 4, st));  // the padding after the last edge
    if (g->csr_w || hw) {
        if ((r = alloc_dev(g, (void**)&w_new, ea * 4))) return r;
        CK(cudaMemsetAsync(w_new + E, 0, (ea - E) * 4, st));
    }
    // stable counting sort of the vertices by key
    k_rl_hist<<<nblk, 256, 0, st>>>(g->csr_off, n, R, hist);
    CK(cudaGetLastError());
    std::vector<uint32_t> h((size_t)nblk * RL_KEYS), p((size_t)nblk * RL_KEYS);
    CK(cudaMemcpyAsync(h.data(), hist, h.size() * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    uint64_t acc = 0;
    for (uint32_t k = 0; k < RL_KEYS; ++k)
        for (uint32_t b = 0; b < nblk; ++b) {
            p[(size_t)b * RL_KEYS + k] = (uint32_t)acc;
            acc += h[(size_t)b * RL_KEYS + k];
        }
    CK(cudaMemcpyAsync(pos, p.data(), p.size() * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(off_new + n, 0, 4, st));
    k_rl_place<<<nblk, 32, 0, st>>>(g->csr_off, n, R, pos, g->new_of_old, g->old_of_new, off_new, start_old);
    CK(cudaGetLastError());
    if ((r = exclusive_scan(g, off_new, (uint64_t)n + 1, st))) return r;  // out-degrees -> offsets
    uint32_t* in_cnt = nullptr;  // in-degrees counted by the host read (directed graphs)
    if (E && hcol) {  // chunks of old positions, read from the host arrays
        if (!g->csc_alias) {
            if ((r = alloc_dev(g, (void**)&in_cnt, ((size_t)n + 1) * 4))) return r;
            CK(cudaMemsetAsync(in_cnt, 0, ((size_t)n + 1) * 4, st));
        }
        k_rl_chunk_src<<<grid_for(g, n_chunks), 256, 0, st>>>(g->csr_off, n, n_chunks, chunk_src);
        CK(cudaGetLastError());
        k_rl_host_edges<<<g->num_sms * 6, 256, in_cnt ? CI_HOT * 4 : 0, st>>>(
            g->csr_off, off_new, g->new_of_old, chunk_src, hcol, hw, n, E, n_chunks, col_new, w_new, in_cnt,
            &g->ctl->err);
        CK(cudaGetLastError());
    } else if (E) {
        k_rl_chunk_src<<<grid_for(g, n_chunks), 256, 0, st>>>(off_new, n, n_chunks, chunk_src);
        CK(cudaGetLastError());
        k_rl_edges<<<grid_for(g, (uint64_t)n_chunks * 32), 256, 0, st>>>(
            off_new, start_old, chunk_src, g->csr_col, g->csr_w, g->new_of_old, n, E, n_chunks, col_new, w_new);
        CK(cudaGetLastError());
    }
    // Every buffer of the old numbering goes back to the device cache (the rebuilt
    // degree bins have the same sizes and take theirs back): the device is idle first.
    CK(cudaDeviceSynchronize());
    if (hcol) {  // the ids read from the host were checked on the way
        unsigned int h = 0;
        CK(cudaMemcpy(&h, &g->ctl->err, sizeof(h), cudaMemcpyDeviceToHost));
        if (h & 2u) {
            DeviceIdleScope idle;
            for (uint32_t* p : {hist, pos, off_new, start_old, chunk_src, col_new, w_new, in_cnt}) free_dev(p);
            g->device_bytes -= (size_t)nblk * RL_KEYS * 8 + ((size_t)n + 1) * 4 + (size_t)n * 4 +
                               (size_t)n_chunks * 4 + ea * 4 * (w_new ? 2 : 1) + (in_cnt ? ((size_t)n + 1) * 4 : 0);
            return IP_E_RANGE;
        }
    }
    const bool alias = g->csc_alias;
    {
        DeviceIdleScope idle;
        free_dev(hist);
        free_dev(pos);
        free_dev(start_old);
        free_dev(chunk_src);
        g->device_bytes -= (size_t)nblk * RL_KEYS * 8 + (size_t)n * 4 + (size_t)n_chunks * 4;
        if (!alias && g->csc_off) {  // (creation with renumbering has not built it yet)
            free_dev(g->csc_off);
            g->device_bytes -= ((size_t)n + 1) * 4;
        }
        if (!alias && g->csc_row) {  // (nor, before a run needs them, the rows)
            free_dev(g->csc_row);
            free_dev(g->csc_w);
            g->device_bytes -= ea * 4 * (g->csc_w ? 2 : 1);
        }
        free_dev(g->csr_off);
        free_dev(g->csr_col);
        free_dev(g->csr_w);
        g->device_bytes -= ((size_t)n + 1) * 4 + (g->csr_col ? ea * 4 : 0) + (g->csr_w ? ea * 4 : 0);
        free_graph_exec(g);
        free_batch_state(g);
        pb_free(g);
        for (BinSet* S : g->binsets) free_binset(g, S);
        g->binsets.clear();
        g->cur = nullptr;
        g->last_app = -1;
    }
    // the renumbered CSR; the CSC is the CSR again (symmetric) or transposed anew
    g->csr_off = off_new;
    g->csr_col = col_new;
    g->csr_w = w_new;
    g->csc_off = g->csc_row = g->csc_w = nullptr;
    g->csc_rows_pending = false;
    if (alias) {
        g->csc_off = g->csr_off;
        g->csc_row = g->csr_col;
        g->csc_w = g->csr_w;
    } else if (in_cnt) {  // counted during the host read: the offsets are their scan
        g->csc_off = in_cnt;
        if ((r = exclusive_scan(g, g->csc_off, (uint64_t)n + 1, st))) return r;
        g->csc_rows_pending = true;
    } else if ((r = build_in_offsets(g, st))) {
        return r;
    }
    k_degrees<<<grid_for(g, n), 256, 0, st>>>(g->csr_off, n, g->inv_outdeg, &g->ctl->err);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(&g->ctl->err, 0, 4, st));
    if ((r = ensure_bins(g, DEFAULT_T1, DEFAULT_T2, st))) return r;
    CK(cudaStreamSynchronize(st));
    return IP_OK;
}

}  // namespace ipg

using namespace ipg;

extern "C" {

void ip_options_default(ip_options_t* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->damping = 0.85f;
    o->pr_iterations = 30;
    o->source = 0;
    o->policy = IP_POLICY_AUTO;
    o->forced_mode = IP_MODE_PULL;
    o->t1 = 0;
    o->t2 = 0;
    o->thr_sparse = 0.00794f;  // cutoffs fitted on measured per-mode superstep times (selector_report.json)
    o->thr_pull = 0.1122f;
    o->use_graph = 1;
    o->collect_labels = 0;
    o->stream = nullptr;
    o->pr_engine = IP_PR_ENGINE_AUTO;
    o->pr_tolerance = 0.0f;
    o->pull_early_exit = 1;
}

void ip_graph_destroy(ip_graph_t* g) {
    if (!g) return;
    int cur = -1;
    (void)cudaGetDevice(&cur);
    (void)cudaSetDevice(g->device);
    (void)cudaDeviceSynchronize();  // no kernel uses the buffers below any more: they can be cached
    DeviceIdleScope idle;
    free_graph_exec(g);
    free_batch_state(g);
    pb_free(g);
    void* bufs[] = {g->ctl,        g->csr_off,    g->csr_col, g->csr_w,      g->inv_outdeg, g->value,
                    g->rank,       g->contrib[0], g->contrib[1], g->mbox,  g->mboxf,      g->recv, g->outbox,
                    g->bcast[0],   g->bcast[1],   g->rq,      g->log,        g->sel,        g->snap_value,
                    g->q[0][0],    g->q[0][1],    g->q[1][0], g->q[1][1],    g->hq[0],      g->hq[1],
                    g->bin_cnt,    g->new_of_old, g->old_of_new};
    for (void* p : bufs) dcache_release(p);
    for (BinSet* S : g->binsets) free_binset(g, S);
    g->binsets.clear();
    if (!g->csc_alias) {
        dcache_release(g->csc_off);
        dcache_release(g->csc_row);
        dcache_release(g->csc_w);
    }
    if (g->ctl_host) cudaFreeHost(g->ctl_host);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    delete g;
    if (cur >= 0) (void)cudaSetDevice(cur);
}

int ip_graph_relabel(ip_graph_t* g, void* stream) {
    if (!g) return IP_E_INVAL;
    return relabel(g, (cudaStream_t)stream);
}

int ip_release_cached_memory(void) {
    DeviceCache& C = dcache();
    std::lock_guard<std::mutex> l(C.m);
    dcache_trim_locked(C, -1);
    return IP_OK;
}

int ip_graph_create(ip_graph_t** out, uint32_t n_vertices, uint64_t n_edges, const uint32_t* csr_offsets,
                    const uint32_t* csr_cols, const uint32_t* csr_weights, const uint32_t* csc_offsets,
                    const uint32_t* csc_rows, const uint32_t* csc_weights, int flags, void* stream) {
    if (!out) return IP_E_INVAL;
    *out = nullptr;
    if (flags & ~(IP_CREATE_DEVICE_PTRS | IP_CREATE_RELABEL)) return IP_E_INVAL;
    if (n_vertices == 0 || n_vertices == 0xFFFFFFFFu || !csr_offsets) return IP_E_INVAL;
    if (n_edges >= 0xFFFFFFFFull) return IP_E_RANGE;
    if (n_edges > 0 && !csr_cols) return IP_E_INVAL;
    if ((csc_offsets == nullptr) != (csc_rows == nullptr) && n_edges > 0) return IP_E_INVAL;
    const bool alias = csc_offsets && csc_offsets == csr_offsets && csc_rows == csr_cols;
    if (alias && csc_weights && csc_weights != csr_weights) return IP_E_INVAL;
    if (csc_offsets && !alias && csr_weights && !csc_weights) return IP_E_INVAL;
    ip_graph* g = new (std::nothrow) ip_graph();
    if (!g) return IP_E_NOMEM;
    int r = create(g, n_vertices, n_edges, csr_offsets, csr_cols, csr_weights, csc_offsets, csc_rows,
                   csr_weights ? csc_weights : nullptr, flags, (cudaStream_t)stream);
    if (r != IP_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        (void)cudaGetLastError();
        ip_graph_destroy(g);
        return r;
    }
    *out = g;
    return IP_OK;
}

int ip_graph_info(const ip_graph_t* g, ip_graph_info_t* info) {
    if (!g || !info) return IP_E_INVAL;
    info->n_vertices = g->V;
    info->n_edges = g->E;
    info->max_out_degree = g->max_out_deg;
    info->max_in_degree = g->max_in_deg;
    info->csc_is_csr = g->csc_alias ? 1u : 0u;
    info->weighted = g->weighted ? 1u : 0u;
    info->num_sms = (uint32_t)g->num_sms;
    info->device_bytes = g->device_bytes;
    // the parts, from the sizes create(), ensure_bins(), ip_graph_relabel() and pb.cu allocate
    const uint64_t nv = g->V, ea = edge_alloc_count(g->E);
    const uint64_t off_b = (nv + 1) * 4, rows_b = ea * 4 * (g->weighted ? 2 : 1);
    uint64_t gb = g->csr_off ? off_b + rows_b : 0;
    if (!g->csc_alias) gb += (g->csc_off ? off_b : 0) + (g->csc_row ? rows_b : 0);  // rows: once a run built them
    info->bytes_graph = gb;
    uint64_t vs = 13 * nv * 4 + 3 * (uint64_t)g->W * 4;  // 13 vertex arrays, recv + 2 broadcast bitmaps
    vs += 2 * (uint64_t)(g->hq_cap + 1) * sizeof(uint2);
    if (g->snap_value) vs += nv * 8;
    info->bytes_vertex_state = g->value ? vs : 0;
    uint64_t bins = 0;
    for (const BinSet* S : g->binsets)
        for (int k = 0; k < 2; ++k)
            for (int i = 0; i < 5; ++i) bins += S->bytes[k][i];
    info->bytes_degree_bins = bins;
    info->bytes_blocked_layout = pb_bytes(g);
    info->bytes_renumbering = g->new_of_old ? 2 * nv * 4 : 0;
    const uint64_t known = info->bytes_graph + info->bytes_vertex_state + info->bytes_degree_bins +
                           info->bytes_blocked_layout + info->bytes_renumbering;
    info->bytes_other = g->device_bytes > known ? g->device_bytes - known : 0;
    return IP_OK;
}

int ip_get_values(ip_graph_t* g, void* dst, size_t dst_bytes, int dst_is_device, void* stream) {
    if (!g || !dst) return IP_E_INVAL;
    if (g->last_app < 0) return IP_E_STATE;
    const size_t need = (size_t)g->V * 4;
    if (dst_bytes < need) return IP_E_RANGE;
    const void* src = g->last_app == IP_PAGERANK ? (const void*)g->rank : (const void*)g->value;
    cudaStream_t st = (cudaStream_t)stream;
    if (g->new_of_old) {  // back to the caller's numbering
        if (!g->snap_value) {
            int r = alloc_dev(g, (void**)&g->snap_value, (size_t)g->V * 8);
            if (r) return r;
        }
        int r = unpermute(g, (const uint32_t*)src, g->snap_value, st);
        if (r) return r;
        src = g->snap_value;
    }
    CK(cudaMemcpyAsync(dst, src, need, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return IP_OK;
}

int ip_set_selector(ip_graph_t* g, const void* blob, size_t bytes) {
    if (!g || !blob) return IP_E_INVAL;
    if (bytes != IP_SELECTOR_BYTES) return IP_E_RANGE;
    CK(cudaMemcpy(g->sel, blob, bytes, cudaMemcpyHostToDevice));
    g->has_selector = true;
    free_graph_exec(g);
    return IP_OK;
}

int ip_run(ip_graph_t* g, ip_app_t app, uint32_t max_supersteps, const ip_options_t* opt, ip_run_stats_t* stats) {
    if (!g) return IP_E_INVAL;
    if (app != IP_PAGERANK && !ipg::program_ops((int)app)) return IP_E_INVAL;  // a registered vertex program
    if (max_supersteps == 0) return IP_E_INVAL;
    return run_app(g, (int)app, max_supersteps, opt, stats);
}

const char* ip_strerror(int code) {
    switch (code) {
        case IP_OK: return "ok";
        case IP_E_INVAL: return "invalid argument or malformed graph";
        case IP_E_RANGE: return "value out of range";
        case IP_E_NOMEM: return "device allocation failed";
        case IP_E_CUDA: return "CUDA runtime error";
        case IP_E_TIMEOUT: return "bounded device wait timed out";
        case IP_E_MAXSTEPS: return "superstep cap reached before global halt";
        case IP_E_DEVICE_ASSERT: return "device-side check failed";
        case IP_E_STATE: return "call not valid in the current state";
        default: return "unknown error code";
    }
}

}  // extern "C"
