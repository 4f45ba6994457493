// Hashmin connected components for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool and may not grow it, or code with a fixed memory
// budget set up once at start. This entry point runs Hashmin (the same
// superstep semantics as ip_run with IP_HASHMIN) with all of its temporary
// state in one fixed-size array that is part of the library image, so it
// allocates nothing on the device. The caller passes the graph and the output
// buffer in device memory.
//
// The scratch array below is a host-side stand-in when named from host code,
// not a device address. Host code looks up its device address once per device
// with cudaGetSymbolAddress (on the first call on that device, with that device
// current) and passes the pointer to the kernels.
//
// Limits and sharing: at most NA_MAX_V vertices. Every call on a device uses the
// same array and leaves its contents behind; each call clears what it needs
// before use. Calls whose work overlaps on the GPU (two streams, two threads)
// race on the array and give wrong results.
//
// The input is checked on the device before and while it is used: offsets that
// do not start at 0, decrease, or do not end at n_edges stop the call before any
// edge is read (IP_E_INVAL); an edge whose destination is not below n_vertices is
// skipped and recorded (IP_E_RANGE). No access ever leaves the caller's arrays or
// the scratch array.
#include <mutex>

#include "internal.h"

namespace {

constexpr uint32_t NA_MAX_V = IP_NOALLOC_MAX_VERTICES;
constexpr uint32_t NA_MAX_W = (NA_MAX_V + 31) / 32;
constexpr uint32_t NA_INF = 0xFFFFFFFFu;
constexpr int NA_BLOCK = 256;

// Layout of the scratch array (32-bit words):
//   [0, MAX_V)                      mailbox, one combined message per vertex
//   [MAX_V, MAX_V + W)              recipient bitmap of the superstep being computed
//   [.. + W, .. + 2W)               broadcast bitmap, even supersteps
//   [.. + 2W, .. + 3W)              broadcast bitmap, odd supersteps
//   [.. + 3W, .. + 3W + 4)          counters: messages sent (64-bit), input error bits, spare
constexpr size_t NA_WORDS = (size_t)NA_MAX_V + 3 * (size_t)NA_MAX_W + 4;
static __device__ __align__(256) uint32_t na_scratch[NA_WORDS];

constexpr uint32_t NA_ERR_OFFSETS = 1u;  // offsets[0] != 0, a decreasing offset, or offsets[n] != n_edges
constexpr uint32_t NA_ERR_IDS = 2u;      // an edge destination >= n_vertices

struct NaPtrs {
    uint32_t* mbox;
    uint32_t* recv;
    uint32_t* bc[2];
    unsigned long long* msgs;
    uint32_t* err;  // right after msgs: one 16-byte read returns both
};

NaPtrs na_layout(uint32_t* base) {
    NaPtrs p;
    p.mbox = base;
    p.recv = base + NA_MAX_V;
    p.bc[0] = p.recv + NA_MAX_W;
    p.bc[1] = p.bc[0] + NA_MAX_W;
    p.msgs = reinterpret_cast<unsigned long long*>(p.bc[1] + NA_MAX_W);
    p.err = p.bc[1] + NA_MAX_W + 2;
    return p;
}

// Offsets check (the err word was zeroed by the host just before): every offset
// pair non-decreasing, the first 0 and the last n_edges, so every later edge
// index lies in [0, n_edges).
__global__ void na_validate(uint32_t n, const uint32_t* off, unsigned long long E, NaPtrs p) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    bool bad = false;
    for (uint32_t v = tid; v < n; v += nth) bad |= off[v + 1] < off[v];
    if (tid == 0) bad |= off[0] != 0u || (unsigned long long)off[n] != E;
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31u) == 0) atomicOr(p.err, NA_ERR_OFFSETS);
}

// Superstep 0 (Fig. 9): label = id, every vertex broadcasts. Clears the
// mailboxes, the recipient bitmap and the counter left by an earlier call.
__global__ void na_init(uint32_t n, uint32_t* label, NaPtrs p, unsigned long long E) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const uint32_t W = (n + 31) / 32;
    for (uint32_t v = tid; v < n; v += nth) {
        label[v] = v;
        p.mbox[v] = NA_INF;
    }
    for (uint32_t w = tid; w < W; w += nth) {
        p.recv[w] = 0;
        const uint64_t lo = (uint64_t)w * 32;
        p.bc[0][w] = lo + 32 <= n ? 0xFFFFFFFFu : ((1u << (n - lo)) - 1u);
    }
    if (tid == 0) *p.msgs = E;
}

// Exchange into superstep s: every broadcaster of s-1 pushes its label along
// its out-edges (min combiner); the bitmap of s is cleared for the apply.
// A warp takes 32 consecutive vertices: a broadcaster with at most NA_LANE_DEG
// out-edges is pushed by its own lane, a larger one by the whole warp (one
// vertex at a time, lanes on consecutive edges), so a hub does not hold up the
// other lanes of its warp. Destinations >= n are skipped and recorded.
constexpr uint32_t NA_LANE_DEG = 8;
__device__ __forceinline__ void na_deliver(uint32_t n, uint32_t v, uint32_t m, const NaPtrs& p, bool& bad) {
    if (v >= n) {
        bad = true;
        return;
    }
    atomicMin(p.mbox + v, m);
    atomicOr(p.recv + (v >> 5), 1u << (v & 31u));
}

__global__ void na_push(uint32_t n, const uint32_t* off, const uint32_t* col, const uint32_t* label, NaPtrs p,
                        uint32_t s) {
    if (*(volatile uint32_t*)p.err) return;  // the host stops before this; kept as a guard
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const uint32_t W = (n + 31) / 32;
    const uint32_t* prev = (s & 1) ? p.bc[0] : p.bc[1];
    uint32_t* next = (s & 1) ? p.bc[1] : p.bc[0];
    for (uint32_t w = tid; w < W; w += nth) next[w] = 0;
    if (tid == 0) *p.msgs = 0;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = nth >> 5;
    bool bad = false;
    for (uint32_t w = tid >> 5; w < W; w += warps) {  // warp-uniform loop over 32-vertex words
        const uint32_t u = w * 32 + lane;
        const bool b = u < n && ((prev[w] >> lane) & 1u);
        uint32_t k0 = 0, k1 = 0, m = 0;
        if (b) {
            k0 = off[u];
            k1 = off[u + 1];
            m = label[u];
        }
        const bool big = b && k1 - k0 > NA_LANE_DEG;
        if (b && !big)
            for (uint32_t k = k0; k < k1; ++k) na_deliver(n, col[k], m, p, bad);
        uint32_t todo = __ballot_sync(0xFFFFFFFFu, big);
        while (todo) {
            const uint32_t src = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint32_t a = __shfl_sync(0xFFFFFFFFu, k0, src), e = __shfl_sync(0xFFFFFFFFu, k1, src);
            const uint32_t mm = __shfl_sync(0xFFFFFFFFu, m, src);
            for (uint32_t k = a + lane; k < e; k += 32) na_deliver(n, col[k], mm, p, bad);
        }
    }
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(p.err, NA_ERR_IDS);
}

// compute() of Fig. 9 for the recipients of superstep s; counts the messages
// the new broadcasters send (the halt test).
__global__ void na_apply(uint32_t n, const uint32_t* off, uint32_t* label, NaPtrs p, uint32_t s) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    uint32_t* next = (s & 1) ? p.bc[1] : p.bc[0];
    unsigned long long sent = 0;
    for (uint32_t v = tid; v < n; v += nth) {
        const uint32_t bit = 1u << (v & 31u);
        if (!(p.recv[v >> 5] & bit)) continue;
        const uint32_t m = p.mbox[v];
        p.mbox[v] = NA_INF;
        if (m < label[v]) {
            label[v] = m;
            atomicOr(next + (v >> 5), bit);
            sent += off[v + 1] - off[v];
        }
    }
    if (sent) atomicAdd(p.msgs, sent);
}

// The recipient bitmap is cleared after the apply has read all of it.
__global__ void na_clear_recv(uint32_t n, NaPtrs p) {
    const uint32_t W = (n + 31) / 32;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < W; w += gridDim.x * blockDim.x) p.recv[w] = 0;
}

std::mutex na_mutex;
uint32_t* na_base[128] = {};

// Device address of the scratch array on the current device (looked up once).
int na_scratch_address(uint32_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IP_E_CUDA;
    if (dev < 0 || dev >= 128) return IP_E_RANGE;
    std::lock_guard<std::mutex> lock(na_mutex);
    if (!na_base[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, na_scratch) != cudaSuccess || ptr == nullptr) {
            (void)cudaGetLastError();
            return IP_E_CUDA;
        }
        na_base[dev] = static_cast<uint32_t*>(ptr);
    }
    *out = na_base[dev];
    return IP_OK;
}

}  // namespace

extern "C" int ip_hashmin_noalloc(uint32_t n_vertices, uint64_t n_edges, const uint32_t* csr_offsets,
                                  const uint32_t* csr_cols, uint32_t* labels, uint32_t max_supersteps,
                                  uint32_t* supersteps_out, void* stream) {
    if (n_vertices == 0 || !csr_offsets || !labels || max_supersteps == 0) return IP_E_INVAL;
    if (n_edges > 0 && !csr_cols) return IP_E_INVAL;
    if (n_vertices > NA_MAX_V) return IP_E_RANGE;
    if (n_edges >= 0xFFFFFFFFull) return IP_E_RANGE;
    uint32_t* base = nullptr;
    int r = na_scratch_address(&base);
    if (r != IP_OK) return r;
    const NaPtrs p = na_layout(base);
    cudaStream_t st = (cudaStream_t)stream;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = sms > 0 ? sms * 4 : 128;
    // {messages sent (64-bit), error bits}, read back after every superstep
    struct {
        unsigned long long sent;
        uint32_t err, spare;
    } ctr = {0, 0, 0};
    auto read_counters = [&]() -> int {
        if (cudaMemcpyAsync(&ctr, p.msgs, sizeof(ctr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return IP_E_CUDA;
        if (ctr.err & NA_ERR_OFFSETS) return IP_E_INVAL;
        if (ctr.err & NA_ERR_IDS) return IP_E_RANGE;
        return IP_OK;
    };
    if (cudaMemsetAsync(p.err, 0, sizeof(uint32_t), st) != cudaSuccess) return IP_E_CUDA;
    na_validate<<<grid, NA_BLOCK, 0, st>>>(n_vertices, csr_offsets, (unsigned long long)n_edges, p);
    na_init<<<grid, NA_BLOCK, 0, st>>>(n_vertices, labels, p, (unsigned long long)n_edges);
    if (cudaGetLastError() != cudaSuccess) return IP_E_CUDA;
    if ((r = read_counters()) != IP_OK) return r;  // bad offsets: no edge has been read
    uint32_t s = 0;  // last completed superstep
    int halted = n_edges == 0;
    while (!halted && s + 1 < max_supersteps) {
        ++s;
        na_push<<<grid, NA_BLOCK, 0, st>>>(n_vertices, csr_offsets, csr_cols, labels, p, s);
        na_apply<<<grid, NA_BLOCK, 0, st>>>(n_vertices, csr_offsets, labels, p, s);
        na_clear_recv<<<grid, NA_BLOCK, 0, st>>>(n_vertices, p);
        if (cudaGetLastError() != cudaSuccess) return IP_E_CUDA;
        if ((r = read_counters()) != IP_OK) return r;
        halted = ctr.sent == 0;
    }
    if (supersteps_out) *supersteps_out = s + 1;
    return halted ? IP_OK : IP_E_MAXSTEPS;
}
