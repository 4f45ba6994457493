// Training kernels of the learned mode selector: an 8 -> 32 -> 32 -> 3 MLP with
// BF16 weights and FP32 accumulation, trained on the per-superstep frontier
// features and per-mode timings that the superstep engine logs.
//
//   xn = (x - mu) / sd
//   h1 = relu(W1 xn + b1),  h2 = relu(W2 h1 + b2),  z = W3 h2 + b3
//   loss = sum_i s_i * (logsumexp(z_i) - z_i[y_i]) / sum_i s_i
//
// The FP32 master parameters are rounded to BF16 (round to nearest even) in the
// forward and backward passes; their gradients update the FP32 masters
// (straight-through). One warp evaluates one sample at a time: lane j owns hidden
// unit j of both layers, exactly as the inference path in the selector kernel
// does, so training and inference compute the same logits.
//
// Parameter vector (IP_MLP_PARAMS floats): W1[32][8], b1[32], W2[32][32], b2[32],
// W3[3][32], b3[3]; normalisation mu[8], sd[8] passed separately.
#include <cuda_bf16.h>

#include "internal.h"

namespace {

constexpr int H = 32, IN = 8, OUT = 3;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + OUT * H, NPARAM = OFF_B3 + OUT;
static_assert(NPARAM == IP_MLP_PARAMS, "parameter count");
constexpr unsigned FULLM = 0xFFFFFFFFu;
constexpr int MLP_WARPS = 8;          // warps per CTA
constexpr int MLP_MAX_CTAS = 256;     // partial-gradient slots of the workspace

__device__ __forceinline__ float rbf(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

// Weights a lane needs, rounded to BF16.
struct LaneW {
    float w1[IN];   // row j of W1
    float w2r[H];   // row j of W2
    float w2c[H];   // column j of W2
    float w3[OUT];  // column j of W3
    float b1, b2, b3[OUT];
};

__device__ __forceinline__ void load_lane_weights(const float* p, LaneW& L) {
    const int j = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < IN; ++i) L.w1[i] = rbf(p[OFF_W1 + j * IN + i]);
#pragma unroll
    for (int k = 0; k < H; ++k) {
        L.w2r[k] = rbf(p[OFF_W2 + j * H + k]);
        L.w2c[k] = rbf(p[OFF_W2 + k * H + j]);
    }
#pragma unroll
    for (int m = 0; m < OUT; ++m) {
        L.w3[m] = rbf(p[OFF_W3 + m * H + j]);
        L.b3[m] = p[OFF_B3 + m];
    }
    L.b1 = p[OFF_B1 + j];
    L.b2 = p[OFF_B2 + j];
}

struct Fwd {
    float xn[IN];
    float a1, h1, a2, h2;
    float z[OUT];
};

// Forward pass of one sample by one warp (lane j = hidden unit j).
__device__ __forceinline__ void forward_one(const LaneW& L, const float* x, const float* musd, Fwd& f) {
#pragma unroll
    for (int i = 0; i < IN; ++i) f.xn[i] = (x[i] - musd[i]) / musd[IN + i];
    float a1 = L.b1;
#pragma unroll
    for (int i = 0; i < IN; ++i) a1 = fmaf(L.w1[i], f.xn[i], a1);
    f.a1 = a1;
    f.h1 = fmaxf(a1, 0.f);
    float a2 = L.b2;
#pragma unroll
    for (int k = 0; k < H; ++k) a2 = fmaf(L.w2r[k], __shfl_sync(FULLM, f.h1, k), a2);
    f.a2 = a2;
    f.h2 = fmaxf(a2, 0.f);
#pragma unroll
    for (int m = 0; m < OUT; ++m) {
        float p = L.w3[m] * f.h2;
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(FULLM, p, o);
        f.z[m] = p + L.b3[m];
    }
}

__global__ void __launch_bounds__(32 * MLP_WARPS) k_mlp_forward(const float* params, const float* musd,
                                                                 const float* X, uint32_t n, float* logits) {
    LaneW L;
    load_lane_weights(params, L);
    float ms[2 * IN];
#pragma unroll
    for (int i = 0; i < 2 * IN; ++i) ms[i] = musd[i];
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = warp; i < n; i += nw) {
        float x[IN];
#pragma unroll
        for (int k = 0; k < IN; ++k) x[k] = X[(size_t)i * IN + k];
        Fwd f;
        forward_one(L, x, ms, f);
        if ((threadIdx.x & 31) < OUT) logits[(size_t)i * OUT + (threadIdx.x & 31)] = f.z[threadIdx.x & 31];
    }
}

// Per-warp gradient accumulation, then one partial per CTA in the workspace.
__global__ void __launch_bounds__(32 * MLP_WARPS) k_mlp_backward(const float* params, const float* musd,
                                                                  const float* X, const int32_t* y, const float* sw,
                                                                  uint32_t n, float inv_total, float* partial) {
    __shared__ float acc[NPARAM + 1];
    for (int i = threadIdx.x; i < NPARAM + 1; i += blockDim.x) acc[i] = 0.f;
    __syncthreads();
    LaneW L;
    load_lane_weights(params, L);
    float ms[2 * IN];
#pragma unroll
    for (int i = 0; i < 2 * IN; ++i) ms[i] = musd[i];
    const int j = threadIdx.x & 31;
    float gw1[IN] = {}, gw2[H] = {}, gw3[OUT] = {}, gb3[OUT] = {};
    float gb1 = 0.f, gb2 = 0.f, lsum = 0.f;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = warp; i < n; i += nw) {
        float x[IN];
#pragma unroll
        for (int k = 0; k < IN; ++k) x[k] = X[(size_t)i * IN + k];
        Fwd f;
        forward_one(L, x, ms, f);
        const int yi = y[i];
        const float wi = sw[i] * inv_total;
        float zmax = fmaxf(fmaxf(f.z[0], f.z[1]), f.z[2]);
        float e[OUT], se = 0.f;
#pragma unroll
        for (int m = 0; m < OUT; ++m) {
            e[m] = expf(f.z[m] - zmax);
            se += e[m];
        }
        lsum += wi * (zmax + logf(se) - f.z[yi]);
        float dz[OUT];
#pragma unroll
        for (int m = 0; m < OUT; ++m) dz[m] = (e[m] / se - (m == yi ? 1.f : 0.f)) * wi;
        // layer 3
        float dh2 = 0.f;
#pragma unroll
        for (int m = 0; m < OUT; ++m) {
            gw3[m] = fmaf(dz[m], f.h2, gw3[m]);
            gb3[m] += dz[m];
            dh2 = fmaf(L.w3[m], dz[m], dh2);
        }
        const float da2 = f.a2 > 0.f ? dh2 : 0.f;
        // layer 2: dW2[j][k] = da2_j * h1_k ; dh1_j = sum_k W2[k][j] * da2_k
        float dh1 = 0.f;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            gw2[k] = fmaf(da2, __shfl_sync(FULLM, f.h1, k), gw2[k]);
            dh1 = fmaf(L.w2c[k], __shfl_sync(FULLM, da2, k), dh1);
        }
        gb2 += da2;
        const float da1 = f.a1 > 0.f ? dh1 : 0.f;
#pragma unroll
        for (int k = 0; k < IN; ++k) gw1[k] = fmaf(da1, f.xn[k], gw1[k]);
        gb1 += da1;
    }
    // reduce the warps of this CTA in shared memory (fixed order: warp 0 first)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        if ((int)(threadIdx.x >> 5) == w) {
#pragma unroll
            for (int k = 0; k < IN; ++k) acc[OFF_W1 + j * IN + k] += gw1[k];
            acc[OFF_B1 + j] += gb1;
#pragma unroll
            for (int k = 0; k < H; ++k) acc[OFF_W2 + j * H + k] += gw2[k];
            acc[OFF_B2 + j] += gb2;
#pragma unroll
            for (int m = 0; m < OUT; ++m) acc[OFF_W3 + m * H + j] += gw3[m];
            if (j == 0) {
#pragma unroll
                for (int m = 0; m < OUT; ++m) acc[OFF_B3 + m] += gb3[m];
                acc[NPARAM] += lsum;
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < NPARAM + 1; i += blockDim.x) partial[(size_t)blockIdx.x * (NPARAM + 1) + i] = acc[i];
}

// Sums the per-CTA partials in CTA order (deterministic).
__global__ void k_mlp_reduce(const float* partial, int nblocks, float* grad, float* loss) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM + 1; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * (NPARAM + 1) + i];
        if (i < NPARAM)
            grad[i] = s;
        else if (loss)
            *loss = s;
    }
}

__global__ void k_mlp_adam(float* p, const float* g, float* m, float* v, uint32_t count, float lr, float b1, float b2,
                           float eps, float c1, float c2) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// FP32 masters -> selector blob (layout of IP_SELECTOR_BYTES).
__global__ void k_mlp_pack(const float* p, const float* musd, ipg::SelectorDev* out) {
    for (int i = threadIdx.x; i < 2 * IN; i += blockDim.x) (i < IN ? out->mu[i] : out->sd[i - IN]) = musd[i];
    for (int i = threadIdx.x; i < H * IN; i += blockDim.x)
        out->W1[i] = __bfloat16_as_ushort(__float2bfloat16_rn(p[OFF_W1 + i]));
    for (int i = threadIdx.x; i < H * H; i += blockDim.x)
        out->W2[i] = __bfloat16_as_ushort(__float2bfloat16_rn(p[OFF_W2 + i]));
    for (int i = threadIdx.x; i < OUT * H; i += blockDim.x)
        out->W3[i] = __bfloat16_as_ushort(__float2bfloat16_rn(p[OFF_W3 + i]));
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        out->b1[i] = p[OFF_B1 + i];
        out->b2[i] = p[OFF_B2 + i];
    }
    if (threadIdx.x < OUT) out->b3[threadIdx.x] = p[OFF_B3 + threadIdx.x];
}

int grid_for_samples(uint32_t n) {
    int ctas = (int)((n + MLP_WARPS - 1) / MLP_WARPS);
    if (ctas > MLP_MAX_CTAS) ctas = MLP_MAX_CTAS;
    return ctas < 1 ? 1 : ctas;
}

}  // namespace

extern "C" {

size_t ip_mlp_workspace_bytes(void) { return (size_t)MLP_MAX_CTAS * (NPARAM + 1) * sizeof(float); }

int ip_mlp_forward(const float* params, const float* mu_sd, const float* X, uint32_t n, float* logits, void* stream) {
    if (!params || !mu_sd || (n && (!X || !logits))) return IP_E_INVAL;
    if (!n) return IP_OK;
    k_mlp_forward<<<grid_for_samples(n), 32 * MLP_WARPS, 0, (cudaStream_t)stream>>>(params, mu_sd, X, n, logits);
    return cudaGetLastError() == cudaSuccess ? IP_OK : IP_E_CUDA;
}

int ip_mlp_backward(const float* params, const float* mu_sd, const float* X, const int32_t* y, const float* w,
                    uint32_t n, float weight_total, float* grad, float* loss, void* workspace, size_t workspace_bytes,
                    void* stream) {
    if (!params || !mu_sd || !grad || !workspace || (n && (!X || !y || !w))) return IP_E_INVAL;
    if (workspace_bytes < ip_mlp_workspace_bytes()) return IP_E_RANGE;
    if (!(weight_total > 0.f)) return IP_E_INVAL;
    const int ctas = grid_for_samples(n);
    cudaStream_t st = (cudaStream_t)stream;
    float* part = (float*)workspace;
    k_mlp_backward<<<ctas, 32 * MLP_WARPS, 0, st>>>(params, mu_sd, X, y, w, n, 1.f / weight_total, part);
    k_mlp_reduce<<<(NPARAM + 1 + 255) / 256, 256, 0, st>>>(part, ctas, grad, loss);
    return cudaGetLastError() == cudaSuccess ? IP_OK : IP_E_CUDA;
}

int ip_mlp_adam(float* params, const float* grad, float* m, float* v, uint32_t count, float lr, float beta1,
                float beta2, float eps, uint32_t step, void* stream) {
    if (!params || !grad || !m || !v || step == 0) return IP_E_INVAL;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_mlp_adam<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, count, lr, beta1, beta2, eps,
                                                                       c1, c2);
    return cudaGetLastError() == cudaSuccess ? IP_OK : IP_E_CUDA;
}

int ip_mlp_pack(const float* params, const float* mu_sd, void* blob, void* stream) {
    if (!params || !mu_sd || !blob) return IP_E_INVAL;
    k_mlp_pack<<<1, 256, 0, (cudaStream_t)stream>>>(params, mu_sd, (ipg::SelectorDev*)blob);
    return cudaGetLastError() == cudaSuccess ? IP_OK : IP_E_CUDA;
}

}  // extern "C"
