// Cost model of the learned switch: FP32 training kernels (forward, backward,
// Adam), the BF16 inference used inside the iteration loop, and the cost
// model installed on a graph.  Plain FMA arithmetic (no tensor cores): the
// model is tiny and runs on at most six rows inside the decision.
#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"
#include "mlp.cuh"

namespace wedge {

constexpr int kGradRows = 128;  // samples per block in the gradient kernel
constexpr int kPad = kMlpHidden + 1;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// FP32 forward, one thread per row.
__global__ void k_mlp_forward(const float* __restrict__ p, const float* __restrict__ X, uint32_t n,
                              float* __restrict__ Y) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float x[kMlpIn], h1[kMlpHidden];
        for (int f = 0; f < kMlpIn; ++f) x[f] = X[(size_t)i * kMlpIn + f];
        for (int j = 0; j < kMlpHidden; ++j) {
            float a = p[kMlpB1 + j];
            for (int f = 0; f < kMlpIn; ++f) a = fmaf(p[kMlpW1 + j * kMlpIn + f], x[f], a);
            h1[j] = fmaxf(a, 0.f);
        }
        float y = p[kMlpB3];
        for (int j = 0; j < kMlpHidden; ++j) {
            float a = p[kMlpB2 + j];
            for (int k = 0; k < kMlpHidden; ++k) a = fmaf(p[kMlpW2 + j * kMlpHidden + k], h1[k], a);
            y = fmaf(p[kMlpW3 + j], fmaxf(a, 0.f), y);
        }
        Y[i] = y;
    }
}

// Inference as the decision runs it: BF16 weights and activations, FP32
// accumulation.  One row per thread (test entry point).
__global__ void k_mlp_forward_bf16(const __nv_bfloat16* __restrict__ w, const float* __restrict__ X, uint32_t n,
                                   float* __restrict__ Y) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float x[kMlpIn], h1[kMlpHidden];
        for (int f = 0; f < kMlpIn; ++f) x[f] = bf16r(X[(size_t)i * kMlpIn + f]);
        for (int j = 0; j < kMlpHidden; ++j) {
            float a = __bfloat162float(w[kMlpB1 + j]);
            for (int f = 0; f < kMlpIn; ++f) a = fmaf(__bfloat162float(w[kMlpW1 + j * kMlpIn + f]), x[f], a);
            h1[j] = bf16r(fmaxf(a, 0.f));
        }
        float y = __bfloat162float(w[kMlpB3]);
        for (int j = 0; j < kMlpHidden; ++j) {
            float a = __bfloat162float(w[kMlpB2 + j]);
            for (int k = 0; k < kMlpHidden; ++k) a = fmaf(__bfloat162float(w[kMlpW2 + j * kMlpHidden + k]), h1[k], a);
            y = fmaf(__bfloat162float(w[kMlpW3 + j]), bf16r(fmaxf(a, 0.f)), y);
        }
        Y[i] = y;
    }
}

// Loss L = mean_i (f(x_i) - t_i)^2 and its gradient, accumulated into
// grad[] (zeroed by the caller) with one atomic per parameter per block.
// A block takes kGradRows rows: activations, then the backward pass as
// small matrix products in shared memory.
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ p, const float* __restrict__ X,
                                                  const float* __restrict__ T, uint32_t n, float* __restrict__ grad,
                                                  float* __restrict__ loss) {
    extern __shared__ float sm[];
    float* xs = sm;                                  // [128][12]
    float* H1 = xs + kGradRows * kMlpIn;             // [128][65]
    float* H2 = H1 + kGradRows * kPad;               // [128][65]
    float* dy = H2 + kGradRows * kPad;               // [128]
    float* red = dy + kGradRows;                     // [32]
    const int tid = threadIdx.x;
    const uint32_t r0 = blockIdx.x * kGradRows;
    const int rows = (int)min((uint32_t)kGradRows, n - r0);
    for (int i = tid; i < kGradRows * kMlpIn; i += blockDim.x)
        xs[i] = (i / kMlpIn) < rows ? X[(size_t)r0 * kMlpIn + i] : 0.f;
    __syncthreads();
    // layer 1
    for (int o = tid; o < kGradRows * kMlpHidden; o += blockDim.x) {
        const int s = o / kMlpHidden, j = o % kMlpHidden;
        float a = p[kMlpB1 + j];
        for (int f = 0; f < kMlpIn; ++f) a = fmaf(p[kMlpW1 + j * kMlpIn + f], xs[s * kMlpIn + f], a);
        H1[s * kPad + j] = fmaxf(a, 0.f);
    }
    __syncthreads();
    // layer 2
    for (int o = tid; o < kGradRows * kMlpHidden; o += blockDim.x) {
        const int s = o / kMlpHidden, j = o % kMlpHidden;
        float a = p[kMlpB2 + j];
        for (int k = 0; k < kMlpHidden; ++k) a = fmaf(p[kMlpW2 + j * kMlpHidden + k], H1[s * kPad + k], a);
        H2[s * kPad + j] = fmaxf(a, 0.f);
    }
    __syncthreads();
    // output, error, dL/dy
    float l = 0.f;
    if (tid < kGradRows) {
        float g = 0.f;
        if (tid < rows) {
            float y = p[kMlpB3];
            for (int j = 0; j < kMlpHidden; ++j) y = fmaf(p[kMlpW3 + j], H2[tid * kPad + j], y);
            const float e = y - T[r0 + tid];
            l = e * e;
            g = 2.f * e / (float)n;
        }
        dy[tid] = g;
    }
    for (int d = 16; d > 0; d >>= 1) l += __shfl_down_sync(0xFFFFFFFFu, l, d);
    if ((tid & 31) == 0) red[tid >> 5] = l;
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s / (float)n);
    }
    // w3, b3
    if (tid < kMlpHidden) {
        float a = 0.f;
        for (int s = 0; s < kGradRows; ++s) a = fmaf(dy[s], H2[s * kPad + tid], a);
        atomicAdd(grad + kMlpW3 + tid, a);
    } else if (tid == kMlpHidden) {
        float a = 0.f;
        for (int s = 0; s < kGradRows; ++s) a += dy[s];
        atomicAdd(grad + kMlpB3, a);
    }
    __syncthreads();
    // dH2 = dy * w3 * [h2 > 0]  (in place)
    for (int o = tid; o < kGradRows * kMlpHidden; o += blockDim.x) {
        const int s = o / kMlpHidden, j = o % kMlpHidden;
        const float h = H2[s * kPad + j];
        H2[s * kPad + j] = h > 0.f ? dy[s] * p[kMlpW3 + j] : 0.f;
    }
    __syncthreads();
    // W2, b2
    for (int o = tid; o < kMlpHidden * kMlpHidden; o += blockDim.x) {
        const int j = o / kMlpHidden, k = o % kMlpHidden;
        float a = 0.f;
        for (int s = 0; s < kGradRows; ++s) a = fmaf(H2[s * kPad + j], H1[s * kPad + k], a);
        atomicAdd(grad + kMlpW2 + o, a);
    }
    if (tid < kMlpHidden) {
        float a = 0.f;
        for (int s = 0; s < kGradRows; ++s) a += H2[s * kPad + tid];
        atomicAdd(grad + kMlpB2 + tid, a);
    }
    __syncthreads();
    // dH1 = (W2^T dH2) * [h1 > 0]  (in place)
    for (int o = tid; o < kGradRows * kMlpHidden; o += blockDim.x) {
        const int s = o / kMlpHidden, k = o % kMlpHidden;
        float a = 0.f;
        for (int j = 0; j < kMlpHidden; ++j) a = fmaf(H2[s * kPad + j], p[kMlpW2 + j * kMlpHidden + k], a);
        H1[s * kPad + k] = H1[s * kPad + k] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // W1, b1
    for (int o = tid; o < kMlpHidden * kMlpIn; o += blockDim.x) {
        const int k = o / kMlpIn, f = o % kMlpIn;
        float a = 0.f;
        for (int s = 0; s < kGradRows; ++s) a = fmaf(H1[s * kPad + k], xs[s * kMlpIn + f], a);
        atomicAdd(grad + kMlpW1 + o, a);
    }
    if (tid < kMlpHidden) {
        float a = 0.f;
        for (int s = 0; s < kGradRows; ++s) a += H1[s * kPad + tid];
        atomicAdd(grad + kMlpB1 + tid, a);
    }
}

__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, float lr, float b1t, float b2t) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMlpParams; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / (1.f - b1t)) / (sqrtf(vi / (1.f - b2t)) + eps);
    }
}

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}

// The in-loop decision's copy of the model: BF16, with W2 stored k-major
// (out[W2 + k*64 + j] = W2[j][k]) so that the deciding block's threads read
// consecutive weights; the rest as laid out in the parameter array.
__global__ void k_to_bf16_decision(const float* __restrict__ in, __nv_bfloat16* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMlpParams; i += gridDim.x * blockDim.x) {
        int o = i;
        if (i >= kMlpW2 && i < kMlpB2) {
            const int jk = i - kMlpW2;
            o = kMlpW2 + (jk % kMlpHidden) * kMlpHidden + jk / kMlpHidden;
        }
        out[o] = __float2bfloat16_rn(in[i]);
    }
}

// Device buffer that holds a caller's parameters (host or device) as FP32.
static wedge_status params_on_device(const float* params, float** dev, bool* owned) {
    *owned = false;
    if (classify(params) == PtrKind::Device) {
        *dev = const_cast<float*>(params);
        return WEDGE_OK;
    }
    WEDGE_TRY(dev_alloc(nullptr, (void**)dev, kMlpParams * sizeof(float)));
    *owned = true;
    WEDGE_TRY_CUDA(cudaMemcpy(*dev, params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice));
    return WEDGE_OK;
}

}  // namespace wedge

using namespace wedge;

extern "C" {

wedge_status wedge_mlp_forward(const float* d_params, const float* d_x, uint32_t n, float* d_y,
                               wedge_stream_t stream) {
    if (!d_params || !d_x || !d_y) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (!n) return WEDGE_OK;
    k_mlp_forward<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d_params, d_x, n, d_y);
    count_launch();
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

wedge_status wedge_mlp_forward_bf16(const float* d_params, const float* d_x, uint32_t n, float* d_y,
                                    wedge_stream_t stream) {
    if (!d_params || !d_x || !d_y) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (!n) return WEDGE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    __nv_bfloat16* w = nullptr;
    WEDGE_TRY(dev_alloc(nullptr, (void**)&w, kMlpParams * sizeof(__nv_bfloat16)));
    k_to_bf16<<<20, 256, 0, s>>>(d_params, w, kMlpParams);
    k_mlp_forward_bf16<<<(n + 127) / 128, 128, 0, s>>>(w, d_x, n, d_y);
    count_launch(2);
    cudaError_t e = cudaStreamSynchronize(s);
    dev_free(w);
    if (e != cudaSuccess) return cuda_error(e, "bf16 forward");
    return WEDGE_OK;
}

wedge_status wedge_mlp_loss_grad(const float* d_params, const float* d_x, const float* d_t, uint32_t n,
                                 float* d_grad, float* d_loss, wedge_stream_t stream) {
    if (!d_params || !d_x || !d_t || !d_grad || !d_loss) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    WEDGE_TRY_CUDA(cudaMemsetAsync(d_grad, 0, kMlpParams * sizeof(float), s));
    WEDGE_TRY_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(float), s));
    if (!n) return WEDGE_OK;
    const int smem = (kGradRows * kMlpIn + 2 * kGradRows * kPad + kGradRows + 32) * (int)sizeof(float);
    static bool attr = false;
    if (!attr) {
        WEDGE_TRY_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = true;
    }
    k_mlp_grad<<<(n + kGradRows - 1) / kGradRows, 256, smem, s>>>(d_params, d_x, d_t, n, d_grad, d_loss);
    count_launch();
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

wedge_status wedge_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, uint32_t t, float lr,
                            wedge_stream_t stream) {
    if (!d_params || !d_grad || !d_m || !d_v || t == 0) return set_error(WEDGE_ERR_INVALID_ARG, "bad argument");
    const float b1t = powf(0.9f, (float)t), b2t = powf(0.999f, (float)t);
    k_mlp_adam<<<20, 256, 0, (cudaStream_t)stream>>>(d_params, d_grad, d_m, d_v, lr, b1t, b2t);
    count_launch();
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

wedge_status wedge_set_learned_band(wedge_graph_t g, float lo, float hi) {
    if (!g) return set_error(WEDGE_ERR_INVALID_ARG, "graph is NULL");
    if (!(lo >= 0.f) || !(hi >= lo)) return set_error(WEDGE_ERR_INVALID_ARG, "band needs 0 <= lo <= hi");
    DeviceGuard dg(g->device);
    WEDGE_TRY_CUDA(cudaDeviceSynchronize());
    // the device-loop graphs captured the previous band: rebuild them
    for (auto& e : g->loop_exec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
    g->loop_failed = false;
    g->band_lo = lo;
    g->band_hi = hi;
    return WEDGE_OK;
}

wedge_status wedge_set_cost_model(wedge_graph_t g, const float* params) {
    if (!g) return set_error(WEDGE_ERR_INVALID_ARG, "graph is NULL");
    DeviceGuard dg(g->device);
    WEDGE_TRY_CUDA(cudaDeviceSynchronize());
    // the device-loop graphs captured the previous model pointer: rebuild them
    for (auto& e : g->loop_exec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
    g->loop_failed = false;
    if (!params) {
        g->has_model = false;
        return WEDGE_OK;
    }
    if (!g->mlp_bf16) WEDGE_TRY(dev_alloc(g, (void**)&g->mlp_bf16, kMlpParams * sizeof(__nv_bfloat16) + 16));
    float* dp = nullptr;
    bool owned = false;
    WEDGE_TRY(params_on_device(params, &dp, &owned));
    k_to_bf16_decision<<<20, 256>>>(dp, reinterpret_cast<__nv_bfloat16*>(g->mlp_bf16));
    count_launch();
    cudaError_t e = cudaDeviceSynchronize();
    if (owned) dev_free(dp);
    if (e != cudaSuccess) return cuda_error(e, "cost model upload");
    g->has_model = true;
    return WEDGE_OK;
}

}  // extern "C"
