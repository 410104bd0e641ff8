// mlp.cu -- the schedule MLP: 6 -> 64 tanh -> 64 tanh -> 1, fp32 master
// parameters, forward and backward with their bf16 roundings and fp32
// accumulation, Adam. Parameters are one flat vector
// [W1 (64x6 row-major), b1 (64), W2 (64x64), b2 (64), W3 (64), b3 (1)].
// The network proposes the next annealing step (Sec. 5.4 cites adaptive
// steps); the histogram overlap judges every proposal.
#include <cuda_bf16.h>

#include "device.cuh"
#include "internal.h"

namespace gbmc {

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// One sample's forward pass with bf16-rounded weights (fp32 sums); h1, h2:
// caller storage of 64 floats each.
__device__ __forceinline__ float mlp_forward_one(const float* __restrict__ p, const float* x, float* h1,
                                                 float* h2) {
    for (int j = 0; j < kMlpHidden; ++j) {
        float a = bf(p[kOffB1 + j]);
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) a += bf(p[kOffW1 + j * kMlpIn + i]) * x[i];
        h1[j] = tanhf(a);
    }
    for (int j = 0; j < kMlpHidden; ++j) {
        float a = bf(p[kOffB2 + j]);
        for (int k = 0; k < kMlpHidden; ++k) a += bf(p[kOffW2 + j * kMlpHidden + k]) * h1[k];
        h2[j] = tanhf(a);
    }
    float y = bf(p[kOffB3]);
    for (int j = 0; j < kMlpHidden; ++j) y += bf(p[kOffW3 + j]) * h2[j];
    return y;
}

// Batch inference: one thread per sample.
__global__ void k_mlp_forward(const float* __restrict__ p, const float* __restrict__ X, uint32_t B,
                              float* __restrict__ Y) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float x[kMlpIn], h1[kMlpHidden], h2[kMlpHidden];
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) x[i] = X[(uint64_t)b * kMlpIn + i];
    Y[b] = mlp_forward_one(p, x, h1, h2);
}

cudaError_t launch_mlp_forward(const float* p, const float* X, uint32_t B, float* Y, cudaStream_t s) {
    k_mlp_forward<<<(B + 127) / 128, 128, 0, s>>>(p, X, B, Y);
    count_launch();
    return cudaGetLastError();
}

// Gradient of (1/B) sum_b (y_b - t_b)^2 / 2 over one minibatch of B <= kMlpMaxBatch
// samples, in one CTA (fixed summation order: deterministic). Shared memory:
// X [B][6], h1, h2, dz2, dz1 [B][64].
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ p, const float* __restrict__ X,
                                                  const float* __restrict__ T, uint32_t B, float* __restrict__ g,
                                                  float* __restrict__ loss) {
    extern __shared__ float sm[];
    float* xs = sm;
    float* h1 = xs + kMlpMaxBatch * kMlpIn;
    float* h2 = h1 + kMlpMaxBatch * kMlpHidden;
    float* dz2 = h2 + kMlpMaxBatch * kMlpHidden;
    float* dz1 = dz2 + kMlpMaxBatch * kMlpHidden;
    __shared__ float dy[kMlpMaxBatch];
    __shared__ float red[32];
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = tid; i < B * kMlpIn; i += blockDim.x) xs[i] = X[i];
    __syncthreads();
    float l = 0.f;
    for (uint32_t b = tid; b < B; b += blockDim.x) {
        const float y = mlp_forward_one(p, xs + b * kMlpIn, h1 + b * kMlpHidden, h2 + b * kMlpHidden);
        const float d = y - T[b];
        l += 0.5f * d * d;
        dy[b] = d / (float)B;
    }
    l = warp_sum(l);
    if ((tid & 31) == 0) red[tid >> 5] = l;
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
        for (uint32_t w = 0; w < blockDim.x / 32; ++w) s += red[w];
        loss[0] = s / (float)B;
    }
    // back through layer 3 and the second tanh
    for (uint32_t b = tid; b < B; b += blockDim.x)
        for (int j = 0; j < kMlpHidden; ++j) {
            const float hv = h2[b * kMlpHidden + j];
            dz2[b * kMlpHidden + j] = dy[b] * bf(p[kOffW3 + j]) * (1.f - hv * hv);
        }
    __syncthreads();
    // through layer 2 and the first tanh
    for (uint32_t b = tid; b < B; b += blockDim.x)
        for (int k = 0; k < kMlpHidden; ++k) {
            float a = 0.f;
            for (int j = 0; j < kMlpHidden; ++j) a += dz2[b * kMlpHidden + j] * bf(p[kOffW2 + j * kMlpHidden + k]);
            const float hv = h1[b * kMlpHidden + k];
            dz1[b * kMlpHidden + k] = a * (1.f - hv * hv);
        }
    __syncthreads();
    // parameter gradients: sums over the batch in sample order
    for (uint32_t q = tid; q < (uint32_t)kMlpParams; q += blockDim.x) {
        float a = 0.f;
        if (q < kOffB1) {
            const uint32_t j = q / kMlpIn, i = q % kMlpIn;
            for (uint32_t b = 0; b < B; ++b) a += dz1[b * kMlpHidden + j] * xs[b * kMlpIn + i];
        } else if (q < kOffW2) {
            const uint32_t j = q - kOffB1;
            for (uint32_t b = 0; b < B; ++b) a += dz1[b * kMlpHidden + j];
        } else if (q < kOffB2) {
            const uint32_t j = (q - kOffW2) / kMlpHidden, k = (q - kOffW2) % kMlpHidden;
            for (uint32_t b = 0; b < B; ++b) a += dz2[b * kMlpHidden + j] * h1[b * kMlpHidden + k];
        } else if (q < kOffW3) {
            const uint32_t j = q - kOffB2;
            for (uint32_t b = 0; b < B; ++b) a += dz2[b * kMlpHidden + j];
        } else if (q < kOffB3) {
            const uint32_t j = q - kOffW3;
            for (uint32_t b = 0; b < B; ++b) a += dy[b] * h2[b * kMlpHidden + j];
        } else {
            for (uint32_t b = 0; b < B; ++b) a += dy[b];
        }
        g[q] = a;
    }
}

size_t mlp_grad_smem() { return sizeof(float) * kMlpMaxBatch * (kMlpIn + 4 * kMlpHidden); }

cudaError_t launch_mlp_grad(const float* p, const float* X, const float* T, uint32_t B, float* g, float* loss,
                            cudaStream_t s) {
    const size_t smem = mlp_grad_smem();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_mlp_grad<<<1, 256, smem, s>>>(p, X, T, B, g, loss);
    count_launch();
    return cudaGetLastError();
}

__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, float lr, float c1, float c2) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (uint32_t)kMlpParams) return;
    const float gq = g[q];
    const float mq = 0.9f * m[q] + 0.1f * gq;
    const float vq = 0.999f * v[q] + 0.001f * gq * gq;
    m[q] = mq;
    v[q] = vq;
    p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + 1e-8f);
}

cudaError_t launch_mlp_adam(float* p, const float* g, float* m, float* v, uint32_t k, float lr, cudaStream_t s) {
    const float c1 = 1.0f - (float)pow(0.9, (double)k);
    const float c2 = 1.0f - (float)pow(0.999, (double)k);
    k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(p, g, m, v, lr, c1, c2);
    count_launch();
    return cudaGetLastError();
}

}  // namespace gbmc
