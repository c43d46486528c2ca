// The learned scheduler's network: an FP32 multilayer perceptron 8 -> 32 -> 32 -> 2 with ReLU
// hidden layers, evaluated and trained by the kernels below (no library calls).
//
// Parameters (1410 floats, row-major, in this order): W1[8][32], b1[32], W2[32][32], b2[32],
// W3[32][2], b3[2]; W[i][j] connects input i to output j. Outputs: out[0] = predicted
// log2(1 + |C|) (cavity size), out[1] = logit of the probability that the point loses a
// conflict at least once. Loss of one sample with targets (y0, y1):
//   (out[0] - y0)^2 + softplus(out[1]) - y1 * out[1]      (squared error + binary cross-entropy)
// averaged over the samples.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace dtg {
namespace {

constexpr int kIn = 8, kH = 32, kOut = 2;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kIn * kH, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kOut, kParams = kOffB3 + kOut;
static_assert(kParams == 1410, "parameter count");
constexpr int kMlpThreads = 256;

__device__ __forceinline__ float softplus(float z) { return z > 20.f ? z : log1pf(__expf(z)); }
__device__ __forceinline__ float sigmoid(float z) { return 1.f / (1.f + __expf(-z)); }

// Forward pass of one sample; h1, h2 keep the post-ReLU activations for the backward pass.
__device__ __forceinline__ void mlp_forward(const float* __restrict__ P, const float* x, float* h1, float* h2,
                                            float* out) {
  for (int j = 0; j < kH; ++j) {
    float a = P[kOffB1 + j];
    for (int i = 0; i < kIn; ++i) a = fmaf(x[i], P[kOffW1 + i * kH + j], a);
    h1[j] = fmaxf(a, 0.f);
  }
  for (int j = 0; j < kH; ++j) {
    float a = P[kOffB2 + j];
    for (int i = 0; i < kH; ++i) a = fmaf(h1[i], P[kOffW2 + i * kH + j], a);
    h2[j] = fmaxf(a, 0.f);
  }
  for (int j = 0; j < kOut; ++j) {
    float a = P[kOffB3 + j];
    for (int i = 0; i < kH; ++i) a = fmaf(h2[i], P[kOffW3 + i * kOut + j], a);
    out[j] = a;
  }
}

__global__ void __launch_bounds__(kMlpThreads) k_mlp_forward(const float* __restrict__ params,
                                                             const float* __restrict__ x, uint64_t n,
                                                             float* __restrict__ out) {
  __shared__ float P[kParams];
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) P[i] = params[i];
  __syncthreads();
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n; s += (uint64_t)gridDim.x * blockDim.x) {
    float xi[kIn], h1[kH], h2[kH], o[kOut];
    for (int i = 0; i < kIn; ++i) xi[i] = x[s * kIn + i];
    mlp_forward(P, xi, h1, h2, o);
    out[s * kOut] = o[0];
    out[s * kOut + 1] = o[1];
  }
}

// Sum over the samples idx[0 .. n) (or 0 .. n when idx is null) of the loss and of its gradient,
// scaled by `scale`, added into grad[kParams] and loss[0]. Each thread takes one sample at a time
// and adds its gradient into the block's shared copy; the block then adds that into grad.
__global__ void __launch_bounds__(kMlpThreads) k_mlp_grad(const float* __restrict__ params, const float* __restrict__ x,
                                                          const float* __restrict__ y, const uint32_t* __restrict__ idx,
                                                          uint64_t n, float scale, float* grad, float* loss) {
  __shared__ float P[kParams];
  __shared__ float G[kParams];
  __shared__ float L;
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) {
    P[i] = params[i];
    G[i] = 0.f;
  }
  if (threadIdx.x == 0) L = 0.f;
  __syncthreads();
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = idx ? idx[k] : k;
    float xi[kIn], h1[kH], h2[kH], o[kOut];
    for (int i = 0; i < kIn; ++i) xi[i] = x[s * kIn + i];
    mlp_forward(P, xi, h1, h2, o);
    const float y0 = y[s * kOut], y1 = y[s * kOut + 1];
    const float e = o[0] - y0;
    atomicAdd(&L, scale * (e * e + softplus(o[1]) - y1 * o[1]));
    // output layer
    const float d0 = 2.f * e * scale, d1 = (sigmoid(o[1]) - y1) * scale;
    atomicAdd(&G[kOffB3], d0);
    atomicAdd(&G[kOffB3 + 1], d1);
    float g2[kH];
    for (int i = 0; i < kH; ++i) {
      atomicAdd(&G[kOffW3 + i * kOut], h2[i] * d0);
      atomicAdd(&G[kOffW3 + i * kOut + 1], h2[i] * d1);
      g2[i] = h2[i] > 0.f ? d0 * P[kOffW3 + i * kOut] + d1 * P[kOffW3 + i * kOut + 1] : 0.f;
    }
    // second hidden layer
    float g1[kH];
    for (int i = 0; i < kH; ++i) g1[i] = 0.f;
    for (int j = 0; j < kH; ++j) {
      const float gj = g2[j];
      if (gj == 0.f) continue;
      atomicAdd(&G[kOffB2 + j], gj);
      for (int i = 0; i < kH; ++i) {
        atomicAdd(&G[kOffW2 + i * kH + j], h1[i] * gj);
        g1[i] = fmaf(gj, P[kOffW2 + i * kH + j], g1[i]);
      }
    }
    // first hidden layer
    for (int j = 0; j < kH; ++j) {
      const float gj = h1[j] > 0.f ? g1[j] : 0.f;
      if (gj == 0.f) continue;
      atomicAdd(&G[kOffB1 + j], gj);
      for (int i = 0; i < kIn; ++i) atomicAdd(&G[kOffW1 + i * kH + j], xi[i] * gj);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kParams; i += blockDim.x)
    if (G[i] != 0.f) atomicAdd(&grad[i], G[i]);
  if (threadIdx.x == 0) atomicAdd(loss, L);
}

// Adam step t (1-based) on all parameters; m and v are the moment estimates.
__global__ void k_mlp_adam(float* params, const float* grad, float* m, float* v, float lr, int t) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Minibatch of b sample indices drawn uniformly (with replacement) by a counter-based hash.
__global__ void k_mlp_draw(uint64_t n, uint32_t b, uint64_t seed, uint32_t* idx) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < b; k += gridDim.x * blockDim.x)
    idx[k] = (uint32_t)(mix64(seed + 0x9E3779B97F4A7C15ull * (k + 1)) % n);
}

unsigned mlp_grid(uint64_t n) {
  uint64_t b = (n + kMlpThreads - 1) / kMlpThreads;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 152ull * 4));
}

}  // namespace

int mlp_params() { return kParams; }

int mlp_forward(const float* params, const float* x, uint64_t n, float* out, cudaStream_t s) {
  if (n == 0) return DT_OK;
  k_mlp_forward<<<mlp_grid(n), kMlpThreads, 0, s>>>(params, x, n, out);
  ++g_kernel_launches;
  return cudaPeekAtLastError() == cudaSuccess ? DT_OK : DT_ECUDA;
}

int mlp_grad(const float* params, const float* x, const float* y, uint64_t n, float* grad, float* loss,
             cudaStream_t s) {
  if (n == 0) return DT_EINVAL;
  cudaMemsetAsync(grad, 0, kParams * sizeof(float), s);
  cudaMemsetAsync(loss, 0, sizeof(float), s);
  k_mlp_grad<<<mlp_grid(n), kMlpThreads, 0, s>>>(params, x, y, nullptr, n, 1.f / (float)n, grad, loss);
  ++g_kernel_launches;
  return cudaPeekAtLastError() == cudaSuccess ? DT_OK : DT_ECUDA;
}

int mlp_train(float* params, const float* x, const float* y, uint64_t n, uint32_t steps, uint32_t batch, float lr,
              uint64_t seed, float* losses_host, cudaStream_t s) {
  if (n == 0 || batch == 0) return DT_EINVAL;
  float *grad = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
  uint32_t* idx = nullptr;
  if (cudaMalloc(&grad, kParams * 4) != cudaSuccess || cudaMalloc(&m, kParams * 4) != cudaSuccess ||
      cudaMalloc(&v, kParams * 4) != cudaSuccess || cudaMalloc(&loss, (size_t)std::max(steps, 1u) * 4) != cudaSuccess ||
      cudaMalloc(&idx, (size_t)batch * 4) != cudaSuccess) {
    cudaFree(grad);
    cudaFree(m);
    cudaFree(v);
    cudaFree(loss);
    cudaFree(idx);
    return DT_ENOMEM;
  }
  cudaMemsetAsync(m, 0, kParams * 4, s);
  cudaMemsetAsync(v, 0, kParams * 4, s);
  cudaMemsetAsync(loss, 0, (size_t)std::max(steps, 1u) * 4, s);
  for (uint32_t t = 0; t < steps; ++t) {
    k_mlp_draw<<<(batch + 255) / 256, 256, 0, s>>>(n, batch, seed + 0x51ED2701ull * (t + 1), idx);
    cudaMemsetAsync(grad, 0, kParams * 4, s);
    k_mlp_grad<<<mlp_grid(batch), kMlpThreads, 0, s>>>(params, x, y, idx, batch, 1.f / (float)batch, grad, loss + t);
    k_mlp_adam<<<6, 256, 0, s>>>(params, grad, m, v, lr, (int)t + 1);
    g_kernel_launches += 3;
  }
  int rc = DT_OK;
  if (losses_host && steps && cudaMemcpyAsync(losses_host, loss, steps * 4ull, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = DT_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = DT_ECUDA;
  cudaFree(grad);
  cudaFree(m);
  cudaFree(v);
  cudaFree(loss);
  cudaFree(idx);
  return rc;
}

}  // namespace dtg
