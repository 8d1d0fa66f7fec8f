// fsort_learned.cu -- the learned CDF model of the learned bucket mapping:
// a 1-64-64-1 multilayer perceptron (ReLU, sigmoid output) that maps a key
// feature x = log2(key + 1) / 64, normalised to [-1, 1], to an estimate of the
// key's rank / n.  Weights are stored in BF16 for the forward passes and
// accumulated in FP32; training keeps FP32 master weights and Adam moments.
//
// Kernels (all hand-written, CUDA cores; the model is tiny):
//   mlp_grad_kernel    forward + backward of a batch, mean squared error;
//                      per-block reduction of every parameter's gradient, the
//                      64x64 layer's gradient as an in-block outer-product sum
//   mlp_adam_kernel    one Adam step on every parameter, refreshing the BF16 copy
//   mlp_eval_kernel    forward of many inputs (BF16 weights)
//   mlp_invert_kernel  splitters: for each quantile q, the smallest key whose
//                      predicted CDF reaches q (bisection on the key feature)
//
// The paper has no learned component; this model serves the learned bucket
// mapping that balances buckets under skew (Sec. IV-A leaves skew open).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fsort_dev.cuh"
#include "fsort_internal.h"

namespace fsort {
namespace {

constexpr int kH = kMlpHidden;  // 64
constexpr int kGradThreads = 64;

struct Layout {
  // parameter offsets inside one flat array
  static constexpr int W1 = 0, B1 = W1 + kH, W2 = B1 + kH, B2 = W2 + kH * kH, W3 = B2 + kH, B3 = W3 + kH;
};
static_assert(Layout::B3 + 1 == kMlpParams, "parameter count");

__device__ __forceinline__ float bf(const __nv_bfloat16* p, int i) { return __bfloat162float(p[i]); }

// Forward one input; h1/h2 receive the post-ReLU activations.
__device__ __forceinline__ float mlp_forward(const __nv_bfloat16* w, float x, float* h1, float* h2) {
#pragma unroll
  for (int i = 0; i < kH; ++i) h1[i] = fmaxf(0.f, fmaf(bf(w, Layout::W1 + i), x, bf(w, Layout::B1 + i)));
  float z = bf(w, Layout::B3);
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float a = bf(w, Layout::B2 + j);
#pragma unroll
    for (int i = 0; i < kH; ++i) a = fmaf(bf(w, Layout::W2 + j * kH + i), h1[i], a);
    h2[j] = fmaxf(0.f, a);
    z = fmaf(bf(w, Layout::W3 + j), h2[j], z);
  }
  return z;
}

__device__ __forceinline__ float sigmoid(float z) { return 1.f / (1.f + expf(-z)); }

// grads (FP32, zero on entry) += d(mean loss)/d(params) over x[0..m), y[0..m).
// Loss = 1/(2m) sum (sigmoid(z) - y)^2.  One thread per sample; its h1 and
// h2 (later dL/dh2) rows live in shared memory (odd row stride: no bank
// conflicts); every parameter's gradient is summed over the block before one
// atomic add per block.
__global__ void __launch_bounds__(kGradThreads) mlp_grad_kernel(const __nv_bfloat16* __restrict__ w,
                                                                const float* __restrict__ x,
                                                                const float* __restrict__ y, uint32_t m,
                                                                float* __restrict__ grads, float* __restrict__ loss) {
  __shared__ float s_h1[kGradThreads][kH + 1];
  __shared__ float s_d2[kGradThreads][kH + 1];
  __shared__ float s_red[kGradThreads / 32];
  const int t = threadIdx.x;
  const uint32_t s = blockIdx.x * kGradThreads + t;
  const bool valid = s < m;
  const float xs = valid ? x[s] : 0.f;
  float* h1 = s_h1[t];
  float* h2 = s_d2[t];
  // forward
#pragma unroll 8
  for (int i = 0; i < kH; ++i) h1[i] = fmaxf(0.f, fmaf(bf(w, Layout::W1 + i), xs, bf(w, Layout::B1 + i)));
  float z = bf(w, Layout::B3);
#pragma unroll 1
  for (int j = 0; j < kH; ++j) {
    float a = bf(w, Layout::B2 + j);
#pragma unroll 16
    for (int i = 0; i < kH; ++i) a = fmaf(bf(w, Layout::W2 + j * kH + i), h1[i], a);
    h2[j] = fmaxf(0.f, a);
    z = fmaf(bf(w, Layout::W3 + j), h2[j], z);
  }
  const float f = sigmoid(z);
  const float err = valid ? (f - y[s]) : 0.f;
  const float dz = err * f * (1.f - f) / float(m);
  auto block_add = [&](float v, int idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) atomicAdd(&grads[idx], v);
  };
  // output layer, then dL/dh2 replaces h2 in place
#pragma unroll 1
  for (int j = 0; j < kH; ++j) {
    const float hj = h2[j];
    block_add(dz * hj, Layout::W3 + j);
    const float d = (hj > 0.f) ? dz * bf(w, Layout::W3 + j) : 0.f;
    h2[j] = d;
    block_add(d, Layout::B2 + j);
  }
  block_add(dz, Layout::B3);
  // first layer: dL/dh1_i = relu'(h1_i) * sum_j dL/dh2_j W2[j][i]
#pragma unroll 1
  for (int i = 0; i < kH; ++i) {
    float a = 0.f;
#pragma unroll 16
    for (int j = 0; j < kH; ++j) a = fmaf(h2[j], bf(w, Layout::W2 + j * kH + i), a);
    const float d1 = (h1[i] > 0.f) ? a : 0.f;
    block_add(d1 * xs, Layout::W1 + i);
    block_add(d1, Layout::B1 + i);
  }
  {
    float l = 0.5f * err * err / float(m);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((t & 31) == 0) s_red[t >> 5] = l;
  }
  __syncthreads();
  if (t == 0 && loss) {
    float l = 0.f;
    for (int k = 0; k < kGradThreads / 32; ++k) l += s_red[k];
    atomicAdd(loss, l);
  }
  // dW2[j][i] = sum over the block's samples of dL/dh2_j * h1_i
  for (int e = t; e < kH * kH; e += kGradThreads) {
    const int j = e / kH, i = e % kH;
    float acc = 0.f;
#pragma unroll 8
    for (int r = 0; r < kGradThreads; ++r) acc = fmaf(s_d2[r][j], s_h1[r][i], acc);
    atomicAdd(&grads[Layout::W2 + e], acc);
  }
}

__global__ void mlp_adam_kernel(float* __restrict__ master, float* __restrict__ grads, float* __restrict__ m1,
                                float* __restrict__ m2, __nv_bfloat16* __restrict__ w, float lr, float beta1,
                                float beta2, float eps, float bias1, float bias2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float g = grads[i];
  grads[i] = 0.f;
  const float a = beta1 * m1[i] + (1.f - beta1) * g;
  const float b = beta2 * m2[i] + (1.f - beta2) * g * g;
  m1[i] = a;
  m2[i] = b;
  const float p = master[i] - lr * (a / bias1) / (sqrtf(b / bias2) + eps);
  master[i] = p;
  w[i] = __float2bfloat16_rn(p);
}

__global__ void mlp_eval_kernel(const __nv_bfloat16* __restrict__ w, const float* __restrict__ x, uint32_t m,
                                float* __restrict__ out) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= m) return;
  float h1[kH], h2[kH];
  out[s] = sigmoid(mlp_forward(w, x[s], h1, h2));
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = __float2bfloat16_rn(src[i]);
}

// Key feature: log2(key + 1) / 64, then affine to [-1, 1] with the model's
// (center, half) from the training sample.  Monotone non-decreasing in key.
__device__ __forceinline__ float key_feature(uint64_t k, float center, float half) {
  const float f = log2f(float(k) + 1.0f) * (1.0f / 64.0f);
  return (f - center) / half;
}

// splitters[j] = smallest key K (on the feature grid) with F(K) >= (j + 1) / B,
// j = 0 .. B-2, found by bisection on the key itself (64 steps, integer).
__global__ void mlp_invert_kernel(const __nv_bfloat16* __restrict__ w, float center, float half, uint64_t lo_key,
                                  uint64_t hi_key, uint32_t buckets, uint64_t* __restrict__ splitters) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j + 1 >= buckets) return;
  const float q = float(j + 1) / float(buckets);
  uint64_t lo = lo_key, hi = hi_key;  // invariant: F(hi) >= q or hi == hi_key
  float h1[kH], h2[kH];
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    const float f = sigmoid(mlp_forward(w, key_feature(mid, center, half), h1, h2));
    if (f >= q) hi = mid; else lo = mid + 1;
  }
  splitters[j] = lo;
}

}  // namespace

cudaError_t launch_mlp_grad(const void* w_bf16, const float* x, const float* y, uint32_t m, float* grads, float* loss,
                            cudaStream_t stream) {
  if (!m) return cudaSuccess;
  const unsigned grid = (m + kGradThreads - 1) / kGradThreads;
  mlp_grad_kernel<<<grid, kGradThreads, 0, stream>>>(static_cast<const __nv_bfloat16*>(w_bf16), x, y, m, grads, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* master, float* grads, float* m1, float* m2, void* w_bf16, float lr, int step,
                            cudaStream_t stream) {
  const float beta1 = 0.9f, beta2 = 0.999f;
  float b1 = 1.f, b2 = 1.f;
  for (int i = 0; i < step; ++i) {
    b1 *= beta1;
    b2 *= beta2;
  }
  mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(master, grads, m1, m2,
                                                                static_cast<__nv_bfloat16*>(w_bf16), lr, beta1, beta2,
                                                                1e-8f, 1.f - b1, 1.f - b2);
  return cudaGetLastError();
}

cudaError_t launch_mlp_eval(const void* w_bf16, const float* x, uint32_t m, float* out, cudaStream_t stream) {
  if (!m) return cudaSuccess;
  mlp_eval_kernel<<<(m + 127) / 128, 128, 0, stream>>>(static_cast<const __nv_bfloat16*>(w_bf16), x, m, out);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* src, void* dst, int count, cudaStream_t stream) {
  to_bf16_kernel<<<(count + 255) / 256, 256, 0, stream>>>(src, static_cast<__nv_bfloat16*>(dst), count);
  return cudaGetLastError();
}

cudaError_t launch_mlp_invert(const void* w_bf16, float center, float half, uint64_t lo_key, uint64_t hi_key,
                              uint32_t buckets, uint64_t* splitters, cudaStream_t stream) {
  if (buckets < 2) return cudaSuccess;
  mlp_invert_kernel<<<(buckets - 1 + 127) / 128, 128, 0, stream>>>(static_cast<const __nv_bfloat16*>(w_bf16), center,
                                                                   half, lo_key, hi_key, buckets, splitters);
  return cudaGetLastError();
}

}  // namespace fsort
