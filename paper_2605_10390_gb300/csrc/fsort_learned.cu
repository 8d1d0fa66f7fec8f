// fsort_learned.cu -- the learned bucket mapping and the exact sort built on it.
//
// Model: a 1-64-64-1 multilayer perceptron (ReLU, sigmoid output) from the key
// feature x = (log2(key + 1) / 64 - center) / half to an estimate of the key's
// rank / count among the non-heavy keys.  Every forward and backward pass reads
// BF16 weights and sums in FP32; training keeps FP32 master weights and Adam
// moments.  It is trained on a stratified sample sorted by this library's plain
// sort.
//
// Map: the model's CDF, mixed with a small floor that is uniform in x, made
// non-decreasing and tabulated (u32 fixed point) at the starts of the 56,320
// cells of an 11-significant-bit floating-point grid over 64-bit keys; inside
// a cell it is interpolated linearly in exact integer arithmetic.  This PLA(k)
// is non-decreasing in k, and b(k) = PLA(k) >> (32 - log2 B).  Keys that are
// frequent in the sample ("heavy") get buckets of their own:
//   id(k) = b(k) + 2 c(k) + e(k),  c(k) = heavy keys below k,  e(k) = [k heavy],
// non-decreasing in k, and a heavy key is the only key of its bucket.
//
// Sort (64-bit keys, keys only, all 64 bits; the result is the sorted
// multiset, exactly what the plain path produces):
//   learn_l1_count_kernel     per input chunk: non-heavy keys per super-bucket
//                             (id >> 10), copies of every heavy key; every
//                             key's id stored (the only map lookup it gets)
//   learn_staged_scatter<1>   non-heavy keys grouped by super-bucket (scratch),
//                             each with its 10-bit fine digit
//   learn_l2_count_kernel     per super-bucket: keys per bucket -- with the
//                             heavy counts, the exact count of every bucket id
//   learn_judge_kernel        largest non-heavy bucket; accept iff <= tau n / B
//                             (else the plain path sorts the untouched input)
//   learn_staged_scatter<2>   per super-bucket: keys to their final buckets
//   learn_fill_kernel         every heavy bucket filled with its key
//   learn_bucket_sort_kernel  every non-heavy bucket sorted on chip (a counting
//                             pass into sub-buckets, ranks by counting inside
//                             small ones, warp splits of large ones)
// Positions inside a bucket are assigned by shared-memory atomics (order
// arbitrary); the on-chip sort then orders each bucket completely.
//
// The paper has no learned component; the mapping addresses the skew it leaves
// open (Sec. IV-A), and its own histogram (Sec. III) is the judge.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "fsort_dev.cuh"
#include "fsort_internal.h"
#include "fsort_rank.cuh"

namespace fsort {
namespace {

constexpr int kH = kMlpHidden;  // 64
constexpr uint32_t kFillSplit = 32768;  // heavy buckets above this are filled by every CTA

struct Layout {
  // parameter offsets inside one flat array
  static constexpr int W1 = 0, B1 = W1 + kH, W2 = B1 + kH, B2 = W2 + kH * kH, W3 = B2 + kH, B3 = W3 + kH;
};
static_assert(Layout::B3 + 1 == kMlpParams, "parameter count");

__device__ __forceinline__ float bf(const __nv_bfloat16* p, int i) { return __bfloat162float(p[i]); }

// splitmix64 finaliser (Steele, Lea and Flood, 2014): a counter-based mixer.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float raw_feature(uint64_t k) {
  return log2f(__ull2float_rn(k) + 1.0f) * (1.0f / 64.0f);
}

// Key feature, non-decreasing in the key.
__device__ __forceinline__ float key_feature(uint64_t k, float center, float half) {
  return (raw_feature(k) - center) / half;
}

__device__ __forceinline__ float sigmoid(float z) { return 1.f / (1.f + expf(-z)); }

// ------------------------------------------------------------- training ----
// Inputs of the gradient kernel: caller arrays, or a stratified minibatch of
// the sorted training sample (stratum s of m covers ranks [s cnt / m, (s+1) cnt / m)).
struct ArrayIn {
  const float* x;
  const float* y;
  __device__ __forceinline__ bool get(uint32_t s, uint32_t m, float& xs, float& ys) const {
    if (s >= m) return false;
    xs = x[s];
    ys = y[s];
    return true;
  }
};

struct SampleIn {
  const uint64_t* train;
  const LearnedState* st;
  uint32_t step;
  uint64_t seed;
  __device__ __forceinline__ bool get(uint32_t s, uint32_t m, float& xs, float& ys) const {
    const uint32_t cnt = st->train_count;
    if (s >= m || cnt == 0) return false;
    const uint64_t r = mix64(seed ^ mix64((uint64_t(step) << 32) | s));
    const double u = double(r >> 11) * (1.0 / 9007199254740992.0);
    uint32_t idx = uint32_t((double(s) + u) * double(cnt) / double(m));
    if (idx >= cnt) idx = cnt - 1;
    xs = key_feature(train[idx], st->center, st->half);
    ys = (float(idx) + 0.5f) / float(cnt);
    return true;
  }
};

__global__ void mlp_adam_kernel(float* __restrict__ master, float* __restrict__ grads, float* __restrict__ m1,
                                float* __restrict__ m2, __nv_bfloat16* __restrict__ w, float lr, float beta1,
                                float beta2, float eps, float bias1, float bias2, LearnedState* st,
                                float* loss_log) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && st) {
    if (loss_log) loss_log[0] = st->loss;
    st->loss = 0.f;
  }
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

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = __float2bfloat16_rn(src[i]);
}

// ------------------------------------------------------ tensor-core MLP ----
// The 64-wide products of the MLP run on the tensor cores: mma.sync m16n8k16
// with BF16 operands and FP32 accumulation.  The weights are BF16 already.  An
// FP32 activation v enters as two BF16 parts, hi = bf16(v) and
// lo = bf16(v - hi): BF16 x BF16 products are exact in FP32, so a product
// taken with both parts keeps about 16 significant bits of v -- the FP32
// arithmetic of the definition (BF16 weights, FP32 sums) up to FP32 rounding.
//
// Fragment layouts of m16n8k16 for lane l = 4 g + t (two BF16 values per
// 32-bit register, the lower k index in the low half):
//   A (16 x 16, row-major)  a0 = A[g][2t, 2t+1]    a1 = A[g+8][2t, 2t+1]
//                            a2 = A[g][2t+8, 2t+9]  a3 = A[g+8][2t+8, 2t+9]
//   B (16 x 8, k-major)     b0 = B[2t, 2t+1][g]    b1 = B[2t+8, 2t+9][g]
//   C (16 x 8)              c0, c1 = C[g][2t, 2t+1]   c2, c3 = C[g+8][2t, 2t+1]
// The accumulators of two adjacent 8-column tiles are, row by row, the B
// fragment of the transposed matrix over one 16-wide k step; the backward pass
// feeds dL/da2 from its accumulators into the next product that way.
constexpr int kTcThreads = 128;  // 4 warps
constexpr int kTcTile = 64;      // samples per CTA step, 16 per warp
constexpr int kTcStride = 72;    // padded row (BF16) of the shared 64 x 64 matrices: conflict-free fragment loads

struct TcSmem {
  __nv_bfloat16 w2[kH * kTcStride];   // W2[j][i] at [j][i]
  __nv_bfloat16 w2t[kH * kTcStride];  // W2[j][i] at [i][j]
  __nv_bfloat16 d2h[kH * kTcStride];  // dL/da2 of the step's samples at [j][sample], high part
  __nv_bfloat16 d2l[kH * kTcStride];  // low part
  float w1[kH], b1[kH], b2[kH], w3[kH];
  float x[kTcTile], y[kTcTile], valid[kTcTile];
  float b3;
};

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) {
  uint32_t r;
  memcpy(&r, &v, 4);
  return r;
}

// (v0, v1) -> high parts and low parts, v0 in the low halves.
__device__ __forceinline__ void split2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
  const float2 hf = __bfloat1622float2(h);
  hi = bf16x2_bits(h);
  lo = bf16x2_bits(__floats2bfloat162_rn(v0 - hf.x, v1 - hf.y));
}

__device__ __forceinline__ uint32_t ld_bf16x2(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// The CTA's copy of the BF16 weights (W2 twice: as is and transposed).
__device__ __forceinline__ void tc_load_weights(const __nv_bfloat16* __restrict__ w, TcSmem& S) {
  for (int e = threadIdx.x; e < kH * kH; e += blockDim.x) {
    const int j = e / kH, i = e % kH;
    const __nv_bfloat16 v = w[Layout::W2 + e];
    S.w2[j * kTcStride + i] = v;
    S.w2t[i * kTcStride + j] = v;
  }
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    S.w1[i] = bf(w, Layout::W1 + i);
    S.b1[i] = bf(w, Layout::B1 + i);
    S.b2[i] = bf(w, Layout::B2 + i);
    S.w3[i] = bf(w, Layout::W3 + i);
  }
  if (threadIdx.x == 0) S.b3 = bf(w, Layout::B3);
}

// acc = the layer-2 products (without b2) of the warp's 16 inputs: x0 in row
// g, x1 in row g + 8; columns j = 8 nt + 2t (+1).
__device__ __forceinline__ void tc_layer2(const TcSmem& S, float x0, float x1, float (&acc)[8][4]) {
  const int l = threadIdx.x & 31, g = l >> 2, t = l & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const int i0 = 16 * kk + 2 * t;
    float h[2][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + (c & 1) + (c >> 1) * 8;
      h[0][c] = fmaxf(0.f, fmaf(S.w1[i], x0, S.b1[i]));
      h[1][c] = fmaxf(0.f, fmaf(S.w1[i], x1, S.b1[i]));
    }
    uint32_t ah[4], al[4];
    split2(h[0][0], h[0][1], ah[0], al[0]);
    split2(h[1][0], h[1][1], ah[1], al[1]);
    split2(h[0][2], h[0][3], ah[2], al[2]);
    split2(h[1][2], h[1][3], ah[3], al[3]);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const __nv_bfloat16* wr = S.w2 + (8 * nt + g) * kTcStride + i0;  // B[k = i][n = j] = W2[j][i]
      const uint32_t b0 = ld_bf16x2(wr), b1 = ld_bf16x2(wr + 8);
      mma_bf16(acc[nt], ah[0], ah[1], ah[2], ah[3], b0, b1);
      mma_bf16(acc[nt], al[0], al[1], al[2], al[3], b0, b1);
    }
  }
}

// z of rows g and g + 8 from the layer-2 products (every lane of the quad gets both).
__device__ __forceinline__ void tc_output(const TcSmem& S, const float (&acc)[8][4], float& z0, float& z1) {
  const int t = threadIdx.x & 3;
  z0 = z1 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int j = 8 * nt + 2 * t + e;
      z0 = fmaf(S.w3[j], fmaxf(0.f, acc[nt][e] + S.b2[j]), z0);
      z1 = fmaf(S.w3[j], fmaxf(0.f, acc[nt][2 + e] + S.b2[j]), z1);
    }
  z0 += __shfl_xor_sync(0xffffffffu, z0, 1);
  z1 += __shfl_xor_sync(0xffffffffu, z1, 1);
  z0 += __shfl_xor_sync(0xffffffffu, z0, 2);
  z1 += __shfl_xor_sync(0xffffffffu, z1, 2);
  z0 += S.b3;
  z1 += S.b3;
}

// grads (FP32) += d(loss)/d(params), loss += 1/(2m) sum (sigmoid(z) - y)^2
// over the m inputs.  Persistent CTAs walk steps of 64 samples; a warp runs
// the forward pass, dL/dz, dL/da2 and dL/da1 of its 16 samples, then each warp
// adds rows 16 w .. 16 w + 15 of dL/dW2 over all 64 samples.  Every gradient
// stays in registers over the CTA's steps; each CTA adds it to `grads` once.
template <typename In>
__global__ void __launch_bounds__(kTcThreads) mlp_grad_tc_kernel(const __nv_bfloat16* __restrict__ w, In in,
                                                                 uint32_t m, float* __restrict__ grads,
                                                                 float* __restrict__ loss) {
  __shared__ TcSmem S;
  tc_load_weights(w, S);
  const int warp = threadIdx.x >> 5, l = threadIdx.x & 31, g = l >> 2, t = l & 3;
  float gw2[8][4];        // dW2[j][i], j = 16 warp + g (+8), i = 8 nt + 2t (+1)
  float gw1[4][2], gb1[4][2];  // dW1, db1 at i = 16 mt + g (+8): this lane's samples
  float gb2[8][2], gw3[8][2];  // db2, dW3 at j = 8 nt + 2t + e: this lane's rows
  float gb3 = 0.f, lsum = 0.f;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    gw2[a][0] = gw2[a][1] = gw2[a][2] = gw2[a][3] = 0.f;
    gb2[a][0] = gb2[a][1] = gw3[a][0] = gw3[a][1] = 0.f;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) gw1[a][0] = gw1[a][1] = gb1[a][0] = gb1[a][1] = 0.f;
  const float inv_m = 1.f / float(m);
  const uint32_t steps = (m + kTcTile - 1) / kTcTile;
  for (uint32_t step = blockIdx.x; step < steps; step += gridDim.x) {
    __syncthreads();  // the weights, and the previous step's use of x and d2, are done
    if (threadIdx.x < kTcTile) {
      float xs = 0.f, ys = 0.f;
      const bool v = in.get(step * kTcTile + threadIdx.x, m, xs, ys);
      S.x[threadIdx.x] = v ? xs : 0.f;
      S.y[threadIdx.x] = v ? ys : 0.f;
      S.valid[threadIdx.x] = v ? 1.f : 0.f;
    }
    __syncthreads();
    // ---- the warp's 16 samples: forward, dL/dz, dL/da2
    const int r0 = 16 * warp + g, r1 = r0 + 8;
    const float x0 = S.x[r0], x1 = S.x[r1];
    float acc[8][4];
    tc_layer2(S, x0, x1, acc);
    float z0, z1;
    tc_output(S, acc, z0, z1);
    const float f0 = sigmoid(z0), f1 = sigmoid(z1);
    const float e0 = S.valid[r0] != 0.f ? f0 - S.y[r0] : 0.f;
    const float e1 = S.valid[r1] != 0.f ? f1 - S.y[r1] : 0.f;
    const float dz0 = e0 * f0 * (1.f - f0) * inv_m, dz1 = e1 * f1 * (1.f - f1) * inv_m;
    if (t == 0) {
      lsum += 0.5f * (e0 * e0 + e1 * e1) * inv_m;
      gb3 += dz0 + dz1;
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int j = 8 * nt + 2 * t + e;
        const float a0 = acc[nt][e] + S.b2[j], a1 = acc[nt][2 + e] + S.b2[j];
        gw3[nt][e] += fmaxf(0.f, a0) * dz0 + fmaxf(0.f, a1) * dz1;
        const float d0 = a0 > 0.f ? dz0 * S.w3[j] : 0.f, d1 = a1 > 0.f ? dz1 * S.w3[j] : 0.f;
        gb2[nt][e] += d0 + d1;
        acc[nt][e] = d0;  // acc now holds dL/da2
        acc[nt][2 + e] = d1;
        const __nv_bfloat16 h0 = __float2bfloat16_rn(d0), h1 = __float2bfloat16_rn(d1);
        S.d2h[j * kTcStride + r0] = h0;
        S.d2h[j * kTcStride + r1] = h1;
        S.d2l[j * kTcStride + r0] = __float2bfloat16_rn(d0 - __bfloat162float(h0));
        S.d2l[j * kTcStride + r1] = __float2bfloat16_rn(d1 - __bfloat162float(h1));
      }
    // ---- dL/da1, transposed: d1t[i][sample] = sum_j W2[j][i] dL/da2[sample][j],
    // rows i = 16 mt + g (+8), columns = the warp's samples 8 ns + 2t (+1)
    {
      float d1t[4][2][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) d1t[a][b][0] = d1t[a][b][1] = d1t[a][b][2] = d1t[a][b][3] = 0.f;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        uint32_t bh[2][2], bl[2][2];  // [ns][reg]: B[k = j][n = sample] from the accumulators
        split2(acc[2 * kk][0], acc[2 * kk][1], bh[0][0], bl[0][0]);
        split2(acc[2 * kk + 1][0], acc[2 * kk + 1][1], bh[0][1], bl[0][1]);
        split2(acc[2 * kk][2], acc[2 * kk][3], bh[1][0], bl[1][0]);
        split2(acc[2 * kk + 1][2], acc[2 * kk + 1][3], bh[1][1], bl[1][1]);
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
          const __nv_bfloat16* ar = S.w2t + (16 * mt + g) * kTcStride + 16 * kk + 2 * t;  // A[i][j] = W2[j][i]
          const uint32_t a0 = ld_bf16x2(ar), a1 = ld_bf16x2(ar + 8 * kTcStride);
          const uint32_t a2 = ld_bf16x2(ar + 8), a3 = ld_bf16x2(ar + 8 * kTcStride + 8);
#pragma unroll
          for (int ns = 0; ns < 2; ++ns) {
            mma_bf16(d1t[mt][ns], a0, a1, a2, a3, bh[ns][0], bh[ns][1]);
            mma_bf16(d1t[mt][ns], a0, a1, a2, a3, bl[ns][0], bl[ns][1]);
          }
        }
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int ns = 0; ns < 2; ++ns)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float xs = S.x[16 * warp + 8 * ns + 2 * t + e];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int i = 16 * mt + g + 8 * h;
              const float v = fmaf(S.w1[i], xs, S.b1[i]) > 0.f ? d1t[mt][ns][2 * h + e] : 0.f;
              gw1[mt][h] = fmaf(v, xs, gw1[mt][h]);
              gb1[mt][h] += v;
            }
          }
    }
    __syncthreads();  // every warp's dL/da2 is in shared memory
    // ---- dW2 rows 16 warp + g (+8): sum over the step's 64 samples of dL/da2[s][j] h1[s][i]
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int row = (16 * warp + g) * kTcStride + 16 * kk + 2 * t;
      const uint32_t ah0 = ld_bf16x2(S.d2h + row), ah1 = ld_bf16x2(S.d2h + row + 8 * kTcStride);
      const uint32_t ah2 = ld_bf16x2(S.d2h + row + 8), ah3 = ld_bf16x2(S.d2h + row + 8 * kTcStride + 8);
      const uint32_t al0 = ld_bf16x2(S.d2l + row), al1 = ld_bf16x2(S.d2l + row + 8 * kTcStride);
      const uint32_t al2 = ld_bf16x2(S.d2l + row + 8), al3 = ld_bf16x2(S.d2l + row + 8 * kTcStride + 8);
      const int s0 = 16 * kk + 2 * t;
      const float xa = S.x[s0], xb = S.x[s0 + 1], xc = S.x[s0 + 8], xd = S.x[s0 + 9];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int i = 8 * nt + g;
        const float wi = S.w1[i], bi = S.b1[i];
        uint32_t bh0, bl0, bh1, bl1;  // B[k = sample][n = i] = h1[sample][i]
        split2(fmaxf(0.f, fmaf(wi, xa, bi)), fmaxf(0.f, fmaf(wi, xb, bi)), bh0, bl0);
        split2(fmaxf(0.f, fmaf(wi, xc, bi)), fmaxf(0.f, fmaf(wi, xd, bi)), bh1, bl1);
        mma_bf16(gw2[nt], ah0, ah1, ah2, ah3, bh0, bh1);
        mma_bf16(gw2[nt], ah0, ah1, ah2, ah3, bl0, bl1);
        mma_bf16(gw2[nt], al0, al1, al2, al3, bh0, bh1);
      }
    }
  }
  // ---- one global addition per parameter per CTA (per warp for the per-warp sums)
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = 16 * warp + g + 8 * (c >> 1), i = 8 * nt + 2 * t + (c & 1);
      atomicAdd(&grads[Layout::W2 + j * kH + i], gw2[nt][c]);
    }
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float a = gw1[mt][h], b = gb1[mt][h];
      a += __shfl_xor_sync(0xffffffffu, a, 1);
      b += __shfl_xor_sync(0xffffffffu, b, 1);
      a += __shfl_xor_sync(0xffffffffu, a, 2);
      b += __shfl_xor_sync(0xffffffffu, b, 2);
      if (t == 0) {
        atomicAdd(&grads[Layout::W1 + 16 * mt + g + 8 * h], a);
        atomicAdd(&grads[Layout::B1 + 16 * mt + g + 8 * h], b);
      }
    }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float a = gb2[nt][e], b = gw3[nt][e];
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
      if (g == 0) {
        atomicAdd(&grads[Layout::B2 + 8 * nt + 2 * t + e], a);
        atomicAdd(&grads[Layout::W3 + 8 * nt + 2 * t + e], b);
      }
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  }
  if (l == 0) {
    atomicAdd(&grads[Layout::B3], gb3);
    if (loss) atomicAdd(loss, lsum);
  }
}

// sigmoid(mlp(x)) for m inputs (x from `in`, see XIn / CellIn), on the tensor cores.
struct XIn {
  const float* x;
  __device__ __forceinline__ bool get(uint32_t s, uint32_t m, float& xs) const {
    if (s >= m) return false;
    xs = x[s];
    return true;
  }
};

__device__ __forceinline__ uint64_t cell_start(uint32_t i);  // first key of grid cell i (below)

// The cell starts of the map's grid as inputs.
struct CellIn {
  const LearnedState* st;
  __device__ __forceinline__ bool get(uint32_t s, uint32_t m, float& xs) const {
    if (s >= m) return false;
    xs = key_feature(cell_start(s), st->center, st->half);
    return true;
  }
};

// kCells: outputs clamped to [0, 1] (NaN from a diverged model counts as 0)
// and out[m] = 1, the closing entry of the map's table.
template <typename In, bool kCells>
__global__ void __launch_bounds__(kTcThreads) mlp_eval_tc_kernel(const __nv_bfloat16* __restrict__ w, In in,
                                                                 uint32_t m, float* __restrict__ out) {
  __shared__ TcSmem S;
  tc_load_weights(w, S);
  if (kCells && blockIdx.x == 0 && threadIdx.x == 0) out[m] = 1.f;
  const int warp = threadIdx.x >> 5, l = threadIdx.x & 31, g = l >> 2, t = l & 3;
  const uint32_t steps = (m + kTcTile - 1) / kTcTile;
  for (uint32_t step = blockIdx.x; step < steps; step += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < kTcTile) {
      float xs = 0.f;
      S.x[threadIdx.x] = in.get(step * kTcTile + threadIdx.x, m, xs) ? xs : 0.f;
    }
    __syncthreads();
    const int r0 = 16 * warp + g, r1 = r0 + 8;
    float acc[8][4];
    tc_layer2(S, S.x[r0], S.x[r1], acc);
    float z0, z1;
    tc_output(S, acc, z0, z1);
    if (t == 0) {
      const uint32_t s0 = step * kTcTile + r0, s1 = step * kTcTile + r1;
      float v0 = sigmoid(z0), v1 = sigmoid(z1);
      if (kCells) {
        v0 = (v0 >= 0.f) ? fminf(v0, 1.f) : 0.f;
        v1 = (v1 >= 0.f) ? fminf(v1, 1.f) : 0.f;
      }
      if (s0 < m) out[s0] = v0;
      if (s1 < m) out[s1] = v1;
    }
  }
}

// ------------------------------------------------------------- sampling ----
// out[j] = keys[pos_j], pos_j uniform in [floor(j n / s), floor((j+1) n / s)).
__global__ void learn_sample_kernel(const uint64_t* __restrict__ keys, uint64_t n, uint32_t s, uint64_t seed,
                                    uint64_t* __restrict__ out) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  const uint64_t lo = uint64_t(j) * n / s, hi = uint64_t(j + 1) * n / s;
  out[j] = keys[lo + mix64(seed + j) % (hi - lo)];
}

// Heavy: a key with at least hmin copies in the sorted sample.
__global__ void learn_split_kernel(const uint64_t* __restrict__ sorted, uint32_t s, uint32_t hmin,
                                   uint32_t* __restrict__ flag_nh, uint32_t* __restrict__ flag_hv) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s) return;
  const uint64_t k = sorted[i];
  uint32_t lo = 0, hi = i;  // first index with sorted >= k
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (sorted[mid] < k) lo = mid + 1; else hi = mid;
  }
  const uint32_t first = lo;
  lo = i + 1;
  hi = s;  // first index with sorted > k
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (sorted[mid] <= k) lo = mid + 1; else hi = mid;
  }
  const bool heavy = lo - first >= hmin;
  flag_nh[i] = heavy ? 0u : 1u;
  flag_hv[i] = (heavy && i == first) ? 1u : 0u;
}

__global__ void learn_compact_kernel(const uint64_t* __restrict__ sorted, uint32_t s,
                                     const uint32_t* __restrict__ flag_nh, const uint32_t* __restrict__ pos_nh,
                                     const uint32_t* __restrict__ flag_hv, const uint32_t* __restrict__ pos_hv,
                                     uint64_t* __restrict__ train, uint64_t* __restrict__ heavy, LearnedState* st) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s) return;
  if (flag_nh[i]) train[pos_nh[i]] = sorted[i];
  if (flag_hv[i] && pos_hv[i] < uint32_t(kLearnMaxHeavy)) heavy[pos_hv[i]] = sorted[i];
  if (i + 1 == s) {
    st->train_count = pos_nh[i] + flag_nh[i];
    const uint32_t hv = pos_hv[i] + flag_hv[i];
    st->heavy_count = hv < uint32_t(kLearnMaxHeavy) ? hv : uint32_t(kLearnMaxHeavy);
    st->sample_count = s;
  }
}

__global__ void learn_norm_kernel(const uint64_t* __restrict__ train, LearnedState* st) {
  const uint32_t c = st->train_count;
  if (c == 0) {
    st->center = 0.f;
    st->half = 1.f;
    return;
  }
  const float lo = raw_feature(train[0]), hi = raw_feature(train[c - 1]);
  st->center = 0.5f * (lo + hi);
  st->half = fmaxf(0.5f * (hi - lo), 1e-4f);
  st->loss = 0.f;
}

// Data-dependent start: the kink of first-layer unit i (where W1_i x + b1_i
// = 0) moves to the feature of the training sample's quantile (i + 0.5) / 64,
// so the kinks are dense where the keys are.  Slopes keep their signs.
__global__ void learn_init_kinks_kernel(const uint64_t* __restrict__ train, const LearnedState* __restrict__ st,
                                        float* __restrict__ master) {
  const int i = threadIdx.x;
  const uint32_t cnt = st->train_count;
  if (i >= kH || cnt == 0) return;
  const uint32_t q = uint32_t((double(i) + 0.5) * double(cnt) / double(kH));
  const float kink = key_feature(train[q < cnt ? q : cnt - 1], st->center, st->half);
  master[Layout::B1 + i] = -master[Layout::W1 + i] * kink;
}

// ------------------------------------------------------------------ map ----
// Cell of a key on the grid with 11 significant bits: keys below 2048 are
// cells of their own; above, the cell is (exponent, next 10 bits), width
// 2^(e-10).  frac16 = position inside the cell in 1/65536 units.
__device__ __forceinline__ uint64_t cell_start(uint32_t i) {
  if (i < 2048u) return i;
  const uint32_t e = (i >> 10) + 9u;
  return uint64_t(1024u + (i & 1023u)) << (e - 10u);
}

// PLA(k): the tabulated CDF interpolated inside k's cell (u32 fixed point);
// hrange receives the cell's heavy range (H_i, H_{i+1}).
__device__ __forceinline__ uint32_t pla_of(uint64_t k, const uint2* __restrict__ cells, uint2& hrange) {
  uint32_t idx, frac;
  if (k < 2048ull) {
    idx = uint32_t(k);
    frac = 0;
  } else {
    const int e = 63 - __clzll(static_cast<long long>(k));
    const int sh = e - 10;
    idx = uint32_t(e - 9) * 1024u + uint32_t((k >> sh) & 1023u);
    const uint64_t rem = k & ((1ull << sh) - 1ull);
    frac = sh >= 16 ? uint32_t(rem >> (sh - 16)) : uint32_t(rem << (16 - sh));
  }
  const uint2 a = __ldg(&cells[idx]);
  const uint2 b = __ldg(&cells[idx + 1]);
  hrange = make_uint2(a.y, b.y);
  return a.x + uint32_t((uint64_t(b.x - a.x) * frac) >> 16);
}

__device__ __forceinline__ uint32_t map_id(uint64_t k, const LearnedMap& mp, bool& hit, uint32_t& t) {
  uint2 hr;
  const uint32_t f = pla_of(k, mp.cells, hr);
  uint32_t c = hr.x;
  hit = false;
  for (uint32_t j = hr.x; j < hr.y; ++j) {
    const uint64_t h = __ldg(&mp.heavy[j]);
    if (h < k) {
      ++c;
    } else {
      hit = (h == k);
      break;
    }
  }
  t = c;
  return (f >> mp.shift) + 2u * c + (hit ? 1u : 0u);
}

// One block: G_i = (1 - eps) max_{j <= i} F(x_j) + eps clamp((x_i + 1) / 2)
// quantised to u32 (non-decreasing, and rising at least with the floor
// wherever the model is flat or dips), and the count of heavy keys below
// every cell start.
constexpr int kCellThreads = 1024;
__global__ void __launch_bounds__(kCellThreads) learn_cells_finish_kernel(const float* __restrict__ fval,
                                                                          const uint64_t* __restrict__ heavy,
                                                                          const LearnedState* __restrict__ st,
                                                                          uint2* __restrict__ cells) {
  constexpr int kN = kLearnCells + 1;
  constexpr int kPer = (kN + kCellThreads - 1) / kCellThreads;
  __shared__ float s_w[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int b0 = t * kPer, b1 = min(b0 + kPer, kN);
  float mx = 0.f;
  for (int i = b0; i < b1; ++i) mx = fmaxf(mx, fval[i]);
  float inc = mx;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc = fmaxf(inc, y);
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    float v = s_w[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v = fmaxf(v, y);
    }
    s_w[lane] = v;
  }
  __syncthreads();
  float run = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) run = 0.f;
  if (warp > 0) run = fmaxf(run, s_w[warp - 1]);
  const uint32_t m = st->heavy_count;
  const float center = st->center, half = st->half;
  for (int i = b0; i < b1; ++i) {
    run = fmaxf(run, fval[i]);
    float v = 1.f;
    if (i < kLearnCells) {
      const float x = key_feature(cell_start(uint32_t(i)), center, half);
      v = (1.f - kLearnEps) * run + kLearnEps * fminf(fmaxf(0.5f * (x + 1.f), 0.f), 1.f);
    }
    uint32_t g = v >= 1.f ? 0xFFFFFFFFu : __float2uint_rz(v * 4294967296.0f);
    if (i == kLearnCells) g = 0xFFFFFFFFu;
    uint32_t hs = m;
    if (i < kLearnCells) {
      const uint64_t c = cell_start(uint32_t(i));
      uint32_t lo = 0, hi = m;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (heavy[mid] < c) lo = mid + 1; else hi = mid;
      }
      hs = lo;
    }
    cells[i] = make_uint2(g, hs);
  }
}

// Model-free map: fval[i] = the empirical CDF of the sorted training sample
// at cell start i (the fraction of its keys below the start), fval[kLearnCells]
// = 1.  Followed by the same table kernel as the model's map, it gives the
// partition the model would give if it matched its training sample exactly.
__global__ void learn_cells_ecdf_kernel(const uint64_t* __restrict__ train, const LearnedState* __restrict__ st,
                                        float* __restrict__ fval) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > uint32_t(kLearnCells)) return;
  if (i == uint32_t(kLearnCells)) {
    fval[i] = 1.f;
    return;
  }
  const uint32_t cnt = st->train_count;
  const uint64_t c = cell_start(i);
  uint32_t lo = 0, hi = cnt;  // first sample key >= c
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (train[mid] < c) lo = mid + 1; else hi = mid;
  }
  fval[i] = cnt ? float(double(lo) / double(cnt)) : 0.f;
}

// --------------------------------------------------------------- sorting ----
// Bucket id = (super-bucket s = id >> f, fine digit d = id & (2^f - 1)), f in 10..12.  Level 1
// groups the non-heavy keys by s into the scratch array: each CTA owns a fixed
// chunk of the input, counts its chunk per s, and after one flattened scan of
// the [s][chunk] counts (super-bucket major, so the scan is the position)
// scatters its chunk through shared-memory cursors.  Level 2 runs one CTA per
// super-bucket: count its keys per d, then (after the judge and a scan over
// all ids) scatter them to their final buckets, again through shared-memory
// cursors.  No per-key global atomic; every write front fits in L2.
constexpr int kFineBitsMin = 6, kFineBitsMax = 12;  // the fine digit's width is chosen per sort
constexpr int kFineMax = 1 << kFineBitsMax;
// most super-buckets: B = 2^22 at 10 fine bits, or up to 2^15 ids at 6 (both well below)
constexpr int kMaxSuper = ((1 << 22) + 2 * kLearnMaxHeavy + (1 << 10) - 1) >> 10;  // 4112
constexpr int kPartThreads = 512;
constexpr int kKeysPerLane = 8;  // keys a lane has in flight: independent table lookups hide latency

__global__ void learn_heavy_ids_kernel(LearnedMap mp, LearnedState* st, uint32_t* __restrict__ hid,
                                       uint32_t* __restrict__ bitmap) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    st->max_nonheavy = 0;
    st->large_heavy = 0;
  }
  if (t >= st->heavy_count) return;
  bool hit;
  uint32_t tt;
  const uint32_t id = map_id(mp.heavy[t], mp, hit, tt);
  hid[t] = id;
  atomicOr(&bitmap[id >> 5], 1u << (id & 31u));
}

// Walk keys[lo, hi) with kKeysPerLane keys per lane in flight; f(key, index, valid).
template <int kThreads, typename F>
__device__ __forceinline__ void for_keys(const uint64_t* __restrict__ keys, uint64_t lo, uint64_t hi, F f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr uint64_t kStep = uint64_t(kThreads) * kKeysPerLane;
  for (uint64_t base = lo + uint64_t(warp) * 32 * kKeysPerLane; base < hi; base += kStep) {
    uint64_t k[kKeysPerLane];
#pragma unroll
    for (int j = 0; j < kKeysPerLane; ++j) {
      const uint64_t i = base + j * 32 + lane;
      k[j] = i < hi ? keys[i] : 0;
    }
#pragma unroll
    for (int j = 0; j < kKeysPerLane; ++j) f(k[j], base + j * 32 + lane, base + j * 32 + lane < hi);
  }
}

// Level 1 count: counts1[s * nch + c] = non-heavy keys of chunk c in super-bucket s;
// hcount[t] += copies of heavy key t; ids[i] = the key's bucket id (kHeavyId
// for heavy keys) -- the only map lookup a key gets.
constexpr uint32_t kHeavyId = 0xFFFFFFFFu;
__global__ void __launch_bounds__(kPartThreads) learn_l1_count_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                                      uint64_t chunk, uint32_t nch, uint32_t nsuper,
                                                                      uint32_t fbits, LearnedMap mp,
                                                                      const LearnedState* __restrict__ st,
                                                                      uint32_t* __restrict__ counts1,
                                                                      uint32_t* __restrict__ hcount,
                                                                      uint32_t* __restrict__ ids, uint32_t heavy_cap) {
  // Shared memory sized to this sort (nsuper + heavy_cap words, heavy_cap the
  // host's count of heavy keys, at most kLearnMaxHeavy): the rest of the SM's
  // L1/shared capacity stays L1 cache for the map lookups.
  extern __shared__ uint32_t l1_smem[];
  const uint32_t m = min(st->heavy_count, heavy_cap);
  uint32_t* s_cnt = l1_smem;             // [nsuper]
  uint32_t* s_heavy = l1_smem + nsuper;  // [m]
  for (uint32_t i = threadIdx.x; i < nsuper + m; i += kPartThreads) l1_smem[i] = 0;
  __syncthreads();
  const uint32_t c = blockIdx.x;
  const uint64_t lo = uint64_t(c) * chunk, hi = lo + chunk < n ? lo + chunk : n;
  for_keys<kPartThreads>(keys, lo, hi, [&](uint64_t k, uint64_t i, bool valid) {
    bool hit = false;
    uint32_t t = 0;
    const uint32_t id = map_id(k, mp, hit, t);
    if (valid) {
      atomicAdd(hit ? &s_heavy[t < m ? t : 0u] : &s_cnt[id >> fbits], 1u);  // t < m whenever the host's count is right
      ids[i] = hit ? kHeavyId : id;
    }
  });
  __syncthreads();
  for (uint32_t s = threadIdx.x; s < nsuper; s += kPartThreads) counts1[uint64_t(s) * nch + c] = s_cnt[s];
  for (uint32_t t = threadIdx.x; t < m; t += kPartThreads)
    if (s_heavy[t]) atomicAdd(&hcount[t], s_heavy[t]);
}

constexpr int kL2Threads = 1024;

// Level 2 count: counts[s * 1024 + d] for super-bucket s = blockIdx.x, whose
// keys are alt[off1[s * nch], off1[(s + 1) * nch]) with fine digits fine[].
__global__ void __launch_bounds__(kL2Threads) learn_l2_count_kernel(const uint16_t* __restrict__ fine,
                                                                    const uint32_t* __restrict__ off1, uint32_t nch,
                                                                    uint32_t fbits, uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_cnt[kFineMax];
  const int nfine = 1 << fbits;
  for (int i = threadIdx.x; i < nfine; i += kL2Threads) s_cnt[i] = 0;
  __syncthreads();
  const uint32_t s = blockIdx.x;
  const uint64_t lo = off1[uint64_t(s) * nch], hi = off1[uint64_t(s + 1) * nch];
  for (uint64_t i = lo + threadIdx.x; i < hi; i += kL2Threads) atomicAdd(&s_cnt[fine[i]], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < nfine; d += kL2Threads) counts[(uint64_t(s) << fbits) + d] = s_cnt[d];
}

// counts[hid[t]] = hcount[t] (heavy ids hold no other key), then the judge:
// largest non-heavy bucket, and the list of heavy buckets filled by every CTA.
__global__ void learn_judge_kernel(uint32_t* __restrict__ counts, uint32_t nb, const uint32_t* __restrict__ bitmap,
                                   const uint32_t* __restrict__ hid, const uint32_t* __restrict__ hcount,
                                   LearnedState* st, uint32_t* __restrict__ large) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t v = 0;
  if (i < nb && !((bitmap[i >> 5] >> (i & 31u)) & 1u)) v = counts[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v) atomicMax(&st->max_nonheavy, v);
  if (i < st->heavy_count) {
    const uint32_t c = hcount[i];
    counts[hid[i]] = c;
    if (c > kFillSplit) large[atomicAdd(&st->large_heavy, 1u)] = i;
  }
}

// Staged scatter of one source range per CTA, tile by tile (8192 keys): each
// tile is counted per digit in shared memory (slot = the old count), staged
// grouped by digit, and written out in runs at the digit's global cursor, so
// consecutive threads write consecutive addresses.  Order inside a digit's run
// follows the shared-memory atomics (arbitrary; the bucket sorts fix it).  The
// next tile's keys are prefetched into shared memory (cp.async).
// No map lookup: the ids come from the level-1 count.
//   level 1: CTA = input chunk c; digit = id >> 10 (heavy keys skipped);
//            cursors from off1[s * nch + c]; keys to alt, fine digit id & 1023
//            to fine_out at the same position
//   level 2: CTA = super-bucket s, keys alt[off1[s nch], off1[(s+1) nch]) with
//            their fine digits; cursors from offsets[s * 1024 + d]; keys to dst
constexpr int kStThreads = 1024;
constexpr int kStIpt = 8;
constexpr int kStTile = kStThreads * kStIpt;
constexpr uint32_t kNoDigit = 0xFFFFu;
constexpr int kStPer = (kMaxSuper + kStThreads - 1) / kStThreads;  // digits a thread owns in the scan
static_assert(kStPer * kStThreads >= kFineMax, "the scan covers the widest fine digit");

// Shared-memory layout for a given digit capacity (bytes from the start).
struct StLayout {
  size_t stage, pre, dig, fine, cnt, cur, delta, warp, bytes;
  __host__ __device__ StLayout(int level, uint32_t cap) {
    stage = 0;
    pre = stage + size_t(kStTile) * 8;
    dig = pre + size_t(kStTile) * 8;
    fine = dig + size_t(kStTile) * 2;
    cnt = fine + (level == 1 ? size_t(kStTile) * 2 : 0);
    cur = cnt + size_t(cap) * 4;
    delta = cur + size_t(cap) * 4;
    warp = delta + size_t(cap) * 4;
    bytes = warp + 33 * 4;
  }
};

__device__ __forceinline__ void prefetch_tile(uint64_t* s_pre, const uint64_t* __restrict__ src, uint64_t base,
                                              uint64_t hi) {
  const uint32_t tn = uint32_t(hi - base < uint64_t(kStTile) ? hi - base : uint64_t(kStTile));
  for (uint32_t i = threadIdx.x; i < tn; i += kStThreads) cp_async8(&s_pre[i], &src[base + i]);
  cp_async_commit();
}

template <int kLevel>
__global__ void __launch_bounds__(kStThreads, 1) learn_staged_scatter_kernel(
    const uint64_t* __restrict__ src, const uint32_t* __restrict__ ids, const uint16_t* __restrict__ fine_in,
    uint64_t n, uint64_t chunk, uint32_t nch, uint32_t nsuper, uint32_t fbits, uint32_t cap,
    const uint32_t* __restrict__ off1,
    const uint32_t* __restrict__ offsets, uint64_t* __restrict__ dst, uint16_t* __restrict__ fine_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const StLayout L(kLevel, cap);
  uint64_t* s_stage = reinterpret_cast<uint64_t*>(smem + L.stage);
  uint64_t* s_pre = reinterpret_cast<uint64_t*>(smem + L.pre);
  uint16_t* s_dig = reinterpret_cast<uint16_t*>(smem + L.dig);
  uint16_t* s_fine = reinterpret_cast<uint16_t*>(smem + L.fine);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + L.cnt);
  uint32_t* s_cur = reinterpret_cast<uint32_t*>(smem + L.cur);
  uint32_t* s_delta = reinterpret_cast<uint32_t*>(smem + L.delta);
  uint32_t* s_warp = reinterpret_cast<uint32_t*>(smem + L.warp);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t ndig = kLevel == 1 ? nsuper : (1u << fbits);
  uint64_t lo, hi;
  if (kLevel == 1) {
    lo = uint64_t(blockIdx.x) * chunk;
    hi = lo + chunk < n ? lo + chunk : n;
  } else {
    lo = off1[uint64_t(blockIdx.x) * nch];
    hi = off1[uint64_t(blockIdx.x + 1) * nch];
  }
  if (lo < hi) prefetch_tile(s_pre, src, lo, hi);
  if (kLevel == 1) {
    for (uint32_t d = tid; d < ndig; d += kStThreads) s_cur[d] = off1[uint64_t(d) * nch + blockIdx.x];
  } else {
    for (uint32_t d = tid; d < ndig; d += kStThreads) s_cur[d] = offsets[(uint64_t(blockIdx.x) << fbits) + d];
  }
  for (uint32_t d = tid; d < ndig; d += kStThreads) s_cnt[d] = 0;
  for (uint64_t base = lo; base < hi; base += kStTile) {
    const uint32_t tn = uint32_t(hi - base < uint64_t(kStTile) ? hi - base : uint64_t(kStTile));
    uint32_t tag[kStIpt];  // the keys' ids (level 1) or fine digits (level 2), loaded while the prefetch lands
#pragma unroll
    for (int j = 0; j < kStIpt; ++j) {
      const uint32_t i = uint32_t(j * kStThreads + tid);
      tag[j] = i < tn ? (kLevel == 1 ? ids[base + i] : uint32_t(fine_in[base + i])) : 0u;
    }
    cp_async_wait_all();
    __syncthreads();
    uint64_t k[kStIpt];
    uint32_t ds[kStIpt];  // digit << 16 | slot inside the tile's digit run
    uint32_t fn[kStIpt];  // level 1: the fine digit travelling with the key
#pragma unroll
    for (int j = 0; j < kStIpt; ++j) {
      const uint32_t i = uint32_t(j * kStThreads + tid);
      k[j] = i < tn ? s_pre[i] : 0;
      uint32_t d = kNoDigit;
      fn[j] = 0;
      if (i < tn) {
        if (kLevel == 1) {
          if (tag[j] != kHeavyId) {
            d = tag[j] >> fbits;
            fn[j] = tag[j] & ((1u << fbits) - 1u);
          }
        } else {
          d = tag[j];
        }
      }
      ds[j] = d << 16;
    }
    __syncthreads();  // the prefetch buffers are free again
    if (base + kStTile < hi) prefetch_tile(s_pre, src, base + kStTile, hi);
#pragma unroll
    for (int j = 0; j < kStIpt; ++j)
      if ((ds[j] >> 16) != kNoDigit) ds[j] |= atomicAdd(&s_cnt[ds[j] >> 16], 1u);
    __syncthreads();
    // exclusive scan of the tile's digit counts (thread t owns digits t*kStPer ...)
    uint32_t own[kStPer], sum = 0;
#pragma unroll
    for (int q = 0; q < kStPer; ++q) {
      const uint32_t d = uint32_t(tid * kStPer + q);
      own[q] = d < ndig ? s_cnt[d] : 0u;
      sum += own[q];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {  // exclusive prefix of the warp totals; the total after them
      static_assert(kStThreads == 1024, "one warp total per lane");
      const uint32_t x = s_warp[lane];
      uint32_t y = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += z;
      }
      s_warp[lane] = y - x;
      if (lane == 31) s_warp[32] = y;
    }
    __syncthreads();
    uint32_t run = inc - sum + s_warp[warp];
    const uint32_t total = s_warp[32];
#pragma unroll
    for (int q = 0; q < kStPer; ++q) {
      const uint32_t d = uint32_t(tid * kStPer + q);
      if (d < ndig) {
        s_cnt[d] = run;  // the tile offset of digit d, for the staging below
        const uint32_t cur = s_cur[d];
        s_delta[d] = cur - run;
        s_cur[d] = cur + own[q];
      }
      run += own[q];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kStIpt; ++j) {
      const uint32_t d = ds[j] >> 16;
      if (d != kNoDigit) {
        const uint32_t p = s_cnt[d] + (ds[j] & 0xFFFFu);
        s_stage[p] = k[j];
        s_dig[p] = uint16_t(d);
        if (kLevel == 1) s_fine[p] = uint16_t(fn[j]);
      }
    }
    __syncthreads();
    for (uint32_t i = tid; i < total; i += kStThreads) {
      const uint32_t pos = s_delta[s_dig[i]] + i;
      dst[pos] = s_stage[i];
      if (kLevel == 1) fine_out[pos] = s_fine[i];
    }
    for (uint32_t d = tid; d < ndig; d += kStThreads) s_cnt[d] = 0;
  }
  cp_async_wait_all();
}

__global__ void __launch_bounds__(256) learn_fill_kernel(LearnedMap mp, const LearnedState* __restrict__ st,
                                                         const uint32_t* __restrict__ hid,
                                                         const uint32_t* __restrict__ large,
                                                         const uint32_t* __restrict__ offsets,
                                                         const uint32_t* __restrict__ counts,
                                                         uint64_t* __restrict__ dst) {
  const uint32_t m = st->heavy_count, nl = st->large_heavy;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t t = gw; t < m; t += nw) {  // one warp per heavy bucket of at most kFillSplit keys
    const uint32_t id = hid[t], c = counts[id];
    if (c > kFillSplit) continue;
    const uint64_t h = mp.heavy[t];
    uint64_t* o = dst + offsets[id];
    for (uint32_t j = lane; j < c; j += 32) o[j] = h;
  }
  for (uint32_t q = 0; q < nl; ++q) {  // every CTA a slice of each larger one
    const uint32_t t = large[q], id = hid[t], c = counts[id];
    const uint64_t h = mp.heavy[t];
    uint64_t* o = dst + offsets[id];
    const uint32_t lo = uint32_t(uint64_t(c) * blockIdx.x / gridDim.x);
    const uint32_t hi = uint32_t(uint64_t(c) * (blockIdx.x + 1) / gridDim.x);
    for (uint32_t j = lo + threadIdx.x; j < hi; j += blockDim.x) o[j] = h;
  }
}

// On-chip sort of the buckets, one unit per CTA iteration, in place.  A unit
// is a run of consecutive non-heavy buckets with at most 4096 keys in all
// (contiguous in memory), sorted by a 512-thread CTA (two per SM), or one
// bucket of 4097 to 8192 keys, sorted by a 1024-thread CTA.  A unit of
// capacity 2^c is split into at most 2^c sub-buckets by the top c bits of
// key - min in one counting pass through shared memory (16-bit counters, two
// to a word: no count or offset exceeds the capacity); a key of a sub-bucket
// of at most 16 keys finds its place by counting the smaller keys there, and
// the larger sub-buckets (in practice a moderately frequent key among a few
// others) are split again by warps.  The next unit's keys are prefetched into
// shared memory (cp.async) while one is sorted.  A unit whose large ranges
// overflow the round list is finished by a bitonic network instead.
template <int kThreadsT, int kCapBits>
struct BsGeom {
  static constexpr int kThreads = kThreadsT;
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kCap = 1 << kCapBits;       // keys of a unit
  static constexpr int kIpt = kCap / kThreads;     // keys per thread
  static constexpr int kSubBits = kCapBits;        // as many sub-buckets as keys
  static constexpr int kSub = 1 << kSubBits;
  static constexpr int kSubPerThread = kSub / kThreads;
  static constexpr uint32_t kMaxBig = kCap / 16;   // large ranges a round holds (more: the bitonic sort)
  static constexpr int kBytes = 3 * kCap * 8;      // dynamic shared memory: the unit, two prefetch buffers
  static constexpr int kMinBlocks = kThreads <= 512 ? 2 : 1;  // resident CTAs per SM (64 registers a thread)
  static_assert(kSub % kThreads == 0 && kSubPerThread == 8, "sub-bucket ownership: four words per thread");
  static_assert(kSub <= 65535 && kCap <= 65535, "16-bit sub-bucket counters and offsets");
  static_assert(kWarps <= 32, "one warp partial per lane");
};
using BsNarrow = BsGeom<512, 12>;  // units of up to 4096 keys, two CTAs per SM
using BsWide = BsGeom<1024, 13>;   // single buckets of up to 8192 keys
static_assert(BsWide::kCap == kLearnBucketCap, "the wide sort takes any bucket the judge accepts");
constexpr int kGroup = 32;  // ids one unit-list thread packs

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

constexpr uint32_t kBigSub = 16;     // larger ranges are split by a warp
constexpr int kSplitBits = 5;        // a warp splits a range into 32 bins
constexpr int kMaxRounds = (64 + kSplitBits - 1) / kSplitBits;  // each round drops 5 bits of key range

template <class G>
struct BsShared {
  uint2 big[2][G::kMaxBig];        // [lo, hi) ranges of more than kBigSub keys: this round's, the next
  uint32_t nbig[2];
  uint32_t bins[G::kWarps][32];    // per-warp bin counters of the split
  __align__(16) uint32_t sub[G::kSub / 2 + 4];  // 16-bit counters, then offsets; entry kSub = the unit's size (uint4-aligned clears)
  uint64_t red[2 * G::kWarps];     // per-warp key min / max
  uint32_t warp_sum[G::kWarps];    // per-warp totals of the sub-bucket counts
  uint32_t flag;
};

// Sorts one unit whose keys the threads hold (key j of thread t is element
// j * G::kThreads + t) into g[0, cnt), 2 <= cnt <= G::kCap; every thread
// calls it.
template <class G>
__device__ void sort_unit(const uint64_t (&k)[G::kIpt], uint64_t* __restrict__ g, uint32_t cnt,
                          uint64_t* __restrict__ s_out, uint64_t* __restrict__ s_tmp, BsShared<G>& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint16_t* sub16 = reinterpret_cast<const uint16_t*>(sh.sub);  // the offsets, after the scan
  uint32_t v[G::kIpt];  // sub-bucket << 16 | slot
  uint64_t kmn = ~0ull, kmx = 0;
#pragma unroll
  for (int j = 0; j < G::kIpt; ++j) {
    const uint32_t i = uint32_t(j * G::kThreads + tid);
    if (i < cnt) {
      kmn = umin64(kmn, k[j]);
      kmx = umax64(kmx, k[j]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kmn = umin64(kmn, __shfl_xor_sync(0xffffffffu, kmn, o));
    kmx = umax64(kmx, __shfl_xor_sync(0xffffffffu, kmx, o));
  }
  if (lane == 0) {
    sh.red[warp] = kmn;
    sh.red[G::kWarps + warp] = kmx;
  }
  if (tid == 0) {
    sh.flag = 0;
    sh.nbig[0] = sh.nbig[1] = 0;
  }
  __syncthreads();
  {  // every warp folds the per-warp partials itself: no second barrier
    kmn = lane < G::kWarps ? sh.red[lane] : ~0ull;
    kmx = lane < G::kWarps ? sh.red[G::kWarps + lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kmn = umin64(kmn, __shfl_xor_sync(0xffffffffu, kmn, o));
      kmx = umax64(kmx, __shfl_xor_sync(0xffffffffu, kmx, o));
    }
  }
  const uint64_t krange = kmx - kmn;
  if (krange == 0) {  // all keys equal: already in order
    for (uint32_t i = tid; i < cnt; i += G::kThreads) g[i] = kmn;
    return;
  }
  // sub-bucket = the top kSubBits bits of key - min: the map is near-linear inside
  // a unit, so the keys spread about evenly over the sub-buckets, except for
  // runs of one key, which the warp split below takes apart cheaply
  const int bits = 64 - __clzll(static_cast<long long>(krange));
  const int shf = bits > G::kSubBits ? bits - G::kSubBits : 0;
#pragma unroll
  for (int j = 0; j < G::kIpt; ++j) {
    const uint32_t i = uint32_t(j * G::kThreads + tid);
    if (i < cnt) {
      const uint32_t sb = uint32_t((k[j] - kmn) >> shf);
      const uint32_t half = (sb & 1u) * 16u;
      v[j] = (sb << 16) | ((atomicAdd(&sh.sub[sb >> 1], 1u << half) >> half) & 0xFFFFu);
    }
  }
  __syncthreads();
  uint32_t own[G::kSubPerThread], sum = 0;
  {
    const uint4 w = reinterpret_cast<const uint4*>(sh.sub)[tid];
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      own[2 * q] = ws[q] & 0xFFFFu;
      own[2 * q + 1] = ws[q] >> 16;
    }
  }
#pragma unroll
  for (int q = 0; q < G::kSubPerThread; ++q) sum += own[q];
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh.warp_sum[warp] = inc;
  __syncthreads();
  uint32_t before;
  {  // every warp scans the warp totals itself: no second barrier
    uint32_t y = lane < G::kWarps ? sh.warp_sum[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    before = __shfl_sync(0xffffffffu, y, warp > 0 ? warp - 1 : 0);
    if (warp == 0) before = 0;
  }
  uint32_t run = inc - sum + before;
  {
    uint32_t ws[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ws[q] = run | ((run + own[2 * q]) << 16);
      run += own[2 * q] + own[2 * q + 1];
    }
    reinterpret_cast<uint4*>(sh.sub)[tid] = make_uint4(ws[0], ws[1], ws[2], ws[3]);
  }
  if (tid == G::kThreads - 1) sh.sub[G::kSub / 2] = cnt;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < G::kIpt; ++j) {
    const uint32_t i = uint32_t(j * G::kThreads + tid);
    if (i < cnt) s_tmp[sub16[v[j] >> 16] + (v[j] & 0xFFFFu)] = k[j];
  }
#pragma unroll
  for (int q = 0; q < G::kSubPerThread; ++q) {  // sub-buckets above kBigSub keys go to the warp split below
    const int sb = tid * G::kSubPerThread + q;
    const uint32_t lo = sub16[sb], hi = sub16[sb + 1];
    if (hi - lo > kBigSub) {
      const uint32_t at = atomicAdd(&sh.nbig[0], 1u);
      if (at < G::kMaxBig) sh.big[0][at] = make_uint2(lo, hi); else sh.flag = 1;
    }
  }
  __syncthreads();
  // the key at position p of a small sub-bucket [lo, hi) goes to lo + the
  // keys there below it + the equal keys before p: independent loads, and
  // the lanes of a warp take consecutive positions, so they mostly read the
  // same words
  for (uint32_t p = uint32_t(tid); p < cnt; p += G::kThreads) {
    const uint64_t key = s_tmp[p];
    const uint32_t sb = uint32_t((key - kmn) >> shf);
    const uint32_t lo = sub16[sb], hi = sub16[sb + 1];
    if (hi - lo > kBigSub) {
      s_out[p] = key;
      continue;
    }
    uint32_t rank = 0;
    for (uint32_t q = lo; q < hi; ++q) {
      const uint64_t y = s_tmp[q];
      rank += (y < key || (y == key && q < p)) ? 1u : 0u;
    }
    s_out[lo + rank] = key;
  }
  __syncthreads();
  // large ranges (mostly a moderately frequent key among a few others), a
  // warp each, in rounds: nothing to do when the keys are all equal; else
  // split into 32 bins by 5 bits of key - min below the range's top bit,
  // lanes insertion-sort the bins of at most kBigSub keys and the larger ones
  // go to the next round with 5 fewer bits of range
  for (int r = 0; r < kMaxRounds; ++r) {
    const int cur = r & 1;
    const uint32_t nr = sh.nbig[cur];
    if (sh.flag || nr == 0) break;
    uint32_t* wb = sh.bins[warp];
    for (uint32_t b = uint32_t(warp); b < nr; b += G::kWarps) {
      const uint2 rg = sh.big[cur][b];
      uint64_t mn = ~0ull, mx = 0;
      for (uint32_t i = rg.x + lane; i < rg.y; i += 32) {
        mn = umin64(mn, s_out[i]);
        mx = umax64(mx, s_out[i]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mn = umin64(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = umax64(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      }
      if (mn == mx) continue;
      const int bits = 64 - __clzll(static_cast<long long>(mx - mn));
      const int shf = bits > kSplitBits ? bits - kSplitBits : 0;
      wb[lane] = 0;
      __syncwarp();
      for (uint32_t i = rg.x + lane; i < rg.y; i += 32) atomicAdd(&wb[uint32_t((s_out[i] - mn) >> shf)], 1u);
      __syncwarp();
      const uint32_t c = wb[lane];
      uint32_t start = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, start, o);
        if (lane >= o) start += y;
      }
      start = rg.x + start - c;
      wb[lane] = start;
      __syncwarp();
      for (uint32_t i = rg.x + lane; i < rg.y; i += 32) {
        const uint64_t key = s_out[i];
        s_tmp[atomicAdd(&wb[uint32_t((key - mn) >> shf)], 1u)] = key;
      }
      __syncwarp();
      for (uint32_t i = rg.x + lane; i < rg.y; i += 32) s_out[i] = s_tmp[i];
      __syncwarp();
      if (c > kBigSub) {
        const uint32_t at = atomicAdd(&sh.nbig[cur ^ 1], 1u);
        if (at < G::kMaxBig) sh.big[cur ^ 1][at] = make_uint2(start, start + c); else sh.flag = 1;
      } else {
        for (uint32_t x = start + 1; x < start + c; ++x) {
          const uint64_t key = s_out[x];
          uint32_t y = x;
          while (y > start && s_out[y - 1] > key) {
            s_out[y] = s_out[y - 1];
            --y;
          }
          s_out[y] = key;
        }
      }
      __syncwarp();
    }
    __syncthreads();
    if (tid == 0) sh.nbig[cur] = 0;
    __syncthreads();
    if (r == kMaxRounds - 1 && sh.nbig[cur ^ 1] != 0) sh.flag = 1;  // cannot happen: 13 rounds use up 64 bits
  }
  __syncthreads();
  if (sh.flag) {  // bitonic network over the next power of two, padded with the largest key
    uint32_t p2 = 2;
    while (p2 < cnt) p2 <<= 1;
    for (uint32_t i = cnt + tid; i < p2; i += G::kThreads) s_out[i] = ~0ull;
    __syncthreads();
    for (uint32_t size = 2; size <= p2; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t i = tid; i < p2 / 2; i += G::kThreads) {
          const uint32_t a = 2 * i - (i & (stride - 1)), c = a + stride;
          const bool up = (a & size) == 0;
          const uint64_t x = s_out[a], y = s_out[c];
          if ((x > y) == up) {
            s_out[a] = y;
            s_out[c] = x;
          }
        }
        __syncthreads();
      }
    }
  }
  for (uint32_t i = tid; i < cnt; i += G::kThreads) g[i] = s_out[i];
  for (int i = tid; i < G::kSub / 2 + 4; i += G::kThreads) sh.sub[i] = 0;
}

// The unit lists (order arbitrary).  units[1 .. units[0].x] are the narrow
// units: each thread walks kGroup consecutive ids and packs runs of
// non-heavy buckets into units of at most BsNarrow::kCap keys (contiguous in
// memory); heavy ids end a unit.  A bucket above that capacity is a wide unit
// of its own, units[nb], units[nb - 1], ... (units[0].y of them).  Every unit
// holds a bucket with two or more keys that no other unit holds, so the two
// lists stay within units[1 .. nb] without meeting.
__global__ void learn_units_kernel(const uint32_t* __restrict__ counts, const uint32_t* __restrict__ offsets,
                                   const uint32_t* __restrict__ bitmap, uint32_t nb, uint2* __restrict__ units,
                                   uint32_t* status) {
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi * kGroup >= nb) return;
  uint32_t* narrow = &units[0].x;
  uint32_t* wide = &units[0].y;
  uint32_t start = 0, tot = 0;
  auto close = [&]() {
    if (tot >= 2) units[1 + atomicAdd(narrow, 1u)] = make_uint2(start, tot);
    tot = 0;
  };
  for (uint32_t id = gi * kGroup; id < nb && id < (gi + 1) * kGroup; ++id) {
    if ((bitmap[id >> 5] >> (id & 31u)) & 1u) {  // heavy: filled elsewhere, never sorted
      close();
      continue;
    }
    const uint32_t c = counts[id];
    if (c > uint32_t(BsWide::kCap)) {  // the judge rejects such maps; never sort past capacity
      atomicOr(status, kDevBadBucket);
      close();
      continue;
    }
    if (c > uint32_t(BsNarrow::kCap)) {
      close();
      units[nb - atomicAdd(wide, 1u)] = make_uint2(offsets[id], c);
      continue;
    }
    if (tot + c > uint32_t(BsNarrow::kCap)) close();
    if (tot == 0) start = offsets[id];
    tot += c;
  }
  close();
}

// Unit u of a list is list[step * u] (step +1: the narrow list from its
// start, -1: the wide list from its end); *count units in all.
template <class G>
__global__ void __launch_bounds__(G::kThreads, G::kMinBlocks)
    learn_bucket_sort_kernel(uint64_t* __restrict__ keys, const uint2* __restrict__ list, int step,
                             const uint32_t* __restrict__ count) {
  extern __shared__ uint64_t s_dyn[];  // [3][G::kCap]: the unit, two prefetch buffers
  uint64_t* s_out = s_dyn;
  __shared__ BsShared<G> sh;
  const int tid = threadIdx.x;
  const uint32_t nunits = *count;
  for (int i = tid; i < G::kSub / 2 + 4; i += G::kThreads) sh.sub[i] = 0;
  auto at = [&](uint32_t u) { return list[ptrdiff_t(step) * ptrdiff_t(u)]; };
  auto prefetch = [&](uint2 x, int buf) {
    uint64_t* dst = s_dyn + (1 + buf) * G::kCap;
    for (uint32_t i = tid; i < x.y; i += G::kThreads) cp_async8(&dst[i], &keys[x.x + i]);
    cp_async_commit();
  };
  uint32_t u = blockIdx.x;
  uint2 cur = make_uint2(0, 0);
  int buf = 0;
  if (u < nunits) {
    cur = at(u);
    prefetch(cur, 0);
  }
  while (u < nunits) {
    const uint32_t nx = u + gridDim.x;
    const uint2 next = nx < nunits ? at(nx) : make_uint2(0, 0);
    cp_async_wait_all();
    __syncthreads();
    const uint64_t* s_pre = s_dyn + (1 + buf) * G::kCap;
    uint64_t k[G::kIpt];
#pragma unroll
    for (int j = 0; j < G::kIpt; ++j) {
      const uint32_t i = uint32_t(j * G::kThreads + tid);
      k[j] = i < cur.y ? s_pre[i] : 0;
    }
    // the other buffer was read in the previous iteration, before the barrier above
    if (nx < nunits) prefetch(next, buf ^ 1);
    // this unit's prefetch buffer is consumed (the keys are in registers): it is the scratch
    sort_unit<G>(k, keys + cur.x, cur.y, s_out, s_dyn + (1 + buf) * G::kCap, sh);
    u = nx;
    cur = next;
    buf ^= 1;
  }
  cp_async_wait_all();
}

__global__ void learn_bucket_ids_kernel(const uint64_t* __restrict__ keys, uint64_t n, LearnedMap mp,
                                        uint32_t* __restrict__ ids) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    bool hit;
    uint32_t t;
    ids[i] = map_id(keys[i], mp, hit, t);
  }
}

// ------------------------------------------------------------------ scan ----
constexpr int kScanThreads = 1024;
constexpr int kScanIpt = 4;
constexpr uint64_t kScanTile = uint64_t(kScanThreads) * kScanIpt;

// Exclusive scan over the block of v; total receives the block sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_w, uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t x = s_w[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_w[lane] = x;
  }
  __syncthreads();
  total = s_w[31];
  return (warp ? s_w[warp - 1] : 0u) + inc - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t* __restrict__ in, uint64_t count,
                                                                   uint32_t* __restrict__ sums) {
  __shared__ uint32_t s_w[32];
  const uint64_t at = blockIdx.x * kScanTile + uint64_t(threadIdx.x) * kScanIpt;
  uint32_t v = 0;
#pragma unroll
  for (int j = 0; j < kScanIpt; ++j)
    if (at + j < count) v += in[at + j];
  uint32_t total;
  block_excl_scan(v, s_w, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Exclusive scan of the block sums in place, kScanTile at a time with a
// running carry; sums[nblocks] receives the grand total.
__global__ void __launch_bounds__(kScanThreads) scan_top_kernel(uint32_t* __restrict__ sums, uint32_t nblocks) {
  __shared__ uint32_t s_w[32];
  uint32_t carry = 0;
  for (uint32_t base = 0; base < nblocks; base += uint32_t(kScanTile)) {
    const uint32_t at = base + threadIdx.x * kScanIpt;
    uint32_t x[kScanIpt], v = 0;
#pragma unroll
    for (int j = 0; j < kScanIpt; ++j) {
      x[j] = (at + j < nblocks) ? sums[at + j] : 0u;
      v += x[j];
    }
    uint32_t total;
    uint32_t run = carry + block_excl_scan(v, s_w, total);
#pragma unroll
    for (int j = 0; j < kScanIpt; ++j) {
      if (at + j < nblocks) sums[at + j] = run;
      run += x[j];
    }
    carry += total;
    __syncthreads();  // s_w is reused by the next segment's scan
  }
  if (threadIdx.x == 0) sums[nblocks] = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t* __restrict__ in, uint64_t count,
                                                                  const uint32_t* __restrict__ sums,
                                                                  uint32_t* __restrict__ out,
                                                                  uint32_t* __restrict__ out2) {
  __shared__ uint32_t s_w[32];
  const uint64_t at = blockIdx.x * kScanTile + uint64_t(threadIdx.x) * kScanIpt;
  uint32_t x[kScanIpt], v = 0;
#pragma unroll
  for (int j = 0; j < kScanIpt; ++j) {
    x[j] = (at + j < count) ? in[at + j] : 0u;
    v += x[j];
  }
  uint32_t total;
  uint32_t run = sums[blockIdx.x] + block_excl_scan(v, s_w, total);
#pragma unroll
  for (int j = 0; j < kScanIpt; ++j) {
    if (at + j < count) {
      out[at + j] = run;
      if (out2) out2[at + j] = run;
    }
    run += x[j];
  }
}

unsigned grid_for(uint64_t n, int threads) { return unsigned((n + threads - 1) / threads); }

}  // namespace

// -------------------------------------------------------------- launchers ----
// Persistent CTAs for the tensor-core MLP kernels: one per SM at most.
unsigned tc_grid(uint32_t m) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 1;
  const uint32_t steps = (m + kTcTile - 1) / kTcTile;
  return steps < uint32_t(sms) ? steps : uint32_t(sms);
}

cudaError_t launch_mlp_grad(const void* w_bf16, const float* x, const float* y, uint32_t m, float* grads, float* loss,
                            cudaStream_t stream) {
  if (!m) return cudaSuccess;
  mlp_grad_tc_kernel<ArrayIn><<<tc_grid(m), kTcThreads, 0, stream>>>(static_cast<const __nv_bfloat16*>(w_bf16),
                                                                      ArrayIn{x, y}, m, grads, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad_sample(const void* w_bf16, const uint64_t* train, const LearnedState* st, uint32_t m,
                                   uint32_t step, uint64_t seed, float* grads, cudaStream_t stream) {
  if (!m) return cudaSuccess;
  float* loss = const_cast<float*>(&st->loss);
  mlp_grad_tc_kernel<SampleIn><<<tc_grid(m), kTcThreads, 0, stream>>>(
      static_cast<const __nv_bfloat16*>(w_bf16), SampleIn{train, st, step, seed}, m, grads, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* master, float* grads, float* m1, float* m2, void* w_bf16, float lr, int step,
                            LearnedState* st, float* loss_log, cudaStream_t stream) {
  const float beta1 = 0.9f, beta2 = 0.999f;
  float b1 = 1.f, b2 = 1.f;
  for (int i = 0; i < step; ++i) {
    b1 *= beta1;
    b2 *= beta2;
  }
  mlp_adam_kernel<<<grid_for(kMlpParams, 256), 256, 0, stream>>>(master, grads, m1, m2,
                                                                 static_cast<__nv_bfloat16*>(w_bf16), lr, beta1, beta2,
                                                                 1e-8f, 1.f - b1, 1.f - b2, st, loss_log);
  return cudaGetLastError();
}

cudaError_t launch_mlp_eval(const void* w_bf16, const float* x, uint32_t m, float* out, cudaStream_t stream) {
  if (!m) return cudaSuccess;
  mlp_eval_tc_kernel<XIn, false><<<tc_grid(m), kTcThreads, 0, stream>>>(static_cast<const __nv_bfloat16*>(w_bf16),
                                                                          XIn{x}, m, out);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* src, void* dst, int count, cudaStream_t stream) {
  to_bf16_kernel<<<grid_for(uint64_t(count), 256), 256, 0, stream>>>(src, static_cast<__nv_bfloat16*>(dst), count);
  return cudaGetLastError();
}

cudaError_t launch_learn_sample(const uint64_t* keys, uint64_t n, uint32_t s, uint64_t seed, uint64_t* out,
                                cudaStream_t stream) {
  if (!s || n < s) return cudaErrorInvalidValue;
  learn_sample_kernel<<<grid_for(s, 256), 256, 0, stream>>>(keys, n, s, seed, out);
  return cudaGetLastError();
}

cudaError_t launch_learn_split(const uint64_t* sorted, uint32_t s, uint32_t hmin, uint32_t* flag_nh,
                               uint32_t* flag_hv, cudaStream_t stream) {
  if (!s) return cudaSuccess;
  learn_split_kernel<<<grid_for(s, 256), 256, 0, stream>>>(sorted, s, hmin, flag_nh, flag_hv);
  return cudaGetLastError();
}

cudaError_t launch_learn_compact(const uint64_t* sorted, uint32_t s, const uint32_t* flag_nh, const uint32_t* pos_nh,
                                 const uint32_t* flag_hv, const uint32_t* pos_hv, uint64_t* train, uint64_t* heavy,
                                 LearnedState* st, cudaStream_t stream) {
  if (!s) return cudaErrorInvalidValue;
  learn_compact_kernel<<<grid_for(s, 256), 256, 0, stream>>>(sorted, s, flag_nh, pos_nh, flag_hv, pos_hv, train,
                                                             heavy, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  learn_norm_kernel<<<1, 1, 0, stream>>>(train, st);
  return cudaGetLastError();
}

cudaError_t launch_learn_init_kinks(const uint64_t* train, const LearnedState* st, float* master,
                                    cudaStream_t stream) {
  learn_init_kinks_kernel<<<1, kH, 0, stream>>>(train, st, master);
  return cudaGetLastError();
}

cudaError_t launch_learn_cells(const void* w_bf16, LearnedState* st, const uint64_t* heavy, float* fval, uint2* cells,
                               cudaStream_t stream) {
  mlp_eval_tc_kernel<CellIn, true><<<tc_grid(kLearnCells), kTcThreads, 0, stream>>>(
      static_cast<const __nv_bfloat16*>(w_bf16), CellIn{st}, uint32_t(kLearnCells), fval);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  learn_cells_finish_kernel<<<1, kCellThreads, 0, stream>>>(fval, heavy, st, cells);
  return cudaGetLastError();
}

cudaError_t launch_learn_cells_ecdf(const uint64_t* train, LearnedState* st, const uint64_t* heavy, float* fval,
                                    uint2* cells, cudaStream_t stream) {
  learn_cells_ecdf_kernel<<<grid_for(kLearnCells + 1, 256), 256, 0, stream>>>(train, st, fval);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  learn_cells_finish_kernel<<<1, kCellThreads, 0, stream>>>(fval, heavy, st, cells);
  return cudaGetLastError();
}

cudaError_t launch_scan_u32(const uint32_t* in, uint64_t count, uint32_t* out, uint32_t* out2, uint32_t* sums,
                            cudaStream_t stream) {
  if (!count) return cudaSuccess;
  const uint64_t blocks = (count + kScanTile - 1) / kScanTile;
  if (blocks >= (1ull << 32)) return cudaErrorInvalidValue;
  scan_reduce_kernel<<<unsigned(blocks), kScanThreads, 0, stream>>>(in, count, sums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scan_top_kernel<<<1, kScanThreads, 0, stream>>>(sums, uint32_t(blocks));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scan_apply_kernel<<<unsigned(blocks), kScanThreads, 0, stream>>>(in, count, sums, out, out2);
  return cudaGetLastError();
}

cudaError_t launch_learn_heavy_ids(const LearnedMap& mp, LearnedState* st, uint32_t* hid, uint32_t* bitmap,
                                   cudaStream_t stream) {
  learn_heavy_ids_kernel<<<grid_for(kLearnMaxHeavy, 256), 256, 0, stream>>>(mp, st, hid, bitmap);
  return cudaGetLastError();
}

LearnedGeom learned_geometry(uint64_t n, uint32_t buckets) {
  LearnedGeom g{};
  g.nb = buckets + 2u * kLearnMaxHeavy;
  // At most 10 fine bits: on 2^30 mixture keys 11 and 12 bits shorten level
  // 1's write runs but lengthen level 2's by more (both scatters: 21.1 ms at
  // 10 bits, 21.7 at 11, 22.7 at 12).  Fewer for small sorts, so that level 2
  // (one CTA per super-bucket) has 256..1024 CTAs.
  uint32_t lb = 0;
  while ((1u << lb) < g.nb) ++lb;
  g.fbits = lb > 9 + kFineBitsMax ? kFineBitsMax : (lb > 9 + kFineBitsMin ? lb - 9 : kFineBitsMin);
  if (g.fbits > 10) g.fbits = 10;
  if (g.fbits > kFineBitsMax) g.fbits = kFineBitsMax;
  g.nsuper = (g.nb + (1u << g.fbits) - 1) >> g.fbits;
  g.nids = g.nsuper << g.fbits;
  const uint64_t want = (n + kLearnL1Chunks - 1) / kLearnL1Chunks;
  g.chunk = want < 16384 ? 16384 : (want + 4095) / 4096 * 4096;
  g.nch = uint32_t((n + g.chunk - 1) / g.chunk);
  if (g.nch == 0) g.nch = 1;
  return g;
}

cudaError_t launch_learn_l1(const uint64_t* keys, uint64_t n, const LearnedGeom& g, const LearnedMap& mp,
                            const LearnedState* st, uint32_t heavy_count, uint32_t* counts1, uint32_t* hcount,
                            uint32_t* ids, cudaStream_t stream) {
  constexpr int kMaxBytes = (kMaxSuper + kLearnMaxHeavy) * 4;
  static const cudaError_t attr = set_smem_attrs(learn_l1_count_kernel, kMaxBytes, false);
  if (attr != cudaSuccess) return attr;
  if (g.nsuper > uint32_t(kMaxSuper) || heavy_count > uint32_t(kLearnMaxHeavy)) return cudaErrorInvalidValue;
  const size_t bytes = size_t(g.nsuper + heavy_count) * 4;
  learn_l1_count_kernel<<<g.nch, kPartThreads, bytes, stream>>>(keys, n, g.chunk, g.nch, g.nsuper, g.fbits, mp, st,
                                                                counts1, hcount, ids, heavy_count);
  return cudaGetLastError();
}

template <int kLevel>
cudaError_t launch_staged(const uint64_t* src, const uint32_t* ids, const uint16_t* fine_in, uint64_t n,
                          const LearnedGeom& g, const uint32_t* off1, const uint32_t* offsets, uint64_t* dst,
                          uint16_t* fine_out, unsigned grid, cudaStream_t stream) {
  const uint32_t cap = g.nsuper > (1u << g.fbits) ? g.nsuper : (1u << g.fbits);
  const StLayout L(kLevel, cap);
  static const cudaError_t attr =
      set_smem_attrs(learn_staged_scatter_kernel<kLevel>, StLayout(kLevel, kMaxSuper).bytes, true);
  if (attr != cudaSuccess) return attr;
  learn_staged_scatter_kernel<kLevel><<<grid, kStThreads, L.bytes, stream>>>(src, ids, fine_in, n, g.chunk, g.nch,
                                                                            g.nsuper, g.fbits, cap, off1, offsets,
                                                                            dst, fine_out);
  return cudaGetLastError();
}

cudaError_t launch_learn_l1_scatter(const uint64_t* keys, const uint32_t* ids, uint64_t n, const LearnedGeom& g,
                                    const uint32_t* off1, uint64_t* alt, uint16_t* fine, cudaStream_t stream) {
  return launch_staged<1>(keys, ids, nullptr, n, g, off1, nullptr, alt, fine, g.nch, stream);
}

cudaError_t launch_learn_l2_count(const uint16_t* fine, const LearnedGeom& g, const uint32_t* off1, uint32_t* counts,
                                  cudaStream_t stream) {
  learn_l2_count_kernel<<<g.nsuper, kL2Threads, 0, stream>>>(fine, off1, g.nch, g.fbits, counts);
  return cudaGetLastError();
}

cudaError_t launch_learn_judge(uint32_t* counts, const LearnedGeom& g, const uint32_t* bitmap, const uint32_t* hid,
                               const uint32_t* hcount, LearnedState* st, uint32_t* large_list, cudaStream_t stream) {
  const uint32_t threads = g.nids > uint32_t(kLearnMaxHeavy) ? g.nids : uint32_t(kLearnMaxHeavy);
  learn_judge_kernel<<<grid_for(threads, 256), 256, 0, stream>>>(counts, g.nids, bitmap, hid, hcount, st, large_list);
  return cudaGetLastError();
}

cudaError_t launch_learn_l2_scatter(const uint64_t* alt, const uint16_t* fine, const LearnedGeom& g,
                                    const uint32_t* off1, const uint32_t* off2, uint64_t* dst, cudaStream_t stream) {
  return launch_staged<2>(alt, nullptr, fine, 0, g, off1, off2, dst, nullptr, g.nsuper, stream);
}

cudaError_t launch_learn_fill(const LearnedMap& mp, const LearnedState* st, const uint32_t* hid,
                              const uint32_t* large_list, const uint32_t* offsets, const uint32_t* counts,
                              uint64_t* dst, int sms, cudaStream_t stream) {
  learn_fill_kernel<<<unsigned(sms) * 4, 256, 0, stream>>>(mp, st, hid, large_list, offsets, counts, dst);
  return cudaGetLastError();
}

template <class G>
cudaError_t launch_bucket_sort_geom(uint64_t* keys, const uint2* list, int step, const uint32_t* count, int sms,
                                    cudaStream_t stream) {
  static const int per_sm = [] {  // resident CTAs per SM (0: the attributes could not be set)
    int v = 0;
    if (set_smem_attrs(learn_bucket_sort_kernel<G>, G::kBytes, true) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, learn_bucket_sort_kernel<G>, G::kThreads, G::kBytes) !=
        cudaSuccess)
      return 0;
    return v < 1 ? 1 : v;
  }();
  if (!per_sm) return cudaErrorInvalidConfiguration;
  learn_bucket_sort_kernel<G><<<unsigned(sms) * unsigned(per_sm), G::kThreads, G::kBytes, stream>>>(keys, list, step,
                                                                                                     count);
  return cudaGetLastError();
}

cudaError_t launch_learn_bucket_sort(uint64_t* keys, const uint32_t* counts, const uint32_t* offsets,
                                     const uint32_t* bitmap, uint32_t nb, uint2* units, uint32_t* status, int sms,
                                     cudaStream_t stream) {
  const uint32_t ngroups = (nb + kGroup - 1) / kGroup;
  cudaError_t e = cudaMemsetAsync(units, 0, sizeof(uint2), stream);
  if (e != cudaSuccess) return e;
  learn_units_kernel<<<grid_for(ngroups, 256), 256, 0, stream>>>(counts, offsets, bitmap, nb, units, status);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_bucket_sort_geom<BsNarrow>(keys, units + 1, 1, &units[0].x, sms, stream);
  if (e == cudaSuccess) e = launch_bucket_sort_geom<BsWide>(keys, units + nb, -1, &units[0].y, sms, stream);
  return e;
}

cudaError_t launch_learn_bucket_ids(const uint64_t* keys, uint64_t n, const LearnedMap& mp, uint32_t* ids,
                                    cudaStream_t stream) {
  if (!n) return cudaSuccess;
  const uint64_t need = (n + 255) / 256;
  learn_bucket_ids_kernel<<<unsigned(need < 4096 ? need : 4096), 256, 0, stream>>>(keys, n, mp, ids);
  return cudaGetLastError();
}

}  // namespace fsort
