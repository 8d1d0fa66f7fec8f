// fsort_stream.cu -- the streaming histogram: counts of the sort keys s(k) =
// k >> (key_bits - p) accumulated over any number of batches (each batch read
// once, never again: the batch counter update of Sec. III-C/D), with rank and
// select queries on it (Alg. 3 GetIndex and Alg. 2 GetItem) and the sorted
// multiset of everything seen rebuilt from it (Alg. 5 with no trailing bits).
//
//   shist_smem_kernel / shist_global_kernel
//       accumulation: 32-bit per-CTA counters in shared memory flushed into
//       the 64-bit device counts (the tapered widths of Sec. III-D-1), or, for
//       more bins than shared memory holds, warp-aggregated 64-bit atomics
//   scan64_*   the exclusive prefix over all 2^p bins: the index every query
//              uses (rebuilt lazily after an accumulation)
//   shist_rank_kernel    rank(v) = prefix[v]
//   shist_select_kernel  select(r) = the bin v with prefix[v] <= r < prefix[v+1]
//   shist_expand_kernel  output window per CTA; each thread finds its bin by
//                        binary search inside the window's bin range
#include <cuda_runtime.h>

#include <cstdint>
#include <new>

#include "../../include/fsort.h"
#include "fsort_dev.cuh"
#include "fsort_internal.h"

namespace {

constexpr int kSmemBinsMax = 1 << 15;  // 128 KB of 32-bit counters
constexpr int kHistThreads = 512;

template <typename K>
__device__ __forceinline__ uint32_t skey(K k, uint32_t shift) {
  return uint32_t(uint64_t(k) >> shift);
}

template <typename K>
__global__ void __launch_bounds__(kHistThreads) shist_smem_kernel(const K* __restrict__ keys, uint64_t n,
                                                                  uint32_t shift, uint32_t bins,
                                                                  unsigned long long* __restrict__ counts) {
  extern __shared__ uint32_t s_cnt[];
  for (uint32_t i = threadIdx.x; i < bins; i += kHistThreads) s_cnt[i] = 0;
  __syncthreads();
  const uint64_t stride = uint64_t(gridDim.x) * kHistThreads;
  for (uint64_t i = uint64_t(blockIdx.x) * kHistThreads + threadIdx.x; i < n; i += stride)
    atomicAdd(&s_cnt[skey(keys[i], shift)], 1u);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < bins; i += kHistThreads)
    if (s_cnt[i]) atomicAdd(&counts[i], (unsigned long long)s_cnt[i]);
}

template <typename K>
__global__ void __launch_bounds__(kHistThreads) shist_global_kernel(const K* __restrict__ keys, uint64_t n,
                                                                    uint32_t shift,
                                                                    unsigned long long* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const uint64_t stride = uint64_t(gridDim.x) * kHistThreads;
  for (uint64_t base = uint64_t(blockIdx.x) * kHistThreads + (threadIdx.x & ~31u); base < n; base += stride) {
    const uint64_t i = base + lane;
    const bool valid = i < n;
    const uint32_t v = valid ? skey(keys[i], shift) : 0xFFFFFFFFu;
    // equal bins in a warp add once (skewed streams would serialise on one counter)
    const uint32_t peers = __match_any_sync(0xffffffffu, v);
    if (valid && (peers & fsort::lanemask_lt()) == 0) atomicAdd(&counts[v], (unsigned long long)__popc(peers));
  }
}

// ---- exclusive scan of 64-bit counts: prefix[0..m] with prefix[m] = total ----
constexpr int kScanThreads = 1024;
constexpr int kScanIpt = 4;
constexpr uint64_t kScanTile = uint64_t(kScanThreads) * kScanIpt;

__device__ __forceinline__ uint64_t block_excl_scan64(uint64_t v, uint64_t* s_w, uint64_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint64_t x = s_w[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_w[lane] = x;
  }
  __syncthreads();
  total = s_w[31];
  return (warp ? s_w[warp - 1] : 0ull) + inc - v;
}

__global__ void __launch_bounds__(kScanThreads) scan64_reduce_kernel(const unsigned long long* __restrict__ in,
                                                                     uint64_t m, uint64_t* __restrict__ sums) {
  __shared__ uint64_t s_w[32];
  const uint64_t at = blockIdx.x * kScanTile + uint64_t(threadIdx.x) * kScanIpt;
  uint64_t v = 0;
#pragma unroll
  for (int j = 0; j < kScanIpt; ++j)
    if (at + j < m) v += in[at + j];
  uint64_t total;
  block_excl_scan64(v, s_w, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan64_top_kernel(uint64_t* __restrict__ sums, uint32_t nblocks) {
  __shared__ uint64_t s_w[32];
  __shared__ uint64_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t b0 = 0; b0 < nblocks; b0 += kScanThreads) {  // one element per thread per round
    const uint32_t i = b0 + threadIdx.x;
    const uint64_t x = i < nblocks ? sums[i] : 0ull;
    uint64_t total;
    const uint64_t ex = block_excl_scan64(x, s_w, total);
    const uint64_t carry = s_carry;
    if (i < nblocks) sums[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + total;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nblocks] = s_carry;
}

__global__ void __launch_bounds__(kScanThreads) scan64_apply_kernel(const unsigned long long* __restrict__ in,
                                                                    uint64_t m, const uint64_t* __restrict__ sums,
                                                                    uint64_t* __restrict__ out) {
  __shared__ uint64_t s_w[32];
  const uint64_t at = blockIdx.x * kScanTile + uint64_t(threadIdx.x) * kScanIpt;
  uint64_t x[kScanIpt], v = 0;
#pragma unroll
  for (int j = 0; j < kScanIpt; ++j) {
    x[j] = (at + j < m) ? uint64_t(in[at + j]) : 0ull;
    v += x[j];
  }
  uint64_t total;
  uint64_t run = sums[blockIdx.x] + block_excl_scan64(v, s_w, total);
#pragma unroll
  for (int j = 0; j < kScanIpt; ++j) {
    if (at + j < m) out[at + j] = run;
    run += x[j];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[m] = sums[gridDim.x];
}

// ---- queries ---------------------------------------------------------------
// Largest v in [lo, hi] with prefix[v] <= r (prefix non-decreasing, prefix[lo] <= r).
__device__ __forceinline__ uint32_t bin_of(const uint64_t* __restrict__ prefix, uint32_t lo, uint32_t hi, uint64_t r) {
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo + 1) / 2;
    if (prefix[mid] <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void shist_rank_kernel(const uint64_t* __restrict__ prefix, uint32_t bins,
                                  const uint64_t* __restrict__ values, uint64_t count, uint64_t* __restrict__ ranks) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) {
    const uint64_t v = values[i];
    ranks[i] = prefix[v < bins ? v : bins];
  }
}

__global__ void shist_select_kernel(const uint64_t* __restrict__ prefix, uint32_t bins,
                                    const uint64_t* __restrict__ ranks, uint64_t count, uint64_t* __restrict__ out) {
  const uint64_t total = prefix[bins];
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) {
    const uint64_t r = ranks[i];
    out[i] = r < total ? uint64_t(bin_of(prefix, 0, bins - 1, r)) : ~0ull;
  }
}

// keys_out[i] = the bin of sorted position i, windows of kExpandWindow
// positions per CTA iteration: the window's first and last bins bound each
// thread's binary search, so dense windows need few steps.
constexpr int kExpandThreads = 256;
constexpr int kExpandWindow = 4096;

template <typename K>
__global__ void __launch_bounds__(kExpandThreads) shist_expand_kernel(const uint64_t* __restrict__ prefix,
                                                                      uint32_t bins, K* __restrict__ out,
                                                                      uint64_t total) {
  __shared__ uint32_t s_range[2];
  for (uint64_t w0 = uint64_t(blockIdx.x) * kExpandWindow; w0 < total; w0 += uint64_t(gridDim.x) * kExpandWindow) {
    const uint64_t w1 = w0 + kExpandWindow < total ? w0 + kExpandWindow : total;
    if (threadIdx.x == 0) {
      s_range[0] = bin_of(prefix, 0, bins - 1, w0);
      s_range[1] = bin_of(prefix, s_range[0], bins - 1, w1 - 1);
    }
    __syncthreads();
    const uint32_t lo = s_range[0], hi = s_range[1];
    uint32_t v = lo;  // positions ascend with the thread: restart each search from the last bin found
    for (uint64_t i = w0 + threadIdx.x; i < w1; i += kExpandThreads) {
      v = bin_of(prefix, v, hi, i);
      out[i] = K(v);
    }
    __syncthreads();
  }
}

unsigned grid_for(uint64_t n, int threads, unsigned cap) {
  const uint64_t g = (n + threads - 1) / threads;
  return unsigned(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

struct fsort_hist {
  int device = 0;
  int sms = 0;
  int key_bits = 0;
  int precision_bits = 0;
  uint32_t bins = 0;
  unsigned long long* counts = nullptr;  // [bins]
  uint64_t* prefix = nullptr;            // [bins + 1]
  uint64_t* sums = nullptr;              // scan scratch
  uint64_t total = 0;                    // host copy: keys accumulated
  bool dirty = true;                     // prefix out of date
};

namespace {

fsort_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return FSORT_OK;
  if (e == cudaErrorMemoryAllocation) return FSORT_ERR_OOM;
  return FSORT_ERR_CUDA;
}

// Natural alignment of an array read or written element by element (a must be a power of two).
bool aligned_to(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

cudaError_t build_index(fsort_hist* h, cudaStream_t s) {
  if (!h->dirty) return cudaSuccess;
  const uint64_t m = h->bins;
  const uint64_t blocks = (m + kScanTile - 1) / kScanTile;
  scan64_reduce_kernel<<<unsigned(blocks), kScanThreads, 0, s>>>(h->counts, m, h->sums);
  scan64_top_kernel<<<1, kScanThreads, 0, s>>>(h->sums, uint32_t(blocks));
  scan64_apply_kernel<<<unsigned(blocks), kScanThreads, 0, s>>>(h->counts, m, h->sums, h->prefix);
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) h->dirty = false;
  return e;
}

template <typename K>
cudaError_t accumulate_typed(fsort_hist* h, const void* keys, uint64_t n, cudaStream_t s) {
  const uint32_t shift = uint32_t(h->key_bits - h->precision_bits);
  const K* k = static_cast<const K*>(keys);
  if (h->bins <= uint32_t(kSmemBinsMax)) {
    const size_t bytes = size_t(h->bins) * 4;
    static const cudaError_t attr = fsort::set_smem_attrs(shist_smem_kernel<K>, size_t(kSmemBinsMax) * 4, false);
    if (attr != cudaSuccess) return attr;
    // per CTA at most 2^31 keys: its 32-bit counters cannot wrap
    unsigned grid = grid_for(n, kHistThreads, unsigned(h->sms) * 2);
    while (uint64_t(grid) << 31 < n) grid *= 2;
    shist_smem_kernel<K><<<grid, kHistThreads, bytes, s>>>(k, n, shift, h->bins, h->counts);
  } else {
    shist_global_kernel<K><<<grid_for(n, kHistThreads, unsigned(h->sms) * 4), kHistThreads, 0, s>>>(k, n, shift,
                                                                                                   h->counts);
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" {

fsort_status fsort_hist_create(int key_bits, int precision_bits, fsort_hist** out) {
  if (!out || (key_bits != 16 && key_bits != 32 && key_bits != 64)) return FSORT_ERR_INVALID_ARG;
  if (precision_bits < 1 || precision_bits > key_bits) return FSORT_ERR_INVALID_ARG;
  if (precision_bits > 24) return FSORT_ERR_UNSUPPORTED;
  fsort_hist* h = new (std::nothrow) fsort_hist();
  if (!h) return FSORT_ERR_OOM;
  h->key_bits = key_bits;
  h->precision_bits = precision_bits;
  h->bins = 1u << precision_bits;
  const uint64_t blocks = (uint64_t(h->bins) + kScanTile - 1) / kScanTile;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->counts), size_t(h->bins) * 8);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->prefix), (size_t(h->bins) + 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->sums), (blocks + 1) * 8);
  if (e == cudaSuccess) e = cudaMemset(h->counts, 0, size_t(h->bins) * 8);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    fsort_hist_destroy(h);
    return from_cuda(e);
  }
  *out = h;
  return FSORT_OK;
}

fsort_status fsort_hist_destroy(fsort_hist* h) {
  if (!h) return FSORT_OK;
  fsort_status st = FSORT_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) st = FSORT_ERR_CUDA;
  if (h->counts) cudaFree(h->counts);
  if (h->prefix) cudaFree(h->prefix);
  if (h->sums) cudaFree(h->sums);
  delete h;
  return st;
}

fsort_status fsort_hist_reset(fsort_hist* h, void* stream) {
  if (!h) return FSORT_ERR_INVALID_ARG;
  const cudaError_t e = cudaMemsetAsync(h->counts, 0, size_t(h->bins) * 8, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return from_cuda(e);
  h->total = 0;
  h->dirty = true;
  return FSORT_OK;
}

fsort_status fsort_hist_accumulate(fsort_hist* h, const void* keys, uint64_t n, void* stream) {
  if (!h || (n && (!keys || !aligned_to(keys, uintptr_t(h->key_bits / 8))))) return FSORT_ERR_INVALID_ARG;
  if (n == 0) return FSORT_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (h->key_bits == 16) e = accumulate_typed<uint16_t>(h, keys, n, s);
  else if (h->key_bits == 32) e = accumulate_typed<uint32_t>(h, keys, n, s);
  else e = accumulate_typed<uint64_t>(h, keys, n, s);
  if (e != cudaSuccess) return from_cuda(e);
  h->total += n;
  h->dirty = true;
  return FSORT_OK;
}

fsort_status fsort_hist_total(const fsort_hist* h, uint64_t* total) {
  if (!h || !total) return FSORT_ERR_INVALID_ARG;
  *total = h->total;
  return FSORT_OK;
}

fsort_status fsort_hist_counts(fsort_hist* h, uint64_t* counts_out, void* stream) {
  if (!h || !counts_out || !aligned_to(counts_out, 8)) return FSORT_ERR_INVALID_ARG;
  return from_cuda(cudaMemcpyAsync(counts_out, h->counts, size_t(h->bins) * 8, cudaMemcpyDeviceToDevice,
                                   static_cast<cudaStream_t>(stream)));
}

fsort_status fsort_hist_rank(fsort_hist* h, const uint64_t* values, uint64_t count, uint64_t* ranks, void* stream) {
  if (!h || (count && (!values || !ranks || !aligned_to(values, 8) || !aligned_to(ranks, 8))))
    return FSORT_ERR_INVALID_ARG;
  if (count == 0) return FSORT_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = build_index(h, s);
  if (e == cudaSuccess) {
    shist_rank_kernel<<<grid_for(count, 256, unsigned(h->sms) * 8), 256, 0, s>>>(h->prefix, h->bins, values, count,
                                                                                ranks);
    e = cudaGetLastError();
  }
  return from_cuda(e);
}

fsort_status fsort_hist_select(fsort_hist* h, const uint64_t* ranks, uint64_t count, uint64_t* values, void* stream) {
  if (!h || (count && (!values || !ranks || !aligned_to(values, 8) || !aligned_to(ranks, 8))))
    return FSORT_ERR_INVALID_ARG;
  if (count == 0) return FSORT_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = build_index(h, s);
  if (e == cudaSuccess) {
    shist_select_kernel<<<grid_for(count, 256, unsigned(h->sms) * 8), 256, 0, s>>>(h->prefix, h->bins, ranks, count,
                                                                                  values);
    e = cudaGetLastError();
  }
  return from_cuda(e);
}

fsort_status fsort_hist_expand(fsort_hist* h, void* keys_out, uint64_t n, void* stream) {
  if (!h || n != h->total || (n && (!keys_out || !aligned_to(keys_out, uintptr_t(h->key_bits / 8)))))
    return FSORT_ERR_INVALID_ARG;
  if (n == 0) return FSORT_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = build_index(h, s);
  if (e != cudaSuccess) return from_cuda(e);
  const unsigned grid = grid_for(n, kExpandWindow, unsigned(h->sms) * 8);
  if (h->key_bits == 16)
    shist_expand_kernel<uint16_t><<<grid, kExpandThreads, 0, s>>>(h->prefix, h->bins, static_cast<uint16_t*>(keys_out), n);
  else if (h->key_bits == 32)
    shist_expand_kernel<uint32_t><<<grid, kExpandThreads, 0, s>>>(h->prefix, h->bins, static_cast<uint32_t*>(keys_out), n);
  else
    shist_expand_kernel<uint64_t><<<grid, kExpandThreads, 0, s>>>(h->prefix, h->bins, static_cast<uint64_t*>(keys_out), n);
  return from_cuda(cudaGetLastError());
}

}  // extern "C"
