// fsort_batch.cu -- kernels of the batched path: many independent sorts in a
// few launches (the paper's batch stream sorting, Sec. III-C and IV-D: batches
// of the input processed without pre-processing, batch size tuned to the
// device).
//
//  small_sort_kernel   persistent; each CTA takes whole small segments from a
//                      work counter and sorts each one entirely in shared
//                      memory: one read and one write of the segment, every
//                      radix pass a stable in-block counting pass
//  seg_hist_kernel     per-segment per-pass digit histograms of the large
//                      segments (one read of their keys)
//  seg_scan_kernel     per segment and pass, the exclusive scan of the
//                      histogram into 64-bit digit bases
//  (the scatter passes of the large segments are K3 in segmented mode)
#include <cstdint>
#include <cuda_runtime.h>

#include "fsort_dev.cuh"
#include "fsort_internal.h"
#include "fsort_rank.cuh"

namespace fsort {
namespace {

constexpr int kRadix = kRankRadix;

// ------------------------------------------------------------ small sort ---
constexpr int kSmallBlock = 256;  // == kRadix: thread d owns digit d

template <typename K, bool kVals, int kCap>
struct SmallLayout {
  static constexpr int kIpt = kCap / kSmallBlock;
  static constexpr int kWarps = kSmallBlock / 32;
  static constexpr size_t kKeysA = 0;
  static constexpr size_t kKeysB = kKeysA + size_t(kCap) * sizeof(K);
  static constexpr size_t kValsA = kKeysB + size_t(kCap) * sizeof(K);
  static constexpr size_t kValsB = kValsA + (kVals ? size_t(kCap) * 4 : 0);
  static constexpr size_t kMask = kValsB + (kVals ? size_t(kCap) * 4 : 0);
  static constexpr size_t kWcnt = kMask + 2 * size_t(kWarps) * kRadix * 4;
  static constexpr size_t kScan = kWcnt + size_t(kWarps) * kRadix * 4;
  static constexpr size_t kMisc = kScan + 16 * 4;
  static constexpr size_t kBytes = kMisc + 16;
};

template <typename K, bool kVals, int kCap>
__global__ void __launch_bounds__(kSmallBlock) small_sort_kernel(const SegDesc* __restrict__ segs, uint32_t count,
                                                                 DigitPlan plan, uint32_t* counter) {
  using L = SmallLayout<K, kVals, kCap>;
  constexpr int kIpt = L::kIpt;
  constexpr int kWarps = L::kWarps;
  extern __shared__ __align__(16) unsigned char smem[];
  K* keys_buf[2] = {reinterpret_cast<K*>(smem + L::kKeysA), reinterpret_cast<K*>(smem + L::kKeysB)};
  uint32_t* vals_buf[2] = {reinterpret_cast<uint32_t*>(smem + L::kValsA),
                           reinterpret_cast<uint32_t*>(smem + L::kValsB)};
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(smem + L::kMask);
  uint32_t* s_wcnt = reinterpret_cast<uint32_t*>(smem + L::kWcnt);
  uint32_t* s_scan = reinterpret_cast<uint32_t*>(smem + L::kScan);
  uint32_t* s_misc = reinterpret_cast<uint32_t*>(smem + L::kMisc);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* wmask0 = s_mask + warp * kRadix;
  uint32_t* wmask1 = s_mask + (kWarps + warp) * kRadix;
  uint32_t* wcnt = s_wcnt + warp * kRadix;
  const int wbase = warp * 32 * kIpt;
  for (int i = tid; i < 2 * kWarps * kRadix; i += kSmallBlock) s_mask[i] = 0;  // rank_strip leaves them zero

  while (true) {
    if (tid == 0) s_misc[0] = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t si = s_misc[0];
    if (si >= count) return;
    const SegDesc sd = segs[si];
    const uint32_t n = uint32_t(sd.n);
    K* gk = static_cast<K*>(sd.keys);
    for (uint32_t i = tid; i < n; i += kSmallBlock) {
      keys_buf[0][i] = gk[i];
      if (kVals) vals_buf[0][i] = sd.vals[i];
    }
    int cur = 0;
    for (int j = 0; j < plan.passes; ++j) {
      for (int i = tid; i < kWarps * kRadix; i += kSmallBlock) s_wcnt[i] = 0;
      __syncthreads();
      const uint32_t shift = plan.shift[j], mask = plan.mask[j];
      Item<K> it[kIpt];
      rank_strip<K, kIpt>(keys_buf[cur], n, wbase, shift, mask, wmask0, wmask1, wcnt, it);
      __syncthreads();
      // digit d = tid: strip prefixes, segment total, segment-exclusive start
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = s_wcnt[w * kRadix + tid];
        s_wcnt[w * kRadix + tid] = run;
        run += c;
      }
      const uint32_t ex = digit_excl_scan<kSmallBlock>(run, s_scan);
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s_wcnt[w * kRadix + tid] += ex;
      // a pass whose digit is the same for every key is the identity
      const int trivial = __syncthreads_or(run == n);
      if (trivial) continue;
#pragma unroll
      for (int i = 0; i < kIpt; ++i) {
        const int pos = wbase + i * 32 + lane;
        if (uint32_t(pos) < n) {
          const K k = it[i].k();
          const uint32_t p = s_wcnt[warp * kRadix + dig(k, shift, mask)] + it[i].r();
          keys_buf[cur ^ 1][p] = k;
          if (kVals) vals_buf[cur ^ 1][p] = vals_buf[cur][pos];
        }
      }
      __syncthreads();  // every warp has read its offsets before the next pass clears them
      cur ^= 1;
    }
    __syncthreads();
    for (uint32_t i = tid; i < n; i += kSmallBlock) {
      gk[i] = keys_buf[cur][i];
      if (kVals) sd.vals[i] = vals_buf[cur][i];
    }
    __syncthreads();
  }
}

template <typename K, bool kVals, int kCap>
cudaError_t launch_small_typed(const SegDesc* segs, uint32_t count, const DigitPlan& plan, uint32_t* counter, int ctas,
                               cudaStream_t stream) {
  using L = SmallLayout<K, kVals, kCap>;
  static const cudaError_t attr = set_smem_attrs(small_sort_kernel<K, kVals, kCap>, L::kBytes, true);
  if (attr != cudaSuccess) return attr;
  small_sort_kernel<K, kVals, kCap><<<unsigned(ctas), kSmallBlock, L::kBytes, stream>>>(segs, count, plan, counter);
  return cudaGetLastError();
}

template <typename K, bool kVals>
cudaError_t launch_small_cap(const SegDesc* segs, uint32_t count, int capacity, const DigitPlan& plan,
                             uint32_t* counter, int ctas, cudaStream_t stream) {
  switch (capacity) {
    case 1024: return launch_small_typed<K, kVals, 1024>(segs, count, plan, counter, ctas, stream);
    case 2048: return launch_small_typed<K, kVals, 2048>(segs, count, plan, counter, ctas, stream);
    case 4096: return launch_small_typed<K, kVals, 4096>(segs, count, plan, counter, ctas, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <typename K, bool kVals>
size_t small_bytes(int capacity) {
  switch (capacity) {
    case 1024: return SmallLayout<K, kVals, 1024>::kBytes;
    case 2048: return SmallLayout<K, kVals, 2048>::kBytes;
    case 4096: return SmallLayout<K, kVals, 4096>::kBytes;
    default: return 0;
  }
}

// --------------------------------------------------- segmented histogram ---
constexpr int kSegHistThreads = 512;

template <typename K, int P>
__global__ void __launch_bounds__(kSegHistThreads) seg_hist_kernel(const SegDesc* __restrict__ segs,
                                                                   const HistChunk* __restrict__ chunks,
                                                                   DigitPlan plan, uint64_t* __restrict__ hist,
                                                                   uint32_t* clear, uint64_t clear_words) {
  __shared__ uint32_t counts[P * kRadix];
  for (int i = threadIdx.x; i < P * kRadix; i += blockDim.x) counts[i] = 0;
  {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < clear_words; i += stride) clear[i] = 0;
  }
  __syncthreads();
  const HistChunk c = chunks[blockIdx.x];
  const K* keys = static_cast<const K*>(segs[c.seg].keys) + c.start;
  for (uint32_t i = threadIdx.x; i < c.len; i += blockDim.x) {
    const K k = keys[i];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const uint32_t d = (sizeof(K) <= 4 ? (uint32_t(k) >> plan.shift[j]) : uint32_t(uint64_t(k) >> plan.shift[j])) &
                         plan.mask[j];
      atomicAdd(&counts[j * kRadix + d], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P * kRadix; i += blockDim.x) {
    const uint32_t v = counts[i];
    if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&hist[uint64_t(c.seg) * P * kRadix + i]),
                     (unsigned long long)v);
  }
}

__global__ void __launch_bounds__(kRadix) seg_scan_kernel(uint64_t* __restrict__ hist, uint64_t* __restrict__ bases,
                                                          int passes) {
  __shared__ uint32_t s_warp[16];
  const uint64_t row0 = uint64_t(blockIdx.x) * passes;
  for (int j = 0; j < passes; ++j) {
    const uint64_t at = (row0 + j) * kRadix + threadIdx.x;
    const uint64_t c = hist[at];
    hist[at] = 0;
    // segments hold < 2^32 keys: 32-bit scan
    const uint32_t ex = digit_excl_scan<kRadix>(uint32_t(c), s_warp);
    bases[at] = ex;
    __syncthreads();
  }
}

__global__ void fill_tile_seg_kernel(const SegDesc* __restrict__ segs, int tile_keys, uint32_t* __restrict__ tile_seg) {
  const SegDesc sd = segs[blockIdx.x];
  const uint32_t tiles = uint32_t((sd.n + tile_keys - 1) / tile_keys);
  for (uint32_t t = threadIdx.x; t < tiles; t += blockDim.x) tile_seg[sd.first_tile + t] = blockIdx.x;
}

template <typename K>
__global__ void seg_copy_back_kernel(const SegDesc* __restrict__ segs, const K* __restrict__ alt_keys,
                                     const uint32_t* __restrict__ alt_vals) {
  const SegDesc sd = segs[blockIdx.y];
  K* k = static_cast<K*>(sd.keys);
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < sd.n; i += stride) {
    k[i] = alt_keys[sd.alt_off + i];
    if (sd.vals) sd.vals[i] = alt_vals[sd.alt_off + i];
  }
}

}  // namespace

int small_sort_ctas_per_sm(int key_bits, bool has_vals, int capacity) {
  size_t b = 0;
  switch (key_bits) {
    case 16: b = has_vals ? small_bytes<uint16_t, true>(capacity) : small_bytes<uint16_t, false>(capacity); break;
    case 32: b = has_vals ? small_bytes<uint32_t, true>(capacity) : small_bytes<uint32_t, false>(capacity); break;
    case 64: b = has_vals ? small_bytes<uint64_t, true>(capacity) : small_bytes<uint64_t, false>(capacity); break;
    default: return 0;
  }
  if (!b) return 0;
  const size_t per_sm = 227 * 1024;
  int c = int(per_sm / (b + 1024));
  if (c > 8) c = 8;  // 8 CTAs x 256 threads fill an SM
  return c < 1 ? 1 : c;
}

cudaError_t launch_small_sort(const SegDesc* segs, uint32_t count, int key_bits, bool has_vals, int capacity,
                              const DigitPlan& plan, uint32_t* counter, int ctas, cudaStream_t stream) {
  if (!count) return cudaSuccess;
  switch (key_bits) {
    case 16: return has_vals ? launch_small_cap<uint16_t, true>(segs, count, capacity, plan, counter, ctas, stream)
                             : launch_small_cap<uint16_t, false>(segs, count, capacity, plan, counter, ctas, stream);
    case 32: return has_vals ? launch_small_cap<uint32_t, true>(segs, count, capacity, plan, counter, ctas, stream)
                             : launch_small_cap<uint32_t, false>(segs, count, capacity, plan, counter, ctas, stream);
    case 64: return has_vals ? launch_small_cap<uint64_t, true>(segs, count, capacity, plan, counter, ctas, stream)
                             : launch_small_cap<uint64_t, false>(segs, count, capacity, plan, counter, ctas, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <typename K>
cudaError_t seg_hist_passes(const SegDesc* segs, const HistChunk* chunks, uint32_t nchunks, const DigitPlan& plan,
                            uint64_t* hist, uint32_t* clear, uint64_t clear_words, cudaStream_t stream) {
#define FSORT_SEGHIST_CASE(P_)                                                                              \
  case P_:                                                                                                  \
    seg_hist_kernel<K, P_><<<nchunks, kSegHistThreads, 0, stream>>>(segs, chunks, plan, hist, clear, clear_words); \
    break;
  switch (plan.passes) {
    FSORT_SEGHIST_CASE(1)
    FSORT_SEGHIST_CASE(2)
    FSORT_SEGHIST_CASE(3)
    FSORT_SEGHIST_CASE(4)
    FSORT_SEGHIST_CASE(5)
    FSORT_SEGHIST_CASE(6)
    FSORT_SEGHIST_CASE(7)
    FSORT_SEGHIST_CASE(8)
    default:
      return cudaErrorInvalidValue;
  }
#undef FSORT_SEGHIST_CASE
  return cudaGetLastError();
}

cudaError_t launch_seg_histogram(const SegDesc* segs, const HistChunk* chunks, uint32_t nchunks, int key_bits,
                                 const DigitPlan& plan, uint64_t* hist, uint32_t* clear, uint64_t clear_words,
                                 cudaStream_t stream) {
  if (!nchunks) return cudaSuccess;
  switch (key_bits) {
    case 16: return seg_hist_passes<uint16_t>(segs, chunks, nchunks, plan, hist, clear, clear_words, stream);
    case 32: return seg_hist_passes<uint32_t>(segs, chunks, nchunks, plan, hist, clear, clear_words, stream);
    case 64: return seg_hist_passes<uint64_t>(segs, chunks, nchunks, plan, hist, clear, clear_words, stream);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_seg_scan(uint64_t* hist, uint64_t* bases, uint32_t nsegs, int passes, cudaStream_t stream) {
  if (!nsegs) return cudaSuccess;
  seg_scan_kernel<<<nsegs, kRadix, 0, stream>>>(hist, bases, passes);
  return cudaGetLastError();
}

cudaError_t launch_fill_tile_seg(const SegDesc* segs, uint32_t nsegs, int tile_keys, uint32_t* tile_seg,
                                 cudaStream_t stream) {
  if (!nsegs) return cudaSuccess;
  fill_tile_seg_kernel<<<nsegs, 256, 0, stream>>>(segs, tile_keys, tile_seg);
  return cudaGetLastError();
}

cudaError_t launch_seg_copy_back(const SegDesc* segs, uint32_t nsegs, const void* alt_keys, const uint32_t* alt_vals,
                                 int key_bits, int sms, cudaStream_t stream) {
  if (!nsegs) return cudaSuccess;
  const dim3 grid{unsigned(sms > 0 ? (sms + 7) / 8 : 1), nsegs, 1u};
  switch (key_bits) {
    case 16: seg_copy_back_kernel<uint16_t><<<grid, 256, 0, stream>>>(segs, static_cast<const uint16_t*>(alt_keys), alt_vals); break;
    case 32: seg_copy_back_kernel<uint32_t><<<grid, 256, 0, stream>>>(segs, static_cast<const uint32_t*>(alt_keys), alt_vals); break;
    case 64: seg_copy_back_kernel<uint64_t><<<grid, 256, 0, stream>>>(segs, static_cast<const uint64_t*>(alt_keys), alt_vals); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fsort
