// fsort_hist.cu -- histogram, scan and expand kernels of libfsort.
//
//  K1  hist_kernel        every pass's digit histogram from one read of the keys
//                          (Sec. III-A/B: one counter update per key per digit)
//  K1' leaf_hist_kernel   the 65,536-bin histogram of 16-bit keys with 16-bit
//                          tapered counters and exact overflow spills (Sec. III-D-1)
//  K2  scan_schedule      exclusive scan per pass (Alg. 3's rank of every leaf),
//                          the first look-back chunk's bases, the device-side pass schedule
//  K4  expand_kernel      Alg. 5 without trailing bits: key v written C[v] times
#include <cstdint>
#include <cuda_runtime.h>

#include "fsort_dev.cuh"
#include "fsort_internal.h"

namespace fsort {
namespace {

constexpr int kRadix = 256;

// ---------------------------------------------------------------- K1 -------
// Every CTA owns a slice of the keys and keeps one shared-memory counter per
// (pass, digit).  Counts are added with shared-memory reductions
// (red.shared.add: the lanes of a warp that add to one counter are served
// together when no other counter of that bank is hit in the same instruction,
// so a digit shared by the whole warp costs one pass), then merged into the
// global 64-bit histogram with one atomic per non-zero counter.
constexpr int kHistThreads = 512;

// P = number of passes (compile time, so the per-key loop is exactly P
// digit extractions and P shared-memory reductions).
template <typename K, int P>
__global__ void __launch_bounds__(kHistThreads) hist_kernel(const K* __restrict__ keys, uint64_t n, DigitPlan plan,
                                                            uint64_t* __restrict__ hist, uint64_t pass_stride,
                                                            uint32_t* clear, uint64_t clear_words) {
  __shared__ uint32_t counts[P * kRadix];
  for (int i = threadIdx.x; i < P * kRadix; i += blockDim.x) counts[i] = 0;

  // Clear the first pass's look-back region and the tile counters.
  {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t first = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    for (uint64_t i = first; i < clear_words; i += stride) clear[i] = 0;
  }
  __syncthreads();

  // Slice of the input for this CTA, in whole 16-byte vectors.  A CTA counts
  // fewer than 2^32 keys (n <= 2^36, >= 16 CTAs), so 32-bit counters suffice.
  constexpr uint64_t kVec = 16 / sizeof(K);
  const uint64_t vecs = (n + kVec - 1) / kVec;
  const uint64_t per = (vecs + gridDim.x - 1) / gridDim.x;
  const uint64_t v_lo = blockIdx.x * per;
  const uint64_t v_hi = (v_lo + per < vecs) ? v_lo + per : vecs;

  uint32_t shift[P], mask[P];
#pragma unroll
  for (int j = 0; j < P; ++j) {
    shift[j] = plan.shift[j];
    mask[j] = plan.mask[j];
  }

  auto count_key = [&](K k) {
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const uint32_t d = (sizeof(K) <= 4 ? (uint32_t(k) >> shift[j]) : uint32_t(uint64_t(k) >> shift[j])) & mask[j];
      atomicAdd(&counts[j * kRadix + d], 1u);
    }
  };

  // Two 16-byte loads in flight per thread per iteration.
  uint64_t v = v_lo + threadIdx.x;
  for (; v + blockDim.x < v_hi; v += 2 * blockDim.x) {
    const uint64_t e0 = v * kVec, e1 = e0 + uint64_t(blockDim.x) * kVec;
    if (e1 + kVec > n) break;
    const uint4 q0 = __ldg(reinterpret_cast<const uint4*>(keys + e0));
    const uint4 q1 = __ldg(reinterpret_cast<const uint4*>(keys + e1));
    const K* k0 = reinterpret_cast<const K*>(&q0);
    const K* k1 = reinterpret_cast<const K*>(&q1);
#pragma unroll
    for (int e = 0; e < int(kVec); ++e) count_key(k0[e]);
#pragma unroll
    for (int e = 0; e < int(kVec); ++e) count_key(k1[e]);
  }
  for (; v < v_hi; v += blockDim.x) {
    const uint64_t e0 = v * kVec;
    if (e0 + kVec <= n) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(keys + e0));
      const K* kk = reinterpret_cast<const K*>(&q);
#pragma unroll
      for (int e = 0; e < int(kVec); ++e) count_key(kk[e]);
    } else {
      for (uint64_t e = e0; e < n; ++e) count_key(keys[e]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P * kRadix; i += blockDim.x) {
    const uint32_t c = counts[i];
    if (c) {
      const int j = i / kRadix, d = i % kRadix;
      atomicAdd(reinterpret_cast<unsigned long long*>(&hist[j * pass_stride + d]), (unsigned long long)c);
    }
  }
}

// ---------------------------------------------------------------- K2 -------
// 256 threads, thread d owns digit d.  For each pass: a block-wide exclusive
// scan over the digit totals (the rank of every leaf, Alg. 3) gives the 64-bit
// bases of the first look-back chunk; the scatter itself chains the bases of
// later chunks, whose key sets are only known once the previous pass has
// permuted the keys.  A pass whose keys all share one digit is trivial (its stable scatter
// is the identity) and is marked inactive.  Thread 0 then routes the active
// passes through the input, scratch and output buffers so that the last one
// writes the output, adding a final copy only when no assignment can.
__device__ uint64_t block_exclusive_scan_256(uint64_t x, uint64_t* s_warp, uint64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  uint64_t before = 0, all = 0;
  for (int w = 0; w < 8; ++w) {
    if (w < warp) before += s_warp[w];
    all += s_warp[w];
  }
  __syncthreads();
  *total = all;
  return before + inc - x;
}

__global__ void __launch_bounds__(kRadix) scan_schedule_kernel(uint64_t* __restrict__ hist,
                                                               uint64_t* __restrict__ chunk_base,
                                                               uint32_t* __restrict__ chunk_flag, int passes,
                                                               uint32_t chunks, int in_place, Schedule* sched) {
  __shared__ uint64_t s_warp[8];
  __shared__ int s_trivial[kMaxPasses];
  const int d = threadIdx.x;
  for (int j = 0; j < passes; ++j) {
    uint64_t* h = hist + uint64_t(j) * kRadix;
    const uint64_t tot = h[d];
    h[d] = 0;  // leave the accumulator zero for the next call
    uint64_t all;
    const uint64_t excl = block_exclusive_scan_256(tot, s_warp, &all);
    const int nonzero = __syncthreads_count(tot != 0);
    if (d == 0) s_trivial[j] = (nonzero <= 1);
    chunk_base[uint64_t(j) * chunks * kRadix + d] = excl;
    for (uint32_t c = d; c < chunks; c += kRadix) chunk_flag[uint64_t(j) * chunks + c] = 0;
  }
  __syncthreads();
  if (d == 0 && sched) route_passes(s_trivial, passes, in_place, sched);
}

// Generic row-wise exclusive scan: one CTA of 1024 threads per row.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) scan_rows_kernel(const uint64_t* __restrict__ in,
                                                                 uint64_t* __restrict__ out, uint64_t bins) {
  __shared__ uint64_t s_warp[32];
  const uint64_t* r_in = in + blockIdx.x * bins;
  uint64_t* r_out = out + blockIdx.x * bins;
  const uint64_t per = (bins + kScanThreads - 1) / kScanThreads;
  const uint64_t lo = threadIdx.x * per;
  const uint64_t hi = (lo + per < bins) ? lo + per : bins;
  uint64_t sum = 0;
  for (uint64_t i = lo; i < hi; ++i) sum += r_in[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  uint64_t before = 0;
  for (int w = 0; w < warp; ++w) before += s_warp[w];
  uint64_t run = before + inc - sum;
  for (uint64_t i = lo; i < hi; ++i) {
    const uint64_t c = r_in[i];
    r_out[i] = run;
    run += c;
  }
}

// dst[i] = src[i] for i < nv (16-byte vectors, distinct buffers), grid-stride,
// four loads in flight per thread before their stores, with streaming hints
// (neither side is read again soon).
__device__ __forceinline__ void copy_vectors(uint4* __restrict__ dst, const uint4* __restrict__ src, uint64_t nv,
                                             uint64_t tid, uint64_t stride) {
  constexpr int kInFlight = 4;
  uint64_t i = tid;
  for (; i + (kInFlight - 1) * stride < nv; i += kInFlight * stride) {
    uint4 r[kInFlight];
#pragma unroll
    for (int u = 0; u < kInFlight; ++u) r[u] = __ldcs(&src[i + u * stride]);
#pragma unroll
    for (int u = 0; u < kInFlight; ++u) __stcs(&dst[i + u * stride], r[u]);
  }
  for (; i < nv; i += stride) __stcs(&dst[i], __ldcs(&src[i]));
}

// Final copy of keys (and values) between buffers when the schedule asks.
template <typename K>
__global__ void __launch_bounds__(256, 4) schedule_copy_kernel(const K* k0, const K* k1, const K* k2, const uint32_t* v0, const uint32_t* v1,
                                     const uint32_t* v2, uint64_t n, const Schedule* sched) {
  const PassDesc cp = sched->copy;
  if (!cp.active) return;
  // buffers chosen without indexing a local array (which would live in local memory)
  const K* src = cp.src == 0 ? k0 : (cp.src == 1 ? k1 : k2);
  K* dst = const_cast<K*>(cp.dst == 0 ? k0 : (cp.dst == 1 ? k1 : k2));
  const uint32_t* vsrc = cp.src == 0 ? v0 : (cp.src == 1 ? v1 : v2);
  uint32_t* vdst = const_cast<uint32_t*>(cp.dst == 0 ? v0 : (cp.dst == 1 ? v1 : v2));
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  constexpr uint64_t kVec = 16 / sizeof(K);
  const uint64_t nv = n / kVec;
  copy_vectors(reinterpret_cast<uint4*>(dst), reinterpret_cast<const uint4*>(src), nv, tid, stride);
  for (uint64_t i = nv * kVec + tid; i < n; i += stride) dst[i] = src[i];
  if (vsrc && vdst) {
    const uint64_t nv4 = n / 4;
    copy_vectors(reinterpret_cast<uint4*>(vdst), reinterpret_cast<const uint4*>(vsrc), nv4, tid, stride);
    for (uint64_t i = nv4 * 4 + tid; i < n; i += stride) vdst[i] = vsrc[i];
  }
}

// --------------------------------------------------------------- K1' -------
// 65,536 counters of 16 bits, two per 32-bit shared-memory word (128 KB):
// word w holds key w in its low half and key w + 32768 in its high half, so
// the small, frequent keys of skewed inputs sit in different words.
//
// Overflow is exact (the tapered width of Sec. III-D-1 with an exact spill):
// every addition returns the counter's old value, and the one addition that
// takes a counter from below 2^14 to 2^14 subtracts 2^14 from it and adds 2^14
// to the key's global 64-bit spill counter.  Every round ends at a block
// barrier, after which every counter is below 2^14 (each crossing's
// subtraction comes before its thread's barrier); a round adds at most
// kLeafRound = 32,768 keys to any counter, so a counter stays below
// 2^14 + 32,768 < 2^16 (no carry into the neighbouring half).  No pass over
// the table is needed (an earlier form read all 128 KB every 49,152 keys to
// move large counts out).
constexpr int kLeafThreads = 1024;
constexpr int kLeafWords = 32768;
constexpr int kLeafVecPerThread = 4;                                   // uint4 = 8 keys each
constexpr int kLeafRound = kLeafThreads * kLeafVecPerThread * 8;       // 32,768 keys
constexpr uint32_t kLeafSpill = 0x4000u;                               // 2^14: moved to the spill on crossing
static_assert(kLeafSpill + kLeafRound <= 65535, "a round must not carry a counter into its neighbour");

__global__ void __launch_bounds__(kLeafThreads, 1) leaf_hist_kernel(const uint16_t* __restrict__ keys, uint64_t n,
                                                                    uint32_t* __restrict__ partials,
                                                                    unsigned long long* __restrict__ spill) {
  extern __shared__ uint32_t hw[];
  for (int i = threadIdx.x; i < kLeafWords; i += blockDim.x) hw[i] = 0;
  __syncthreads();
  // Rounds are dealt to CTAs round-robin over the whole input; the next
  // round's keys are loaded into registers before this round's keys are
  // counted, so the loads overlap the counting.
  const uint64_t rounds = (n + kLeafRound - 1) / kLeafRound;
  auto add = [&](uint32_t k) {
    const uint32_t sh = (k >> 15) * 16;
    const uint32_t old = (atomicAdd(&hw[k & 32767u], 1u << sh) >> sh) & 0xFFFFu;
    if (old == kLeafSpill - 1u) {  // this addition took the counter to kLeafSpill
      atomicSub(&hw[k & 32767u], kLeafSpill << sh);
      atomicAdd(&spill[k], (unsigned long long)kLeafSpill);
    }
  };
  auto full = [&](uint64_t r) { return (r + 1) * kLeafRound <= n; };
  uint4 q[kLeafVecPerThread];
  auto load = [&](uint64_t r) {
#pragma unroll
    for (int u = 0; u < kLeafVecPerThread; ++u)
      q[u] = __ldg(reinterpret_cast<const uint4*>(keys + r * kLeafRound) + u * kLeafThreads + threadIdx.x);
  };
  uint64_t r = blockIdx.x;
  if (r < rounds && full(r)) load(r);
  for (; r < rounds; r += gridDim.x) {
    const uint64_t next = r + gridDim.x;
    if (full(r)) {
      uint4 cur[kLeafVecPerThread];
#pragma unroll
      for (int u = 0; u < kLeafVecPerThread; ++u) cur[u] = q[u];
      if (next < rounds && full(next)) load(next);
#pragma unroll
      for (int u = 0; u < kLeafVecPerThread; ++u) {
        const uint32_t w[4] = {cur[u].x, cur[u].y, cur[u].z, cur[u].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          add(w[e] & 0xFFFFu);
          add(w[e] >> 16);
        }
      }
    } else {
      for (uint64_t i = r * kLeafRound + threadIdx.x; i < n; i += blockDim.x) add(keys[i]);
    }
    __syncthreads();  // every counter is below kLeafSpill again (see above)
  }
  for (int i = threadIdx.x; i < kLeafWords; i += blockDim.x) partials[uint64_t(blockIdx.x) * kLeafWords + i] = hw[i];
}

// counts[k] = spill[k] + the CTAs' partial counters of key k (word k & 32767,
// low half for k < 32768, high half above).
__global__ void leaf_reduce_kernel(const uint32_t* __restrict__ partials, const uint64_t* __restrict__ spill,
                                   int grid, uint64_t* __restrict__ counts) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= kLeafWords) return;
  uint64_t lo = spill[w], hi = spill[w + 32768];
  for (int c = 0; c < grid; ++c) {
    const uint32_t x = partials[uint64_t(c) * kLeafWords + w];
    lo += x & 0xFFFFu;
    hi += x >> 16;
  }
  counts[w] = lo;
  counts[w + 32768] = hi;
}

// ---------------------------------------------------------------- K4 -------
// Output-centric and persistent: CTA c writes one contiguous stretch of the
// output.  Thread 0 finds the bins of the stretch's first and last position by
// binary search over the 65,536 bin starts; each thread then writes 8
// consecutive keys per step (one 16-byte store, the warp's stores contiguous)
// and follows the bin boundary forward as its positions advance.
constexpr int kExpandThreads = 256;
constexpr int kExpandPerThread = 8;
constexpr uint64_t kExpandStep = uint64_t(kExpandThreads) * kExpandPerThread;  // keys per CTA step

__device__ __forceinline__ uint32_t bin_of(const uint64_t* off, uint32_t lo, uint32_t hi, uint64_t pos) {
  // largest v in [lo, hi] with off[v] <= pos (off ascending, off[lo] <= pos)
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= pos) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kExpandThreads) expand_kernel(const uint64_t* __restrict__ offsets,
                                                                uint16_t* __restrict__ out, uint64_t n,
                                                                uint64_t per_cta) {
  __shared__ uint32_t s_range[2];
  const uint64_t c0 = uint64_t(blockIdx.x) * per_cta;
  if (c0 >= n) return;
  const uint64_t c1 = (c0 + per_cta < n) ? c0 + per_cta : n;
  if (threadIdx.x == 0) {
    s_range[0] = bin_of(offsets, 0, 65535, c0);
    s_range[1] = bin_of(offsets, s_range[0], 65535, c1 - 1);
  }
  __syncthreads();
  const uint32_t b_lo = s_range[0], b_hi = s_range[1];
  uint64_t p0 = c0 + uint64_t(threadIdx.x) * kExpandPerThread;
  if (p0 >= c1) return;
  uint32_t b = bin_of(offsets, b_lo, b_hi, p0);
  uint64_t next = (b < 65535) ? offsets[b + 1] : n;
  for (; p0 < c1; p0 += kExpandStep) {
    while (p0 >= next) {  // positions only move forward: walk to the bin holding p0
      ++b;
      next = (b < 65535) ? offsets[b + 1] : n;
    }
    if (p0 + kExpandPerThread <= c1 && p0 + kExpandPerThread <= next) {
      const uint32_t v2 = uint32_t(b) | (uint32_t(b) << 16);  // all 8 keys in one bin
      *reinterpret_cast<uint4*>(out + p0) = make_uint4(v2, v2, v2, v2);
    } else {
      uint16_t v[kExpandPerThread];
      uint32_t bb = b;
      uint64_t nx = next;
#pragma unroll
      for (int e = 0; e < kExpandPerThread; ++e) {
        while (p0 + e >= nx && bb < 65535) {
          ++bb;
          nx = (bb < 65535) ? offsets[bb + 1] : n;
        }
        v[e] = uint16_t(bb);
      }
      if (p0 + kExpandPerThread <= c1) {
        uint4 qv;
        qv.x = uint32_t(v[0]) | (uint32_t(v[1]) << 16);
        qv.y = uint32_t(v[2]) | (uint32_t(v[3]) << 16);
        qv.z = uint32_t(v[4]) | (uint32_t(v[5]) << 16);
        qv.w = uint32_t(v[6]) | (uint32_t(v[7]) << 16);
        *reinterpret_cast<uint4*>(out + p0) = qv;
      } else {
        for (int e = 0; e < kExpandPerThread && p0 + e < c1; ++e) out[p0 + e] = v[e];
      }
    }
  }
}

}  // namespace

// ------------------------------------------------------------ launchers ----

template <typename K, int P>
void launch_hist_typed(unsigned grid, cudaStream_t stream, const void* keys, uint64_t n, const DigitPlan& plan,
                       uint64_t* hist, uint64_t pass_stride, uint32_t* clear, uint64_t clear_words) {
  hist_kernel<K, P><<<grid, kHistThreads, 0, stream>>>(static_cast<const K*>(keys), n, plan, hist, pass_stride,
                                                       clear, clear_words);
}

template <typename K>
cudaError_t launch_hist_passes(unsigned grid, cudaStream_t stream, const void* keys, uint64_t n,
                               const DigitPlan& plan, uint64_t* hist, uint64_t pass_stride, uint32_t* clear,
                               uint64_t clear_words) {
#define FSORT_HIST_CASE(P_)                                                                          \
  case P_:                                                                                           \
    launch_hist_typed<K, P_>(grid, stream, keys, n, plan, hist, pass_stride, clear, clear_words); \
    break;
  switch (plan.passes) {
    FSORT_HIST_CASE(1)
    FSORT_HIST_CASE(2)
    FSORT_HIST_CASE(3)
    FSORT_HIST_CASE(4)
    FSORT_HIST_CASE(5)
    FSORT_HIST_CASE(6)
    FSORT_HIST_CASE(7)
    FSORT_HIST_CASE(8)
    default:
      return cudaErrorInvalidValue;
  }
#undef FSORT_HIST_CASE
  return cudaGetLastError();
}

cudaError_t launch_histogram(const void* keys, int key_bits, uint64_t n, const DigitPlan& plan, uint64_t* hist,
                             uint64_t pass_stride, uint32_t* clear, uint64_t clear_words, int sms,
                             cudaStream_t stream) {
  // About four resident CTAs per SM, at least 4096 keys each, at least 16 CTAs.
  uint64_t grid = uint64_t(sms) * 4;
  const uint64_t useful = (n + 8 * kHistThreads - 1) / (8 * kHistThreads);
  if (grid > useful) grid = useful;
  if (grid < 16) grid = 16;
  switch (key_bits) {
    case 16: return launch_hist_passes<uint16_t>(unsigned(grid), stream, keys, n, plan, hist, pass_stride, clear,
                                                 clear_words);
    case 32: return launch_hist_passes<uint32_t>(unsigned(grid), stream, keys, n, plan, hist, pass_stride, clear,
                                                 clear_words);
    case 64: return launch_hist_passes<uint64_t>(unsigned(grid), stream, keys, n, plan, hist, pass_stride, clear,
                                                 clear_words);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_scan_schedule(uint64_t* hist, uint64_t* chunk_base, uint32_t* chunk_flag, int passes,
                                 uint32_t chunks, int in_place, Schedule* sched, cudaStream_t stream) {
  scan_schedule_kernel<<<1, kRadix, 0, stream>>>(hist, chunk_base, chunk_flag, passes, chunks, in_place, sched);
  return cudaGetLastError();
}

cudaError_t launch_scan_rows(const uint64_t* in, uint64_t* out, uint64_t rows, uint64_t bins, cudaStream_t stream) {
  if (!rows || !bins) return cudaSuccess;
  scan_rows_kernel<<<unsigned(rows), kScanThreads, 0, stream>>>(in, out, bins);
  return cudaGetLastError();
}

cudaError_t launch_schedule_copy(const void* const keys[3], const uint32_t* const vals[3], int key_bits,
                                 bool has_vals, uint64_t n, const Schedule* sched, int sms, cudaStream_t stream) {
  const unsigned grid = unsigned(sms) * 4;  // all resident at once (256 threads, four CTAs per SM)
  const uint32_t* v0 = has_vals ? vals[0] : nullptr;
  const uint32_t* v1 = has_vals ? vals[1] : nullptr;
  const uint32_t* v2 = has_vals ? vals[2] : nullptr;
  switch (key_bits) {
    case 16:
      schedule_copy_kernel<uint16_t><<<grid, 256, 0, stream>>>(
          static_cast<const uint16_t*>(keys[0]), static_cast<const uint16_t*>(keys[1]),
          static_cast<const uint16_t*>(keys[2]), v0, v1, v2, n, sched);
      break;
    case 32:
      schedule_copy_kernel<uint32_t><<<grid, 256, 0, stream>>>(
          static_cast<const uint32_t*>(keys[0]), static_cast<const uint32_t*>(keys[1]),
          static_cast<const uint32_t*>(keys[2]), v0, v1, v2, n, sched);
      break;
    case 64:
      schedule_copy_kernel<uint64_t><<<grid, 256, 0, stream>>>(
          static_cast<const uint64_t*>(keys[0]), static_cast<const uint64_t*>(keys[1]),
          static_cast<const uint64_t*>(keys[2]), v0, v1, v2, n, sched);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int leaf_hist_grid(int sms) { return sms; }

cudaError_t launch_leaf_histogram(const uint16_t* keys, uint64_t n, uint32_t* partials, uint64_t* spill, int sms,
                                  cudaStream_t stream) {
  const size_t smem = size_t(kLeafWords) * 4;
  static const cudaError_t attr = set_smem_attrs(leaf_hist_kernel, smem, false);
  if (attr != cudaSuccess) return attr;
  cudaError_t e = cudaMemsetAsync(spill, 0, sizeof(uint64_t) * 65536, stream);
  if (e != cudaSuccess) return e;
  leaf_hist_kernel<<<leaf_hist_grid(sms), kLeafThreads, smem, stream>>>(
      keys, n, partials, reinterpret_cast<unsigned long long*>(spill));
  return cudaGetLastError();
}

cudaError_t launch_leaf_reduce(const uint32_t* partials, const uint64_t* spill, int grid, uint64_t* counts,
                               cudaStream_t stream) {
  leaf_reduce_kernel<<<kLeafWords / 256, 256, 0, stream>>>(partials, spill, grid, counts);
  return cudaGetLastError();
}

cudaError_t launch_expand(const uint64_t* offsets, uint16_t* keys_out, uint64_t n, cudaStream_t stream) {
  if (!n) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // Eight CTAs per SM, each a stretch that is a whole number of 16-byte steps.
  const uint64_t want = uint64_t(sms) * 8;
  uint64_t per = (n + want - 1) / want;
  per = (per + kExpandStep - 1) / kExpandStep * kExpandStep;
  const uint64_t grid = (n + per - 1) / per;
  expand_kernel<<<unsigned(grid), kExpandThreads, 0, stream>>>(offsets, keys_out, n, per);
  return cudaGetLastError();
}

}  // namespace fsort
