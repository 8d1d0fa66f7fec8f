// fsort_onesweep.cu -- K3, the stable scatter of one radix pass (Sec. II:
// "stable scatter"), in a single read and write of keys and values.
//
// One CTA per tile of kTile consecutive keys, tiles taken in order from a
// dynamic counter so that a tile only ever waits for tiles already running.
//
//  1. A bulk async copy (cp.async.bulk + mbarrier) stages the tile's keys and
//     values in shared memory.
//  2. The tile is stably sorted by the pass's 8-bit digit inside shared
//     memory with two counting passes on 4-bit halves of the digit (low half
//     first): each thread owns kIpt consecutive keys and counts them in sixteen
//     4-bit fields of one 64-bit register, a block-wide exclusive scan over
//     (nibble, thread) turns the counts into positions, and one scatter per
//     half moves (key, source index) records.  No shared-memory atomics or warp
//     votes are needed for stability: order within a thread is its key order,
//     and threads are scanned in order.  The tile's digit counts are gathered
//     on the way with shared-memory reductions.
//  3. The digit counts are published at once to the decoupled look-back
//     (2-bit flag | 30-bit count, the tapered counter width of Sec. III-D-1: a
//     chunk never holds 2^30 keys), and scanned into tile-local digit starts.
//  4. The look-back reads a window of predecessor tiles at a time (bounded
//     wait) to find each digit's exclusive prefix among earlier tiles of the
//     chunk, and publishes its inclusive prefix.  The 64-bit base of the chunk
//     comes from the scan (chunk 0) or from the last tile of the previous chunk,
//     which publishes the next chunk's bases (a 64-bit running total per digit)
//     once its own prefix is known.
//  5. The sorted tile is written out in digit runs, consecutive threads to
//     consecutive addresses; values are gathered through the source index.
#include <cstdint>
#include <cuda_runtime.h>

#include "fsort_dev.cuh"
#include "fsort_internal.h"

namespace fsort {
namespace {

constexpr int kRadix = 256;  // threads 0..255 own one digit each in the per-digit steps
constexpr int kNib = 16;     // bins of one 4-bit counting step
constexpr int kWindow = 16;  // predecessor tiles read per look-back round trip

// Threads per CTA and keys per thread (<= 15: per-thread counts live in 4-bit
// fields).  Two CTAs per SM.
template <typename K>
struct TileShape;
template <>
struct TileShape<uint16_t> { static constexpr int kBlock = 512, kIpt = 15, kMinBlocks = 2; };
template <>
struct TileShape<uint32_t> { static constexpr int kBlock = 512, kIpt = 15, kMinBlocks = 2; };
template <>
struct TileShape<uint64_t> { static constexpr int kBlock = 512, kIpt = 8, kMinBlocks = 2; };

// Sorted records: 16-bit keys travel packed with their 13-bit source index in
// one 32-bit word; wider keys stay in the input buffer and only a 16-bit
// source index moves.
template <typename K>
struct Rec {
  using T = uint16_t;
  static constexpr bool kPacked = false;
};
template <>
struct Rec<uint16_t> {
  using T = uint32_t;
  static constexpr bool kPacked = true;
};

template <typename K, bool kVals>
struct SmemLayout {
  static constexpr int kBlock = TileShape<K>::kBlock;
  static constexpr int kIpt = TileShape<K>::kIpt;
  static constexpr int kTile = kBlock * kIpt;
  using R = typename Rec<K>::T;
  static constexpr size_t align(size_t x) { return (x + 1023) / 1024 * 1024; }
  // Packed records reuse the input-key region (the keys are in registers by
  // the time the first scatter writes); otherwise records get their own.
  static constexpr size_t kKeys = 0;
  static constexpr size_t kKeyBytes = Rec<K>::kPacked ? size_t(kTile) * sizeof(R) : size_t(kTile) * sizeof(K);
  static constexpr size_t kRecs = Rec<K>::kPacked ? kKeys : align(kKeys + kKeyBytes);
  static constexpr size_t kVals_ = align(Rec<K>::kPacked ? kKeys + kKeyBytes : kRecs + size_t(kTile) * sizeof(R));
  static constexpr size_t kCnt16 = align(kVals_ + (kVals ? size_t(kTile) * 4 : 0));  // [16][kBlock] u16
  static constexpr size_t kHist = align(kCnt16 + size_t(kNib) * kBlock * 2);          // [256] u32
  static constexpr size_t kExcl = kHist + kRadix * 4;
  static constexpr size_t kOff = kExcl + kRadix * 4;  // 8-byte aligned
  static constexpr size_t kScan = kOff + kRadix * 8;  // 16 warp totals
  static constexpr size_t kBar = kScan + 16 * 4;
  static constexpr size_t kTileId = kBar + 8;
  static constexpr size_t kBytes = kTileId + 16;
};

// Exclusive scan of x over threads 0..255 (the digits); every thread of the
// block must call it (it contains a barrier).
__device__ __forceinline__ uint32_t digit_excl_scan(uint32_t x, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31 && warp < kRadix / 32) s_warp[warp] = inc;
  __syncthreads();
  uint32_t before = 0;
#pragma unroll
  for (int w = 0; w < kRadix / 32; ++w)
    if (w < warp) before += s_warp[w];
  return before + inc - x;
}

// In-place exclusive scan of the [16][kBlock] u16 count matrix in row-major
// order (nibble-major, then thread), i.e. the stable counting-sort positions.
// Thread t rakes the 16 consecutive entries [16t, 16t + 16).  Contains
// barriers; every thread calls it.
template <int kBlock>
__device__ __forceinline__ void scan_counts(uint16_t* cnt, uint32_t* s_warp) {
  static_assert(kNib * kBlock == 16 * kBlock, "one 16-entry segment per thread");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint4* seg = reinterpret_cast<uint4*>(cnt + 16 * tid);
  uint4 q0 = seg[0], q1 = seg[1];
  uint32_t w[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
  uint32_t total = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) total += (w[i] & 0xFFFFu) + (w[i] >> 16);
  uint32_t inc = total;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  uint32_t run = inc - total;
#pragma unroll
  for (int v = 0; v < kBlock / 32; ++v)
    if (v < warp) run += s_warp[v];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t lo = w[i] & 0xFFFFu, hi = w[i] >> 16;
    w[i] = run | ((run + lo) << 16);
    run += lo + hi;
  }
  seg[0] = make_uint4(w[0], w[1], w[2], w[3]);
  seg[1] = make_uint4(w[4], w[5], w[6], w[7]);
  __syncthreads();
}

template <typename K>
__device__ __forceinline__ uint32_t dig(K k, uint32_t shift, uint32_t mask) {
  if (sizeof(K) <= 4) return (uint32_t(k) >> shift) & mask;
  return uint32_t(uint64_t(k) >> shift) & mask;
}

// 4-bit field of a 64-bit counter word.
__device__ __forceinline__ uint32_t field4(uint64_t c, uint32_t v) { return uint32_t(c >> (4 * v)) & 15u; }

template <typename K, bool kVals>
__global__ void __launch_bounds__(TileShape<K>::kBlock, TileShape<K>::kMinBlocks)
    onesweep_kernel(const OnesweepArgs a) {
  using L = SmemLayout<K, kVals>;
  using R = typename L::R;
  constexpr bool kPacked = Rec<K>::kPacked;
  constexpr int kBlock = L::kBlock;
  constexpr int kIpt = L::kIpt;
  constexpr int kTile = L::kTile;
  static_assert(kIpt <= 15, "per-thread counts are 4-bit fields");
  static_assert(kTile <= 8192, "packed records carry a 13-bit source index");
  extern __shared__ __align__(1024) unsigned char smem[];
  K* s_keys = reinterpret_cast<K*>(smem + L::kKeys);
  R* s_rec = reinterpret_cast<R*>(smem + L::kRecs);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(smem + L::kVals_);
  uint16_t* s_cnt16 = reinterpret_cast<uint16_t*>(smem + L::kCnt16);
  uint32_t* s_hist = reinterpret_cast<uint32_t*>(smem + L::kHist);
  uint32_t* s_excl = reinterpret_cast<uint32_t*>(smem + L::kExcl);
  unsigned long long* s_off = reinterpret_cast<unsigned long long*>(smem + L::kOff);
  uint32_t* s_scan = reinterpret_cast<uint32_t*>(smem + L::kScan);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + L::kBar);
  uint32_t* s_tile = reinterpret_cast<uint32_t*>(smem + L::kTileId);

  const int tid = threadIdx.x;

  int src = kBufIn, dst = kBufOut, active = 1;
  if (a.sched) {
    const PassDesc pd = a.sched->pass[a.pass];
    active = pd.active;
    src = pd.src;
    dst = pd.dst;
  }
  // The next pass uses the other look-back region: clear this block's slot of
  // it (one block per tile, so the slots cover every tile) and its counter.
  if (a.next_lookback && tid < kRadix) a.next_lookback[uint64_t(blockIdx.x) * kRadix + tid] = 0;
  if (a.next_counter && blockIdx.x == 0 && tid == 0) *a.next_counter = 0;
  if (!active) return;

  if (tid == 0) {
    *s_tile = atomicAdd(a.tile_counter, 1u);
    mbar_init(s_bar, 1);
    fence_mbar_init();
  }
  if (tid < kRadix) s_hist[tid] = 0;
  __syncthreads();

  const uint32_t tile = *s_tile;
  if (tile >= gridDim.x) {  // counter not reset: never index past the look-back region
    if (tid == 0) atomicOr(a.status, kDevBadTile);
    return;
  }
  const uint64_t t0 = uint64_t(tile) * kTile;
  const uint32_t tile_n = uint32_t((a.n - t0 < uint64_t(kTile)) ? (a.n - t0) : uint64_t(kTile));
  const K* kin = static_cast<const K*>(a.keys[src]);
  const uint32_t* vin = a.vals[src];

  // 1. stage the tile: bulk copies for the 16-byte-aligned body, plain loads
  // for a ragged end.
  const uint32_t kbody = (tile_n * uint32_t(sizeof(K))) & ~15u;
  const uint32_t vbody = kVals ? ((tile_n * 4u) & ~15u) : 0u;
  if (tid == 0) {
    mbar_arrive_expect_tx(s_bar, kbody + vbody);
    if (kbody) bulk_copy_g2s(s_keys, kin + t0, kbody, s_bar);
    if (vbody) bulk_copy_g2s(s_vals, vin + t0, vbody, s_bar);
  }
  for (uint32_t i = kbody / sizeof(K) + tid; i < tile_n; i += kBlock) s_keys[i] = kin[t0 + i];
  if (kVals)
    for (uint32_t i = vbody / 4 + tid; i < tile_n; i += kBlock) s_vals[i] = vin[t0 + i];
  if (!mbar_wait_bounded(s_bar, 0)) atomicOr(a.status, kDevTimeoutLoad);
  __syncthreads();

  // 2. stable in-tile sort by the digit: two 4-bit counting steps.
  const uint32_t shift = a.shift, mask = a.mask;
  const uint32_t first = uint32_t(tid) * kIpt;  // this thread's keys [first, first + kIpt)
  R rec[kIpt];
  uint64_t c = 0;
  // Step A (low nibble), counting: key order within the thread is input order.
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    const uint32_t pos = first + i;
    const bool valid = pos < tile_n;
    const K k = valid ? s_keys[pos] : K(0);
    const uint32_t d = dig(k, shift, mask);
    if (valid) atomicAdd(&s_hist[d], 1u);  // tile digit counts (same-address adds combine)
    if (valid) c += 1ull << (4 * (d & 15u));
    if (kPacked) rec[i] = R(uint32_t(k) | (pos << 16));
    else rec[i] = R(pos);
  }
#pragma unroll
  for (int v = 0; v < kNib; ++v) s_cnt16[v * kBlock + tid] = uint16_t(field4(c, v));
  __syncthreads();
  scan_counts<kBlock>(s_cnt16, s_scan);
  // Scatter A.  For packed records this overwrites the input keys, all of
  // which were read before the barriers inside scan_counts.  The counter is
  // replayed to recover each key's rank within the thread.
  c = 0;
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    if (first + i < tile_n) {
      const K k = kPacked ? K(uint32_t(rec[i]) & 0xFFFFu) : s_keys[first + i];
      const uint32_t v = dig(k, shift, mask) & 15u;
      s_rec[s_cnt16[v * kBlock + tid] + field4(c, v)] = rec[i];
      c += 1ull << (4 * v);
    }
  }
  __syncthreads();
  // Step B (high nibble) over the low-nibble order.
  c = 0;
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    const uint32_t pos = first + i;
    const bool valid = pos < tile_n;
    const R r = valid ? s_rec[pos] : R(0);
    rec[i] = r;
    const K k = kPacked ? K(uint32_t(r) & 0xFFFFu) : s_keys[uint32_t(r)];
    if (valid) c += 1ull << (4 * ((dig(k, shift, mask) >> 4) & 15u));
  }
#pragma unroll
  for (int v = 0; v < kNib; ++v) s_cnt16[v * kBlock + tid] = uint16_t(field4(c, v));
  __syncthreads();
  scan_counts<kBlock>(s_cnt16, s_scan);
  c = 0;
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    if (first + i < tile_n) {
      const K k = kPacked ? K(uint32_t(rec[i]) & 0xFFFFu) : s_keys[uint32_t(rec[i])];
      const uint32_t v = (dig(k, shift, mask) >> 4) & 15u;
      s_rec[s_cnt16[v * kBlock + tid] + field4(c, v)] = rec[i];
      c += 1ull << (4 * v);
    }
  }

  // 3. per-digit: publish the tile's counts, tile-exclusive digit starts
  const uint32_t tpc = a.tiles_per_chunk;
  const uint32_t chunk = tile / tpc;
  const uint32_t chunk_first = chunk * tpc;
  const bool first_in_chunk = tile == chunk_first;
  const bool last_in_chunk = (tile - chunk_first == tpc - 1) && (tile + 1 < gridDim.x);
  uint32_t* lb = a.lookback + uint64_t(tile) * kRadix;
  uint32_t cnt = 0;
  if (tid < kRadix) {
    cnt = s_hist[tid];
    st_relaxed_gpu(lb + tid, (first_in_chunk ? kFlagPrefix : kFlagAggregate) | cnt);
  }
  {
    const uint32_t ex = digit_excl_scan(cnt, s_scan);
    if (tid < kRadix) s_excl[tid] = ex;
  }

  // 4. decoupled look-back for digit d = tid, kWindow predecessors per round trip
  if (tid < kRadix) {
    const int d = tid;
    uint32_t excl = 0;
    if (!first_in_chunk) {
      uint32_t t = tile;  // tiles [chunk_first, t) are still to the left
      uint64_t t_wait = 0;
      while (true) {
        const uint32_t left = t - chunk_first;
        const uint32_t w = left < uint32_t(kWindow) ? left : uint32_t(kWindow);
        uint32_t v[kWindow];
#pragma unroll
        for (int i = 0; i < kWindow; ++i)
          v[i] = (uint32_t(i) < w) ? ld_relaxed_gpu(a.lookback + uint64_t(t - 1 - i) * kRadix + d) : 0u;
        bool stop = false, found = false;
        uint32_t used = 0;
#pragma unroll
        for (int i = 0; i < kWindow; ++i) {
          if (!stop && uint32_t(i) < w) {
            const uint32_t f = v[i] & ~kCountMask;
            if (f == 0) {
              stop = true;  // not published yet: read again from here
            } else {
              excl += v[i] & kCountMask;
              ++used;
              if (f == kFlagPrefix) stop = found = true;
            }
          }
        }
        if (found) break;
        t -= used;
        if (t == chunk_first) {  // a chunk's first tile always publishes a prefix
          atomicOr(a.status, kDevBadLookback);
          break;
        }
        if (used < w) {  // blocked on an unpublished predecessor
          if (t_wait == 0) {
            t_wait = global_timer_ns();
          } else if (global_timer_ns() - t_wait > kWaitLimitNs) {
            atomicOr(a.status, kDevTimeoutLookback);
            break;
          }
          __nanosleep(64);
        } else {
          t_wait = 0;
        }
      }
      st_relaxed_gpu(lb + d, kFlagPrefix | (excl + cnt));
    }
    // 64-bit base of this digit in this chunk.
    unsigned long long base;
    if (chunk == 0) {
      base = a.chunk_base[d];
    } else {
      const uint32_t* flag = a.chunk_flag + chunk;
      if (!ld_acquire_gpu(flag)) {
        const uint64_t t_wait = global_timer_ns();
        while (!ld_acquire_gpu(flag)) {
          if (global_timer_ns() - t_wait > kWaitLimitNs) {
            atomicOr(a.status, kDevTimeoutLookback);
            break;
          }
          __nanosleep(128);
        }
      }
      base = a.chunk_base[uint64_t(chunk) * kRadix + d];
    }
    s_off[d] = base + excl - s_excl[d];
    if (last_in_chunk) {  // hand the next chunk its 64-bit bases
      a.chunk_base[uint64_t(chunk + 1) * kRadix + d] = base + excl + cnt;
      __threadfence();
    }
  }
  __syncthreads();
  if (last_in_chunk && tid == 0) st_release_gpu(a.chunk_flag + chunk + 1, 1u);

  // 5. write the sorted tile out in digit runs
  K* kout = const_cast<K*>(static_cast<const K*>(a.keys[dst]));
  uint32_t* vout = const_cast<uint32_t*>(a.vals[dst]);
  bool out_of_range = false;
#pragma unroll 4
  for (uint32_t s = tid; s < tile_n; s += kBlock) {
    const R r = s_rec[s];
    const uint32_t from = kPacked ? (uint32_t(r) >> 16) : uint32_t(r);
    const K k = kPacked ? K(uint32_t(r) & 0xFFFFu) : s_keys[from];
    const uint64_t o = s_off[dig(k, shift, mask)] + s;
    if (o >= a.n) {  // only reachable after a timed-out wait; never write outside the output
      out_of_range = true;
      continue;
    }
    kout[o] = k;
    if (kVals) vout[o] = s_vals[from];
  }
  if (out_of_range) atomicOr(a.status, kDevBadOutput);
}

template <typename K, bool kVals>
cudaError_t launch_typed(const OnesweepArgs& a, cudaStream_t stream) {
  using L = SmemLayout<K, kVals>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(onesweep_kernel<K, kVals>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(L::kBytes));
    if (e == cudaSuccess)  // all of the unified L1/shared capacity as shared memory
      e = cudaFuncSetAttribute(onesweep_kernel<K, kVals>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const uint64_t tiles = (a.n + L::kTile - 1) / L::kTile;
  if (!tiles) return cudaSuccess;
  onesweep_kernel<K, kVals><<<unsigned(tiles), L::kBlock, L::kBytes, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

int tile_keys_for(int key_bits) {
  switch (key_bits) {
    case 16: return SmemLayout<uint16_t, true>::kTile;
    case 32: return SmemLayout<uint32_t, true>::kTile;
    case 64: return SmemLayout<uint64_t, true>::kTile;
    default: return 0;
  }
}

uint64_t chunk_keys_for(int key_bits) {
  const uint64_t t = uint64_t(tile_keys_for(key_bits));
  return t ? (kMaxChunkKeys / t) * t : 0;
}

cudaError_t launch_onesweep(const OnesweepArgs& args, int key_bits, bool has_vals, cudaStream_t stream) {
  switch (key_bits) {
    case 16: return has_vals ? launch_typed<uint16_t, true>(args, stream) : launch_typed<uint16_t, false>(args, stream);
    case 32: return has_vals ? launch_typed<uint32_t, true>(args, stream) : launch_typed<uint32_t, false>(args, stream);
    case 64: return has_vals ? launch_typed<uint64_t, true>(args, stream) : launch_typed<uint64_t, false>(args, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fsort
