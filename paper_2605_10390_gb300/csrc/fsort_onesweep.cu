// fsort_onesweep.cu -- K3, the stable scatter of one radix pass (Sec. II:
// "stable scatter"), in a single read and write of keys and values.
//
// One CTA per tile of kTile consecutive keys, tiles taken in order from a
// dynamic counter so that a tile only ever waits for tiles already running.
//
//  1. A bulk async copy (cp.async.bulk + mbarrier) stages the tile's keys and
//     values in shared memory.
//  2. Stable rank within each warp's strip of the tile: for every round of 32
//     keys, the lanes that share a digit form a group (the __match_any_sync
//     peer mask, found through two small warp-private tables, see
//     digit_group); the group's winner adds the group size to the warp's digit
//     counter and broadcasts the old value; a lane's rank is that value plus
//     its peers below it.  (The hardware match.any instruction computes the
//     same mask but measured 6-7x slower on uniform 8-bit digits on GB300.)
//  3. Warp counters -> per-warp exclusive prefixes and the tile's digit counts,
//     published at once to the decoupled look-back (2-bit flag | 30-bit count,
//     the tapered counter width of Sec. III-D-1: a chunk never holds 2^30 keys).
//  4. Keys are permuted into digit order inside shared memory, each with its
//     source position (values are gathered through it when written out).
//  5. The look-back reads a window of predecessor tiles at a time (bounded
//     wait) to find each digit's exclusive prefix among earlier tiles of the
//     chunk, and publishes its inclusive prefix.  The 64-bit base of the chunk
//     comes from the scan (chunk 0) or from the last tile of the previous chunk,
//     which publishes the next chunk's bases (a 64-bit running total per digit)
//     once its own prefix is known.
//  6. The staged tile is written out in digit runs, consecutive threads to
//     consecutive addresses.
#include <cstdint>
#include <cuda_runtime.h>

#include "fsort_dev.cuh"
#include "fsort_internal.h"
#include "fsort_rank.cuh"

namespace fsort {
namespace {

constexpr int kRadix = 256;  // threads 0..255 own one digit each in the per-digit steps
constexpr int kWindow = 16;  // predecessor tiles read per look-back round trip

// Threads per CTA, keys per thread, and the CTAs per SM the register budget
// is sized for.  Two 16-warp CTAs per SM keep 32 ranking chains of kIpt
// items in flight per SM.
template <typename K>
struct TileShape;
template <>
struct TileShape<uint16_t> { static constexpr int kBlock = 512, kIpt = 16, kMinBlocks = 2; };
template <>
struct TileShape<uint32_t> { static constexpr int kBlock = 512, kIpt = 12, kMinBlocks = 2; };
template <>
struct TileShape<uint64_t> { static constexpr int kBlock = 512, kIpt = 8, kMinBlocks = 2; };

template <typename K, bool kVals>
struct SmemLayout {
  static constexpr int kBlock = TileShape<K>::kBlock;
  static constexpr int kIpt = TileShape<K>::kIpt;
  static constexpr int kTile = kBlock * kIpt;
  static constexpr int kWarps = kBlock / 32;
  static constexpr size_t kKeys = 0;
  static constexpr size_t kVals_ = kKeys + size_t(kTile) * sizeof(K);
  // records in digit order: 16-bit keys packed with their source position
  // (4 bytes), wider keys permuted in place plus a 16-bit source position
  static constexpr size_t kRec = kVals_ + (kVals ? size_t(kTile) * 4 : 0);
  static constexpr size_t kWcnt = kRec + (size_t(kTile) * (sizeof(K) == 2 ? 4 : 2) + 1023) / 1024 * 1024;
  static constexpr size_t kWin = kWcnt + size_t(kWarps) * kRadix * 4;  // digit-group tables (rank_strip_grouped)
  static constexpr size_t kGrp = kWin + size_t(kWarps) * kRadix;
  static constexpr size_t kExcl = kGrp + size_t(kWarps) * 32 * 4;
  static constexpr size_t kCnt = kExcl + kRadix * 4;
  static constexpr size_t kOff = kCnt + kRadix * 4;  // 8-byte aligned: all above are multiples of 1 KB
  static constexpr size_t kScan = kOff + kRadix * 8;
  static constexpr size_t kBar = kScan + 16 * 4;
  static constexpr size_t kTileId = kBar + 8;  // tile id, then a failed-wait flag
  static constexpr size_t kBytes = kTileId + 16;
};

// Look-back for digit d of `tile` (kWindow predecessors per round trip,
// bounded wait), publication of the tile's inclusive prefix, and the digit's
// 64-bit output offset s_off[d] = chunk base + exclusive prefix - tile
// position.  The last tile of a chunk hands the next chunk its bases.
// Returns false when a wait gave up (the device status records why).
__device__ __forceinline__ bool digit_offset(const OnesweepArgs& a, uint32_t tile, uint32_t chunk,
                                             uint32_t chunk_first, bool first_in_chunk, bool last_in_chunk,
                                             const unsigned long long* base_row, uint32_t d, uint32_t cnt,
                                             uint32_t tile_excl, uint32_t* lb, unsigned long long* s_off) {
  bool ok = true;
  uint32_t excl = 0;
  const uint64_t limit = a.wait_limit_ns ? a.wait_limit_ns : kWaitLimitNs;
  const bool publish = tile != a.withhold_tile;
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
        ok = false;
        break;
      }
      if (used < w) {  // blocked on an unpublished predecessor
        if (t_wait == 0) {
          t_wait = global_timer_ns();
        } else if (global_timer_ns() - t_wait > limit) {
          atomicOr(a.status, kDevTimeoutLookback);
          ok = false;
          break;
        } else if (ld_relaxed_gpu(a.status) & kDevTimeoutLookback) {  // another wait gave up: so do we
          ok = false;
          break;
        }
        __nanosleep(64);
      } else {
        t_wait = 0;
      }
    }
    if (publish) st_relaxed_gpu(lb + d, kFlagPrefix | (excl + cnt));
  }
  // 64-bit base of this digit in this chunk.
  unsigned long long base;
  if (base_row) {
    base = base_row[d];
  } else {
    const uint32_t* flag = a.chunk_flag + chunk;
    if (!ld_acquire_gpu(flag)) {
      const uint64_t t_wait = global_timer_ns();
      while (!ld_acquire_gpu(flag)) {
        if (global_timer_ns() - t_wait > limit) {
          atomicOr(a.status, kDevTimeoutLookback);
          ok = false;
          break;
        }
        if (ld_relaxed_gpu(a.status) & kDevTimeoutLookback) {
          ok = false;
          break;
        }
        __nanosleep(128);
      }
    }
    base = a.chunk_base[uint64_t(chunk) * kRadix + d];
  }
  s_off[d] = base + excl - tile_excl;
  if (last_in_chunk) {  // hand the next chunk its 64-bit bases
    a.chunk_base[uint64_t(chunk + 1) * kRadix + d] = base + excl + cnt;
    __threadfence();
  }
  return ok;
}

template <typename K, bool kVals>
__global__ void __launch_bounds__(TileShape<K>::kBlock, TileShape<K>::kMinBlocks)
    onesweep_kernel(const OnesweepArgs a) {
  using L = SmemLayout<K, kVals>;
  constexpr int kBlock = L::kBlock;
  constexpr int kIpt = L::kIpt;
  constexpr int kTile = L::kTile;
  constexpr int kWarps = L::kWarps;
  static_assert(kTile <= 65536, "in-warp ranks are kept in 16 bits");
  static_assert(sizeof(K) != 2 || kTile <= 65536, "packed records carry a 16-bit source position");
  extern __shared__ __align__(1024) unsigned char smem[];
  K* s_keys = reinterpret_cast<K*>(smem + L::kKeys);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(smem + L::kVals_);
  uint32_t* s_rec = reinterpret_cast<uint32_t*>(smem + L::kRec);
  uint32_t* s_wcnt = reinterpret_cast<uint32_t*>(smem + L::kWcnt);
  uint32_t* s_excl = reinterpret_cast<uint32_t*>(smem + L::kExcl);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + L::kCnt);
  unsigned long long* s_off = reinterpret_cast<unsigned long long*>(smem + L::kOff);
  uint32_t* s_scan = reinterpret_cast<uint32_t*>(smem + L::kScan);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + L::kBar);
  uint32_t* s_tile = reinterpret_cast<uint32_t*>(smem + L::kTileId);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

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
    s_tile[1] = 0;  // set when a bounded wait of this tile gave up
    mbar_init(s_bar, 1);
    fence_mbar_init();
  }
  for (int i = tid; i < kWarps * kRadix; i += kBlock) s_wcnt[i] = 0;
  __syncthreads();

  const uint32_t tile = *s_tile;
  if (tile >= gridDim.x) {  // counter not reset: never index past the look-back region
    if (tid == 0) atomicOr(a.status, kDevBadTile);
    return;
  }
  // Where this tile's keys live, where they go, and its look-back chunk.
  const K* kin;
  const uint32_t* vin;
  K* kout;
  uint32_t* vout;
  uint64_t t0, n_bound;
  uint32_t chunk, chunk_first;
  bool last_in_chunk;
  const unsigned long long* base_row;  // 64-bit digit bases of this tile's chunk, if already known
  if (a.segs) {
    const uint32_t seg = a.tile_seg[tile];
    const SegDesc sd = a.segs[seg];
    K* user_k = static_cast<K*>(sd.keys);
    K* alt_k = const_cast<K*>(static_cast<const K*>(a.keys[kBufAlt])) + sd.alt_off;
    uint32_t* alt_v = kVals ? const_cast<uint32_t*>(a.vals[kBufAlt]) + sd.alt_off : nullptr;
    const bool even = (a.pass & 1) == 0;
    kin = even ? user_k : alt_k;
    vin = even ? sd.vals : alt_v;
    kout = even ? alt_k : user_k;
    vout = even ? alt_v : sd.vals;
    t0 = uint64_t(tile - sd.first_tile) * kTile;
    n_bound = sd.n;
    chunk = seg;
    chunk_first = sd.first_tile;
    last_in_chunk = false;  // a segment is one chunk (< 2^30 keys)
    base_row = reinterpret_cast<const unsigned long long*>(a.chunk_base) + (uint64_t(seg) * a.passes + a.pass) * kRadix;
  } else {
    kin = static_cast<const K*>(a.keys[src]);
    vin = a.vals[src];
    kout = const_cast<K*>(static_cast<const K*>(a.keys[dst]));
    vout = const_cast<uint32_t*>(a.vals[dst]);
    t0 = uint64_t(tile) * kTile;
    n_bound = a.n;
    chunk = tile / a.tiles_per_chunk;
    chunk_first = chunk * a.tiles_per_chunk;
    last_in_chunk = (tile - chunk_first == a.tiles_per_chunk - 1) && (tile + 1 < gridDim.x);
    base_row = chunk == 0 ? reinterpret_cast<const unsigned long long*>(a.chunk_base) : nullptr;
  }
  const uint32_t tile_n = uint32_t((n_bound - t0 < uint64_t(kTile)) ? (n_bound - t0) : uint64_t(kTile));

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
  // A copy that has not landed within the bound: the tile still ranks and
  // publishes (so that later tiles do not wait on it) but writes nothing.
  const bool landed = mbar_wait_bounded(s_bar, 0);
  if (!landed) {
    atomicOr(a.status, kDevTimeoutLoad);
    s_tile[1] = 1;
  }
  __syncthreads();

  // 2. stable in-warp ranks
  const uint32_t shift = a.shift, mask = a.mask;
  (void)lane;
  uint32_t* wcnt = s_wcnt + warp * kRadix;
  const int wbase = warp * 32 * kIpt;
  Item<K> it[kIpt];
  rank_strip_grouped<K, kIpt>(s_keys, tile_n, wbase, shift, mask, reinterpret_cast<uint8_t*>(smem + L::kWin) + warp * kRadix,
                              reinterpret_cast<uint32_t*>(smem + L::kGrp) + warp * 32, wcnt, it);
  __syncthreads();

  // 3. per-digit: warp prefixes, tile count, publish, tile-exclusive prefix
  const bool first_in_chunk = tile == chunk_first;
  uint32_t* lb = a.lookback + uint64_t(tile) * kRadix;
  {
    const int d = tid;
    uint32_t run = 0;
    if (d < kRadix) {
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = s_wcnt[w * kRadix + d];
        s_wcnt[w * kRadix + d] = run;
        run += c;
      }
      s_cnt[d] = run;
      if (tile != a.withhold_tile) st_relaxed_gpu(lb + d, (first_in_chunk ? kFlagPrefix : kFlagAggregate) | run);
    }
    const uint32_t ex = digit_excl_scan<kBlock>(run, s_scan);
    if (d < kRadix) {
      s_excl[d] = ex;
      // warp offsets become tile positions: one lookup per key in the permute
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s_wcnt[w * kRadix + d] += ex;
    }
  }
  __syncthreads();

  // 4. permute into digit order in shared memory.  The record area holds the
  // sorted records: 16-bit keys packed with
  // their source position, wider keys in place plus a 16-bit source position.
  // Values stay where they are and are gathered once, in the output loop.
  uint32_t* s_rec32 = s_rec;
  uint16_t* s_src16 = reinterpret_cast<uint16_t*>(s_rec);
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    const int pos = wbase + i * 32 + lane;
    if (uint32_t(pos) < tile_n) {
      const K k = it[i].k();
      const uint32_t p = s_wcnt[warp * kRadix + dig(k, shift, mask)] + it[i].r();
      if (sizeof(K) == 2) {
        s_rec32[p] = uint32_t(k) | (uint32_t(pos) << 16);
      } else {
        s_keys[p] = k;
        s_src16[p] = uint16_t(pos);
      }
    }
  }

  // 5. decoupled look-back for digit d = tid, kWindow predecessors per round trip
  if (tid < kRadix)
    if (!digit_offset(a, tile, chunk, chunk_first, first_in_chunk, last_in_chunk, base_row, uint32_t(tid), s_cnt[tid],
                      s_excl[tid], lb, s_off))
      s_tile[1] = 1;
  __syncthreads();
  if (last_in_chunk && tid == 0) st_release_gpu(a.chunk_flag + chunk + 1, 1u);

  // 6. write the staged tile out in digit runs.  Without a failed wait every
  // offset is exact (each digit's run lies inside the output); after one the
  // tile writes nothing, so a partial prefix can never address past it.
  if (s_tile[1]) {
    if (tid == 0) atomicOr(a.status, kDevBadOutput);
    // a copy that had not landed gets a second bounded wait, so that it cannot
    // land in shared memory that another CTA has been given after this one exits
    if (!landed) mbar_wait_bounded(s_bar, 0);
    return;
  }
#pragma unroll 4
  for (uint32_t s = tid; s < tile_n; s += kBlock) {
    K k;
    uint32_t from;
    if (sizeof(K) == 2) {
      const uint32_t r = s_rec32[s];
      k = K(r & 0xFFFFu);
      from = r >> 16;
    } else {
      k = s_keys[s];
      from = s_src16[s];
    }
    const uint64_t o = s_off[dig(k, shift, mask)] + s;
    kout[o] = k;
    if (kVals) vout[o] = s_vals[from];
  }
}

template <typename K, bool kVals>
cudaError_t launch_typed(const OnesweepArgs& a, cudaStream_t stream) {
  using L = SmemLayout<K, kVals>;
  static const cudaError_t attr = set_smem_attrs(onesweep_kernel<K, kVals>, L::kBytes, true);
  if (attr != cudaSuccess) return attr;
  const uint64_t tiles = a.segs ? uint64_t(a.total_tiles) : (a.n + L::kTile - 1) / L::kTile;
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
