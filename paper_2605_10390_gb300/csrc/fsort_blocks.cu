// fsort_blocks.cu -- the scatter passes (Sec. II: "stable scatter") as
// reduce-then-scan over a table of per-tile digit offsets: no chain between
// tiles.
//
//  KT1 tile_count_kernel      one read of a pass's input, one CTA per chunk of
//                             consecutive tiles: for every tile the counts of
//                             each digit in the chunk's earlier tiles and in
//                             each of the tile's 16 warp strips, the chunk's
//                             totals, the pass's totals; on the first read of
//                             the input also the OR and AND of all keys
//  table_schedule_kernel      trivial passes (OR and AND agree on the digit)
//                             and the buffer routing
//  KT2 chunk_scan_kernel      per digit, the keys of lower digits plus the
//                             exclusive scan of the chunk totals (Alg. 3's rank
//                             of every leaf, split over chunks)
//  KT3 tile_scatter_kernel    one CTA per tile: bulk copy of keys and values
//                             into shared memory, the per-warp digit counts
//                             from KT1's strip table, the tile's digit
//                             prefixes, stable ranks placed
//                             straight into digit order in shared memory, and
//                             the write-out in digit runs at the tile's offsets
//                             (chunk offset + offset within the chunk).
//
// The tile-local steps follow the chained scatter (fsort_onesweep.cu); what
// differs is where a tile's digit offsets come from: the chained form waits
// for its predecessors' prefixes (decoupled look-back), this form reads them
// from a table that one read of the pass input (kb bytes per key) and a small
// scan made before the pass.  Tiles run in launch order, so the runs that
// neighbouring tiles write into the same output lines meet in L2 at about the
// same time.
#include <cstdint>
#include <cuda_runtime.h>

#include "fsort_dev.cuh"
#include "fsort_internal.h"
#include "fsort_rank.cuh"

namespace fsort {
namespace {

constexpr int kRadix = 256;
constexpr int kScanThreads = 1024;

// Scatter tiles: threads, keys per thread, CTAs per SM.  A tile's shared
// memory is 8 bytes per key for 16-bit keys with values (records, values)
// plus 17 KB; 23 keys per thread is the most two CTAs per SM can hold.
template <typename K>
struct TileShape;
template <>
struct TileShape<uint16_t> { static constexpr int kBlock = 512, kIpt = 22, kMinBlocks = 2; };
template <>
struct TileShape<uint32_t> { static constexpr int kBlock = 512, kIpt = 16, kMinBlocks = 2; };
template <>
struct TileShape<uint64_t> { static constexpr int kBlock = 512, kIpt = 12, kMinBlocks = 2; };

// Buffer `sel` of a by-BufSel triple, selected without indexing the
// parameter array (which would copy it to local memory).
template <typename T>
__device__ __forceinline__ T* pick(T* const (&b)[3], int sel) {
  return sel == kBufIn ? b[0] : (sel == kBufAlt ? b[1] : b[2]);
}

// ------------------------------------------------------------------ KT1 ----
// One digit (shift, mask) per launch.  CTA c walks the tiles of chunk c in
// order and writes for each tile the counts of its digits in the chunk's
// earlier tiles (tilerel[t][256]) and the digit counts of each of the tile's
// 16 strips (stripcnt[t][w][256], 16 bits: strip w is the keys KT3's warp w
// ranks, so KT3 needs no counting pass of its own), then the chunk's totals
// (chunksum[c][256]) and adds them to the pass's digit totals (totals[256],
// zero on entry).
// kOrAnd (the first read of the input) also folds every key into
// orand[0] |= k and orand[1] &= k: a pass is trivial (all keys share its
// digit) exactly when the two agree on the digit's bits, so the schedule needs
// no histogram of the other passes.  The chunk streams through kCountStages
// shared-memory buffers of one tile each, filled by bulk copies while earlier
// tiles are counted.  Each thread counts count_vecs 16-byte vectors of a full
// tile, so the count CTA has tile / (16-byte vector keys * count_vecs) threads.
constexpr int kCountStages = 3;

// Count CTAs per SM: two for 16-bit keys (3 x 22 KB of buffers and 32 KB of
// counters each), one for wider keys.
template <typename K>
__host__ __device__ constexpr int count_ctas_per_sm() { return sizeof(K) == 2 ? 2 : 1; }
template <typename K>
__host__ __device__ constexpr uint32_t count_tile_keys() {
  return uint32_t(TileShape<K>::kBlock) * TileShape<K>::kIpt;
}
// 16-byte vectors per count thread per tile: the fewest that keep the CTA at
// 1024 threads or fewer.
template <typename K>
__host__ __device__ constexpr int count_vecs() {
  return int((count_tile_keys<K>() / (16 / sizeof(K)) + 1023) / 1024);
}
template <typename K>
__host__ __device__ constexpr int count_threads() {
  return int(count_tile_keys<K>() / (16 / sizeof(K)) / count_vecs<K>());
}
template <typename K>
__host__ __device__ constexpr size_t count_smem_bytes() {
  return size_t(kCountStages) * count_tile_keys<K>() * sizeof(K);
}

// Key e of a 16-byte vector, by shifts (no address taken, so the vector stays
// in registers).
template <typename K>
__device__ __forceinline__ K vec_key(const uint4& q, int e) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
  if (sizeof(K) == 2) return K((w[e >> 1] >> ((e & 1) * 16)) & 0xFFFFu);
  if (sizeof(K) == 4) return K(w[e]);
  return K(uint64_t(w[2 * e]) | (uint64_t(w[2 * e + 1]) << 32));
}

template <typename K, bool kOrAnd>
__global__ void __launch_bounds__(count_threads<K>(), count_ctas_per_sm<K>()) tile_count_kernel(TileCountArgs a) {
  constexpr int kThreads = count_threads<K>();
  constexpr uint32_t kTileKeys = count_tile_keys<K>();
  constexpr uint32_t kVec = 16 / sizeof(K);
  static_assert(kThreads >= kRadix && kThreads % 32 == 0 && kThreads <= 1024, "one thread per digit");
  constexpr int kCountVecs = count_vecs<K>();
  static_assert(uint32_t(kThreads) * kVec * kCountVecs == kTileKeys, "threads cover a tile exactly");
  extern __shared__ __align__(128) unsigned char smem[];  // [kCountStages][tile keys]
  // Counts of one tile per strip and digit, tiles alternating between two
  // sets: the thread of digit d reads its 16 strip counts after the tile's
  // barrier and clears them, and the set is counted into again two tiles later
  // (after another barrier).
  constexpr uint32_t kStripKeys = 32u * uint32_t(TileShape<K>::kIpt);  // keys of one KT3 warp strip
  constexpr int kStrips = TileShape<K>::kBlock / 32;
  static_assert(kStrips == kTableStrips && kStripKeys % kVec == 0 && kStrips * kStripKeys == kTileKeys,
                "strips of whole vectors tile the tile");
  __shared__ __align__(128) uint32_t s_cnt[2][kStrips][kRadix];
  __shared__ uint64_t s_bar[kCountStages];
  __shared__ uint32_t s_fail[2];  // by tile parity: a tile reads only its own flag after its barrier
  K* buf = reinterpret_cast<K*>(smem);
  // The chunk: tiles [t_begin, t_end) of an array of n_keys keys; g_tile0 is
  // the global index (into tilerel) of tile t_begin.
  const K* keys;
  uint32_t t_begin, t_end, g_tile0;
  uint64_t n_keys;
  if (a.segs) {
    const SegDesc sd = a.segs[a.chunk_seg[blockIdx.x]];
    keys = (a.pass & 1) ? static_cast<const K*>(a.keys[kBufAlt]) + sd.alt_off : static_cast<const K*>(sd.keys);
    n_keys = sd.n;
    const uint32_t seg_tiles = uint32_t((sd.n + kTileKeys - 1) / kTileKeys);
    t_begin = (blockIdx.x - sd.first_chunk) * a.chunk_tiles;
    t_end = (t_begin + a.chunk_tiles < seg_tiles) ? t_begin + a.chunk_tiles : seg_tiles;
    g_tile0 = sd.first_tile + t_begin;
  } else {
    if (a.sched) {
      const PassDesc pd = a.sched->pass[a.pass];
      if (!pd.active) return;
      keys = static_cast<const K*>(pick(a.keys, pd.src));
    } else {
      keys = static_cast<const K*>(a.keys[kBufIn]);
    }
    n_keys = a.n;
    t_begin = blockIdx.x * a.chunk_tiles;
    t_end = (t_begin + a.chunk_tiles < a.tiles) ? t_begin + a.chunk_tiles : a.tiles;
    g_tile0 = t_begin;
  }
  const int tid = threadIdx.x;
  const uint32_t steps = t_end - t_begin;
  // step s counts tile t_begin + s: keys [e0, e1); its body of whole 16-byte vectors is copied in bulk
  auto step_range = [&](uint32_t st, uint64_t& e0, uint64_t& e1) {
    e0 = uint64_t(t_begin + st) * kTileKeys;
    e1 = (e0 + kTileKeys < n_keys) ? e0 + kTileKeys : n_keys;
  };
  auto issue = [&](uint32_t st) {  // thread 0 only
    uint64_t e0, e1;
    step_range(st, e0, e1);
    const uint32_t bytes = uint32_t((e1 - e0) * sizeof(K)) & ~15u;
    uint64_t* bar = &s_bar[st % kCountStages];
    mbar_arrive_expect_tx(bar, bytes);
    if (bytes) bulk_copy_g2s(buf + size_t(st % kCountStages) * kTileKeys, keys + e0, bytes, bar);
  };
  if (tid == 0) {
    for (int i = 0; i < kCountStages; ++i) mbar_init(&s_bar[i], 1);
    fence_mbar_init();
    s_fail[0] = s_fail[1] = 0;
    for (uint32_t st = 0; st < steps && st < uint32_t(kCountStages); ++st) issue(st);
  }
  for (int i = tid; i < 2 * kStrips * kRadix; i += kThreads) (&s_cnt[0][0][0])[i] = 0;
  __syncthreads();

  const uint32_t shift = a.shift, mask = a.mask;
  uint64_t k_or = 0, k_and = ~0ull;  // this thread's keys of ragged ends folded
  // Whole 16-byte vectors are folded word by word: w_or[h] / w_and[h] cover the
  // vector words of parity h (for 64-bit keys the low and high halves; for
  // narrower keys both hold whole keys, two 16-bit keys to a word).
  uint32_t w_or[2] = {0u, 0u}, w_and[2] = {~0u, ~0u};
  auto fold_vec = [&](const uint4& q) {
    if (kOrAnd) {
      w_or[0] |= q.x | q.z;
      w_or[1] |= q.y | q.w;
      w_and[0] &= q.x & q.z;
      w_and[1] &= q.y & q.w;
    }
  };
  uint32_t set = 0;
  auto count_key = [&](K k, uint32_t strip) { atomicAdd(&s_cnt[set][strip][dig(k, shift, mask)], 1u); };
  auto count_ragged = [&](K k, uint32_t strip) {
    count_key(k, strip);
    if (kOrAnd) {
      k_or |= uint64_t(k);
      k_and &= uint64_t(k);
    }
  };
  uint32_t acc = 0;  // thread d < 256: digit d in the chunk's tiles so far
  for (uint32_t st = 0; st < steps; ++st) {
    uint64_t e0, e1;
    step_range(st, e0, e1);
    const uint32_t keys_n = uint32_t(e1 - e0);
    const uint32_t body = (keys_n * uint32_t(sizeof(K)) & ~15u) / sizeof(K);
    if (!mbar_wait_bounded(&s_bar[st % kCountStages], (st / kCountStages) & 1u)) s_fail[st & 1u] = 1;
    const uint4* bv = reinterpret_cast<const uint4*>(buf + size_t(st % kCountStages) * kTileKeys);
    if (body == kTileKeys) {
#pragma unroll
      for (int j = 0; j < kCountVecs; ++j) {
        const uint32_t v = uint32_t(tid + j * kThreads);
        const uint4 q = bv[v];
        fold_vec(q);
        const uint32_t strip = v * kVec / kStripKeys;  // a vector lies in one strip
#pragma unroll
        for (int e = 0; e < int(kVec); ++e) count_key(vec_key<K>(q, e), strip);
      }
    } else {  // the last, short tile
      for (uint32_t v = tid; v < body / kVec; v += kThreads) {
        const uint4 q = bv[v];
        fold_vec(q);
        const uint32_t strip = v * kVec / kStripKeys;
#pragma unroll
        for (int e = 0; e < int(kVec); ++e) count_key(vec_key<K>(q, e), strip);
      }
      for (uint32_t i = body + tid; i < keys_n; i += kThreads) count_ragged(keys[e0 + i], i / kStripKeys);  // ragged end
    }
    __syncthreads();
    if (s_fail[st & 1u]) {  // the table would be wrong: mark it so that no scatter uses it
      if (tid == 0) atomicOr(a.status, kDevTimeoutLoad | kDevBadTable);
      // copies still in flight get a second bounded wait before this CTA exits
      if (tid == 0)
        for (uint32_t q = st; q < steps && q < st + kCountStages; ++q)
          mbar_wait_bounded(&s_bar[q % kCountStages], (q / kCountStages) & 1u);
      return;
    }
    if (tid < kRadix) {  // meanwhile the next tile counts into the other set
      const uint64_t g_tile = uint64_t(g_tile0 + st);
      a.tilerel[g_tile * kRadix + tid] = acc;
      uint16_t* sc = a.stripcnt + g_tile * (kStrips * kRadix) + tid;
      uint32_t c = 0;
#pragma unroll
      for (int w = 0; w < kStrips; ++w) {
        const uint32_t x = s_cnt[set][w][tid];
        s_cnt[set][w][tid] = 0;  // counted into again two tiles later, after another barrier
        sc[w * kRadix] = uint16_t(x);
        c += x;
      }
      acc += c;
    }
    if (tid == 0 && st + kCountStages < steps) {  // every thread has read this buffer (barrier above)
      fence_proxy_async_smem();
      issue(st + kCountStages);
    }
    set ^= 1u;
  }
  if (tid < kRadix) {
    a.chunksum[uint64_t(blockIdx.x) * kRadix + tid] = acc;
    if (acc && a.totals) atomicAdd(&a.totals[tid], acc);
  }
  if (kOrAnd) {
    if (sizeof(K) == 8) {
      k_or |= uint64_t(w_or[0]) | (uint64_t(w_or[1]) << 32);
      k_and &= uint64_t(w_and[0]) | (uint64_t(w_and[1]) << 32);
    } else {
      uint32_t o = w_or[0] | w_or[1], n = w_and[0] & w_and[1];
      if (sizeof(K) == 2) {
        o = (o | (o >> 16)) & 0xFFFFu;
        n = n & (n >> 16) & 0xFFFFu;
      }
      k_or |= uint64_t(o);
      k_and &= uint64_t(n) | (sizeof(K) == 2 ? ~0xFFFFull : ~0xFFFFFFFFull);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      k_or |= __shfl_xor_sync(0xffffffffu, k_or, o);
      k_and &= __shfl_xor_sync(0xffffffffu, k_and, o);
    }
    if ((tid & 31) == 0) {
      atomicOr(reinterpret_cast<unsigned long long*>(&a.orand[0]), (unsigned long long)k_or);
      atomicAnd(reinterpret_cast<unsigned long long*>(&a.orand[1]), (unsigned long long)k_and);
    }
  }
}

// ------------------------------------------------------------------ KT2 ----
// The schedule from the keys' OR and AND (one thread): pass j is trivial when
// no bit of its digit differs between keys; then the buffer routing.  Leaves
// the accumulators at OR = 0, AND = all ones for the next call.
__global__ void table_schedule_kernel(uint64_t* __restrict__ orand, DigitPlan plan, int in_place, Schedule* sched) {
  const uint64_t diff = orand[0] ^ orand[1];
  int trivial[kMaxPasses];
  for (int j = 0; j < kMaxPasses; ++j)
    trivial[j] = j < plan.passes ? (((diff >> plan.shift[j]) & uint64_t(plan.mask[j])) == 0) : 1;
  route_passes(trivial, plan.passes, in_place, sched);
  orand[0] = 0;
  orand[1] = ~0ull;
}

// One CTA per digit d: chunkoff[c][d] = (keys of digits below d, from the
// pass's totals) + (keys of digit d in chunks before c) (Alg. 3's rank of
// every leaf, split over chunks; 32-bit, exact modulo 2^32).
__global__ void __launch_bounds__(kScanThreads) chunk_scan_kernel(const uint32_t* __restrict__ sum,
                                                                  const uint32_t* __restrict__ totals,
                                                                  uint32_t chunks, const Schedule* sched,
                                                                  int32_t pass, uint32_t* __restrict__ off) {
  if (sched && !sched->pass[pass].active) return;
  __shared__ uint32_t s_warp[32];
  const int d = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // keys of the digits below d
  uint32_t below = threadIdx.x < uint32_t(d) ? totals[threadIdx.x] : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
  if (lane == 0) s_warp[warp] = below;
  __syncthreads();
  uint32_t running = 0;
#pragma unroll
  for (int w = 0; w < kRadix / 32; ++w) running += s_warp[w];
  __syncthreads();
  for (uint32_t c0 = 0; c0 < chunks; c0 += kScanThreads) {
    const uint32_t c = c0 + threadIdx.x;
    const uint32_t x = c < chunks ? sum[uint64_t(c) * kRadix + d] : 0u;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
      const uint32_t t = s_warp[w];
      before += w < warp ? t : 0u;
      all += t;
    }
    if (c < chunks) off[uint64_t(c) * kRadix + d] = running + before + inc - x;
    running += all;
    __syncthreads();
  }
}

// Segmented KT2, one CTA (256 threads, thread d = digit d) per segment: the
// segment's count of digit d is the sum over its chunks; its exclusive scan
// over the digits places the segment's digit runs, and each chunk's offset
// adds the counts of d in the segment's earlier chunks (offsets relative to
// the segment's start; a segment holds fewer than 2^31 keys).
__global__ void __launch_bounds__(kRadix) seg_chunk_scan_kernel(const uint32_t* __restrict__ sum,
                                                               const SegDesc* __restrict__ segs, uint32_t tile,
                                                               uint32_t chunk_tiles, uint32_t* __restrict__ off) {
  __shared__ uint32_t s_warp[kRadix / 32];
  const SegDesc sd = segs[blockIdx.x];
  const uint32_t d = threadIdx.x;
  const uint32_t seg_tiles = uint32_t((sd.n + tile - 1) / tile);
  const uint32_t c0 = sd.first_chunk, c1 = c0 + (seg_tiles + chunk_tiles - 1) / chunk_tiles;
  uint32_t total = 0;
  for (uint32_t c = c0; c < c1; ++c) total += sum[uint64_t(c) * kRadix + d];
  uint32_t run = digit_excl_scan<kRadix>(total, s_warp);
  for (uint32_t c = c0; c < c1; ++c) {
    const uint32_t x = sum[uint64_t(c) * kRadix + d];
    off[uint64_t(c) * kRadix + d] = run;
    run += x;
  }
}

// ------------------------------------------------------------------ KT3 ----
template <typename K, bool kVals>
struct TileSmem {
  static constexpr int kBlock = TileShape<K>::kBlock;
  static constexpr int kIpt = TileShape<K>::kIpt;
  static constexpr int kTile = kBlock * kIpt;
  static constexpr int kWarps = kBlock / 32;
  // The staged keys, later (16-bit keys) records key | source slot << 16 over
  // the keys and source areas together, or (wider keys) the keys in digit
  // order plus their 16-bit source slots; the staged values; per-warp digit
  // counters; per-warp digit-group tables (winner bytes, group masks); the
  // tile's output offsets; scan scratch; the copy barrier.
  static constexpr size_t kKeys = 0;
  static constexpr size_t kSrc = kKeys + size_t(kTile) * sizeof(K);
  static constexpr size_t kVals_ = kSrc + size_t(kTile) * 2;
  static constexpr size_t kWcnt = kVals_ + (kVals ? size_t(kTile) * 4 : 0);
  static constexpr size_t kWin = kWcnt + size_t(kWarps) * kRadix * 4;
  static constexpr size_t kGrp = kWin + size_t(kWarps) * kRadix;
  static constexpr size_t kOff = kGrp + size_t(kWarps) * 32 * 4;
  static constexpr size_t kScan = kOff + kRadix * 4;
  static constexpr size_t kBar = kScan + 16 * 4;
  static constexpr size_t kBytes = kBar + 16;
};

// Compile-time flag for code paths that differ only for a short last tile.
template <bool B>
struct FullTile {
  static constexpr bool value = B;
};

// kIpt keys of one thread in registers; 16-bit keys two to a word.
template <typename K, int kIpt>
struct KeyRegs {
  K k[kIpt];
  __device__ __forceinline__ void set(int i, K v) { k[i] = v; }
  __device__ __forceinline__ K get(int i) const { return k[i]; }
};
template <int kIpt>
struct KeyRegs<uint16_t, kIpt> {
  uint32_t w[(kIpt + 1) / 2];
  __device__ __forceinline__ void set(int i, uint16_t v) {
    if (i & 1) w[i >> 1] |= uint32_t(v) << 16;
    else w[i >> 1] = v;
  }
  __device__ __forceinline__ uint16_t get(int i) const { return uint16_t((i & 1) ? (w[i >> 1] >> 16) : (w[i >> 1] & 0xFFFFu)); }
};

template <typename K, bool kVals>
__global__ void __launch_bounds__(TileShape<K>::kBlock, TileShape<K>::kMinBlocks)
    tile_scatter_kernel(const TileScatterArgs a) {
  using L = TileSmem<K, kVals>;
  constexpr int kBlock = L::kBlock;
  constexpr int kIpt = L::kIpt;
  constexpr int kTile = L::kTile;
  constexpr int kWarps = L::kWarps;
  static_assert(kTile <= 65536, "in-warp ranks and source positions are kept in 16 bits");
  static_assert(kWarps == kTableStrips, "one warp per strip of KT1's strip counts");
  static_assert(L::kVals_ % 16 == 0 && L::kWcnt % 16 == 0 && L::kGrp % 128 == 0,
                "bulk-copy targets, 16-byte clears, one bank per group word");
  extern __shared__ __align__(1024) unsigned char smem[];
  K* s_keys = reinterpret_cast<K*>(smem + L::kKeys);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(smem + L::kVals_);
  uint32_t* s_wcnt = reinterpret_cast<uint32_t*>(smem + L::kWcnt);
  uint32_t* s_off = reinterpret_cast<uint32_t*>(smem + L::kOff);
  uint32_t* s_scan = reinterpret_cast<uint32_t*>(smem + L::kScan);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + L::kBar);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // the chunk scan of this pass has read the totals: leave them zero for the next count
  if (blockIdx.x == 0 && tid < kRadix && a.totals) a.totals[tid] = 0;
  // Where the tile's keys come from and go to: t0 is its first key in an
  // array of n_keys keys, chunk its count chunk.
  const uint32_t tile = blockIdx.x;
  const K* kin;
  const uint32_t* vin;
  K* kout;
  uint32_t* vout;
  uint64_t t0, n_keys;
  uint32_t chunk;
  if (a.segs) {
    const SegDesc sd = a.segs[a.tile_seg[tile]];
    K* own_k = static_cast<K*>(sd.keys);
    K* alt_k = const_cast<K*>(static_cast<const K*>(a.keys[kBufAlt])) + sd.alt_off;
    uint32_t* alt_v = kVals ? const_cast<uint32_t*>(a.vals[kBufAlt]) + sd.alt_off : nullptr;
    const bool even = (a.pass & 1) == 0;
    kin = even ? own_k : alt_k;
    vin = even ? sd.vals : alt_v;
    kout = even ? alt_k : own_k;
    vout = even ? alt_v : sd.vals;
    t0 = uint64_t(tile - sd.first_tile) * kTile;
    n_keys = sd.n;
    chunk = sd.first_chunk + (tile - sd.first_tile) / a.chunk_tiles;
  } else {
    int src = kBufIn, dst = kBufOut;
    if (a.sched) {
      const PassDesc pd = a.sched->pass[a.pass];
      if (!pd.active) return;
      src = pd.src;
      dst = pd.dst;
    }
    kin = static_cast<const K*>(pick(a.keys, src));
    vin = pick(a.vals, src);
    kout = const_cast<K*>(static_cast<const K*>(pick(a.keys, dst)));
    vout = const_cast<uint32_t*>(pick(a.vals, dst));
    t0 = uint64_t(tile) * kTile;
    n_keys = a.n;
    chunk = tile / a.chunk_tiles;
  }
  if (ld_relaxed_gpu(a.status) & kDevBadTable) return;  // the offsets are not trustworthy: write nothing
  const uint32_t tile_n = uint32_t((n_keys - t0 < uint64_t(kTile)) ? (n_keys - t0) : uint64_t(kTile));

  // 1. stage the tile: bulk copies for the 16-byte-aligned body, plain loads
  // for a ragged end; meanwhile read the tile's offsets and its strips' digit
  // counts (KT1 counted them) from the table.
  const uint32_t kbody = (tile_n * uint32_t(sizeof(K))) & ~15u;
  const uint32_t vbody = kVals ? ((tile_n * 4u) & ~15u) : 0u;
  if (tid == 0) {
    mbar_init(s_bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(s_bar, kbody + vbody);
    if (kbody) bulk_copy_g2s(s_keys, kin + t0, kbody, s_bar);
    if (vbody) bulk_copy_g2s(s_vals, vin + t0, vbody, s_bar);
  }
  {
    const uint16_t* sc = a.stripcnt + uint64_t(tile) * (kWarps * kRadix);
#pragma unroll
    for (int i = tid; i < kWarps * kRadix; i += kBlock) s_wcnt[i] = sc[i];
  }
  if (tid < kRadix)  // lands while the copy does
    s_off[tid] = a.chunkoff[uint64_t(chunk) * kRadix + tid] + a.tilerel[uint64_t(tile) * kRadix + tid];
  for (uint32_t i = kbody / sizeof(K) + tid; i < tile_n; i += kBlock) s_keys[i] = kin[t0 + i];
  if (kVals)
    for (uint32_t i = vbody / 4 + tid; i < tile_n; i += kBlock) s_vals[i] = vin[t0 + i];
  __syncthreads();  // the mbarrier's init is visible before anyone waits on it
  const bool landed = mbar_wait_bounded(s_bar, 0);
  if (__syncthreads_or(!landed)) {
    // Staged data not known complete: write nothing.  Give the copies still in
    // flight a second bounded wait, so that none lands in shared memory after
    // this CTA has exited and its space has gone to another CTA.
    if (tid == 0) atomicOr(a.status, kDevTimeoutLoad | kDevBadOutput);
    if (!landed) mbar_wait_bounded(s_bar, 0);
    return;
  }

  // 2. each warp loads its strip (item i of lane l is the key at
  // wbase + i*32 + l) into registers
  const uint32_t shift = a.shift, mask = a.mask;
  uint32_t* wcnt = s_wcnt + warp * kRadix;
  const int wbase = warp * 32 * kIpt;
  KeyRegs<K, kIpt> kr;
  // steps 2 and 4 are compiled twice: for whole tiles (every position valid) and the short last one
  auto load_step = [&](auto full) {
    constexpr bool kFull = decltype(full)::value;
#pragma unroll
    for (int i = 0; i < kIpt; ++i) {
      const int pos = wbase + i * 32 + lane;
      const bool valid = kFull || uint32_t(pos) < tile_n;
      kr.set(i, valid ? s_keys[pos] : K(0));
    }
  };
  if (tile_n == uint32_t(kTile)) load_step(FullTile<true>{});
  else load_step(FullTile<false>{});
  // No barrier here: the warp counts came from the table before the copy
  // barrier, and the scan below holds a block barrier that every warp reaches
  // only after its loads, so no record store of the rank step (they overwrite
  // the staged keys) can come before another warp's load.

  // 3. per digit: each warp's first position of the digit in the tile's
  // digit order (warp prefixes on top of the tile's exclusive digit prefix),
  // and the output offset of the digit's run (the table entry minus the run's
  // start inside the tile, modulo 2^32)
  {
    const int d = tid;
    uint32_t c[kWarps];
    uint32_t run = 0;
    if (d < kRadix) {
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        c[w] = s_wcnt[w * kRadix + d];
        run += c[w];
      }
    }
    const uint32_t ex = digit_excl_scan<kBlock>(run, s_scan);
    if (d < kRadix) {
      uint32_t acc = ex;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        s_wcnt[w * kRadix + d] = acc;
        acc += c[w];
      }
      s_off[d] -= ex;
    }
  }
  __syncthreads();

  // 4. stable ranks, straight to the key's slot in digit order: per round of
  // 32 keys the lanes that share a digit form a group (digit_group: its
  // winner and peer mask; the hardware match.any on locally skewed strips,
  // where it is the faster one); the winner takes the group's slots from the warp's
  // running position of the digit, and each lane's slot is the first one plus
  // its peers below it.  16-bit keys are stored as one record
  // key | source slot << 16 over the keys and source areas, wider keys in
  // place plus a 16-bit source slot; values stay where they are and are
  // gathered once, in the write-out.
  auto rank_step = [&](auto full) {
    constexpr bool kFull = decltype(full)::value;
    const uint32_t lt = lanemask_lt();
    bool skewed;
    {
      const uint32_t d0 = (kFull || uint32_t(wbase + lane) < tile_n) ? dig(kr.get(0), shift, mask) : 0xFFFFFFFFu;
      skewed = __popc(__ballot_sync(0xffffffffu, d0 == __shfl_sync(0xffffffffu, d0, 0))) >= 16;
    }
    uint8_t* win = reinterpret_cast<uint8_t*>(smem + L::kWin) + warp * kRadix;
    uint32_t* grp = reinterpret_cast<uint32_t*>(smem + L::kGrp) + warp * 32;
    uint32_t* s_rec32 = reinterpret_cast<uint32_t*>(smem + L::kKeys);
    uint16_t* s_src = reinterpret_cast<uint16_t*>(smem + L::kSrc);
#pragma unroll
    for (int i = 0; i < kIpt; ++i) {
      const int pos = wbase + i * 32 + lane;
      const bool valid = kFull || uint32_t(pos) < tile_n;
      const K k = kr.get(i);
      const uint32_t d = dig(k, shift, mask);
      uint32_t w;
      const uint32_t peers = digit_group_any(skewed, d, valid, win, grp, &w);
      uint32_t base = 0;
      if (valid && w == uint32_t(lane)) base = atomicAdd(&wcnt[d], uint32_t(__popc(peers)));
      base = __shfl_sync(0xffffffffu, base, w);
      if (valid) {
        const uint32_t p = base + __popc(peers & lt);
        if (sizeof(K) == 2) {
          s_rec32[p] = uint32_t(k) | (uint32_t(pos) << 16);
        } else {
          s_keys[p] = k;
          if (kVals) s_src[p] = uint16_t(pos);
        }
      }
    }
  };
  if (tile_n == uint32_t(kTile)) rank_step(FullTile<true>{});
  else rank_step(FullTile<false>{});
  __syncthreads();

  // 5. write-out in digit runs, consecutive threads to consecutive addresses
  const uint32_t* s_rec32 = reinterpret_cast<const uint32_t*>(smem + L::kKeys);
  const uint16_t* s_src = reinterpret_cast<const uint16_t*>(smem + L::kSrc);
  auto write_slot = [&](uint32_t s) {
    K k;
    uint32_t from = 0;
    if (sizeof(K) == 2) {
      const uint32_t r = s_rec32[s];
      k = K(r & 0xFFFFu);
      from = r >> 16;
    } else {
      k = s_keys[s];
      if (kVals) from = s_src[s];
    }
    const uint32_t o = s_off[dig(k, shift, mask)] + s;
    kout[o] = k;
    if (kVals) vout[o] = s_vals[from];
  };
  if (tile_n == uint32_t(kTile)) {
#pragma unroll
    for (int j = 0; j < kIpt; ++j) write_slot(uint32_t(tid + j * kBlock));
  } else {
#pragma unroll 4
    for (uint32_t s = tid; s < tile_n; s += kBlock) write_slot(s);
  }
}

template <typename K, bool kVals>
cudaError_t launch_scatter_typed(const TileScatterArgs& a, uint32_t tiles, cudaStream_t stream) {
  using L = TileSmem<K, kVals>;
  static const cudaError_t attr = set_smem_attrs(tile_scatter_kernel<K, kVals>, L::kBytes, true);
  if (attr != cudaSuccess) return attr;
  tile_scatter_kernel<K, kVals><<<tiles, L::kBlock, L::kBytes, stream>>>(a);
  return cudaGetLastError();
}

template <typename K, bool kOrAnd>
cudaError_t launch_count_variant(const TileCountArgs& a, uint32_t grid, cudaStream_t stream) {
  static const cudaError_t attr = set_smem_attrs(tile_count_kernel<K, kOrAnd>, count_smem_bytes<K>(), false);
  if (attr != cudaSuccess) return attr;
  tile_count_kernel<K, kOrAnd><<<grid, count_threads<K>(), count_smem_bytes<K>(), stream>>>(a);
  return cudaGetLastError();
}

template <typename K>
cudaError_t launch_count_typed(const TileCountArgs& a, uint32_t grid, cudaStream_t stream) {
  return a.orand ? launch_count_variant<K, true>(a, grid, stream) : launch_count_variant<K, false>(a, grid, stream);
}

}  // namespace

int table_tile_keys_for(int key_bits) {
  switch (key_bits) {
    case 16: return TileSmem<uint16_t, true>::kTile;
    case 32: return TileSmem<uint32_t, true>::kTile;
    case 64: return TileSmem<uint64_t, true>::kTile;
    default: return 0;
  }
}

TableGeom table_geometry(uint64_t n, int key_bits, int sms) {
  TableGeom g{};
  g.tile = uint32_t(table_tile_keys_for(key_bits));
  if (!g.tile || !n) return g;
  g.tiles = uint32_t((n + g.tile - 1) / g.tile);
  const int per_sm = key_bits == 16 ? count_ctas_per_sm<uint16_t>() : count_ctas_per_sm<uint64_t>();
  const uint32_t want = uint32_t(sms) * uint32_t(per_sm);  // one chunk per resident count CTA
  g.chunk_tiles = (g.tiles + want - 1) / want;
  g.chunks = (g.tiles + g.chunk_tiles - 1) / g.chunk_tiles;
  return g;
}

cudaError_t launch_tile_count(const TileCountArgs& a, int key_bits, uint32_t chunks, cudaStream_t stream) {
  if (!chunks) return cudaSuccess;
  switch (key_bits) {
    case 16: return launch_count_typed<uint16_t>(a, chunks, stream);
    case 32: return launch_count_typed<uint32_t>(a, chunks, stream);
    case 64: return launch_count_typed<uint64_t>(a, chunks, stream);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_table_schedule(uint64_t* orand, const DigitPlan& plan, int in_place, Schedule* sched,
                                  cudaStream_t stream) {
  table_schedule_kernel<<<1, 1, 0, stream>>>(orand, plan, in_place, sched);
  return cudaGetLastError();
}

cudaError_t launch_chunk_scan(const uint32_t* chunksum, const uint32_t* totals, uint32_t chunks,
                              const Schedule* sched, int pass, uint32_t* chunkoff, cudaStream_t stream) {
  if (!chunks) return cudaSuccess;
  chunk_scan_kernel<<<kRadix, kScanThreads, 0, stream>>>(chunksum, totals, chunks, sched, pass, chunkoff);
  return cudaGetLastError();
}

cudaError_t launch_seg_chunk_scan(const uint32_t* chunksum, const SegDesc* segs, uint32_t nsegs, uint32_t tile,
                                  uint32_t chunk_tiles, uint32_t* chunkoff, cudaStream_t stream) {
  if (!nsegs) return cudaSuccess;
  seg_chunk_scan_kernel<<<nsegs, kRadix, 0, stream>>>(chunksum, segs, tile, chunk_tiles, chunkoff);
  return cudaGetLastError();
}

cudaError_t launch_tile_scatter(const TileScatterArgs& a, int key_bits, bool has_vals, cudaStream_t stream) {
  if (!a.tiles) return cudaSuccess;
  switch (key_bits) {
    case 16: return has_vals ? launch_scatter_typed<uint16_t, true>(a, a.tiles, stream)
                             : launch_scatter_typed<uint16_t, false>(a, a.tiles, stream);
    case 32: return has_vals ? launch_scatter_typed<uint32_t, true>(a, a.tiles, stream)
                             : launch_scatter_typed<uint32_t, false>(a, a.tiles, stream);
    case 64: return has_vals ? launch_scatter_typed<uint64_t, true>(a, a.tiles, stream)
                             : launch_scatter_typed<uint64_t, false>(a, a.tiles, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fsort
