// fsort_rank.cuh -- stable ranking of keys by one radix digit inside a
// thread block: the building block shared by the scatter pass (K3) and the
// on-chip segment sort of the batched path.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fsort_dev.cuh"

namespace fsort {

constexpr int kRankRadix = 256;  // 8-bit digits; threads 0..255 own one digit each in per-digit steps

// Exclusive scan of x over threads 0..255 (the digits); every thread of the
// block must call it (it contains a barrier).
template <int kBlock>
__device__ __forceinline__ uint32_t digit_excl_scan(uint32_t x, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31 && warp < kRankRadix / 32) s_warp[warp] = inc;
  __syncthreads();
  uint32_t before = 0;
#pragma unroll
  for (int w = 0; w < kRankRadix / 32; ++w)
    if (w < warp) before += s_warp[w];
  return before + inc - x;
}

template <typename K>
__device__ __forceinline__ uint32_t dig(K k, uint32_t shift, uint32_t mask) {
  if (sizeof(K) <= 4) return (uint32_t(k) >> shift) & mask;
  return uint32_t(uint64_t(k) >> shift) & mask;
}

// Per-item key and in-warp rank.  16-bit keys share one register with their
// rank (ranks stay below the tile size); wider keys keep two.
template <typename K>
struct Item {
  K key;
  uint32_t rank;
  __device__ __forceinline__ void set(K k, uint32_t r) { key = k; rank = r; }
  __device__ __forceinline__ K k() const { return key; }
  __device__ __forceinline__ uint32_t r() const { return rank; }
  __device__ __forceinline__ void set_r(uint32_t r) { rank = r; }
};
template <>
struct Item<uint16_t> {
  uint32_t packed;
  __device__ __forceinline__ void set(uint16_t k, uint32_t r) { packed = uint32_t(k) | (r << 16); }
  __device__ __forceinline__ uint16_t k() const { return uint16_t(packed & 0xFFFFu); }
  __device__ __forceinline__ uint32_t r() const { return packed >> 16; }
  __device__ __forceinline__ void set_r(uint32_t r) { packed = (packed & 0xFFFFu) | (r << 16); }
};


// Groups of the lanes of a warp that share a digit, through two small
// warp-private tables that need no clearing between uses:
//   win[256] (bytes): every lane writes its lane id to win[d]; one write per
//       digit survives, naming the group's winner.  Four digits share a
//       32-bit word, so this table spreads 32 lanes over 64 words and its
//       accesses meet fewer bank conflicts than a word per digit would.
//   grp[32] (words, indexed by the winner lane, one bank each): the winner
//       resets its word, every member adds its lane bit, and the word is then
//       the group's peer mask -- what __match_any_sync returns.
// Returns the peer mask (0 for an invalid lane, which joins no group) and the
// winner lane in *winner.  Every lane of the warp must call it; neither table
// needs initialising, and calls may follow each other directly.
__device__ __forceinline__ uint32_t digit_group(uint32_t d, bool valid, uint8_t* win, uint32_t* grp,
                                                uint32_t* winner) {
  const uint32_t lane = threadIdx.x & 31;
  if (valid) win[d] = uint8_t(lane);
  __syncwarp();
  const uint32_t w = valid ? uint32_t(win[d]) : lane;
  if (valid && w == lane) grp[w] = 0u;
  __syncwarp();
  if (valid) atomicAdd(&grp[w], 1u << lane);
  __syncwarp();
  *winner = w;
  return valid ? grp[w] : 0u;
}

// Whether a warp's strip is locally skewed: at least half of its first
// round shares lane 0's digit (presorted runs, constant digits).  There the
// group words of digit_group take one same-address addition per member,
// while the hardware match.any is fast when a round has few distinct digits;
// elsewhere match.any is several times slower.  The choice changes speed
// only.  Every lane of the warp must call it.
template <typename K>
__device__ __forceinline__ bool strip_skewed(const K* s_keys, uint32_t tile_n, int wbase, uint32_t shift,
                                             uint32_t mask) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t d0 = uint32_t(wbase) + lane < tile_n ? dig(s_keys[wbase + lane], shift, mask) : 0xFFFFFFFFu;
  const uint32_t lead = __shfl_sync(0xffffffffu, d0, 0);
  return __popc(__ballot_sync(0xffffffffu, d0 == lead)) >= 16;
}

// digit_group, or the hardware match.any on a skewed strip (same groups; the
// winner is then the group's lowest lane).
__device__ __forceinline__ uint32_t digit_group_any(bool skewed, uint32_t d, bool valid, uint8_t* win,
                                                    uint32_t* grp, uint32_t* winner) {
  if (!skewed) return digit_group(d, valid, win, grp, winner);
  const uint32_t lane = threadIdx.x & 31;
  uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 0x100u + lane);  // invalid lanes match nobody
  if (!valid) peers = 0;
  *winner = valid ? uint32_t(__ffs(peers) - 1) : lane;
  return peers;
}

// Stable in-warp ranks of one warp's strip of a tile held in shared memory,
// with digit groups from digit_group.  Item i of lane l is the key at position
// wbase + i*32 + l; positions >= tile_n are padding.  Per round of 32 keys the
// group's winner adds the group size to the strip's counter of the digit and
// broadcasts the old value; each lane's rank is that value plus its peers
// below it.  On return it[i] holds the key and its rank among the strip's keys
// with the same digit (input order), and wcnt[d] (zero on entry) the strip's
// count of digit d.
template <typename K, int kIpt>
__device__ __forceinline__ void rank_strip_grouped(const K* s_keys, uint32_t tile_n, int wbase, uint32_t shift,
                                                   uint32_t mask, uint8_t* win, uint32_t* grp, uint32_t* wcnt,
                                                   Item<K> (&it)[kIpt]) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const bool skewed = strip_skewed(s_keys, tile_n, wbase, shift, mask);
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    const int first = wbase + i * 32;
    const int left = int(tile_n) - first;  // keys in this round (warp-uniform)
    if (left <= 0) {
      it[i].set(K(0), 0);
      continue;
    }
    const bool valid = lane < left;
    const K k = valid ? s_keys[first + lane] : K(0);
    const uint32_t d = dig(k, shift, mask);
    uint32_t w;
    const uint32_t peers = digit_group_any(skewed, d, valid, win, grp, &w);
    uint32_t base = 0;
    if (valid && w == uint32_t(lane)) base = atomicAdd(&wcnt[d], uint32_t(__popc(peers)));
    base = __shfl_sync(0xffffffffu, base, w);
    it[i].set(k, base + __popc(peers & lt));
  }
}

// Stable in-warp ranks of one warp's strip of a tile held in shared memory.
// Item i of lane l is the key at position wbase + i*32 + l (positions >=
// tile_n are padding).  On return it[i] holds the key and its rank among the
// strip's keys with the same digit (input order), and wcnt[d] the strip's
// count of digit d (wcnt must start at zero).  wmask0/wmask1 are two
// 256-word scratch arrays that must start at zero; they are zero again on
// return.
//
// For every round of 32 keys each lane adds its lane bit to the word of its
// digit: the word is then exactly the __match_any_sync peer mask of the lane.
// The lowest peer adds the group size to the strip's digit counter and
// broadcasts the old value; a lane's rank is that value plus its peers below
// it.  Locally skewed strips (presorted runs, constant digits) serialise the
// same-address additions, while the hardware match.any is fast when a round
// has few distinct digits: the warp picks the method for its whole strip from
// its first round (a speed choice only; both give the same ranks).
//
// kDyn: the strip has only `rounds` (<= kIpt) rounds (a warp-uniform bound);
// items of later rounds are left untouched.
template <typename K, int kIpt, bool kDyn = false>
__device__ __forceinline__ void rank_strip(const K* s_keys, uint32_t tile_n, int wbase, uint32_t shift, uint32_t mask,
                                           uint32_t* wmask0, uint32_t* wmask1, uint32_t* wcnt, Item<K> (&it)[kIpt],
                                           int rounds = kIpt) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt(), me = 1u << lane;
  // Locally skewed strips (presorted runs, constant digits): same-address
  // mask additions serialise, while the hardware match.any is fast when a
  // round has few distinct digits.  The warp picks the method for its whole
  // strip from its first round (a speed choice only; both give the same ranks).
  bool use_match;
  {
    const bool v0 = uint32_t(wbase + lane) < tile_n;
    const uint32_t d0 = v0 ? dig(s_keys[wbase + lane], shift, mask) : 0xFFFFFFFFu;
    const uint32_t lead = __shfl_sync(0xffffffffu, d0, 0);
    use_match = __popc(__ballot_sync(0xffffffffu, d0 == lead)) >= 16;
  }
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    if (kDyn && i >= rounds) break;
    const int pos = wbase + i * 32 + lane;
    const bool valid = uint32_t(pos) < tile_n;
    const K k = valid ? s_keys[pos] : K(0);
    const uint32_t d = dig(k, shift, mask);
    uint32_t peers;
    if (use_match) {
      peers = __match_any_sync(0xffffffffu, valid ? d : (0x100u + lane));  // invalid lanes match nobody
      if (!valid) peers = 0;
    } else {
      uint32_t* wmask = (i & 1) ? wmask1 : wmask0;
      if (valid) atomicAdd(&wmask[d], me);
      __syncwarp();
      peers = valid ? wmask[d] : 0u;
      __syncwarp();
      if (valid && (peers & lt) == 0) wmask[d] = 0;
    }
    const uint32_t below = __popc(peers & lt);
    uint32_t base = 0;
    if (valid && below == 0) base = atomicAdd(&wcnt[d], uint32_t(__popc(peers)));
    base = __shfl_sync(0xffffffffu, base, valid ? (__ffs(peers) - 1) : lane);
    it[i].set(k, base + below);
  }
}

}  // namespace fsort
