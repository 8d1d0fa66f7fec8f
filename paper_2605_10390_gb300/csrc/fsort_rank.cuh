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
