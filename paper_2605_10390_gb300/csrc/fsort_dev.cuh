// fsort_dev.cuh -- device-side building blocks shared by libfsort's kernels:
// inline-PTX wrappers (bulk async copies, mbarriers, relaxed GPU-scope
// loads/stores, the global timer) and the descriptors the kernels exchange.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fsort {

// ---- device status word bits (latched, read by the host) -------------------
constexpr uint32_t kDevTimeoutLookback = 1u;  // a look-back wait gave up
constexpr uint32_t kDevTimeoutLoad = 2u;      // a bulk-copy wait gave up
constexpr uint32_t kDevBadTile = 4u;          // a dynamic tile id beyond the grid (counter not reset)
constexpr uint32_t kDevBadLookback = 8u;      // a look-back walk reached its chunk's first tile without a prefix
constexpr uint32_t kDevBadOutput = 16u;       // a tile skipped its output after a failed bounded wait
constexpr uint32_t kDevBadBucket = 32u;       // a learned-path bucket exceeded the on-chip capacity (judge bypassed)
constexpr uint32_t kDevBadTable = 64u;        // a tile-offset table is incomplete (a count wait gave up)

// Bounded waits give up after this many nanoseconds of %globaltimer.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// ---- look-back status words -------------------------------------------------
// One 32-bit word per (tile, digit): 2-bit flag | 30-bit count.  Counts inside
// one look-back chunk never reach 2^30 (chunks hold fewer keys than that), so
// the word never overflows; the chunk's base is added as a 64-bit number.
constexpr uint32_t kFlagShift = 30;
constexpr uint32_t kFlagAggregate = 1u << kFlagShift;  // tile's own count only
constexpr uint32_t kFlagPrefix = 2u << kFlagShift;     // inclusive prefix through this tile
constexpr uint32_t kCountMask = (1u << kFlagShift) - 1;
constexpr uint64_t kMaxChunkKeys = (1ull << 30) - 1;

// Which buffer a pass reads or writes.
enum BufSel : int32_t { kBufIn = 0, kBufAlt = 1, kBufOut = 2 };

// Per-pass schedule written by the scan kernel on the device, so that trivial
// passes (every key has the same digit) are skipped without a host round trip.
struct PassDesc {
  int32_t active;   // 1: run the scatter; 0: skip
  int32_t src;      // BufSel
  int32_t dst;      // BufSel
  int32_t pad;
};

constexpr int kMaxPasses = 16;

struct Schedule {
  PassDesc pass[kMaxPasses];
  PassDesc copy;       // final copy when the result would end in the wrong buffer
  int32_t active_passes;
  int32_t pad[3];
};

// Route the active passes through the input, scratch and output buffers so
// that the last one writes the result where it belongs, adding a final copy
// only when no assignment can (one thread).  Buffer sequence b_0 = input,
// ..., b_k = the buffer holding the result (k active passes).  In place
// (input == output): alternate scratch/input; odd k ends in the scratch buffer
// and needs the copy back.  Out of place: count backwards from the output so
// the last active pass writes it; k == 0 copies.
__host__ __device__ inline void route_passes(const int* trivial, int passes, int in_place, Schedule* sched) {
  int k = 0;
  for (int j = 0; j < passes; ++j) k += trivial[j] ? 0 : 1;
  int cur = kBufIn, idx = 0;
  for (int j = 0; j < kMaxPasses; ++j) {
    PassDesc pd{0, kBufIn, kBufIn, 0};
    if (j < passes && !trivial[j]) {
      ++idx;
      int nxt;
      if (in_place) nxt = (idx & 1) ? kBufAlt : kBufIn;
      else nxt = ((k - idx) & 1) ? kBufAlt : kBufOut;
      pd.active = 1;
      pd.src = cur;
      pd.dst = nxt;
      cur = nxt;
    }
    sched->pass[j] = pd;
  }
  PassDesc cp{0, cur, in_place ? kBufIn : kBufOut, 0};
  if (in_place) cp.active = (cur != kBufIn);
  else cp.active = (cur != kBufOut);
  sched->copy = cp;
  sched->active_passes = k;
}

// ---- PTX wrappers ------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_gpu(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait that lets the hardware suspend the thread for up to ~1 ms while
// the phase is incomplete, instead of spinning.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier to complete; gives up after
// kWaitLimitNs and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait_suspend(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (!mbar_try_wait_suspend(bar, parity)) {
    if (global_timer_ns() - t0 > kWaitLimitNs) return false;
  }
  return true;
}

// Bulk (non-tensor) async copy global -> this CTA's shared memory, completing
// `bytes` of transaction count on `bar`.  dst, src and bytes must be multiples
// of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Asynchronous 8-byte copy global -> shared; completes at cp_async_wait_all
// (per thread; a barrier afterwards publishes it to the block).
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace fsort
