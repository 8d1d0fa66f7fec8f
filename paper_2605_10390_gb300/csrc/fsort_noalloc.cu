// fsort_noalloc.cu -- fsort_scatter_pass_noalloc: one stable scatter pass with
// its scratch in a fixed device array that this library owns, so the call
// itself allocates nothing.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// sort -- for example code running under another component's memory budget (a
// framework's caching allocator that already holds nearly all of HBM),
// latency-critical paths that must not take cudaMalloc's implicit device
// synchronisation, or plugin hosts that forbid device allocation after start
// up.  They cannot create a plan either (fsort_plan_create allocates), so this
// entry point needs none.
//
// The scratch (look-back words, tile counters, the histogram accumulator,
// chunk bases, a status word) lives in g_noalloc_scratch below.  Every GPU
// that loads the library holds it until the process exits.  Host code must
// not pass the array's name to a kernel: in host code it is a host-side
// stand-in, not a device address.  The device address is looked up once per
// device with cudaGetSymbolAddress, with that device current.  A device reset
// (cudaDeviceReset, or a reset of the primary context) reloads the module and
// invalidates the cached address: calls after one are not supported.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/fsort.h"
#include "fsort_dev.cuh"
#include "fsort_internal.h"

namespace fsort {
namespace {

constexpr int kRadix = 256;
constexpr uint64_t kMaxTiles = (FSORT_NOALLOC_MAX_KEYS + 4095) / 4096;  // the smallest tile holds 4096 keys

// Byte layout of the scratch array.
constexpr size_t kOffCounters = 0;                        // 2 tile counters, padded (cleared by K1)
constexpr size_t kOffLookback = 256;                      // kMaxTiles x 256 look-back words (cleared by K1)
constexpr size_t kOffHist = kOffLookback + kMaxTiles * kRadix * 4;  // 256 u64, zeroed every call
constexpr size_t kOffChunkBase = kOffHist + kRadix * 8;   // 1 chunk x 256 u64 (written by K2)
constexpr size_t kOffChunkFlag = kOffChunkBase + kRadix * 8;
constexpr size_t kOffStatus = kOffChunkFlag + 256;        // zeroed every call
constexpr size_t kScratchBytes = kOffStatus + 256;
static_assert(kScratchBytes == FSORT_NOALLOC_SCRATCH_BYTES, "header and layout disagree");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_call_lock[kMaxDevices];  // one call at a time per device: they share the array

// Device address of g_noalloc_scratch on device `dev`, the current device
// (looked up once).
cudaError_t scratch_for_device(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return cudaSuccess;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool overlaps(const void* a, size_t an, const void* b, size_t bn) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bn && y < x + an;
}

}  // namespace
}  // namespace fsort

using namespace fsort;

extern "C" fsort_status fsort_scatter_pass_noalloc(const void* keys_in, const uint32_t* vals_in, void* keys_out,
                                                   uint32_t* vals_out, uint64_t n, int key_bits, int shift,
                                                   int width, void* stream) {
  if (key_bits != 16 && key_bits != 32 && key_bits != 64) return FSORT_ERR_INVALID_ARG;
  if ((vals_in == nullptr) != (vals_out == nullptr)) return FSORT_ERR_INVALID_ARG;
  if (width < 1 || width > 8 || shift < 0 || shift + width > key_bits) return FSORT_ERR_INVALID_ARG;
  if (n > FSORT_NOALLOC_MAX_KEYS) return FSORT_ERR_INVALID_ARG;
  if (n == 0) return FSORT_OK;
  if (!keys_in || !keys_out || !aligned16(keys_in) || !aligned16(keys_out)) return FSORT_ERR_INVALID_ARG;
  if (vals_in && (!aligned16(vals_in) || !aligned16(vals_out))) return FSORT_ERR_INVALID_ARG;
  const size_t kbytes = size_t(n) * (key_bits / 8);
  if (overlaps(keys_in, kbytes, keys_out, kbytes)) return FSORT_ERR_INVALID_ARG;
  if (vals_in && overlaps(vals_in, n * 4, vals_out, n * 4)) return FSORT_ERR_INVALID_ARG;

  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FSORT_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return FSORT_ERR_UNSUPPORTED;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FSORT_ERR_CUDA;
  unsigned char* w = nullptr;
  cudaError_t e = scratch_for_device(dev, &w);
  if (e != cudaSuccess) return FSORT_ERR_CUDA;
  // Calls from several host threads take turns: the call is synchronous, so
  // holding the lock until it returns keeps every other call off the array.
  std::lock_guard<std::mutex> turn(g_call_lock[dev]);

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* counters = reinterpret_cast<uint32_t*>(w + kOffCounters);
  uint32_t* lookback = reinterpret_cast<uint32_t*>(w + kOffLookback);
  uint64_t* hist = reinterpret_cast<uint64_t*>(w + kOffHist);
  uint64_t* chunk_base = reinterpret_cast<uint64_t*>(w + kOffChunkBase);
  uint32_t* chunk_flag = reinterpret_cast<uint32_t*>(w + kOffChunkFlag);
  uint32_t* status = reinterpret_cast<uint32_t*>(w + kOffStatus);

  const uint64_t tile = uint64_t(tile_keys_for(key_bits));
  const uint64_t tiles = (n + tile - 1) / tile;
  // The array keeps the previous call's contents: zero the histogram
  // accumulator and the status word; K1 zeroes the counters and look-back words.
  e = cudaMemsetAsync(hist, 0, kRadix * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 4, s);
  DigitPlan dp{};
  dp.passes = 1;
  dp.shift[0] = uint32_t(shift);
  dp.mask[0] = (1u << width) - 1u;
  if (e == cudaSuccess)
    e = launch_histogram(keys_in, key_bits, n, dp, hist, kRadix, counters,
                         (kOffLookback - kOffCounters) / 4 + tiles * kRadix, sms, s);
  if (e == cudaSuccess) e = launch_scan_schedule(hist, chunk_base, chunk_flag, 1, 1u, 0, nullptr, s);
  if (e == cudaSuccess) {
    OnesweepArgs a{};
    a.keys[0] = keys_in;
    a.keys[2] = keys_out;
    a.vals[0] = vals_in;
    a.vals[2] = vals_out;
    a.n = n;
    a.shift = dp.shift[0];
    a.mask = dp.mask[0];
    a.lookback = lookback;
    a.tile_counter = counters;
    a.chunk_base = chunk_base;
    a.chunk_flag = chunk_flag;
    a.sched = nullptr;
    a.pass = 0;
    a.tiles_per_chunk = uint32_t(chunk_keys_for(key_bits) / tile);
    a.status = status;
    e = launch_onesweep(a, key_bits, vals_in != nullptr, s);
  }
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FSORT_ERR_OOM : FSORT_ERR_CUDA;
  // Synchronous: read the status word back on the caller's stream (no
  // legacy-stream copy, which would wait for every blocking stream of the
  // device), wait for the stream, then report a device-side error.
  uint32_t flags = 0;
  if (cudaMemcpyAsync(&flags, status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return FSORT_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FSORT_ERR_CUDA;
  if (flags & (kDevTimeoutLookback | kDevTimeoutLoad)) return FSORT_ERR_TIMEOUT;
  return flags ? FSORT_ERR_INTERNAL : FSORT_OK;
}
