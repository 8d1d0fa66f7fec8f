// Device side of the seeded workload generators (see wl_gen.h): the same
// integer-only recipe, one thread per element, so a multi-GB workload is made
// in HBM without a host round trip.  Its bytes equal wl_fill's.
#include <cuda_runtime.h>
#include "wl_gen.h"

namespace {

template <typename K>
__global__ void wl_fill_kernel(K* out, uint64_t start, uint64_t count, wl_params p) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < count; j += stride)
    out[j] = K(wl_key(&p, start + j));
}

__global__ void wl_iota_kernel(uint32_t* out, uint64_t start, uint64_t count) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < count; j += stride)
    out[j] = uint32_t(start + j);
}

}  // namespace

// `p` is a host struct whose table pointers are device pointers.
extern "C" int wl_fill_device(void* out, uint64_t start, uint64_t count, const wl_params* p, void* stream) {
  if (!count) return 0;
  if (!out || !p) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 2;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
  const unsigned grid = unsigned(sms) * 8u;
  switch (p->key_bits) {
    case 16: wl_fill_kernel<uint16_t><<<grid, 256, 0, s>>>((uint16_t*)out, start, count, *p); break;
    case 32: wl_fill_kernel<uint32_t><<<grid, 256, 0, s>>>((uint32_t*)out, start, count, *p); break;
    case 64: wl_fill_kernel<uint64_t><<<grid, 256, 0, s>>>((uint64_t*)out, start, count, *p); break;
    default: return 1;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int wl_iota_device(uint32_t* out, uint64_t start, uint64_t count, void* stream) {
  if (!count) return 0;
  if (!out) return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 2;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
  wl_iota_kernel<<<unsigned(sms) * 8u, 256, 0, (cudaStream_t)stream>>>(out, start, count);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
