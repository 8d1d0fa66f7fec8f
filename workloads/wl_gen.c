/* Host side of the seeded workload generators (see wl_gen.h). */
#include "wl_gen.h"

int wl_fill(void* out, uint64_t start, uint64_t count, const wl_params* p) {
  if (!out && count) return 1;
  if (p->key_bits != 16 && p->key_bits != 32 && p->key_bits != 64) return 1;
  if ((p->dist == WL_TABLE || p->dist == WL_HOTSET) && !p->table) return 1;
  if ((p->dist == WL_QUANTILE || p->dist == WL_HOTSET) && !p->quant) return 1;
  if (p->dist == WL_HOTSET && !p->hot) return 1;
  for (uint64_t j = 0; j < count; ++j) {
    const uint64_t k = wl_key(p, start + j);
    if (p->key_bits == 16) ((uint16_t*)out)[j] = (uint16_t)k;
    else if (p->key_bits == 32) ((uint32_t*)out)[j] = (uint32_t)k;
    else ((uint64_t*)out)[j] = k;
  }
  return 0;
}

uint64_t wl_raw(uint64_t base, uint64_t i) { return wl_draw_raw(base, i); }
uint64_t wl_stream_base(uint64_t seed, uint64_t stream, uint64_t sub) { return wl_base(seed, stream, sub); }
