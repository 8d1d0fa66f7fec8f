/* Seeded, counter-based synthetic key generators shared by the CPU oracle's
 * tests, the CUDA parity tests and the benchmark.
 *
 * This module holds none of the sort's arithmetic: it only turns
 * (seed, stream, element index) into a key.  Element i of a stream depends on
 * nothing but (seed, stream, i), so any slice of a workload can be regenerated
 * on its own, on the host (wl_gen.c) or on the device (wl_gen_device.cu), and
 * both produce the same bytes.
 *
 * Random source: the SplitMix64 output function of Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators" (OOPSLA 2014), applied to
 * the Weyl sequence state_i = base + (i + 1) * GAMMA.  With base = 0 the
 * outputs are the published SplitMix64 sequence seeded with 0
 * (0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, ...).
 *
 * Distributions (dist codes):
 *   WL_UNIFORM    every key bit from the random source
 *   WL_TABLE      top 16 bits from an inverse-CDF threshold table over the
 *                 65,536 values (Zipf, discretised Gaussian, ...); key =
 *                 smallest t with u < table[t] (table has 65,535 entries,
 *                 the last bucket is implicit); lower bits uniform
 *   WL_PRESORTED  top 16 bits = floor(i * 65536 / n) (an ascending ramp); with
 *                 probability 1/10 per element the top 16 bits are instead a
 *                 uniform draw (the "10 % random swaps"); lower bits uniform
 *   WL_CONSTANT   every key equal to the 0xA5 byte pattern
 *   WL_QUANTILE   full-width key from a piecewise-linear inverse CDF: a table
 *                 of 65,537 ascending u64 quantile points q[0..65536]; the top
 *                 16 bits of u pick the segment, the low 48 bits interpolate
 *                 (integer arithmetic only)
 *   WL_HOTSET     with probability num/2^32 (hot_prob) the key is
 *                 hot_values[rank] with rank from the threshold table,
 *                 otherwise a WL_QUANTILE draw (used for mixtures with a set
 *                 of heavy hitters)
 *
 * Only integer arithmetic is used, so the host and the device agree bit for
 * bit.  Tables are plain data computed once by the caller.
 */
#ifndef WL_GEN_H
#define WL_GEN_H

#include <stdint.h>

#if defined(__CUDACC__)
#define WL_HD __host__ __device__ __forceinline__
#else
#define WL_HD static inline
#endif

#define WL_GAMMA 0x9E3779B97F4A7C15ULL

enum { WL_UNIFORM = 0, WL_TABLE = 1, WL_PRESORTED = 2, WL_CONSTANT = 3, WL_QUANTILE = 4, WL_HOTSET = 5 };

typedef struct wl_params {
  uint64_t seed;
  uint64_t stream;
  uint64_t n_total;      /* workload length (the ramp of WL_PRESORTED spans it) */
  int32_t dist;
  int32_t key_bits;      /* 16, 32 or 64 */
  uint32_t hot_prob;     /* WL_HOTSET: probability of a hot key, in units of 2^-32 */
  uint32_t pad;
  const uint64_t* table; /* WL_TABLE / WL_HOTSET: 65,535 thresholds */
  const uint64_t* quant; /* WL_QUANTILE / WL_HOTSET: 65,537 quantile points */
  const uint64_t* hot;   /* WL_HOTSET: 65,536 hot values */
} wl_params;

WL_HD uint64_t wl_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Base of sub-stream `sub` of (seed, stream); base(0, 0, 0) is not 0, the
 * raw SplitMix64 sequence is reachable through wl_draw_raw. */
WL_HD uint64_t wl_base(uint64_t seed, uint64_t stream, uint64_t sub) {
  return wl_mix(wl_mix(seed + WL_GAMMA) ^ (stream * 0xD1B54A32D192ED03ULL) ^ (sub * 0xA0761D6478BD642FULL));
}

WL_HD uint64_t wl_draw_raw(uint64_t base, uint64_t i) { return wl_mix(base + (i + 1) * WL_GAMMA); }

WL_HD uint32_t wl_table_lookup(const uint64_t* table, uint64_t u) {
  /* smallest t in [0, 65535] with u < table[t]; table[65535] is +infinity */
  uint32_t lo = 0, hi = 65535;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (u < table[mid]) hi = mid; else lo = mid + 1;
  }
  return lo;
}

WL_HD uint64_t wl_quantile(const uint64_t* q, uint64_t u) {
  uint32_t seg = (uint32_t)(u >> 48);
  uint64_t frac = u & 0xFFFFFFFFFFFFULL;            /* 48 bits */
  uint64_t a = q[seg], b = q[seg + 1];
  uint64_t span = b - a;                             /* q is ascending */
  /* a + span * frac / 2^48 without 128-bit types: split span into 32-bit halves */
  uint64_t s_hi = span >> 32, s_lo = span & 0xFFFFFFFFULL;
  uint64_t f_hi = frac >> 24, f_lo = frac & 0xFFFFFFULL;  /* frac = f_hi*2^24 + f_lo */
  /* span*frac/2^48 = (s_hi*2^32 + s_lo)*(f_hi*2^24 + f_lo)/2^48, truncated term by term */
  uint64_t t1 = (s_hi * f_hi) << 8;                  /* s_hi*f_hi*2^56/2^48 */
  uint64_t t2 = (s_hi * f_lo) >> 16;                 /* s_hi*f_lo*2^32/2^48 */
  uint64_t t3 = (s_lo * f_hi) >> 24;                 /* s_lo*f_hi*2^24/2^48 */
  uint64_t t4 = (s_lo * f_lo) >> 48;
  uint64_t off = t1 + t2 + t3 + t4;
  if (off > span) off = span;
  return a + off;
}

/* Element i (absolute index within the workload) as a key of p->key_bits bits. */
WL_HD uint64_t wl_key(const wl_params* p, uint64_t i) {
  const int kb = p->key_bits;
  const uint64_t kmask = kb == 64 ? ~0ULL : ((1ULL << kb) - 1);
  const uint64_t u0 = wl_draw_raw(wl_base(p->seed, p->stream, 0), i);
  const uint64_t u1 = wl_draw_raw(wl_base(p->seed, p->stream, 1), i);
  const int low_bits = kb - 16;
  const uint64_t low = low_bits > 0 ? (u1 >> (64 - low_bits)) : 0;
  uint64_t top;
  switch (p->dist) {
    case WL_UNIFORM:
      return (u0 >> (64 - kb)) & kmask;
    case WL_TABLE:
      top = wl_table_lookup(p->table, u0);
      return ((top << low_bits) | low) & kmask;
    case WL_PRESORTED: {
      const uint64_t u2 = wl_draw_raw(wl_base(p->seed, p->stream, 2), i);
      /* floor(i * 65536 / n) without overflow for n < 2^48 */
      top = p->n_total ? ((i << 16) / p->n_total) : 0;
      if (u2 < 0x199999999999999AULL) top = u0 >> 48;   /* 2^64 / 10, rounded up */
      return ((top << low_bits) | low) & kmask;
    }
    case WL_CONSTANT:
      return 0xA5A5A5A5A5A5A5A5ULL & kmask;
    case WL_QUANTILE:
      return (wl_quantile(p->quant, u0) >> (64 - kb)) & kmask;
    case WL_HOTSET: {
      const uint64_t u2 = wl_draw_raw(wl_base(p->seed, p->stream, 2), i);
      if ((uint32_t)(u2 >> 32) < p->hot_prob)
        return (p->hot[wl_table_lookup(p->table, u1)] >> (64 - kb)) & kmask;
      return (wl_quantile(p->quant, u0) >> (64 - kb)) & kmask;
    }
    default:
      return 0;
  }
}

#endif /* WL_GEN_H */
