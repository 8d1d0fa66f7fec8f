/*
 * oracle.c -- plain, slow, single-threaded CPU reference for the compressed
 * radix sort hot path of "FractalSortCPU: Bandwidth-Efficient Compressed Radix
 * Sort on CPU" (arXiv 2605.10390).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: it exists so that the CUDA library can be compared, element
 * by element, against an implementation a reader can check against the paper
 * by eye.  It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (readings of the paper are marked R1..R9 and listed in
 * the project's design notes):
 *   - Sort key.  A key of key_bits bits is ordered by its top p =
 *     precision_bits bits, s(k) = k >> (key_bits - p) (Sec. I on reduced
 *     precision sorting; R2).  Ties keep input order (R3: the radix sort of
 *     Sec. II is histogram, prefix sum and *stable* scatter), which makes the
 *     output unique.  Order is ascending unsigned numeric order of s(k) (R1).
 *   - oracle_sort: LSD radix sort built from exactly the three phases named in
 *     Sec. II -- histogram, exclusive prefix sum, stable scatter -- with a
 *     fixed 8-bit digit (the last digit narrower when 8 does not divide p).
 *   - oracle_digit_histograms: the per-pass digit counts C_j[v] (the leaf
 *     level of the histogram tree of Sec. III-B restricted to one digit).
 *   - oracle_exclusive_scan: B[v] = sum_{u<v} C[u]; the rank of leaf v, i.e.
 *     what GetIndex (Alg. 3) returns for value v (R6).
 *   - oracle_scatter_pass: one stable counting pass on one digit.
 *   - oracle_tree_*: the dense histogram tree of Sec. III-B ("Fractal RMW":
 *     every node on a key's root-to-leaf path counts it, R4) in the
 *     computable-pointer layout of Sec. III-F-1 / Alg. 4 (node ids implied by
 *     position), with rank (Alg. 3, R6) and select (Alg. 2, R5).
 *   - oracle_expand: Alg. 5 with no trailing bits (t = 0, R7): bin b's key is
 *     written C[b] times, bins in ascending order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

static int valid_widths(int key_bits, int precision_bits) {
  if (key_bits != 16 && key_bits != 32 && key_bits != 64) return 0;
  if (precision_bits < 1 || precision_bits > key_bits) return 0;
  return 1;
}

static uint64_t get_key(const void* keys, int key_bits, uint64_t i) {
  if (key_bits == 16) return ((const uint16_t*)keys)[i];
  if (key_bits == 32) return ((const uint32_t*)keys)[i];
  return ((const uint64_t*)keys)[i];
}

static void put_key(void* keys, int key_bits, uint64_t i, uint64_t k) {
  if (key_bits == 16) ((uint16_t*)keys)[i] = (uint16_t)k;
  else if (key_bits == 32) ((uint32_t*)keys)[i] = (uint32_t)k;
  else ((uint64_t*)keys)[i] = k;
}

/* s(k): the top p bits of the key, as an unsigned number (R1, R2). */
static uint64_t sort_key(uint64_t k, int key_bits, int p) { return k >> (key_bits - p); }

/* Digit j of the sort key for digit width d: bits [j*d, min((j+1)*d, p)). */
static uint64_t digit_of(uint64_t s, int p, int d, int j) {
  const int lo = j * d;
  const int width = (p - lo < d) ? (p - lo) : d;
  const uint64_t mask = (width >= 64) ? ~0ULL : ((1ULL << width) - 1);
  return (s >> lo) & mask;
}

int oracle_num_passes(int precision_bits, int digit_bits) {
  return (precision_bits + digit_bits - 1) / digit_bits;
}

/* Per-pass digit histograms: counts[j * 2^d + v] = #{i : digit_j(s(k_i)) = v}
 * for every pass j of a digit width d (Sec. III-A/B: one counter increment per
 * key per level; here only the leaf level of each digit is kept). */
int oracle_digit_histograms(const void* keys, uint64_t n, int key_bits, int precision_bits,
                            int digit_bits, uint64_t* counts) {
  if (!valid_widths(key_bits, precision_bits) || digit_bits < 1 || digit_bits > 16) return ORACLE_EINVAL;
  const int passes = oracle_num_passes(precision_bits, digit_bits);
  const uint64_t bins = 1ULL << digit_bits;
  memset(counts, 0, sizeof(uint64_t) * bins * (uint64_t)passes);
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t s = sort_key(get_key(keys, key_bits, i), key_bits, precision_bits);
    for (int j = 0; j < passes; ++j) counts[(uint64_t)j * bins + digit_of(s, precision_bits, digit_bits, j)] += 1;
  }
  return ORACLE_OK;
}

/* Exclusive prefix sum over the bins (Sec. II "prefix sum"; Alg. 3 rank). */
void oracle_exclusive_scan(const uint64_t* counts, uint64_t bins, uint64_t* out) {
  uint64_t running = 0;
  for (uint64_t v = 0; v < bins; ++v) {
    const uint64_t c = counts[v];
    out[v] = running;
    running += c;
  }
}

/* One stable counting pass on bits [shift, shift + width) of the raw key:
 * histogram, exclusive prefix sum, then an in-order scatter (Sec. II). */
int oracle_scatter_pass(const void* keys_in, const uint32_t* vals_in, void* keys_out, uint32_t* vals_out,
                        uint64_t n, int key_bits, int shift, int width) {
  if (key_bits != 16 && key_bits != 32 && key_bits != 64) return ORACLE_EINVAL;
  if (width < 1 || width > 16 || shift < 0 || shift + width > key_bits) return ORACLE_EINVAL;
  const uint64_t bins = 1ULL << width, mask = bins - 1;
  uint64_t* count = (uint64_t*)calloc(bins, sizeof(uint64_t));
  uint64_t* next = (uint64_t*)calloc(bins, sizeof(uint64_t));
  if (!count || !next) { free(count); free(next); return ORACLE_ENOMEM; }
  for (uint64_t i = 0; i < n; ++i) count[(get_key(keys_in, key_bits, i) >> shift) & mask] += 1;
  oracle_exclusive_scan(count, bins, next);
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t k = get_key(keys_in, key_bits, i);
    const uint64_t pos = next[(k >> shift) & mask]++;
    put_key(keys_out, key_bits, pos, k);
    if (vals_in) vals_out[pos] = vals_in[i];
  }
  free(count);
  free(next);
  return ORACLE_OK;
}

/* Full stable sort on the top p bits: LSD passes of 8-bit digits, least
 * significant digit first (Sec. II), each pass a stable counting pass.
 * keys_out/vals_out receive the result; the inputs are not modified.
 * vals_in may be NULL (keys only). */
int oracle_sort(const void* keys_in, const uint32_t* vals_in, void* keys_out, uint32_t* vals_out,
                uint64_t n, int key_bits, int precision_bits) {
  if (!valid_widths(key_bits, precision_bits)) return ORACLE_EINVAL;
  const size_t kb = (size_t)key_bits / 8;
  void* ka = malloc(n ? n * kb : 1);
  void* kt = malloc(n ? n * kb : 1);
  uint32_t* va = vals_in ? (uint32_t*)malloc(n ? n * 4 : 1) : NULL;
  uint32_t* vt = vals_in ? (uint32_t*)malloc(n ? n * 4 : 1) : NULL;
  if (!ka || !kt || (vals_in && (!va || !vt))) {
    free(ka); free(kt); free(va); free(vt);
    return ORACLE_ENOMEM;
  }
  memcpy(ka, keys_in, n * kb);
  if (vals_in) memcpy(va, vals_in, n * 4);
  const int d = 8;
  const int passes = oracle_num_passes(precision_bits, d);
  const int base = key_bits - precision_bits;  /* bit where the sort key starts */
  for (int j = 0; j < passes; ++j) {
    const int lo = j * d;
    const int width = (precision_bits - lo < d) ? (precision_bits - lo) : d;
    int rc = oracle_scatter_pass(ka, va, kt, vt, n, key_bits, base + lo, width);
    if (rc) { free(ka); free(kt); free(va); free(vt); return rc; }
    void* t = ka; ka = kt; kt = t;
    uint32_t* u = va; va = vt; vt = u;
  }
  memcpy(keys_out, ka, n * kb);
  if (vals_in) memcpy(vals_out, va, n * 4);
  free(ka); free(kt); free(va); free(vt);
  return ORACLE_OK;
}

/* ---- Histogram tree (Sec. III-B, Alg. 1-4), dense layout ----------------
 * Level l (0 = root) has 2^l nodes; node x at level l counts the keys whose
 * sort key has x as its top l bits.  Stored level by level: level l starts at
 * offset 2^l - 1 (the computable-pointer layout: a node's id is its place). */

static uint64_t level_base(int l) { return (1ULL << l) - 1; }

uint64_t oracle_tree_size(int precision_bits) { return (1ULL << (precision_bits + 1)) - 1; }

/* Insert every key along its root-to-leaf path, one increment per level
 * (Fractal RMW, Sec. III-B-1; Alg. 1 with every path node +1 per key, R4). */
int oracle_tree_build(const void* keys, uint64_t n, int key_bits, int precision_bits, uint64_t* tree) {
  if (!valid_widths(key_bits, precision_bits) || precision_bits > 24) return ORACLE_EINVAL;
  const int p = precision_bits;
  memset(tree, 0, sizeof(uint64_t) * oracle_tree_size(p));
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t s = sort_key(get_key(keys, key_bits, i), key_bits, p);
    for (int l = 0; l <= p; ++l) tree[level_base(l) + (s >> (p - l))] += 1;
  }
  return ORACLE_OK;
}

/* Count stored at node `prefix` of level l. */
uint64_t oracle_tree_count(const uint64_t* tree, int precision_bits, int level, uint64_t prefix) {
  (void)precision_bits;
  return tree[level_base(level) + prefix];
}

/* rank(v) = #{i : s(k_i) < v}: descend along v's bits; wherever v's path
 * turns right, add the left sibling's count (Alg. 3, R6). */
uint64_t oracle_tree_rank(const uint64_t* tree, int precision_bits, uint64_t v) {
  const int p = precision_bits;
  uint64_t idx = 0, prefix = 0;
  for (int l = 0; l < p; ++l) {
    const uint64_t bit = (v >> (p - 1 - l)) & 1;
    if (bit) idx += tree[level_base(l + 1) + (prefix << 1)];
    prefix = (prefix << 1) | bit;
  }
  return idx;
}

/* select(r): the sort key at sorted position r (0 <= r < n).  Go left while r
 * is below the left child's count, else subtract it and go right (Alg. 2, R5).
 * Returns UINT64_MAX when r is out of range. */
uint64_t oracle_tree_select(const uint64_t* tree, int precision_bits, uint64_t r) {
  const int p = precision_bits;
  if (r >= tree[0]) return UINT64_MAX;
  uint64_t prefix = 0;
  for (int l = 0; l < p; ++l) {
    const uint64_t left = tree[level_base(l + 1) + (prefix << 1)];
    if (r < left) {
      prefix = prefix << 1;
    } else {
      r -= left;
      prefix = (prefix << 1) | 1;
    }
  }
  return prefix;
}

/* Alg. 5 with t = 0 (R7): for bins b in ascending order write key b, C[b]
 * times.  Output length = sum of counts. */
int oracle_expand(const uint64_t* counts, uint64_t bins, int key_bits, void* keys_out) {
  if (key_bits != 16 && key_bits != 32 && key_bits != 64) return ORACLE_EINVAL;
  uint64_t idx = 0;
  for (uint64_t b = 0; b < bins; ++b)
    for (uint64_t c = 0; c < counts[b]; ++c) put_key(keys_out, key_bits, idx++, b);
  return ORACLE_OK;
}
