// fsort_internal.h -- launchers shared between the kernel translation units
// and the C-ABI layer.  Host-only declarations; no CUDA types beyond streams.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fsort_dev.cuh"

namespace fsort {

// A kernel's dynamic shared-memory limit and, with max_carveout, all of the
// unified L1/shared capacity as shared memory.  Callers keep the result in a
// function-local static, so each kernel is set up once per process, and
// thread-safely (C++ static initialisation), whichever host thread calls first.
template <typename F>
inline cudaError_t set_smem_attrs(F* kernel, size_t bytes, bool max_carveout) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e == cudaSuccess && max_carveout)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

// Digit plan of one sort: pass j extracts bits [shift[j], shift[j] + width[j]).
struct DigitPlan {
  int32_t passes;
  int32_t pad;
  uint32_t shift[kMaxPasses];
  uint32_t mask[kMaxPasses];
};

// Keys per scatter tile for each key width (also sizes the look-back regions).
int tile_keys_for(int key_bits);
// Keys per look-back chunk: whole tiles, fewer than 2^30 keys.
uint64_t chunk_keys_for(int key_bits);

// K1: per-pass digit histograms of keys[0, n): hist[j * pass_stride + d] +=
// count of digit d of pass j.  Also zeroes clear_words words at `clear` (the
// first pass's look-back region and the tile counters) on the way.
cudaError_t launch_histogram(const void* keys, int key_bits, uint64_t n, const DigitPlan& plan, uint64_t* hist,
                             uint64_t pass_stride, uint32_t* clear, uint64_t clear_words, int sms,
                             cudaStream_t stream);

// K2: per pass, exclusive scan over digits of the histogram (hist[j][256]),
// written as the 64-bit bases of look-back chunk 0 (chunk_base[j][chunks][256]),
// the chunk-ready flags of later chunks zeroed (chunk_flag[j][chunks]), and the
// device-side pass schedule.  hist is left all zero.  in_place: the result must
// land in the input buffer.  sched may be null (the one-pass step).
cudaError_t launch_scan_schedule(uint64_t* hist, uint64_t* chunk_base, uint32_t* chunk_flag, int passes,
                                 uint32_t chunks, int in_place, Schedule* sched, cudaStream_t stream);

// Row-wise exclusive scan, one CTA per row (bins <= 65536).
cudaError_t launch_scan_rows(const uint64_t* in, uint64_t* out, uint64_t rows, uint64_t bins, cudaStream_t stream);

// One segment of a batched sort (segmented scatter mode of K3).
struct SegDesc {
  void* keys;           // the caller's keys (sorted in place)
  uint32_t* vals;       // the caller's values, or null
  uint64_t n;           // keys in the segment
  uint64_t alt_off;     // element offset of the segment's ping-pong space in the plan scratch
  uint32_t first_tile;   // global index of the segment's first scatter tile
  uint32_t first_chunk;  // table form: global index of the segment's first count chunk
};

// K3: one stable scatter pass.
struct OnesweepArgs {
  const void* keys[3];     // by BufSel: input, plan scratch, output
  const uint32_t* vals[3];
  uint64_t n;
  uint32_t shift;
  uint32_t mask;
  uint32_t* lookback;      // this pass's region, [tiles][256] words, zero on entry
  uint32_t* tile_counter;  // this pass's dynamic tile counter, zero on entry
  uint32_t* next_lookback; // region the next pass will use (cleared here), or null
  uint32_t* next_counter;  // the next pass's counter (cleared here), or null
  uint64_t* chunk_base;    // [chunks][256] 64-bit digit bases; chunk 0 from the scan, later chunks
                           // written by the last tile of the chunk before
  uint32_t* chunk_flag;    // [chunks] set once a chunk's bases are written (entry 0 unused)
  const Schedule* sched;   // null: always run, input -> output
  int32_t pass;
  uint32_t tiles_per_chunk;
  uint32_t* status;
  // Segmented mode (segs != null): global tiles of many independent segments;
  // tile t belongs to segment tile_seg[t]; even passes read the segment's own
  // buffers and write its scratch space, odd passes the reverse; the segment's
  // 64-bit digit bases are chunk_base[seg * passes * 256 + pass * 256 + d].
  const SegDesc* segs;
  const uint32_t* tile_seg;
  uint32_t passes;
  uint32_t total_tiles;  // segmented mode: tiles over all segments (the grid)
  // Failure-detection test hook: tile `withhold_tile` never publishes its
  // look-back words (0xFFFFFFFF: none).  Look-back waits give up after
  // wait_limit_ns (0: kWaitLimitNs), and at once when another wait of this
  // plan already gave up.
  uint32_t withhold_tile = 0xFFFFFFFFu;
  uint32_t pad3 = 0;
  uint64_t wait_limit_ns = 0;
};
cudaError_t launch_onesweep(const OnesweepArgs& args, int key_bits, bool has_vals, cudaStream_t stream);

// ---- scatter passes over a table of per-tile offsets (fsort_blocks.cu) ----
// For n <= 2^32 keys: `tiles` tiles of `tile` keys, grouped in `chunks` runs of
// `chunk_tiles` consecutive tiles (one count CTA each; the last may be shorter).
struct TableGeom {
  uint32_t tile;
  uint32_t tiles;
  uint32_t chunk_tiles;
  uint32_t chunks;
};
int table_tile_keys_for(int key_bits);
TableGeom table_geometry(uint64_t n, int key_bits, int sms);
// Warp strips of a table-form tile (KT3's warps): KT1 counts every tile's
// digits per strip, 16-bit counts in stripcnt[tile][strip][256].
constexpr int kTableStrips = 16;

// KT1: for the digit (shift, mask), per tile the counts of each digit in the
// earlier tiles of its chunk (tilerel[t][256]), per chunk the digit totals
// (chunksum[c][256]) and over all chunks totals[256] += them (zero on entry);
// with orand set, also orand[0] |= every key and orand[1]
// &= every key (accumulators: 0 and all ones on entry).  sched set: the keys
// are those pass `pass` reads, and an inactive pass counts nothing; else
// keys[kBufIn].
struct TileCountArgs {
  const void* keys[3];
  uint64_t n;
  uint32_t shift;
  uint32_t mask;
  uint32_t tile;
  uint32_t tiles;
  uint32_t chunk_tiles;
  uint32_t pad;
  uint32_t* tilerel;
  uint32_t* chunksum;
  uint32_t* totals;
  uint64_t* orand;
  const Schedule* sched;
  int32_t pass;
  int32_t pad2;
  uint32_t* status;  // a failed bounded wait sets kDevBadTable: the scatter then writes nothing
  // Segmented mode (segs != null; batched sorts): chunk c belongs to segment
  // chunk_seg[c] and covers chunk_tiles of its tiles (the segment's last chunk
  // may hold fewer); even passes read the segment's own keys, odd passes its
  // scratch space keys[kBufAlt] + alt_off; tilerel is indexed by global tile
  // (SegDesc::first_tile), totals and orand are unused.
  const SegDesc* segs = nullptr;
  const uint32_t* chunk_seg = nullptr;
  // Digit counts of every tile's 16 strips (the keys KT3's warp w ranks):
  // stripcnt[t][w][256], 16 bits, indexed by global tile like tilerel.
  uint16_t* stripcnt = nullptr;
};
cudaError_t launch_tile_count(const TileCountArgs& a, int key_bits, uint32_t chunks, cudaStream_t stream);
// Segmented KT2: for every segment (one CTA each) and digit d, the exclusive
// scan over digits of the segment's totals (the sums of its chunks' counts)
// plus the counts of d in its earlier chunks: chunkoff[c][d], relative to the
// segment's start.
cudaError_t launch_seg_chunk_scan(const uint32_t* chunksum, const SegDesc* segs, uint32_t nsegs, uint32_t tile,
                                  uint32_t chunk_tiles, uint32_t* chunkoff, cudaStream_t stream);
// The pass schedule from the keys' OR and AND (a pass is trivial when they
// agree on its digit); resets the accumulators.
cudaError_t launch_table_schedule(uint64_t* orand, const DigitPlan& plan, int in_place, Schedule* sched,
                                  cudaStream_t stream);
// KT2: chunkoff[c][d] = keys of digits below d (from totals) + keys of digit d
// in chunks before c (32-bit, exact modulo 2^32).
cudaError_t launch_chunk_scan(const uint32_t* chunksum, const uint32_t* totals, uint32_t chunks,
                              const Schedule* sched, int pass, uint32_t* chunkoff, cudaStream_t stream);
// KT3: one stable scatter pass, one CTA per tile, tile t writing digit d from
// chunkoff[t / chunk_tiles][d] + tilerel[t][d] on.
struct TileScatterArgs {
  const void* keys[3];  // by BufSel: input, plan scratch, output
  const uint32_t* vals[3];
  uint64_t n;
  uint32_t shift;
  uint32_t mask;
  uint32_t tiles;
  uint32_t chunk_tiles;
  const uint32_t* tilerel;
  const uint32_t* chunkoff;
  uint32_t* totals;  // this pass's digit totals, zeroed here once the chunk scan has read them
  const Schedule* sched;  // null: always run, input -> output
  int32_t pass;
  int32_t pad2;
  uint32_t* status;
  // Segmented mode (segs != null): tile t belongs to segment tile_seg[t]; its
  // offsets are chunkoff[first_chunk + local tile / chunk_tiles] + tilerel[t];
  // even passes write the segment's scratch space, odd passes its own buffers.
  const SegDesc* segs = nullptr;
  const uint32_t* tile_seg = nullptr;
  // The tile's per-strip digit counts from KT1 (stripcnt[t][w][256]).
  const uint16_t* stripcnt = nullptr;
};
cudaError_t launch_tile_scatter(const TileScatterArgs& a, int key_bits, bool has_vals, cudaStream_t stream);

// Final copy when the schedule leaves the result in the wrong buffer.
cudaError_t launch_schedule_copy(const void* const keys[3], const uint32_t* const vals[3], int key_bits,
                                 bool has_vals, uint64_t n, const Schedule* sched, int sms, cudaStream_t stream);

// Expand path (16-bit keys, precision 16, keys only).
// K1 leaf histogram with 16-bit tapered counters: per-CTA packed partials
// [grid][32768] words plus exact overflow spills [65536] (spill zeroed here).
int leaf_hist_grid(int sms);
cudaError_t launch_leaf_histogram(const uint16_t* keys, uint64_t n, uint32_t* partials, uint64_t* spill, int sms,
                                  cudaStream_t stream);
// Sum the partials and spills into counts[65536].
cudaError_t launch_leaf_reduce(const uint32_t* partials, const uint64_t* spill, int grid, uint64_t* counts,
                               cudaStream_t stream);
// K4: keys_out[offsets[v] .. offsets[v] + counts[v]) = v.
cudaError_t launch_expand(const uint64_t* offsets, uint16_t* keys_out, uint64_t n, cudaStream_t stream);

// ---- batched sorts (fsort_batch.cu) ----
// Small segments sorted entirely in shared memory by one CTA each.
// capacity: 1024, 2048 or 4096 keys.  segs[0..count) all have n <= capacity.
// counter: a device word, zero on entry (work distribution).
cudaError_t launch_small_sort(const SegDesc* segs, uint32_t count, int key_bits, bool has_vals, int capacity,
                              const DigitPlan& plan, uint32_t* counter, int ctas, cudaStream_t stream);
int small_sort_ctas_per_sm(int key_bits, bool has_vals, int capacity);

// One entry of the segmented histogram's work list.
struct HistChunk {
  uint32_t seg;
  uint32_t len;
  uint64_t start;
};
// Per-segment per-pass digit histograms: hist[(seg * passes + j) * 256 + d]
// (accumulated; zero on entry).  Also zeroes clear_words words at `clear`.
cudaError_t launch_seg_histogram(const SegDesc* segs, const HistChunk* chunks, uint32_t nchunks, int key_bits,
                                 const DigitPlan& plan, uint64_t* hist, uint32_t* clear, uint64_t clear_words,
                                 cudaStream_t stream);
// Per segment and pass: exclusive scan of the histogram into 64-bit bases
// (same layout); leaves hist zero.
cudaError_t launch_seg_scan(uint64_t* hist, uint64_t* bases, uint32_t nsegs, int passes, cudaStream_t stream);
// tile_seg[t] = segment of global tile t.
cudaError_t launch_fill_tile_seg(const SegDesc* segs, uint32_t nsegs, int tile_keys, uint32_t* tile_seg,
                                 cudaStream_t stream);
// Copy each segment's scratch space back to its own buffers (odd pass count).
cudaError_t launch_seg_copy_back(const SegDesc* segs, uint32_t nsegs, const void* alt_keys,
                                 const uint32_t* alt_vals, int key_bits, int sms, cudaStream_t stream);

// ---- learned bucket mapping (fsort_learned.cu) ----
constexpr int kMlpHidden = 64;
constexpr int kMlpParams = 1 * kMlpHidden + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden + kMlpHidden + 1;
constexpr int kLearnCells = 56320;        // cells of the 11-significant-bit grid over 64-bit keys
constexpr int kLearnMaxHeavy = 8192;      // keys that get a bucket of their own
constexpr int kLearnBucketCap = 8192;     // keys one CTA sorts on chip
constexpr int kLearnKeysPerBucket = 1024; // B = smallest power of two >= n / 1024 (mean load in (512, 1024])
constexpr int kLearnTau = 8;              // judge: accept iff max non-heavy bucket <= tau * n / B (<= capacity)
constexpr float kLearnEps = 1.0f / 16.0f; // weight of the uniform-in-feature floor mixed into the model's CDF

// Device-resident model and judge state.
struct LearnedState {
  float center, half;          // feature normalisation: x = (log2(k + 1) / 64 - center) / half
  uint32_t heavy_count;        // m (<= kLearnMaxHeavy)
  uint32_t train_count;        // non-heavy sample keys the model is trained on
  uint32_t sample_count;
  uint32_t max_nonheavy;       // judge: largest non-heavy bucket of the last histogram
  uint32_t large_heavy;        // judge: heavy buckets above the fill split (listed in large_list)
  uint32_t pad;
  float loss;                  // accumulated by the gradient kernel, moved to the loss log by Adam
  float pad2[3];
};

// The bucket map: cells[i] = (G_i, H_i) for i in [0, kLearnCells]: G = model
// CDF at cell start (u32 fixed point, non-decreasing), H = heavy keys below
// the cell start; heavy[] ascending; id = (PLA(k) >> shift) + 2 c(k) + e(k).
struct LearnedMap {
  const uint2* cells;
  const uint64_t* heavy;
  uint32_t shift;  // 32 - log2(B)
};

// grads += gradient of the mean (over m) of 0.5 (sigmoid(mlp(x)) - y)^2; loss += that mean.
cudaError_t launch_mlp_grad(const void* w_bf16, const float* x, const float* y, uint32_t m, float* grads, float* loss,
                            cudaStream_t stream);
// Same on a stratified minibatch of m keys of the sorted training sample (step selects the draw).
cudaError_t launch_mlp_grad_sample(const void* w_bf16, const uint64_t* train, const LearnedState* st, uint32_t m,
                                   uint32_t step, uint64_t seed, float* grads, cudaStream_t stream);
// One Adam step (step >= 1): master/m1/m2 FP32, grads zeroed, BF16 copy
// refreshed; if loss_log: loss_log[0] = st->loss, st->loss = 0.
cudaError_t launch_mlp_adam(float* master, float* grads, float* m1, float* m2, void* w_bf16, float lr, int step,
                            LearnedState* st, float* loss_log, cudaStream_t stream);
cudaError_t launch_mlp_eval(const void* w_bf16, const float* x, uint32_t m, float* out, cudaStream_t stream);
cudaError_t launch_to_bf16(const float* src, void* dst, int count, cudaStream_t stream);

// Fitting: stratified sample of s keys; heavy/non-heavy split of the sorted
// sample; compaction; the tabulated map.
cudaError_t launch_learn_sample(const uint64_t* keys, uint64_t n, uint32_t s, uint64_t seed, uint64_t* out,
                                cudaStream_t stream);
cudaError_t launch_learn_split(const uint64_t* sorted, uint32_t s, uint32_t hmin, uint32_t* flag_nh,
                               uint32_t* flag_hv, cudaStream_t stream);
cudaError_t launch_learn_compact(const uint64_t* sorted, uint32_t s, const uint32_t* flag_nh, const uint32_t* pos_nh,
                                 const uint32_t* flag_hv, const uint32_t* pos_hv, uint64_t* train, uint64_t* heavy,
                                 LearnedState* st, cudaStream_t stream);
// Move the first-layer kinks to quantiles of the training sample (FP32 master weights).
cudaError_t launch_learn_init_kinks(const uint64_t* train, const LearnedState* st, float* master,
                                    cudaStream_t stream);
cudaError_t launch_learn_cells(const void* w_bf16, LearnedState* st, const uint64_t* heavy, float* fval, uint2* cells,
                               cudaStream_t stream);
// The same table from the sorted training sample's empirical CDF (no model).
cudaError_t launch_learn_cells_ecdf(const uint64_t* train, LearnedState* st, const uint64_t* heavy, float* fval,
                                    uint2* cells, cudaStream_t stream);

// Exclusive scan of count u32 words (count <= 2^24): out (and out2 if not
// null); sums: scratch of >= count / 4096 + 1 words.
cudaError_t launch_scan_u32(const uint32_t* in, uint64_t count, uint32_t* out, uint32_t* out2, uint32_t* sums,
                            cudaStream_t stream);

// Sorting with the map: two-level partition geometry for a sort of n keys.
constexpr uint32_t kLearnL1Chunks = 16384;  // most level-1 chunks (input ranges owned by one CTA)
struct LearnedGeom {
  uint32_t nb;      // bucket ids in use: B + 2 * kLearnMaxHeavy
  uint32_t fbits;   // fine digit width (10..12)
  uint32_t nsuper;  // super-buckets (id >> fbits)
  uint32_t nids;    // nsuper << fbits (ids beyond nb are empty)
  uint32_t nch;     // level-1 chunks
  uint64_t chunk;   // keys per level-1 chunk
};
LearnedGeom learned_geometry(uint64_t n, uint32_t buckets);
cudaError_t launch_learn_heavy_ids(const LearnedMap& mp, LearnedState* st, uint32_t* hid, uint32_t* bitmap,
                                   cudaStream_t stream);
// counts1[nsuper * nch] (super-bucket major), hcount[kLearnMaxHeavy] accumulated,
// ids[n] every key's bucket id (all ones for heavy keys).
cudaError_t launch_learn_l1(const uint64_t* keys, uint64_t n, const LearnedGeom& g, const LearnedMap& mp,
                            const LearnedState* st, uint32_t heavy_count, uint32_t* counts1, uint32_t* hcount,
                            uint32_t* ids, cudaStream_t stream);
// off1: exclusive scan of counts1 with one extra entry (the total); fine[] receives
// each scattered key's fine digit (id & (2^fbits - 1)) at the key's position in alt.
cudaError_t launch_learn_l1_scatter(const uint64_t* keys, const uint32_t* ids, uint64_t n, const LearnedGeom& g,
                                    const uint32_t* off1, uint64_t* alt, uint16_t* fine, cudaStream_t stream);
cudaError_t launch_learn_l2_count(const uint16_t* fine, const LearnedGeom& g, const uint32_t* off1, uint32_t* counts,
                                  cudaStream_t stream);
cudaError_t launch_learn_judge(uint32_t* counts, const LearnedGeom& g, const uint32_t* bitmap, const uint32_t* hid,
                               const uint32_t* hcount, LearnedState* st, uint32_t* large_list, cudaStream_t stream);
cudaError_t launch_learn_l2_scatter(const uint64_t* alt, const uint16_t* fine, const LearnedGeom& g,
                                    const uint32_t* off1, const uint32_t* off2, uint64_t* dst, cudaStream_t stream);
cudaError_t launch_learn_fill(const LearnedMap& mp, const LearnedState* st, const uint32_t* hid,
                              const uint32_t* large_list, const uint32_t* offsets, const uint32_t* counts,
                              uint64_t* dst, int sms, cudaStream_t stream);
// units: scratch of 1 + 4 * ceil(nb / 4) uint2 (the unit list).
cudaError_t launch_learn_bucket_sort(uint64_t* keys, const uint32_t* counts, const uint32_t* offsets,
                                     const uint32_t* bitmap, uint32_t nb, uint2* units, uint32_t* status, int sms,
                                     cudaStream_t stream);
cudaError_t launch_learn_bucket_ids(const uint64_t* keys, uint64_t n, const LearnedMap& mp, uint32_t* ids,
                                    cudaStream_t stream);

}  // namespace fsort
