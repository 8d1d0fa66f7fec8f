// fsort_api.cu -- the C ABI of libfsort (include/fsort.h): argument checks,
// plan-owned scratch, the digit plan, kernel sequencing and status latching.
// Every step of a sort runs in this library's CUDA kernels; the host only
// validates, enqueues and reports.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fsort.h"
#include "fsort_dev.cuh"
#include "fsort_internal.h"

using namespace fsort;

// The library's own sizes are the ones the header publishes.
static_assert(kMlpParams == FSORT_MLP_PARAMS, "MLP parameter count");
static_assert(kLearnCells == FSORT_LEARN_CELLS, "map table cells");
static_assert(kLearnMaxHeavy == FSORT_LEARN_MAX_HEAVY, "frequent keys with buckets of their own");

namespace {

// Per-kernel timing: events recorded around launches, reported on demand.
struct TimingRec {
  int32_t kind, pass, call, slot;
  uint64_t n;
  int32_t ev0, ev1;
};

struct Timing {
  static constexpr int kEvents = 8192;
  static constexpr int kSlots = 2048;
  bool on = false;
  std::vector<cudaEvent_t> ev;
  int next_ev = 0;
  fsort::Schedule* h_sched = nullptr;  // pinned copies of the device schedule, one per recorded call
  int next_slot = 0;
  int calls = 0;
  std::vector<TimingRec> recs;
};

// Learned bucket mapping (FSORT_FLAG_LEARNED): device buffers carved from
// the plan's allocation, and the host view of the last fit and judge.
struct LearnedWs {
  static constexpr uint32_t kMaxSample = 1u << 22;
  static constexpr uint32_t kMaxSteps = 16384;
  uint32_t sample_max = 0;
  uint32_t nids_max = 0;
  uint64_t l1_max = 0;
  uint64_t* sample = nullptr;
  uint64_t* train = nullptr;
  uint32_t *flag_nh = nullptr, *flag_hv = nullptr, *pos_nh = nullptr, *pos_hv = nullptr;
  uint32_t* sums = nullptr;
  uint64_t* heavy = nullptr;
  uint32_t *hid = nullptr, *large = nullptr;
  uint2* cells = nullptr;
  float* fval = nullptr;
  uint32_t *counts1 = nullptr, *off1 = nullptr;   // level 1: [nsuper][nch] + 1
  uint32_t *counts = nullptr, *offsets = nullptr;  // every bucket id (+ 1)
  uint32_t *hcount = nullptr, *bitmap = nullptr;
  uint2* units = nullptr;                          // bucket-sort unit list
  uint32_t* ids = nullptr;                         // [max_n] bucket id of every input key
  uint16_t* fine = nullptr;                        // [max_n] fine digit of every key in alt
  void* w_bf16 = nullptr;
  float *master = nullptr, *m1 = nullptr, *m2 = nullptr, *grads = nullptr, *loss_log = nullptr;
  fsort::LearnedState* st = nullptr;
  fsort::LearnedState* h_st = nullptr;  // pinned
  bool fitted = false;
  int32_t used = -1;
  // Host bound on st->heavy_count for the level-1 count's shared memory: the
  // maximum after a fit (the fit is stream-ordered), exact after a model is
  // set or a learned sort has read the state back.
  uint32_t heavy_count = kLearnMaxHeavy;
  uint32_t steps = 0, last_b = 0, last_limit = 0, last_max = 0, last_heavy = 0;
  double last_imbalance = 0.0;
};

}  // namespace

struct fsort_plan {
  int device = 0;
  int sms = 0;
  fsort_plan_desc desc{};
  int digit_bits = 8;
  int tile = 0;
  uint64_t chunk_keys = 0;
  uint64_t max_tiles = 0;
  uint64_t max_chunks = 0;

  unsigned char* ws = nullptr;  // one allocation holds all device scratch
  size_t ws_bytes = 0;
  void* alt_keys = nullptr;
  uint32_t* alt_vals = nullptr;
  uint32_t* counters = nullptr;  // [2] tile counters, directly followed by look-back region 0
  uint32_t* lookback[2] = {nullptr, nullptr};
  uint64_t* hist = nullptr;       // [kMaxPasses][256], all zero between calls
  uint64_t* chunk_base = nullptr; // [kMaxPasses][max_chunks][256]
  uint32_t* chunk_flag = nullptr; // [kMaxPasses][max_chunks]
  Schedule* sched = nullptr;
  uint32_t* status = nullptr;    // sticky device error bits
  uint64_t table_tiles = 0;      // tiles of the largest sort the offset table serves (n < 2^32)
  uint32_t table_chunks = 0;     // chunks of the count kernel (at most two per SM)
  uint32_t* tilerel = nullptr;   // [table_tiles][256] per-tile digit offsets within the tile's chunk
  uint16_t* stripcnt = nullptr;  // [table_tiles][16][256] per-tile digit counts of each warp strip
  uint32_t* chunksum = nullptr;  // [table_chunks][256] per-chunk digit totals
  uint32_t* chunkoff = nullptr;  // [table_chunks][256] per-chunk digit output offsets
  uint64_t* orand = nullptr;     // [2] OR and AND of the keys of one sort (0 and all ones between calls)
  uint32_t* totals = nullptr;    // [2][256] digit totals of a pass (by pass parity; zero between uses)
  bool chained = false;          // FSORT_FLAG_CHAINED_SCATTER: always the look-back scatter
  uint32_t* leaf_part = nullptr; // expand path (16-bit keys)
  uint64_t* leaf_spill = nullptr;
  uint64_t* leaf_counts = nullptr;
  uint64_t* leaf_off = nullptr;
  void* io_keys = nullptr;       // FSORT_FLAG_HOST_IO
  uint32_t* io_vals = nullptr;

  uint32_t* h_status = nullptr;  // pinned copy of *status
  cudaEvent_t done = nullptr;
  bool pending = false;
  uint32_t last_device_flags = 0;  // raw bits of the last latched device error
  uint32_t withhold_tile = 0xFFFFFFFFu;  // failure-detection test hook (fsort_plan_set_fault_hook)
  uint64_t wait_limit_ns = 0;            // 0: the kernels' default bound

  // batched sorts (max_segments > 0)
  uint32_t max_segments = 0;
  uint64_t max_hist_chunks = 0;
  SegDesc* d_seg_large = nullptr;
  SegDesc* d_seg_small = nullptr;
  HistChunk* d_chunks = nullptr;
  uint32_t* d_tile_seg = nullptr;
  uint64_t* d_bhist = nullptr;   // [max_segments][passes][256], zero between calls
  uint64_t* d_bbases = nullptr;
  uint32_t* d_small_counter = nullptr;
  SegDesc* h_seg_large = nullptr;  // pinned staging
  SegDesc* h_seg_small = nullptr;
  HistChunk* h_chunks = nullptr;
  // table form of the large segments (fsort_batch_config::large_form = 1)
  uint64_t max_ttiles = 0, max_tchunks = 0;
  uint32_t* bt_tilerel = nullptr;   // [tiles][256] per-tile digit offsets within the tile's chunk
  uint16_t* bt_stripcnt = nullptr;  // [tiles][16][256] per-tile digit counts of each warp strip
  uint32_t* bt_chunksum = nullptr;  // [chunks][256]
  uint32_t* bt_chunkoff = nullptr;  // [chunks][256], relative to the segment's start
  uint32_t* d_chunk_seg = nullptr;  // [chunks] segment of each chunk
  uint32_t* h_chunk_seg = nullptr;  // pinned staging
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  fsort_batch_config bcfg{};
  cudaGraphExec_t gexec = nullptr;  // last captured batch
  uint64_t gkey[10] = {};

  Timing timing;
  LearnedWs* learn = nullptr;  // FSORT_FLAG_LEARNED
};

namespace {

constexpr int kRadix = 256;
constexpr size_t kCounterBytes = 256;  // two counters, padded
constexpr uint64_t kBatchHistChunk = 262144;  // keys per work item of the segmented histogram
constexpr uint32_t kBatchChunkTiles = 16;     // table form: tiles per count chunk of a large segment

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool valid_key_bits(int kb) { return kb == 16 || kb == 32 || kb == 64; }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Natural alignment of an array read or written element by element (a must be a power of two).
bool aligned_to(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

fsort_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return FSORT_OK;
  if (e == cudaErrorMemoryAllocation) return FSORT_ERR_OOM;
  return FSORT_ERR_CUDA;
}

// B for a learned sort of n keys: the smallest power of two >= n / 1024,
// clamped to [2^8, 2^22].
uint32_t learned_buckets(uint64_t n) {
  const uint64_t want = (n + kLearnKeysPerBucket - 1) / kLearnKeysPerBucket;
  uint32_t b = 256;
  while (b < want && b < (1u << 22)) b <<= 1;
  return b;
}

uint32_t log2u(uint32_t v) {
  uint32_t l = 0;
  while ((1u << l) < v) ++l;
  return l;
}

DigitPlan make_plan(int key_bits, int precision_bits, int d) {
  DigitPlan p{};
  p.passes = (precision_bits + d - 1) / d;
  const int base = key_bits - precision_bits;
  for (int j = 0; j < p.passes; ++j) {
    const int lo = j * d;
    const int width = (precision_bits - lo < d) ? (precision_bits - lo) : d;
    p.shift[j] = uint32_t(base + lo);
    p.mask[j] = (1u << width) - 1u;
  }
  return p;
}

bool use_expand(int key_bits, int precision_bits, bool has_vals) {
  return key_bits == 16 && precision_bits == 16 && !has_vals;
}

// Report (and clear) a device error latched by earlier work of this plan.
// wait: block until that work is done; otherwise look only if it already is.
fsort_status take_latched(fsort_plan* p, bool wait, cudaStream_t stream) {
  if (!p->pending) return FSORT_OK;
  if (wait) {
    if (cudaEventSynchronize(p->done) != cudaSuccess) return FSORT_ERR_CUDA;
  } else {
    const cudaError_t q = cudaEventQuery(p->done);
    if (q == cudaErrorNotReady) return FSORT_OK;
    if (q != cudaSuccess) return FSORT_ERR_CUDA;
  }
  p->pending = false;
  const uint32_t s = *p->h_status;
  if (!s) return FSORT_OK;
  p->last_device_flags = s;
  *p->h_status = 0;
  if (cudaMemsetAsync(p->status, 0, sizeof(uint32_t), stream) != cudaSuccess) return FSORT_ERR_CUDA;
  if (wait && cudaStreamSynchronize(stream) != cudaSuccess) return FSORT_ERR_CUDA;
  return (s & (kDevTimeoutLookback | kDevTimeoutLoad)) ? FSORT_ERR_TIMEOUT : FSORT_ERR_INTERNAL;
}

// After enqueuing work: copy the sticky device status back and mark the call.
fsort_status finish_call(fsort_plan* p, cudaStream_t stream) {
  cudaError_t e = cudaMemcpyAsync(p->h_status, p->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaEventRecord(p->done, stream);
  if (e != cudaSuccess) return from_cuda(e);
  p->pending = true;
  return FSORT_OK;
}

fsort_status check_call(const fsort_plan* p, uint64_t n, int key_bits, int precision_bits, bool has_vals) {
  if (!p) return FSORT_ERR_INVALID_ARG;
  if (key_bits != p->desc.key_bits) return FSORT_ERR_INVALID_ARG;
  if (precision_bits < 1 || precision_bits > key_bits) return FSORT_ERR_INVALID_ARG;
  if (n > p->desc.max_n) return FSORT_ERR_INVALID_ARG;
  if (has_vals && !p->desc.has_values) return FSORT_ERR_INVALID_ARG;
  return FSORT_OK;
}

bool overlaps(const void* a, size_t an, const void* b, size_t bn) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bn && y < x + an;
}

// Records the device time of each launch of one call when timing is on.
class CallTimer {
 public:
  CallTimer(fsort_plan* p, uint64_t n, cudaStream_t s, bool has_schedule) : p_(p), n_(n), s_(s) {
    Timing& t = p->timing;
    if (!t.on || t.next_ev + 40 > Timing::kEvents || t.next_slot >= Timing::kSlots) return;
    on_ = true;
    call_ = t.calls++;
    slot_ = has_schedule ? t.next_slot++ : -1;
    prev_ = t.next_ev++;
    cudaEventRecord(t.ev[prev_], s_);
  }
  void mark(int kind, int pass) {
    if (!on_) return;
    Timing& t = p_->timing;
    const int e = t.next_ev++;
    cudaEventRecord(t.ev[e], s_);
    t.recs.push_back(TimingRec{kind, pass, call_, slot_, n_, prev_, e});
    prev_ = e;
  }
  void finish() {
    if (on_ && slot_ >= 0)
      cudaMemcpyAsync(&p_->timing.h_sched[slot_], p_->sched, sizeof(Schedule), cudaMemcpyDeviceToHost, s_);
  }

 private:
  fsort_plan* p_;
  uint64_t n_;
  cudaStream_t s_;
  bool on_ = false;
  int call_ = -1, slot_ = -1, prev_ = -1;
};

// The whole sort, keys_in -> keys_out (equal pointers: in place).
fsort_status enqueue_sort(fsort_plan* p, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                          uint32_t* vals_out, uint64_t n, int key_bits, int precision_bits, cudaStream_t s) {
  const bool has_vals = vals_in != nullptr;
  const bool in_place = keys_in == keys_out;
  cudaError_t e = cudaSuccess;
  if (use_expand(key_bits, precision_bits, has_vals)) {
    // Expand path: the 65,536-bin histogram is the whole sorted multiset.
    CallTimer tm(p, n, s, false);
    e = launch_leaf_histogram(static_cast<const uint16_t*>(keys_in), n, p->leaf_part, p->leaf_spill, p->sms, s);
    tm.mark(FSORT_KERNEL_LEAF_HIST, -1);
    if (e == cudaSuccess) e = launch_leaf_reduce(p->leaf_part, p->leaf_spill, leaf_hist_grid(p->sms), p->leaf_counts, s);
    tm.mark(FSORT_KERNEL_LEAF_REDUCE, -1);
    if (e == cudaSuccess) e = launch_scan_rows(p->leaf_counts, p->leaf_off, 1, 65536, s);
    tm.mark(FSORT_KERNEL_LEAF_SCAN, -1);
    if (e == cudaSuccess) e = launch_expand(p->leaf_off, static_cast<uint16_t*>(keys_out), n, s);
    tm.mark(FSORT_KERNEL_EXPAND, -1);
    if (e != cudaSuccess) return from_cuda(e);
    return finish_call(p, s);
  }
  CallTimer tm(p, n, s, true);
  const DigitPlan plan = make_plan(key_bits, precision_bits, p->digit_bits);
  const void* kb[3] = {keys_in, p->alt_keys, keys_out};
  const uint32_t* vb[3] = {vals_in, p->alt_vals, vals_out};
  if (!p->chained && n <= (1ull << 32)) {  // output positions fit 32 bits (offsets are exact modulo 2^32)
    // Scatter passes over a table of per-tile offsets: one read of the input
    // for every pass's histogram and the first pass's table; before each later
    // pass, one read of its input for its table.
    const TableGeom g = table_geometry(n, key_bits, p->sms);
    TileCountArgs ca{};
    for (int b = 0; b < 3; ++b) ca.keys[b] = kb[b];
    ca.n = n;
    ca.shift = plan.shift[0];
    ca.mask = plan.mask[0];
    ca.tile = g.tile;
    ca.tiles = g.tiles;
    ca.chunk_tiles = g.chunk_tiles;
    ca.tilerel = p->tilerel;
    ca.stripcnt = p->stripcnt;
    ca.chunksum = p->chunksum;
    ca.totals = p->totals;
    ca.orand = p->orand;
    ca.status = p->status;
    // totals left dirty by an interrupted call would misplace every key: clear them
    e = cudaMemsetAsync(p->totals, 0, 2 * kRadix * 4, s);
    if (e == cudaSuccess) e = launch_tile_count(ca, key_bits, g.chunks, s);
    tm.mark(FSORT_KERNEL_HISTOGRAM, -1);
    if (e == cudaSuccess) e = launch_table_schedule(p->orand, plan, in_place ? 1 : 0, p->sched, s);
    tm.mark(FSORT_KERNEL_SCAN, -1);
    for (int j = 0; j < plan.passes && e == cudaSuccess; ++j) {
      if (j > 0) {
        TileCountArgs cj = ca;
        cj.shift = plan.shift[j];
        cj.mask = plan.mask[j];
        cj.orand = nullptr;
        cj.totals = p->totals + (j & 1) * kRadix;
        cj.sched = p->sched;
        cj.pass = j;
        e = launch_tile_count(cj, key_bits, g.chunks, s);
        tm.mark(FSORT_KERNEL_TILE_COUNT, j);
      }
      if (e == cudaSuccess)
        e = launch_chunk_scan(p->chunksum, p->totals + (j & 1) * kRadix, g.chunks, p->sched, j, p->chunkoff, s);
      tm.mark(FSORT_KERNEL_TILE_SCAN, j);
      TileScatterArgs a{};
      for (int b = 0; b < 3; ++b) {
        a.keys[b] = kb[b];
        a.vals[b] = has_vals ? vb[b] : nullptr;
      }
      a.n = n;
      a.shift = plan.shift[j];
      a.mask = plan.mask[j];
      a.tiles = g.tiles;
      a.chunk_tiles = g.chunk_tiles;
      a.tilerel = p->tilerel;
      a.stripcnt = p->stripcnt;
      a.chunkoff = p->chunkoff;
      a.totals = p->totals + (j & 1) * kRadix;
      a.sched = p->sched;
      a.pass = j;
      a.status = p->status;
      if (e == cudaSuccess) e = launch_tile_scatter(a, key_bits, has_vals, s);
      tm.mark(FSORT_KERNEL_SCATTER, j);
    }
    if (e == cudaSuccess) e = launch_schedule_copy(kb, vb, key_bits, has_vals, n, p->sched, p->sms, s);
    tm.mark(FSORT_KERNEL_COPY, -1);
    tm.finish();
    if (e != cudaSuccess) return from_cuda(e);
    return finish_call(p, s);
  }
  const uint64_t tiles = (n + p->tile - 1) / p->tile;
  const uint64_t chunks = (n + p->chunk_keys - 1) / p->chunk_keys;
  const uint64_t clear_words = kCounterBytes / 4 + tiles * kRadix;
  e = launch_histogram(keys_in, key_bits, n, plan, p->hist, kRadix, p->counters, clear_words, p->sms, s);
  tm.mark(FSORT_KERNEL_HISTOGRAM, -1);
  if (e == cudaSuccess)
    e = launch_scan_schedule(p->hist, p->chunk_base, p->chunk_flag, plan.passes, uint32_t(chunks),
                             in_place ? 1 : 0, p->sched, s);
  tm.mark(FSORT_KERNEL_SCAN, -1);
  for (int j = 0; j < plan.passes && e == cudaSuccess; ++j) {
    OnesweepArgs a{};
    for (int b = 0; b < 3; ++b) {
      a.keys[b] = kb[b];
      a.vals[b] = has_vals ? vb[b] : nullptr;
    }
    a.n = n;
    a.shift = plan.shift[j];
    a.mask = plan.mask[j];
    a.lookback = p->lookback[j & 1];
    a.tile_counter = p->counters + (j & 1);
    const bool last = (j + 1 == plan.passes);
    a.next_lookback = last ? nullptr : p->lookback[(j + 1) & 1];
    a.next_counter = last ? nullptr : p->counters + ((j + 1) & 1);
    a.chunk_base = p->chunk_base + uint64_t(j) * chunks * kRadix;
    a.chunk_flag = p->chunk_flag + uint64_t(j) * chunks;
    a.sched = p->sched;
    a.pass = j;
    a.tiles_per_chunk = uint32_t(p->chunk_keys / p->tile);
    a.status = p->status;
    a.withhold_tile = p->withhold_tile;
    a.wait_limit_ns = p->wait_limit_ns;
    e = launch_onesweep(a, key_bits, has_vals, s);
    tm.mark(FSORT_KERNEL_SCATTER, j);
  }
  if (e == cudaSuccess) e = launch_schedule_copy(kb, vb, key_bits, has_vals, n, p->sched, p->sms, s);
  tm.mark(FSORT_KERNEL_COPY, -1);
  tm.finish();
  if (e != cudaSuccess) return from_cuda(e);
  return finish_call(p, s);
}

// ---- learned bucket mapping ----
bool learned_eligible(const fsort_plan* p, const uint32_t* vals, uint64_t n, int key_bits, int precision_bits) {
  return p->learn && p->learn->fitted && !vals && key_bits == 64 && precision_bits == 64 && n > 0 &&
         n < (1ull << 32);
}

LearnedMap learned_map(const LearnedWs& L, uint64_t n) {
  return LearnedMap{L.cells, L.heavy, 32u - log2u(learned_buckets(n))};
}

// Level-1 and level-2 counts, the judge (host read-back); on acceptance the
// scatters, the heavy fill and the bucket sorts, else the plain path on the
// untouched input.  keys_in == keys_out: in place.
fsort_status enqueue_learned(fsort_plan* p, const void* keys_in, void* keys_out, uint64_t n, cudaStream_t s) {
  LearnedWs& L = *p->learn;
  const uint32_t B = learned_buckets(n);
  const LearnedGeom g = learned_geometry(n, B);
  const LearnedMap mp = learned_map(L, n);
  const uint64_t* kin = static_cast<const uint64_t*>(keys_in);
  uint64_t* kout = static_cast<uint64_t*>(keys_out);
  uint64_t* alt = static_cast<uint64_t*>(p->alt_keys);
  const uint64_t l1n = uint64_t(g.nsuper) * g.nch;
  CallTimer tm(p, n, s, false);
  cudaError_t e = cudaMemsetAsync(L.hcount, 0, size_t(kLearnMaxHeavy) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.bitmap, 0, size_t(g.nids / 32 + 1) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.counts1 + l1n, 0, 4, s);
  if (e == cudaSuccess) e = launch_learn_heavy_ids(mp, L.st, L.hid, L.bitmap, s);
  if (e == cudaSuccess) e = launch_learn_l1(kin, n, g, mp, L.st, L.heavy_count, L.counts1, L.hcount, L.ids, s);
  tm.mark(FSORT_KERNEL_LEARN_COUNT1, -1);
  if (e == cudaSuccess) e = launch_scan_u32(L.counts1, l1n + 1, L.off1, nullptr, L.sums, s);
  if (e == cudaSuccess) e = launch_learn_l1_scatter(kin, L.ids, n, g, L.off1, alt, L.fine, s);
  tm.mark(FSORT_KERNEL_LEARN_SCATTER1, -1);
  if (e == cudaSuccess) e = launch_learn_l2_count(L.fine, g, L.off1, L.counts, s);
  tm.mark(FSORT_KERNEL_LEARN_COUNT2, -1);
  if (e == cudaSuccess) e = launch_learn_judge(L.counts, g, L.bitmap, L.hid, L.hcount, L.st, L.large, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.h_st, L.st, sizeof(LearnedState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  tm.mark(FSORT_KERNEL_LEARN_JUDGE, -1);
  if (e != cudaSuccess) return from_cuda(e);
  const uint64_t limit = uint64_t(kLearnTau) * n / B;
  const uint32_t mx = L.h_st->max_nonheavy;
  const bool accept = mx <= limit && mx <= uint32_t(kLearnBucketCap);
  L.used = accept ? 1 : 0;
  L.last_b = B;
  L.last_limit = uint32_t(limit);
  L.last_max = mx;
  L.last_heavy = L.h_st->heavy_count;
  L.heavy_count = L.h_st->heavy_count < uint32_t(kLearnMaxHeavy) ? L.h_st->heavy_count : uint32_t(kLearnMaxHeavy);
  L.last_imbalance = double(mx) * double(B) / double(n);
  if (!accept) return enqueue_sort(p, keys_in, nullptr, keys_out, nullptr, n, 64, 64, s);
  e = launch_scan_u32(L.counts, g.nids, L.offsets, nullptr, L.sums, s);
  if (e == cudaSuccess) e = launch_learn_l2_scatter(alt, L.fine, g, L.off1, L.offsets, kout, s);
  tm.mark(FSORT_KERNEL_LEARN_SCATTER2, -1);
  if (e == cudaSuccess) e = launch_learn_fill(mp, L.st, L.hid, L.large, L.offsets, L.counts, kout, p->sms, s);
  tm.mark(FSORT_KERNEL_LEARN_FILL, -1);
  if (e == cudaSuccess)
    e = launch_learn_bucket_sort(kout, L.counts, L.offsets, L.bitmap, g.nids, L.units, p->status, p->sms, s);
  tm.mark(FSORT_KERNEL_LEARN_BUCKETS, -1);
  if (e != cudaSuccess) return from_cuda(e);
  return finish_call(p, s);
}

// Every sort entry point: the learned path where it applies, else the plain one.
fsort_status enqueue_any(fsort_plan* p, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                         uint32_t* vals_out, uint64_t n, int key_bits, int precision_bits, cudaStream_t s) {
  if (learned_eligible(p, vals_in, n, key_bits, precision_bits)) return enqueue_learned(p, keys_in, keys_out, n, s);
  return enqueue_sort(p, keys_in, vals_in, keys_out, vals_out, n, key_bits, precision_bits, s);
}

// Seeded initial weights: first-layer kinks spread evenly over the feature
// range [-1, 1], He-scaled hidden layer, small output layer.
void learned_init_params(std::vector<float>& w, uint64_t seed) {
  w.assign(kMlpParams, 0.f);
  uint64_t z = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  auto next = [&]() {  // splitmix64 (Steele, Lea and Flood, 2014) -> uniform [0, 1)
    z += 0x9E3779B97F4A7C15ull;
    uint64_t x = z;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return double(x >> 11) * (1.0 / 9007199254740992.0);
  };
  auto normal = [&]() {  // Box-Muller
    const double u1 = next() + 1e-300, u2 = next();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  const int H = kMlpHidden;
  for (int i = 0; i < H; ++i) {
    const double slope = (2.0 + 6.0 * next()) * ((i & 1) ? -1.0 : 1.0);
    const double kink = -1.0 + 2.0 * (i + 0.5) / H;
    w[i] = float(slope);                 // W1
    w[H + i] = float(-slope * kink);     // b1
  }
  const int w2 = 2 * H, b2 = w2 + H * H, w3 = b2 + H;
  for (int i = 0; i < H * H; ++i) w[w2 + i] = float(normal() * std::sqrt(2.0 / H));
  for (int i = 0; i < H; ++i) w[b2 + i] = 0.f;
  for (int i = 0; i < H; ++i) w[w3 + i] = float(normal() * std::sqrt(1.0 / H));
  w[w3 + H] = 0.f;  // b3
}

// Batched sorts: build the segment lists on the host (pinned staging), then
// enqueue the small-segment kernel on a side stream and the large-segment
// passes on `s`, joined at the end.  With FSORT_FLAG_GRAPH and a non-default
// stream, the enqueued work is captured once per batch shape and replayed: the
// kernels read the segment lists from plan memory, so one graph serves every
// batch of the same shape.
struct BatchShape {
  uint32_t n_large = 0, n_small = 0, n_chunks = 0, total_tiles = 0;
  uint32_t n_tchunks = 0;  // table form: count chunks over all large segments
  uint64_t alt_total = 0;
  bool has_vals = false;
};

fsort_status build_batch(fsort_plan* p, const fsort_segment* segs, uint32_t count, int key_bits, BatchShape* out) {
  const int cap = p->bcfg.small_capacity;
  const bool table = p->bcfg.large_form == 1;
  const uint64_t tile = table ? uint64_t(table_tile_keys_for(key_bits)) : uint64_t(p->tile);
  BatchShape b;
  int vals_state = -1;  // -1 unknown, 0 none, 1 all
  for (uint32_t i = 0; i < count; ++i) {
    const fsort_segment& g = segs[i];
    if (g.n == 0) continue;
    if (!g.keys || g.n >= (1ull << 31)) return FSORT_ERR_INVALID_ARG;
    const int hv = g.vals != nullptr;
    if (vals_state < 0) vals_state = hv;
    if (vals_state != hv) return FSORT_ERR_INVALID_ARG;
    if (hv && !p->desc.has_values) return FSORT_ERR_INVALID_ARG;
    const uintptr_t ka = reinterpret_cast<uintptr_t>(g.keys);
    if (ka % uintptr_t(key_bits / 8)) return FSORT_ERR_INVALID_ARG;
    if (hv && (reinterpret_cast<uintptr_t>(g.vals) & 3u)) return FSORT_ERR_INVALID_ARG;
    SegDesc d{g.keys, g.vals, g.n, 0, 0, 0};
    if (cap > 0 && g.n <= uint64_t(cap)) {
      p->h_seg_small[b.n_small++] = d;
      continue;
    }
    if (!aligned16(g.keys) || (hv && !aligned16(g.vals))) return FSORT_ERR_INVALID_ARG;
    d.alt_off = b.alt_total;
    d.first_tile = b.total_tiles;
    b.alt_total += (g.n + 7) / 8 * 8;  // keeps every segment's scratch 16-byte aligned
    if (b.alt_total > p->desc.max_n) return FSORT_ERR_INVALID_ARG;
    const uint64_t tiles = (g.n + tile - 1) / tile;
    if (uint64_t(b.total_tiles) + tiles > (table ? p->max_ttiles : p->max_tiles)) return FSORT_ERR_INVALID_ARG;
    b.total_tiles += uint32_t(tiles);
    if (table) {  // count chunks of the segment, and nothing for the segmented histogram
      const uint64_t nch = (tiles + kBatchChunkTiles - 1) / kBatchChunkTiles;
      if (uint64_t(b.n_tchunks) + nch > p->max_tchunks) return FSORT_ERR_INVALID_ARG;
      d.first_chunk = b.n_tchunks;
      for (uint64_t c = 0; c < nch; ++c) p->h_chunk_seg[b.n_tchunks++] = b.n_large;
      p->h_seg_large[b.n_large++] = d;
      continue;
    }
    for (uint64_t st = 0; st < g.n; st += kBatchHistChunk) {
      if (b.n_chunks >= p->max_hist_chunks) return FSORT_ERR_INVALID_ARG;
      const uint64_t len = (g.n - st < kBatchHistChunk) ? g.n - st : kBatchHistChunk;
      p->h_chunks[b.n_chunks++] = HistChunk{b.n_large, uint32_t(len), st};
    }
    p->h_seg_large[b.n_large++] = d;
  }
  b.has_vals = vals_state == 1;
  *out = b;
  return FSORT_OK;
}

// Digit width of the batched path's passes (fsort_batch_config::digit_bits, 0 = 8).
int batch_digits(const fsort_plan* p) { return p->bcfg.digit_bits ? p->bcfg.digit_bits : 8; }

// Most passes a batch of this key width can take: at 6-bit digits for 16- and
// 32-bit keys, at 8-bit digits for 64-bit keys.
int batch_max_passes(int key_bits) { return key_bits == 64 ? 8 : (key_bits + 5) / 6; }

cudaError_t enqueue_batch(fsort_plan* p, const BatchShape& b, int key_bits, int precision_bits, cudaStream_t s) {
  const DigitPlan plan = make_plan(key_bits, precision_bits, batch_digits(p));
  cudaError_t e = cudaSuccess;
  if (b.n_large) e = cudaMemcpyAsync(p->d_seg_large, p->h_seg_large, sizeof(SegDesc) * b.n_large,
                                     cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && b.n_small)
    e = cudaMemcpyAsync(p->d_seg_small, p->h_seg_small, sizeof(SegDesc) * b.n_small, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && b.n_chunks)
    e = cudaMemcpyAsync(p->d_chunks, p->h_chunks, sizeof(HistChunk) * b.n_chunks, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && b.n_small) e = cudaMemsetAsync(p->d_small_counter, 0, 4, s);
  if (e == cudaSuccess && b.n_small) {
    e = cudaEventRecord(p->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side, p->ev_fork, 0);
    if (e == cudaSuccess)
      e = launch_small_sort(p->d_seg_small, b.n_small, key_bits, b.has_vals, p->bcfg.small_capacity, plan,
                            p->d_small_counter, p->bcfg.small_ctas_per_sm * p->sms, p->side);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_join, p->side);
  }
  if (e == cudaSuccess && b.n_large && p->bcfg.large_form == 1) {
    // Table form: per pass, one read of the segments' keys counts every tile
    // (chunks of kBatchChunkTiles tiles inside one segment), a per-segment
    // scan turns the counts into offsets, and every tile scatters at once.
    const uint32_t tile = uint32_t(table_tile_keys_for(key_bits));
    e = cudaMemcpyAsync(p->d_chunk_seg, p->h_chunk_seg, sizeof(uint32_t) * b.n_tchunks, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_fill_tile_seg(p->d_seg_large, b.n_large, int(tile), p->d_tile_seg, s);
    for (int j = 0; j < plan.passes && e == cudaSuccess; ++j) {
      TileCountArgs ca{};
      ca.keys[kBufAlt] = p->alt_keys;
      ca.shift = plan.shift[j];
      ca.mask = plan.mask[j];
      ca.tile = tile;
      ca.tiles = b.total_tiles;
      ca.chunk_tiles = kBatchChunkTiles;
      ca.tilerel = p->bt_tilerel;
      ca.stripcnt = p->bt_stripcnt;
      ca.chunksum = p->bt_chunksum;
      ca.pass = j;
      ca.status = p->status;
      ca.segs = p->d_seg_large;
      ca.chunk_seg = p->d_chunk_seg;
      e = launch_tile_count(ca, key_bits, b.n_tchunks, s);
      if (e == cudaSuccess)
        e = launch_seg_chunk_scan(p->bt_chunksum, p->d_seg_large, b.n_large, tile, kBatchChunkTiles, p->bt_chunkoff, s);
      TileScatterArgs a{};
      a.keys[kBufAlt] = p->alt_keys;
      a.vals[kBufAlt] = b.has_vals ? p->alt_vals : nullptr;
      a.shift = plan.shift[j];
      a.mask = plan.mask[j];
      a.tiles = b.total_tiles;
      a.chunk_tiles = kBatchChunkTiles;
      a.tilerel = p->bt_tilerel;
      a.stripcnt = p->bt_stripcnt;
      a.chunkoff = p->bt_chunkoff;
      a.pass = j;
      a.status = p->status;
      a.segs = p->d_seg_large;
      a.tile_seg = p->d_tile_seg;
      if (e == cudaSuccess) e = launch_tile_scatter(a, key_bits, b.has_vals, s);
    }
    if (e == cudaSuccess && (plan.passes & 1))
      e = launch_seg_copy_back(p->d_seg_large, b.n_large, p->alt_keys, b.has_vals ? p->alt_vals : nullptr, key_bits,
                               p->sms, s);
  } else if (e == cudaSuccess && b.n_large) {  // chained form: segmented decoupled look-back
    e = launch_fill_tile_seg(p->d_seg_large, b.n_large, p->tile, p->d_tile_seg, s);
    if (e == cudaSuccess)
      e = launch_seg_histogram(p->d_seg_large, p->d_chunks, b.n_chunks, key_bits, plan, p->d_bhist, p->counters,
                               kCounterBytes / 4 + uint64_t(b.total_tiles) * kRadix, s);
    if (e == cudaSuccess) e = launch_seg_scan(p->d_bhist, p->d_bbases, b.n_large, plan.passes, s);
    for (int j = 0; j < plan.passes && e == cudaSuccess; ++j) {
      OnesweepArgs a{};
      a.keys[kBufAlt] = p->alt_keys;
      a.vals[kBufAlt] = b.has_vals ? p->alt_vals : nullptr;
      a.n = b.alt_total;
      a.shift = plan.shift[j];
      a.mask = plan.mask[j];
      a.lookback = p->lookback[j & 1];
      a.tile_counter = p->counters + (j & 1);
      const bool last = (j + 1 == plan.passes);
      a.next_lookback = last ? nullptr : p->lookback[(j + 1) & 1];
      a.next_counter = last ? nullptr : p->counters + ((j + 1) & 1);
      a.chunk_base = p->d_bbases;
      a.chunk_flag = nullptr;
      a.sched = nullptr;
      a.pass = j;
      a.tiles_per_chunk = 1;
      a.status = p->status;
      a.segs = p->d_seg_large;
      a.tile_seg = p->d_tile_seg;
      a.passes = uint32_t(plan.passes);
      a.total_tiles = b.total_tiles;
      a.withhold_tile = p->withhold_tile;
      a.wait_limit_ns = p->wait_limit_ns;
      e = launch_onesweep(a, key_bits, b.has_vals, s);
    }
    if (e == cudaSuccess && (plan.passes & 1))
      e = launch_seg_copy_back(p->d_seg_large, b.n_large, p->alt_keys, b.has_vals ? p->alt_vals : nullptr, key_bits,
                               p->sms, s);
  }
  if (e == cudaSuccess && b.n_small) e = cudaStreamWaitEvent(s, p->ev_join, 0);
  return e;
}

fsort_status run_batch(fsort_plan* p, const fsort_segment* segs, uint32_t count, int key_bits, int precision_bits,
                       cudaStream_t s, bool allow_graph) {
  // The pinned staging is rewritten below: let the previous call finish with it.
  if (p->pending && cudaEventSynchronize(p->done) != cudaSuccess) return FSORT_ERR_CUDA;
  BatchShape b;
  fsort_status st = build_batch(p, segs, count, key_bits, &b);
  if (st != FSORT_OK) return st;
  if (!b.n_large && !b.n_small) return FSORT_OK;
  const bool graph = allow_graph && (p->desc.flags & FSORT_FLAG_GRAPH) && s != nullptr;
  if (!graph) {
    const cudaError_t e = enqueue_batch(p, b, key_bits, precision_bits, s);
    if (e != cudaSuccess) return from_cuda(e);
    return finish_call(p, s);
  }
  const uint64_t key[10] = {b.n_large, b.n_small, uint64_t(b.n_chunks) << 32 | b.n_tchunks, b.total_tiles, b.alt_total,
                            uint64_t(b.has_vals) | uint64_t(p->bcfg.large_form) << 1,
                            uint64_t(key_bits) << 8 | uint64_t(precision_bits), uint64_t(p->bcfg.small_capacity),
                            uint64_t(p->bcfg.small_ctas_per_sm) | uint64_t(batch_digits(p)) << 32,
                            reinterpret_cast<uint64_t>(s)};
  if (!p->gexec || std::memcmp(key, p->gkey, sizeof(key)) != 0) {
    if (p->gexec) {
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return from_cuda(e);
    const cudaError_t ee = enqueue_batch(p, b, key_bits, precision_bits, s);
    e = cudaStreamEndCapture(s, &g);
    if (ee != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return FSORT_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      p->gexec = nullptr;
      return from_cuda(e);
    }
    std::memcpy(p->gkey, key, sizeof(key));
  }
  const cudaError_t e = cudaGraphLaunch(p->gexec, s);
  if (e != cudaSuccess) return from_cuda(e);
  return finish_call(p, s);
}

}  // namespace

extern "C" {

fsort_status fsort_sort_batch(fsort_plan* plan, const fsort_segment* segments, uint32_t count, int key_bits,
                              int precision_bits, void* stream) {
  if (!plan || !plan->max_segments) return FSORT_ERR_INVALID_ARG;
  if (count > plan->max_segments || (count && !segments)) return FSORT_ERR_INVALID_ARG;
  fsort_status st = check_call(plan, 0, key_bits, precision_bits, false);
  if (st != FSORT_OK) return st;
  if (count == 0) return FSORT_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = take_latched(plan, false, s);
  if (st != FSORT_OK) return st;
  return run_batch(plan, segments, count, key_bits, precision_bits, s, true);
}

fsort_status fsort_batch_set_config(fsort_plan* plan, const fsort_batch_config* config) {
  if (!plan || !config || !plan->max_segments) return FSORT_ERR_INVALID_ARG;
  const int c = config->small_capacity;
  if (c != 0 && c != 1024 && c != 2048 && c != 4096) return FSORT_ERR_INVALID_ARG;
  if (config->small_ctas_per_sm < 1 || config->small_ctas_per_sm > 8) return FSORT_ERR_INVALID_ARG;
  if (c && config->small_ctas_per_sm > small_sort_ctas_per_sm(plan->desc.key_bits, plan->desc.has_values != 0, c))
    return FSORT_ERR_INVALID_ARG;  // more CTAs than shared memory holds at once
  if (config->large_form != 0 && config->large_form != 1) return FSORT_ERR_INVALID_ARG;
  const int w = config->digit_bits;
  if (w != 0 && w != 6 && w != 7 && w != 8) return FSORT_ERR_INVALID_ARG;
  if (plan->desc.key_bits == 64 && w != 0 && w != 8) return FSORT_ERR_INVALID_ARG;  // more passes than the buffers hold
  plan->bcfg = *config;
  return FSORT_OK;
}

fsort_status fsort_batch_get_config(const fsort_plan* plan, fsort_batch_config* config) {
  if (!plan || !config || !plan->max_segments) return FSORT_ERR_INVALID_ARG;
  *config = plan->bcfg;
  return FSORT_OK;
}

fsort_status fsort_batch_autotune(fsort_plan* plan, const fsort_segment* segments, uint32_t count, int key_bits,
                                  int precision_bits, void* stream, fsort_batch_config* best, float* best_ms) {
  if (!plan || !plan->max_segments || !best) return FSORT_ERR_INVALID_ARG;
  if (count > plan->max_segments || (count && !segments)) return FSORT_ERR_INVALID_ARG;
  fsort_status st = check_call(plan, 0, key_bits, precision_bits, false);
  if (st != FSORT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = take_latched(plan, true, s);
  if (st != FSORT_OK) return st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return FSORT_ERR_CUDA;
  const fsort_batch_config saved = plan->bcfg;
  fsort_batch_config winner = saved;
  float winner_ms = -1.f;
  const bool hv = plan->desc.has_values != 0;
  // one timed batch (after a warm-up one) under the plan's current config
  auto time_config = [&](float* ms) -> fsort_status {
    fsort_status r = run_batch(plan, segments, count, key_bits, precision_bits, s, false);  // warm-up
    if (r == FSORT_OK && cudaEventRecord(e0, s) != cudaSuccess) r = FSORT_ERR_CUDA;
    if (r == FSORT_OK) r = run_batch(plan, segments, count, key_bits, precision_bits, s, false);
    if (r == FSORT_OK && cudaEventRecord(e1, s) != cudaSuccess) r = FSORT_ERR_CUDA;
    if (r == FSORT_OK && cudaEventSynchronize(e1) != cudaSuccess) r = FSORT_ERR_CUDA;
    if (r == FSORT_OK && cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) r = FSORT_ERR_CUDA;
    return r;
  };
  auto consider = [&](float ms) {
    if (winner_ms < 0.f || ms < winner_ms) {
      winner_ms = ms;
      winner = plan->bcfg;
    }
  };
  // Coordinate search: the large segments' form under the current small-segment
  // configuration, then every small-segment configuration under that form.
  for (int form : {1, 0}) {
    plan->bcfg = saved;
    plan->bcfg.large_form = form;
    float ms = 0.f;
    st = time_config(&ms);
    if (st != FSORT_OK) break;
    consider(ms);
  }
  const int form = winner.large_form, width = saved.digit_bits;
  for (int cap : {0, 1024, 2048, 4096}) {
    if (st != FSORT_OK) break;
    const int most = cap ? small_sort_ctas_per_sm(key_bits, hv, cap) : 1;
    for (int ctas : {most, (most + 1) / 2}) {
      if (cap == 0 && ctas != most) continue;
      plan->bcfg.small_capacity = cap;
      plan->bcfg.small_ctas_per_sm = ctas;
      plan->bcfg.large_form = form;
      plan->bcfg.digit_bits = width;
      float ms = 0.f;
      st = time_config(&ms);
      if (st != FSORT_OK) break;
      consider(ms);
    }
  }
  // then the digit width under the best of those (the current width is measured already)
  const fsort_batch_config best_so_far = winner;
  for (int w : {8, 7, 6}) {
    if (st != FSORT_OK || key_bits == 64) break;
    if (w == (width ? width : 8)) continue;
    plan->bcfg = best_so_far;
    plan->bcfg.digit_bits = w;
    float ms = 0.f;
    st = time_config(&ms);
    if (st != FSORT_OK) break;
    consider(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan->bcfg = (st == FSORT_OK) ? winner : saved;
  if (st != FSORT_OK) return st;
  *best = winner;
  if (best_ms) *best_ms = winner_ms;
  return take_latched(plan, true, s);
}


fsort_status fsort_plan_create(const fsort_plan_desc* desc, fsort_plan** out_plan) {
  if (!desc || !out_plan) return FSORT_ERR_INVALID_ARG;
  if (!valid_key_bits(desc->key_bits) || desc->max_n < 1) return FSORT_ERR_INVALID_ARG;
  if (desc->has_values != 0 && desc->has_values != 1) return FSORT_ERR_INVALID_ARG;
  if (desc->digit_bits != 0 && desc->digit_bits != 8) return FSORT_ERR_UNSUPPORTED;
  if (desc->flags & ~(FSORT_FLAG_HOST_IO | FSORT_FLAG_GRAPH | FSORT_FLAG_LEARNED | FSORT_FLAG_CHAINED_SCATTER))
    return FSORT_ERR_INVALID_ARG;
  if ((desc->flags & FSORT_FLAG_LEARNED) && desc->key_bits != 64) return FSORT_ERR_UNSUPPORTED;
  if (desc->max_n > (1ull << 36)) return FSORT_ERR_UNSUPPORTED;

  fsort_plan* p = new (std::nothrow) fsort_plan();
  if (!p) return FSORT_ERR_OOM;
  p->desc = *desc;
  p->digit_bits = 8;
  if (cudaGetDevice(&p->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    delete p;
    return FSORT_ERR_CUDA;
  }
  const int kb = desc->key_bits / 8;
  const uint64_t n = desc->max_n;
  p->chained = (desc->flags & FSORT_FLAG_CHAINED_SCATTER) != 0;
  if (!p->chained) {
    const uint64_t tn = n < (1ull << 32) ? n : (1ull << 32);
    const uint64_t tt = uint64_t(table_tile_keys_for(desc->key_bits));
    p->table_tiles = (tn + tt - 1) / tt;
    p->table_chunks = uint32_t(p->sms) * 2;
  }
  p->tile = tile_keys_for(desc->key_bits);
  p->chunk_keys = chunk_keys_for(desc->key_bits);
  p->max_tiles = (n + p->tile - 1) / p->tile;
  p->max_chunks = (n + p->chunk_keys - 1) / p->chunk_keys;
  if (desc->max_segments > 0) {
    p->max_segments = desc->max_segments;
    p->max_tiles += desc->max_segments;  // every batch segment may add one partial tile
  }

  // Carve the scratch out of one allocation.
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  const size_t o_alt_k = take(n * kb);
  const size_t o_alt_v = desc->has_values ? take(n * 4) : 0;
  const size_t o_cnt = take(kCounterBytes + p->max_tiles * kRadix * 4);  // counters + region 0
  const size_t o_lb1 = take(p->max_tiles * kRadix * 4);
  const size_t hist_bytes = size_t(kMaxPasses) * kRadix * 8;
  const size_t o_hist = take(hist_bytes);
  const size_t o_cbase = take(size_t(kMaxPasses) * p->max_chunks * kRadix * 8);
  const size_t o_cflag = take(size_t(kMaxPasses) * p->max_chunks * 4);
  const size_t o_sched = take(sizeof(Schedule));
  const size_t o_status = take(sizeof(uint32_t));
  const size_t o_trel = take(size_t(p->table_tiles) * kRadix * 4);
  const size_t o_csum = take(size_t(p->table_chunks) * kRadix * 4);
  const size_t o_coff = take(size_t(p->table_chunks) * kRadix * 4);
  const size_t o_orand = take(2 * sizeof(uint64_t));
  const size_t o_totals = take(2 * kRadix * 4);
  size_t o_lpart = 0, o_lspill = 0, o_lcnt = 0, o_loff = 0;
  const bool batch = desc->max_segments > 0;
  if (desc->max_segments > 65535) {
    delete p;
    return FSORT_ERR_INVALID_ARG;
  }
  const int pmax = batch_max_passes(desc->key_bits);
  size_t o_bsl = 0, o_bss = 0, o_bch = 0, o_bts = 0, o_bh = 0, o_bb = 0, o_bctr = 0;
  size_t o_btr = 0, o_btcs = 0, o_btco = 0, o_btseg = 0, o_btsc = 0;
  if (batch) {
    p->max_hist_chunks = n / kBatchHistChunk + desc->max_segments + 1;
    o_bsl = take(size_t(desc->max_segments) * sizeof(SegDesc));
    o_bss = take(size_t(desc->max_segments) * sizeof(SegDesc));
    o_bch = take(size_t(p->max_hist_chunks) * sizeof(HistChunk));
    o_bts = take(size_t(p->max_tiles) * 4);
    o_bh = take(size_t(desc->max_segments) * pmax * kRadix * 8);
    o_bb = take(size_t(desc->max_segments) * pmax * kRadix * 8);
    o_bctr = take(4);
    const uint64_t tt = uint64_t(table_tile_keys_for(desc->key_bits));
    p->max_ttiles = n / tt + desc->max_segments + 1;  // every segment may add one partial tile
    p->max_tchunks = p->max_ttiles / kBatchChunkTiles + desc->max_segments + 1;
    o_btr = take(size_t(p->max_ttiles) * kRadix * 4);
    o_btsc = take(size_t(p->max_ttiles) * kTableStrips * kRadix * 2);
    o_btcs = take(size_t(p->max_tchunks) * kRadix * 4);
    o_btco = take(size_t(p->max_tchunks) * kRadix * 4);
    o_btseg = take(size_t(p->max_tchunks) * 4);
  }
  const bool leaf = desc->key_bits == 16;
  if (leaf) {
    o_lpart = take(size_t(leaf_hist_grid(p->sms)) * 32768 * 4);
    o_lspill = take(65536 * 8);
    o_lcnt = take(65536 * 8);
    o_loff = take(65536 * 8);
  }
  size_t o_iok = 0, o_iov = 0;
  const bool hio = (desc->flags & FSORT_FLAG_HOST_IO) != 0;
  if (hio) {
    o_iok = take(n * kb);
    if (desc->has_values) o_iov = take(n * 4);
  }
  const bool learned = (desc->flags & FSORT_FLAG_LEARNED) != 0;
  LearnedWs lw;
  size_t o_l[28] = {};
  if (learned) {
    lw.sample_max = uint32_t(n < LearnedWs::kMaxSample ? n : LearnedWs::kMaxSample);
    // the largest id table and level-1 count table over every B a sort on this plan may use
    for (uint32_t b = 256; b <= learned_buckets(n); b <<= 1) {
      const LearnedGeom gm = learned_geometry(n, b);
      if (gm.nids > lw.nids_max) lw.nids_max = gm.nids;
      if (uint64_t(gm.nsuper) * kLearnL1Chunks + 1 > lw.l1_max) lw.l1_max = uint64_t(gm.nsuper) * kLearnL1Chunks + 1;
    }
    const size_t sm = lw.sample_max, nb = lw.nids_max + 1, l1 = lw.l1_max;
    const size_t big = sm > nb ? (sm > l1 ? sm : l1) : (nb > l1 ? nb : l1);
    const size_t scan_words = big / 4096 + 2;
    o_l[0] = take(sm * 8);
    o_l[1] = take(sm * 8);
    o_l[2] = take(sm * 4);
    o_l[3] = take(sm * 4);
    o_l[4] = take(sm * 4);
    o_l[5] = take(sm * 4);
    o_l[6] = take(scan_words * 4);
    o_l[7] = take(size_t(kLearnMaxHeavy) * 8);
    o_l[8] = take(size_t(kLearnMaxHeavy) * 4);
    o_l[9] = take(size_t(kLearnMaxHeavy) * 4);
    o_l[10] = take(size_t(kLearnCells + 1) * 8);
    o_l[11] = take(size_t(kLearnCells + 1) * 4);
    o_l[12] = take(nb * 4);
    o_l[13] = take(nb * 4);
    o_l[14] = take(size_t(kLearnMaxHeavy) * 4);
    o_l[15] = take((nb / 32 + 1) * 4);
    o_l[23] = take(l1 * 4);
    o_l[24] = take(l1 * 4);
    o_l[25] = take(((nb + 3) / 4 * 4 + 1) * 8);
    o_l[26] = take(size_t(n) * 4);
    o_l[27] = take(size_t(n) * 2);
    o_l[16] = take(size_t(kMlpParams) * 2);
    o_l[17] = take(size_t(kMlpParams) * 4);
    o_l[18] = take(size_t(kMlpParams) * 4);
    o_l[19] = take(size_t(kMlpParams) * 4);
    o_l[20] = take(size_t(kMlpParams) * 4);
    o_l[21] = take(size_t(LearnedWs::kMaxSteps) * 4);
    o_l[22] = take(sizeof(LearnedState));
  }
  // The strip table last: placed before the learned arrays, it moved them and
  // the learned level-1 count measured a sixth slower; here it leaves every
  // other array where it was.
  const size_t o_tsc = take(size_t(p->table_tiles) * kTableStrips * kRadix * 2);
  p->ws_bytes = off;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p->ws), p->ws_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return FSORT_ERR_OOM;
  }
  unsigned char* w = p->ws;
  p->alt_keys = w + o_alt_k;
  p->alt_vals = desc->has_values ? reinterpret_cast<uint32_t*>(w + o_alt_v) : nullptr;
  p->counters = reinterpret_cast<uint32_t*>(w + o_cnt);
  p->lookback[0] = reinterpret_cast<uint32_t*>(w + o_cnt + kCounterBytes);
  p->lookback[1] = reinterpret_cast<uint32_t*>(w + o_lb1);
  p->hist = reinterpret_cast<uint64_t*>(w + o_hist);
  p->chunk_base = reinterpret_cast<uint64_t*>(w + o_cbase);
  p->chunk_flag = reinterpret_cast<uint32_t*>(w + o_cflag);
  p->sched = reinterpret_cast<Schedule*>(w + o_sched);
  p->status = reinterpret_cast<uint32_t*>(w + o_status);
  p->tilerel = reinterpret_cast<uint32_t*>(w + o_trel);
  p->stripcnt = reinterpret_cast<uint16_t*>(w + o_tsc);
  p->chunksum = reinterpret_cast<uint32_t*>(w + o_csum);
  p->chunkoff = reinterpret_cast<uint32_t*>(w + o_coff);
  p->orand = reinterpret_cast<uint64_t*>(w + o_orand);
  p->totals = reinterpret_cast<uint32_t*>(w + o_totals);
  if (batch) {
    p->d_seg_large = reinterpret_cast<SegDesc*>(w + o_bsl);
    p->d_seg_small = reinterpret_cast<SegDesc*>(w + o_bss);
    p->d_chunks = reinterpret_cast<HistChunk*>(w + o_bch);
    p->d_tile_seg = reinterpret_cast<uint32_t*>(w + o_bts);
    p->d_bhist = reinterpret_cast<uint64_t*>(w + o_bh);
    p->d_bbases = reinterpret_cast<uint64_t*>(w + o_bb);
    p->d_small_counter = reinterpret_cast<uint32_t*>(w + o_bctr);
    p->bt_tilerel = reinterpret_cast<uint32_t*>(w + o_btr);
    p->bt_stripcnt = reinterpret_cast<uint16_t*>(w + o_btsc);
    p->bt_chunksum = reinterpret_cast<uint32_t*>(w + o_btcs);
    p->bt_chunkoff = reinterpret_cast<uint32_t*>(w + o_btco);
    p->d_chunk_seg = reinterpret_cast<uint32_t*>(w + o_btseg);
  }
  if (leaf) {
    p->leaf_part = reinterpret_cast<uint32_t*>(w + o_lpart);
    p->leaf_spill = reinterpret_cast<uint64_t*>(w + o_lspill);
    p->leaf_counts = reinterpret_cast<uint64_t*>(w + o_lcnt);
    p->leaf_off = reinterpret_cast<uint64_t*>(w + o_loff);
  }
  if (hio) {
    p->io_keys = w + o_iok;
    p->io_vals = desc->has_values ? reinterpret_cast<uint32_t*>(w + o_iov) : nullptr;
  }
  if (learned) {
    p->learn = new (std::nothrow) LearnedWs(lw);
    if (!p->learn) {
      fsort_plan_destroy(p);
      return FSORT_ERR_OOM;
    }
    LearnedWs& L = *p->learn;
    L.sample = reinterpret_cast<uint64_t*>(w + o_l[0]);
    L.train = reinterpret_cast<uint64_t*>(w + o_l[1]);
    L.flag_nh = reinterpret_cast<uint32_t*>(w + o_l[2]);
    L.flag_hv = reinterpret_cast<uint32_t*>(w + o_l[3]);
    L.pos_nh = reinterpret_cast<uint32_t*>(w + o_l[4]);
    L.pos_hv = reinterpret_cast<uint32_t*>(w + o_l[5]);
    L.sums = reinterpret_cast<uint32_t*>(w + o_l[6]);
    L.heavy = reinterpret_cast<uint64_t*>(w + o_l[7]);
    L.hid = reinterpret_cast<uint32_t*>(w + o_l[8]);
    L.large = reinterpret_cast<uint32_t*>(w + o_l[9]);
    L.cells = reinterpret_cast<uint2*>(w + o_l[10]);
    L.fval = reinterpret_cast<float*>(w + o_l[11]);
    L.counts = reinterpret_cast<uint32_t*>(w + o_l[12]);
    L.offsets = reinterpret_cast<uint32_t*>(w + o_l[13]);
    L.hcount = reinterpret_cast<uint32_t*>(w + o_l[14]);
    L.bitmap = reinterpret_cast<uint32_t*>(w + o_l[15]);
    L.counts1 = reinterpret_cast<uint32_t*>(w + o_l[23]);
    L.off1 = reinterpret_cast<uint32_t*>(w + o_l[24]);
    L.units = reinterpret_cast<uint2*>(w + o_l[25]);
    L.ids = reinterpret_cast<uint32_t*>(w + o_l[26]);
    L.fine = reinterpret_cast<uint16_t*>(w + o_l[27]);
    L.w_bf16 = w + o_l[16];
    L.master = reinterpret_cast<float*>(w + o_l[17]);
    L.m1 = reinterpret_cast<float*>(w + o_l[18]);
    L.m2 = reinterpret_cast<float*>(w + o_l[19]);
    L.grads = reinterpret_cast<float*>(w + o_l[20]);
    L.loss_log = reinterpret_cast<float*>(w + o_l[21]);
    L.st = reinterpret_cast<LearnedState*>(w + o_l[22]);
    e = cudaMallocHost(reinterpret_cast<void**>(&L.h_st), sizeof(LearnedState));
    if (e != cudaSuccess) L.h_st = nullptr;
    if (e == cudaSuccess) e = cudaMemset(L.st, 0, sizeof(LearnedState));
    if (e == cudaSuccess) e = cudaMemset(L.heavy, 0, size_t(kLearnMaxHeavy) * 8);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fsort_plan_destroy(p);
      return FSORT_ERR_OOM;
    }
  }
  // Zero what must start at zero: histogram accumulators, status, counters.
  e = cudaMemset(p->hist, 0, hist_bytes);
  if (e == cudaSuccess) e = cudaMemset(p->orand, 0, sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMemset(p->orand + 1, 0xFF, sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMemset(p->totals, 0, 2 * kRadix * 4);
  if (e == cudaSuccess) e = cudaMemset(p->status, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(p->counters, 0, kCounterBytes);
  if (e == cudaSuccess && batch) e = cudaMemset(p->d_bhist, 0, size_t(desc->max_segments) * pmax * kRadix * 8);
  if (e == cudaSuccess && batch)
    e = cudaMallocHost(reinterpret_cast<void**>(&p->h_seg_large), sizeof(SegDesc) * desc->max_segments);
  if (e == cudaSuccess && batch)
    e = cudaMallocHost(reinterpret_cast<void**>(&p->h_seg_small), sizeof(SegDesc) * desc->max_segments);
  if (e == cudaSuccess && batch)
    e = cudaMallocHost(reinterpret_cast<void**>(&p->h_chunks), sizeof(HistChunk) * p->max_hist_chunks);
  if (e == cudaSuccess && batch)
    e = cudaMallocHost(reinterpret_cast<void**>(&p->h_chunk_seg), sizeof(uint32_t) * p->max_tchunks);
  if (e == cudaSuccess && batch) e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
  if (e == cudaSuccess && batch) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess && batch) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&p->h_status), sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    fsort_plan_destroy(p);
    return FSORT_ERR_CUDA;
  }
  *p->h_status = 0;
  if (batch) {
    p->bcfg.small_capacity = 4096;
    p->bcfg.small_ctas_per_sm = small_sort_ctas_per_sm(desc->key_bits, desc->has_values != 0, 4096);
    p->bcfg.large_form = 1;
    p->bcfg.digit_bits = 8;
  }
  *out_plan = p;
  return FSORT_OK;
}

fsort_status fsort_plan_destroy(fsort_plan* plan) {
  if (!plan) return FSORT_OK;
  fsort_status st = FSORT_OK;
  if (plan->pending && cudaEventSynchronize(plan->done) != cudaSuccess) st = FSORT_ERR_CUDA;
  if (plan->side) cudaStreamSynchronize(plan->side);
  if (plan->gexec) cudaGraphExecDestroy(plan->gexec);
  if (plan->side) cudaStreamDestroy(plan->side);
  if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
  if (plan->ev_join) cudaEventDestroy(plan->ev_join);
  if (plan->h_seg_large) cudaFreeHost(plan->h_seg_large);
  if (plan->h_seg_small) cudaFreeHost(plan->h_seg_small);
  if (plan->h_chunks) cudaFreeHost(plan->h_chunks);
  if (plan->h_chunk_seg) cudaFreeHost(plan->h_chunk_seg);
  if (plan->done) cudaEventDestroy(plan->done);
  if (plan->h_status) cudaFreeHost(plan->h_status);
  fsort_plan_set_timing(plan, 0);
  if (plan->learn) {
    if (plan->learn->h_st) cudaFreeHost(plan->learn->h_st);
    delete plan->learn;
  }
  if (plan->ws && cudaFree(plan->ws) != cudaSuccess) st = FSORT_ERR_CUDA;
  delete plan;
  return st;
}

fsort_status fsort_plan_sync(fsort_plan* plan) {
  if (!plan) return FSORT_ERR_INVALID_ARG;
  return take_latched(plan, true, nullptr);
}

fsort_status fsort_plan_describe(const fsort_plan* plan, uint64_t n, int key_bits, int precision_bits,
                                 int has_values, fsort_plan_info* out) {
  if (!out) return FSORT_ERR_INVALID_ARG;
  const fsort_status st = check_call(plan, n, key_bits, precision_bits, has_values != 0);
  if (st != FSORT_OK) return st;
  std::memset(out, 0, sizeof(*out));
  const uint64_t kb = uint64_t(key_bits) / 8, vb = has_values ? 4 : 0;
  const bool table = !plan->chained && n <= (1ull << 32);  // the form enqueue_sort takes
  const int tile = table ? table_tile_keys_for(key_bits) : plan->tile;
  out->digit_bits = plan->digit_bits;
  out->tile_keys = tile;
  out->chunk_keys = plan->chunk_keys;
  out->workspace_bytes = plan->ws_bytes;
  out->scatter_form = table ? 0 : 1;
  if (use_expand(key_bits, precision_bits, has_values != 0)) {
    out->expand_path = 1;
    out->passes = 0;
    out->num_tiles = 0;
    out->algorithmic_bytes = 2 * kb * n;
  } else {
    out->passes = (precision_bits + plan->digit_bits - 1) / plan->digit_bits;
    out->num_tiles = (n + tile - 1) / tile;
    out->algorithmic_bytes = kb * n + uint64_t(out->passes) * 2 * (kb + vb) * n;
  }
  return FSORT_OK;
}

fsort_status fsort_sort_pairs(fsort_plan* plan, void* keys, uint32_t* vals, uint64_t n, int key_bits,
                              int precision_bits, void* stream) {
  fsort_status st = check_call(plan, n, key_bits, precision_bits, vals != nullptr);
  if (st != FSORT_OK) return st;
  if (n == 0) return FSORT_OK;
  if (!keys || !aligned16(keys) || (vals && !aligned16(vals))) return FSORT_ERR_INVALID_ARG;
  if (vals && overlaps(keys, n * (key_bits / 8), vals, n * 4)) return FSORT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = take_latched(plan, false, s);
  if (st != FSORT_OK) return st;
  return enqueue_any(plan, keys, vals, keys, vals, n, key_bits, precision_bits, s);
}

fsort_status fsort_sort_pairs_out(fsort_plan* plan, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                                  uint32_t* vals_out, uint64_t n, int key_bits, int precision_bits, void* stream) {
  if ((vals_in == nullptr) != (vals_out == nullptr)) return FSORT_ERR_INVALID_ARG;
  fsort_status st = check_call(plan, n, key_bits, precision_bits, vals_in != nullptr);
  if (st != FSORT_OK) return st;
  if (n == 0) return FSORT_OK;
  if (!keys_in || !keys_out || !aligned16(keys_in) || !aligned16(keys_out)) return FSORT_ERR_INVALID_ARG;
  if (vals_in && (!aligned16(vals_in) || !aligned16(vals_out))) return FSORT_ERR_INVALID_ARG;
  const size_t kbytes = size_t(n) * (key_bits / 8);
  if (overlaps(keys_in, kbytes, keys_out, kbytes)) return FSORT_ERR_INVALID_ARG;
  if (vals_in && (overlaps(vals_in, n * 4, vals_out, n * 4) || overlaps(keys_out, kbytes, vals_out, n * 4) ||
                  overlaps(keys_in, kbytes, vals_out, n * 4) || overlaps(vals_in, n * 4, keys_out, kbytes)))
    return FSORT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = take_latched(plan, false, s);
  if (st != FSORT_OK) return st;
  return enqueue_any(plan, keys_in, vals_in, keys_out, vals_out, n, key_bits, precision_bits, s);
}

fsort_status fsort_sort_pairs_host(fsort_plan* plan, void* keys_host, uint32_t* vals_host, uint64_t n, int key_bits,
                                   int precision_bits, void* stream) {
  fsort_status st = check_call(plan, n, key_bits, precision_bits, vals_host != nullptr);
  if (st != FSORT_OK) return st;
  if (!(plan->desc.flags & FSORT_FLAG_HOST_IO)) return FSORT_ERR_INVALID_ARG;
  if (n == 0) return FSORT_OK;
  if (!keys_host) return FSORT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = take_latched(plan, false, s);
  if (st != FSORT_OK) return st;
  const size_t kbytes = size_t(n) * (key_bits / 8);
  // The caller may reuse its host buffers once this returns, on an error too:
  // every copy enqueued so far is drained before any return.
  cudaError_t e = cudaMemcpyAsync(plan->io_keys, keys_host, kbytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && vals_host) e = cudaMemcpyAsync(plan->io_vals, vals_host, n * 4, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(s);
    return from_cuda(e);
  }
  st = enqueue_any(plan, plan->io_keys, vals_host ? plan->io_vals : nullptr, plan->io_keys,
                   vals_host ? plan->io_vals : nullptr, n, key_bits, precision_bits, s);
  if (st != FSORT_OK) {
    cudaStreamSynchronize(s);
    return st;
  }
  e = cudaMemcpyAsync(keys_host, plan->io_keys, kbytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && vals_host) e = cudaMemcpyAsync(vals_host, plan->io_vals, n * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  return take_latched(plan, true, s);
}

fsort_status fsort_histogram(fsort_plan* plan, const void* keys, uint64_t n, int key_bits, int precision_bits,
                             int digit_bits, uint64_t* counts_out, void* stream) {
  fsort_status st = check_call(plan, n, key_bits, precision_bits, false);
  if (st != FSORT_OK) return st;
  if (!counts_out || !aligned_to(counts_out, 8) || (n && (!keys || !aligned16(keys)))) return FSORT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = take_latched(plan, false, s);
  if (st != FSORT_OK) return st;
  cudaError_t e;
  if (digit_bits == 16) {
    if (key_bits != 16 || precision_bits != 16) return FSORT_ERR_INVALID_ARG;
    e = launch_leaf_histogram(static_cast<const uint16_t*>(keys), n, plan->leaf_part, plan->leaf_spill, plan->sms, s);
    if (e == cudaSuccess)
      e = launch_leaf_reduce(plan->leaf_part, plan->leaf_spill, leaf_hist_grid(plan->sms), counts_out, s);
  } else {
    if (digit_bits != plan->digit_bits) return FSORT_ERR_INVALID_ARG;
    const DigitPlan dp = make_plan(key_bits, precision_bits, digit_bits);
    e = cudaMemsetAsync(counts_out, 0, sizeof(uint64_t) * dp.passes * (1u << digit_bits), s);
    if (e == cudaSuccess && n)
      e = launch_histogram(keys, key_bits, n, dp, counts_out, uint64_t(1) << digit_bits, nullptr, 0, plan->sms, s);
  }
  if (e != cudaSuccess) return from_cuda(e);
  return finish_call(plan, s);
}

fsort_status fsort_exclusive_scan(fsort_plan* plan, const uint64_t* counts, uint64_t rows, uint64_t bins,
                                  uint64_t* offsets_out, void* stream) {
  if (!plan || !counts || !offsets_out || !aligned_to(counts, 8) || !aligned_to(offsets_out, 8))
    return FSORT_ERR_INVALID_ARG;
  if (bins != (1ull << plan->digit_bits) && bins != 65536) return FSORT_ERR_INVALID_ARG;
  if (rows < 1 || rows > 65535) return FSORT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  fsort_status st = take_latched(plan, false, s);
  if (st != FSORT_OK) return st;
  const cudaError_t e = launch_scan_rows(counts, offsets_out, rows, bins, s);
  if (e != cudaSuccess) return from_cuda(e);
  return finish_call(plan, s);
}

fsort_status fsort_scatter_pass(fsort_plan* plan, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                                uint32_t* vals_out, uint64_t n, int key_bits, int shift, int width, void* stream) {
  if ((vals_in == nullptr) != (vals_out == nullptr)) return FSORT_ERR_INVALID_ARG;
  fsort_status st = check_call(plan, n, key_bits, key_bits, vals_in != nullptr);
  if (st != FSORT_OK) return st;
  if (width < 1 || width > plan->digit_bits || shift < 0 || shift + width > key_bits) return FSORT_ERR_INVALID_ARG;
  if (n == 0) return FSORT_OK;
  if (!keys_in || !keys_out || !aligned16(keys_in) || !aligned16(keys_out)) return FSORT_ERR_INVALID_ARG;
  if (vals_in && (!aligned16(vals_in) || !aligned16(vals_out))) return FSORT_ERR_INVALID_ARG;
  const size_t kbytes = size_t(n) * (key_bits / 8);
  if (overlaps(keys_in, kbytes, keys_out, kbytes)) return FSORT_ERR_INVALID_ARG;
  if (vals_in && overlaps(vals_in, n * 4, vals_out, n * 4)) return FSORT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = take_latched(plan, false, s);
  if (st != FSORT_OK) return st;
  DigitPlan dp{};
  dp.passes = 1;
  dp.shift[0] = uint32_t(shift);
  dp.mask[0] = (1u << width) - 1u;
  const uint64_t tiles = (n + plan->tile - 1) / plan->tile;
  const uint64_t chunks = (n + plan->chunk_keys - 1) / plan->chunk_keys;
  cudaError_t e = launch_histogram(keys_in, key_bits, n, dp, plan->hist, kRadix, plan->counters,
                                   kCounterBytes / 4 + tiles * kRadix, plan->sms, s);
  if (e == cudaSuccess)
    e = launch_scan_schedule(plan->hist, plan->chunk_base, plan->chunk_flag, 1, uint32_t(chunks), 0, nullptr, s);
  if (e == cudaSuccess) {
    OnesweepArgs a{};
    a.keys[0] = keys_in;
    a.keys[1] = nullptr;
    a.keys[2] = keys_out;
    a.vals[0] = vals_in;
    a.vals[1] = nullptr;
    a.vals[2] = vals_out;
    a.n = n;
    a.shift = dp.shift[0];
    a.mask = dp.mask[0];
    a.lookback = plan->lookback[0];
    a.tile_counter = plan->counters;
    a.next_lookback = nullptr;
    a.next_counter = nullptr;
    a.chunk_base = plan->chunk_base;
    a.chunk_flag = plan->chunk_flag;
    a.sched = nullptr;
    a.pass = 0;
    a.tiles_per_chunk = uint32_t(plan->chunk_keys / plan->tile);
    a.status = plan->status;
    a.withhold_tile = plan->withhold_tile;
    a.wait_limit_ns = plan->wait_limit_ns;
    e = launch_onesweep(a, key_bits, vals_in != nullptr, s);
  }
  if (e != cudaSuccess) return from_cuda(e);
  return finish_call(plan, s);
}

fsort_status fsort_expand(fsort_plan* plan, const uint64_t* counts, void* keys_out, uint64_t n, int key_bits,
                          void* stream) {
  fsort_status st = check_call(plan, n, key_bits, key_bits, false);
  if (st != FSORT_OK) return st;
  if (key_bits != 16 || !counts || !aligned_to(counts, 8)) return FSORT_ERR_INVALID_ARG;
  if (n == 0) return FSORT_OK;
  if (!keys_out || !aligned16(keys_out)) return FSORT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = take_latched(plan, false, s);
  if (st != FSORT_OK) return st;
  cudaError_t e = launch_scan_rows(counts, plan->leaf_off, 1, 65536, s);
  if (e == cudaSuccess) e = launch_expand(plan->leaf_off, static_cast<uint16_t*>(keys_out), n, s);
  if (e != cudaSuccess) return from_cuda(e);
  return finish_call(plan, s);
}

namespace {
// The learned fit (ecdf false) or its model-free counterpart (ecdf true: the
// map tabulates the sorted sample's empirical CDF; no training).
fsort_status learned_fit_impl(fsort_plan* plan, const void* keys, uint64_t n, const fsort_learned_opts* opts,
                              void* stream, bool ecdf);
}  // namespace

fsort_status fsort_learned_fit(fsort_plan* plan, const void* keys, uint64_t n, const fsort_learned_opts* opts,
                               void* stream) {
  return learned_fit_impl(plan, keys, n, opts, stream, false);
}

fsort_status fsort_learned_fit_ecdf(fsort_plan* plan, const void* keys, uint64_t n, const fsort_learned_opts* opts,
                                    void* stream) {
  return learned_fit_impl(plan, keys, n, opts, stream, true);
}

namespace {
fsort_status learned_fit_impl(fsort_plan* plan, const void* keys, uint64_t n, const fsort_learned_opts* opts,
                              void* stream, bool ecdf) {
  if (!plan || !plan->learn) return FSORT_ERR_INVALID_ARG;
  if (!keys || !aligned16(keys) || n < 1 || n > plan->desc.max_n) return FSORT_ERR_INVALID_ARG;
  fsort_learned_opts o{};
  if (opts) o = *opts;
  LearnedWs& L = *plan->learn;
  uint32_t S = o.sample_keys ? o.sample_keys : LearnedWs::kMaxSample;
  if (S > L.sample_max) S = L.sample_max;
  if (uint64_t(S) > n) S = uint32_t(n);
  const uint32_t steps = o.steps ? o.steps : 4000u;
  const uint32_t batch = o.batch ? o.batch : 65536u;
  const float lr = o.lr > 0.f ? o.lr : 0.01f;
  if (steps > LearnedWs::kMaxSteps || batch > (1u << 20) || !(lr < 1.f)) return FSORT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  fsort_status st = take_latched(plan, false, s);
  if (st != FSORT_OK) return st;
  L.fitted = false;
  std::vector<float> init;
  learned_init_params(init, o.seed);
  cudaError_t e = cudaMemcpyAsync(L.master, init.data(), size_t(kMlpParams) * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // `init` is pageable and about to go away
  if (e == cudaSuccess) e = cudaMemsetAsync(L.m1, 0, size_t(kMlpParams) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.m2, 0, size_t(kMlpParams) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.grads, 0, size_t(kMlpParams) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.loss_log, 0, size_t(LearnedWs::kMaxSteps) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.st, 0, sizeof(LearnedState), s);
  if (e == cudaSuccess) e = launch_to_bf16(L.master, L.w_bf16, kMlpParams, s);
  // the sample, sorted by the plain path
  if (e == cudaSuccess) e = launch_learn_sample(static_cast<const uint64_t*>(keys), n, S, o.seed, L.sample, s);
  if (e != cudaSuccess) return from_cuda(e);
  st = enqueue_sort(plan, L.sample, nullptr, L.sample, nullptr, S, 64, 64, s);
  if (st != FSORT_OK) return st;
  // frequent keys: at least 1024 copies expected among the n keys
  uint64_t hmin = (uint64_t(S) * 1024 + n - 1) / n;
  if (hmin < 2) hmin = 2;
  e = launch_learn_split(L.sample, S, uint32_t(hmin), L.flag_nh, L.flag_hv, s);
  if (e == cudaSuccess) e = launch_scan_u32(L.flag_nh, S, L.pos_nh, nullptr, L.sums, s);
  if (e == cudaSuccess) e = launch_scan_u32(L.flag_hv, S, L.pos_hv, nullptr, L.sums, s);
  if (e == cudaSuccess)
    e = launch_learn_compact(L.sample, S, L.flag_nh, L.pos_nh, L.flag_hv, L.pos_hv, L.train, L.heavy, L.st, s);
  if (ecdf) {
    if (e == cudaSuccess) e = launch_learn_cells_ecdf(L.train, L.st, L.heavy, L.fval, L.cells, s);
    if (e != cudaSuccess) return from_cuda(e);
    L.fitted = true;
    L.steps = 0;
    L.used = -1;
    L.heavy_count = kLearnMaxHeavy;
    return finish_call(plan, s);
  }
  if (e == cudaSuccess) e = launch_learn_init_kinks(L.train, L.st, L.master, s);
  if (e == cudaSuccess) e = launch_to_bf16(L.master, L.w_bf16, kMlpParams, s);
  // training: Adam on stratified minibatches, cosine decay to lr / 10
  for (uint32_t t = 1; t <= steps && e == cudaSuccess; ++t) {
    const double c = 0.5 * (1.0 + std::cos(3.141592653589793 * double(t - 1) / double(steps)));
    const float lr_t = float(lr * (0.1 + 0.9 * c));
    e = launch_mlp_grad_sample(L.w_bf16, L.train, L.st, batch, t, o.seed, L.grads, s);
    if (e == cudaSuccess)
      e = launch_mlp_adam(L.master, L.grads, L.m1, L.m2, L.w_bf16, lr_t, int(t), L.st, L.loss_log + (t - 1), s);
  }
  if (e == cudaSuccess) e = launch_learn_cells(L.w_bf16, L.st, L.heavy, L.fval, L.cells, s);
  if (e != cudaSuccess) return from_cuda(e);
  L.fitted = true;
  L.steps = steps;
  L.used = -1;
  L.heavy_count = kLearnMaxHeavy;
  return finish_call(plan, s);
}
}  // namespace

fsort_status fsort_learned_get_stats(fsort_plan* plan, fsort_learned_stats* out) {
  if (!plan || !plan->learn || !out) return FSORT_ERR_INVALID_ARG;
  LearnedWs& L = *plan->learn;
  std::memset(out, 0, sizeof(*out));
  if (cudaDeviceSynchronize() != cudaSuccess) return FSORT_ERR_CUDA;
  out->fitted = L.fitted ? 1 : 0;
  out->used = L.used;
  out->buckets = L.last_b;
  out->max_bucket = L.last_max;
  out->limit = L.last_limit;
  out->imbalance = L.last_imbalance;
  out->tau = double(kLearnTau);
  out->steps = L.steps;
  if (L.fitted) {
    LearnedState h{};
    if (cudaMemcpy(&h, L.st, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return FSORT_ERR_CUDA;
    out->heavy_keys = h.heavy_count;
    out->sample_keys = h.sample_count;
    out->train_keys = h.train_count;
    if (L.steps) {
      if (cudaMemcpy(&out->loss_first, L.loss_log, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(&out->loss_last, L.loss_log + (L.steps - 1), 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return FSORT_ERR_CUDA;
    }
  }
  return FSORT_OK;
}

fsort_status fsort_learned_get_model(fsort_plan* plan, float* params_host, uint32_t* cells_host, uint64_t* heavy_host,
                                     uint32_t* heavy_count, float* norm) {
  if (!plan || !plan->learn) return FSORT_ERR_INVALID_ARG;
  LearnedWs& L = *plan->learn;
  if (cudaDeviceSynchronize() != cudaSuccess) return FSORT_ERR_CUDA;
  LearnedState h{};
  cudaError_t e = cudaMemcpy(&h, L.st, sizeof(h), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && params_host)
    e = cudaMemcpy(params_host, L.master, size_t(kMlpParams) * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && cells_host)
    e = cudaMemcpy(cells_host, L.cells, size_t(kLearnCells + 1) * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && heavy_host)
    e = cudaMemcpy(heavy_host, L.heavy, size_t(kLearnMaxHeavy) * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return FSORT_ERR_CUDA;
  if (heavy_count) *heavy_count = h.heavy_count;
  if (norm) {
    norm[0] = h.center;
    norm[1] = h.half;
  }
  return FSORT_OK;
}

fsort_status fsort_learned_set_model(fsort_plan* plan, const float* params_host, const uint32_t* cells_host,
                                     const uint64_t* heavy_host, uint32_t heavy_count, const float* norm,
                                     void* stream) {
  if (!plan || !plan->learn || !norm || !(norm[1] > 0.f)) return FSORT_ERR_INVALID_ARG;
  if (heavy_count > uint32_t(kLearnMaxHeavy) || (heavy_count && !heavy_host)) return FSORT_ERR_INVALID_ARG;
  if (!cells_host && !params_host) return FSORT_ERR_INVALID_ARG;
  for (uint32_t t = 1; t < heavy_count; ++t)
    if (heavy_host[t - 1] >= heavy_host[t]) return FSORT_ERR_INVALID_ARG;
  if (cells_host) {  // G non-decreasing, last = all ones, H = frequent keys below each cell start
    if (cells_host[2 * kLearnCells] != 0xFFFFFFFFu || cells_host[2 * kLearnCells + 1] != heavy_count)
      return FSORT_ERR_INVALID_ARG;
    uint32_t below = 0;
    for (int i = 0; i < kLearnCells; ++i) {
      if (cells_host[2 * i] > cells_host[2 * i + 2]) return FSORT_ERR_INVALID_ARG;
      const uint64_t c = i < 2048 ? uint64_t(i) : uint64_t(1024 + (i & 1023)) << ((i >> 10) - 1);
      while (below < heavy_count && heavy_host[below] < c) ++below;
      if (cells_host[2 * i + 1] != below) return FSORT_ERR_INVALID_ARG;
    }
  }
  LearnedWs& L = *plan->learn;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  fsort_status st = take_latched(plan, true, s);
  if (st != FSORT_OK) return st;
  LearnedState h{};
  h.center = norm[0];
  h.half = norm[1];
  h.heavy_count = heavy_count;
  L.fitted = false;
  cudaError_t e = cudaMemcpyAsync(L.st, &h, sizeof(h), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.heavy, 0, size_t(kLearnMaxHeavy) * 8, s);
  if (e == cudaSuccess && heavy_count)
    e = cudaMemcpyAsync(L.heavy, heavy_host, size_t(heavy_count) * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && params_host) {
    e = cudaMemcpyAsync(L.master, params_host, size_t(kMlpParams) * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_to_bf16(L.master, L.w_bf16, kMlpParams, s);
  }
  if (e == cudaSuccess) {
    if (cells_host)
      e = cudaMemcpyAsync(L.cells, cells_host, size_t(kLearnCells + 1) * 8, cudaMemcpyHostToDevice, s);
    else
      e = launch_learn_cells(L.w_bf16, L.st, L.heavy, L.fval, L.cells, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  L.fitted = true;
  L.steps = 0;
  L.used = -1;
  L.heavy_count = heavy_count;
  return FSORT_OK;
}

fsort_status fsort_learned_bucket_ids(fsort_plan* plan, const void* keys, uint64_t n, uint32_t* ids, void* stream) {
  if (!plan || !plan->learn || !plan->learn->fitted) return FSORT_ERR_INVALID_ARG;
  if (n == 0) return FSORT_OK;
  if (!keys || !ids || !aligned_to(keys, 8) || !aligned_to(ids, 4) || n >= (1ull << 32)) return FSORT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e = launch_learn_bucket_ids(static_cast<const uint64_t*>(keys), n,
                                                learned_map(*plan->learn, n), ids, s);
  return from_cuda(e);
}

fsort_status fsort_mlp_forward(const void* w_bf16, const float* x, uint32_t m, float* out, void* stream) {
  if (!w_bf16 || !x || !out || m < 1) return FSORT_ERR_INVALID_ARG;
  if (!aligned_to(w_bf16, 2) || !aligned_to(x, 4) || !aligned_to(out, 4)) return FSORT_ERR_INVALID_ARG;
  return from_cuda(launch_mlp_eval(w_bf16, x, m, out, static_cast<cudaStream_t>(stream)));
}

fsort_status fsort_mlp_grad(const void* w_bf16, const float* x, const float* y, uint32_t m, float* grads, float* loss,
                            void* stream) {
  if (!w_bf16 || !x || !y || !grads || m < 1) return FSORT_ERR_INVALID_ARG;
  if (!aligned_to(w_bf16, 2) || !aligned_to(x, 4) || !aligned_to(y, 4) || !aligned_to(grads, 4) ||
      (loss && !aligned_to(loss, 4)))
    return FSORT_ERR_INVALID_ARG;
  return from_cuda(launch_mlp_grad(w_bf16, x, y, m, grads, loss, static_cast<cudaStream_t>(stream)));
}

fsort_status fsort_plan_set_fault_hook(fsort_plan* plan, uint32_t withhold_tile, uint64_t wait_limit_ns) {
  if (!plan) return FSORT_ERR_INVALID_ARG;
  plan->withhold_tile = withhold_tile;
  plan->wait_limit_ns = wait_limit_ns;
  return FSORT_OK;
}

fsort_status fsort_plan_set_timing(fsort_plan* plan, int enable) {
  if (!plan) return FSORT_ERR_INVALID_ARG;
  Timing& t = plan->timing;
  if (enable && !t.on) {
    t.ev.assign(Timing::kEvents, nullptr);
    for (auto& e : t.ev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        fsort_plan_set_timing(plan, 0);
        return FSORT_ERR_CUDA;
      }
    if (cudaMallocHost(reinterpret_cast<void**>(&t.h_sched), sizeof(Schedule) * Timing::kSlots) != cudaSuccess) {
      t.h_sched = nullptr;
      fsort_plan_set_timing(plan, 0);
      return FSORT_ERR_OOM;
    }
    t.on = true;
    t.next_ev = t.next_slot = t.calls = 0;
    t.recs.clear();
  } else if (!enable) {
    if (!t.ev.empty()) cudaDeviceSynchronize();
    for (auto& e : t.ev)
      if (e) cudaEventDestroy(e);
    t.ev.clear();
    if (t.h_sched) cudaFreeHost(t.h_sched);
    t.h_sched = nullptr;
    t.on = false;
    t.recs.clear();
  }
  return FSORT_OK;
}

fsort_status fsort_plan_timing_report(fsort_plan* plan, fsort_kernel_time* out, uint32_t capacity,
                                      uint32_t* count) {
  if (!plan || !count || (capacity && !out)) return FSORT_ERR_INVALID_ARG;
  Timing& t = plan->timing;
  *count = 0;
  if (!t.on) return FSORT_ERR_INVALID_ARG;
  if (!t.recs.empty() && cudaEventSynchronize(t.ev[t.recs.back().ev1]) != cudaSuccess) return FSORT_ERR_CUDA;
  if (plan->pending && cudaEventSynchronize(plan->done) != cudaSuccess) return FSORT_ERR_CUDA;
  uint32_t k = 0;
  for (const TimingRec& r : t.recs) {
    if (k >= capacity) break;
    fsort_kernel_time& o = out[k++];
    o.kind = r.kind;
    o.pass = r.pass;
    o.call = r.call;
    o.n = r.n;
    o.reserved = 0.f;
    o.active = 1;
    if (r.slot >= 0 && r.pass >= 0 &&
        (r.kind == FSORT_KERNEL_SCATTER || r.kind == FSORT_KERNEL_TILE_COUNT || r.kind == FSORT_KERNEL_TILE_SCAN))
      o.active = t.h_sched[r.slot].pass[r.pass].active;
    if (r.slot >= 0 && r.kind == FSORT_KERNEL_COPY) o.active = t.h_sched[r.slot].copy.active;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.ev[r.ev0], t.ev[r.ev1]) != cudaSuccess) return FSORT_ERR_CUDA;
    o.ms = ms;
  }
  *count = k;
  t.recs.clear();
  t.next_ev = t.next_slot = t.calls = 0;
  return FSORT_OK;
}

const char* fsort_status_string(fsort_status status) {
  switch (status) {
    case FSORT_OK: return "FSORT_OK";
    case FSORT_ERR_INVALID_ARG: return "FSORT_ERR_INVALID_ARG";
    case FSORT_ERR_OOM: return "FSORT_ERR_OOM";
    case FSORT_ERR_CUDA: return "FSORT_ERR_CUDA";
    case FSORT_ERR_TIMEOUT: return "FSORT_ERR_TIMEOUT";
    case FSORT_ERR_BUSY: return "FSORT_ERR_BUSY";
    case FSORT_NOT_READY: return "FSORT_NOT_READY";
    case FSORT_ERR_INTERNAL: return "FSORT_ERR_INTERNAL";
    case FSORT_ERR_UNSUPPORTED: return "FSORT_ERR_UNSUPPORTED";
    default: return "FSORT_UNKNOWN_STATUS";
  }
}

uint32_t fsort_plan_device_flags(const fsort_plan* plan) { return plan ? plan->last_device_flags : 0u; }

int fsort_version(void) { return 200; }  // 2.0: fsort_plan_info gained scatter_form; table-form scatter passes

}  // extern "C"
