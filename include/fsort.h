/*
 * fsort.h -- C ABI of libfsort, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of the compressed radix sort of "FractalSortCPU:
 * Bandwidth-Efficient Compressed Radix Sort on CPU" (arXiv 2605.10390).
 *
 * Problem (paper Sec. I and II): sort n keys of key_bits bits, optionally
 * carrying one 32-bit value each, in ascending order of their top
 * precision_bits bits ("arbitrary-precision keys"; a reduced precision gives
 * the approximate sort of Sec. I).  The sort is stable: keys whose top bits are
 * equal keep their input order, which makes the result unique.  Full keys and
 * values are moved.
 *
 * The hot path (every step a CUDA kernel of this library):
 *   1. digit plan: least-significant-digit-first passes of d-bit digits over
 *      bits [key_bits - precision_bits, key_bits) (Sec. II);
 *   2. digit histograms (the leaf level of the histogram tree of Sec.
 *      III-A/B, with counters whose width tapers with the size of what they
 *      count, Sec. III-D-1).  Sorts of up to 2^32 keys count each pass's
 *      digits per tile, in one read of that pass's input just before it (the
 *      first read also marks the passes whose digit is the same for every key);
 *      larger sorts, and plans with FSORT_FLAG_CHAINED_SCATTER, count every
 *      pass's digits in one upfront read of the keys;
 *   3. exclusive scan of each histogram (the rank of Alg. 3 for every leaf):
 *      per tile from the table of tile counts, or chained between tiles by
 *      decoupled look-back;
 *   4. one stable scatter per pass (Sec. II), skipped on the device when a
 *      pass's digit is the same for every key;
 *   5. keys-only 16-bit sorts at full precision instead rebuild the output from
 *      the 65,536-bin histogram (Alg. 5 with no trailing bits).
 *
 * Conventions for every entry point:
 *   - Pointers named keys/vals/counts/... are DEVICE pointers (e.g. a torch
 *     tensor's data_ptr()) unless the name ends in _host.  Key arrays hold
 *     uint16_t, uint32_t or uint64_t elements for key_bits 16, 32, 64; values
 *     are uint32_t.  Key and value arrays given to the sorts and the scatter
 *     pass must be 16-byte aligned; every other device array (histogram
 *     counts and offsets, ranks, bucket ids, the streaming histogram's keys,
 *     the model's inputs) must be aligned to its element size.  A pointer
 *     that breaks either rule is FSORT_ERR_INVALID_ARG.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered: they enqueue work and return; the
 *     caller owns and keeps alive every buffer until the stream reaches it.
 *   - The plan owns all scratch memory (allocated by fsort_plan_create, freed
 *     by fsort_plan_destroy); no call allocates device memory afterwards, and
 *     the caller owns every buffer it passes.  One plan serves one stream at a
 *     time: concurrent calls on one plan race on its scratch.
 *   - Argument errors are returned synchronously and nothing is enqueued.
 *     Errors found on the device (a bounded wait that timed out) are latched
 *     in a plan-owned status word and returned by fsort_plan_sync or by the
 *     first call that finds the previous call's work finished.
 *   - No C++ exception crosses this interface.
 */
#ifndef FSORT_H
#define FSORT_H

#include <stdint.h>

#if defined(__GNUC__)
#define FSORT_API __attribute__((visibility("default")))
#else
#define FSORT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fsort_status {
  FSORT_OK = 0,
  FSORT_ERR_INVALID_ARG = 1, /* bad size, width, pointer, alignment or plan */
  FSORT_ERR_OOM = 2,         /* device or pinned host memory could not be allocated */
  FSORT_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  FSORT_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up; output is invalid */
  FSORT_ERR_BUSY = 5,        /* no free slot / memory to admit the request now */
  FSORT_NOT_READY = 6,       /* the queried work has not finished */
  FSORT_ERR_INTERNAL = 7,    /* an invariant of the library was violated */
  FSORT_ERR_UNSUPPORTED = 8  /* valid request this build does not support */
} fsort_status;

/* fsort_plan_desc.flags */
#define FSORT_FLAG_HOST_IO 0x4u /* also allocate device buffers of max_n keys (+values) for fsort_sort_pairs_host */
#define FSORT_FLAG_GRAPH 0x2u   /* batched sorts replay a captured CUDA graph when the batch shape repeats */
#define FSORT_FLAG_LEARNED 0x8u /* allocate the learned bucket mapping (64-bit keys only); see fsort_learned_fit */
#define FSORT_FLAG_CHAINED_SCATTER 0x10u /* every scatter pass in the chained (decoupled look-back) form; by
                                            default sorts of n <= 2^32 keys read their tiles' digit offsets from
                                            a table of per-tile counts made before each pass */

typedef struct fsort_plan fsort_plan;

typedef struct fsort_plan_desc {
  uint64_t max_n;     /* largest n any call on this plan will pass (>= 1) */
  int32_t key_bits;   /* 16, 32 or 64 */
  int32_t has_values; /* 1 if calls may carry uint32_t values, else 0 */
  int32_t digit_bits; /* radix digit width of the scatter passes: 0 = library default (8), or 8 */
  uint32_t flags;     /* FSORT_FLAG_* */
  uint32_t max_segments; /* largest segment count of fsort_sort_batch (0: no batched sorts), <= 65535 */
} fsort_plan_desc;

/* What a call with these arguments will do (filled by fsort_plan_describe). */
typedef struct fsort_plan_info {
  int32_t passes;          /* scatter passes of the digit plan (before device-side skipping) */
  int32_t digit_bits;      /* d */
  int32_t expand_path;     /* 1: keys-only full-precision 16-bit sort rebuilt from the histogram */
  int32_t tile_keys;       /* keys per scatter tile */
  uint64_t num_tiles;      /* tiles per scatter pass */
  uint64_t chunk_keys;     /* keys per look-back chunk (counts inside a chunk fit 30 bits) */
  uint64_t workspace_bytes;/* device scratch owned by the plan */
  uint64_t algorithmic_bytes; /* bytes the hot path must move: key read for the histogram plus
                                 read+write of keys(+values) per pass (expand: read + write of keys) */
  int32_t scatter_form;    /* 0: per-tile offsets from a table of tile counts (n <= 2^32), 1: chained by
                              decoupled look-back (tile_keys and num_tiles describe this form) */
  int32_t reserved;
} fsort_plan_info;

/* Create a plan: validates desc, allocates all device scratch for sorts of up
 * to max_n keys of key_bits bits on the current device.  Returns
 * FSORT_ERR_INVALID_ARG for a bad desc, FSORT_ERR_OOM if scratch cannot be
 * allocated; *out_plan is set only on FSORT_OK. */
FSORT_API fsort_status fsort_plan_create(const fsort_plan_desc* desc, fsort_plan** out_plan);

/* Synchronise with the plan's last stream and free everything it owns.
 * NULL is accepted (no-op). */
FSORT_API fsort_status fsort_plan_destroy(fsort_plan* plan);

/* Wait for all work enqueued by this plan, then return and clear the latched
 * device status: FSORT_OK, FSORT_ERR_TIMEOUT (a bounded wait gave up),
 * FSORT_ERR_INTERNAL (another device check failed; fsort_plan_device_flags
 * gives the bits) or FSORT_ERR_CUDA. */
FSORT_API fsort_status fsort_plan_sync(fsort_plan* plan);

/* Describe the schedule of a sort of n keys (no work is enqueued). */
FSORT_API fsort_status fsort_plan_describe(const fsort_plan* plan, uint64_t n, int key_bits, int precision_bits,
                                 int has_values, fsort_plan_info* out_info);

/* Stable in-place sort of keys[0..n) (and vals, if not NULL) by the top
 * precision_bits bits of each key (paper Sec. I-II).  1 <= precision_bits <=
 * key_bits; key_bits must equal the plan's; n <= max_n; vals requires a plan
 * with has_values.  n == 0 returns FSORT_OK without enqueuing work. */
FSORT_API fsort_status fsort_sort_pairs(fsort_plan* plan, void* keys, uint32_t* vals, uint64_t n, int key_bits,
                              int precision_bits, void* stream);

/* Out-of-place form: keys_in/vals_in are read only; the result lands in
 * keys_out/vals_out.  Input and output ranges must not overlap.  vals_in and
 * vals_out are both NULL (keys only) or both set. */
FSORT_API fsort_status fsort_sort_pairs_out(fsort_plan* plan, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                                  uint32_t* vals_out, uint64_t n, int key_bits, int precision_bits, void* stream);

/* Host-buffer form (plan created with FSORT_FLAG_HOST_IO): copies keys_host
 * (and vals_host) to the plan's device buffers, sorts them and copies the
 * result back in place, all on `stream`, and returns after the stream has
 * finished (the call is synchronous).  Pinned host memory makes the copies
 * asynchronous DMA; pageable memory works but is slower. */
FSORT_API fsort_status fsort_sort_pairs_host(fsort_plan* plan, void* keys_host, uint32_t* vals_host, uint64_t n,
                                   int key_bits, int precision_bits, void* stream);

/* ---- batched sorts ---------------------------------------------------------
 * Many independent stable sorts in one call (the paper's batch stream
 * sorting: batches processed without pre-processing, batch size tuned to the
 * device, Sec. III-C and IV-D).  Each segment is sorted in place, exactly as
 * fsort_sort_pairs would sort it alone.  Segments of at most
 * small_capacity keys are sorted whole in shared memory by one persistent
 * kernel; larger segments share one histogram launch, one scan launch and one
 * scatter launch per pass.  The two groups run concurrently on the device.
 * Requirements: a plan created with max_segments >= count; the sum of the
 * large segments' lengths (each rounded up to a multiple of 8) <= max_n;
 * each segment shorter than 2^31 keys; large segments' key/value pointers
 * 16-byte aligned; either every segment has values or none. */
typedef struct fsort_segment {
  void* keys;     /* device pointer, key_bits-wide keys */
  uint32_t* vals; /* device pointer or NULL */
  uint64_t n;
} fsort_segment;

typedef struct fsort_batch_config {
  int32_t small_capacity;    /* 0 (no on-chip path), 1024, 2048 or 4096 keys */
  int32_t small_ctas_per_sm; /* CTAs per SM of the persistent small-segment kernel (1..8) */
  int32_t large_form;        /* scatter passes of the larger segments: 1 = from a table of per-tile offsets
                                (one count read per pass), 0 = chained (decoupled look-back) */
  int32_t digit_bits;        /* digit width of every pass of the batch (both groups): 0 or 8 (the default;
                                ceil(p / 8) passes), 7 or 6 (ceil(p / 7), ceil(p / 6) passes with fewer
                                distinct digits each; 16- and 32-bit keys only).  The output is the same. */
} fsort_batch_config;

/* Sort count segments (host array of descriptors; the keys and values are on
 * the device).  A segment of n == 0 is skipped.  A broken requirement returns
 * FSORT_ERR_INVALID_ARG and enqueues nothing.  With FSORT_FLAG_GRAPH and a
 * non-default stream, the first batch of a shape is captured as a CUDA graph
 * and later batches of that shape replay it. */
FSORT_API fsort_status fsort_sort_batch(fsort_plan* plan, const fsort_segment* segments, uint32_t count, int key_bits,
                                        int precision_bits, void* stream);

/* Set / read the batched path's configuration (defaults: 4096 keys, the most
 * CTAs per SM that shared memory allows, the table form, 8-bit digits). */
FSORT_API fsort_status fsort_batch_set_config(fsort_plan* plan, const fsort_batch_config* config);
FSORT_API fsort_status fsort_batch_get_config(const fsort_plan* plan, fsort_batch_config* config);

/* Autotuner: time fsort_sort_batch on these segments under candidate
 * configurations -- the larger segments' form (table or chained) under the
 * current small-segment configuration, then every small-segment capacity (the
 * on-chip tile) x CTAs per SM under the faster form, then the digit widths 8,
 * 7 and 6 (16- and 32-bit keys) under the best of those -- keep the fastest in
 * the plan and return it (and its time in ms, if best_ms is not NULL).  The
 * segments are sorted in place several times; the result is the sorted batch.
 * Synchronous. */
FSORT_API fsort_status fsort_batch_autotune(fsort_plan* plan, const fsort_segment* segments, uint32_t count,
                                            int key_bits, int precision_bits, void* stream,
                                            fsort_batch_config* best, float* best_ms);

/* ---- learned bucket mapping -----------------------------------------------
 * The paper has no learned component; this extends it where it leaves skewed
 * inputs open (Sec. IV-A).  A small CDF model (a 1-64-64-1 ReLU perceptron with
 * a sigmoid output, BF16 weights, FP32 sums) is trained on the GPU by this
 * library's own forward and backward kernels on a stratified sample that the
 * plain sort has sorted.  Its CDF is tabulated into a monotone bucket map;
 * keys frequent in the sample get buckets of their own.  A keys-only sort of
 * 64-bit keys at precision 64 on a plan with a fitted model then:
 *   1. counts every bucket exactly (the plain path's histogram, Sec. III, used
 *      as the judge of the model's error),
 *   2. accepts the map iff the largest bucket of non-frequent keys holds at
 *      most tau * n / B keys (tau = 8, B = the power of two >= n / 1024; one
 *      CTA sorts up to 8,192 keys on chip), else runs the plain path (the
 *      fallback),
 *   3. partitions the keys into their buckets, fills the frequent-key buckets
 *      and sorts every other bucket on chip.
 * The result is the sorted multiset, identical to the plain path's.  The
 * judge's decision is read back by the host: such a call synchronises with
 * `stream` once, midway, and cannot be captured into a CUDA graph.  Calls
 * with values, precision < 64 or n >= 2^32 always take the plain path. */
typedef struct fsort_learned_opts {
  uint32_t sample_keys; /* keys sampled from the input: 0 = min(n, 4,194,304); at most that */
  uint32_t steps;       /* Adam steps: 0 = 4000; at most 16384 */
  uint32_t batch;       /* minibatch (stratified over the sorted sample): 0 = 65536; at most 1,048,576 */
  float lr;             /* peak learning rate (cosine decay to a tenth): 0 = 0.01 */
  uint64_t seed;        /* sample, initial weights and minibatches */
} fsort_learned_opts;

typedef struct fsort_learned_stats {
  int32_t fitted;        /* a model has been fitted on this plan */
  int32_t used;          /* last eligible sort: 1 learned path, 0 fallback, -1 none yet */
  uint32_t buckets;      /* B of the last judged sort (frequent keys add 2 ids each) */
  uint32_t heavy_keys;   /* keys with buckets of their own */
  uint32_t max_bucket;   /* largest bucket of non-frequent keys in the last judged sort */
  uint32_t limit;        /* floor(tau * n / B) of that sort */
  double imbalance;      /* max_bucket / (n / B) */
  double tau;            /* threshold on imbalance (8) */
  uint32_t sample_keys;  /* keys sampled by the last fit */
  uint32_t train_keys;   /* non-frequent sample keys the model was trained on */
  uint32_t steps;        /* Adam steps of the last fit */
  uint32_t reserved;
  float loss_first;      /* training loss (mean of 0.5 (F(x) - rank/count)^2) of the first step */
  float loss_last;       /* and of the last step */
} fsort_learned_stats;

/* Number of MLP parameters and their order in a flat array: W1[64], b1[64],
 * W2[64][64] (row j feeds hidden unit j of layer 2), b2[64], W3[64], b3. */
#define FSORT_MLP_PARAMS 4353
#define FSORT_LEARN_CELLS 56320    /* cells of the map table (which has one more, closing entry) */
#define FSORT_LEARN_MAX_HEAVY 8192 /* most frequent keys a model keeps buckets of their own for */

/* Fit the plan's model to keys[0..n) (64-bit keys, device, 16-byte aligned,
 * 1 <= n <= max_n): sample, sort the sample with the plain path, find the
 * frequent keys, train, tabulate the map.  opts may be NULL (all defaults).
 * Stream-ordered (no host synchronisation).  FSORT_ERR_INVALID_ARG: a plan
 * without FSORT_FLAG_LEARNED, bad keys or n, or options beyond their limits. */
FSORT_API fsort_status fsort_learned_fit(fsort_plan* plan, const void* keys, uint64_t n,
                                         const fsort_learned_opts* opts, void* stream);

/* The model-free counterpart of fsort_learned_fit, for measuring what the
 * network adds (no paper counterpart): the same sample, sorted by the plain
 * path, the same frequent keys, but the map's table is the sorted sample's
 * empirical CDF at the cell starts (fraction of its non-frequent keys below
 * each start) instead of the trained model, with the same uniform floor,
 * running maximum and judge.  No training runs; the model parameters are left
 * as they were.  Same arguments, options (steps, batch and lr unused) and
 * errors as fsort_learned_fit. */
FSORT_API fsort_status fsort_learned_fit_ecdf(fsort_plan* plan, const void* keys, uint64_t n,
                                              const fsort_learned_opts* opts, void* stream);

/* Statistics of the last fit and the last judged sort.  Waits for the device. */
FSORT_API fsort_status fsort_learned_get_stats(fsort_plan* plan, fsort_learned_stats* out);

/* Copy of the fitted model (waits for the device): params_host[FSORT_MLP_PARAMS]
 * FP32 master weights (the sorts use their BF16 rounding); cells_host
 * [2 * (FSORT_LEARN_CELLS + 1)] the map table (G_i, H_i) pairs; heavy_host
 * [8192] the frequent keys ascending, *heavy_count of them; norm[2] = (center,
 * half) of the feature.  Any pointer may be NULL. */
FSORT_API fsort_status fsort_learned_get_model(fsort_plan* plan, float* params_host, uint32_t* cells_host,
                                               uint64_t* heavy_host, uint32_t* heavy_count, float* norm);

/* Install a model instead of fitting one (synchronous; host pointers).
 * heavy_host[heavy_count] ascending distinct frequent keys (heavy_count <=
 * 8192, NULL if 0); norm[2] = (center, half > 0).  If cells_host is NULL the
 * map table is built on the GPU from params_host exactly as a fit builds it;
 * otherwise cells_host[2 * (FSORT_LEARN_CELLS + 1)] is used as the table: G
 * non-decreasing with G[FSORT_LEARN_CELLS] = 0xFFFFFFFF, H_i = frequent keys
 * below the start of cell i (checked; FSORT_ERR_INVALID_ARG otherwise), and
 * params_host may be NULL. */
FSORT_API fsort_status fsort_learned_set_model(fsort_plan* plan, const float* params_host, const uint32_t* cells_host,
                                               const uint64_t* heavy_host, uint32_t heavy_count, const float* norm,
                                               void* stream);

/* ids[i] = bucket id of keys[i] under the fitted map, with the B that a sort
 * of n keys uses (device pointers: 64-bit keys, uint32_t ids; n < 2^32).
 * FSORT_ERR_INVALID_ARG without a fitted or installed model. */
FSORT_API fsort_status fsort_learned_bucket_ids(fsort_plan* plan, const void* keys, uint64_t n, uint32_t* ids,
                                                void* stream);

/* The model's kernels on caller data (device pointers), for checking them:
 * out[i] = sigmoid(mlp(x[i])) with BF16 weights w_bf16[FSORT_MLP_PARAMS];
 * grads[FSORT_MLP_PARAMS] += gradient of L = 1/(2m) sum_i (out_i - y_i)^2 and
 * *loss += L (loss may be NULL).  1 <= m. */
FSORT_API fsort_status fsort_mlp_forward(const void* w_bf16, const float* x, uint32_t m, float* out, void* stream);
FSORT_API fsort_status fsort_mlp_grad(const void* w_bf16, const float* x, const float* y, uint32_t m, float* grads,
                                      float* loss, void* stream);

/* ---- serving: a request loop with continuous batching --------------------
 * A server runs `lanes` workers, each with its own CUDA stream and plan.
 * Requests (host buffers) wait in a FIFO queue; a free worker takes the head
 * request as soon as its device buffers fit into the server's memory arena
 * (admission by free HBM), copies it in, sorts it, copies the result out and
 * frees the buffers -- requests that arrive while others run are admitted as
 * lanes and memory free up, and the lanes' work overlaps on the device.  A
 * worker that finds several small requests (at most batch_keys keys each) at
 * the head of the queue sorts them together in one fsort_sort_batch call.
 * Every result equals what fsort_sort_pairs returns for that request alone.
 * All entry points are thread-safe. */
typedef struct fsort_server fsort_server;

typedef struct fsort_serve_desc {
  uint64_t max_request_keys; /* largest n of any request (>= 1) */
  uint64_t hbm_budget_bytes; /* device bytes for admitted requests' buffers; 0 = a quarter of free memory */
  int32_t key_bits;          /* 16, 32 or 64 */
  int32_t has_values;        /* requests may carry uint32_t values */
  uint32_t lanes;            /* workers (stream + plan + thread each); 0 = 4 */
  uint32_t max_queue;        /* waiting requests before submit answers FSORT_ERR_BUSY; 0 = 65536 */
  uint32_t batch_keys;       /* requests of at most this many keys may share a batch; 0 = 1,048,576 */
  uint32_t max_batch;        /* requests per batch (1..1024); 0 = 64 */
  uint32_t flags;            /* FSORT_FLAG_LEARNED: 64-bit keys, lanes take the learned path once a
                                model is installed with fsort_serve_set_model */
  uint32_t reserved;
} fsort_serve_desc;

typedef struct fsort_request {
  const void* keys_host;     /* n keys (host memory; pinned memory makes the copies asynchronous) */
  const uint32_t* vals_host; /* n values or NULL */
  void* keys_out_host;       /* receives the sorted keys (may equal keys_host) */
  uint32_t* vals_out_host;   /* receives the values (NULL iff vals_host is NULL) */
  uint64_t n;
  int32_t precision_bits;
  uint32_t reserved;
} fsort_request;

typedef struct fsort_result {
  int32_t status;    /* fsort_status of the request */
  int32_t batched;   /* 1 if it was sorted inside a batch of several requests */
  uint64_t n;
  double latency_ms; /* submit -> result ready */
  double queue_ms;   /* submit -> admitted */
  double run_ms;     /* admitted -> result ready (copies in, sort, copies out) */
} fsort_result;

typedef struct fsort_serve_stats {
  uint64_t submitted, completed, keys_completed, batches;
  uint64_t bytes_in_use, peak_bytes, budget_bytes;
  uint32_t max_inflight; /* most requests admitted at once */
  uint32_t reserved;
  double p50_ms, p99_ms;                  /* latency percentiles (nearest rank) over the most recent
                                             1,048,576 completed requests */
  double mean_ms, max_ms;                 /* latency over all completed requests */
  double span_s;                          /* first submit -> last completion */
  double keys_per_s;                      /* keys_completed / span_s */
} fsort_serve_stats;

/* Create a server on the current device: one device arena of hbm_budget_bytes
 * (rounded up to 256 bytes), and per lane a plan for max_request_keys keys, a
 * stream and a worker thread.  FSORT_ERR_INVALID_ARG for a bad desc,
 * FSORT_ERR_OOM when the arena cannot be allocated; *out is set only on
 * FSORT_OK. */
FSORT_API fsort_status fsort_serve_create(const fsort_serve_desc* desc, fsort_server** out);
/* Finishes every admitted and queued request, then frees the server. */
FSORT_API fsort_status fsort_serve_destroy(fsort_server* server);
/* Queue a request; *ticket identifies it.  The buffers must stay valid until
 * the request is reported done.  FSORT_ERR_BUSY: the queue is full;
 * FSORT_ERR_INVALID_ARG: n > max_request_keys, bad pointers or precision, or
 * buffers larger than the whole budget. */
FSORT_API fsort_status fsort_serve_submit(fsort_server* server, const fsort_request* req, uint64_t* ticket);
/* FSORT_NOT_READY while the request runs; FSORT_OK once done (out filled, the
 * ticket retired); FSORT_ERR_INVALID_ARG for an unknown ticket. */
FSORT_API fsort_status fsort_serve_poll(fsort_server* server, uint64_t ticket, fsort_result* out);
/* Like poll, but waits up to timeout_ms (negative: no limit). */
FSORT_API fsort_status fsort_serve_wait(fsort_server* server, uint64_t ticket, double timeout_ms, fsort_result* out);
/* Counters and latency statistics so far (does not wait for the device). */
FSORT_API fsort_status fsort_serve_stats_get(fsort_server* server, fsort_serve_stats* out);
/* Install the fitted model of `source` (a plan with FSORT_FLAG_LEARNED) on
 * every lane; call while no request runs. */
FSORT_API fsort_status fsort_serve_set_model(fsort_server* server, fsort_plan* source);

/* ---- streaming histogram with rank / select --------------------------------
 * Counts of the sort keys s(k) = k >> (key_bits - precision_bits) accumulated
 * over any number of batches; each batch is read once and never again (the
 * batch counter update of Sec. III-C/D: the histogram of the batches so far
 * is kept and extended).  Queries (device arrays, stream-ordered):
 *   rank(v)   = #{accumulated keys with s(k) < v}            (Alg. 3, GetIndex)
 *   select(r) = s(k) of the key at sorted position r         (Alg. 2, GetItem)
 *               (UINT64_MAX when r >= the number accumulated)
 *   expand    = the sorted multiset of every s(k) seen, as key_bits-wide keys
 *               (for precision_bits == key_bits: the sorted keys themselves;
 *                Alg. 5 with no trailing bits)
 * precision_bits <= 24 (2^p 64-bit counters).  One object serves one stream at
 * a time.  The paper defines these on its histogram tree; the GPU keeps the
 * leaf level plus a prefix index rebuilt after each accumulation. */
typedef struct fsort_hist fsort_hist;
/* Allocate 2^precision_bits counters (zero) on the current device.
 * FSORT_ERR_INVALID_ARG for bad widths, FSORT_ERR_UNSUPPORTED for
 * precision_bits > 24, FSORT_ERR_OOM when the counters cannot be allocated. */
FSORT_API fsort_status fsort_hist_create(int key_bits, int precision_bits, fsort_hist** out);
/* Wait for the device, then free the object (NULL: no-op). */
FSORT_API fsort_status fsort_hist_destroy(fsort_hist* hist);
/* Zero the counts (stream-ordered); the total restarts at 0. */
FSORT_API fsort_status fsort_hist_reset(fsort_hist* hist, void* stream);
/* Add the counts of keys[0..n) (device). */
FSORT_API fsort_status fsort_hist_accumulate(fsort_hist* hist, const void* keys, uint64_t n, void* stream);
/* Keys accumulated so far (host-side count; no synchronisation). */
FSORT_API fsort_status fsort_hist_total(const fsort_hist* hist, uint64_t* total);
/* counts_out[v] (device, 2^precision_bits uint64_t) = accumulated keys with s(k) = v. */
FSORT_API fsort_status fsort_hist_counts(fsort_hist* hist, uint64_t* counts_out, void* stream);
/* ranks[i] = rank(values[i]) (values >= 2^p give the total). */
FSORT_API fsort_status fsort_hist_rank(fsort_hist* hist, const uint64_t* values, uint64_t count, uint64_t* ranks,
                                       void* stream);
/* values[i] = select(ranks[i]). */
FSORT_API fsort_status fsort_hist_select(fsort_hist* hist, const uint64_t* ranks, uint64_t count, uint64_t* values,
                                         void* stream);
/* keys_out[0..n) (device, key_bits wide) = the sorted multiset of s(k); n must
 * equal the total accumulated. */
FSORT_API fsort_status fsort_hist_expand(fsort_hist* hist, void* keys_out, uint64_t n, void* stream);

/* ---- the hot-path steps one at a time (same kernels as the full sort) ---- */

/* Step 2: per-pass digit histograms of keys[0..n).  counts_out (device, uint64_t)
 * receives passes x 2^digit_bits counts, pass-major, where passes =
 * ceil(precision_bits / digit_bits) and pass j counts bits [key_bits -
 * precision_bits + j*digit_bits, ...) (the last digit may be narrower; its
 * unused bins are 0).  digit_bits must be the plan's digit width, or 16 for the
 * 65,536-bin histogram of 16-bit keys at precision 16 (the expand path). */
FSORT_API fsort_status fsort_histogram(fsort_plan* plan, const void* keys, uint64_t n, int key_bits, int precision_bits,
                             int digit_bits, uint64_t* counts_out, void* stream);

/* Step 3: row-wise exclusive scan (Alg. 3's rank of every leaf):
 * offsets_out[r*bins + v] = sum_{u<v} counts[r*bins + u] for r < rows.
 * bins must be 2^digit_bits of the plan or 65536; device pointers, uint64_t. */
FSORT_API fsort_status fsort_exclusive_scan(fsort_plan* plan, const uint64_t* counts, uint64_t rows, uint64_t bins,
                                  uint64_t* offsets_out, void* stream);

/* Step 4: one stable scatter pass on raw key bits [shift, shift + width),
 * 1 <= width <= the plan's digit width, out of place.  vals_in/vals_out both
 * NULL or both set. */
FSORT_API fsort_status fsort_scatter_pass(fsort_plan* plan, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                                uint32_t* vals_out, uint64_t n, int key_bits, int shift, int width, void* stream);

/* Step 5: write key v counts[v] times for v = 0..65535 in ascending order
 * (Alg. 5 with no trailing bits); n must equal the sum of counts (device,
 * uint64_t, 65,536 entries).  16-bit keys only. */
FSORT_API fsort_status fsort_expand(fsort_plan* plan, const uint64_t* counts, void* keys_out, uint64_t n, int key_bits,
                          void* stream);

/* ---- per-kernel device timing (instrumentation) --------------------------- */

/* Kernel kinds reported by fsort_plan_timing_report. */
#define FSORT_KERNEL_HISTOGRAM 1   /* step 2, per-pass digit histograms */
#define FSORT_KERNEL_SCAN 2        /* step 3 with the pass schedule */
#define FSORT_KERNEL_SCATTER 3     /* step 4, one pass */
#define FSORT_KERNEL_COPY 4        /* final copy when the schedule needs one */
#define FSORT_KERNEL_LEAF_HIST 5   /* expand path: 65,536-bin histogram */
#define FSORT_KERNEL_LEAF_REDUCE 6 /* expand path: sum of per-CTA partial counts */
#define FSORT_KERNEL_LEAF_SCAN 7   /* expand path: exclusive scan of 65,536 bins */
#define FSORT_KERNEL_EXPAND 8      /* step 5 */
#define FSORT_KERNEL_LEARN_COUNT1 9    /* learned path: per-chunk super-bucket counts, heavy counts */
#define FSORT_KERNEL_LEARN_SCATTER1 10 /* learned path: scan + keys grouped by super-bucket */
#define FSORT_KERNEL_LEARN_COUNT2 11   /* learned path: per-bucket counts */
#define FSORT_KERNEL_LEARN_JUDGE 12    /* learned path: the judge, with the host read-back */
#define FSORT_KERNEL_LEARN_SCATTER2 13 /* learned path: scan + keys to their buckets */
#define FSORT_KERNEL_LEARN_FILL 14     /* learned path: heavy buckets */
#define FSORT_KERNEL_LEARN_BUCKETS 15  /* learned path: on-chip sort of every bucket */
#define FSORT_KERNEL_TILE_COUNT 16     /* table scatter: per-tile digit counts of a later pass's input */
#define FSORT_KERNEL_TILE_SCAN 17      /* table scatter: per-chunk digit offsets (scan of the chunk totals) */

typedef struct fsort_kernel_time {
  int32_t kind;   /* FSORT_KERNEL_* */
  int32_t pass;   /* scatter, tile count and tile scan: the pass index, else -1 */
  int32_t active; /* per-pass kernels and copy: 1 if the device schedule ran it (0: exited at once); others 1 */
  int32_t call;   /* index of the sort call since timing was enabled or last reported */
  uint64_t n;     /* keys of that call */
  float ms;       /* device time between CUDA events recorded around the launch on the call's stream */
  float reserved;
} fsort_kernel_time;

/* Enable (1) or disable (0) per-kernel timing on this plan.  While enabled,
 * every sort call records a CUDA event before its first kernel and after each
 * kernel on the call's stream (a pool of 8192 events, allocated here; calls
 * beyond the pool are not recorded).  Disabling frees the pool. */
FSORT_API fsort_status fsort_plan_set_timing(fsort_plan* plan, int enable);

/* Wait for the recorded calls, write up to `capacity` records to `out` (host
 * memory), set *count to the number written, and start a new recording. */
FSORT_API fsort_status fsort_plan_timing_report(fsort_plan* plan, fsort_kernel_time* out, uint32_t capacity,
                                                uint32_t* count);

/* ---- allocation-free entry point --------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot
 * call cudaMalloc where they sort: code running under another component's
 * memory budget (a caching allocator that already holds nearly all device
 * memory), latency-critical paths that must not take cudaMalloc's implicit
 * device synchronisation, and hosts that forbid device allocation after start
 * up.  Such callers cannot create a plan either, so this call needs none.
 *
 * fsort_scatter_pass_noalloc performs exactly what fsort_scatter_pass does
 * (one stable scatter pass on raw key bits [shift, shift + width),
 * 1 <= width <= 8, out of place, same argument rules) but keeps its scratch in
 * a fixed array of FSORT_NOALLOC_SCRATCH_BYTES (about 4 MiB) that the library
 * declares in device memory.  Every GPU that loads libfsort holds that array
 * until the process exits.  The call allocates nothing: no cudaMalloc or
 * cudaFree, no allocating library routine.
 *   - n must not exceed FSORT_NOALLOC_MAX_KEYS; larger n returns
 *     FSORT_ERR_INVALID_ARG without doing anything.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current) and keeps it for the life of the
 *     process; after a device or primary-context reset (cudaDeviceReset) the
 *     address is stale and calls are not supported.
 *   - The call is synchronous: it enqueues its kernels and the read-back of
 *     its status word on `stream`, waits for that stream (and for nothing
 *     else), and returns FSORT_ERR_TIMEOUT if a device-side wait gave up.
 *   - All calls on one device share its array, which keeps the last call's
 *     contents (the call clears what must start at zero).  The library lets
 *     one call at a time per device use it: calls from several host threads
 *     of a process take turns (each waits until the previous one has
 *     returned).  Devices with an index of 64 or more return
 *     FSORT_ERR_UNSUPPORTED. */
#define FSORT_NOALLOC_MAX_KEYS 16777216ull
#define FSORT_NOALLOC_SCRATCH_BYTES 4199168ull
FSORT_API fsort_status fsort_scatter_pass_noalloc(const void* keys_in, const uint32_t* vals_in, void* keys_out,
                                                  uint32_t* vals_out, uint64_t n, int key_bits, int shift, int width,
                                                  void* stream);

/* Failure-detection test hook, for tests of the error path only (no paper
 * counterpart).  After this call, scatter tile `withhold_tile` of every
 * chained-form scatter pass of this plan (FSORT_FLAG_CHAINED_SCATTER plans,
 * sorts of more than 2^32 keys, batched and one-pass calls) never publishes
 * its look-back words, so the tiles after it wait for a flag that nothing
 * sets.  Each such wait gives up after `wait_limit_ns` nanoseconds of the
 * device's global timer (0 restores the default bound of 2 s) and sets status
 * bit 1; a wait that sees the bit set by another gives up at once, so the whole
 * pass ends within about one bound.  The tiles that gave up write nothing, and
 * the next fsort_plan_sync (or call) returns FSORT_ERR_TIMEOUT.  No wait is
 * unbounded and nothing faults: the plan and the CUDA context stay usable.
 * withhold_tile = 0xFFFFFFFF removes the hook.  Not stream-ordered: set it
 * while no call of this plan is in flight. */
FSORT_API fsort_status fsort_plan_set_fault_hook(fsort_plan* plan, uint32_t withhold_tile, uint64_t wait_limit_ns);

/* Raw device flag bits behind the last FSORT_ERR_TIMEOUT / FSORT_ERR_INTERNAL
 * this plan reported (0 if none): 1 look-back wait timed out, 2 bulk-copy wait
 * timed out, 4 tile id beyond the grid, 8 look-back walk found no prefix at its
 * chunk's first tile, 16 a tile skipped its output after a wait gave up, 32 a
 * learned-path bucket exceeded the on-chip capacity, 64 a tile-offset table was
 * incomplete (its scatter wrote nothing). */
FSORT_API uint32_t fsort_plan_device_flags(const fsort_plan* plan);

/* Human-readable name of a status code (static storage). */
FSORT_API const char* fsort_status_string(fsort_status status);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH (for this 0.x series: 100 = first release, 200 =
 * fsort_plan_info with scatter_form, scatter passes from a table of per-tile offsets by default). */
FSORT_API int fsort_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FSORT_H */
