// fsort_serve.cu -- the request loop (host runtime; the sorting itself is
// this library's kernels, reached through its own C ABI).
//
//   lanes     one worker thread, CUDA stream and plan each; the lanes' copies
//             and kernels overlap on the device
//   arena     one device allocation of hbm_budget_bytes, carved first-fit
//             with coalescing on free; a request is admitted when its key
//             and value buffers fit (admission by free HBM)
//   queue     FIFO; a free lane takes the head request as soon as it fits,
//             together with every compatible small request waiting anywhere
//             behind it that fits too (continuous batching: nothing waits for
//             a batch to fill or to drain)
//   latency   steady-clock stamps at submit, admission and completion
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/fsort.h"
#include "fsort_serve_host.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

using fsort_serve::Arena;
using fsort_serve::LatencyLog;

struct Req {
  uint64_t ticket = 0;
  fsort_request r{};
  size_t bytes = 0;  // device bytes (keys + values)
  size_t off = 0;    // arena offset once admitted
  Clock::time_point t_submit, t_admit, t_done;
  fsort_status status = FSORT_OK;
  bool done = false;
  bool batched = false;
};

struct Lane {
  cudaStream_t stream = nullptr;
  fsort_plan* plan = nullptr;
};

}  // namespace

struct fsort_server {
  fsort_serve_desc desc{};
  int device = 0;
  unsigned char* mem = nullptr;  // the arena
  Arena arena;
  std::mutex mu;
  std::condition_variable cv_work;  // a request was queued, memory was freed, or stop
  std::condition_variable cv_done;  // a request finished
  std::deque<Req*> pending;
  std::unordered_map<uint64_t, Req*> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::vector<Lane> lanes;
  std::vector<std::thread> threads;
  // statistics
  uint64_t submitted = 0, completed = 0, keys_completed = 0, batches = 0;
  uint32_t inflight = 0, max_inflight = 0;
  LatencyLog latencies;  // ms, submit -> completion
  bool any = false;
  Clock::time_point t_first, t_last;
};

namespace {

size_t key_bytes(const fsort_server* s) { return size_t(s->desc.key_bits) / 8; }

size_t request_bytes(const fsort_server* s, const fsort_request& r) {
  return Arena::round(size_t(r.n) * key_bytes(s)) + (r.vals_host ? Arena::round(size_t(r.n) * 4) : 0);
}

// Enqueue admitted requests on one lane: copy in, sort (alone or as one
// batch), copy out.
fsort_status enqueue_requests(fsort_server* s, Lane& lane, std::vector<Req*>& batch) {
  const size_t kb = key_bytes(s);
  cudaError_t e = cudaSuccess;
  std::vector<fsort_segment> segs;
  for (Req* q : batch) {
    unsigned char* base = s->mem + q->off;
    const size_t kbytes = size_t(q->r.n) * kb;
    uint32_t* vals = q->r.vals_host ? reinterpret_cast<uint32_t*>(base + Arena::round(kbytes)) : nullptr;
    if (e == cudaSuccess) e = cudaMemcpyAsync(base, q->r.keys_host, kbytes, cudaMemcpyHostToDevice, lane.stream);
    if (e == cudaSuccess && vals)
      e = cudaMemcpyAsync(vals, q->r.vals_host, size_t(q->r.n) * 4, cudaMemcpyHostToDevice, lane.stream);
    segs.push_back(fsort_segment{base, vals, q->r.n});
  }
  if (e != cudaSuccess) return FSORT_ERR_CUDA;
  fsort_status st = FSORT_OK;
  if (batch.size() == 1) {
    const Req* q = batch[0];
    st = fsort_sort_pairs(lane.plan, segs[0].keys, segs[0].vals, q->r.n, s->desc.key_bits, q->r.precision_bits,
                          lane.stream);
  } else {
    st = fsort_sort_batch(lane.plan, segs.data(), uint32_t(segs.size()), s->desc.key_bits,
                          batch[0]->r.precision_bits, lane.stream);
  }
  if (st != FSORT_OK) return st;
  for (size_t i = 0; i < batch.size() && e == cudaSuccess; ++i) {
    const Req* q = batch[i];
    e = cudaMemcpyAsync(q->r.keys_out_host, segs[i].keys, size_t(q->r.n) * kb, cudaMemcpyDeviceToHost, lane.stream);
    if (e == cudaSuccess && segs[i].vals)
      e = cudaMemcpyAsync(q->r.vals_out_host, segs[i].vals, size_t(q->r.n) * 4, cudaMemcpyDeviceToHost, lane.stream);
  }
  return e == cudaSuccess ? FSORT_OK : FSORT_ERR_CUDA;
}

// Run admitted requests on one lane and wait for them.  The lane's stream is
// drained on every outcome: the requests' arena blocks are freed next and may
// go to another lane at once, so no copy or kernel of this batch may still be
// in flight, even after a failed enqueue.
fsort_status run_requests(fsort_server* s, Lane& lane, std::vector<Req*>& batch) {
  const fsort_status st = enqueue_requests(s, lane, batch);
  const cudaError_t e = cudaStreamSynchronize(lane.stream);
  if (st != FSORT_OK) return st;
  if (e != cudaSuccess) return FSORT_ERR_CUDA;
  return fsort_plan_sync(lane.plan);
}

void lane_main(fsort_server* s, size_t li) {
  cudaSetDevice(s->device);
  Lane& lane = s->lanes[li];
  const uint32_t max_batch = s->desc.max_batch;
  for (;;) {
    std::vector<Req*> batch;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (!s->pending.empty()) {
          Req* head = s->pending.front();
          size_t off = 0;
          if (s->arena.alloc(head->bytes, &off)) {
            head->off = off;
            s->pending.pop_front();
            batch.push_back(head);
            break;
          }
        } else if (s->stop) {
          return;
        }
        s->cv_work.wait(lk);
      }
      // A small head takes every compatible small request still waiting into
      // its batch, in arrival order, as far as each fits the arena (same
      // precision and values; a batch's keys, each segment rounded up to 8,
      // fit the lane plan's max_n).  Requests that do not match or do not fit
      // keep their place in the queue for the next free lane.
      Req* head = batch[0];
      uint64_t total = (head->r.n + 7) / 8 * 8;
      if (head->r.n <= s->desc.batch_keys) {
        for (auto it = s->pending.begin(); it != s->pending.end() && batch.size() < max_batch;) {
          Req* q = *it;
          const uint64_t padded = (q->r.n + 7) / 8 * 8;
          size_t off = 0;
          if (q->r.n > s->desc.batch_keys || q->r.precision_bits != head->r.precision_bits ||
              (q->r.vals_host == nullptr) != (head->r.vals_host == nullptr) ||
              total + padded > s->desc.max_request_keys || !s->arena.alloc(q->bytes, &off)) {
            ++it;
            continue;
          }
          total += padded;
          q->off = off;
          it = s->pending.erase(it);
          batch.push_back(q);
        }
      }
      const Clock::time_point now = Clock::now();
      for (Req* q : batch) {
        q->t_admit = now;
        q->batched = batch.size() > 1;
      }
      s->inflight += uint32_t(batch.size());
      s->max_inflight = std::max(s->max_inflight, s->inflight);
      if (batch.size() > 1) ++s->batches;
    }
    const fsort_status st = run_requests(s, lane, batch);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      const Clock::time_point now = Clock::now();
      for (Req* q : batch) {
        q->status = st;
        q->t_done = now;
        q->done = true;
        s->arena.release(q->off, q->bytes);
        ++s->completed;
        s->keys_completed += q->r.n;
        s->latencies.record(ms_between(q->t_submit, now));
      }
      s->inflight -= uint32_t(batch.size());
      s->t_last = now;
    }
    s->cv_work.notify_all();  // memory came free
    s->cv_done.notify_all();
  }
}

fsort_status take_result(fsort_server* s, uint64_t ticket, fsort_result* out) {
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return FSORT_ERR_INVALID_ARG;
  Req* q = it->second;
  if (!q->done) return FSORT_NOT_READY;
  if (out) {
    out->status = q->status;
    out->batched = q->batched ? 1 : 0;
    out->n = q->r.n;
    out->latency_ms = ms_between(q->t_submit, q->t_done);
    out->queue_ms = ms_between(q->t_submit, q->t_admit);
    out->run_ms = ms_between(q->t_admit, q->t_done);
  }
  s->reqs.erase(it);
  delete q;
  return FSORT_OK;
}

}  // namespace

extern "C" {

fsort_status fsort_serve_create(const fsort_serve_desc* desc, fsort_server** out) {
  if (!desc || !out || desc->max_request_keys < 1) return FSORT_ERR_INVALID_ARG;
  if (desc->key_bits != 16 && desc->key_bits != 32 && desc->key_bits != 64) return FSORT_ERR_INVALID_ARG;
  if (desc->has_values != 0 && desc->has_values != 1) return FSORT_ERR_INVALID_ARG;
  if (desc->flags & ~FSORT_FLAG_LEARNED) return FSORT_ERR_INVALID_ARG;
  if ((desc->flags & FSORT_FLAG_LEARNED) && desc->key_bits != 64) return FSORT_ERR_UNSUPPORTED;
  if (desc->max_batch > 1024 || desc->lanes > 64) return FSORT_ERR_INVALID_ARG;
  fsort_server* s = new (std::nothrow) fsort_server();
  if (!s) return FSORT_ERR_OOM;
  s->desc = *desc;
  if (!s->desc.lanes) s->desc.lanes = 4;
  if (!s->desc.max_queue) s->desc.max_queue = 65536;
  if (!s->desc.batch_keys) s->desc.batch_keys = 1u << 20;
  if (!s->desc.max_batch) s->desc.max_batch = 64;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return FSORT_ERR_CUDA;
  }
  size_t budget = desc->hbm_budget_bytes;
  if (!budget) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      delete s;
      return FSORT_ERR_CUDA;
    }
    budget = free_b / 4;
  }
  budget = Arena::round(budget);
  if (cudaMalloc(reinterpret_cast<void**>(&s->mem), budget) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return FSORT_ERR_OOM;
  }
  s->arena.reset(budget);
  s->desc.hbm_budget_bytes = budget;
  // lanes: a plan sized for the largest request (batches are bounded by it too)
  fsort_plan_desc pd{};
  pd.max_n = desc->max_request_keys;
  pd.key_bits = desc->key_bits;
  pd.has_values = desc->has_values;
  pd.flags = desc->flags & FSORT_FLAG_LEARNED;
  pd.max_segments = s->desc.max_batch;
  s->lanes.resize(s->desc.lanes);
  for (Lane& l : s->lanes) {
    fsort_status st = fsort_plan_create(&pd, &l.plan);
    if (st == FSORT_OK && cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess)
      st = FSORT_ERR_CUDA;
    if (st != FSORT_OK) {
      fsort_serve_destroy(s);
      return st;
    }
  }
  for (size_t i = 0; i < s->lanes.size(); ++i) s->threads.emplace_back(lane_main, s, i);
  *out = s;
  return FSORT_OK;
}

fsort_status fsort_serve_destroy(fsort_server* s) {
  if (!s) return FSORT_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (std::thread& t : s->threads) t.join();
  fsort_status st = FSORT_OK;
  for (Lane& l : s->lanes) {
    if (l.plan && fsort_plan_destroy(l.plan) != FSORT_OK) st = FSORT_ERR_CUDA;
    if (l.stream) cudaStreamDestroy(l.stream);
  }
  for (auto& kv : s->reqs) delete kv.second;
  if (s->mem && cudaFree(s->mem) != cudaSuccess) st = FSORT_ERR_CUDA;
  delete s;
  return st;
}

fsort_status fsort_serve_submit(fsort_server* s, const fsort_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return FSORT_ERR_INVALID_ARG;
  const fsort_request& r = *req;
  if (r.n > s->desc.max_request_keys) return FSORT_ERR_INVALID_ARG;
  if (r.precision_bits < 1 || r.precision_bits > s->desc.key_bits) return FSORT_ERR_INVALID_ARG;
  if ((r.vals_host == nullptr) != (r.vals_out_host == nullptr)) return FSORT_ERR_INVALID_ARG;
  if (r.vals_host && !s->desc.has_values) return FSORT_ERR_INVALID_ARG;
  if (r.n && (!r.keys_host || !r.keys_out_host)) return FSORT_ERR_INVALID_ARG;
  const size_t bytes = request_bytes(s, r);
  if (bytes > s->arena.size()) return FSORT_ERR_INVALID_ARG;
  Req* q = new (std::nothrow) Req();
  if (!q) return FSORT_ERR_OOM;
  q->r = r;
  q->bytes = bytes ? bytes : 256;
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->pending.size() >= s->desc.max_queue) {
      delete q;
      return FSORT_ERR_BUSY;
    }
    q->ticket = s->next_ticket++;
    s->reqs[q->ticket] = q;
    ++s->submitted;
    if (!s->any) {
      s->any = true;
      s->t_first = q->t_submit;
    }
    if (r.n == 0) {  // nothing to sort: done at once
      q->done = true;
      q->t_admit = q->t_done = q->t_submit;
      ++s->completed;
      s->latencies.record(0.0);
      s->t_last = q->t_done;
    } else {
      s->pending.push_back(q);
    }
    *ticket = q->ticket;
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  return FSORT_OK;
}

fsort_status fsort_serve_poll(fsort_server* s, uint64_t ticket, fsort_result* out) {
  if (!s) return FSORT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  return take_result(s, ticket, out);
}

fsort_status fsort_serve_wait(fsort_server* s, uint64_t ticket, double timeout_ms, fsort_result* out) {
  if (!s) return FSORT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const Clock::time_point until =
      Clock::now() + std::chrono::microseconds(int64_t(timeout_ms < 0 ? 0 : timeout_ms * 1000.0));
  for (;;) {
    const fsort_status st = take_result(s, ticket, out);
    if (st != FSORT_NOT_READY) return st;
    if (timeout_ms < 0) {
      s->cv_done.wait(lk);
    } else if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout) {
      return take_result(s, ticket, out);
    }
  }
}

fsort_status fsort_serve_stats_get(fsort_server* s, fsort_serve_stats* out) {
  if (!s || !out) return FSORT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->keys_completed = s->keys_completed;
  out->batches = s->batches;
  out->bytes_in_use = s->arena.used();
  out->peak_bytes = s->arena.peak();
  out->budget_bytes = s->arena.size();
  out->max_inflight = s->max_inflight;
  if (s->latencies.count()) {
    const std::vector<double> p = s->latencies.percentiles({0.50, 0.99});
    out->p50_ms = p[0];
    out->p99_ms = p[1];
    out->max_ms = s->latencies.max();
    out->mean_ms = s->latencies.mean();
  }
  if (s->any) {
    out->span_s = std::chrono::duration<double>(s->t_last - s->t_first).count();
    if (out->span_s > 0) out->keys_per_s = double(s->keys_completed) / out->span_s;
  }
  return FSORT_OK;
}

fsort_status fsort_serve_set_model(fsort_server* s, fsort_plan* source) {
  if (!s || !source || !(s->desc.flags & FSORT_FLAG_LEARNED)) return FSORT_ERR_INVALID_ARG;
  std::vector<float> params(FSORT_MLP_PARAMS);
  std::vector<uint32_t> cells(2 * (FSORT_LEARN_CELLS + 1));
  std::vector<uint64_t> heavy(8192);
  uint32_t m = 0;
  float norm[2] = {0.f, 1.f};
  fsort_status st = fsort_learned_get_model(source, params.data(), cells.data(), heavy.data(), &m, norm);
  fsort_learned_stats ls{};
  if (st == FSORT_OK) st = fsort_learned_get_stats(source, &ls);
  if (st != FSORT_OK) return st;
  if (!ls.fitted) return FSORT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->inflight || !s->pending.empty()) return FSORT_ERR_BUSY;
  for (Lane& l : s->lanes) {
    st = fsort_learned_set_model(l.plan, params.data(), cells.data(), heavy.data(), m, norm, l.stream);
    if (st != FSORT_OK) return st;
  }
  return FSORT_OK;
}

}  // extern "C"
