// fsort_serve_host.h -- host-only parts of the request loop: the device-memory
// arena that admission draws on, and the latency log behind p50/p99.  Plain
// C++ (no CUDA), so the host tests compile and check them on their own.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>
#include <vector>

namespace fsort_serve {

// First-fit allocator over [0, size) in 256-byte granules.  Free ranges are
// kept coalesced (no two adjacent), so each is a maximal run of free granules
// and first fit takes the lowest-addressed run that is long enough.
class Arena {
 public:
  static constexpr size_t kGranule = 256;
  static size_t round(size_t b) { return (b + kGranule - 1) / kGranule * kGranule; }

  void reset(size_t size) {
    size_ = size / kGranule * kGranule;
    free_.clear();
    if (size_) free_[0] = size_;
    used_ = peak_ = 0;
  }
  // Offset of `bytes` (rounded up to granules) at the first free range that
  // holds them; false (nothing changed) if none does.
  bool alloc(size_t bytes, size_t* off) {
    bytes = round(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  // Return a range that alloc gave out (same offset and size).
  void release(size_t off, size_t bytes) {
    bytes = round(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  size_t free_ranges() const { return free_.size(); }

 private:
  size_t size_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
};

// Request latencies: percentiles over a window of the most recent ones (a
// ring, so a long-running server's statistics take bounded memory), mean and
// maximum over all of them.
class LatencyLog {
 public:
  explicit LatencyLog(size_t window = size_t(1) << 20) : window_(window ? window : 1) {}

  void record(double ms) {
    if (ring_.size() < window_)
      ring_.push_back(ms);
    else
      ring_[next_] = ms;
    next_ = (next_ + 1) % window_;
    ++count_;
    sum_ += ms;
    max_ = count_ == 1 ? ms : std::max(max_, ms);
  }
  uint64_t count() const { return count_; }
  double mean() const { return count_ ? sum_ / double(count_) : 0.0; }
  double max() const { return max_; }
  // Nearest-rank percentiles (p in (0, 1]) of the window, one per entry of ps.
  std::vector<double> percentiles(const std::vector<double>& ps) const {
    std::vector<double> out(ps.size(), 0.0);
    if (ring_.empty()) return out;
    std::vector<double> v = ring_;
    for (size_t k = 0; k < ps.size(); ++k) {
      size_t i = size_t(ps[k] * double(v.size()) + 0.999999);
      i = std::min(std::max(i, size_t(1)), v.size());
      std::nth_element(v.begin(), v.begin() + (i - 1), v.end());
      out[k] = v[i - 1];
    }
    return out;
  }

 private:
  size_t window_;
  std::vector<double> ring_;
  size_t next_ = 0;
  uint64_t count_ = 0;
  double sum_ = 0.0, max_ = 0.0;
};

}  // namespace fsort_serve
