// Host-side scheduling structures of the solve server, free of CUDA so that they
// build and test on any host: a first-fit range allocator over the server's
// device-memory budget, and latency statistics.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <iterator>
#include <map>
#include <vector>

namespace dpt {

// First-fit allocator over the byte range [0, capacity).  Every range starts on
// an `align` boundary and its size is rounded up to `align`; freed ranges merge
// with free neighbours.  It hands out offsets only: the owner adds them to the
// base address of one device allocation, so admitting a request never calls
// cudaMalloc.
class RangeAllocator {
 public:
  explicit RangeAllocator(uint64_t capacity = 0, uint64_t align = 256) : align_(align) {
    reset(capacity);
  }

  void reset(uint64_t capacity) {
    cap_ = capacity / align_ * align_;
    free_.clear();
    used_.clear();
    in_use_ = 0;
    if (cap_) free_[0] = cap_;
  }

  // Rounds `bytes` up to the alignment; false when no free range is large enough.
  bool alloc(uint64_t bytes, uint64_t* off) {
    const uint64_t need = round(bytes == 0 ? 1 : bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const uint64_t o = it->first, sz = it->second;
      free_.erase(it);
      if (sz > need) free_[o + need] = sz - need;
      used_[o] = need;
      in_use_ += need;
      peak_ = std::max(peak_, in_use_);
      *off = o;
      return true;
    }
    return false;
  }

  // Returns false (and changes nothing) for an offset alloc() did not hand out.
  bool free(uint64_t off) {
    auto u = used_.find(off);
    if (u == used_.end()) return false;
    uint64_t o = off, sz = u->second;
    used_.erase(u);
    in_use_ -= sz;
    auto next = free_.lower_bound(o);
    if (next != free_.end() && o + sz == next->first) {
      sz += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == o) {
        prev->second += sz;
        return true;
      }
    }
    free_[o] = sz;
    return true;
  }

  // Bytes a request of `bytes` takes (after alignment).
  uint64_t footprint(uint64_t bytes) const { return round(bytes == 0 ? 1 : bytes); }
  uint64_t capacity() const { return cap_; }
  uint64_t in_use() const { return in_use_; }
  uint64_t peak() const { return peak_; }
  uint64_t largest_free() const {
    uint64_t m = 0;
    for (const auto& f : free_) m = std::max(m, f.second);
    return m;
  }
  size_t free_ranges() const { return free_.size(); }
  size_t live() const { return used_.size(); }

 private:
  uint64_t round(uint64_t b) const { return (b + align_ - 1) / align_ * align_; }
  uint64_t align_;
  uint64_t cap_ = 0;
  uint64_t in_use_ = 0;
  uint64_t peak_ = 0;
  std::map<uint64_t, uint64_t> free_;   // offset -> size
  std::map<uint64_t, uint64_t> used_;   // offset -> size
};

// Nearest-rank percentile (q in [0, 1]) of a sample; 0 for an empty sample.
inline double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double r = std::ceil(q * (double)v.size());
  size_t k = r < 1.0 ? 0 : (size_t)r - 1;
  if (k >= v.size()) k = v.size() - 1;
  return v[k];
}

}  // namespace dpt
