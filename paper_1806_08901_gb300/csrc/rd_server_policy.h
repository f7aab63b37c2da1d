// rd_server_policy.h -- admission of selection requests under a device-memory
// budget, for the serving loop (rd_server_*).  Plain C++, no CUDA: the
// serving runtime calls it under its lock, and the CPU tests drive it
// directly.
//
// Resident fields are keyed by the caller's field key.  A request for a key
// that is resident and loaded is admitted at once (a hit) and pins the entry
// while it runs.  A request for a key not resident needs `bytes` of budget:
// unpinned resident entries are evicted, least recently used first, until it
// fits; the new entry is pinned and marked loading until the runtime has
// copied the field in (mark_loaded).  A request for a key that is still
// loading waits (not admissible yet).  Transient requests (key 0) hold
// their bytes only while they run.  A request larger than the whole budget
// can never be admitted (the runtime rejects it at submission).  A budget
// of 0 means no bound.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <unordered_map>
#include <utility>
#include <vector>

namespace rdk {

class AdmissionPolicy {
 public:
  struct Decision {
    bool admitted = false;
    bool hit = false;               // the field was resident and loaded
    std::vector<uint64_t> evicted;  // keys whose storage the runtime frees
  };

  explicit AdmissionPolicy(size_t budget) : budget_(budget) {}

  size_t budget() const { return budget_; }
  size_t used() const { return used_; }
  size_t resident_count() const { return entries_.size(); }
  uint64_t evictions() const { return evictions_; }
  bool fits_at_all(size_t bytes) const { return budget_ == 0 || bytes <= budget_; }

  // Try to admit a request for `key` (0: transient) needing `bytes` when not
  // resident.  On success the entry is pinned (and, when new, loading).
  Decision admit(uint64_t key, size_t bytes) {
    Decision d;
    if (key != 0) {
      auto it = entries_.find(key);
      if (it != entries_.end()) {
        if (!it->second.loaded) return d;  // another request is loading it
        it->second.pins++;
        it->second.last_use = ++clock_;
        d.admitted = true;
        d.hit = true;
        return d;
      }
    }
    if (!fits_at_all(bytes)) return d;
    std::vector<uint64_t> victims;
    if (budget_ != 0 && used_ + bytes > budget_) {
      // evict unpinned loaded entries, least recently used first, until it fits
      std::vector<std::pair<uint64_t, uint64_t>> order;  // (last use, key)
      for (const auto& kv : entries_)
        if (kv.second.pins == 0 && kv.second.loaded) order.push_back({kv.second.last_use, kv.first});
      std::sort(order.begin(), order.end());
      size_t freed = 0;
      for (const auto& o : order) {
        if (used_ - freed + bytes <= budget_) break;
        victims.push_back(o.second);
        freed += entries_[o.second].bytes;
      }
      if (used_ - freed + bytes > budget_) return d;  // pinned or loading entries hold the budget
    }
    for (uint64_t v : victims) {
      used_ -= entries_[v].bytes;
      entries_.erase(v);
      evictions_++;
    }
    used_ += bytes;
    if (key != 0) {
      Entry e;
      e.bytes = bytes;
      e.pins = 1;
      e.loaded = false;
      e.last_use = ++clock_;
      entries_[key] = e;
    }
    d.admitted = true;
    d.evicted = std::move(victims);
    return d;
  }

  // The runtime copied the field of `key` in; requests for it may now hit.
  void mark_loaded(uint64_t key) {
    auto it = entries_.find(key);
    if (it != entries_.end()) it->second.loaded = true;
  }

  // A load failed: drop the entry with its pin and bytes.
  void drop(uint64_t key) {
    auto it = entries_.find(key);
    if (it == entries_.end()) return;
    used_ -= it->second.bytes;
    entries_.erase(it);
  }

  // The request for `key` ended (transient requests give their bytes back).
  void release(uint64_t key, size_t bytes) {
    if (key == 0) {
      used_ -= bytes;
      return;
    }
    auto it = entries_.find(key);
    if (it != entries_.end() && it->second.pins > 0) it->second.pins--;
  }

  bool is_resident(uint64_t key) const { return entries_.count(key) != 0; }
  int pins(uint64_t key) const {
    auto it = entries_.find(key);
    return it == entries_.end() ? 0 : it->second.pins;
  }

 private:
  struct Entry {
    size_t bytes = 0;
    int pins = 0;
    bool loaded = false;
    uint64_t last_use = 0;
  };

  size_t budget_;
  size_t used_ = 0;
  uint64_t clock_ = 0;
  uint64_t evictions_ = 0;
  std::unordered_map<uint64_t, Entry> entries_;
};

}  // namespace rdk
