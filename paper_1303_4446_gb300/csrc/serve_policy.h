// Scheduling policy of the X2C server (continuous batching under a device-memory budget),
// kept free of CUDA so that it can be compiled and checked on a host without a GPU.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <vector>

namespace x2c {
namespace serve {

// One queued request as the policy sees it.
struct Candidate {
  size_t bytes;     // device memory the request needs of its own (copied inputs, outputs)
  uint64_t group;   // requests with equal group keys can be built in one launch
  bool batchable;   // false: always built alone (full X2C, molecular-block DLU)
};

// Requests to start together on one free slot, as indexes into `queue` (arrival order).
// The head of the queue always comes first: if it does not fit into `free_bytes` nothing
// starts (first come, first served; a large request is never starved by smaller ones behind
// it).  After the head, later requests of the same group join while the batch holds fewer
// than `max_batch` requests and their bytes still fit; the scan stops at the first one of
// that group that does not fit, so requests of a group keep their order.  Requests of other
// groups are passed over and keep their places for the next free slot.
inline std::vector<size_t> choose_batch(const std::vector<Candidate> &queue, size_t free_bytes,
                                        int max_batch) {
  std::vector<size_t> pick;
  if (queue.empty() || max_batch < 1 || queue[0].bytes > free_bytes) return pick;
  pick.push_back(0);
  size_t used = queue[0].bytes;
  if (!queue[0].batchable) return pick;
  for (size_t i = 1; i < queue.size() && (int)pick.size() < max_batch; ++i) {
    const Candidate &c = queue[i];
    if (!c.batchable || c.group != queue[0].group) continue;
    if (c.bytes > free_bytes - used) break;
    pick.push_back(i);
    used += c.bytes;
  }
  return pick;
}

// Nearest-rank percentile (p in [0, 100]) of the samples: the smallest sample such that at
// least p percent of the samples are <= it.  NaN for no samples.
inline double percentile(std::vector<double> v, double p) {
  if (v.empty()) return std::nan("");
  std::sort(v.begin(), v.end());
  const double r = std::ceil(p / 100.0 * static_cast<double>(v.size()));
  size_t k = r < 1.0 ? 0 : static_cast<size_t>(r) - 1;
  if (k >= v.size()) k = v.size() - 1;
  return v[k];
}

// Least-recently-used cache entries to evict, oldest first, until `need` bytes are freed:
// entries are (last use, bytes, evictable); returns their indexes, or nothing if even all
// evictable entries together do not free enough.
struct CacheView {
  uint64_t last_use;
  size_t bytes;
  bool evictable;  // ready and used by no request in flight
};
inline std::vector<size_t> choose_evictions(const std::vector<CacheView> &entries, size_t need) {
  std::vector<size_t> idx;
  for (size_t i = 0; i < entries.size(); ++i)
    if (entries[i].evictable) idx.push_back(i);
  std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
    return entries[a].last_use != entries[b].last_use ? entries[a].last_use < entries[b].last_use : a < b;
  });
  std::vector<size_t> out;
  size_t freed = 0;
  for (size_t i : idx) {
    if (freed >= need) break;
    out.push_back(i);
    freed += entries[i].bytes;
  }
  if (freed < need) out.clear();
  return out;
}

}  // namespace serve
}  // namespace x2c
