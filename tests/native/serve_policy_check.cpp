// Host-only checks of the server's scheduling policy (no CUDA): prints "ok" or the first
// failed check and exits non-zero.
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../paper_1303_4446_gb300/csrc/serve_policy.h"

using x2c::serve::Candidate;
using x2c::serve::CacheView;

static int fails = 0;
#define CHECK(cond)                                           \
  do {                                                        \
    if (!(cond)) {                                            \
      std::printf("FAIL line %d: %s\n", __LINE__, #cond);     \
      ++fails;                                                \
    }                                                         \
  } while (0)

static bool same(const std::vector<size_t> &a, const std::vector<size_t> &b) { return a == b; }

int main() {
  using x2c::serve::choose_batch;
  // empty queue, no slots of memory, bad batch size
  CHECK(choose_batch({}, 100, 4).empty());
  CHECK(choose_batch({{10, 1, true}}, 9, 4).empty());         // head does not fit: nothing starts
  CHECK(choose_batch({{10, 1, true}}, 100, 0).empty());
  // head alone when it is not batchable
  CHECK(same(choose_batch({{10, 0, false}, {10, 0, false}}, 100, 4), {0}));
  // same group joins, other groups are passed over, order kept
  std::vector<Candidate> q = {{10, 7, true}, {10, 8, true}, {10, 7, true}, {10, 0, false}, {10, 7, true}};
  CHECK(same(choose_batch(q, 100, 8), {0, 2, 4}));
  CHECK(same(choose_batch(q, 100, 2), {0, 2}));                // max_batch
  CHECK(same(choose_batch(q, 25, 8), {0, 2}));                 // memory stops the scan
  // the scan stops at the first same-group request that does not fit (no overtaking)
  std::vector<Candidate> q2 = {{10, 7, true}, {50, 7, true}, {5, 7, true}};
  CHECK(same(choose_batch(q2, 30, 8), {0}));
  // a large head is never skipped for small requests behind it
  std::vector<Candidate> q3 = {{90, 7, true}, {1, 7, true}};
  CHECK(choose_batch(q3, 50, 8).empty());

  using x2c::serve::percentile;
  CHECK(std::isnan(percentile({}, 50)));
  CHECK(percentile({5.0}, 99) == 5.0);
  std::vector<double> v;
  for (int i = 100; i >= 1; --i) v.push_back(i);              // 1..100, unsorted
  CHECK(percentile(v, 50) == 50.0);
  CHECK(percentile(v, 99) == 99.0);
  CHECK(percentile(v, 100) == 100.0);
  CHECK(percentile(v, 0) == 1.0);
  CHECK(percentile({3, 1, 2}, 50) == 2.0);
  CHECK(percentile({1, 2, 3, 4}, 50) == 2.0);                 // nearest rank: ceil(0.5 * 4) = 2

  using x2c::serve::choose_evictions;
  std::vector<CacheView> c = {{5, 10, true}, {1, 10, false}, {3, 10, true}, {2, 10, true}};
  CHECK(same(choose_evictions(c, 10), {3}));                   // oldest evictable first
  CHECK(same(choose_evictions(c, 15), {3, 2}));
  CHECK(same(choose_evictions(c, 30), {3, 2, 0}));
  CHECK(choose_evictions(c, 31).empty());                       // not enough even with all
  CHECK(choose_evictions(c, 0).empty());

  if (fails == 0) std::printf("ok\n");
  return fails == 0 ? 0 : 1;
}
