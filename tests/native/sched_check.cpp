// Host-side checks of the server's scheduling structures (dpt_sched.h): the
// first-fit range allocator against a byte-map model under random traffic, and
// the nearest-rank percentile.  Prints "ok" and exits 0 on success.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "dpt_sched.h"

#define REQUIRE(c)                                                   \
  do {                                                               \
    if (!(c)) {                                                      \
      std::fprintf(stderr, "check failed line %d: %s\n", __LINE__, #c); \
      return 1;                                                      \
    }                                                                \
  } while (0)

int main() {
  using dpt::RangeAllocator;
  const uint64_t align = 256, cap = 256 * 1000;
  RangeAllocator a(cap + 100, align);        // capacity rounds down to the alignment
  REQUIRE(a.capacity() == cap);
  REQUIRE(a.largest_free() == cap && a.free_ranges() == 1 && a.in_use() == 0);

  // byte map: owner id of each 256-byte unit (0 = free)
  std::vector<int> map(cap / align, 0);
  struct Live { uint64_t off, units; int id; };
  std::vector<Live> live;
  std::mt19937_64 rng(2002);
  int next = 1;
  uint64_t model_used = 0;
  for (int step = 0; step < 20000; ++step) {
    const bool do_alloc = live.empty() || (rng() % 100) < 55;
    if (do_alloc) {
      const uint64_t bytes = 1 + rng() % (align * 40);
      const uint64_t units = (bytes + align - 1) / align;
      uint64_t off;
      // first fit in the model
      long first = -1;
      for (size_t u = 0, run = 0; u < map.size(); ++u) {
        run = map[u] ? 0 : run + 1;
        if (run == units) { first = (long)(u + 1 - units); break; }
      }
      const bool ok = a.alloc(bytes, &off);
      REQUIRE(ok == (first >= 0));
      if (!ok) continue;
      REQUIRE(off % align == 0);
      REQUIRE((long)(off / align) == first);
      for (uint64_t u = off / align; u < off / align + units; ++u) {
        REQUIRE(map[u] == 0);
        map[u] = next;
      }
      live.push_back({off, units, next++});
      model_used += units * align;
    } else {
      const size_t k = rng() % live.size();
      const Live l = live[k];
      REQUIRE(a.free(l.off));
      REQUIRE(!a.free(l.off));                 // double free is refused
      for (uint64_t u = l.off / align; u < l.off / align + l.units; ++u) map[u] = 0;
      live.erase(live.begin() + (long)k);
      model_used -= l.units * align;
    }
    REQUIRE(a.in_use() == model_used);
    REQUIRE(a.live() == live.size());
    // free ranges are maximal: count runs of free units in the model
    size_t runs = 0;
    uint64_t longest = 0, cur = 0;
    for (size_t u = 0; u < map.size(); ++u) {
      if (!map[u]) {
        if (cur == 0) ++runs;
        ++cur;
        if (cur > longest) longest = cur;
      } else {
        cur = 0;
      }
    }
    REQUIRE(a.free_ranges() == runs);
    REQUIRE(a.largest_free() == longest * align);
  }
  for (const Live& l : live) REQUIRE(a.free(l.off));
  REQUIRE(a.in_use() == 0 && a.free_ranges() == 1 && a.largest_free() == cap);
  REQUIRE(a.peak() <= cap && a.peak() > 0);
  REQUIRE(!a.free(12345));
  uint64_t off;
  REQUIRE(!a.alloc(cap + 1, &off));
  REQUIRE(a.alloc(cap, &off) && off == 0 && a.largest_free() == 0);

  // nearest-rank percentiles
  std::vector<double> v;
  for (int i = 100; i >= 1; --i) v.push_back(i);
  REQUIRE(dpt::percentile(v, 0.50) == 50.0);
  REQUIRE(dpt::percentile(v, 0.99) == 99.0);
  REQUIRE(dpt::percentile(v, 1.0) == 100.0);
  REQUIRE(dpt::percentile(v, 0.0) == 1.0);
  REQUIRE(dpt::percentile({}, 0.5) == 0.0);
  REQUIRE(dpt::percentile({7.0}, 0.99) == 7.0);
  std::printf("ok\n");
  return 0;
}
