// Stand-alone check of the factorization's host thread pool (csrc/host_pool.h),
// compiled and run by tests/test_host_pool.py: every index of a region runs
// exactly once, exceptions come back to the caller after the whole region has
// finished, the pool stays usable after one, and two callers at once (the pool
// busy for one of them) both complete.
#include <chrono>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "host_pool.h"

using ifmm::parallel_ranges;

static int fails = 0;
#define CHECK(cond, what)                     \
  do {                                        \
    if (!(cond)) {                            \
      std::printf("FAIL: %s\n", what);        \
      ++fails;                                \
    }                                         \
  } while (0)

// one caller's regions of 1..16 threads; each index records its own visit
static void regions(int reps, int seed) {
  for (int rep = 0; rep < reps; ++rep)
    for (int nth = 1; nth <= 16; ++nth) {
      std::vector<int> hits(nth, 0);
      std::vector<long> part(nth, 0);
      const int n = 1000 + seed + rep;
      parallel_ranges(nth, [&](int t) {
        hits[t] += 1;
        const int i0 = (int)((long)n * t / nth), i1 = (int)((long)n * (t + 1) / nth);
        long s = 0;
        for (int i = i0; i < i1; ++i) s += i;
        part[t] = s;
      });
      long total = 0;
      for (int t = 0; t < nth; ++t) {
        CHECK(hits[t] == 1, "every index of a region runs exactly once");
        total += part[t];
      }
      CHECK(total == (long)n * (n - 1) / 2, "the ranges cover the items once");
    }
}

int main() {
  regions(50, 0);

  // an exception from a worker index and one from the caller's index: the
  // first in index order comes back, after every other index has finished
  for (int thrower : {7, 0}) {
    std::vector<int> hits(8, 0);
    bool caught = false;
    try {
      parallel_ranges(8, [&](int t) {
        if (t == thrower || t == 5) throw std::runtime_error(t == thrower ? "first" : "second");
        std::this_thread::sleep_for(std::chrono::milliseconds(2));
        hits[t] = 1;
      });
    } catch (const std::runtime_error& e) {
      caught = true;
      const char* want = thrower < 5 ? "first" : "second";
      CHECK(std::string(e.what()) == want, "the exception of the lowest index is rethrown");
      for (int t = 0; t < 8; ++t)
        if (t != thrower && t != 5) CHECK(hits[t] == 1, "the region finished before the rethrow");
    }
    CHECK(caught, "an exception in a region reaches the caller");
  }
  regions(5, 1);  // the pool is usable after an exception

  // two callers at once: one gets the pool, the other its own threads
  std::thread a([] { regions(20, 2); });
  std::thread b([] { regions(20, 3); });
  a.join();
  b.join();

  if (fails == 0) std::printf("host_pool ok\n");
  return fails ? 1 : 0;
}
