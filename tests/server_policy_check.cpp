// Checks of the serving loop's admission policy (rd_server_policy.h), built
// and run by test_server_policy.py with the host compiler (no GPU).
#include <stdio.h>
#include <stdlib.h>

#include "rd_server_policy.h"

#define CHECK(c)                                                   \
  do {                                                             \
    if (!(c)) {                                                    \
      fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #c); \
      exit(1);                                                     \
    }                                                              \
  } while (0)

using rdk::AdmissionPolicy;

int main() {
  // a new key is admitted and loading; a second request waits until loaded
  {
    AdmissionPolicy p(100);
    auto d = p.admit(1, 40);
    CHECK(d.admitted && !d.hit && d.evicted.empty() && p.used() == 40);
    CHECK(!p.admit(1, 40).admitted);  // still loading
    p.mark_loaded(1);
    auto h = p.admit(1, 40);
    CHECK(h.admitted && h.hit && p.pins(1) == 2 && p.used() == 40);
    p.release(1, 40);
    p.release(1, 40);
    CHECK(p.pins(1) == 0 && p.is_resident(1));
  }
  // eviction: least recently used unpinned entries go first
  {
    AdmissionPolicy p(100);
    for (uint64_t k = 1; k <= 3; k++) {
      CHECK(p.admit(k, 30).admitted);
      p.mark_loaded(k);
      p.release(k, 30);
    }
    CHECK(p.admit(2, 30).hit);  // 2 is now the most recently used (and pinned)
    p.release(2, 30);
    auto d = p.admit(4, 50);    // needs 40 more: evict 1 (oldest), then 3
    CHECK(d.admitted && d.evicted.size() == 2 && d.evicted[0] == 1 && d.evicted[1] == 3);
    CHECK(p.used() == 80 && p.is_resident(2) && p.is_resident(4) && !p.is_resident(1));
    CHECK(p.evictions() == 2);
  }
  // pinned and loading entries are never evicted; the request waits
  {
    AdmissionPolicy p(100);
    CHECK(p.admit(1, 60).admitted);  // loading, pinned
    CHECK(!p.admit(2, 50).admitted);
    p.mark_loaded(1);
    CHECK(!p.admit(2, 50).admitted);  // still pinned
    p.release(1, 60);
    auto d = p.admit(2, 50);
    CHECK(d.admitted && d.evicted.size() == 1 && d.evicted[0] == 1 && p.used() == 50);
  }
  // transient requests hold bytes only while they run
  {
    AdmissionPolicy p(100);
    CHECK(p.admit(0, 70).admitted && p.used() == 70);
    CHECK(!p.admit(0, 40).admitted);
    p.release(0, 70);
    CHECK(p.used() == 0 && p.resident_count() == 0);
    CHECK(p.admit(0, 100).admitted);
    CHECK(!p.fits_at_all(101));
  }
  // a failed load drops its entry
  {
    AdmissionPolicy p(100);
    CHECK(p.admit(5, 80).admitted);
    p.drop(5);
    CHECK(p.used() == 0 && !p.is_resident(5));
  }
  // no bound when the budget is 0
  {
    AdmissionPolicy p(0);
    for (uint64_t k = 1; k <= 100; k++) CHECK(p.admit(k, 1ull << 40).admitted);
    CHECK(p.evictions() == 0 && p.resident_count() == 100);
  }
  // a request that cannot fit even after evicting everything unpinned waits
  // without evicting anything
  {
    AdmissionPolicy p(100);
    CHECK(p.admit(1, 50).admitted);
    p.mark_loaded(1);  // pinned
    CHECK(p.admit(2, 30).admitted);
    p.mark_loaded(2);
    p.release(2, 30);  // unpinned, resident
    auto d = p.admit(3, 60);  // needs 40 more; only 30 evictable
    CHECK(!d.admitted && p.is_resident(2) && p.evictions() == 0);
  }
  printf("ok\n");
  return 0;
}
