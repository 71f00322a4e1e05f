// CPU test of the service's scheduling policy (serve_sched.h): admission order, deferral of
// solves whose factors are not ready, slot reuse, the memory budget with LRU eviction, and the
// failure codes.  The "device work" is a fake: start() only records what was started.
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "serve_sched.h"

using hq::ServeScheduler;
static int failures = 0;
#define CHECK(c)                                                   \
  do {                                                             \
    if (!(c)) {                                                    \
      std::printf("FAIL %s:%d: %s\n", __FILE__, __LINE__, #c);     \
      ++failures;                                                  \
    }                                                              \
  } while (0)

struct Fake {
  std::vector<long long> started;
  std::vector<long long> evicted;
  std::vector<int> slots;
  int fail_id = -1, fail_code = 0;
  std::function<int(const ServeScheduler::Request&)> start() {
    return [this](const ServeScheduler::Request& r) {
      started.push_back(r.id);
      slots.push_back(r.slot);
      return r.id == fail_id ? fail_code : 0;
    };
  }
  std::function<void(long long)> evict() {
    return [this](long long k) { evicted.push_back(k); };
  }
};

static void fifo_and_slot_reuse() {
  ServeScheduler S(2, 100);
  Fake f;
  long long a = S.submit(ServeScheduler::kFactor, -1, 10), b = S.submit(ServeScheduler::kFactor, -1, 10),
            c = S.submit(ServeScheduler::kFactor, -1, 10);
  S.admit(f.start(), f.evict());
  CHECK(f.started == std::vector<long long>({a, b}));
  CHECK(S.running() == 2 && S.waiting() == 1 && S.used() == 20);
  S.finish(a, 0, 0, f.evict());
  S.admit(f.start(), f.evict());
  CHECK(f.started.size() == 3 && f.started[2] == c && f.slots[2] == f.slots[0]);   // a's slot
  CHECK(S.find(a)->state == ServeScheduler::kDone && S.used() == 20);
}

static void solve_waits_for_its_factors() {
  ServeScheduler S(3, 1000);
  Fake f;
  long long fk = S.submit(ServeScheduler::kFactor, 5, 10);
  long long s1 = S.submit(ServeScheduler::kSolve, 5, 3);
  long long g = S.submit(ServeScheduler::kFactor, -1, 10);
  S.admit(f.start(), f.evict());
  CHECK(f.started == std::vector<long long>({fk, g}));            // the solve let g pass
  S.finish(fk, 0, 20, f.evict());
  CHECK(S.is_resident(5) && S.used() == 10 + 20);
  S.admit(f.start(), f.evict());
  CHECK(f.started.back() == s1);
  // a second solve on the same factors waits while the first runs
  long long s2 = S.submit(ServeScheduler::kSolve, 5, 3);
  S.admit(f.start(), f.evict());
  CHECK(f.started.back() == s1 && S.find(s2)->state == ServeScheduler::kWaiting);
  S.finish(s1, 0, 0, f.evict());
  S.admit(f.start(), f.evict());
  CHECK(f.started.back() == s2);
}

static void unknown_key_fails() {
  ServeScheduler S(2, 100);
  Fake f;
  long long s = S.submit(ServeScheduler::kSolve, 42, 1);
  S.admit(f.start(), f.evict());
  CHECK(f.started.empty() && S.find(s)->state == ServeScheduler::kFailed && S.find(s)->error == 7);
}

static void budget_evicts_lru_then_waits_then_fails() {
  ServeScheduler S(4, 100);
  Fake f;
  long long k1 = S.submit(ServeScheduler::kFactor, 1, 30), k2 = S.submit(ServeScheduler::kFactor, 2, 30);
  S.admit(f.start(), f.evict());
  S.finish(k1, 0, 40, f.evict());
  S.finish(k2, 0, 40, f.evict());
  CHECK(S.used() == 80 && S.resident_count() == 2);
  // a solve on key 1 makes 2 the least recently used
  long long s1 = S.submit(ServeScheduler::kSolve, 1, 5);
  S.admit(f.start(), f.evict());
  S.finish(s1, 0, 0, f.evict());
  long long big = S.submit(ServeScheduler::kFactor, -1, 50);      // needs key 2 evicted
  S.admit(f.start(), f.evict());
  CHECK(f.evicted == std::vector<long long>({2}) && S.find(big)->state == ServeScheduler::kRunning);
  CHECK(S.used() == 40 + 50);
  long long wait = S.submit(ServeScheduler::kFactor, -1, 60);     // fits only after big finishes
  S.admit(f.start(), f.evict());
  CHECK(S.find(wait)->state == ServeScheduler::kWaiting);         // key 1 evicted, still no room
  CHECK(f.evicted == std::vector<long long>({2, 1}));
  S.finish(big, 0, 0, f.evict());
  S.admit(f.start(), f.evict());
  CHECK(S.find(wait)->state == ServeScheduler::kRunning);
  S.finish(wait, 0, 0, f.evict());
  long long never = S.submit(ServeScheduler::kFactor, -1, 101);
  S.admit(f.start(), f.evict());
  CHECK(S.find(never)->state == ServeScheduler::kFailed && S.find(never)->error == 2);
  CHECK(S.used() == 0 && S.running() == 0);
}

static void solve_never_evicts_its_own_factors() {
  ServeScheduler S(2, 100);
  Fake f;
  long long k = S.submit(ServeScheduler::kFactor, 7, 10);
  S.admit(f.start(), f.evict());
  S.finish(k, 0, 90, f.evict());
  long long s = S.submit(ServeScheduler::kSolve, 7, 20);          // 90 + 20 > 100
  S.admit(f.start(), f.evict());
  CHECK(f.evicted.empty() && S.find(s)->state == ServeScheduler::kFailed && S.find(s)->error == 2);
  CHECK(S.is_resident(7));
}

static void replacement_waits_for_users() {
  ServeScheduler S(3, 1000);
  Fake f;
  long long k = S.submit(ServeScheduler::kFactor, 3, 10);
  S.admit(f.start(), f.evict());
  S.finish(k, 0, 20, f.evict());
  long long s = S.submit(ServeScheduler::kSolve, 3, 1);
  long long r = S.submit(ServeScheduler::kFactor, 3, 10);         // replaces key 3
  S.admit(f.start(), f.evict());
  CHECK(S.find(s)->state == ServeScheduler::kRunning && S.find(r)->state == ServeScheduler::kWaiting);
  long long s2 = S.submit(ServeScheduler::kSolve, 3, 1);          // must see the new factors
  S.finish(s, 0, 0, f.evict());
  S.admit(f.start(), f.evict());
  CHECK(S.find(r)->state == ServeScheduler::kRunning && S.find(s2)->state == ServeScheduler::kWaiting);
  S.finish(r, 0, 25, f.evict());
  CHECK(f.evicted == std::vector<long long>({3}) && S.is_resident(3) && S.used() == 25);
  S.admit(f.start(), f.evict());
  CHECK(S.find(s2)->state == ServeScheduler::kRunning);
}

static void start_failure_frees_the_slot() {
  ServeScheduler S(1, 100);
  Fake f;
  long long a = S.submit(ServeScheduler::kFactor, -1, 10), b = S.submit(ServeScheduler::kFactor, -1, 10);
  f.fail_id = (int)a;
  f.fail_code = 6;
  S.admit(f.start(), f.evict());
  CHECK(S.find(a)->state == ServeScheduler::kFailed && S.find(a)->error == 6);
  CHECK(S.find(b)->state == ServeScheduler::kRunning && S.used() == 10);
}

int main() {
  fifo_and_slot_reuse();
  solve_waits_for_its_factors();
  unknown_key_fails();
  budget_evicts_lru_then_waits_then_fails();
  solve_never_evicts_its_own_factors();
  replacement_waits_for_users();
  start_failure_frees_the_slot();
  if (failures) return 1;
  std::printf("serve_sched: all checks passed\n");
  return 0;
}
