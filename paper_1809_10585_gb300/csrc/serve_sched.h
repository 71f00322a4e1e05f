// Scheduling policy of the continuously batched factorize/solve service (host only, no CUDA),
// used by the C ABI server in server.cpp.  It decides which waiting request starts in which
// slot, tracks device bytes against a budget, and keeps factors resident for later solves:
//
//  * Requests are served first come, first served, except that a solve whose factors are not
//    resident yet (their factorization is waiting or running), are busy with another request,
//    or are about to be replaced by a running factorization under the same key lets later
//    requests pass, and so does a factorization that would replace factors still in use.  A
//    solve for a key that no request will produce fails.
//  * A request starts when a slot is free and its device bytes fit the budget.  To make room,
//    least recently used resident factors that no running request uses are evicted.  If the
//    request still does not fit it waits for running requests to finish; if nothing runs, it
//    can never fit and fails.
//  * A finished factorization that asked to keep its factors becomes resident under its key
//    (replacing older factors under the same key); otherwise its bytes are released.
//
// Error codes are those of include/hodlr_qr.h.
#pragma once

#include <cstddef>
#include <cstdint>
#include <deque>
#include <functional>
#include <list>
#include <map>
#include <vector>

namespace hq {

class ServeScheduler {
 public:
  enum Kind { kFactor = 0, kSolve = 1 };
  enum State { kWaiting = 0, kRunning = 1, kDone = 2, kFailed = 3 };
  struct Request {
    long long id = 0;
    int kind = kFactor;
    long long key = -1;        // factor: keep under key (-1: do not keep); solve: resident key
    size_t bytes = 0;          // device bytes while running
    int state = kWaiting;
    int error = 0;             // HODLR_* code when failed
    int slot = -1;
  };
  struct Resident {
    size_t bytes = 0;
    long long busy_with = -1;  // id of the running request using the factors, or -1
  };

  ServeScheduler(int slots, size_t budget) : budget_(budget) {
    for (int s = 0; s < slots; ++s) free_.push_back(s);
  }

  long long submit(int kind, long long key, size_t bytes) {
    Request r;
    r.id = next_++;
    r.kind = kind;
    r.key = key;
    r.bytes = bytes;
    reqs_[r.id] = r;
    waiting_.push_back(r.id);
    return r.id;
  }

  // Start every request that can start now.  `start(request)` begins its work in request.slot
  // and returns HODLR_OK or an error code (the request then fails).  `evict(key)` releases
  // resident factors.  Returns the ids started.
  std::vector<long long> admit(const std::function<int(const Request&)>& start,
                               const std::function<void(long long)>& evict) {
    std::vector<long long> started;
    for (auto it = waiting_.begin(); it != waiting_.end();) {
      if (free_.empty()) break;
      Request& r = reqs_[*it];
      if (r.kind == kSolve) {
        auto res = resident_.find(r.key);
        if (res == resident_.end()) {
          if (producer_pending(r.key)) {
            ++it;
            continue;
          }
          fail(r, 7);                             // HODLR_ESTATE: nothing will produce the key
          it = waiting_.erase(it);
          continue;
        }
        // one request per resident matrix at a time; a solve waits for a running factorization
        // that will replace the factors under its key
        if (res->second.busy_with >= 0 || producer_running(r.key)) {
          ++it;
          continue;
        }
        res->second.busy_with = r.id;             // its own factors are never evicted for it
      } else if (r.key >= 0) {
        auto res = resident_.find(r.key);         // replaces factors in use: wait for them
        if (res != resident_.end() && res->second.busy_with >= 0) {
          ++it;
          continue;
        }
      }
      if (!make_room(r.bytes, evict)) {
        if (r.kind == kSolve) resident_[r.key].busy_with = -1;
        if (running_ > 0) break;                  // wait for memory to free up
        fail(r, 2);                               // HODLR_ENOMEM: can never fit
        it = waiting_.erase(it);
        continue;
      }
      r.slot = free_.front();
      free_.pop_front();
      used_ += r.bytes;
      r.state = kRunning;
      ++running_;
      if (r.kind == kSolve) touch(r.key);
      const int rc = start(r);
      if (rc != 0) {
        finish(r.id, rc, 0, evict);
      } else {
        started.push_back(r.id);
      }
      it = waiting_.erase(it);
    }
    return started;
  }

  // The request `id` finished (error = 0) or failed.  For a factorization that keeps its
  // factors, `resident_bytes` is what they hold from now on.
  void finish(long long id, int error, size_t resident_bytes, const std::function<void(long long)>& evict) {
    Request& r = reqs_[id];
    if (r.state != kRunning) return;
    used_ -= r.bytes;
    --running_;
    free_.push_back(r.slot);
    if (r.kind == kSolve) {
      auto res = resident_.find(r.key);
      if (res != resident_.end()) res->second.busy_with = -1;
    }
    if (error) {
      fail(r, error);
      return;
    }
    r.state = kDone;
    if (r.kind == kFactor && r.key >= 0) {
      auto old = resident_.find(r.key);
      if (old != resident_.end()) {
        used_ -= old->second.bytes;
        evict(r.key);
        resident_.erase(old);
        lru_.remove(r.key);
      }
      Resident res;
      res.bytes = resident_bytes;
      resident_[r.key] = res;
      lru_.push_back(r.key);
      used_ += resident_bytes;
    }
  }

  // Resident factors of `key` now hold `bytes` (e.g. a solve plan grew them).
  void resize_resident(long long key, size_t bytes) {
    auto res = resident_.find(key);
    if (res == resident_.end()) return;
    used_ += bytes;
    used_ -= res->second.bytes;
    res->second.bytes = bytes;
  }

  const Request* find(long long id) const {
    auto it = reqs_.find(id);
    return it == reqs_.end() ? nullptr : &it->second;
  }
  void forget(long long id) { reqs_.erase(id); }
  bool is_resident(long long key) const { return resident_.count(key) != 0; }
  size_t used() const { return used_; }
  int running() const { return running_; }
  int waiting() const { return (int)waiting_.size(); }
  int resident_count() const { return (int)resident_.size(); }
  std::vector<long long> resident_keys() const { return std::vector<long long>(lru_.begin(), lru_.end()); }

 private:
  bool producer_pending(long long key) const {
    for (auto& kv : reqs_) {
      const Request& q = kv.second;
      if (q.kind == kFactor && q.key == key && (q.state == kWaiting || q.state == kRunning)) return true;
    }
    return false;
  }
  bool producer_running(long long key) const {
    for (auto& kv : reqs_) {
      const Request& q = kv.second;
      if (q.kind == kFactor && q.key == key && q.state == kRunning) return true;
    }
    return false;
  }
  bool make_room(size_t need, const std::function<void(long long)>& evict) {
    while (used_ + need > budget_) {
      long long victim = -1;
      for (long long k : lru_)
        if (resident_[k].busy_with < 0) {
          victim = k;
          break;
        }
      if (victim < 0) return false;
      used_ -= resident_[victim].bytes;
      evict(victim);
      resident_.erase(victim);
      lru_.remove(victim);
    }
    return true;
  }
  void touch(long long key) {
    lru_.remove(key);
    lru_.push_back(key);
  }
  void fail(Request& r, int error) {
    r.state = kFailed;
    r.error = error;
  }

  size_t budget_;
  size_t used_ = 0;
  int running_ = 0;
  long long next_ = 1;
  std::deque<int> free_;
  std::list<long long> waiting_;
  std::map<long long, Request> reqs_;
  std::map<long long, Resident> resident_;
  std::list<long long> lru_;                    // resident keys, least recently used first
};

}  // namespace hq
