// Host-side retry rule for batches of problems that share one device: a problem whose attempt
// reports out-of-memory while other problems hold device memory waits until one of them finishes
// and runs again.  When every other problem of the pool is waiting as well (nobody can finish),
// the waiting problems run again one at a time -- alone on the device -- and those results stand;
// a problem that is alone from the start keeps its out-of-memory result.  Plain C++ (no CUDA), so
// the rule is tested on the host with a simulated memory budget.
#pragma once
#include <condition_variable>
#include <mutex>

namespace nh {

class MemoryRetry {
 public:
  // a problem enters / leaves the pool
  void begin() {
    std::lock_guard<std::mutex> lk(mu_);
    active_++;
  }
  void end() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      active_--;
      finished_++;
    }
    cv_.notify_all();
  }
  // attempt() until it returns something other than `oom`, by the rule above; returns the last status
  template <typename A> int run(A&& attempt, int oom) {
    int s = attempt();
    while (s == oom) {
      std::unique_lock<std::mutex> lk(mu_);
      if (active_ <= 1) break;            // alone on the device: the failure stands
      const long seen = finished_;
      active_--;
      cv_.notify_all();                   // the others may now all be waiting
      cv_.wait(lk, [&] { return finished_ > seen || active_ == 0; });
      const bool progress = finished_ > seen;
      active_++;
      lk.unlock();
      if (progress) {
        s = attempt();
        continue;
      }
      // every other problem was waiting too: run again one at a time; this result stands
      std::lock_guard<std::mutex> one(alone_);
      s = attempt();
      break;
    }
    return s;
  }

 private:
  std::mutex mu_, alone_;
  std::condition_variable cv_;
  int active_ = 0;
  long finished_ = 0;
};

}  // namespace nh
