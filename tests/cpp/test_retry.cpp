// Host test of the batch retry rule (csrc/retry.h) with a simulated device-memory budget: tasks take
// `need` units for a short while; an attempt that does not fit reports out-of-memory.  Prints one
// line per scenario: the final status of every task.  The test driver checks the lines.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <thread>
#include <vector>

#include "retry.h"

namespace {
constexpr int OK = 0, OOM = 2;

struct Budget {
  std::atomic<int> free_units;
  explicit Budget(int u) : free_units(u) {}
  bool take(int n) {
    int cur = free_units.load();
    while (cur >= n)
      if (free_units.compare_exchange_weak(cur, cur - n)) return true;
    return false;
  }
  void give(int n) { free_units += n; }
};

// run `need.size()` tasks on `threads` threads; returns each task's status
std::vector<int> scenario(int budget, const std::vector<int>& need, int threads, int hold_ms) {
  Budget b(budget);
  nh::MemoryRetry retry;
  std::vector<int> st(need.size(), -1);
  std::atomic<int> next{0};
  auto work = [&] {
    for (int i = next++; i < (int)need.size(); i = next++) {
      retry.begin();
      st[i] = retry.run(
          [&]() -> int {
            // a first allocation, then the rest after a while (both must fit)
            const int half = need[i] / 2;
            if (!b.take(half)) return OOM;
            std::this_thread::sleep_for(std::chrono::milliseconds(hold_ms));
            if (!b.take(need[i] - half)) {
              b.give(half);
              return OOM;
            }
            std::this_thread::sleep_for(std::chrono::milliseconds(hold_ms));
            b.give(need[i]);
            return OK;
          },
          OOM);
      retry.end();
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t) pool.emplace_back(work);
  for (auto& t : pool) t.join();
  return st;
}

void print(const char* name, const std::vector<int>& st) {
  std::printf("%s", name);
  for (int s : st) std::printf(" %d", s);
  std::printf("\n");
}
}  // namespace

int main() {
  // every task fits alone, no two fit together: all must finish OK (no livelock)
  print("pairwise_conflict", scenario(10, {6, 6, 6, 6, 6, 6}, 4, 5));
  // plenty of memory: all OK
  print("ample", scenario(100, {10, 10, 10, 10}, 4, 2));
  // one task needs more than the device has: it alone fails, the others finish
  print("too_big", scenario(10, {6, 12, 6, 4}, 3, 3));
  // a single thread: a task that does not fit fails at once (nobody to wait for)
  print("single_thread", scenario(10, {12, 4}, 1, 1));
  return 0;
}
