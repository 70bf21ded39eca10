// Test harness (CPU, no CUDA): the host thread pool (host_pool.cpp) when
// tasks throw.  Every task must still run once, the caller must receive one
// of the exceptions after all tasks are over, and the pool must stay usable.
// Exits 0 when all checks hold, else the number of the failed check.
#include <atomic>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "host_pool.h"

using namespace hif;

int main() {
  if (host_threads() < 1) return 1;
  for (int round = 0; round < 200; ++round) {
    const int n = 257 + round;
    std::vector<std::atomic<int>> runs(n);
    for (auto& r : runs) r = 0;
    bool caught = false;
    try {
      parallel_tasks(n, [&](int t) {
        runs[t].fetch_add(1);
        if (t % 97 == round % 97) throw std::runtime_error("task " + std::to_string(t));
      });
    } catch (const std::runtime_error& e) {
      caught = std::string(e.what()).rfind("task ", 0) == 0;
    }
    if (!caught) return 2;
    for (auto& r : runs)
      if (r.load() != 1) return 3;
    // the pool still works, with no exception
    std::atomic<long> sum{0};
    parallel_tasks(n, [&](int t) { sum.fetch_add(t); });
    if (sum.load() != (long)n * (n - 1) / 2) return 4;
  }
  // a single task (serial path) that throws
  try {
    parallel_tasks(1, [](int) { throw std::logic_error("serial"); });
    return 5;
  } catch (const std::logic_error&) {
  }
  std::printf("ok %d threads\n", host_threads());
  return 0;
}
