// A process-wide pool of host threads for the data-parallel parts of the
// tree and block-index builder (per-DOF counting and filling, per-cell and
// per-front index lists).  The caller takes part in its own job; a second
// caller that finds the pool busy (concurrent factorizations of the batched
// API) runs its tasks itself, so nothing ever waits for another caller's job.
#pragma once
#include <cstdint>
#include <functional>

namespace hif {

// Threads of the pool, the caller included (1: no pool).
int host_threads();

// fn(t) for t = 0 .. ntasks-1, each exactly once, in any order and on any of
// the pool's threads; returns when all have returned.  If tasks throw, the
// others still run and the first exception is rethrown here afterwards.
void parallel_tasks(int ntasks, const std::function<void(int)>& fn);

// Tasks for `work` items: about one per `grain` items, at most host_threads().
int task_count(int64_t work, int64_t grain);

// [lo, hi) of task t when n items are cut into `tasks` contiguous ranges.
inline void task_range(int64_t n, int tasks, int t, int64_t& lo, int64_t& hi) {
  lo = n * t / tasks;
  hi = n * (t + 1) / tasks;
}

}  // namespace hif
