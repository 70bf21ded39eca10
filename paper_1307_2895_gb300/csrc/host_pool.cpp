// Process-wide host thread pool (see host_pool.h).
#include "host_pool.h"

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <exception>
#include <mutex>
#include <thread>
#include <vector>

namespace hif {
namespace {

// One parallel_tasks call: lives on the caller's stack; a worker touches it
// only while registered (users > 0), and the caller returns only after every
// task has run and every registered worker has left.  A task that throws
// still counts as run; the first exception is kept and rethrown to the
// caller once the job is over.
struct Job {
  const std::function<void(int)>* fn;
  int ntasks;
  std::mutex* m;   // the pool mutex
  std::atomic<int> next{0};
  int done = 0;    // tasks finished (guarded by the pool mutex)
  int users = 0;   // workers registered on the job (guarded by the pool mutex)
  std::exception_ptr error;   // first exception of a task (guarded by the pool mutex)
  int run_some() {
    int mine = 0;
    for (int t; (t = next.fetch_add(1)) < ntasks; ++mine) {
      try {
        (*fn)(t);
      } catch (...) {
        std::lock_guard<std::mutex> g(*m);
        if (!error) error = std::current_exception();
      }
    }
    return mine;
  }
};

class Pool {
 public:
  explicit Pool(int nthreads) {
    try {
      for (int i = 1; i < nthreads; ++i) workers_.emplace_back([this] { work(); });
    } catch (const std::exception&) {
      // a thread that cannot start: the pool runs with those that did
    }
  }
  int size() const { return (int)workers_.size() + 1; }

  void run(int ntasks, const std::function<void(int)>& fn) {
    std::unique_lock<std::mutex> job(busy_, std::try_to_lock);
    if (!job.owns_lock() || workers_.empty() || ntasks <= 1) {
      for (int t = 0; t < ntasks; ++t) fn(t);
      return;
    }
    Job j;
    j.fn = &fn;
    j.ntasks = ntasks;
    j.m = &m_;
    {
      std::lock_guard<std::mutex> g(m_);
      cur_ = &j;
      ++gen_;
    }
    cv_work_.notify_all();
    const int mine = j.run_some();
    std::unique_lock<std::mutex> lk(m_);
    j.done += mine;
    cur_ = nullptr;   // late wakers find no job
    cv_done_.wait(lk, [&] { return j.done == j.ntasks && j.users == 0; });
    if (j.error) std::rethrow_exception(j.error);
  }

 private:
  void work() {
    uint64_t seen = 0;
    std::unique_lock<std::mutex> lk(m_);
    for (;;) {
      cv_work_.wait(lk, [&] { return cur_ != nullptr && gen_ != seen; });
      seen = gen_;
      Job* j = cur_;
      ++j->users;
      lk.unlock();
      const int mine = j->run_some();
      lk.lock();
      j->done += mine;
      --j->users;
      if (j->done == j->ntasks && j->users == 0) cv_done_.notify_all();
    }
  }

  std::vector<std::thread> workers_;
  std::mutex busy_;   // one job at a time
  std::mutex m_;
  std::condition_variable cv_work_, cv_done_;
  Job* cur_ = nullptr;
  uint64_t gen_ = 0;
};

Pool& pool() {
  // never destroyed: the workers sleep until the process ends
  static Pool* p = new Pool(std::max(1, std::min(8, (int)std::thread::hardware_concurrency())));
  return *p;
}

}  // namespace

int host_threads() { return pool().size(); }

void parallel_tasks(int ntasks, const std::function<void(int)>& fn) { pool().run(ntasks, fn); }

int task_count(int64_t work, int64_t grain) {
  const int64_t t = work / std::max<int64_t>(grain, 1);
  return (int)std::max<int64_t>(1, std::min<int64_t>(t, host_threads()));
}

}  // namespace hif
