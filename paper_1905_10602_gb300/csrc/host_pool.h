// Host thread pool of the factorization's parallel loops (csrc/factor.cpp).
// Standard C++ only, so that a CPU test can compile it on its own.
#pragma once

#include <atomic>
#include <condition_variable>
#include <exception>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace ifmm {

// Worker threads kept for the life of the process, so that the per-color
// parallel loops do not create and join threads each time (a few hundred loops
// per factorization).  One parallel region at a time: a caller that finds the
// pool busy (another thread's factorization) creates threads for its region.
class HostPool {
 public:
  static HostPool& get() {
    static HostPool* p = new HostPool();  // never destroyed: idle workers end with the process
    return *p;
  }
  // starts f(t) for t in [1, nth) on the workers (exceptions into ex[t]);
  // false, with nothing started, if another region is running
  bool start(int nth, const std::function<void(int)>* f, std::vector<std::exception_ptr>* ex) {
    if (busy_.exchange(true)) return false;
    {
      std::lock_guard<std::mutex> lk(mu_);
      while ((int)nworkers_ < nth - 1) {
        const int id = ++nworkers_;
        std::thread([this, id] { loop(id); }).detach();
      }
      job_ = f;
      exc_ = ex;
      nth_ = nth;
      pending_ = nth - 1;
      ++gen_;
    }
    cv_.notify_all();
    return true;
  }
  // waits for the started region and frees the pool
  void finish() {
    {
      std::unique_lock<std::mutex> lk(mu_);
      done_cv_.wait(lk, [this] { return pending_ == 0; });
      job_ = nullptr;
      exc_ = nullptr;
    }
    busy_.store(false);
  }

 private:
  void loop(int id) {
    unsigned long seen = 0;
    for (;;) {
      const std::function<void(int)>* f;
      std::vector<std::exception_ptr>* ex;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return gen_ != seen && id < nth_; });
        seen = gen_;
        f = job_;
        ex = exc_;
      }
      try {
        (*f)(id);
      } catch (...) {
        (*ex)[id] = std::current_exception();
      }
      std::lock_guard<std::mutex> lk(mu_);
      if (--pending_ == 0) done_cv_.notify_all();
    }
  }
  std::atomic<bool> busy_{false};
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  int nworkers_ = 0;
  const std::function<void(int)>* job_ = nullptr;
  std::vector<std::exception_ptr>* exc_ = nullptr;
  int nth_ = 0, pending_ = 0;
  unsigned long gen_ = 0;
};

// f(t) for t in [0, nth) on nth threads (t = 0 on the caller); the first
// exception any of them threw is rethrown after all have finished
template <class Fn>
void parallel_ranges(int nth, Fn&& f) {
  if (nth <= 1) {
    f(0);
    return;
  }
  std::vector<std::exception_ptr> ex(nth);
  const std::function<void(int)> job = [&](int t) { f(t); };
  HostPool& pool = HostPool::get();
  const bool pooled = pool.start(nth, &job, &ex);
  std::vector<std::thread> th;
  if (!pooled)
    for (int t = 1; t < nth; ++t)
      th.emplace_back([&, t] {
        try {
          f(t);
        } catch (...) {
          ex[t] = std::current_exception();
        }
      });
  try {
    f(0);
  } catch (...) {
    ex[0] = std::current_exception();
  }
  if (pooled)
    pool.finish();
  else
    for (auto& x : th) x.join();
  for (auto& e : ex)
    if (e) std::rethrow_exception(e);
}

}  // namespace ifmm
