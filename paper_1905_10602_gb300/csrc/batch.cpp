// Many independent problems at once: every worker thread owns a CUDA stream
// and takes the next problem from a shared counter, so the kernels of
// different problems interleave on the GPU and one problem's host-side work
// and per-color synchronisation hide behind the others' kernels.
#include <atomic>
#include <mutex>
#include <thread>

#include "fact.h"

namespace {

struct StreamPool {
  std::vector<cudaStream_t> s;
  explicit StreamPool(int n) {
    s.resize(n, nullptr);
    for (auto& x : s)
      if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess)
        throw ifmm::Error(IFMM_ECUDA, "cudaStreamCreate failed");
  }
  ~StreamPool() {
    for (auto x : s)
      if (x) cudaStreamDestroy(x);
  }
};

template <class F>
ifmm_status run_workers(int nprob, int nworkers, F&& body) {
  const int nw = std::max(1, std::min(nworkers > 0 ? nworkers : 8, nprob));
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    ifmm::set_last_error("no CUDA device");
    return IFMM_ECUDA;
  }
  std::atomic<int> next{0};
  std::mutex mu;
  ifmm_status first = IFMM_OK;
  std::string msg;
  try {
    StreamPool pool(nw);
    std::vector<std::thread> th;
    for (int w = 0; w < nw; ++w)
      th.emplace_back([&, w] {
        cudaSetDevice(dev);
        if (nw > 1) ifmm::host_thread_cap() = 1;  // the workers already share the host
        for (;;) {
          const int i = next.fetch_add(1);
          if (i >= nprob) break;
          ifmm_status st = body(i, pool.s[w]);
          if (st != IFMM_OK) {
            std::lock_guard<std::mutex> lock(mu);
            if (first == IFMM_OK) {
              first = st;
              msg = "problem " + std::to_string(i) + ": " + ifmm_last_error();
            }
          }
        }
      });
    for (auto& t : th) t.join();
  } catch (const ifmm::Error& e) {
    ifmm::set_last_error(e.what());
    return e.code;
  }
  if (first != IFMM_OK) ifmm::set_last_error(msg);
  return first;
}

}  // namespace

extern "C" {

ifmm_status ifmm_factor_batched(const ifmm_tree* const* trees, const ifmm_kernel* kernels, const ifmm_opts* opts,
                                int nprob, int nworkers, ifmm_fact** out) {
  if (!trees || !kernels || !opts || !out || nprob < 0) {
    ifmm::set_last_error("bad argument");
    return IFMM_EINVAL;
  }
  for (int i = 0; i < nprob; ++i) out[i] = nullptr;
  // device copies of the trees first (one thread): they are shared state
  for (int i = 0; i < nprob; ++i) {
    try {
      IFMM_REQUIRE(trees[i] != nullptr, IFMM_EINVAL, "NULL tree");
      const_cast<ifmm_tree*>(trees[i])->ensure_device();
    } catch (const ifmm::Error& e) {
      ifmm::set_last_error(e.what());
      return e.code;
    }
  }
  const ifmm_status st = run_workers(nprob, nworkers, [&](int i, cudaStream_t s) {
    return ifmm_factor(trees[i], &kernels[i], &opts[i], (void*)s, &out[i]);
  });
  if (st != IFMM_OK)
    for (int i = 0; i < nprob; ++i) {
      ifmm_fact_free(out[i]);
      out[i] = nullptr;
    }
  return st;
}

ifmm_status bem_gmres_batched(const ifmm_tree* const* trees, const ifmm_kernel* kernels, const ifmm_fact* const* precond,
                              const double* const* b, double* const* x, int nprob, int restart, double tol, int maxit,
                              int* iters, double* relres, int nworkers) {
  if (!trees || !kernels || !b || !x || nprob < 0) {
    ifmm::set_last_error("bad argument");
    return IFMM_EINVAL;
  }
  for (int i = 0; i < nprob; ++i) {
    try {
      IFMM_REQUIRE(trees[i] != nullptr, IFMM_EINVAL, "NULL tree");
      const_cast<ifmm_tree*>(trees[i])->ensure_device();
    } catch (const ifmm::Error& e) {
      ifmm::set_last_error(e.what());
      return e.code;
    }
  }
  return run_workers(nprob, nworkers, [&](int i, cudaStream_t s) {
    return bem_gmres(trees[i], &kernels[i], precond ? precond[i] : nullptr, b[i], x[i], restart, tol, maxit,
                     iters ? &iters[i] : nullptr, relres ? &relres[i] : nullptr, (void*)s);
  });
}

}  // extern "C"
