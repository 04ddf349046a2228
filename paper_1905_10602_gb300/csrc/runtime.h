// Device memory arenas and batched-launch helpers.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.h"
#include "descs.h"

namespace ifmm {

#define CK(x)                                                                                \
  do {                                                                                       \
    cudaError_t e_ = (x);                                                                    \
    if (e_ != cudaSuccess)                                                                   \
      throw ::ifmm::Error(e_ == cudaErrorMemoryAllocation ? IFMM_ENOMEM : IFMM_ECUDA,        \
                          std::string(#x) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

// Optional host-side bounds check of every launch (IFMM_CHECK=1): allocations
// are registered, and each descriptor's address range must fall inside one of
// them before the kernel is launched.
struct Registry {
  bool on = false;
  std::map<uintptr_t, uintptr_t> iv;  // start -> end
  std::mutex mu;
  void add(const void* p, size_t bytes) {
    if (!on) return;
    std::lock_guard<std::mutex> lock(mu);
    iv[(uintptr_t)p] = (uintptr_t)p + bytes;
  }
  void remove_range(const void* lo, size_t bytes) {
    if (!on) return;
    std::lock_guard<std::mutex> lock(mu);
    auto a = iv.lower_bound((uintptr_t)lo);
    auto b = iv.lower_bound((uintptr_t)lo + bytes);
    iv.erase(a, b);
  }
  bool contains(const void* p, size_t bytes) {
    if (!on) return true;
    std::lock_guard<std::mutex> lock(mu);
    uintptr_t lo = (uintptr_t)p, hi = lo + bytes;
    auto it = iv.upper_bound(lo);
    if (it == iv.begin()) return false;
    --it;
    return it->first <= lo && hi <= it->second;
  }
};
Registry& registry();

// Optional poisoning of new arena memory (IFMM_POISON=1): every allocation is
// filled with the byte 0x7e (about 1e301 as a double, 2e38 as a float), so that
// a kernel reading memory nothing wrote turns its results into overflow.
// Debugging aid; it synchronizes the device on every allocation.
bool poison_on();
void poison_fill(void* p, size_t bytes);

// Bump allocator over cudaMalloc'd chunks.  reset() makes the memory reusable;
// callers only reset at points where all earlier work on the stream that uses
// the memory has been ordered before later work (one stream) .
struct DeviceArena {
  struct Chunk {
    char* p;
    size_t size;
  };
  std::vector<Chunk> chunks;
  size_t ci = 0, off = 0;
  size_t min_chunk = (size_t)256 << 20;
  size_t high = 0;
  void* alloc_bytes(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    while (ci < chunks.size()) {
      if (off + bytes <= chunks[ci].size) {
        void* r = chunks[ci].p + off;
        off += bytes;
        registry().add(r, bytes);
        if (poison_on()) poison_fill(r, bytes);
        return r;
      }
      ++ci;
      off = 0;
    }
    size_t sz = std::max(min_chunk, bytes);
    void* p = nullptr;
    CK(cudaMalloc(&p, sz));
    chunks.push_back({(char*)p, sz});
    ci = chunks.size() - 1;
    off = bytes;
    high += sz;
    registry().add(p, bytes);
    if (poison_on()) poison_fill(p, bytes);
    return p;
  }
  double* alloc(size_t n) { return (double*)alloc_bytes(n * sizeof(double)); }
  void reset() {
    for (auto& c : chunks) registry().remove_range(c.p, c.size);
    ci = 0;
    off = 0;
  }
  void release() {
    for (auto& c : chunks) registry().remove_range(c.p, c.size);
    for (auto& c : chunks) cudaFree(c.p);
    chunks.clear();
    ci = off = 0;
  }
  void swap(DeviceArena& o) {
    std::swap(chunks, o.chunks);
    std::swap(ci, o.ci);
    std::swap(off, o.off);
    std::swap(min_chunk, o.min_chunk);
    std::swap(high, o.high);
  }
  DeviceArena() = default;
  DeviceArena(const DeviceArena&) = delete;
  DeviceArena& operator=(const DeviceArena&) = delete;
  ~DeviceArena() { release(); }
};

// Pinned host staging + device buffer for launch descriptors.  push() copies a
// vector into pinned memory and enqueues its upload; reset() only after a
// stream synchronization.
struct DescStage {
  cudaStream_t stream = nullptr;
  std::vector<std::pair<char*, size_t>> host;  // pinned chunks
  size_t hci = 0, hoff = 0;
  DeviceArena dev;
  DescStage() { dev.min_chunk = (size_t)64 << 20; }
  void* host_alloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    while (hci < host.size()) {
      if (hoff + bytes <= host[hci].second) {
        void* r = host[hci].first + hoff;
        hoff += bytes;
        return r;
      }
      ++hci;
      hoff = 0;
    }
    size_t sz = std::max<size_t>((size_t)64 << 20, bytes);
    void* p = nullptr;
    CK(cudaMallocHost(&p, sz));
    host.push_back({(char*)p, sz});
    hci = host.size() - 1;
    hoff = bytes;
    return p;
  }
  template <class T>
  T* push(const T* data, size_t n) {
    if (n == 0) return nullptr;
    T* h = (T*)host_alloc(n * sizeof(T));
    memcpy(h, data, n * sizeof(T));
    return upload(h, n);
  }
  // enqueues the upload of n elements that the caller wrote into memory from
  // host_alloc (written completely before this call)
  template <class T>
  T* upload(const T* h, size_t n) {
    if (n == 0) return nullptr;
    void* d = dev.alloc_bytes(n * sizeof(T));
    CK(cudaMemcpyAsync(d, h, n * sizeof(T), cudaMemcpyHostToDevice, stream));
    return (T*)d;
  }
  template <class T>
  T* push(const std::vector<T>& v) {
    return push(v.data(), v.size());
  }
  void reset() {
    hci = hoff = 0;
    dev.reset();
  }
  void release() {
    for (auto& h : host) cudaFreeHost(h.first);
    host.clear();
    dev.release();
  }
  ~DescStage() { release(); }
};

// P16: FP32 arithmetic on bfloat16-rounded operands (GEMM launches only)
enum Prec { P64 = 0, P32 = 1, P16 = 2 };

// Per-kernel launch counts and (when enabled) CUDA-event durations measured on
// the launching stream around every launch.
enum KernelKind {
  KK_COPY = 0, KK_GEMM64, KK_GEMM32, KK_INV, KK_QR64, KK_QR32, KK_SVD64, KK_SVD32, KK_GEMV, KK_GEMV_SUM, KK_P2P,
  KK_INTERP, KK_TABLES, KK_MATVEC, KK_PERM, KK_GJ_BIG, KK_SOLVE_GRAPH, KK_QRG64, KK_QRG32, KK_QRC64, KK_QRC32, KK_ALL, KK_COUNT
};
struct Profiler {
  bool timing = false;
  std::vector<std::pair<int, long>> pending_tags;
  long launches[KK_COUNT] = {0};
  long events_kernels[KK_COUNT] = {0};
  double ms[KK_COUNT] = {0};
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  cudaEvent_t begin(int kind, cudaStream_t s, long count = 1);
  void end(int kind, cudaStream_t s, cudaEvent_t b);
  void collect();  // synchronizes pending events and accumulates
  void collect_locked();
  void count(int kind, long n);
  void reset();
};
Profiler& profiler();
// per-thread cap on the host threads a factorization may use for its own
// loops (0: as many as useful; batch workers set 1, as they already share the host)
int& host_thread_cap();
// per-thread tags of the per-launch log: level being factored, batch size
int& prof_level_tag();
long& prof_batch_tag();
const char* kernel_kind_name(int k);

void launch_copy(DescStage& st, const std::vector<CopyDesc>& v);
// launch_copy splits its list into the copies of at most 1024 elements (one
// warp each) and the larger ones (one CTA each)
inline bool copy_is_small(const CopyDesc& x) { return (long)x.rows * x.cols <= 1024; }
// The same launches for descriptors that the caller already wrote, sorted, into
// memory from st.host_alloc: the ns copies with copy_is_small first, then the nb
// others.
void launch_copy_sorted(DescStage& st, const CopyDesc* h, size_t ns, size_t nb);
void launch_gemm(DescStage& st, const std::vector<GemmDesc>& v, int prec);
void launch_inv(DescStage& st, const std::vector<InvDesc>& v);
void launch_qr(DescStage& st, const std::vector<QrDesc>& v, int prec);
void launch_gemv(DescStage& st, const std::vector<GemvDesc>& v);
void launch_qrcp(DescStage& st, const std::vector<QrcpDesc>& v, int prec);
void launch_svd_rt(DescStage& st, const std::vector<SvdRtDesc>& v, int prec);
void launch_sketch(DescStage& st, const std::vector<SketchDesc>& v);
void launch_frob(DescStage& st, const std::vector<FrobDesc>& v);
// checks the launches just issued and counts nkernels of them (profile kind "kernels")
void check_launch(const char* what, long nkernels = 1);

inline CopyDesc cpy(const double* src, int lds, double* dst, int ldd, int rows, int cols, double alpha = 1.0,
                    double beta = 0.0, int trans = 0) {
  CopyDesc d;
  d.src = src;
  d.dst = dst;
  d.lds = lds;
  d.ldd = ldd;
  d.rows = rows;
  d.cols = cols;
  d.alpha = alpha;
  d.beta = beta;
  d.trans = trans;
  d.pad = 0;
  return d;
}

inline GemmDesc gmm(const double* A, int lda, int ta, const double* B, int ldb, int tb, double* C, int ldc, int m,
                    int n, int k, double alpha, double beta) {
  GemmDesc d;
  d.A = A;
  d.B = B;
  d.C = C;
  d.lda = lda;
  d.ldb = ldb;
  d.ldc = ldc;
  d.m = m;
  d.n = n;
  d.k = k;
  d.ta = ta;
  d.tb = tb;
  d.alpha = alpha;
  d.beta = beta;
  return d;
}

inline GemvDesc gmv(const double* A, int lda, int m, int n, int trans, const double* x, double* y, double alpha,
                    double beta) {
  GemvDesc d;
  d.A = A;
  d.lda = lda;
  d.m = m;
  d.n = n;
  d.trans = trans;
  d.x = x;
  d.y = y;
  d.alpha = alpha;
  d.beta = beta;
  return d;
}

}  // namespace ifmm
