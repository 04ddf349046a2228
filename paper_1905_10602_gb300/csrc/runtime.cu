// Every device kernel of the library lives in this translation unit: the
// batched dense primitives (dense.cuh) and the IFMM-specific kernels below,
// plus their launchers.
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>

#include "dense.cuh"
#include "pairs.cuh"
#include "ifmm_kernels.h"
#include "runtime.h"

namespace ifmm {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }

Registry& registry() {
  static Registry r;
  static bool init = false;
  if (!init) {
    const char* e = getenv("IFMM_CHECK");
    r.on = e && e[0] == '1';
    init = true;
  }
  return r;
}

bool poison_on() {
  static const bool on = [] {
    const char* e = getenv("IFMM_POISON");
    return e && e[0] == '1';
  }();
  return on;
}
void poison_fill(void* p, size_t bytes) {
  // earlier work on any stream may still use the memory being handed out again
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemset(p, 0x7e, bytes) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess)
    (void)cudaGetLastError();  // e.g. during a stream capture: left unpoisoned
}

// bytes spanned by an m x n column-major block with leading dimension ld
static size_t span(int m, int n, long ld) {
  if (m <= 0 || n <= 0) return 0;
  return sizeof(double) * ((size_t)(n - 1) * ld + m);
}
static void req(const void* p, size_t bytes, const char* what, size_t idx) {
  if (!bytes || registry().contains(p, bytes)) return;
  throw Error(IFMM_EINVAL, std::string("bounds check failed: ") + what + " descriptor " + std::to_string(idx) +
                               " touches " + std::to_string(bytes) + " bytes outside any allocation");
}
static void check_copy(const CopyDesc* v, size_t n) {
  if (!registry().on) return;
  for (size_t i = 0; i < n; ++i) {
    const CopyDesc& d = v[i];
    if (d.rows < 0 || d.cols < 0) throw Error(IFMM_EINVAL, "negative copy size");
    if (d.src) req(d.src, d.trans ? span(d.cols, d.rows, d.lds) : span(d.rows, d.cols, d.lds), "copy.src", i);
    req(d.dst, span(d.rows, d.cols, d.ldd), "copy.dst", i);
    if (d.ldd < d.rows || (d.src && d.lds < (d.trans ? d.cols : d.rows))) throw Error(IFMM_EINVAL, "copy ld too small");
  }
}
static void check_gemm(const std::vector<GemmDesc>& v) {
  if (!registry().on) return;
  for (size_t i = 0; i < v.size(); ++i) {
    const GemmDesc& d = v[i];
    if (d.m <= 0 || d.n <= 0) continue;
    if (d.k > 0) {
      req(d.A, d.ta ? span(d.k, d.m, d.lda) : span(d.m, d.k, d.lda), "gemm.A", i);
      req(d.B, d.tb ? span(d.n, d.k, d.ldb) : span(d.k, d.n, d.ldb), "gemm.B", i);
      if (d.lda < (d.ta ? d.k : d.m) || d.ldb < (d.tb ? d.n : d.k)) throw Error(IFMM_EINVAL, "gemm ld too small");
    }
    req(d.C, span(d.m, d.n, d.ldc), "gemm.C", i);
    if (d.ldc < d.m) throw Error(IFMM_EINVAL, "gemm ldc too small");
  }
}

static const char* kKindNames[KK_COUNT] = {"copy", "gemm_fp64", "gemm_fp32", "gauss_jordan", "qr_fp64", "qr_fp32",
                                           "svd_fp64", "svd_fp32", "gemv", "gemv_sum", "p2p", "interp", "tables",
                                           "matvec", "permute", "gauss_jordan_big", "solve_graph",
                                           "qr_global_fp64", "qr_global_fp32", "qr_cluster_fp64", "qr_cluster_fp32", "kernels"};
const char* kernel_kind_name(int k) { return (k >= 0 && k < KK_COUNT) ? kKindNames[k] : nullptr; }
int& host_thread_cap() {
  static thread_local int c = 0;
  return c;
}
int& prof_level_tag() {
  static thread_local int t = -1;
  return t;
}
long& prof_batch_tag() {
  static thread_local long t = 0;
  return t;
}
Profiler& profiler() {
  static Profiler p;
  return p;
}
static std::mutex g_prof_mutex;
cudaEvent_t Profiler::begin(int kind, cudaStream_t s, long count) {
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  launches[kind] += count;
  if (!timing) return nullptr;
  cudaEvent_t e;
  CK(cudaEventCreate(&e));
  CK(cudaEventRecord(e, s));
  return e;
}
void Profiler::end(int kind, cudaStream_t s, cudaEvent_t b) {
  if (!timing || !b) return;
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  cudaEvent_t e;
  CK(cudaEventCreate(&e));
  CK(cudaEventRecord(e, s));
  pending.push_back({kind, {b, e}});
  pending_tags.push_back({prof_level_tag(), prof_batch_tag()});
  if (pending.size() > 4096) collect_locked();
}
void Profiler::collect() {
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  collect_locked();
}
void Profiler::collect_locked() {
  static FILE* log = nullptr;
  static bool log_init = false;
  if (!log_init) {
    const char* path = getenv("IFMM_PROFILE_LOG");
    if (path && path[0]) log = fopen(path, "a");
    log_init = true;
  }
  for (size_t i = 0; i < pending.size(); ++i) {
    auto& p = pending[i];
    CK(cudaEventSynchronize(p.second.second));
    float t = 0;
    CK(cudaEventElapsedTime(&t, p.second.first, p.second.second));
    ms[p.first] += t;
    events_kernels[p.first] += 1;
    if (log) fprintf(log, "%s %d %ld %.4f\n", kKindNames[p.first], pending_tags[i].first, pending_tags[i].second, t);
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  if (log) fflush(log);
  pending.clear();
  pending_tags.clear();
}
void Profiler::count(int kind, long n) {
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  launches[kind] += n;
}
void Profiler::reset() {
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  collect_locked();
  for (int k = 0; k < KK_COUNT; ++k) {
    launches[k] = 0;
    events_kernels[k] = 0;
    ms[k] = 0;
  }
}

// checks the launches just issued and counts them (profile kind "kernels")
void check_launch(const char* what, long nkernels) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error(IFMM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  profiler().count(KK_ALL, nkernels);
}

// Independent launches of one batch on side streams of the caller's stream:
// fork() orders the side streams after everything already on the main stream
// (descriptor uploads included), join() orders the main stream after them.
// The side streams and events belong to the calling thread.
struct ForkJoin {
  static constexpr int kSide = 4;
  cudaStream_t main;
  int used = 0;
  struct Side {
    cudaStream_t s[kSide] = {};
    cudaEvent_t done[kSide] = {};
    cudaEvent_t fork = nullptr;
    int dev = -1;
    ~Side() {
      if (dev < 0) return;
      for (int i = 0; i < kSide; ++i) {
        cudaStreamDestroy(s[i]);
        cudaEventDestroy(done[i]);
      }
      cudaEventDestroy(fork);
    }
  };
  static Side& side() {
    static thread_local Side sd;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (sd.dev != dev) {
      for (int i = 0; i < kSide; ++i) {
        CK(cudaStreamCreateWithFlags(&sd.s[i], cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&sd.done[i], cudaEventDisableTiming));
      }
      CK(cudaEventCreateWithFlags(&sd.fork, cudaEventDisableTiming));
      sd.dev = dev;
    }
    return sd;
  }
  explicit ForkJoin(cudaStream_t m) : main(m) {
    CK(cudaEventRecord(side().fork, main));
  }
  // the i-th independent launch goes to stream(i)
  cudaStream_t stream(int i) {
    Side& sd = side();
    const int k = i % kSide;
    if (k >= used) {
      CK(cudaStreamWaitEvent(sd.s[k], sd.fork, 0));
      used = k + 1;
    }
    return sd.s[k];
  }
  void join() {
    Side& sd = side();
    for (int k = 0; k < used; ++k) {
      CK(cudaEventRecord(sd.done[k], sd.s[k]));
      CK(cudaStreamWaitEvent(main, sd.done[k], 0));
    }
    used = 0;
  }
};

// ------------------------------------------------------------------ launchers
void launch_copy(DescStage& st, const std::vector<CopyDesc>& v) {
  if (v.empty()) return;
  // blocks of at most 1024 elements first, then the rest (each in list order),
  // sorted straight into the pinned staging buffer: one upload
  size_t ns = 0;
  for (auto& x : v) ns += copy_is_small(x);
  CopyDesc* h = (CopyDesc*)st.host_alloc(sizeof(CopyDesc) * v.size());
  size_t js = 0, jb = ns;
  for (auto& x : v) h[copy_is_small(x) ? js++ : jb++] = x;
  launch_copy_sorted(st, h, ns, v.size() - ns);
}

void launch_copy_sorted(DescStage& st, const CopyDesc* h, size_t ns, size_t nb) {
  if (ns + nb == 0) return;
  check_copy(h, ns + nb);
  const CopyDesc* d = st.upload(h, ns + nb);
  prof_batch_tag() = (long)(ns + nb);
  cudaEvent_t pe = profiler().begin(KK_COPY, st.stream);
  if (ns) k_copy_small<<<(unsigned)((ns + 7) / 8), 256, 0, st.stream>>>(d, (int)ns);
  if (nb) k_copy<<<(unsigned)nb, 256, 0, st.stream>>>(d + ns, (int)nb);
  check_launch("k_copy", (long)(ns > 0) + (long)(nb > 0));
  profiler().end(KK_COPY, st.stream, pe);
}

// Large reduced-precision GEMMs on the tensor cores (k_gemm_tc, 128 x 128 tiles).
static void launch_gemm_tc(DescStage& st, const std::vector<GemmDesc>& v, int prec) {
  if (v.empty()) return;
  static thread_local std::vector<int> tp;
  tp.assign(v.size() + 1, 0);
  for (size_t i = 0; i < v.size(); ++i)
    tp[i + 1] = tp[i] + (int)((long)((v[i].m + kTcBM - 1) / kTcBM) * ((v[i].n + kTcBN - 1) / kTcBN));
  const GemmDesc* d = st.push(v);
  const int* p = st.push(tp);
  static bool attr = false;  // set once per process (the attribute is per function)
  if (!attr) {
    CK(cudaFuncSetAttribute(k_gemm_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, gemm_tc_smem_bytes(0)));
    CK(cudaFuncSetAttribute(k_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, gemm_tc_smem_bytes(1)));
    attr = true;
  }
  prof_batch_tag() = (long)v.size();
  cudaEvent_t pe = profiler().begin(KK_GEMM32, st.stream);
  if (prec == P16)
    k_gemm_tc<1><<<(unsigned)tp.back(), 256, gemm_tc_smem_bytes(1), st.stream>>>(d, p, (int)v.size());
  else
    k_gemm_tc<0><<<(unsigned)tp.back(), 256, gemm_tc_smem_bytes(0), st.stream>>>(d, p, (int)v.size());
  check_launch("k_gemm_tc");
  profiler().end(KK_GEMM32, st.stream, pe);
}

void launch_gemm(DescStage& st, const std::vector<GemmDesc>& v0, int prec) {
  if (v0.empty()) return;
  check_gemm(v0);
  // products of at most 32 x 32 go straight into the pinned staging buffer
  // (list order); the larger ones (few) are sorted further below
  static thread_local std::vector<GemmDesc> v;
  static thread_local std::vector<int> tp;
  auto is_small = [](const GemmDesc& x) { return x.m > 0 && x.n > 0 && x.m <= 32 && x.n <= 32; };
  size_t ns = 0;
  for (auto& x : v0) ns += is_small(x);
  GemmDesc* hs = ns ? (GemmDesc*)st.host_alloc(sizeof(GemmDesc) * ns) : nullptr;
  size_t js = 0;
  v.clear();
  for (auto& x : v0) {
    if (x.m <= 0 || x.n <= 0) continue;
    if (is_small(x))
      hs[js++] = x;
    else
      v.push_back(x);
  }
  if (ns) {
    const GemmDesc* d = st.upload(hs, ns);
    const int kk = prec == P64 ? KK_GEMM64 : KK_GEMM32;
    prof_batch_tag() = (long)ns;
    cudaEvent_t pe = profiler().begin(kk, st.stream);
    if (prec == P32)
      k_gemm_small<float><<<(unsigned)((ns + 3) / 4), 128, 0, st.stream>>>(d, (int)ns);
    else if (prec == P16)
      k_gemm_small<float, true><<<(unsigned)((ns + 3) / 4), 128, 0, st.stream>>>(d, (int)ns);
    else
      k_gemm_small<double><<<(unsigned)((ns + 3) / 4), 128, 0, st.stream>>>(d, (int)ns);
    check_launch("k_gemm_small");
    profiler().end(kk, st.stream, pe);
  }
  if (v.empty()) return;
  if (prec != P64) {
    // large products on the tensor cores; the rest stay on the 64 x 64 FMA tiles
    static thread_local std::vector<GemmDesc> tc, fma;
    tc.clear();
    fma.clear();
    for (auto& x : v) (x.m > 64 && x.n > 64 && x.k >= 32 ? tc : fma).push_back(x);
    launch_gemm_tc(st, tc, prec);
    v.swap(fma);
    if (v.empty()) return;
  }
  tp.assign(v.size() + 1, 0);
  for (size_t i = 0; i < v.size(); ++i) {
    long t = (long)((v[i].m + 63) / 64) * ((v[i].n + 63) / 64);
    if (v[i].m <= 0 || v[i].n <= 0) t = 0;
    tp[i + 1] = tp[i] + (int)t;
  }
  if (tp.back() == 0) return;
  // descriptors with zero tiles are never selected: find_desc returns the last
  // descriptor whose start <= tile, and empty ones share their start with the next
  const GemmDesc* d = st.push(v);
  prof_batch_tag() = (long)v.size();
  const int* p = st.push(tp);
  const int kk = prec == P64 ? KK_GEMM64 : KK_GEMM32;
  cudaEvent_t pe = profiler().begin(kk, st.stream);
  if (prec == P32)
    k_gemm<float><<<(unsigned)tp.back(), 256, 0, st.stream>>>(d, p, (int)v.size());
  else if (prec == P16)
    k_gemm<float, true><<<(unsigned)tp.back(), 256, 0, st.stream>>>(d, p, (int)v.size());
  else
    k_gemm<double><<<(unsigned)tp.back(), 256, 0, st.stream>>>(d, p, (int)v.size());
  check_launch("k_gemm");
  profiler().end(kk, st.stream, pe);
}

// A cluster launch of k_inv_cluster (R CTAs per matrix); false when no cluster of
// that shape and shared memory can be resident.
static bool launch_inv_cluster(const InvDesc* d, int nd, int R, size_t smem, cudaStream_t s, bool probe_only) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nd * R), 1, 1);
  cfg.blockDim = dim3(512, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)R;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (probe_only) {
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_inv_cluster, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return ncl > 0;
  }
  CK(cudaLaunchKernelEx(&cfg, k_inv_cluster, d, nd));
  return true;
}

void launch_inv(DescStage& st, const std::vector<InvDesc>& v) {
  if (v.empty()) return;
  for (size_t i = 0; i < v.size() && registry().on; ++i) {
    req(v[i].A, span(v[i].n, v[i].n, v[i].ld), "inv.A", i);
    req(v[i].info, sizeof(int), "inv.info", i);
  }
  // Size classes.  Blocks of n <= 32: one CTA each in shared memory.  Larger
  // ones: the FP64 elimination of one block on one SM is bound by that SM's FP64
  // pipe, so when a color has fewer large blocks than SMs each block is spread
  // over a cluster of R CTAs (R ~ SMs / blocks, at most 16 -- a non-portable
  // cluster size, used when the GPU can host it -- and at least what its rows
  // need to fit); R = 1 is one CTA in shared memory (n <= 160).  Blocks that fit
  // no cluster take the batched multi-CTA kernels below.
  static constexpr int kInvCta = 0;
  static constexpr size_t kInvClusterSmem = 220 * 1024;
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    CK(cudaFuncSetAttribute(k_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024));
    CK(cudaFuncSetAttribute(k_inv_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInvClusterSmem));
    if (cudaFuncSetAttribute(k_inv_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
      cudaGetLastError();  // then the residency probe rejects R = 16
  });
  static int cl_ok[5] = {0, 0, 0, 0, 0};  // per R = 1, 2, 4, 8, 16: 0 unknown, 1 yes, -1 no
  static std::mutex cl_mu;
  // IFMM_INV_FALLBACK_N=n (read once per process; tests) sends every block of
  // at least n rows to the batched multi-CTA kernels
  static const int fallback_n = [] {
    const char* e = getenv("IFMM_INV_FALLBACK_N");
    const long n = e ? atol(e) : 0;
    return n >= 1 ? (int)std::min(n, 1L << 30) : 0;
  }();
  int nbig = 0;
  for (auto& x : v) nbig += x.n > 32;
  int rwant = 1;
  while (rwant < 16 && nbig * rwant * 2 <= 152) rwant *= 2;
  std::vector<InvDesc> cls[3], ccl[5];
  size_t csm[5] = {16, 16, 16, 16, 16};
  for (auto& x : v) {
    if (fallback_n && x.n >= fallback_n) {
      cls[2].push_back(x);
      continue;
    }
    if (x.n <= 32) {
      cls[0].push_back(x);
      continue;
    }
    int R = rwant, q = 0;
    while ((1 << q) < R) ++q;
    int qmin = 0;  // the smallest cluster whose slots hold the rows
    while (qmin < 5 && inv_cluster_slot_bytes(x.n, 1 << qmin) > kInvClusterSmem) ++qmin;
    if (q < qmin) q = qmin;
    if (q == 0 && x.n <= 160) {
      cls[1].push_back(x);
      continue;
    }
    if (q == 0) q = 1;
    bool ok = false;
    {
      std::lock_guard<std::mutex> lock(cl_mu);
      // the wanted size, else the next smaller one that still holds the rows
      for (; q < 5 && q >= std::max(1, qmin); --q) {
        if (cl_ok[q] == 0)
          cl_ok[q] = launch_inv_cluster(nullptr, 1, 1 << q, kInvClusterSmem, st.stream, true) ? 1 : -1;
        if (cl_ok[q] > 0) {
          ok = true;
          break;
        }
      }
    }
    if (ok) {
      ccl[q].push_back(x);
      csm[q] = std::max(csm[q], inv_cluster_slot_bytes(x.n, 1 << q));
    } else {
      cls[x.n <= 160 ? 1 : 2].push_back(x);
    }
  }
  (void)kInvCta;
  const InvDesc* dcl[5] = {};
  for (int q = 1; q < 5; ++q)
    if (!ccl[q].empty()) dcl[q] = st.push(ccl[q]);
  int ncl = 0;
  for (int q = 1; q < 5; ++q) ncl += (int)ccl[q].size();
  if (ncl) {
    prof_batch_tag() = (long)ncl;
    cudaEvent_t pe = profiler().begin(KK_INV, st.stream);
    ForkJoin fj(st.stream);
    int li = 0;
    for (int q = 1; q < 5; ++q) {
      if (ccl[q].empty()) continue;
      launch_inv_cluster(dcl[q], (int)ccl[q].size(), 1 << q, csm[q], fj.stream(li++), false);
      check_launch("k_inv_cluster");
    }
    fj.join();
    profiler().end(KK_INV, st.stream, pe);
  }
  for (int c = 0; c < 2; ++c) {
    if (cls[c].empty()) continue;
    int nmax = 0;
    for (auto& x : cls[c]) nmax = std::max(nmax, x.n);
    const int smem_mat = nmax * nmax * (int)sizeof(double);
    const size_t smem = (size_t)smem_mat + sizeof(double) * 2 * nmax + sizeof(int) * nmax + 16;
    const InvDesc* d = st.push(cls[c]);
    prof_batch_tag() = (long)cls[c].size();
    cudaEvent_t pe = profiler().begin(KK_INV, st.stream);
    k_inv<<<(unsigned)cls[c].size(), c == 0 ? 128 : 256, smem, st.stream>>>(d, (int)cls[c].size(), smem_mat);
    check_launch("k_inv");
    profiler().end(KK_INV, st.stream, pe);
  }
  if (!cls[2].empty()) {
    const std::vector<InvDesc>& L = cls[2];
    int nmax = 0;
    std::vector<long> off(L.size());
    long tot = 0;
    for (size_t i = 0; i < L.size(); ++i) {
      nmax = std::max(nmax, L[i].n);
      off[i] = tot;
      tot += 3 * (long)L[i].n + 2;
    }
    double* work = (double*)st.dev.alloc_bytes(sizeof(double) * tot);
    const InvDesc* d = st.push(L);
    const long* o = st.push(off);
    const int nb = (int)L.size();
    const int gx = (int)std::max<long>(1, std::min<long>(((long)nmax + 7) / 8, 64));
    prof_batch_tag() = (long)nb;
    cudaEvent_t pe = profiler().begin(KK_GJ_BIG, st.stream, 2L * nmax + 1);
    for (int k = 0; k < nmax; ++k) {
      k_gjb_pivot<<<nb, 256, 0, st.stream>>>(d, nb, k, work, o);
      k_gjb_update<<<dim3(gx, nb), 256, 0, st.stream>>>(d, nb, k, work, o);
    }
    k_gjb_colswap<<<nb, 256, 0, st.stream>>>(d, nb, work, o);
    check_launch("k_gjb", 2L * nmax + 1);
    profiler().end(KK_GJ_BIG, st.stream, pe);
  }
}

// Size buckets of the Householder QR launches.  A problem whose shared-memory
// slot (block + norms, in the arithmetic type) is at most kQrWarpSlot bytes is
// factorised by one warp; one of at most kQrCtaSmem bytes by one CTA with the
// block in shared memory.  A taller block is first reduced in place: its rows
// are cut into chunks that fit, each chunk is factorised (unpivoted), and the
// stacked chunk R factors -- the same column space, column norms and R up to
// signs -- are factorised as the logical matrix (rows addressed through
// QrcpDesc::rb, rs), when they fit.  Anything else goes to the global-memory
// kernels.
static constexpr size_t kQrWarpSlot = 12 * 1024;
static constexpr size_t kQrCtaSmem = 220 * 1024;
// Shared memory a QR problem may use per CTA; IFMM_QR_CTA_LIMIT_KB (<= 220)
// lowers it, which routes smaller problems through the tall reduction, the
// cluster and the global-memory kernels (used by the tests of those paths).
static size_t qr_cta_limit() {
  static const size_t lim = [] {
    const char* e = getenv("IFMM_QR_CTA_LIMIT_KB");
    const long kb = e ? atol(e) : 0;
    return (kb >= 4 && kb <= 220) ? (size_t)kb * 1024 : kQrCtaSmem;
  }();
  return lim;
}

static void qr_smem_attrs() {
  static std::once_flag once;
  std::call_once(once, [] {
    const int big = (int)kQrCtaSmem;
    const int wmax = (int)(8 * kQrWarpSlot);
    CK(cudaFuncSetAttribute(k_qr_cta<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    CK(cudaFuncSetAttribute(k_qr_cta<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    CK(cudaFuncSetAttribute(k_qr_cta<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    CK(cudaFuncSetAttribute(k_qr_cta<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    CK(cudaFuncSetAttribute(k_qr_warp<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, wmax));
    CK(cudaFuncSetAttribute(k_qr_warp<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, wmax));
    CK(cudaFuncSetAttribute(k_qr_warp<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, wmax));
    CK(cudaFuncSetAttribute(k_qr_warp<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, wmax));
    CK(cudaFuncSetAttribute(k_qr_cluster<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    CK(cudaFuncSetAttribute(k_qr_cluster<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    CK(cudaFuncSetAttribute(k_qr_cluster<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    CK(cudaFuncSetAttribute(k_qr_cluster<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  });
}

// A cluster launch of k_qr_cluster (R CTAs per problem); false when no cluster
// of that shape and shared memory can be resident (the caller then falls back).
template <typename TC, bool PIV>
static bool launch_qr_cluster(const QrcpDesc* d, int nd, int R, size_t smem, cudaStream_t s, bool probe_only) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nd * R), 1, 1);
  cfg.blockDim = dim3(512, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)R;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (probe_only) {
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_qr_cluster<TC, PIV>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return ncl > 0;
  }
  CK(cudaLaunchKernelEx(&cfg, k_qr_cluster<TC, PIV>, d, nd));
  return true;
}

// Launches problems that all fit in kQrCtaSmem: the warp bucket, then the CTA bucket.
static constexpr int kQrClusterSizes[3] = {2, 4, 8};

template <bool PIV>
static void launch_qr_fitting(DescStage& st, const std::vector<QrcpDesc>& v, int prec,
                              const std::vector<QrcpDesc>* clus = nullptr) {
  const int tcb = prec == P32 ? 4 : 8;
  // classes: warp per problem (slot <= kQrWarpSlot), then CTA per problem in
  // shared-memory size classes (<= 24, 48, 96, 220 KB).  A launch reserves its
  // largest slot for every CTA, so one large block must not set the occupancy of
  // many small ones; classes with few CTAs per SM get more threads to hide the
  // latency of each column step.  The classes run concurrently.
  const size_t lim = qr_cta_limit();
  const size_t cls[5] = {std::min(kQrWarpSlot, lim), std::min<size_t>(24 * 1024, lim), std::min<size_t>(48 * 1024, lim),
                         std::min<size_t>(96 * 1024, lim), lim};
  // (a launch of fewer problems than SMs gives every CTA 1024 threads)
  const bool few = v.size() < 152;
  const int thr[5] = {0, few ? 1024 : 256, few ? 1024 : 256, few ? 1024 : 512, 1024};
  std::vector<QrcpDesc> part[5];
  size_t smax[5] = {16, 16, 16, 16, 16};
  for (auto& x : v) {
    const size_t b = qr_slot_bytes(x.m, x.n, tcb);
    int c = 0;
    while (c < 4 && b > cls[c]) ++c;
    part[c].push_back(x);
    smax[c] = std::max(smax[c], b);
  }
  const QrcpDesc* d[5] = {};
  for (int c = 0; c < 5; ++c)
    if (!part[c].empty()) d[c] = st.push(part[c]);
  const QrcpDesc* dcl[3] = {};
  size_t scl[3] = {16, 16, 16};
  for (int c = 0; clus && c < 3; ++c) {
    if (clus[c].empty()) continue;
    dcl[c] = st.push(clus[c]);
    for (auto& x : clus[c]) scl[c] = std::max(scl[c], qr_cluster_slot_bytes(x.m, x.n, kQrClusterSizes[c], tcb));
  }
  ForkJoin fj(st.stream);
  int li = 0;
  for (int c = 0; clus && c < 3; ++c) {
    if (clus[c].empty()) continue;
    cudaStream_t s = fj.stream(li++);
    const int nd = (int)clus[c].size();
    if (prec == P32)
      launch_qr_cluster<float, PIV>(dcl[c], nd, kQrClusterSizes[c], scl[c], s, false);
    else
      launch_qr_cluster<double, PIV>(dcl[c], nd, kQrClusterSizes[c], scl[c], s, false);
    check_launch("k_qr_cluster");
    profiler().count(prec == P32 ? KK_QRC32 : KK_QRC64, 1);
  }
  for (int c = 0; c < 5; ++c) {
    if (part[c].empty()) continue;
    const int nd = (int)part[c].size();
    cudaStream_t s = fj.stream(li++);
    if (c == 0) {
      // warps per CTA: as many slots as fit in 48 KB, 1..8
      const int nwp = (int)std::max<size_t>(1, std::min<size_t>(8, (48 * 1024) / smax[0]));
      const unsigned grid = (unsigned)((nd + nwp - 1) / nwp);
      const size_t smem = smax[0] * nwp;
      if (prec == P32)
        k_qr_warp<float, PIV><<<grid, 32 * nwp, smem, s>>>(d[0], nd, (int)smax[0]);
      else
        k_qr_warp<double, PIV><<<grid, 32 * nwp, smem, s>>>(d[0], nd, (int)smax[0]);
      check_launch("k_qr_warp");
    } else {
      if (prec == P32)
        k_qr_cta<float, PIV><<<(unsigned)nd, thr[c], smax[c], s>>>(d[c], nd);
      else
        k_qr_cta<double, PIV><<<(unsigned)nd, thr[c], smax[c], s>>>(d[c], nd);
      check_launch("k_qr_cta");
    }
  }
  fj.join();
}

// Launches the shared-memory part of a QR batch (reducing tall blocks first);
// returns the indices of the descriptors left for the global-memory kernel.
template <bool PIV>
static std::vector<size_t> launch_qr_smem(DescStage& st, const std::vector<QrcpDesc>& v, int prec) {
  const int tcb = prec == P32 ? 4 : 8;
  const size_t lim = qr_cta_limit();
  qr_smem_attrs();
  std::vector<QrcpDesc> pre, fit;
  std::vector<size_t> rest;
  for (size_t i = 0; i < v.size(); ++i) {
    const QrcpDesc& x = v[i];
    if (qr_slot_bytes(x.m, x.n, tcb) <= lim) {
      fit.push_back(x);
      continue;
    }
    // largest chunk height c with a fitting slot
    long c = (long)((lim - sizeof(int) * (size_t)x.n - 16) / tcb) / std::max(1, x.n) - 2;
    while (c > 0 && qr_slot_bytes((int)c, x.n, tcb) > lim) --c;
    if (x.rb > 0 || x.m <= x.n || c < x.n) {
      rest.push_back(i);
      continue;
    }
    const int nch = (int)((x.m + c - 1) / c);
    const int last = x.m - (nch - 1) * (int)c;
    const int mv = (nch - 1) * x.n + std::min(x.n, last);
    if (qr_slot_bytes(mv, x.n, tcb) > lim) {
      rest.push_back(i);
      continue;
    }
    for (int j = 0; j < nch; ++j) {
      QrcpDesc q{};
      q.A = x.A + (long)j * c;
      q.ld = x.ld;
      q.m = std::min((int)c, x.m - j * (int)c);
      q.n = x.n;
      pre.push_back(q);
    }
    QrcpDesc y = x;
    y.m = mv;
    y.rb = x.n;
    y.rs = (int)c;
    fit.push_back(y);
  }
  // what neither fits nor reduces goes to a cluster of 2, 4 or 8 CTAs when its
  // rows fit their shared memory (rows addressed plainly: rb == 0)
  std::vector<QrcpDesc> clus[3];
  std::vector<size_t> left;
  for (size_t i : rest) {
    const QrcpDesc& x = v[i];
    int c = -1;
    if (x.rb == 0)
      for (int q = 0; q < 3 && c < 0; ++q)
        if (qr_cluster_slot_bytes(x.m, x.n, kQrClusterSizes[q], tcb) <= lim) c = q;
    if (c >= 0) {
      // residency of the largest cluster slot of each size (probed once)
      static std::mutex mu;
      static int ok_cache[2][2][3] = {};  // 0 unknown, 1 yes, -1 no
      int& ok = ok_cache[prec == P32 ? 0 : 1][PIV ? 1 : 0][c];
      std::lock_guard<std::mutex> lock(mu);
      if (ok == 0) {
        const bool r = prec == P32
                           ? launch_qr_cluster<float, PIV>(nullptr, 1, kQrClusterSizes[c], kQrCtaSmem, st.stream, true)
                           : launch_qr_cluster<double, PIV>(nullptr, 1, kQrClusterSizes[c], kQrCtaSmem, st.stream, true);
        ok = r ? 1 : -1;
      }
      if (ok < 0) c = -1;
    }
    if (c >= 0)
      clus[c].push_back(x);
    else
      left.push_back(i);
  }
  if (!pre.empty()) launch_qr_fitting<false>(st, pre, prec);
  launch_qr_fitting<PIV>(st, fit, prec, clus);
  return left;
}

void launch_qr(DescStage& st, const std::vector<QrDesc>& v, int prec) {
  if (v.empty()) return;
  for (auto& x : v) IFMM_REQUIRE(x.n <= 1024, IFMM_EINVAL, "QR wider than 1024 columns");
  for (size_t i = 0; i < v.size() && registry().on; ++i) {
    req(v[i].A, span(v[i].m, v[i].n, v[i].ld), "qr.A", i);
    if (v[i].ld < v[i].m) throw Error(IFMM_EINVAL, "qr ld too small");
  }
  prof_batch_tag() = (long)v.size();
  const int kk = prec == P32 ? KK_QR32 : KK_QR64;
  cudaEvent_t pe = profiler().begin(kk, st.stream);
  std::vector<QrcpDesc> as(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    QrcpDesc q{};
    q.A = v[i].A;
    q.ld = v[i].ld;
    q.m = v[i].m;
    q.n = v[i].n;
    as[i] = q;
  }
  const std::vector<size_t> rest = launch_qr_smem<false>(st, as, prec);
  profiler().end(kk, st.stream, pe);
  if (!rest.empty()) {
    std::vector<QrDesc> g;
    for (size_t i : rest) g.push_back(v[i]);
    const QrDesc* d = st.push(g);
    prof_batch_tag() = (long)g.size();
    const int kg = prec == P32 ? KK_QRG32 : KK_QRG64;
    cudaEvent_t pg = profiler().begin(kg, st.stream);
    if (prec == P32)
      k_qr<float><<<(unsigned)g.size(), 512, 0, st.stream>>>(d, (int)g.size());
    else
      k_qr<double><<<(unsigned)g.size(), 512, 0, st.stream>>>(d, (int)g.size());
    check_launch("k_qr");
    profiler().end(kg, st.stream, pg);
  }
}

void launch_qrcp(DescStage& st, const std::vector<QrcpDesc>& v, int prec) {
  if (v.empty()) return;
  for (auto& x : v) IFMM_REQUIRE(x.n <= 1024, IFMM_EINVAL, "pivoted QR wider than 1024 columns");
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    CK(cudaFuncSetAttribute(k_qrcp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    CK(cudaFuncSetAttribute(k_qrcp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  });
  for (size_t i = 0; i < v.size() && registry().on; ++i) {
    req(v[i].A, span(v[i].m, v[i].n, v[i].ld), "qrcp.A", i);
    req(v[i].jpvt, sizeof(int) * v[i].n, "qrcp.jpvt", i);
    req(v[i].kout, sizeof(int), "qrcp.kout", i);
    if (v[i].ld < v[i].m) throw Error(IFMM_EINVAL, "qrcp ld too small");
  }
  prof_batch_tag() = (long)v.size();
  const int kk = prec == P32 ? KK_QR32 : KK_QR64;
  cudaEvent_t pe = profiler().begin(kk, st.stream);
  const std::vector<size_t> rest = launch_qr_smem<true>(st, v, prec);
  profiler().end(kk, st.stream, pe);
  if (!rest.empty()) {
    std::vector<QrcpDesc> g;
    int nmax = 0;
    for (size_t i : rest) {
      g.push_back(v[i]);
      nmax = std::max(nmax, v[i].n);
    }
    const size_t smem = sizeof(double) * 2 * nmax + sizeof(int) * nmax + 16;
    IFMM_REQUIRE(smem <= 200 * 1024, IFMM_EINVAL, "pivoted QR too wide");
    const QrcpDesc* d = st.push(g);
    prof_batch_tag() = (long)g.size();
    const int kg = prec == P32 ? KK_QRG32 : KK_QRG64;
    cudaEvent_t pg = profiler().begin(kg, st.stream);
    if (prec == P32)
      k_qrcp<float><<<(unsigned)g.size(), 512, smem, st.stream>>>(d, (int)g.size());
    else
      k_qrcp<double><<<(unsigned)g.size(), 512, smem, st.stream>>>(d, (int)g.size());
    check_launch("k_qrcp");
    profiler().end(kg, st.stream, pg);
  }
}

void launch_svd_rt(DescStage& st, const std::vector<SvdRtDesc>& v, int prec) {
  if (v.empty()) return;
  static constexpr int smem_cap = 160 * 1024;
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    CK(cudaFuncSetAttribute(k_svd_rt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_cap));
    CK(cudaFuncSetAttribute(k_svd_rt<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_cap));
  });
  int nmax = 1;
  for (size_t i = 0; i < v.size(); ++i) {
    IFMM_REQUIRE(v[i].n <= 1024, IFMM_EINVAL, "SVD wider than 1024 columns");
    nmax = std::max(nmax, v[i].n);
    if (!registry().on) continue;
    const SvdRtDesc& x = v[i];
    req(x.A, span(x.n, x.n, x.ld) > 0 ? sizeof(double) : 0, "svd_rt.A", i);
    if (x.jpvt) req(x.jpvt, sizeof(int) * x.n, "svd_rt.jpvt", i);
    req(x.V, span(x.n, x.n, x.ldv), "svd_rt.V", i);
    req(x.sig, sizeof(double) * x.n, "svd_rt.sig", i);
    req(x.work, sizeof(double) * (size_t)x.n * x.n, "svd_rt.work", i);
  }
  // B is n x k with k <= n: n^2 elements bound what a problem keeps in shared
  // memory (larger ones use their global work buffer).  The batch is launched in
  // width classes so that a wide problem does not set the shared memory (and so
  // the occupancy) of many narrow ones; one warp per column pair of the widest
  // problem of a class
  const int tcb = prec == P32 ? 4 : 8;
  prof_batch_tag() = (long)v.size();
  const int kk = prec == P32 ? KK_SVD32 : KK_SVD64;
  cudaEvent_t pe = profiler().begin(kk, st.stream);
  const int wcls[4] = {16, 48, 128, 1024};
  std::vector<SvdRtDesc> part[4];
  int nmx[4] = {1, 1, 1, 1};
  for (auto& x : v) {
    int c = 0;
    while (c < 3 && x.n > wcls[c]) ++c;
    part[c].push_back(x);
    nmx[c] = std::max(nmx[c], x.n);
  }
  (void)nmax;
  const SvdRtDesc* d[4] = {};
  for (int c = 0; c < 4; ++c)
    if (!part[c].empty()) d[c] = st.push(part[c]);
  ForkJoin fj(st.stream);
  int li = 0;
  for (int c = 0; c < 4; ++c) {
    if (part[c].empty()) continue;
    const int smem = (int)std::min<size_t>(smem_cap, ((size_t)nmx[c] * nmx[c] * tcb + 15) & ~(size_t)15);
    const unsigned g = (unsigned)part[c].size();
    // one warp per column pair of the widest problem, up to 16 warps; up to 32
    // when the class has fewer problems than SMs (nothing else to hide latency)
    const int threads = std::min(g < 152 ? 1024 : 512, std::max(64, 32 * ((nmx[c] + 1) / 2)));
    cudaStream_t s = fj.stream(li++);
    if (prec == P32)
      k_svd_rt<float><<<g, threads, smem, s>>>(d[c], (int)g, 60, smem);
    else
      k_svd_rt<double><<<g, threads, smem, s>>>(d[c], (int)g, 60, smem);
    check_launch("k_svd_rt");
  }
  fj.join();
  profiler().end(kk, st.stream, pe);
}

// Level-start M2L blocks: one CTA per chunk of entries sharing an offset o, the
// translation block K_o staged once in shared memory (arithmetic type TC); per
// entry the CTA stages T_b and T'_a, forms W = K_o T_b (rc x kb) and then
// M2L_ab = T'_a W.  Every rank at a level start is <= rc <= 64.
template <typename TC>
__global__ void __launch_bounds__(256) k_m2l_init(const M2lChunk* __restrict__ ch, int nch, M2lTables t) {
  if ((int)blockIdx.x >= nch) return;
  const M2lChunk C = ch[blockIdx.x];
  const int rc = t.rc, tid = threadIdx.x, nt = blockDim.x;
  extern __shared__ __align__(16) unsigned char msm[];
  TC* K = (TC*)msm;       // rc x rc
  TC* Tb = K + rc * rc;   // rc x kb, ld rc
  TC* Tp = Tb + rc * rc;  // ka x rc, ld ka
  TC* Wm = Tp + rc * rc;  // rc x kb, ld rc
  const double* Kg = t.tab + (long)C.off * rc * rc;
  for (int x = tid; x < rc * rc; x += nt) K[x] = ld_tc<TC>(Kg[x]);
  for (int q = 0; q < C.count; ++q) {
    const int e = t.ent[C.first + q];
    const int a = t.il_row[e], b = t.il[e];
    const int ka = t.k[a], kb = t.k[b];
    if (!ka || !kb) continue;  // the same for every thread of the CTA
    __syncthreads();           // K staged; the previous entry is done with Tb, Tp, Wm
    const double* Tg = t.T[b];
    const double* Pg = t.Tp[a];
    for (int x = tid; x < rc * kb; x += nt) Tb[x] = ld_tc<TC>(Tg[x]);
    for (int x = tid; x < ka * rc; x += nt) Tp[x] = ld_tc<TC>(Pg[x]);
    __syncthreads();
    for (int x = tid; x < rc * kb; x += nt) {
      const int r = x % rc, j = x / rc;
      TC acc = 0;
      for (int k = 0; k < rc; ++k) acc += K[r + k * rc] * Tb[k + j * rc];
      Wm[x] = acc;
    }
    __syncthreads();
    double* M = t.far[e];
    const long ld = t.capr[a];
    for (int x = tid; x < ka * kb; x += nt) {
      const int i = x % ka, j = x / ka;
      TC acc = 0;
      for (int r = 0; r < rc; ++r) acc += Tp[i + r * ka] * Wm[r + j * rc];
      M[i + (long)j * ld] = st_tc<TC>(acc);
    }
  }
}

void launch_m2l_init(DescStage& st, const std::vector<M2lChunk>& chunks, const M2lTables& t, int prec) {
  if (chunks.empty()) return;
  IFMM_REQUIRE(t.rc <= 64, IFMM_EINVAL, "internal: level-start M2L kernel needs rc <= 64");
  const M2lChunk* d = st.push(chunks);
  const int kk = prec == P64 ? KK_GEMM64 : KK_GEMM32;
  prof_batch_tag() = (long)chunks.size();
  cudaEvent_t pe = profiler().begin(kk, st.stream);
  static bool attr = false;  // once per process: both instantiations may need > 48 KB
  if (!attr) {
    CK(cudaFuncSetAttribute(k_m2l_init<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 64 * 64 * 8));
    CK(cudaFuncSetAttribute(k_m2l_init<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 64 * 64 * 4));
    attr = true;
  }
  const size_t smem = (size_t)4 * t.rc * t.rc * (prec == P64 ? 8 : 4);
  if (prec == P64)
    k_m2l_init<double><<<(unsigned)chunks.size(), 256, smem, st.stream>>>(d, (int)chunks.size(), t);
  else
    k_m2l_init<float><<<(unsigned)chunks.size(), 256, smem, st.stream>>>(d, (int)chunks.size(), t);
  check_launch("k_m2l_init");
  profiler().end(kk, st.stream, pe);
}

void launch_il_transform(DescStage& st, const std::vector<int>& list, const IlTables& t, int md, int prec) {
  if (list.empty()) return;
  IFMM_REQUIRE(md >= 1 && md <= 64, IFMM_EINVAL, "IL transform tile out of range");
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    CK(cudaFuncSetAttribute(k_il_transform<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 64 * 64 * 8));
    CK(cudaFuncSetAttribute(k_il_transform<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 64 * 64 * 4));
  });
  const int* d = st.push(list);
  prof_batch_tag() = (long)list.size();
  const int kk = prec == P32 ? KK_GEMM32 : KK_GEMM64;
  cudaEvent_t pe = profiler().begin(kk, st.stream);
  const unsigned g = (unsigned)list.size();
  if (prec == P32)
    k_il_transform<float><<<g, 128, 3 * md * md * sizeof(float), st.stream>>>(d, (int)g, t, md);
  else
    k_il_transform<double><<<g, 128, 3 * md * md * sizeof(double), st.stream>>>(d, (int)g, t, md);
  check_launch("k_il_transform");
  profiler().end(kk, st.stream, pe);
}

void launch_zgather(DescStage& st, const std::vector<ZGatherDesc>& v, const ZTables& t) {
  if (v.empty()) return;
  const ZGatherDesc* d = st.push(v);
  prof_batch_tag() = (long)v.size();
  cudaEvent_t pe = profiler().begin(KK_COPY, st.stream);
  k_zgather<<<(unsigned)v.size(), 256, 0, st.stream>>>(d, (int)v.size(), t);
  check_launch("k_zgather");
  profiler().end(KK_COPY, st.stream, pe);
}

void launch_schur_scatter(DescStage& st, const std::vector<ScatterDesc>& v, const ScatterTables& t, int maxdeg) {
  if (v.empty() || maxdeg <= 0) return;
  IFMM_REQUIRE(maxdeg <= 32, IFMM_EINVAL, "more than 32 neighbours");
  const ScatterDesc* d = st.push(v);
  prof_batch_tag() = (long)v.size();
  cudaEvent_t pe = profiler().begin(KK_COPY, st.stream);
  k_schur_scatter<<<dim3((unsigned)v.size(), (unsigned)maxdeg), 256, 0, st.stream>>>(d, (int)v.size(), t);
  check_launch("k_schur_scatter");
  profiler().end(KK_COPY, st.stream, pe);
}

void launch_sketch(DescStage& st, const std::vector<SketchDesc>& v) {
  if (v.empty()) return;
  const SketchDesc* d = st.push(v);
  profiler().count(KK_TABLES, 1);
  k_sketch<<<(unsigned)v.size(), 256, 0, st.stream>>>(d, (int)v.size());
  check_launch("k_sketch");
}
void launch_frob(DescStage& st, const std::vector<FrobDesc>& v) {
  if (v.empty()) return;
  const FrobDesc* d = st.push(v);
  profiler().count(KK_TABLES, 1);
  k_frob<<<(unsigned)v.size(), 256, 0, st.stream>>>(d, (int)v.size());
  check_launch("k_frob");
}

void launch_gemv(DescStage& st, const std::vector<GemvDesc>& v) {
  if (v.empty()) return;
  for (size_t i = 0; i < v.size() && registry().on; ++i) {
    const GemvDesc& x = v[i];
    req(x.A, span(x.m, x.n, x.lda), "gemv.A", i);
    req(x.x, sizeof(double) * (x.trans ? x.m : x.n), "gemv.x", i);
    req(x.y, sizeof(double) * (x.trans ? x.n : x.m), "gemv.y", i);
  }
  const GemvDesc* d = st.push(v);
  prof_batch_tag() = (long)v.size();
  cudaEvent_t pe = profiler().begin(KK_GEMV, st.stream);
  k_gemv<<<(unsigned)v.size(), 128, 0, st.stream>>>(d, (int)v.size());
  check_launch("k_gemv");
  profiler().end(KK_GEMV, st.stream, pe);
}

// ------------------------------------------------------------------ IFMM kernels
__device__ __forceinline__ double cheb_root(int a, int p) {
  // first-kind Chebyshev roots t_a = cos((2a+1) pi / (2p)), a = 0..p-1
  return cospi((2.0 * a + 1.0) / (2.0 * p));
}

// Lagrange basis on the p roots: l_a(u) = prod_{b != a} (u - t_b)/(t_a - t_b)
__device__ __forceinline__ double lagrange(int a, int p, double u) {
  const double ta = cheb_root(a, p);
  double v = 1.0;
  for (int b = 0; b < p; ++b)
    if (b != a) {
      const double tb = cheb_root(b, p);
      v *= (u - tb) / (ta - tb);
    }
  return v;
}

// Near-field blocks: A_ij = scale/|x_i - x_j|, A_ii = diag (same leaf).  With
// dof = 2 (Helmholtz, wavenumber k) the entry is z = scale e^{ik r}/r (A_ii =
// diag + i diag_im) in the real 2 x 2 form [[Re z, -Im z], [Im z, Re z]] acting
// on the (real, imaginary) pair of each point: rows and columns 2a, 2a + 1.
__global__ void k_p2p(const P2pDesc* __restrict__ d, int nd, const double* __restrict__ px,
                      const double* __restrict__ py, const double* __restrict__ pz, double scale, double diag,
                      double diag_im, double k, int dof) {
  if ((int)blockIdx.x >= nd) return;
  const P2pDesc D = d[blockIdx.x];
  const int total = D.ni * D.nj;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int a = e % D.ni, b = e / D.ni;
    const int i = D.i0 + a, j = D.j0 + b;
    const bool self = D.same && a == b;
    double r = 1.0;
    if (!self) {
      const double dx = px[i] - px[j], dy = py[i] - py[j], dz = pz[i] - pz[j];
      r = sqrt(dx * dx + dy * dy + dz * dz);
    }
    if (dof == 1) {
      D.dst[a + (long)b * D.ld] = self ? diag : scale / r;
    } else {
      double zr = diag, zi = diag_im;
      if (!self) {
        double sn, cs;
        sincos(k * r, &sn, &cs);
        zr = scale * cs / r;
        zi = scale * sn / r;
      }
      double* o = D.dst + 2 * a + (long)(2 * b) * D.ld;
      o[0] = zr;
      o[1] = zi;
      o[D.ld] = -zi;
      o[D.ld + 1] = zr;
    }
  }
}

// 32 x 32 tiles of the self blocks of the block-diagonal preconditioner
__global__ void k_bd_fill(const BdBlockDesc* __restrict__ d, const int* __restrict__ tile_ptr, int nd,
                          const double* __restrict__ px, const double* __restrict__ py, const double* __restrict__ pz,
                          double scale, double diag) {
  const int di = find_desc(tile_ptr, nd, blockIdx.x);
  const BdBlockDesc D = d[di];
  const int local = blockIdx.x - tile_ptr[di];
  const int tr = (D.n + 31) >> 5;
  const int r0 = (local % tr) * 32, c0 = (local / tr) * 32;
  for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
    const int a = r0 + (e & 31), b = c0 + (e >> 5);
    if (a >= D.n || b >= D.n) continue;
    double v = diag;
    if (a != b) {
      const int i = D.idx[a], j = D.idx[b];
      const double dx = px[i] - px[j], dy = py[i] - py[j], dz = pz[i] - pz[j];
      v = scale / sqrt(dx * dx + dy * dy + dz * dz);
    }
    D.dst[a + (long)b * D.n] = v;
  }
}

// Leaf interpolation matrix S (p^3 x n): S(m, j) = l_a(u_x) l_b(u_y) l_c(u_z),
// m = (c p + b) p + a, u = (x_j - centre)/halfwidth.
// With dof = 2 the matrix is S (x) I_2 (each node and point carries a real and
// an imaginary part).
__global__ void k_interp(const InterpDesc* __restrict__ d, int nd, const double* __restrict__ px,
                         const double* __restrict__ py, const double* __restrict__ pz, int p, int dof) {
  if ((int)blockIdx.x >= nd) return;
  const InterpDesc D = d[blockIdx.x];
  const int r = p * p * p;
  const int total = r * D.n;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int m = e % r, j = e / r;
    const int a = m % p, b = (m / p) % p, c = m / (p * p);
    const int pt = D.p0 + j;
    const double ux = (px[pt] - D.cx) / D.h, uy = (py[pt] - D.cy) / D.h, uz = (pz[pt] - D.cz) / D.h;
    const double v = lagrange(a, p, ux) * lagrange(b, p, uy) * lagrange(c, p, uz);
    if (dof == 1) {
      D.dst[m + (long)j * D.ld] = v;
    } else {
      double* o = D.dst + 2 * m + (long)(2 * j) * D.ld;
      o[0] = v;
      o[1] = 0.0;
      o[D.ld] = 0.0;
      o[D.ld + 1] = v;
    }
  }
}

// M2L translation table of one level: for the 7^3 target-minus-source cell
// offsets o, K_o(m, k) = scale / |h (2 o + t_m - t_k)| between the Chebyshev
// nodes of two cells of half-width h (offsets with max |o| <= 1 stay zero).
// With dof = 2 (Helmholtz) the entry is scale e^{ik r}/r, r = h |2 o + t_m - t_k|,
// in the real 2 x 2 form (ld 2 r^3).
__global__ void k_m2l_table(double* __restrict__ out, int p, double h, double scale, double wk, int dof) {
  const int r = p * p * p, rd = dof * r;
  const int o = blockIdx.x;  // 0..342
  const int ox = o % 7 - 3, oy = (o / 7) % 7 - 3, oz = o / 49 - 3;
  const bool near = abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1;
  double* T = out + (long)o * rd * rd;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int m = e % r, k = e / r;
    double v = 0.0, vi = 0.0;
    if (!near) {
      const int ma = m % p, mb = (m / p) % p, mc = m / (p * p);
      const int ka = k % p, kb = (k / p) % p, kc = k / (p * p);
      const double dx = 2.0 * ox + cheb_root(ma, p) - cheb_root(ka, p);
      const double dy = 2.0 * oy + cheb_root(mb, p) - cheb_root(kb, p);
      const double dz = 2.0 * oz + cheb_root(mc, p) - cheb_root(kc, p);
      const double dist = h * sqrt(dx * dx + dy * dy + dz * dz);
      if (dof == 1) {
        v = scale / dist;
      } else {
        double sn, cs;
        sincos(wk * dist, &sn, &cs);
        v = scale * cs / dist;
        vi = scale * sn / dist;
      }
    }
    if (dof == 1) {
      T[e] = v;
    } else {
      double* q = T + 2 * m + (long)(2 * k) * rd;
      q[0] = v;
      q[1] = vi;
      q[rd] = -vi;
      q[rd + 1] = v;
    }
  }
}

// M2M of the 8 child octants: M(m, k) = S_parent(child node k, parent node m),
// the child node at u = (o - 1/2) + t_k / 2 in parent coordinates.
// (with dof = 2: M (x) I_2, ld 2 r^3)
__global__ void k_m2m_table(double* __restrict__ out, int p, int dof) {
  const int r = p * p * p, rd = dof * r;
  const int oct = blockIdx.x;  // 0..7, bit 0 = x, bit 1 = y, bit 2 = z
  const double sx = (oct & 1) - 0.5, sy = ((oct >> 1) & 1) - 0.5, sz = ((oct >> 2) & 1) - 0.5;
  double* T = out + (long)oct * rd * rd;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int m = e % r, k = e / r;
    const int ma = m % p, mb = (m / p) % p, mc = m / (p * p);
    const int ka = k % p, kb = (k / p) % p, kc = k / (p * p);
    const double ux = sx + 0.5 * cheb_root(ka, p), uy = sy + 0.5 * cheb_root(kb, p), uz = sz + 0.5 * cheb_root(kc, p);
    const double v = lagrange(ma, p, ux) * lagrange(mb, p, uy) * lagrange(mc, p, uz);
    if (dof == 1) {
      T[e] = v;
    } else {
      double* q = T + 2 * m + (long)(2 * k) * rd;
      q[0] = v;
      q[1] = 0.0;
      q[rd] = 0.0;
      q[rd + 1] = v;
    }
  }
}

// ---------------------------------------------------------------- FMM matvec
// y = A~ x through the FMM representation (Sec. 2.2, Eq. (1)) with the
// Chebyshev operators the factorization uses: P2M at the leaves, M2M up to
// level 2, M2L over the interaction lists of levels 2..depth, L2L down, then
// L2P plus the near field (A_ij for i, j in the same or adjacent leaves).  M
// and L of a level are node-major (rc per node); S (rc x n per leaf, ld rc)
// at soff[leaf].  FP64 throughout; a CTA per node, threads over the rc
// coefficients (or the leaf's points).
__device__ __forceinline__ int octant_of(const int* cells, int c) {
  return (cells[3 * c] & 1) | ((cells[3 * c + 1] & 1) << 1) | ((cells[3 * c + 2] & 1) << 2);
}
__global__ void k_fmm_p2m(const double* __restrict__ S, const long* __restrict__ soff, const int* __restrict__ leaf_ptr,
                          const double* __restrict__ x, double* __restrict__ M, int rc) {
  const int leaf = blockIdx.x;
  const int p0 = leaf_ptr[leaf], n = leaf_ptr[leaf + 1] - p0;
  const double* Sl = S + soff[leaf];
  for (int m = threadIdx.x; m < rc; m += blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc = fma(Sl[m + (long)j * rc], x[p0 + j], acc);
    M[(long)leaf * rc + m] = acc;
  }
}
__global__ void k_fmm_m2m(const int* __restrict__ child_ptr, const int* __restrict__ child,
                          const int* __restrict__ ccells, const double* __restrict__ m2m,
                          const double* __restrict__ Mc, double* __restrict__ Mp, int rc) {
  const int a = blockIdx.x;
  const long r2 = (long)rc * rc;
  for (int m = threadIdx.x; m < rc; m += blockDim.x) {
    double acc = 0.0;
    for (int x = child_ptr[a]; x < child_ptr[a + 1]; ++x) {
      const int c = child[x];
      const double* T = m2m + octant_of(ccells, c) * r2;
      const double* v = Mc + (long)c * rc;
      for (int k = 0; k < rc; ++k) acc = fma(T[m + (long)k * rc], v[k], acc);
    }
    Mp[(long)a * rc + m] = acc;
  }
}
__global__ void k_fmm_m2l(const int* __restrict__ il_ptr, const int* __restrict__ il, const int* __restrict__ cells,
                          const double* __restrict__ tab, const double* __restrict__ M, double* __restrict__ L,
                          int rc) {
  const int a = blockIdx.x;
  const long r2 = (long)rc * rc;
  const int ax = cells[3 * a], ay = cells[3 * a + 1], az = cells[3 * a + 2];
  for (int m = threadIdx.x; m < rc; m += blockDim.x) {
    double acc = 0.0;
    for (int e = il_ptr[a]; e < il_ptr[a + 1]; ++e) {
      const int b = il[e];
      const int o = (az - cells[3 * b + 2] + 3) * 49 + (ay - cells[3 * b + 1] + 3) * 7 + (ax - cells[3 * b] + 3);
      const double* K = tab + o * r2;
      const double* v = M + (long)b * rc;
      for (int k = 0; k < rc; ++k) acc = fma(K[m + (long)k * rc], v[k], acc);
    }
    L[(long)a * rc + m] = acc;
  }
}
__global__ void k_fmm_l2l(const int* __restrict__ parent, const int* __restrict__ cells, const double* __restrict__ m2m,
                          const double* __restrict__ Lp, double* __restrict__ Lc, int rc) {
  const int c = blockIdx.x;
  const long r2 = (long)rc * rc;
  const double* T = m2m + octant_of(cells, c) * r2;  // L2L = M2M^T
  const double* v = Lp + (long)parent[c] * rc;
  for (int m = threadIdx.x; m < rc; m += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < rc; ++k) acc = fma(T[k + (long)m * rc], v[k], acc);
    Lc[(long)c * rc + m] += acc;
  }
}
__global__ void k_fmm_l2p(const double* __restrict__ S, const long* __restrict__ soff, const int* __restrict__ leaf_ptr,
                          const int* __restrict__ nbr_ptr, const int* __restrict__ nbr, const double* __restrict__ L,
                          const double* __restrict__ px, const double* __restrict__ py, const double* __restrict__ pz,
                          const double* __restrict__ x, double* __restrict__ y, int rc, double scale, double diag) {
  const int leaf = blockIdx.x;
  const int p0 = leaf_ptr[leaf], n = leaf_ptr[leaf + 1] - p0;
  const double* Sl = S + soff[leaf];
  const double* Ll = L + (long)leaf * rc;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int i = p0 + j;
    double far = 0.0;
    for (int m = 0; m < rc; ++m) far = fma(Sl[m + (long)j * rc], Ll[m], far);
    const double xi = px[i], yi = py[i], zi = pz[i];
    double near = 0.0;
    for (int q = -1; q < nbr_ptr[leaf + 1] - nbr_ptr[leaf]; ++q) {
      const int lq = q < 0 ? leaf : nbr[nbr_ptr[leaf] + q];
      for (int s = leaf_ptr[lq]; s < leaf_ptr[lq + 1]; ++s) {
        if (s == i) continue;
        const double dx = xi - px[s], dy = yi - py[s], dz = zi - pz[s];
        near = fma(x[s], rsqrt(dx * dx + dy * dy + dz * dz), near);
      }
    }
    y[i] = far + scale * near + diag * x[i];
  }
}

void launch_fmm_p2m(cudaStream_t s, const double* S, const long* soff, const int* leaf_ptr, const double* x, double* M,
                    int nleaf, int rc) {
  if (nleaf) k_fmm_p2m<<<nleaf, 64, 0, s>>>(S, soff, leaf_ptr, x, M, rc);
}
void launch_fmm_m2m(cudaStream_t s, const int* child_ptr, const int* child, const int* ccells, const double* m2m,
                    const double* Mc, double* Mp, int nparent, int rc) {
  if (nparent) k_fmm_m2m<<<nparent, 64, 0, s>>>(child_ptr, child, ccells, m2m, Mc, Mp, rc);
}
void launch_fmm_m2l(cudaStream_t s, const int* il_ptr, const int* il, const int* cells, const double* tab,
                    const double* M, double* L, int n, int rc) {
  if (n) k_fmm_m2l<<<n, 64, 0, s>>>(il_ptr, il, cells, tab, M, L, rc);
}
void launch_fmm_l2l(cudaStream_t s, const int* parent, const int* cells, const double* m2m, const double* Lp,
                    double* Lc, int n, int rc) {
  if (n) k_fmm_l2l<<<n, 64, 0, s>>>(parent, cells, m2m, Lp, Lc, rc);
}
void launch_fmm_l2p(cudaStream_t s, const double* S, const long* soff, const int* leaf_ptr, const int* nbr_ptr,
                    const int* nbr, const double* L, const double* pts, int N, const double* x, double* y, int nleaf,
                    int rc, double scale, double diag) {
  if (nleaf)
    k_fmm_l2p<<<nleaf, 64, 0, s>>>(S, soff, leaf_ptr, nbr_ptr, nbr, L, pts, pts + N, pts + 2 * (long)N, x, y, rc,
                                   scale, diag);
}

// y = diag x + scale * sum_{j != i} x_j / |p_i - p_j|: a thread per target,
// sources staged through shared memory in tiles of blockDim.x.
__global__ void __launch_bounds__(256) k_matvec(const double* __restrict__ px, const double* __restrict__ py,
                                                const double* __restrict__ pz, const double* __restrict__ x,
                                                double* __restrict__ y, int n, double scale, double diag) {
  __shared__ double sx[256], sy[256], sz[256], sq[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double xi = 0, yi = 0, zi = 0;
  if (i < n) {
    xi = px[i];
    yi = py[i];
    zi = pz[i];
  }
  double acc = 0.0;
  for (int j0 = 0; j0 < n; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    if (j < n) {
      sx[threadIdx.x] = px[j];
      sy[threadIdx.x] = py[j];
      sz[threadIdx.x] = pz[j];
      sq[threadIdx.x] = x[j];
    } else {
      sx[threadIdx.x] = sy[threadIdx.x] = sz[threadIdx.x] = 0.0;
      sq[threadIdx.x] = 0.0;
    }
    __syncthreads();
    const int cnt = min((int)blockDim.x, n - j0);
    for (int t = 0; t < cnt; ++t) {
      const double dx = xi - sx[t], dy = yi - sy[t], dz = zi - sz[t];
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (j0 + t != i) acc += sq[t] * rsqrt(r2);
    }
    __syncthreads();
  }
  if (i < n) y[i] = diag * x[i] + scale * acc;
}

// Helmholtz: y = A x with A_ij = scale e^{ik r_ij}/r_ij, A_ii = diag + i diag_im,
// complex vectors interleaved (re, im); FP64, a thread per target, sources
// staged through shared memory.
__global__ void __launch_bounds__(256) k_matvec_c(const double* __restrict__ px, const double* __restrict__ py,
                                                  const double* __restrict__ pz, const double* __restrict__ x,
                                                  double* __restrict__ y, int n, double scale, double diag,
                                                  double diag_im, double wk) {
  __shared__ double sx[256], sy[256], sz[256], sr[256], si[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double xi = 0, yi = 0, zi = 0;
  if (i < n) {
    xi = px[i];
    yi = py[i];
    zi = pz[i];
  }
  double ar = 0.0, ai = 0.0;
  for (int j0 = 0; j0 < n; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    if (j < n) {
      sx[threadIdx.x] = px[j];
      sy[threadIdx.x] = py[j];
      sz[threadIdx.x] = pz[j];
      sr[threadIdx.x] = x[2 * j];
      si[threadIdx.x] = x[2 * j + 1];
    }
    __syncthreads();
    const int cnt = min((int)blockDim.x, n - j0);
    for (int t = 0; t < cnt; ++t) {
      if (j0 + t == i) continue;
      const double dx = xi - sx[t], dy = yi - sy[t], dz = zi - sz[t];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      double sn, cs;
      sincos(wk * r, &sn, &cs);
      const double w = 1.0 / r;
      ar += (cs * sr[t] - sn * si[t]) * w;
      ai += (sn * sr[t] + cs * si[t]) * w;
    }
    __syncthreads();
  }
  if (i < n) {
    const double xr = x[2 * i], xim = x[2 * i + 1];
    y[2 * i] = diag * xr - diag_im * xim + scale * ar;
    y[2 * i + 1] = diag * xim + diag_im * xr + scale * ai;
  }
}

// ---------------------------------------------------------------- double-float matvec
// The same sum with every quantity carried as a float pair (pairs.cuh);
// 1/sqrt(r^2) from rsqrtf refined by one Newton step in pair arithmetic.
// FP64-level accuracy at FP32 throughput.
__global__ void k_split_df(const double* __restrict__ in, float* __restrict__ hi, float* __restrict__ lo, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double v = in[i];
    const float h = (float)v;
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
  }
}

// pts: 6 float arrays (xh, xl, yh, yl, zh, zl) of length n; q: (qh, ql).
// BS threads per CTA = sources per shared-memory tile; TPT targets per thread
// (TPT = 2: each source read from shared memory serves two independent
// accumulation chains).  A source tile is two float4 per source (x, y / z, q as
// pairs), read as two broadcast 16-byte loads.  Both autotuned per tree.
template <int BS, int TPT>
__global__ void __launch_bounds__(BS) k_matvec_df(const float* __restrict__ pts, const float* __restrict__ qh,
                                                  const float* __restrict__ ql, const double* __restrict__ x,
                                                  double* __restrict__ y, int n, double scale, double diag) {
  __shared__ float4 sa[BS], sb[BS];  // (xh, xl, yh, yl), (zh, zl, qh, ql)
  const float* xh = pts;
  const float* xl = pts + n;
  const float* yh = pts + 2 * (long)n;
  const float* yl = pts + 3 * (long)n;
  const float* zh = pts + 4 * (long)n;
  const float* zl = pts + 5 * (long)n;
  int ii[TPT];
  df px[TPT], py[TPT], pz[TPT], acc[TPT];
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int i = blockIdx.x * (BS * TPT) + u * BS + threadIdx.x;
    ii[u] = i;
    px[u] = py[u] = pz[u] = acc[u] = {0.f, 0.f};
    if (i < n) {
      px[u] = {xh[i], xl[i]};
      py[u] = {yh[i], yl[i]};
      pz[u] = {zh[i], zl[i]};
    }
  }
  for (int j0 = 0; j0 < n; j0 += BS) {
    const int j = j0 + threadIdx.x;
    if (j < n) {
      sa[threadIdx.x] = make_float4(xh[j], xl[j], yh[j], yl[j]);
      sb[threadIdx.x] = make_float4(zh[j], zl[j], qh[j], ql[j]);
    }
    __syncthreads();
    const int cnt = min(BS, n - j0);
    for (int t = 0; t < cnt; ++t) {
      const float4 a = sa[t], b = sb[t];
#pragma unroll
      for (int u = 0; u < TPT; ++u) {
        // d = p_i - p_j per axis: two-sum of the high parts plus the low parts
        // (not renormalised: it is squared next)
        const df dx = df_diff(px[u], a.x, a.y);
        const df dy = df_diff(py[u], a.z, a.w);
        const df dz = df_diff(pz[u], b.x, b.y);
        // r^2 = sum d^2: FMA two-product of the high parts, 2 h l for the rest
        const df r2 = df_sum3(df_sq(dx), df_sq(dy), df_sq(dz));
        const df w = df_rsqrt_fast(r2);
        // q_j / r as a pair, added with a two-sum
        const float ph = b.z * w.h;
        const float pl = fmaf(b.z, w.h, -ph) + fmaf(b.z, w.l, b.w * w.h);
        if (j0 + t != ii[u]) acc[u] = df_acc(acc[u], ph, pl);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < TPT; ++u)
    if (ii[u] < n) y[ii[u]] = diag * x[ii[u]] + scale * ((double)acc[u].h + (double)acc[u].l);
}

// The same sum with each unordered pair (i, j), i != j, evaluated once: the
// kernel is symmetric (1/|x_i - x_j|), so one 1/r serves both q_j / r (row i)
// and q_i / r (row j).  The points are cut into tiles of kSymTile; a CTA takes
// one pair of tiles (I <= J): every warp holds 32 targets of tile I and walks
// the 128 sources of tile J in four chunks of 32, lane l meeting source
// (l + step) mod 32 of the chunk at each step, so that the 32 lanes touch 32
// different sources and add their q_i / r into per-warp shared-memory column
// sums without atomics (a __syncwarp between steps orders them).  Each CTA
// writes its row sums as tile J's partial of the targets and its column sums,
// combined over the warps in a fixed order, as tile I's partial of the sources:
// part[B * n + p] is tile B's contribution to point p, written exactly once.  A
// diagonal tile (I == J) takes every ordered pair once, rows only.  The second
// kernel adds the T partials of each point in tile order.  Both orders are
// fixed, so the result does not depend on scheduling.
constexpr int kSymTile = 128;
__device__ __forceinline__ df sym_w(df px, df py, df pz, float4 a, float4 b) {
  const df dx = df_diff(px, a.x, a.y);
  const df dy = df_diff(py, a.z, a.w);
  const df dz = df_diff(pz, b.x, b.y);
  return df_rsqrt_fast(df_sum3(df_sq(dx), df_sq(dy), df_sq(dz)));
}
// q w as a pair added to acc (q a pair, w a pair)
__device__ __forceinline__ df sym_add(df acc, float qh, float ql, df w) {
  const float ph = qh * w.h;
  const float pl = fmaf(qh, w.h, -ph) + fmaf(qh, w.l, ql * w.h);
  return df_acc(acc, ph, pl);
}
__global__ void __launch_bounds__(kSymTile) k_matvec_sym(const float* __restrict__ pts, const float* __restrict__ qh,
                                                         const float* __restrict__ ql, int n, int T,
                                                         float2* __restrict__ part) {
  constexpr int TB = kSymTile;
  __shared__ float4 sa[TB], sb[TB];
  __shared__ float2 col[TB / 32][TB];
  // tile pair of this CTA: b = I T - I (I - 1) / 2 + (J - I), I <= J
  const long bid = blockIdx.x;
  int I = (int)((2.0 * T + 1.0 - sqrt((2.0 * T + 1.0) * (2.0 * T + 1.0) - 8.0 * (double)bid)) / 2.0);
  auto first = [&](int i) { return (long)i * T - (long)i * (i - 1) / 2; };
  if (I < 0) I = 0;
  if (I > T - 1) I = T - 1;
  while (I > 0 && first(I) > bid) --I;
  while (I < T - 1 && first(I + 1) <= bid) ++I;
  const int J = I + (int)(bid - first(I));
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float* xh = pts;
  const float* xl = pts + n;
  const float* yh = pts + 2 * (long)n;
  const float* yl = pts + 3 * (long)n;
  const float* zh = pts + 4 * (long)n;
  const float* zl = pts + 5 * (long)n;
  // outside the points: far away (finite distances) with zero charge
  constexpr float kFar = 1e15f;
  const int i = I * TB + tid, j = J * TB + tid;
  df px = {kFar, 0.f}, py = {kFar, 0.f}, pz = {kFar, 0.f};
  float qih = 0.f, qil = 0.f;
  if (i < n) {
    px = {xh[i], xl[i]};
    py = {yh[i], yl[i]};
    pz = {zh[i], zl[i]};
    qih = qh[i];
    qil = ql[i];
  }
  if (j < n) {
    sa[tid] = make_float4(xh[j], xl[j], yh[j], yl[j]);
    sb[tid] = make_float4(zh[j], zl[j], qh[j], ql[j]);
  } else {
    sa[tid] = make_float4(-kFar, 0.f, -kFar, 0.f);
    sb[tid] = make_float4(-kFar, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int u = 0; u < TB / 32; ++u) col[u][tid] = make_float2(0.f, 0.f);
  __syncthreads();
  df acc = {0.f, 0.f};
  if (I == J) {
    for (int t = 0; t < TB; ++t) {
      const float4 a = sa[t], b = sb[t];
      const df wr = sym_w(px, py, pz, a, b);
      if (t != tid) acc = sym_add(acc, b.z, b.w, wr);
    }
  } else {
    float2* mycol = col[w];
    for (int c = 0; c < TB; c += 32) {
      for (int r = 0; r < 32; ++r) {
        const int sidx = c + ((lane + r) & 31);
        const float4 a = sa[sidx], b = sb[sidx];
        const df wr = sym_w(px, py, pz, a, b);
        acc = sym_add(acc, b.z, b.w, wr);
        const float2 cv = mycol[sidx];
        const df cs = sym_add({cv.x, cv.y}, qih, qil, wr);
        mycol[sidx] = make_float2(cs.h, cs.l);
        __syncwarp();
      }
    }
  }
  if (i < n) part[(long)J * n + i] = make_float2(acc.h, acc.l);
  if (I != J) {
    __syncthreads();
    if (j < n) {
      df cs = {col[0][tid].x, col[0][tid].y};
#pragma unroll
      for (int u = 1; u < TB / 32; ++u) cs = df_acc(cs, col[u][tid].x, col[u][tid].y);
      part[(long)I * n + j] = make_float2(cs.h, cs.l);
    }
  }
}
__global__ void k_matvec_sym_sum(const float2* __restrict__ part, int n, int T, const double* __restrict__ x,
                                 double* __restrict__ y, double scale, double diag) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  df acc = {0.f, 0.f};
  for (int b = 0; b < T; ++b) {
    const float2 v = part[(long)b * n + p];
    acc = df_acc(acc, v.x, v.y);
  }
  y[p] = diag * x[p] + scale * ((double)acc.h + (double)acc.l);
}

// floats of partial sums the symmetric float-pair matvec needs for n points
size_t matvec_sym_part_floats(int n) {
  const long T = (n + kSymTile - 1) / kSymTile;
  return (size_t)T * (size_t)n * 2;
}

// ---------------------------------------------------------------- the solve's row operations
// out[r] = beta base[r] + alpha sum_c M[r][c] v(c) for the rows of every op of a
// launch.  `lanes` lanes share a row: each reads 16-byte vectors of the row
// (4 FP32 or 2 FP64 coefficients) at a stride of lanes vectors, two vectors per
// step, and the partial sums are combined by shuffles in a fixed order.  A warp
// covers 32 / lanes rows of one op; warp_ptr gives each op's first warp.
// PAIRS: FP32 coefficients, float-pair vectors and accumulation (the product of
// an exact float by a pair is formed with FMAs, so the operator applied is the
// stored FP32 matrix to ~2^-44); otherwise FP64 throughout.
// s + a v(c) with a exact and v(c) a pair: the FMA two-product of a and the
// high part plus a times the low part, added with a two-sum
__device__ __forceinline__ df pair_term(df s, float a, const float2* __restrict__ X, const int* __restrict__ xidx,
                                        int c) {
  const float2 xv = xidx ? X[xidx[c]] : X[c];
  const float p = a * xv.x;
  return df_acc(s, p, fmaf(a, xv.y, fmaf(a, xv.x, -p)));
}
template <bool PAIRS>
__global__ void __launch_bounds__(256) k_solve_rows(const SolveOp* __restrict__ ops, const int* __restrict__ warp_ptr,
                                                    int nops) {
  const int gw = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  if (gw >= warp_ptr[nops]) return;  // whole warps
  const int oi = find_desc(warp_ptr, nops, gw);
  const SolveOp& O = ops[oi];
  const int lane = threadIdx.x & 31;
  const int G = O.lanes;
  const int sub = lane & (G - 1);
  const int r = (gw - warp_ptr[oi]) * (32 / G) + lane / G;
  const bool live = r < O.rows;
  const int nc = live ? O.ncols : 0;
  if constexpr (PAIRS) {
    const float2* X = (const float2*)O.x;
    const int* xi = O.xidx;
    const float* row = (const float*)O.M + (long)r * O.ldm;
    df s = {0.f, 0.f};
    int c = sub * 4;
    for (; c + G * 4 < nc; c += 2 * G * 4) {
      const float4 u = *(const float4*)(row + c);
      const float4 w = *(const float4*)(row + c + G * 4);
      const int c2 = c + G * 4;
      s = pair_term(s, u.x, X, xi, c);
      if (c + 1 < nc) s = pair_term(s, u.y, X, xi, c + 1);
      if (c + 2 < nc) s = pair_term(s, u.z, X, xi, c + 2);
      if (c + 3 < nc) s = pair_term(s, u.w, X, xi, c + 3);
      s = pair_term(s, w.x, X, xi, c2);
      if (c2 + 1 < nc) s = pair_term(s, w.y, X, xi, c2 + 1);
      if (c2 + 2 < nc) s = pair_term(s, w.z, X, xi, c2 + 2);
      if (c2 + 3 < nc) s = pair_term(s, w.w, X, xi, c2 + 3);
    }
    if (c < nc) {
      const float4 u = *(const float4*)(row + c);
      s = pair_term(s, u.x, X, xi, c);
      if (c + 1 < nc) s = pair_term(s, u.y, X, xi, c + 1);
      if (c + 2 < nc) s = pair_term(s, u.z, X, xi, c + 2);
      if (c + 3 < nc) s = pair_term(s, u.w, X, xi, c + 3);
    }
    for (int o = G >> 1; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, s.h, o), ol = __shfl_xor_sync(0xffffffffu, s.l, o);
      s = df_acc(s, oh, ol);
    }
    if (live && sub == 0) {
      const int orow = O.oidx ? O.oidx[r] : r;
      if (O.alpha < 0.0) s = {-s.h, -s.l};
      if (O.beta != 0.0) {
        const float2 b = ((const float2*)O.base)[orow];
        s = df_acc(s, b.x, b.y);
      }
      ((float2*)O.out)[orow] = make_float2(s.h, s.l);
    }
  } else {
    const double* X = (const double*)O.x;
    const double* row = (const double*)O.M + (long)r * O.ldm;
    double s0 = 0.0, s1 = 0.0;
    auto xv = [&](int c) { return O.xidx ? X[O.xidx[c]] : X[c]; };
    int c = sub * 2;
    for (; c + G * 2 < nc; c += 2 * G * 2) {
      const double2 u = *(const double2*)(row + c);
      const double2 w = *(const double2*)(row + c + G * 2);
      const int c2 = c + G * 2;
      s0 = fma(u.x, xv(c), s0);
      if (c + 1 < nc) s1 = fma(u.y, xv(c + 1), s1);
      s0 = fma(w.x, xv(c2), s0);
      if (c2 + 1 < nc) s1 = fma(w.y, xv(c2 + 1), s1);
    }
    if (c < nc) {
      const double2 u = *(const double2*)(row + c);
      s0 = fma(u.x, xv(c), s0);
      if (c + 1 < nc) s1 = fma(u.y, xv(c + 1), s1);
    }
    double s = s0 + s1;
    for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (live && sub == 0) {
      const int orow = O.oidx ? O.oidx[r] : r;
      const double v = O.alpha * s;
      ((double*)O.out)[orow] = O.beta == 0.0 ? v : O.beta * ((const double*)O.base)[orow] + v;
    }
  }
}

// 32 x 32 tiles of column-major FP64 blocks written row-major (FP64 or FP32),
// through shared memory so both sides are coalesced
template <bool F32>
__global__ void __launch_bounds__(256) k_pack_rows(const PackDesc* __restrict__ d, const int* __restrict__ tile_ptr,
                                                   int nd) {
  __shared__ double tile[32][33];
  const int di = find_desc(tile_ptr, nd, blockIdx.x);
  const PackDesc D = d[di];
  const int local = blockIdx.x - tile_ptr[di];
  const int tr = (D.rows + 31) >> 5;
  const int r0 = (local % tr) * 32, c0 = (local / tr) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int j = ty; j < 32; j += 8) {
    const int r = r0 + tx, c = c0 + j;
    tile[j][tx] = (r < D.rows && c < D.cols) ? D.src[r + (long)c * D.lds] : 0.0;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + tx;
    if (r < D.rows && c < D.cols) {
      if constexpr (F32)
        ((float*)D.dst)[(long)r * D.ldd + c] = d2f_pow2(tile[tx][i], 0);
      else
        ((double*)D.dst)[(long)r * D.ldd + c] = tile[tx][i];
    }
  }
}

__global__ void k_pair_split(const double* __restrict__ in, float2* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const double v = in[i];
    const float h = d2f_pow2(v, 0);
    out[i] = make_float2(h, d2f_pow2(v - st_tc<float>(h), 0));
  }
}
__global__ void k_pair_join(const float2* __restrict__ in, double* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const float2 v = in[i];
    out[i] = st_tc<float>(v.x) + st_tc<float>(v.y);
  }
}

void launch_solve_ops(cudaStream_t s, const SolveOp* ops, const int* warp_ptr, int nops, int nwarps, bool pairs) {
  if (!nops || !nwarps) return;
  const unsigned blocks = (unsigned)((nwarps + 7) / 8);
  if (pairs)
    k_solve_rows<true><<<blocks, 256, 0, s>>>(ops, warp_ptr, nops);
  else
    k_solve_rows<false><<<blocks, 256, 0, s>>>(ops, warp_ptr, nops);
}

void launch_pack(DescStage& st, const std::vector<PackDesc>& v, bool fp32) {
  if (v.empty()) return;
  std::vector<int> tp(v.size() + 1, 0);
  for (size_t i = 0; i < v.size(); ++i)
    tp[i + 1] = tp[i] + (int)((long)((v[i].rows + 31) / 32) * ((v[i].cols + 31) / 32));
  if (!tp.back()) return;
  const PackDesc* d = st.push(v);
  const int* p = st.push(tp);
  if (fp32)
    k_pack_rows<true><<<(unsigned)tp.back(), 256, 0, st.stream>>>(d, p, (int)v.size());
  else
    k_pack_rows<false><<<(unsigned)tp.back(), 256, 0, st.stream>>>(d, p, (int)v.size());
  check_launch("k_pack_rows");
}

void launch_pair_split(cudaStream_t s, const double* in, void* out, int64_t n) {
  if (n > 0) k_pair_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, (float2*)out, n);
}
void launch_pair_join(cudaStream_t s, const void* in, double* out, int64_t n) {
  if (n > 0) k_pair_join<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const float2*)in, out, n);
}

void launch_split_df(cudaStream_t s, const double* in, float* hi, float* lo, int n) {
  k_split_df<<<(n + 255) / 256, 256, 0, s>>>(in, hi, lo, n);
  check_launch("k_split_df");
}

// the tile code: BS | TPT << 16; TPT = 3 is the symmetric kernel (part != NULL)
static void matvec_df_bs(int code, cudaStream_t s, const float* pts_df, const float* qh, const float* ql,
                         const double* x, double* y, int N, double scale, double diag, float2* part) {
  const int bs = code & 0xffff, tpt = code >> 16;
  if (tpt == 3 && part) {
    const long T = (N + kSymTile - 1) / kSymTile;
    k_matvec_sym<<<(unsigned)(T * (T + 1) / 2), kSymTile, 0, s>>>(pts_df, qh, ql, N, (int)T, part);
    k_matvec_sym_sum<<<(N + 255) / 256, 256, 0, s>>>(part, N, (int)T, x, y, scale, diag);
  } else if (tpt == 2) {
    if (bs == 128)
      k_matvec_df<128, 2><<<(N + 255) / 256, 128, 0, s>>>(pts_df, qh, ql, x, y, N, scale, diag);
    else
      k_matvec_df<256, 2><<<(N + 511) / 512, 256, 0, s>>>(pts_df, qh, ql, x, y, N, scale, diag);
  } else if (bs == 128) {
    k_matvec_df<128, 1><<<(N + 127) / 128, 128, 0, s>>>(pts_df, qh, ql, x, y, N, scale, diag);
  } else if (bs == 512) {
    k_matvec_df<512, 1><<<(N + 511) / 512, 512, 0, s>>>(pts_df, qh, ql, x, y, N, scale, diag);
  } else {
    k_matvec_df<256, 1><<<(N + 255) / 256, 256, 0, s>>>(pts_df, qh, ql, x, y, N, scale, diag);
  }
}

// Autotuner: times each candidate (source-tile width and targets per thread;
// the symmetric kernel when a partial-sum buffer is given) twice on the
// caller's data (after one untimed launch of each) and returns the fastest as
// BS | TPT << 16; y is overwritten.
int autotune_matvec_df(cudaStream_t s, const float* pts_df, const float* qh, const float* ql, const double* x,
                       double* y, int N, double scale, double diag, float2* part) {
  std::vector<int> cand = {128 | 1 << 16, 256 | 1 << 16, 512 | 1 << 16, 128 | 2 << 16, 256 | 2 << 16};
  if (part) cand.push_back(kSymTile | 3 << 16);
  float best = 1e30f;
  int pick = 256 | 1 << 16;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  for (int c : cand) matvec_df_bs(c, s, pts_df, qh, ql, x, y, N, scale, diag, part);
  for (int c : cand) {
    CK(cudaEventRecord(a, s));
    for (int r = 0; r < 2; ++r) matvec_df_bs(c, s, pts_df, qh, ql, x, y, N, scale, diag, part);
    CK(cudaEventRecord(b, s));
    CK(cudaEventSynchronize(b));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, a, b));
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  check_launch("autotune_matvec_df", 9);
  return pick;
}

void launch_matvec_df(cudaStream_t s, const float* pts_df, const float* qh, const float* ql, const double* x, double* y,
                      int N, double scale, double diag, int bs, float2* part) {
  cudaEvent_t pe = profiler().begin(KK_MATVEC, s);
  matvec_df_bs(bs, s, pts_df, qh, ql, x, y, N, scale, diag, part);
  check_launch("k_matvec_df");
  profiler().end(KK_MATVEC, s, pe);
}

// ---------------------------------------------------------------- Gram sums, Cholesky
// dst (r x r) = sum of the listed r x r matrices (one CTA per output).
__global__ void k_gram_sum(double* const* __restrict__ dst, const double* const* __restrict__ terms,
                           const int* __restrict__ first, int nd, int r) {
  const int b = blockIdx.x;
  if (b >= nd) return;
  const int t0 = first[b], t1 = first[b + 1];
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    double s = 0.0;
    for (int t = t0; t < t1; ++t) s += terms[t][e];
    dst[b][e] = s;
  }
}

// Upper Cholesky factor R (R^T R = G + delta * max_i G_ii * I) of each r x r
// matrix, r <= 128, in shared memory; a pivot that is still not positive is
// replaced by delta * max_i G_ii (the direction then carries almost no weight).
__global__ void k_chol(double* const* __restrict__ mats, int nd, int r, double delta) {
  const int b = blockIdx.x;
  if (b >= nd) return;
  extern __shared__ double G[];
  double* M = mats[b];
  __shared__ double s_diag, s_piv;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) G[e] = M[e];
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < r; ++i) mx = fmax(mx, G[i + i * r]);
    s_diag = mx > 0.0 ? delta * mx : 1e-300;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x) G[i + i * r] += s_diag;
  __syncthreads();
  // right-looking: column-major G, upper factor stored in the upper triangle
  for (int k = 0; k < r; ++k) {
    if (threadIdx.x == 0) {
      double d = G[k + k * r];
      if (!(d > s_diag * 1e-3)) d = s_diag;
      s_piv = sqrt(d);
      G[k + k * r] = s_piv;
    }
    __syncthreads();
    const double pv = s_piv;
    for (int j = k + 1 + threadIdx.x; j < r; j += blockDim.x) G[k + j * r] /= pv;  // row k of R
    __syncthreads();
    for (int e = threadIdx.x; e < (r - k - 1) * (r - k - 1); e += blockDim.x) {
      const int i = k + 1 + e % (r - k - 1), j = k + 1 + e / (r - k - 1);
      if (i <= j) G[i + j * r] -= G[k + i * r] * G[k + j * r];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    M[e] = (i <= j) ? G[e] : 0.0;
  }
}

void launch_gram_sum(DescStage& st, const std::vector<double*>& dst, const std::vector<const double*>& terms,
                     const std::vector<int>& first, int r) {
  if (dst.empty()) return;
  double* const* d = st.push(dst);
  const double* const* t = st.push(terms);
  const int* f = st.push(first);
  profiler().count(KK_TABLES, 1);
  k_gram_sum<<<(unsigned)dst.size(), 256, 0, st.stream>>>(d, t, f, (int)dst.size(), r);
  check_launch("k_gram_sum");
}

void launch_chol(DescStage& st, const std::vector<double*>& mats, int r, double delta) {
  if (mats.empty()) return;
  IFMM_REQUIRE(r <= 128, IFMM_EINVAL, "Cholesky block too large");
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    CK(cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024));
  });
  double* const* d = st.push(mats);
  profiler().count(KK_TABLES, 1);
  k_chol<<<(unsigned)mats.size(), 256, sizeof(double) * r * r, st.stream>>>(d, (int)mats.size(), r, delta);
  check_launch("k_chol");
}

// point permutations of vectors with dof entries per point
__global__ void k_gather_perm(const double* __restrict__ src, const int* __restrict__ perm, double* __restrict__ dst,
                              int n, int dof) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n * dof) {
    const int pt = k / dof, c = k - pt * dof;
    dst[k] = src[(long)perm[pt] * dof + c];
  }
}
__global__ void k_scatter_perm(const double* __restrict__ src, const int* __restrict__ perm, double* __restrict__ dst,
                               int n, int dof) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n * dof) {
    const int pt = k / dof, c = k - pt * dof;
    dst[(long)perm[pt] * dof + c] = src[k];
  }
}

// ---------------------------------------------------------------- big Gauss-Jordan
// Inverse of one large n x n matrix with one launch pair per pivot step:
// k_gj_pivot (one CTA) picks and swaps the pivot row and scales it, then
// k_gj_update (many CTAs) eliminates column k from every other row.
__global__ void k_gj_pivot(double* A, long ld, int n, int k, int* piv, double* rowk, double* colk, int* info) {
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_p;
  if (info[0] != 0) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  double best = -1.0;
  int bi = n;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double v = fabs(A[i + k * ld]);
    if (v > best || (v == best && i < bi)) { best = v; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
  }
  if (lane == 0) { red_v[w] = best; red_i[w] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bv = -1.0;
    int b = n;
    for (int i = 0; i < nw; ++i)
      if (red_v[i] > bv || (red_v[i] == bv && red_i[i] < b)) { bv = red_v[i]; b = red_i[i]; }
    if (!(bv > 0.0) || b >= n) {
      info[0] = k + 1;
      b = k;
    }
    s_p = b;
    piv[k] = b;
  }
  __syncthreads();
  if (info[0] != 0) return;
  const int p = s_p;
  if (p != k) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double t = A[k + j * ld];
      A[k + j * ld] = A[p + j * ld];
      A[p + j * ld] = t;
    }
    __syncthreads();  // p is the same in every thread: rows k and p swapped before they are read below
  }
  __shared__ double s_inv;
  if (threadIdx.x == 0) s_inv = 1.0 / A[k + k * ld];  // once: an FP64 divide is a long FP64 sequence
  __syncthreads();
  const double inv = s_inv;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = (j == k) ? inv : A[k + j * ld] * inv;
    rowk[j] = v;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = (i == k) ? 0.0 : A[i + k * ld];
}

__global__ void k_gj_update(double* A, long ld, int n, int k, const double* rowk, const double* colk,
                            const int* info) {
  if (info[0] != 0) return;
  // (column, 256-row segment) items over (CTA, warp), lanes over rows
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nseg = (n + 255) / 256;
  for (int it = blockIdx.x * nw + (threadIdx.x >> 5); it < n * nseg; it += gridDim.x * nw) {
    const int j = it / nseg, seg = it % nseg;
    const double rj = rowk[j];
    double* cj = A + (long)j * ld;
    const int i1 = min(n, (seg + 1) * 256);
    for (int i = seg * 256 + lane; i < i1; i += 32) {
      if (i == k) {
        cj[i] = rj;
      } else {
        const double a = (j == k) ? 0.0 : cj[i];
        cj[i] = a - colk[i] * rj;
      }
    }
  }
}

__global__ void k_gj_colswap(double* A, long ld, int n, const int* piv, const int* info) {
  if (info[0] != 0) return;
  // one CTA: apply the column interchanges in reverse order
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double t = A[i + k * ld];
        A[i + k * ld] = A[i + p * ld];
        A[i + p * ld] = t;
      }
    __syncthreads();
  }
}

void big_inverse(cudaStream_t s, double* A, int ld, int n, int* d_work_int, double* d_work, int* d_info) {
  // d_work_int: n ints (pivots); d_work: 2n doubles; d_info: 1 int (zeroed here)
  CK(cudaMemsetAsync(d_info, 0, sizeof(int), s));
  const int upd_blocks = (int)std::max<long>(1, std::min<long>(152L * 8, ((long)n * ((n + 255) / 256) + 7) / 8));
  cudaEvent_t pe = profiler().begin(KK_GJ_BIG, s, 2L * n + 1);
  for (int k = 0; k < n; ++k) {
    k_gj_pivot<<<1, 1024, 0, s>>>(A, ld, n, k, d_work_int, d_work, d_work + n, d_info);
    k_gj_update<<<upd_blocks, 256, 0, s>>>(A, ld, n, k, d_work, d_work + n, d_info);
  }
  k_gj_colswap<<<1, 1024, 0, s>>>(A, ld, n, d_work_int, d_info);
  check_launch("big_inverse", 2L * n + 1);
  profiler().end(KK_GJ_BIG, s, pe);
}

void launch_p2p(DescStage& st, const std::vector<P2pDesc>& v, const double* pts, int N, const ifmm_kernel& k) {
  if (v.empty()) return;
  const int dof = kernel_dof(k);
  for (size_t i = 0; i < v.size() && registry().on; ++i) {
    req(v[i].dst, span(dof * v[i].ni, dof * v[i].nj, v[i].ld), "p2p.dst", i);
    if (v[i].i0 < 0 || v[i].j0 < 0 || v[i].i0 + v[i].ni > N || v[i].j0 + v[i].nj > N)
      throw Error(IFMM_EINVAL, "p2p point range");
  }
  const P2pDesc* d = st.push(v);
  prof_batch_tag() = (long)v.size();
  profiler().count(KK_P2P, 1);
  k_p2p<<<(unsigned)v.size(), 128, 0, st.stream>>>(d, (int)v.size(), pts, pts + N, pts + 2 * (long)N, k.scale, k.diag,
                                                   k.diag_im, k.wavenumber, dof);
  check_launch("k_p2p");
}

void launch_bd_fill(DescStage& st, const std::vector<BdBlockDesc>& v, const double* pts, int N, double scale,
                    double diag) {
  if (v.empty()) return;
  std::vector<int> tp(v.size() + 1, 0);
  for (size_t i = 0; i < v.size(); ++i) {
    const long t = (long)((v[i].n + 31) / 32) * ((v[i].n + 31) / 32);
    IFMM_REQUIRE(tp[i] + t < (1L << 31), IFMM_EINVAL, "block-diagonal blocks too large");
    tp[i + 1] = tp[i] + (int)t;
  }
  if (!tp.back()) return;
  const BdBlockDesc* d = st.push(v);
  const int* p = st.push(tp);
  cudaEvent_t pe = profiler().begin(KK_P2P, st.stream);
  k_bd_fill<<<(unsigned)tp.back(), 256, 0, st.stream>>>(d, p, (int)v.size(), pts, pts + N, pts + 2 * (long)N, scale,
                                                        diag);
  check_launch("k_bd_fill");
  profiler().end(KK_P2P, st.stream, pe);
}

void launch_interp(DescStage& st, const std::vector<InterpDesc>& v, const double* pts, int N, int p, int dof) {
  if (v.empty()) return;
  for (size_t i = 0; i < v.size() && registry().on; ++i) {
    req(v[i].dst, span(dof * p * p * p, dof * v[i].n, v[i].ld), "interp.dst", i);
    if (v[i].p0 < 0 || v[i].p0 + v[i].n > N) throw Error(IFMM_EINVAL, "interp point range");
  }
  const InterpDesc* d = st.push(v);
  prof_batch_tag() = (long)v.size();
  profiler().count(KK_INTERP, 1);
  k_interp<<<(unsigned)v.size(), 256, 0, st.stream>>>(d, (int)v.size(), pts, pts + N, pts + 2 * (long)N, p, dof);
  check_launch("k_interp");
}

void launch_m2l_table(cudaStream_t s, double* out, int p, double h, const ifmm_kernel& k) {
  profiler().count(KK_TABLES, 1);
  k_m2l_table<<<343, 256, 0, s>>>(out, p, h, k.scale, k.wavenumber, kernel_dof(k));
  check_launch("k_m2l_table");
}

void launch_m2m_table(cudaStream_t s, double* out, int p, int dof) {
  profiler().count(KK_TABLES, 1);
  k_m2m_table<<<8, 256, 0, s>>>(out, p, dof);
  check_launch("k_m2m_table");
}

void launch_matvec(cudaStream_t s, const double* pts, int N, const double* x, double* y, const ifmm_kernel& k) {
  cudaEvent_t pe = profiler().begin(KK_MATVEC, s);
  if (kernel_dof(k) == 2)
    k_matvec_c<<<(N + 255) / 256, 256, 0, s>>>(pts, pts + N, pts + 2 * (long)N, x, y, N, k.scale, k.diag, k.diag_im,
                                               k.wavenumber);
  else
    k_matvec<<<(N + 255) / 256, 256, 0, s>>>(pts, pts + N, pts + 2 * (long)N, x, y, N, k.scale, k.diag);
  check_launch("k_matvec");
  profiler().end(KK_MATVEC, s, pe);
}

void launch_gather_perm(cudaStream_t s, const double* src, const int* perm, double* dst, int n, int dof) {
  profiler().count(KK_PERM, 1);
  k_gather_perm<<<(n * dof + 255) / 256, 256, 0, s>>>(src, perm, dst, n, dof);
  check_launch("k_gather_perm");
}
void launch_scatter_perm(cudaStream_t s, const double* src, const int* perm, double* dst, int n, int dof) {
  profiler().count(KK_PERM, 1);
  k_scatter_perm<<<(n * dof + 255) / 256, 256, 0, s>>>(src, perm, dst, n, dof);
  check_launch("k_scatter_perm");
}

// raw launches with device-resident descriptors (solve plans, graph capture)
__global__ void k_conv_check(const double* x, int n, int sh, float* f, double* back) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = d2f_pow2(x[i], sh);
  f[i] = v;
  back[i] = f2d_pow2(v, -sh);
}

void launch_copy_dev(cudaStream_t s, const CopyDesc* d, int n) {
  if (n) k_copy<<<n, 256, 0, s>>>(d, n);
}

}  // namespace ifmm

extern "C" {
const char* ifmm_last_error(void) { return ifmm::last_error(); }

ifmm_status ifmm_gemm_check(int precision, int m, int n, int k, int ta, int tb, double alpha, const double* A, int lda,
                            const double* B, int ldb, double beta, double* C, int ldc) {
  using namespace ifmm;
  try {
    IFMM_REQUIRE(precision >= 0 && precision <= 2 && m >= 0 && n >= 0 && k >= 0 && m <= 8192 && n <= 8192 &&
                     k <= 8192 && A && B && C,
                 IFMM_EINVAL, "bad arguments");
    IFMM_REQUIRE(lda >= std::max(1, ta ? k : m) && ldb >= std::max(1, tb ? n : k) && ldc >= std::max(1, m),
                 IFMM_EINVAL, "leading dimension too small");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      cudaGetLastError();
      throw Error(IFMM_ECUDA, "no CUDA device");
    }
    const size_t na = (size_t)lda * (ta ? m : k), nb = (size_t)ldb * (tb ? k : n), nc = (size_t)ldc * n;
    DescStage st;
    cudaStream_t s;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    st.stream = s;
    DeviceArena mem;
    double* dA = mem.alloc(std::max<size_t>(na, 1));
    double* dB = mem.alloc(std::max<size_t>(nb, 1));
    double* dC = mem.alloc(std::max<size_t>(nc, 1));
    CK(cudaMemcpyAsync(dA, A, sizeof(double) * na, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dB, B, sizeof(double) * nb, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dC, C, sizeof(double) * nc, cudaMemcpyHostToDevice, s));
    std::vector<GemmDesc> v{gmm(dA, lda, ta, dB, ldb, tb, dC, ldc, m, n, k, alpha, beta)};
    launch_gemm(st, v, precision == IFMM_PREC_FP64 ? P64 : (precision == IFMM_PREC_FP32 ? P32 : P16));
    CK(cudaMemcpyAsync(C, dC, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    st.release();
    mem.release();
    CK(cudaStreamDestroy(s));
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

ifmm_status ifmm_qr_check(int precision, int pivoted, int m, int n, double* A, int ld, int* jpvt, int* k) {
  using namespace ifmm;
  try {
    IFMM_REQUIRE((precision == IFMM_PREC_FP64 || precision == IFMM_PREC_FP32) && m >= 1 && n >= 1 && m <= 65536 &&
                     n <= 1024 && ld >= m && A && (!pivoted || (jpvt && k)),
                 IFMM_EINVAL, "bad arguments");
    IFMM_REQUIRE((size_t)ld * n <= ((size_t)1 << 27), IFMM_EINVAL, "matrix too large");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      cudaGetLastError();
      throw Error(IFMM_ECUDA, "no CUDA device");
    }
    const int prec = precision == IFMM_PREC_FP64 ? P64 : P32;
    DescStage st;
    cudaStream_t s;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    st.stream = s;
    DeviceArena mem;
    const size_t na = (size_t)ld * n;
    double* dA = mem.alloc(na);
    int* dj = (int*)mem.alloc_bytes(sizeof(int) * (size_t)n);
    int* dk = (int*)mem.alloc_bytes(sizeof(int));
    CK(cudaMemcpyAsync(dA, A, sizeof(double) * na, cudaMemcpyHostToDevice, s));
    if (pivoted) {
      QrcpDesc q{};
      q.A = dA;
      q.ld = ld;
      q.m = m;
      q.n = n;
      q.tau_rel = 0.0;
      q.jpvt = dj;
      q.kout = dk;
      launch_qrcp(st, std::vector<QrcpDesc>{q}, prec);
    } else {
      launch_qr(st, std::vector<QrDesc>{QrDesc{dA, ld, m, n}}, prec);
    }
    CK(cudaMemcpyAsync(A, dA, sizeof(double) * na, cudaMemcpyDeviceToHost, s));
    if (pivoted) {
      CK(cudaMemcpyAsync(jpvt, dj, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(k, dk, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    st.release();
    mem.release();
    CK(cudaStreamDestroy(s));
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

ifmm_status ifmm_inv_check(int nmat, const int* n, double* A, int* info) {
  using namespace ifmm;
  try {
    IFMM_REQUIRE(nmat >= 0 && nmat <= 4096 && (nmat == 0 || (n && A && info)), IFMM_EINVAL, "bad arguments");
    size_t tot = 0;
    for (int i = 0; i < nmat; ++i) {
      IFMM_REQUIRE(n[i] >= 1 && n[i] <= 4096, IFMM_EINVAL, "matrix order must be in [1, 4096]");
      tot += (size_t)n[i] * n[i];
    }
    IFMM_REQUIRE(tot <= ((size_t)1 << 28), IFMM_EINVAL, "batch too large");
    if (nmat == 0) return IFMM_OK;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      cudaGetLastError();
      throw Error(IFMM_ECUDA, "no CUDA device");
    }
    DescStage st;
    cudaStream_t s;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    st.stream = s;
    DeviceArena mem;
    double* dA = mem.alloc(tot);
    int* dinfo = (int*)mem.alloc_bytes(sizeof(int) * (size_t)nmat);
    CK(cudaMemcpyAsync(dA, A, sizeof(double) * tot, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(dinfo, 0, sizeof(int) * (size_t)nmat, s));
    std::vector<InvDesc> v;
    size_t off = 0;
    for (int i = 0; i < nmat; ++i) {
      v.push_back(InvDesc{dA + off, n[i], n[i], dinfo + i, 0});
      off += (size_t)n[i] * n[i];
    }
    launch_inv(st, v);
    CK(cudaMemcpyAsync(A, dA, sizeof(double) * tot, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(info, dinfo, sizeof(int) * (size_t)nmat, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    st.release();
    mem.release();
    CK(cudaStreamDestroy(s));
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

ifmm_status ifmm_convert_check(const double* x, int64_t n, int shift, float* f, double* back) {
  try {
    IFMM_REQUIRE(x && f && back && n >= 0 && n <= (1 << 26), IFMM_EINVAL, "bad arguments");
    IFMM_REQUIRE(shift >= -200 && shift <= 200, IFMM_EINVAL, "shift out of range");
    if (n == 0) return IFMM_OK;
    double *dx = nullptr, *db = nullptr;
    float* df = nullptr;
    CK(cudaMalloc(&dx, sizeof(double) * n));
    CK(cudaMalloc(&db, sizeof(double) * n));
    CK(cudaMalloc(&df, sizeof(float) * n));
    cudaError_t e = cudaMemcpy(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      ifmm::k_conv_check<<<(unsigned)((n + 255) / 256), 256>>>(dx, (int)n, shift, df, db);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(f, df, sizeof(float) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(back, db, sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(db);
    cudaFree(df);
    CK(e);
    return IFMM_OK;
  } catch (const ifmm::Error& e) {
    ifmm::set_last_error(e.what());
    return e.code;
  }
}

ifmm_status ifmm_profile(int timing) {
  try {
    ifmm::profiler().reset();
    ifmm::profiler().timing = timing != 0;
    return IFMM_OK;
  } catch (const ifmm::Error& e) {
    ifmm::set_last_error(e.what());
    return e.code;
  }
}

ifmm_status ifmm_profile_query(int index, const char** name, int64_t* launches, double* ms) {
  try {
    if (index < 0 || index >= ifmm::KK_COUNT) {
      ifmm::set_last_error("profile index out of range");
      return IFMM_EINVAL;
    }
    ifmm::profiler().collect();
    if (name) *name = ifmm::kernel_kind_name(index);
    if (launches) *launches = ifmm::profiler().launches[index];
    if (ms) *ms = ifmm::profiler().ms[index];
    return IFMM_OK;
  } catch (const ifmm::Error& e) {
    ifmm::set_last_error(e.what());
    return e.code;
  }
}
}
