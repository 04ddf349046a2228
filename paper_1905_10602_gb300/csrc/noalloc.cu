// bem_matvec_noalloc: the direct-summation product y = A x without any device
// allocation, for callers that cannot allocate device memory -- code running
// where a memory pool is owned and sized by someone else (a host framework or
// runtime that forbids cudaMalloc/cudaFree during its own execution), or code
// that must not trigger the implicit synchronisation an allocation can cause.
//
// Scratch: a file-scope device array of NOALLOC_MAX_N * 16 bytes (4 MiB),
// holding the input in tree order (doubles) and its float-pair split.  Every
// GPU that loads this library keeps the array until the process exits.  Every
// element of the scratch that a call reads is written earlier in that same call,
// so nothing has to be cleared between calls; but all calls share the one array,
// so calls that overlap on the GPU (different streams, or threads) race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "common.h"
#include "pairs.cuh"

namespace {

constexpr int64_t NOALLOC_MAX_N = 262144;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_matvec_scratch[NOALLOC_MAX_N * 16];

std::mutex g_setup_mutex;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};

// x (caller order) -> scratch: tree-ordered doubles, then their float pairs
__global__ void k_na_prepare(const double* __restrict__ x, const int* __restrict__ perm, unsigned char* scratch,
                             int n) {
  double* a = (double*)scratch;
  float* qh = (float*)(a + NOALLOC_MAX_N);
  float* ql = qh + NOALLOC_MAX_N;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    const double v = x[perm[k]];
    a[k] = v;
    const float h = (float)v;
    qh[k] = h;
    ql[k] = (float)(v - (double)h);
  }
}

// one thread per target (tree order), sources through shared memory; the
// result goes straight to the caller's order through perm
__global__ void __launch_bounds__(256) k_na_matvec(const double* __restrict__ p64, const float* __restrict__ pdf,
                                                   const int* __restrict__ perm, const unsigned char* scratch,
                                                   double* __restrict__ y, int n, double scale, double diag,
                                                   int use_pairs) {
  const double* a = (const double*)scratch;
  const float* qh = (const float*)(a + NOALLOC_MAX_N);
  const float* ql = qh + NOALLOC_MAX_N;
  __shared__ float s[8][256];
  __shared__ double d[4][256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (use_pairs) {
    ifmm::df px = {0.f, 0.f}, py = {0.f, 0.f}, pz = {0.f, 0.f};
    if (i < n) {
      px = {pdf[i], pdf[n + i]};
      py = {pdf[2 * n + i], pdf[3 * n + i]};
      pz = {pdf[4 * n + i], pdf[5 * n + i]};
    }
    ifmm::df acc = {0.f, 0.f};
    for (int j0 = 0; j0 < n; j0 += blockDim.x) {
      const int j = j0 + threadIdx.x;
      if (j < n) {
        s[0][threadIdx.x] = pdf[j];
        s[1][threadIdx.x] = pdf[n + j];
        s[2][threadIdx.x] = pdf[2 * n + j];
        s[3][threadIdx.x] = pdf[3 * n + j];
        s[4][threadIdx.x] = pdf[4 * n + j];
        s[5][threadIdx.x] = pdf[5 * n + j];
        s[6][threadIdx.x] = qh[j];
        s[7][threadIdx.x] = ql[j];
      }
      __syncthreads();
      const int cnt = min((int)blockDim.x, n - j0);
      for (int t = 0; t < cnt; ++t) {
        // the pair arithmetic of the main float-pair matvec (pairs.cuh)
        const ifmm::df dx = ifmm::df_diff(px, s[0][t], s[1][t]);
        const ifmm::df dy = ifmm::df_diff(py, s[2][t], s[3][t]);
        const ifmm::df dz = ifmm::df_diff(pz, s[4][t], s[5][t]);
        const ifmm::df w = ifmm::df_rsqrt_fast(ifmm::df_sum3(ifmm::df_sq(dx), ifmm::df_sq(dy), ifmm::df_sq(dz)));
        const float ph = s[6][t] * w.h;
        const float pl = fmaf(s[6][t], w.h, -ph) + fmaf(s[6][t], w.l, s[7][t] * w.h);
        if (j0 + t != i) acc = ifmm::df_acc(acc, ph, pl);
      }
      __syncthreads();
    }
    if (i < n) y[perm[i]] = diag * a[i] + scale * ((double)acc.h + (double)acc.l);
  } else {
    double xi = 0, yi = 0, zi = 0;
    if (i < n) {
      xi = p64[i];
      yi = p64[n + i];
      zi = p64[2 * n + i];
    }
    double acc = 0.0;
    for (int j0 = 0; j0 < n; j0 += blockDim.x) {
      const int j = j0 + threadIdx.x;
      if (j < n) {
        d[0][threadIdx.x] = p64[j];
        d[1][threadIdx.x] = p64[n + j];
        d[2][threadIdx.x] = p64[2 * n + j];
        d[3][threadIdx.x] = a[j];
      }
      __syncthreads();
      const int cnt = min((int)blockDim.x, n - j0);
      for (int t = 0; t < cnt; ++t) {
        const double dx = xi - d[0][t], dy = yi - d[1][t], dz = zi - d[2][t];
        if (j0 + t != i) acc += d[3][t] * rsqrt(dx * dx + dy * dy + dz * dz);
      }
      __syncthreads();
    }
    if (i < n) y[perm[i]] = diag * a[i] + scale * acc;
  }
}

bool is_device_pointer(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

// Once per device, with that device current: the scratch array's device
// address.  Looking it up loads this file's module (the array and the kernel
// images), which the CUDA runtime otherwise does lazily at first use; the two
// kernels are loaded here too.  That load is the only allocation tied to this
// entry point, so it is done where the library allocates anyway.
cudaError_t setup_device(int dev, void** addr) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_matvec_scratch);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_prepare);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_matvec);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    }
    g_scratch_addr[dev] = p;
  }
  *addr = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

namespace ifmm {
// Called when a tree is first made resident on a device (ifmm_tree::ensure_device),
// so that a later bem_matvec_noalloc on that device finds its module loaded.  A
// failure here is not an error of the caller's call: bem_matvec_noalloc retries
// and reports it.
void noalloc_prepare_device(int dev) {
  if (dev < 0 || dev >= MAX_DEVICES) return;
  void* p = nullptr;
  (void)setup_device(dev, &p);
}
}  // namespace ifmm

extern "C" ifmm_status bem_matvec_noalloc(const ifmm_tree* t, const ifmm_kernel* k, const double* x, double* y,
                                          void* stream) {
  if (!t || !k || !x || !y) {
    ifmm::set_last_error("bem_matvec_noalloc: NULL argument");
    return IFMM_EINVAL;
  }
  if ((k->arith != IFMM_ARITH_FP64 && k->arith != IFMM_ARITH_DF) || k->wavenumber != 0.0) {
    ifmm::set_last_error("bem_matvec_noalloc: only the Laplace direct sums (IFMM_ARITH_FP64, IFMM_ARITH_DF) run "
                         "without allocating");
    return IFMM_EINVAL;
  }
  if (t->N > NOALLOC_MAX_N) {
    ifmm::set_last_error("bem_matvec_noalloc: the tree has more points than the " +
                         std::to_string(NOALLOC_MAX_N) + " its fixed scratch holds; use bem_matvec");
    return IFMM_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    cudaGetLastError();
    ifmm::set_last_error("bem_matvec_noalloc: no usable CUDA device");
    return IFMM_ECUDA;
  }
  if (!t->d_pts || !t->d_pts_df || !t->d_perm || t->device != dev) {
    ifmm::set_last_error("bem_matvec_noalloc: the tree is not resident on the current device "
                         "(an earlier ifmm_factor, bem_matvec or bem_gmres on it uploads it)");
    return IFMM_EINVAL;
  }
  if (!is_device_pointer(x, dev) || !is_device_pointer(y, dev)) {
    ifmm::set_last_error("bem_matvec_noalloc: x and y must be device memory of the current device");
    return IFMM_EINVAL;
  }
  if (x == y) {
    ifmm::set_last_error("bem_matvec_noalloc: x and y must not alias");
    return IFMM_EINVAL;
  }
  void* scratch = nullptr;
  const cudaError_t se = setup_device(dev, &scratch);
  if (se != cudaSuccess) {
    ifmm::set_last_error(std::string("bem_matvec_noalloc: device set-up failed: ") + cudaGetErrorString(se));
    return IFMM_ECUDA;
  }
  const int n = (int)t->N;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (n + 255) / 256;
  k_na_prepare<<<blocks, 256, 0, s>>>(x, t->d_perm, (unsigned char*)scratch, n);
  k_na_matvec<<<blocks, 256, 0, s>>>(t->d_pts, t->d_pts_df, t->d_perm, (const unsigned char*)scratch, y, n,
                                     k->scale, k->diag, k->arith == IFMM_ARITH_DF ? 1 : 0);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ifmm::set_last_error(std::string("bem_matvec_noalloc: launch failed: ") + cudaGetErrorString(e));
    return IFMM_ECUDA;
  }
  return IFMM_OK;
}
