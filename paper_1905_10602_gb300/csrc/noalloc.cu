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

namespace {

constexpr int64_t NOALLOC_MAX_N = 262144;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_matvec_scratch[NOALLOC_MAX_N * 16];

std::mutex g_setup_mutex;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};

struct fpair {
  float h, l;
};
__device__ __forceinline__ fpair fp_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ fpair fp_quick(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ fpair fp_add(fpair a, fpair b) {
  fpair s = fp_two_sum(a.h, b.h);
  return fp_quick(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ fpair fp_sub(fpair a, fpair b) {
  fpair s = fp_two_sum(a.h, -b.h);
  return fp_quick(s.h, s.l + (a.l - b.l));
}
__device__ __forceinline__ fpair fp_mul(fpair a, fpair b) {
  const float p = a.h * b.h;
  const float e = fmaf(a.h, b.h, -p);
  return fp_quick(p, e + (a.h * b.l + a.l * b.h));
}
__device__ __forceinline__ fpair fp_rsqrt(fpair x) {
  const float y0 = rsqrtf(x.h);
  const fpair t = fp_mul(x, fp_mul({y0, 0.f}, {y0, 0.f}));
  const fpair e = fp_sub({1.f, 0.f}, t);
  return fp_add({y0, 0.f}, fp_mul({0.5f * y0, 0.f}, e));
}

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
    fpair px = {0.f, 0.f}, py = {0.f, 0.f}, pz = {0.f, 0.f};
    if (i < n) {
      px = {pdf[i], pdf[n + i]};
      py = {pdf[2 * n + i], pdf[3 * n + i]};
      pz = {pdf[4 * n + i], pdf[5 * n + i]};
    }
    fpair acc = {0.f, 0.f};
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
        const fpair dx = fp_sub(px, {s[0][t], s[1][t]});
        const fpair dy = fp_sub(py, {s[2][t], s[3][t]});
        const fpair dz = fp_sub(pz, {s[4][t], s[5][t]});
        const fpair r2 = fp_add(fp_add(fp_mul(dx, dx), fp_mul(dy, dy)), fp_mul(dz, dz));
        if (j0 + t != i) acc = fp_add(acc, fp_mul({s[6][t], s[7][t]}, fp_rsqrt(r2)));
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

}  // namespace

extern "C" ifmm_status bem_matvec_noalloc(const ifmm_tree* t, const ifmm_kernel* k, const double* x, double* y,
                                          void* stream) {
  if (!t || !k || !x || !y) {
    ifmm::set_last_error("bem_matvec_noalloc: NULL argument");
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
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_matvec_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        ifmm::set_last_error(std::string("bem_matvec_noalloc: cudaGetSymbolAddress failed: ") +
                             cudaGetErrorString(e));
        return IFMM_ECUDA;
      }
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
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
