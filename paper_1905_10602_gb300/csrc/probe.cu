// Arithmetic peaks of the current GPU, measured by the library itself: the
// denominators of the per-phase rooflines (FP32 and FP64 FMA pipes, the
// TF32 / BF16 / FP64 warp-level tensor-core MMAs).  Each probe kernel runs
// independent dependency chains in registers (no memory traffic inside the
// loop), on enough CTAs to fill every SM several times over, and is timed with
// CUDA events after one warm-up launch.
#include <cuda_runtime.h>

#include <string>

#include "common.h"

namespace {

constexpr int kIters = 4096;

// 8 independent FMA chains per thread
template <typename T>
__global__ void __launch_bounds__(256) k_peak_fma(T* out, T seed) {
  T a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = seed + (T)(threadIdx.x + c);
  const T m = (T)0.999999, d = (T)1e-7;
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = a[c] * m + d;
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  if (s == (T)-12345.0) out[blockIdx.x] = s;
}

// 4 independent accumulator tiles per warp
__global__ void __launch_bounds__(256) k_peak_tf32(float* out, unsigned seed) {
  unsigned a[4] = {seed, seed ^ 1u, seed ^ 2u, seed ^ 3u}, b[2] = {seed ^ 5u, seed ^ 7u};
  float c[4][4] = {};
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int t = 0; t < 4; ++t)
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(c[t][0]), "+f"(c[t][1]), "+f"(c[t][2]), "+f"(c[t][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  float s = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) s += c[t][0] + c[t][1] + c[t][2] + c[t][3];
  if (s == -12345.f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_bf16(float* out, unsigned seed) {
  unsigned a[4] = {seed, seed ^ 1u, seed ^ 2u, seed ^ 3u}, b[2] = {seed ^ 5u, seed ^ 7u};
  float c[4][4] = {};
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int t = 0; t < 4; ++t)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(c[t][0]), "+f"(c[t][1]), "+f"(c[t][2]), "+f"(c[t][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  float s = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) s += c[t][0] + c[t][1] + c[t][2] + c[t][3];
  if (s == -12345.f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_dmma(double* out, double seed) {
  const double a = seed, b = seed * 0.5;
  double c[4][2] = {};
  for (int it = 0; it < kIters / 4; ++it)
#pragma unroll
    for (int t = 0; t < 4; ++t)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(c[t][0]), "+d"(c[t][1])
                   : "d"(a), "d"(b));
  double s = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) s += c[t][0] + c[t][1];
  if (s == -12345.0) out[blockIdx.x] = s;
}

}  // namespace

extern "C" ifmm_status ifmm_probe_peak(int kind, double* tflops) {
  if (!tflops || kind < 0 || kind > 4) {
    ifmm::set_last_error("ifmm_probe_peak: bad argument");
    return IFMM_EINVAL;
  }
  *tflops = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
    cudaGetLastError();
    ifmm::set_last_error("ifmm_probe_peak: no CUDA device");
    return IFMM_ECUDA;
  }
  const int blocks = sms * 8, threads = 256;
  void* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double flops = 0.0;
  float ms = 0.f;
  cudaError_t err = cudaMalloc(&out, sizeof(double) * blocks);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
    cudaEventRecord(e0);
    switch (kind) {
      case 0:  // FP32 FFMA
        k_peak_fma<float><<<blocks, threads>>>((float*)out, 1.0f);
        flops = 2.0 * 8 * kIters * (double)blocks * threads;
        break;
      case 1:  // FP64 DFMA
        k_peak_fma<double><<<blocks, threads>>>((double*)out, 1.0);
        flops = 2.0 * 8 * kIters * (double)blocks * threads;
        break;
      case 2:  // TF32 mma.sync m16n8k8
        k_peak_tf32<<<blocks, threads>>>((float*)out, 0x3f800000u);
        flops = 2.0 * 16 * 8 * 8 * 4 * (double)kIters * blocks * (threads / 32);
        break;
      case 3:  // BF16 mma.sync m16n8k16
        k_peak_bf16<<<blocks, threads>>>((float*)out, 0x3f803f80u);
        flops = 2.0 * 16 * 8 * 16 * 4 * (double)kIters * blocks * (threads / 32);
        break;
      case 4:  // FP64 mma.sync m8n8k4
        k_peak_dmma<<<blocks, threads>>>((double*)out, 1.0);
        flops = 2.0 * 8 * 8 * 4 * 4 * (double)(kIters / 4) * blocks * (threads / 32);
        break;
    }
    cudaEventRecord(e1);
    err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) {
    cudaGetLastError();
    ifmm::set_last_error(std::string("ifmm_probe_peak: ") + cudaGetErrorString(err));
    return IFMM_ECUDA;
  }
  *tflops = flops / (ms * 1e-3) / 1e12;
  return IFMM_OK;
}
