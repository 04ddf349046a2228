// Batched dense linear algebra used by every step of the factorization and
// the solve: block copies, variable-size GEMM, Gauss-Jordan inversion with
// partial pivoting, Householder QR (R factor), one-sided Jacobi SVD, GEMV.
//
// Every matrix is column-major with a leading dimension (BLAS convention).
// One descriptor describes one problem; a launch covers a batch of problems of
// different sizes (the nodes of one color of one level).  Kernels never wait
// on anything but __syncthreads, and every index is bounded by the sizes in
// the descriptor.
#pragma once

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "descs.h"

namespace ifmm {

__device__ __forceinline__ int find_desc(const int* ptr, int ndesc, int t) {
  int lo = 0, hi = ndesc - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (ptr[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- copies
__global__ void k_copy(const CopyDesc* __restrict__ d, int nd) {
  const int b = blockIdx.x;
  if (b >= nd) return;
  const CopyDesc D = d[b];
  // warps over columns, lanes over rows (no per-element index division); the
  // common alpha = 1, beta in {0, 1} cases take no FP64 multiply
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int mode = (D.alpha == 1.0 && D.beta == 0.0) ? 0 : ((D.alpha == 1.0 && D.beta == 1.0) ? 1 : 2);
  for (int j = threadIdx.x >> 5; j < D.cols; j += nw)
    for (int i = lane; i < D.rows; i += 32) {
      double v = 0.0;
      if (D.src) v = D.trans ? D.src[j + (long)i * D.lds] : D.src[i + (long)j * D.lds];
      double* o = D.dst + i + (long)j * D.ldd;
      *o = mode == 0 ? v : (mode == 1 ? *o + v : ((D.beta == 0.0) ? D.alpha * v : D.alpha * v + D.beta * (*o)));
    }
}

// ---------------------------------------------------------------- small problems
// A warp per descriptor (8 per CTA) for blocks of at most 1024 elements.
__global__ void k_copy_small(const CopyDesc* __restrict__ d, int nd) {
  const int di = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (di >= nd) return;
  const CopyDesc D = d[di];
  const int total = D.rows * D.cols;
  const int mode = (D.alpha == 1.0 && D.beta == 0.0) ? 0 : ((D.alpha == 1.0 && D.beta == 1.0) ? 1 : 2);
  for (int e = lane; e < total; e += 32) {
    const int i = e % D.rows, j = e / D.rows;
    double v = 0.0;
    if (D.src) v = D.trans ? D.src[j + (long)i * D.lds] : D.src[i + (long)j * D.lds];
    double* o = D.dst + i + (long)j * D.ldd;
    *o = mode == 0 ? v : (mode == 1 ? *o + v : ((D.beta == 0.0) ? D.alpha * v : D.alpha * v + D.beta * (*o)));
  }
}

// ---------------------------------------------------------------- FP64 <-> FP32 on the integer pipes
// GB300 executes double arithmetic and double<->float conversions on its narrow
// FP64 pipe (about 2 operations per clock per SM).  The FP32 kernels read and
// write FP64 storage, so they convert with integer operations on the IEEE-754
// fields instead, folding an optional power-of-two scale 2^sh into the
// exponent.  No path of either function uses a floating-point instruction (the
// compiler would evaluate a rare-path hardware conversion on every call and
// select).  d2f_pow2 rounds to nearest with ties away from zero (IEEE binary64
// -> binary32 keeps the top 23 of 52 fraction bits; the first dropped bit
// decides); results below the binary32 normal range become signed zero, above
// it infinity; infinity and NaN stay infinity and (quiet) NaN.  f2d_pow2 widens
// exactly (binary32 subnormals included); results below the binary64 normal
// range become signed zero, above it infinity.
__device__ __forceinline__ float d2f_pow2(double d, int sh) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned ah = hi & 0x7fffffffu, sg = hi & 0x80000000u;
  if (ah >= 0x7ff00000u) {
    const bool nan = ah > 0x7ff00000u || lo != 0u;
    return __uint_as_float(sg | 0x7f800000u | (nan ? 0x400000u | ((ah & 0x000fffffu) << 3) : 0u));
  }
  const int e = (int)(ah >> 20) + sh;  // biased binary64 exponent after scaling
  if (ah < 0x00100000u || e <= 896) return __uint_as_float(sg);
  if (e >= 1151) return __uint_as_float(sg | 0x7f800000u);
  unsigned f = ((unsigned)(e - 896) << 23) | ((ah & 0x000fffffu) << 3) | (lo >> 29);
  f += (lo >> 28) & 1u;  // a carry into the exponent is the correct rounding
  return __uint_as_float(sg | f);
}
__device__ __forceinline__ double f2d_pow2(float f, int sh) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7fffffffu, sg = u & 0x80000000u;
  if (a == 0) return __hiloint2double((int)sg, 0);
  if (a >= 0x7f800000u) {
    const unsigned m = a & 0x007fffffu;  // NaN payload (0: infinity)
    return __hiloint2double((int)(sg | 0x7ff00000u | (m ? 0x80000u | (m >> 3) : 0u)), (int)(m << 29));
  }
  unsigned mant;
  int e;  // biased binary64 exponent
  if (a < 0x00800000u) {  // subnormal: a 2^-149, normalised
    const int lz = __clz((int)a) - 8;
    mant = (a << lz) & 0x007fffffu;
    e = 897 - lz + sh;
  } else {
    mant = a & 0x007fffffu;
    e = (int)(a >> 23) + 896 + sh;
  }
  if (e <= 0) return __hiloint2double((int)sg, 0);
  if (e >= 2047) return __hiloint2double((int)(sg | 0x7ff00000u), 0);
  return __hiloint2double((int)(sg | ((unsigned)e << 20) | (mant >> 3)), (int)(mant << 29));
}
// biased binary64 exponent of |d| (0 for zero and subnormals, 2047 for inf/NaN)
__device__ __forceinline__ int dexp(double d) { return (int)(((unsigned)__double2hiint(d) & 0x7fffffffu) >> 20); }

// value of a double as the arithmetic type TC, times 2^sh
template <typename TC>
__device__ __forceinline__ TC ld_tc(double d, int sh = 0) {
  if constexpr (sizeof(TC) == 4)
    return d2f_pow2(d, sh);
  else
    return sh ? ldexp(d, sh) : d;
}
// a TC value times 2^sh, as a double
template <typename TC>
__device__ __forceinline__ double st_tc(TC v, int sh = 0) {
  if constexpr (sizeof(TC) == 4)
    return f2d_pow2(v, sh);
  else
    return sh ? ldexp(v, sh) : v;
}

// RB: the operands are rounded to bfloat16 before the (FP32) multiply-add.
__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
template <typename TC, bool RB>
__device__ __forceinline__ TC stage_val(double v) {
  if constexpr (RB)
    return (TC)round_bf16(d2f_pow2(v, 0));
  else
    return ld_tc<TC>(v);
}

// One warp per GEMM with m, n <= 32 (any k), four warps per CTA.  The operands
// are staged in chunks of 16 along k through the warp's shared memory (one
// load and conversion per element); lane j accumulates column j of C in
// registers, reading the A chunk by broadcast.
template <typename TC, bool RB = false>
__global__ void __launch_bounds__(128) k_gemm_small(const GemmDesc* __restrict__ d, int nd) {
  constexpr int KC = 16;
  __shared__ TC As[4][32][KC + 1];
  __shared__ TC Bs[4][KC][33];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int di = blockIdx.x * 4 + w;
  if (di >= nd) return;
  const GemmDesc D = d[di];
  const int m = D.m, n = D.n;
  TC acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = (TC)0;
  for (int k0 = 0; k0 < D.k; k0 += KC) {
    const int kc = min(KC, D.k - k0);
    // A chunk: row i = lane, columns k0..k0+kc-1 (rows >= m and columns >= kc zero)
    for (int kk = 0; kk < KC; ++kk) {
      double v = 0.0;
      if (lane < m && kk < kc) {
        const int c = k0 + kk;
        v = D.ta ? D.A[c + (long)lane * D.lda] : D.A[lane + (long)c * D.lda];
      }
      As[w][lane][kk] = stage_val<TC, RB>(v);
    }
    // B chunk: rows k0..k0+kc-1 (kk = lane % 16), columns j
    for (int x = lane; x < KC * 32; x += 32) {
      const int kk = x % KC, j = x / KC;
      double v = 0.0;
      if (kk < kc && j < n) {
        const int r = k0 + kk;
        v = D.tb ? D.B[j + (long)r * D.ldb] : D.B[r + (long)j * D.ldb];
      }
      Bs[w][kk][j] = stage_val<TC, RB>(v);
    }
    __syncwarp();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      const TC b = Bs[w][kk][lane];
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] += As[w][i][kk] * b;
    }
    __syncwarp();
  }
  if (lane < n) {
    double* o = D.C + (long)lane * D.ldc;
    const TC al = ld_tc<TC>(D.alpha);
    const int bm = D.beta == 0.0 ? 0 : (D.beta == 1.0 ? 1 : 2);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      if (i >= m) break;
      const double v = st_tc<TC>(al * acc[i]);
      o[i] = bm == 0 ? v : (bm == 1 ? o[i] + v : v + D.beta * o[i]);
    }
  }
}

// ---------------------------------------------------------------- GEMM
// 64 x 64 output tile per CTA, 256 threads, 4 x 4 outputs per thread, K in
// slices of 16 staged through shared memory.  TC is the arithmetic type
// (double for the FP64 path, float for the reduced-precision modes).
template <typename TC, bool RB = false>
__global__ void __launch_bounds__(256) k_gemm(const GemmDesc* __restrict__ d, const int* __restrict__ tile_ptr, int nd) {
  const int di = find_desc(tile_ptr, nd, blockIdx.x);
  const GemmDesc D = d[di];
  const int local = blockIdx.x - tile_ptr[di];
  const int tiles_m = (D.m + 63) >> 6;
  const int tm = local % tiles_m, tn = local / tiles_m;
  const int row0 = tm * 64, col0 = tn * 64;
  __shared__ TC As[16][64 + 1];
  __shared__ TC Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  TC acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (TC)0;
  for (int k0 = 0; k0 < D.k; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      {
        const int i = e & 63, kk = e >> 6;
        const int r = row0 + i, c = k0 + kk;
        double v = 0.0;
        if (r < D.m && c < D.k) v = D.ta ? D.A[c + (long)r * D.lda] : D.A[r + (long)c * D.lda];
        As[kk][i] = stage_val<TC, RB>(v);
      }
      {
        const int kk = e & 15, j = e >> 4;
        const int r = k0 + kk, c = col0 + j;
        double v = 0.0;
        if (r < D.k && c < D.n) v = D.tb ? D.B[c + (long)r * D.ldb] : D.B[r + (long)c * D.ldb];
        Bs[kk][j] = stage_val<TC, RB>(v);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      TC a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
    }
    __syncthreads();
  }
  const TC al = ld_tc<TC>(D.alpha);
  const int bm = D.beta == 0.0 ? 0 : (D.beta == 1.0 ? 1 : 2);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= D.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx + 16 * j;
      if (c >= D.n) continue;
      double* o = D.C + r + (long)c * D.ldc;
      const double v = st_tc<TC>(al * acc[i][j]);
      *o = bm == 0 ? v : (bm == 1 ? *o + v : v + D.beta * (*o));
    }
  }
}

// ---------------------------------------------------------------- tensor-core GEMM (reduced precision)
// C = alpha op(A) op(B) + beta C on the warp-level tensor cores, FP32
// accumulation, FP64 storage.  MODE 0 (the FP32 mode): each operand x is split
// into a TF32 head h = rn_tf32(x) and a TF32-rounded tail l = rn_tf32(x - h),
// and a*b is taken as a_l*b_h + a_h*b_l + a_h*b_h (the l*l term, below
// 2^-22 |a b|, is dropped: Ootomo and Yokota's 3xTF32 scheme), three
// m16n8k8 MMAs per product tile.  MODE 1 (the BF16 mode): the operands are
// rounded to bfloat16 and multiplied by one m16n8k16 MMA.
//
// A 128 x 128 output tile per CTA of 8 warps (2 x 4, 64 x 32 per warp), K in
// slices of 16.  The FP64 slices are copied to shared memory with cp.async
// (8-byte copies, zero-filled outside the matrices) into two stages, so the
// next slice is in flight while the current one is used; each slice is then
// converted once to FP32 on the integer pipes (d2f_pow2) and, in MODE 0, split
// into TF32 head and tail, k-major with 8 words of padding (fragment loads
// free of bank conflicts).  The epilogue goes through shared memory as a
// column-major tile and every warp writes whole column segments of C.
// x rounded to TF32 (10 fraction bits), to nearest with ties away from zero,
// by integer operations on its bits: adding half a TF32 unit to the magnitude
// and clearing the 13 dropped bits (a carry into the exponent is the correct
// rounding).  Infinity stays infinity and NaN stays NaN (its quiet bit, which
// survives the truncation, is set).  The conversion instruction would run on
// the narrow FP64 pipe.
__device__ __forceinline__ unsigned tf32_rn(float x) {
  const unsigned u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return (u & 0x7fffffu) ? ((u | 0x400000u) & 0xffffe000u) : u;
  return (u + 0x1000u) & 0xffffe000u;
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};\n"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};\n"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// two floats as a bfloat16 pair (round to nearest even), lo in the low half
__device__ __forceinline__ unsigned bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}
// 8-byte asynchronous copy global -> shared; nbytes 0 writes zeros
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, int nbytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(nbytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 16, kTcPad = 136, kTcPC = 132;
// shared memory: two FP64 stages (A and B slices), then the converted slice
// (MODE 0: A head, A tail, B head, B tail; MODE 1: A, B); the epilogue tile
// (128 x 132 floats) reuses the FP64 stages
constexpr int kTcStageBytes = 2 * (kTcBM * kTcBK + kTcBK * kTcBN) * 8;
constexpr int kTcEpiBytes = kTcBN * kTcPC * 4;
constexpr int kTcLowBytes = kTcStageBytes > kTcEpiBytes ? kTcStageBytes : kTcEpiBytes;
constexpr int gemm_tc_smem_bytes(int mode) { return kTcLowBytes + (mode == 0 ? 4 : 2) * kTcBK * kTcPad * 4; }

template <int MODE>
__global__ void __launch_bounds__(256, 2) k_gemm_tc(const GemmDesc* __restrict__ d, const int* __restrict__ tile_ptr,
                                                     int nd) {
  constexpr int BM = kTcBM, BN = kTcBN, BK = kTcBK, P = kTcPad;
  extern __shared__ __align__(16) unsigned char tcsm[];
  double* S64 = (double*)tcsm;                   // [2][BM*BK + BK*BN]
  unsigned* Cv = (unsigned*)(tcsm + kTcLowBytes);  // converted slice
  const int di = find_desc(tile_ptr, nd, blockIdx.x);
  const GemmDesc& D = d[di];
  const int local = blockIdx.x - tile_ptr[di];
  const int tiles_m = (D.m + BM - 1) / BM;
  const int row0 = (local % tiles_m) * BM, col0 = (local / tiles_m) * BN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;  // 2 x 4 warps, warp tile 64 x 32
  const int g = lane >> 2, t = lane & 3;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
  // staging order of a slice: A element (i, kk) at sa(i, kk), B element (kk, j)
  // at sb(kk, j), along the contiguous axis of each matrix in memory
  auto issue = [&](int k0, int stage) {
    double* SA = S64 + stage * (BM * BK + BK * BN);
    double* SB = SA + BM * BK;
#pragma unroll
    for (int x = 0; x < BM * BK / 256; ++x) {
      const int e = tid + x * 256;
      int i, kk;
      if (D.ta) { kk = e % BK; i = e / BK; } else { i = e % BM; kk = e / BM; }
      const int r = row0 + i, c = k0 + kk;
      const bool in = r < D.m && c < D.k;
      const double* src = in ? (D.ta ? D.A + c + (long)r * D.lda : D.A + r + (long)c * D.lda) : D.A;
      cp_async8(SA + e, src, in ? 8 : 0);
    }
#pragma unroll
    for (int x = 0; x < BK * BN / 256; ++x) {
      const int e = tid + x * 256;
      int kk, j;
      if (D.tb) { j = e % BN; kk = e / BN; } else { kk = e % BK; j = e / BK; }
      const int r = k0 + kk, c = col0 + j;
      const bool in = r < D.k && c < D.n;
      const double* src = in ? (D.tb ? D.B + c + (long)r * D.ldb : D.B + r + (long)c * D.ldb) : D.B;
      cp_async8(SB + e, src, in ? 8 : 0);
    }
    cp_async_commit();
  };
  // converts stage `stage` into Cv: k-major rows of P words
  auto convert = [&](int stage) {
    const double* SA = S64 + stage * (BM * BK + BK * BN);
    const double* SB = SA + BM * BK;
#pragma unroll
    for (int x = 0; x < BM * BK / 256; ++x) {
      const int e = tid + x * 256;
      const int i = e % BM, kk = e / BM;
      const float f = d2f_pow2(D.ta ? SA[kk + i * BK] : SA[i + kk * BM], 0);
      if constexpr (MODE == 0) {
        const unsigned h = tf32_rn(f);
        Cv[kk * P + i] = h;
        Cv[(BK + kk) * P + i] = tf32_rn(f - __uint_as_float(h));
      } else {
        Cv[kk * P + i] = __float_as_uint(f);
      }
    }
    unsigned* CB = Cv + (MODE == 0 ? 2 : 1) * BK * P;
#pragma unroll
    for (int x = 0; x < BK * BN / 256; ++x) {
      const int e = tid + x * 256;
      const int j = e % BN, kk = e / BN;
      const float f = d2f_pow2(D.tb ? SB[j + kk * BN] : SB[kk + j * BK], 0);
      if constexpr (MODE == 0) {
        const unsigned h = tf32_rn(f);
        CB[kk * P + j] = h;
        CB[(BK + kk) * P + j] = tf32_rn(f - __uint_as_float(h));
      } else {
        CB[kk * P + j] = __float_as_uint(f);
      }
    }
  };
  const int nk = (D.k + BK - 1) / BK;
  if (nk > 0) issue(0, 0);
  for (int ks = 0; ks < nk; ++ks) {
    if (ks + 1 < nk) {
      issue((ks + 1) * BK, (ks + 1) & 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // slice ks landed for every thread; the previous MMAs are done with Cv
    convert(ks & 1);
    __syncthreads();
    const unsigned* Ah = Cv + wm * 64;
    const unsigned* Bh = Cv + (MODE == 0 ? 2 : 1) * BK * P + wn * 32;
    if constexpr (MODE == 0) {
      const unsigned* Al = Ah + BK * P;
      const unsigned* Bl = Bh + BK * P;
#pragma unroll
      for (int k8 = 0; k8 < BK; k8 += 8) {
        unsigned bh[4][2], bl[4][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          bh[j][0] = Bh[(k8 + t) * P + j * 8 + g];
          bh[j][1] = Bh[(k8 + t + 4) * P + j * 8 + g];
          bl[j][0] = Bl[(k8 + t) * P + j * 8 + g];
          bl[j][1] = Bl[(k8 + t + 4) * P + j * 8 + g];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int m0 = i * 16 + g;
          const unsigned ah[4] = {Ah[(k8 + t) * P + m0], Ah[(k8 + t) * P + m0 + 8], Ah[(k8 + t + 4) * P + m0],
                                  Ah[(k8 + t + 4) * P + m0 + 8]};
          const unsigned al[4] = {Al[(k8 + t) * P + m0], Al[(k8 + t) * P + m0 + 8], Al[(k8 + t + 4) * P + m0],
                                  Al[(k8 + t + 4) * P + m0 + 8]};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            mma_tf32(acc[i][j], al, bh[j]);
            mma_tf32(acc[i][j], ah, bl[j]);
            mma_tf32(acc[i][j], ah, bh[j]);
          }
        }
      }
    } else {
      const float* As = (const float*)Ah;
      const float* Bs = (const float*)Bh;
      unsigned b[4][2];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float* bb = Bs + j * 8 + g;
        b[j][0] = bf16x2(bb[(2 * t) * P], bb[(2 * t + 1) * P]);
        b[j][1] = bf16x2(bb[(2 * t + 8) * P], bb[(2 * t + 9) * P]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float* aa = As + i * 16 + g;
        unsigned a[4];
        a[0] = bf16x2(aa[(2 * t) * P], aa[(2 * t + 1) * P]);
        a[1] = bf16x2(aa[(2 * t) * P + 8], aa[(2 * t + 1) * P + 8]);
        a[2] = bf16x2(aa[(2 * t + 8) * P], aa[(2 * t + 9) * P]);
        a[3] = bf16x2(aa[(2 * t + 8) * P + 8], aa[(2 * t + 9) * P + 8]);
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a, b[j]);
      }
    }
  }
  __syncthreads();  // every warp is done with the stages before the epilogue reuses them
  float* Cs = (float*)tcsm;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = wm * 64 + i * 16 + g, c = wn * 32 + j * 8 + 2 * t;
      Cs[c * kTcPC + r] = acc[i][j][0];
      Cs[(c + 1) * kTcPC + r] = acc[i][j][1];
      Cs[c * kTcPC + r + 8] = acc[i][j][2];
      Cs[(c + 1) * kTcPC + r + 8] = acc[i][j][3];
    }
  __syncthreads();
  const float al = d2f_pow2(D.alpha, 0);
  const int bm = D.beta == 0.0 ? 0 : (D.beta == 1.0 ? 1 : 2);
  const int mr = min(BM, D.m - row0), nc = min(BN, D.n - col0);
  for (int c = warp; c < nc; c += 8) {
    double* o = D.C + row0 + (long)(col0 + c) * D.ldc;
    for (int r = lane; r < mr; r += 32) {
      const double v = f2d_pow2(al * Cs[c * kTcPC + r], 0);
      o[r] = bm == 0 ? v : (bm == 1 ? o[r] + v : v + D.beta * o[r]);
    }
  }
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum; scratch holds >= 32 doubles; every thread gets the result
__device__ double block_sum(double v, double* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += scratch[i];
  return s;
}

// ---------------------------------------------------------------- Gauss-Jordan inverse
// One CTA per matrix.  Step k: pick the row of largest |A(i,k)|, i >= k (ties:
// smallest i), swap it into row k, scale row k, eliminate column k from every
// other row; finally undo the row interchanges as column interchanges in
// reverse order.  The matrix is worked on in shared memory when n*n doubles fit
// in smem_mat bytes, else in place in global memory.  Dynamic shared memory:
// smem_mat bytes + 2n doubles + n ints.
__global__ void k_inv(const InvDesc* __restrict__ d, int nd, int smem_mat) {
  if ((int)blockIdx.x >= nd) return;
  const InvDesc D = d[blockIdx.x];
  const int n = D.n;
  extern __shared__ double sm[];
  const bool in_smem = (size_t)n * n * sizeof(double) <= (size_t)smem_mat;
  double* A = in_smem ? sm : D.A;
  const long ld = in_smem ? n : D.ld;
  double* rowk = sm + smem_mat / sizeof(double);
  double* colk = rowk + n;
  int* piv = (int*)(colk + n);
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_p;
  __shared__ int s_bad;
  __shared__ double s_inv;
  if (threadIdx.x == 0) s_bad = 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (in_smem)
    for (int j = w; j < n; j += nw)
      for (int i = lane; i < n; i += 32) A[i + (long)j * n] = D.A[i + (long)j * D.ld];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
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
      if (!(bv > 0.0) || b >= n) { s_bad = k + 1; b = k; }
      s_p = b;
      piv[k] = b;
    }
    __syncthreads();
    if (s_bad) break;
    const int p = s_p;
    if (p != k) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double t = A[k + j * ld];
        A[k + j * ld] = A[p + j * ld];
        A[p + j * ld] = t;
      }
      __syncthreads();  // p is the same in every thread: row k complete before it is read below
    }
    // the reciprocal of the pivot once (an FP64 divide is a long FP64 sequence)
    if (threadIdx.x == 0) s_inv = 1.0 / A[k + k * ld];
    __syncthreads();
    const double inv = s_inv;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double v = (j == k) ? inv : A[k + j * ld] * inv;
      rowk[j] = v;
      A[k + j * ld] = v;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = (i == k) ? 0.0 : A[i + k * ld];
    __syncthreads();
    // warps over columns, lanes over rows (no per-element index division)
    for (int j = w; j < n; j += nw) {
      const double rj = rowk[j];
      double* cj = A + (long)j * ld;
      for (int i = lane; i < n; i += 32) {
        if (i == k) continue;
        const double a = (j == k) ? 0.0 : cj[i];
        cj[i] = a - colk[i] * rj;
      }
    }
    __syncthreads();
  }
  if (s_bad) {
    if (threadIdx.x == 0) D.info[0] = s_bad;
    return;
  }
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
  if (in_smem)
    for (int j = w; j < n; j += nw)
      for (int i = lane; i < n; i += 32) D.A[i + (long)j * D.ld] = A[i + (long)j * n];
  if (threadIdx.x == 0) D.info[0] = 0;
}

// Batched Gauss-Jordan for matrices too large for shared memory: one launch
// pair per pivot step k over all matrices of the batch (k_gjb_pivot: a CTA per
// matrix picks, swaps and scales the pivot row; k_gjb_update: a 2-D grid, one
// row of CTAs per matrix, eliminates column k), then k_gjb_colswap.  work holds
// 2n doubles and n ints per matrix at work_off[b].
__global__ void k_gjb_pivot(const InvDesc* __restrict__ d, int nd, int k, double* __restrict__ work,
                            const long* __restrict__ work_off) {
  const int b = blockIdx.x;
  if (b >= nd) return;
  const InvDesc D = d[b];
  const int n = D.n;
  if (k >= n || D.info[0] != 0) return;
  double* A = D.A;
  const long ld = D.ld;
  double* rowk = work + work_off[b];
  double* colk = rowk + n;
  int* piv = (int*)(colk + n);
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_p;
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
    int bb = n;
    for (int i = 0; i < nw; ++i)
      if (red_v[i] > bv || (red_v[i] == bv && red_i[i] < bb)) { bv = red_v[i]; bb = red_i[i]; }
    if (!(bv > 0.0) || bb >= n) {
      D.info[0] = k + 1;
      bb = k;
    }
    s_p = bb;
    piv[k] = bb;
  }
  __syncthreads();
  if (D.info[0] != 0) return;
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
  for (int j = threadIdx.x; j < n; j += blockDim.x) rowk[j] = (j == k) ? inv : A[k + j * ld] * inv;
  for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = (i == k) ? 0.0 : A[i + k * ld];
}

__global__ void k_gjb_update(const InvDesc* __restrict__ d, int nd, int k, const double* __restrict__ work,
                             const long* __restrict__ work_off) {
  const int b = blockIdx.y;
  if (b >= nd) return;
  const InvDesc D = d[b];
  const int n = D.n;
  if (k >= n || D.info[0] != 0) return;
  double* A = D.A;
  const long ld = D.ld;
  const double* rowk = work + work_off[b];
  const double* colk = rowk + n;
  // columns over (CTA, warp), lanes over rows (no per-element index division)
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = blockIdx.x * nw + (threadIdx.x >> 5); j < n; j += gridDim.x * nw) {
    const double rj = rowk[j];
    double* cj = A + (long)j * ld;
    for (int i = lane; i < n; i += 32) {
      if (i == k) {
        cj[i] = rj;
      } else {
        const double a = (j == k) ? 0.0 : cj[i];
        cj[i] = a - colk[i] * rj;
      }
    }
  }
}

__global__ void k_gjb_colswap(const InvDesc* __restrict__ d, int nd, const double* __restrict__ work,
                              const long* __restrict__ work_off) {
  const int b = blockIdx.x;
  if (b >= nd) return;
  const InvDesc D = d[b];
  const int n = D.n;
  if (D.info[0] != 0) return;
  double* A = D.A;
  const long ld = D.ld;
  const int* piv = (const int*)(work + work_off[b] + 2 * n);
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

// ---------------------------------------------------------------- Householder QR
// One CTA per matrix.  Column k: v = x - alpha e1 with alpha = -sign(x_0)||x||,
// H = I - 2 v v^T / (v^T v) applied to the trailing columns (one warp per column).
// Storage is double; TC is the arithmetic type of the dot products and updates.
template <typename TC>
__device__ __forceinline__ TC warp_sum_t(TC v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Apply H = I - t v v^T (v_0 = 1, v_i = x_i for i >= 1) to the trailing
// columns k+1..n-1 of A (rows k..k+len-1).  Each column's dot product and
// update is split into S row segments when there are fewer trailing columns
// than warps; the S partial sums are added in a fixed order (deterministic).
// partial: shared memory of >= max(n, warps) doubles.  Ends with __syncthreads.
template <typename TC>
__device__ void apply_reflector(double* A, long ld, int k, int n, int len, const double* x, TC t, double* partial) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const int nt = n - k - 1;
  if (nt <= 0) return;
  int S = nw / nt;
  const int smax = (len + 63) / 64;
  if (S > smax) S = smax;
  if (S < 1) S = 1;
  const int seg = (len + S - 1) / S;
  const int items = nt * S;
  for (int it = w; it < items; it += nw) {
    const int jj = it / S, sg = it % S;
    const double* y = A + k + (long)(k + 1 + jj) * ld;
    const int r0 = sg * seg, r1 = min(len, r0 + seg);
    TC dot = 0;
    for (int i = r0 + lane; i < r1; i += 32) dot += (i == 0 ? (TC)1 : (TC)x[i]) * (TC)y[i];
    dot = warp_sum_t<TC>(dot);
    if (lane == 0) partial[it] = (double)dot;
  }
  __syncthreads();
  for (int it = w; it < items; it += nw) {
    const int jj = it / S, sg = it % S;
    double* y = A + k + (long)(k + 1 + jj) * ld;
    TC dot = 0;
    for (int q = 0; q < S; ++q) dot += (TC)partial[jj * S + q];
    dot *= t;
    const int r0 = sg * seg, r1 = min(len, r0 + seg);
    for (int i = r0 + lane; i < r1; i += 32) y[i] = (double)((TC)y[i] - dot * (i == 0 ? (TC)1 : (TC)x[i]));
  }
  __syncthreads();
}

template <typename TC>
__global__ void k_qr(const QrDesc* __restrict__ d, int nd) {
  if ((int)blockIdx.x >= nd) return;
  const QrDesc D = d[blockIdx.x];
  const int m = D.m, n = D.n;
  const long ld = D.ld;
  double* A = D.A;
  __shared__ double scratch[32];
  __shared__ double partial[1024];
  __shared__ double s_alpha, s_beta, s_scale;
  const int kmax = m < n ? m : n;
  for (int k = 0; k < kmax; ++k) {
    double* x = A + k + k * ld;
    const int len = m - k;
    double ss = 0.0;
    for (int i = 1 + threadIdx.x; i < len; i += blockDim.x) ss += x[i] * x[i];
    ss = block_sum(ss, scratch);
    // reflector in the normalised form H = I - tau v v^T, v_0 = 1,
    // v_i = x_i / (x_0 - alpha), tau = (alpha - x_0) / alpha in [1, 2]
    if (threadIdx.x == 0) {
      const double x0 = x[0];
      const double nrm = sqrt(x0 * x0 + ss);
      if (nrm == 0.0 || ss == 0.0) {
        s_alpha = x0;
        s_beta = 0.0;
      } else {
        const double alpha = (x0 >= 0.0) ? -nrm : nrm;
        s_alpha = alpha;
        s_beta = (alpha - x0) / alpha;
        s_scale = 1.0 / (x0 - alpha);
      }
    }
    __syncthreads();
    const double tau = s_beta;
    if (tau != 0.0) {
      const double sc = s_scale;
      for (int i = 1 + threadIdx.x; i < len; i += blockDim.x) x[i] *= sc;
      __syncthreads();
      apply_reflector<TC>(A, ld, k, n, len, x, (TC)tau, partial);
    }
    __syncthreads();
    if (threadIdx.x == 0) x[0] = s_alpha;
    for (int i = 1 + threadIdx.x; i < len; i += blockDim.x) x[i] = 0.0;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- pivoted QR (truncated), global memory
// One CTA per matrix, the block in global memory (the fallback for blocks that
// fit neither one CTA's nor a cluster's shared memory).  Column norms live in
// shared memory and are downdated after each step (recomputed when
// cancellation has eaten two digits).  Dynamic shared memory: 2n doubles + n ints.
template <typename TC>
__global__ void k_qrcp(const QrcpDesc* __restrict__ d, int nd) {
  if ((int)blockIdx.x >= nd) return;
  const QrcpDesc D = d[blockIdx.x];
  const int m = D.m, n = D.n;
  const long ld = D.ld;
  double* A = D.A;
  extern __shared__ double sm[];
  double* nrm = sm;
  double* ref = sm + n;
  int* jp = (int*)(sm + 2 * n);
  __shared__ double scratch[32];
  __shared__ double partial[1024];
  __shared__ char flag[1024];
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ double s_tau2, s_alpha, s_tau, s_scale, s_first, s_tailv;
  __shared__ int s_p, s_stop, s_capped;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int j = w; j < n; j += nw) {
    const double* c = A + (long)j * ld;
    double ss = 0.0;
    for (int i = lane; i < m; i += 32) ss += c[i] * c[i];
    ss = warp_sum(ss);
    if (lane == 0) {
      nrm[j] = ss;
      ref[j] = ss;
      jp[j] = j;
    }
  }
  __syncthreads();
  const int kmax = m < n ? m : n;
  int k = 0;
  for (; k < kmax; ++k) {
    double best = -1.0;
    int bi = n;
    for (int j = k + threadIdx.x; j < n; j += blockDim.x) {
      const double v = nrm[j];
      if (v > best || (v == best && j < bi)) { best = v; bi = j; }
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
      if (k == 0) s_tau2 = D.tau_rel * D.tau_rel * bv;
      if (k == 0) s_first = bv;
      s_stop = !(bv > s_tau2) || !(bv > 0.0) || b >= n;
      s_capped = 0;
      if (!s_stop && D.kcap > 0 && k >= D.kcap) {
        s_stop = 1;
        s_capped = 1;
        s_tailv = (s_first > 0.0) ? sqrt(bv / s_first) : 0.0;
      }
      s_p = b;
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_p;
    if (p != k) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double t = A[i + k * ld];
        A[i + k * ld] = A[i + p * ld];
        A[i + p * ld] = t;
      }
      if (threadIdx.x == 0) {
        double t = nrm[k]; nrm[k] = nrm[p]; nrm[p] = t;
        t = ref[k]; ref[k] = ref[p]; ref[p] = t;
        const int q = jp[k]; jp[k] = jp[p]; jp[p] = q;
      }
    }
    __syncthreads();
    double* x = A + k + k * ld;
    const int len = m - k;
    double ss = 0.0;
    for (int i = 1 + threadIdx.x; i < len; i += blockDim.x) ss += x[i] * x[i];
    ss = block_sum(ss, scratch);
    if (threadIdx.x == 0) {
      const double x0 = x[0];
      const double nr = sqrt(x0 * x0 + ss);
      if (nr == 0.0 || ss == 0.0) {
        s_alpha = x0;
        s_tau = 0.0;
      } else {
        const double alpha = (x0 >= 0.0) ? -nr : nr;
        s_alpha = alpha;
        s_tau = (alpha - x0) / alpha;
        s_scale = 1.0 / (x0 - alpha);
      }
    }
    __syncthreads();
    const double tau = s_tau;
    if (tau != 0.0) {
      const double sc = s_scale;
      for (int i = 1 + threadIdx.x; i < len; i += blockDim.x) x[i] *= sc;
      __syncthreads();
    }
    if (tau != 0.0) apply_reflector<TC>(A, ld, k, n, len, x, (TC)tau, partial);
    // downdate the column norms with the new row k of R; recompute a norm when
    // cancellation has removed two digits
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
      const double rkj = A[k + (long)j * ld];
      const double v = nrm[j] - rkj * rkj;
      flag[j] = !(v > 1e-2 * ref[j]);
      nrm[j] = v;
    }
    __syncthreads();
    for (int j = k + 1 + w; j < n; j += nw) {
      if (!flag[j]) continue;
      const double* y = A + k + (long)j * ld;
      double s2 = 0.0;
      for (int i = 1 + lane; i < len; i += 32) s2 += y[i] * y[i];
      s2 = warp_sum(s2);
      if (lane == 0) {
        nrm[j] = s2;
        ref[j] = s2;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) x[0] = s_alpha;
    for (int i = 1 + threadIdx.x; i < len; i += blockDim.x) x[i] = 0.0;
    __syncthreads();
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) D.jpvt[j] = jp[j];
  if (threadIdx.x == 0) {
    D.kout[0] = k;
    if (D.tail) D.tail[0] = (k < kmax && s_capped) ? s_tailv : 0.0;
  }
}

// ---------------------------------------------------------------- Householder QR in shared memory
// The factorisations of k_qr (PIV = false) and k_qrcp (PIV = true) for blocks
// that fit in shared memory in the arithmetic type TC: the block is read from
// global memory once, factorised in shared memory, and written back once.
// On the way in it is multiplied by a power of two (exact) that brings its
// largest magnitude into [0.5, 1): squared column norms of FP32 blocks whose
// entries are ~1e-12 would otherwise fall out of the FP32 normal range.  R is
// scaled back (exactly) on the way out.  The Householder vector of step k,
// v_0 = 1, v_i = sc x_i, is formed on the fly from the untouched column and
// never stored; the column is zeroed below the diagonal on write-back.  The
// norm of every pivot candidate is downdated right after its column has been
// updated, in the same pass.
// Slot of one problem: A (m x n, ld m) | nrm (n) | ref (n), in TC | jp (n ints).
__host__ __device__ __forceinline__ size_t qr_slot_bytes(int m, int n, int tc_bytes) {
  return (((size_t)m * n + 2 * (size_t)n) * tc_bytes + sizeof(int) * (size_t)n + 15) & ~(size_t)15;
}

// exponent shift that brings a block whose largest |entry| has biased binary64
// exponent emax into [0.5, 1) (0 for an all-zero block or one with inf/NaN)
__device__ __forceinline__ int pow2_shift(int emax) { return (emax <= 0 || emax >= 2047) ? 0 : 1022 - emax; }

// Applies H = I - tau v v^T (v_0 = 1, v_i = sc x_i) to the cnt <= G columns
// j0.. of the trailing block (rows k..k+len-1, ld m) with one warp: G independent
// dot products per row sweep and G interleaved butterfly reductions, so the
// shared-memory and shuffle latencies of the columns overlap.
template <typename TC, int G>
__device__ __forceinline__ void reflect_group(TC* A, int m, int k, int len, const TC* x, TC sc, TC tau, int j0,
                                              int cnt, int lane) {
  TC* y[G];
#pragma unroll
  for (int u = 0; u < G; ++u) y[u] = A + k + (size_t)(j0 + (u < cnt ? u : cnt - 1)) * m;
  TC acc[G];
#pragma unroll
  for (int u = 0; u < G; ++u) acc[u] = 0;
  for (int i = lane; i < len; i += 32) {
    const TC vi = (i == 0) ? (TC)1 : sc * x[i];
#pragma unroll
    for (int u = 0; u < G; ++u) acc[u] += vi * y[u][i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int u = 0; u < G; ++u) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
  for (int i = lane; i < len; i += 32) {
    const TC vi = (i == 0) ? (TC)1 : sc * x[i];
#pragma unroll
    for (int u = 0; u < G; ++u)
      if (u < cnt) y[u][i] -= (acc[u] * tau) * vi;
  }
}

// (row, column) of the flat column-major index e = i + j m, advanced by a fixed
// stride without a division per step
struct FlatIdx {
  int i, j, di, dj, m;
  __device__ __forceinline__ FlatIdx(int e0, int stride, int m_) : m(m_ > 0 ? m_ : 1) {
    i = e0 % m;
    j = e0 / m;
    di = stride % m;
    dj = stride / m;
  }
  __device__ __forceinline__ void next() {
    i += di;
    j += dj;
    if (i >= m) {
      i -= m;
      ++j;
    }
  }
};

// physical row of logical row i (QrcpDesc::rb, rs)
__device__ __forceinline__ long qr_row(const QrcpDesc& D, int i) {
  return D.rb > 0 ? (long)(i / D.rb) * D.rs + i % D.rb : (long)i;
}

// One warp per problem; blockDim.x / 32 problems per CTA; slot_bytes of
// dynamic shared memory per warp.  Only __syncwarp is used.
template <typename TC, bool PIV>
__global__ void k_qr_warp(const QrcpDesc* __restrict__ d, int nd, int slot_bytes) {
  extern __shared__ __align__(16) unsigned char qsm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int di = blockIdx.x * (blockDim.x >> 5) + w;
  if (di >= nd) return;
  const QrcpDesc D = d[di];
  const int m = D.m, n = D.n;
  const long ld = D.ld;
  const int mn = m * n;
  TC* A = (TC*)(qsm + (size_t)w * slot_bytes);
  TC* nrm = A + mn;
  TC* ref = nrm + n;
  int* jp = (int*)(ref + n);
  int em = 0;
  {
    FlatIdx x(lane, 32, m);
    for (int e = lane; e < mn; e += 32, x.next()) em = max(em, dexp(D.A[qr_row(D, x.i) + (long)x.j * ld]));
  }
  const int sh = pow2_shift((int)__reduce_max_sync(0xffffffffu, (unsigned)em));
  {
    FlatIdx x(lane, 32, m);
    for (int e = lane; e < mn; e += 32, x.next()) A[e] = ld_tc<TC>(D.A[qr_row(D, x.i) + (long)x.j * ld], sh);
  }
  __syncwarp();
  if (PIV) {
    for (int j = 0; j < n; ++j) {
      const TC* c = A + (size_t)j * m;
      TC ss = 0;
      for (int i = lane; i < m; i += 32) ss += c[i] * c[i];
      ss = warp_sum_t<TC>(ss);
      if (lane == 0) {
        nrm[j] = ss;
        ref[j] = ss;
        jp[j] = j;
      }
    }
    __syncwarp();
  }
  const int kmax = m < n ? m : n;
  TC tau2 = 0, first = 0;
  double tailv = 0.0;
  bool capped = false;
  int k = 0;
  for (; k < kmax; ++k) {
    if (PIV) {
      TC best = -1;
      int bi = n;
      for (int j = k + lane; j < n; j += 32) {
        const TC v = nrm[j];
        if (v > best || (v == best && j < bi)) { best = v; bi = j; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const TC ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (k == 0) {
        tau2 = (TC)(D.tau_rel * D.tau_rel) * best;
        first = best;
      }
      bool stop = !(best > tau2) || !(best > (TC)0) || bi >= n;
      if (!stop && D.kcap > 0 && k >= D.kcap) {
        stop = true;
        capped = true;
        tailv = (first > (TC)0) ? sqrt((double)best / (double)first) : 0.0;
      }
      if (stop) break;
      if (bi != k) {
        TC* ck = A + (size_t)k * m;
        TC* cp = A + (size_t)bi * m;
        for (int i = lane; i < m; i += 32) {
          const TC t = ck[i];
          ck[i] = cp[i];
          cp[i] = t;
        }
        if (lane == 0) {
          TC t = nrm[k]; nrm[k] = nrm[bi]; nrm[bi] = t;
          t = ref[k]; ref[k] = ref[bi]; ref[bi] = t;
          const int q = jp[k]; jp[k] = jp[bi]; jp[bi] = q;
        }
        __syncwarp();
      }
    }
    TC* x = A + k + (size_t)k * m;
    const int len = m - k;
    TC ss = 0;
    for (int i = lane; i < len; i += 32)
      if (i > 0) ss += x[i] * x[i];
    ss = warp_sum_t<TC>(ss);
    const TC x0 = x[0];
    const TC nr = sqrt(x0 * x0 + ss);
    TC alpha = x0, tau = 0, sc = 0;
    if (!(nr == (TC)0 || ss == (TC)0)) {
      alpha = (x0 >= (TC)0) ? -nr : nr;
      tau = (alpha - x0) / alpha;
      sc = (TC)1 / (x0 - alpha);
    }
    for (int j0 = k + 1; j0 < n; j0 += 4) {
      const int cnt = min(4, n - j0);
      if (tau != (TC)0) reflect_group<TC, 4>(A, m, k, len, x, sc, tau, j0, cnt, lane);
      if (PIV) {
        for (int u = 0; u < cnt; ++u) {
          const int j = j0 + u;
          const TC* y = A + k + (size_t)j * m;
          const TC nj = nrm[j], rj = ref[j];
          const TC r = __shfl_sync(0xffffffffu, lane == 0 ? y[0] : (TC)0, 0);
          TC nv = nj - r * r;
          if (!(nv > (TC)1e-2 * rj)) {  // two digits lost: recompute from the column
            TC s2 = 0;
            for (int i = lane; i < len; i += 32)
              if (i > 0) s2 += y[i] * y[i];
            nv = warp_sum_t<TC>(s2);
            if (lane == 0) ref[j] = nv;
          }
          if (lane == 0) nrm[j] = nv;
        }
      }
    }
    if (lane == 0) x[0] = alpha;
    __syncwarp();
  }
  {
    FlatIdx x(lane, 32, m);
    for (int e = lane; e < mn; e += 32, x.next()) {
      const TC v = (x.j < k && x.i > x.j) ? (TC)0 : A[e];
      D.A[qr_row(D, x.i) + (long)x.j * ld] = st_tc<TC>(v, -sh);
    }
  }
  if (PIV) {
    for (int j = lane; j < n; j += 32) D.jpvt[j] = jp[j];
    if (lane == 0) {
      D.kout[0] = k;
      if (D.tail) D.tail[0] = (k < kmax && capped) ? tailv : 0.0;
    }
  }
}

// One CTA (<= 1024 threads) per problem, the block in dynamic shared memory.
// Per column step: one barrier for the pivot search, one after a column swap,
// one for the reflector norm, one between the segment dot products and the
// update, and one closing the step (plus one more in the rare step where a
// downdated norm has to be recomputed).
template <typename TC, bool PIV>
__global__ void __launch_bounds__(1024) k_qr_cta(const QrcpDesc* __restrict__ d, int nd) {
  if ((int)blockIdx.x >= nd) return;
  const QrcpDesc D = d[blockIdx.x];
  const int m = D.m, n = D.n;
  const long ld = D.ld;
  const int mn = m * n;
  extern __shared__ __align__(16) unsigned char qsm[];
  TC* A = (TC*)qsm;
  TC* nrm = A + mn;
  TC* ref = nrm + n;
  int* jp = (int*)(ref + n);
  __shared__ TC part[32];
  __shared__ unsigned char flag[1024];
  __shared__ TC red_s[32], red_v[32];
  __shared__ int red_i[32];
  const int tid = threadIdx.x, nt_ = blockDim.x;
  const int lane = tid & 31, w = tid >> 5, nw = nt_ >> 5;
  int em = 0;
  {
    FlatIdx x(tid, nt_, m);
    for (int e = tid; e < mn; e += nt_, x.next()) em = max(em, dexp(D.A[qr_row(D, x.i) + (long)x.j * ld]));
  }
  em = (int)__reduce_max_sync(0xffffffffu, (unsigned)em);
  if (lane == 0) red_i[w] = em;
  __syncthreads();
  em = 0;
  for (int i = 0; i < nw; ++i) em = max(em, red_i[i]);
  const int sh = pow2_shift(em);
  {
    FlatIdx x(tid, nt_, m);
    for (int e = tid; e < mn; e += nt_, x.next()) A[e] = ld_tc<TC>(D.A[qr_row(D, x.i) + (long)x.j * ld], sh);
  }
  for (int j = tid; j < n; j += nt_) flag[j] = 0;
  __syncthreads();
  if (PIV) {
    for (int j = w; j < n; j += nw) {
      const TC* c = A + (size_t)j * m;
      TC ss = 0;
      for (int i = lane; i < m; i += 32) ss += c[i] * c[i];
      ss = warp_sum_t<TC>(ss);
      if (lane == 0) {
        nrm[j] = ss;
        ref[j] = ss;
        jp[j] = j;
      }
    }
    __syncthreads();
  }
  const int kmax = m < n ? m : n;
  TC tau2 = 0, first = 0;
  double tailv = 0.0;
  bool capped = false;
  int k = 0;
  for (; k < kmax; ++k) {
    if (PIV) {
      TC best = -1;
      int bi = n;
      for (int j = k + tid; j < n; j += nt_) {
        const TC v = nrm[j];
        if (v > best || (v == best && j < bi)) { best = v; bi = j; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const TC ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) {
        red_v[w] = best;
        red_i[w] = bi;
      }
      __syncthreads();
      best = -1;
      bi = n;
      for (int i = 0; i < nw; ++i)
        if (red_v[i] > best || (red_v[i] == best && red_i[i] < bi)) { best = red_v[i]; bi = red_i[i]; }
      if (k == 0) {
        tau2 = (TC)(D.tau_rel * D.tau_rel) * best;
        first = best;
      }
      bool stop = !(best > tau2) || !(best > (TC)0) || bi >= n;
      if (!stop && D.kcap > 0 && k >= D.kcap) {
        stop = true;
        capped = true;
        tailv = (first > (TC)0) ? sqrt((double)best / (double)first) : 0.0;
      }
      if (stop) break;
      if (bi != k) {
        TC* ck = A + (size_t)k * m;
        TC* cp = A + (size_t)bi * m;
        for (int i = tid; i < m; i += nt_) {
          const TC t = ck[i];
          ck[i] = cp[i];
          cp[i] = t;
        }
        if (tid == 0) {
          TC t = nrm[k]; nrm[k] = nrm[bi]; nrm[bi] = t;
          t = ref[k]; ref[k] = ref[bi]; ref[bi] = t;
          const int q = jp[k]; jp[k] = jp[bi]; jp[bi] = q;
        }
        __syncthreads();
      }
    }
    TC* x = A + k + (size_t)k * m;
    const int len = m - k;
    TC ss = 0;
    for (int i = tid; i < len; i += nt_)
      if (i > 0) ss += x[i] * x[i];
    ss = warp_sum_t<TC>(ss);
    if (lane == 0) red_s[w] = ss;
    __syncthreads();
    ss = 0;
    for (int i = 0; i < nw; ++i) ss += red_s[i];
    const TC x0 = x[0];
    const TC nr = sqrt(x0 * x0 + ss);
    TC alpha = x0, tau = 0, sc = 0;
    if (!(nr == (TC)0 || ss == (TC)0)) {
      alpha = (x0 >= (TC)0) ? -nr : nr;
      tau = (alpha - x0) / alpha;
      sc = (TC)1 / (x0 - alpha);
    }
    const int ntr = n - k - 1;
    int need = 0;
    if (ntr > 0 && tau != (TC)0) {
      // a trailing column is split into S row segments when there are fewer
      // columns than warps (then ntr * S <= nw); segment sums are added in a
      // fixed order
      int S = nw / ntr;
      const int smax = (len + 63) / 64;
      if (S > smax) S = smax;
      if (S < 1) S = 1;
      if (S == 1) {
        // groups of G consecutive columns, round-robin over the warps
        const int G = ntr >= 4 * nw ? 4 : (ntr >= 2 * nw ? 2 : 1);
        const int ng = (ntr + G - 1) / G;
        for (int g = w; g < ng; g += nw) {
          const int j0 = k + 1 + g * G;
          const int cnt = min(G, n - j0);
          if (G == 4)
            reflect_group<TC, 4>(A, m, k, len, x, sc, tau, j0, cnt, lane);
          else if (G == 2)
            reflect_group<TC, 2>(A, m, k, len, x, sc, tau, j0, cnt, lane);
          else
            reflect_group<TC, 1>(A, m, k, len, x, sc, tau, j0, cnt, lane);
          if (PIV && lane == 0) {
            for (int u = 0; u < cnt; ++u) {
              const int j = j0 + u;
              const TC r = A[k + (size_t)j * m];
              const TC nv = nrm[j] - r * r;
              nrm[j] = nv;
              if (!(nv > (TC)1e-2 * ref[j])) {
                flag[j] = 1;
                need = 1;
              }
            }
          }
        }
      } else {
        const int seg = (len + S - 1) / S;
        const int items = ntr * S;
        for (int it = w; it < items; it += nw) {
          const int jj = it / S, sg = it % S;
          const TC* y = A + k + (size_t)(k + 1 + jj) * m;
          const int r0 = sg * seg, r1 = min(len, r0 + seg);
          TC dot = 0;
          for (int i = r0 + lane; i < r1; i += 32) dot += (i == 0 ? (TC)1 : sc * x[i]) * y[i];
          dot = warp_sum_t<TC>(dot);
          if (lane == 0) part[it] = dot;
        }
        __syncthreads();
        for (int it = w; it < items; it += nw) {
          const int jj = it / S, sg = it % S;
          const int j = k + 1 + jj;
          TC* y = A + k + (size_t)j * m;
          TC dot = 0;
          for (int q = 0; q < S; ++q) dot += part[jj * S + q];
          dot *= tau;
          const int r0 = sg * seg, r1 = min(len, r0 + seg);
          for (int i = r0 + lane; i < r1; i += 32) y[i] -= dot * (i == 0 ? (TC)1 : sc * x[i]);
          if (PIV && sg == 0 && lane == 0) {
            const TC r = y[0];
            const TC nv = nrm[j] - r * r;
            nrm[j] = nv;
            if (!(nv > (TC)1e-2 * ref[j])) {
              flag[j] = 1;
              need = 1;
            }
          }
        }
      }
    } else if (PIV && ntr > 0) {
      for (int j = k + 1 + tid; j < n; j += nt_) {
        const TC r = A[k + (size_t)j * m];
        const TC nv = nrm[j] - r * r;
        nrm[j] = nv;
        if (!(nv > (TC)1e-2 * ref[j])) {
          flag[j] = 1;
          need = 1;
        }
      }
    }
    const int any = __syncthreads_or(need);
    if (PIV && any) {  // two digits lost: recompute those norms from the columns
      for (int j = k + 1 + w; j < n; j += nw) {
        if (!flag[j]) continue;
        const TC* y = A + k + (size_t)j * m;
        TC s2 = 0;
        for (int i = lane; i < len; i += 32)
          if (i > 0) s2 += y[i] * y[i];
        s2 = warp_sum_t<TC>(s2);
        if (lane == 0) {
          nrm[j] = s2;
          ref[j] = s2;
          flag[j] = 0;
        }
      }
      __syncthreads();
    }
    if (tid == 0) x[0] = alpha;
  }
  __syncthreads();
  {
    FlatIdx x(tid, nt_, m);
    for (int e = tid; e < mn; e += nt_, x.next()) {
      const TC v = (x.j < k && x.i > x.j) ? (TC)0 : A[e];
      D.A[qr_row(D, x.i) + (long)x.j * ld] = st_tc<TC>(v, -sh);
    }
  }
  if (PIV) {
    for (int j = tid; j < n; j += nt_) D.jpvt[j] = jp[j];
    if (tid == 0) {
      D.kout[0] = k;
      if (D.tail) D.tail[0] = (k < kmax && capped) ? tailv : 0.0;
    }
  }
}

// ---------------------------------------------------------------- Householder QR across a cluster
// The same factorisations as k_qr_cta for blocks too large for one CTA's shared
// memory: the rows are split over the R CTAs of a thread-block cluster (CTA r
// holds logical rows [r*chunk, (r+1)*chunk) of all n columns, chunk = ceil(m/R)),
// and the CTAs exchange through distributed shared memory.  Every CTA keeps the
// column norms, the pivot order and the reflector scalars replicated, computed by
// the same operations in the same order, so every decision (pivot, stop, norm
// recompute) is identical cluster-wide.  Per column step there are two cluster
// barriers: after the partial reflector norms (plus the diagonal entry from the
// CTA that owns row k), and after the partial dot products (plus the owner's row k,
// from which every CTA forms row k of R for the norm downdate).  The exchange
// buffers alternate between even and odd steps, so a buffer is rewritten only
// after every CTA has passed the barrier that follows its last read.
// Slot: A (chunk x n, ld chunk) | nrm, ref (n) | xd (2n) | xr (2n) | xs (8), in TC | jp (n ints).
__host__ __device__ __forceinline__ size_t qr_cluster_slot_bytes(int m, int n, int R, int tc_bytes) {
  const size_t chunk = ((size_t)m + R - 1) / R;
  return ((chunk * n + 6 * (size_t)n + 8) * tc_bytes + sizeof(int) * (size_t)n + 15) & ~(size_t)15;
}

template <typename TC, bool PIV>
__global__ void __launch_bounds__(512) k_qr_cluster(const QrcpDesc* __restrict__ d, int nd) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int R = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int pi = (int)(blockIdx.x / R);
  const QrcpDesc D = d[pi < nd ? pi : nd - 1];
  const int m = D.m, n = D.n;
  const long ld = D.ld;
  const int chunk = (m + R - 1) / R;
  const int r0 = min(m, rank * chunk), ml = min(m, r0 + chunk) - r0;
  const int mlp = chunk > 0 ? chunk : 1;
  extern __shared__ __align__(16) unsigned char qsm[];
  TC* A = (TC*)qsm;
  TC* nrm = A + (size_t)mlp * n;
  TC* ref = nrm + n;
  TC* xd = ref + n;
  TC* xr = xd + 2 * n;
  TC* xs = xr + 2 * n;
  int* jp = (int*)(xs + 8);
  __shared__ unsigned char flag[1024];
  __shared__ TC red_s[32], red_v[32];
  __shared__ int red_i[32];
  __shared__ int xg;
  const int tid = threadIdx.x, nt_ = blockDim.x;
  const int lane = tid & 31, w = tid >> 5, nw = nt_ >> 5;
  // power-of-two scale from the cluster-wide largest magnitude
  int em = 0;
  for (int e = tid; e < ml * n; e += nt_) em = max(em, dexp(D.A[(r0 + e % ml) + (long)(e / ml) * ld]));
  em = (int)__reduce_max_sync(0xffffffffu, (unsigned)em);
  if (lane == 0) red_i[w] = em;
  __syncthreads();
  if (tid == 0) {
    int g = 0;
    for (int i = 0; i < nw; ++i) g = max(g, red_i[i]);
    xg = g;
  }
  for (int j = tid; j < n; j += nt_) flag[j] = 0;
  cl.sync();
  em = 0;
  for (int r = 0; r < R; ++r) em = max(em, *cl.map_shared_rank(&xg, r));
  const int sh = pow2_shift(em);
  for (int e = tid; e < ml * n; e += nt_) {
    const int li = e % ml, j = e / ml;
    A[li + (size_t)j * mlp] = ld_tc<TC>(D.A[(r0 + li) + (long)j * ld], sh);
  }
  __syncthreads();
  if (PIV) {
    for (int j = w; j < n; j += nw) {
      const TC* c = A + (size_t)j * mlp;
      TC ss = 0;
      for (int i = lane; i < ml; i += 32) ss += c[i] * c[i];
      ss = warp_sum_t<TC>(ss);
      if (lane == 0) xd[j] = ss;
    }
    cl.sync();
    for (int j = tid; j < n; j += nt_) {
      TC s = 0;
      for (int r = 0; r < R; ++r) s += cl.map_shared_rank(xd, r)[j];
      nrm[j] = s;
      ref[j] = s;
      jp[j] = j;
    }
    __syncthreads();
  }
  const int kmax = m < n ? m : n;
  TC tau2 = 0, first = 0;
  double tailv = 0.0;
  bool capped = false;
  int k = 0;
  for (; k < kmax; ++k) {
    const int buf = k & 1;
    if (PIV) {
      TC best = -1;
      int bi = n;
      for (int j = k + tid; j < n; j += nt_) {
        const TC v = nrm[j];
        if (v > best || (v == best && j < bi)) { best = v; bi = j; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const TC ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) {
        red_v[w] = best;
        red_i[w] = bi;
      }
      __syncthreads();
      best = -1;
      bi = n;
      for (int i = 0; i < nw; ++i)
        if (red_v[i] > best || (red_v[i] == best && red_i[i] < bi)) { best = red_v[i]; bi = red_i[i]; }
      if (k == 0) {
        tau2 = (TC)(D.tau_rel * D.tau_rel) * best;
        first = best;
      }
      bool stop = !(best > tau2) || !(best > (TC)0) || bi >= n;
      if (!stop && D.kcap > 0 && k >= D.kcap) {
        stop = true;
        capped = true;
        tailv = (first > (TC)0) ? sqrt((double)best / (double)first) : 0.0;
      }
      if (stop) break;
      if (bi != k) {
        TC* ck = A + (size_t)k * mlp;
        TC* cp = A + (size_t)bi * mlp;
        for (int i = tid; i < ml; i += nt_) {
          const TC t = ck[i];
          ck[i] = cp[i];
          cp[i] = t;
        }
        if (tid == 0) {
          TC t = nrm[k]; nrm[k] = nrm[bi]; nrm[bi] = t;
          t = ref[k]; ref[k] = ref[bi]; ref[bi] = t;
          const int q = jp[k]; jp[k] = jp[bi]; jp[bi] = q;
        }
        __syncthreads();
      }
    }
    const int owner = k / chunk;
    const int lk = k - r0;  // local row of k (in [0, ml) on the owner)
    // local rows li >= l0 hold logical rows >= k
    const int l0 = max(0, k - r0);
    const TC* xk = A + (size_t)k * mlp;
    TC ss = 0;
    for (int li = l0 + tid; li < ml; li += nt_)
      if (r0 + li > k) ss += xk[li] * xk[li];
    ss = warp_sum_t<TC>(ss);
    if (lane == 0) red_s[w] = ss;
    __syncthreads();
    if (tid == 0) {
      TC s = 0;
      for (int i = 0; i < nw; ++i) s += red_s[i];
      xs[4 * buf] = s;
      if (rank == owner) xs[4 * buf + 1] = xk[lk];
    }
    cl.sync();
    ss = 0;
    for (int r = 0; r < R; ++r) ss += cl.map_shared_rank(xs, r)[4 * buf];
    const TC x0 = cl.map_shared_rank(xs, owner)[4 * buf + 1];
    const TC nr = sqrt(x0 * x0 + ss);
    TC alpha = x0, tau = 0, sc = 0;
    if (!(nr == (TC)0 || ss == (TC)0)) {
      alpha = (x0 >= (TC)0) ? -nr : nr;
      tau = (alpha - x0) / alpha;
      sc = (TC)1 / (x0 - alpha);
    }
    const int ntr = n - k - 1;
    TC* xdb = xd + (size_t)buf * n;
    TC* xrb = xr + (size_t)buf * n;
    if (ntr > 0 && tau != (TC)0) {
      for (int j = k + 1 + w; j < n; j += nw) {
        const TC* y = A + (size_t)j * mlp;
        TC acc = 0;
        for (int li = l0 + lane; li < ml; li += 32) {
          const TC vi = (r0 + li == k) ? (TC)1 : sc * xk[li];
          acc += vi * y[li];
        }
        acc = warp_sum_t<TC>(acc);
        if (lane == 0) xdb[j] = acc;
      }
    }
    if (rank == owner)
      for (int j = k + 1 + tid; j < n; j += nt_) xrb[j] = A[lk + (size_t)j * mlp];
    cl.sync();
    int need = 0;
    if (ntr > 0) {
      const TC* xro = cl.map_shared_rank(xrb, owner);
      for (int j = k + 1 + w; j < n; j += nw) {
        TC dj = 0;
        if (tau != (TC)0) {
          for (int r = 0; r < R; ++r) dj += cl.map_shared_rank(xdb, r)[j];
          dj *= tau;
          TC* y = A + (size_t)j * mlp;
          for (int li = l0 + lane; li < ml; li += 32) {
            const TC vi = (r0 + li == k) ? (TC)1 : sc * xk[li];
            y[li] -= dj * vi;
          }
        }
        if (PIV && lane == 0) {
          const TC rkj = xro[j] - dj;  // row k of R: the owner's row k minus d_j v_k, v_k = 1
          const TC nv = nrm[j] - rkj * rkj;
          nrm[j] = nv;
          if (!(nv > (TC)1e-2 * ref[j])) {
            flag[j] = 1;
            need = 1;
          }
        }
      }
    }
    const int any = __syncthreads_or(need);
    if (PIV && any) {  // two digits lost (identically in every CTA): recompute
      TC* xdo = xd + (size_t)(buf ^ 1) * n;
      for (int j = k + 1 + w; j < n; j += nw) {
        if (!flag[j]) continue;
        const TC* y = A + (size_t)j * mlp;
        TC s2 = 0;
        for (int li = l0 + lane; li < ml; li += 32)
          if (r0 + li > k) s2 += y[li] * y[li];
        s2 = warp_sum_t<TC>(s2);
        if (lane == 0) xdo[j] = s2;
      }
      cl.sync();
      for (int j = k + 1 + tid; j < n; j += nt_) {
        if (!flag[j]) continue;
        TC s = 0;
        for (int r = 0; r < R; ++r) s += cl.map_shared_rank(xdo, r)[j];
        nrm[j] = s;
        ref[j] = s;
        flag[j] = 0;
      }
    }
    if (rank == owner && tid == 0) A[lk + (size_t)k * mlp] = alpha;
    __syncthreads();
  }
  // no CTA leaves while another may still read its shared memory
  cl.sync();
  for (int e = tid; e < ml * n; e += nt_) {
    const int li = e % ml, j = e / ml;
    const int i = r0 + li;
    const TC v = (j < k && i > j) ? (TC)0 : A[li + (size_t)j * mlp];
    D.A[i + (long)j * ld] = st_tc<TC>(v, -sh);
  }
  if (PIV && rank == 0) {
    for (int j = tid; j < n; j += nt_) D.jpvt[j] = jp[j];
    if (tid == 0) {
      D.kout[0] = k;
      if (D.tail) D.tail[0] = (k < kmax && capped) ? tailv : 0.0;
    }
  }
}

// ---------------------------------------------------------------- Gauss-Jordan across a cluster
// The inverse of k_inv (partial pivoting, in place, the row interchanges undone
// as column interchanges at the end) with the rows split over the R CTAs of a
// thread-block cluster (CTA r holds rows [r*chunk, (r+1)*chunk), chunk =
// ceil(n/R), all n columns, column-major with ld chunk), so that a color with
// few large pivot blocks still occupies many SMs of GB300's narrow FP64 pipes.
// Step k: each CTA publishes its best |A(i,k)|, i >= k (barrier 1); every CTA
// picks the same pivot row p (ties: smallest i); the CTAs owning rows k and p
// publish copies of them (barrier 2); every CTA forms the scaled pivot row from
// the copy of row p and eliminates column k from its rows, the owner of p first
// taking in the copy of row k.  Exchange buffers alternate between even and odd
// steps.  Every element sees the same operations as in k_inv.
// Slot: A (chunk x n) | ck (chunk) | prow (n) | xrk, xrp (2 x n each) | xv (2),
// in double | piv (n), xi (2) ints.
__host__ __device__ __forceinline__ size_t inv_cluster_slot_bytes(int n, int R) {
  const size_t chunk = ((size_t)n + R - 1) / R;
  return ((chunk * n + chunk + 5 * (size_t)n + 2) * sizeof(double) + sizeof(int) * ((size_t)n + 2) + 15) &
         ~(size_t)15;
}

__global__ void __launch_bounds__(512) k_inv_cluster(const InvDesc* __restrict__ d, int nd) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int R = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int pi = (int)(blockIdx.x / R);
  const InvDesc D = d[pi < nd ? pi : nd - 1];
  const int n = D.n;
  const long ld = D.ld;
  const int chunk = (n + R - 1) / R;
  const int r0 = min(n, rank * chunk), ml = min(n, r0 + chunk) - r0;
  const int cp = chunk > 0 ? chunk : 1;
  extern __shared__ __align__(16) unsigned char ism2[];
  double* A = (double*)ism2;
  double* ck = A + (size_t)cp * n;
  double* prow = ck + cp;
  double* xrk = prow + n;
  double* xrp = xrk + 2 * n;
  double* xv = xrp + 2 * n;
  int* piv = (int*)(xv + 2);
  int* xi = piv + n;
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ double s_inv;
  __shared__ int s_p;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  for (int j = w; j < n; j += nw)
    for (int li = lane; li < ml; li += 32) A[li + (size_t)j * cp] = D.A[(r0 + li) + (long)j * ld];
  __syncthreads();
  int bad = 0;
  const int tot = ml * n;
  for (int k = 0; k < n; ++k) {
    const int b = k & 1;
    double best = -1.0;
    int bi = n;
    for (int li = max(0, k - r0) + tid; li < ml; li += nt) {
      const double v = fabs(A[li + (size_t)k * cp]);
      const int i = r0 + li;
      if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) {
      red_v[w] = best;
      red_i[w] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double bv = -1.0;
      int bb = n;
      for (int i = 0; i < nw; ++i)
        if (red_v[i] > bv || (red_v[i] == bv && red_i[i] < bb)) { bv = red_v[i]; bb = red_i[i]; }
      xv[b] = bv;
      xi[b] = bb;
    }
    cl.sync();
    // one warp reads the R candidates and decides (the same decision in every CTA)
    if (w == 0) {
      double v = -1.0;
      int i = n;
      if (lane < R) {
        v = cl.map_shared_rank(xv, lane)[b];
        i = cl.map_shared_rank(xi, lane)[b];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
      }
      if (lane == 0) {
        s_p = (!(v > 0.0) || i >= n) ? -1 : i;
        if (s_p >= 0) piv[k] = i;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p < 0) {
      bad = k + 1;
      break;
    }
    const int ok = k / chunk, op = p / chunk;
    if (rank == ok)
      for (int j = tid; j < n; j += nt) xrk[(size_t)b * n + j] = A[(k - r0) + (size_t)j * cp];
    if (rank == op)
      for (int j = tid; j < n; j += nt) xrp[(size_t)b * n + j] = A[(p - r0) + (size_t)j * cp];
    cl.sync();
    const double* rp = cl.map_shared_rank(xrp, op) + (size_t)b * n;
    if (tid == 0) s_inv = 1.0 / rp[k];  // once per CTA: an FP64 divide is a long FP64 sequence
    // multipliers of column k (the owner of p takes in the copy of row k there)
    const double* rk = (rank == op && p != k) ? cl.map_shared_rank(xrk, ok) + (size_t)b * n : nullptr;
    for (int li = tid; li < ml; li += nt) ck[li] = (rk && r0 + li == p) ? rk[k] : A[li + (size_t)k * cp];
    if (rk)
      for (int j = tid; j < n; j += nt) A[(p - r0) + (size_t)j * cp] = rk[j];
    __syncthreads();
    const double inv = s_inv;
    for (int j = tid; j < n; j += nt) prow[j] = (j == k) ? inv : rp[j] * inv;
    __syncthreads();
    // eliminate column k from every local row but k; (li, j) walked with
    // incremental indices; the owner of k writes the scaled pivot row
    {
      int li = tid % max(ml, 1), j = tid / max(ml, 1);
      const int di = nt % max(ml, 1), dj = nt / max(ml, 1);
      for (int e = tid; e < tot; e += nt) {
        const int i = r0 + li;
        double* a = A + li + (size_t)j * cp;
        if (i == k)
          *a = prow[j];
        else
          *a = ((j == k) ? 0.0 : *a) - ck[li] * prow[j];
        li += di;
        j += dj;
        if (li >= ml) {
          li -= ml;
          ++j;
        }
      }
    }
    __syncthreads();
  }
  if (!bad) {
    for (int k = n - 1; k >= 0; --k) {
      const int p = piv[k];
      if (p != k)
        for (int li = tid; li < ml; li += nt) {
          const double t = A[li + (size_t)k * cp];
          A[li + (size_t)k * cp] = A[li + (size_t)p * cp];
          A[li + (size_t)p * cp] = t;
        }
      __syncthreads();
    }
  }
  // no CTA leaves while another may still read its shared memory
  cl.sync();
  if (!bad)
    for (int j = w; j < n; j += nw)
      for (int li = lane; li < ml; li += 32) D.A[(r0 + li) + (long)j * ld] = A[li + (size_t)j * cp];
  if (rank == 0 && tid == 0) D.info[0] = bad;
}

// ---------------------------------------------------------------- IL basis changes
// One CTA per touched IL entry e of a color: M2L_ab <- T'_a M2L_ab T_b, with
// the identity for an endpoint that was not re-based and a zero block when an
// old rank is zero.  The block is staged in shared memory (it is overwritten in
// place); md >= every rank involved is the stride of the staging tiles.
template <typename TC>
__global__ void __launch_bounds__(128) k_il_transform(const int* __restrict__ list, int nlist, IlTables t, int md) {
  if ((int)blockIdx.x >= nlist) return;
  const int e = list[blockIdx.x];
  const int a = t.il_row[e], b = t.il[e];
  const int ra = t.rbefore[a], rb = t.rbefore[b], na = t.newk[a], nb = t.newk[b];
  const int ka = na >= 0 ? na : ra, kb = nb >= 0 ? nb : rb;
  if (ka == 0 || kb == 0) return;
  double* M = t.far[e];
  const long ld = t.capr[a];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (ra == 0 || rb == 0) {
    for (int x = tid; x < ka * kb; x += nt) M[(x % ka) + (long)(x / ka) * ld] = 0.0;
    return;
  }
  extern __shared__ __align__(16) unsigned char ism[];
  TC* Ms = (TC*)ism;       // ra x rb, ld ra
  TC* t1 = Ms + md * md;   // ka x rb, ld ka
  TC* X = t1 + md * md;    // T'_a (ka x ra, ld ka), then T_b (rb x kb, ld rb)
  for (int x = tid; x < ra * rb; x += nt) Ms[x] = ld_tc<TC>(M[(x % ra) + (long)(x / ra) * ld]);
  if (na >= 0) {
    const double* Tp = t.Tp[a];
    for (int x = tid; x < ka * ra; x += nt) X[x] = ld_tc<TC>(Tp[x]);
  }
  __syncthreads();
  if (na >= 0) {
    for (int x = tid; x < ka * rb; x += nt) {
      const int i = x % ka, j = x / ka;
      TC acc = 0;
      for (int l = 0; l < ra; ++l) acc += X[i + l * ka] * Ms[l + j * ra];
      t1[x] = acc;
    }
  } else {
    for (int x = tid; x < ka * rb; x += nt) t1[x] = Ms[x];
  }
  __syncthreads();
  if (nb >= 0) {
    const double* Tb = t.T[b];
    for (int x = tid; x < rb * kb; x += nt) X[x] = ld_tc<TC>(Tb[x]);
    __syncthreads();
    for (int x = tid; x < ka * kb; x += nt) {
      const int i = x % ka, j = x / ka;
      TC acc = 0;
      for (int l = 0; l < rb; ++l) acc += t1[i + l * ka] * X[l + j * rb];
      M[i + (long)j * ld] = st_tc<TC>(acc);
    }
  } else {
    for (int x = tid; x < ka * kb; x += nt) M[(x % ka) + (long)(x / ka) * ld] = st_tc<TC>(t1[x]);
  }
}

// One CTA per (event, side): gathers the weight stack of ZGatherDesc from the
// level's IL blocks on the device.
__global__ void __launch_bounds__(256) k_zgather(const ZGatherDesc* __restrict__ d, int nd, ZTables t) {
  if ((int)blockIdx.x >= nd) return;
  const ZGatherDesc D = d[blockIdx.x];
  const int q = D.q, rq = t.r[q];
  const long ldz = D.ldz;
  const int tid = threadIdx.x, nt = blockDim.x;
  int off = 0;
  for (int e = t.il_ptr[q]; e < t.il_ptr[q + 1]; ++e) {
    const int l = t.il[e], rl = t.r[l];
    if (rl == 0) continue;
    if (D.side == 0) {
      const double* src = t.far[t.il_T[e]];
      const long lds = t.capr[l];
      for (int x = tid; x < rl * rq; x += nt) {
        const int i = x % rl, j = x / rl;
        D.Z[off + i + j * ldz] = src[i + j * lds];
      }
    } else {
      const double* src = t.far[e];
      const long lds = t.capr[q];
      for (int x = tid; x < rl * rq; x += nt) {
        const int i = x % rl, j = x / rl;
        D.Z[off + i + j * ldz] = src[j + i * lds];
      }
    }
    off += rl;
  }
  if (t.tail) {
    const int rc = t.rc;
    if (D.side == 0) {
      const double* src = t.M2M[q];
      for (int x = tid; x < rc * rq; x += nt) {
        const int i = x % rc, j = x / rc;
        D.Z[off + i + j * ldz] = src[i + (long)j * rc];
      }
    } else {
      const double* src = t.L2L[q];
      const long lds = t.capr[q];
      for (int x = tid; x < rc * rq; x += nt) {
        const int i = x % rc, j = x / rc;
        D.Z[off + i + j * ldz] = src[j + i * lds];
      }
    }
  }
}

// One CTA per (eliminated node, neighbour a): adds the row block of neighbour a
// of F into its near blocks (ScatterDesc).  The slot of (q, q2) is found by a
// binary search of q2 in q's sorted neighbour list.
__global__ void __launch_bounds__(256) k_schur_scatter(const ScatterDesc* __restrict__ d, int nd, ScatterTables t) {
  const int di = blockIdx.x;
  if (di >= nd) return;
  const ScatterDesc D = d[di];
  const int i = D.i;
  const int c0 = t.nbr_ptr[i], deg = t.nbr_ptr[i + 1] - c0;
  const int a = blockIdx.y;
  if (a >= deg) return;
  __shared__ int roff[32], dims[32], cl[32];
  if (threadIdx.x == 0) {
    int off = 0;
    for (int b = 0; b < deg && b < 32; ++b) {
      const int q = t.nbr[c0 + b];
      const int dq = t.elim[q] ? t.r[q] : t.n[q];
      cl[b] = q;
      roff[b] = off;
      dims[b] = dq;
      off += dq;
    }
  }
  __syncthreads();
  const int q = cl[a], mq = dims[a];
  if (mq == 0 || t.n[i] == 0) return;
  const int q0 = t.nbr_ptr[q], q1 = t.nbr_ptr[q + 1];
  const long ldd = t.n[q];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = 0; b < deg; ++b) {
    const int q2 = cl[b], mq2 = dims[b];
    if (mq2 == 0) continue;
    int slot = -1;
    if (q2 == q) {
      slot = t.slot_ptr[q];
    } else {
      int lo = q0, hi = q1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (t.nbr[mid] < q2) lo = mid + 1; else hi = mid;
      }
      if (lo < q1 && t.nbr[lo] == q2) slot = t.slot_ptr[q] + 1 + (lo - q0);
    }
    if (slot < 0) continue;  // a far pair: consumed by the recompression
    const int stg = t.elim[q] + t.elim[q2];
    double* dst = (stg == 0 ? t.nb0 : (stg == 1 ? t.nb1 : t.nb2))[slot];
    const double* src = D.F + roff[a] + (long)roff[b] * D.M;
    for (int j = w; j < mq2; j += nw)
      for (int x = lane; x < mq; x += 32) dst[x + (long)j * ldd] += src[x + (long)j * D.M];
  }
}

// ---------------------------------------------------------------- Jacobi on P R_k^T
// Hestenes' one-sided Jacobi: rotate column pairs of B until all pairs are
// orthogonal to working precision.  Pairs are taken in the round-robin order
// (k' = k rounded up to even; in round r, position p > 0 holds column
// 1 + ((p - 1 - r) mod (k'-1)); pair i joins positions i and k'-1-i), so the k'/2
// pairs of a round are disjoint and handled by different warps.
// B (n x k, column-major, ld n) lives in dynamic shared memory when it fits in
// smem_bytes, else in the descriptor's global work buffer.  Columns are rotated
// in place (no rotation matrix is accumulated: the rotated columns themselves,
// normalised, are the singular vectors sought).  n <= 1024.
template <typename TC>
__global__ void k_svd_rt(const SvdRtDesc* __restrict__ d, int nd, int max_sweeps, int smem_bytes) {
  if ((int)blockIdx.x >= nd) return;
  const SvdRtDesc D = d[blockIdx.x];
  const int n = D.n;
  int k = D.kin[0];
  k = k < 0 ? 0 : (k > n ? n : k);
  extern __shared__ double smraw[];
  __shared__ TC nrm[1024];
  __shared__ TC rnv[1024];
  __shared__ int ord[1024];
  __shared__ int s_em[32];
  __shared__ int s_rot;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const bool in_smem = (size_t)n * k * sizeof(TC) <= (size_t)smem_bytes;
  TC* B = in_smem ? (TC*)smraw : (TC*)D.work;
  const long ld = D.ld;
  // B = P R_k^T (or the explicit matrix), scaled by a power of two 2^sh that
  // brings its largest entry into [0.5, 1); warps over columns, lanes over rows
  int em = 0;
  for (int i = w; i < k; i += nw)
    for (int pos = lane; pos < n; pos += 32) {
      const double v = D.jpvt ? ((i <= pos) ? D.A[i + (long)pos * ld] : 0.0) : D.A[pos + (long)i * ld];
      em = max(em, dexp(v));
    }
  em = (int)__reduce_max_sync(0xffffffffu, (unsigned)em);
  if (lane == 0) s_em[w] = em;
  __syncthreads();
  em = 0;
  for (int i = 0; i < nw; ++i) em = max(em, s_em[i]);
  const int sh = pow2_shift(em);
  for (int i = w; i < k; i += nw)
    for (int pos = lane; pos < n; pos += 32) {
      if (D.jpvt)
        B[D.jpvt[pos] + (long)i * n] = ld_tc<TC>((i <= pos) ? D.A[i + (long)pos * ld] : 0.0, sh);
      else
        B[pos + (long)i * n] = ld_tc<TC>(D.A[pos + (long)i * ld], sh);
    }
  __syncthreads();
  const TC tol = sizeof(TC) == 8 ? (TC)1e-15 : (TC)4e-7;
  const TC tiny = sizeof(TC) == 8 ? (TC)1e-300 : (TC)1e-36;
  const int kp = k + (k & 1);
  for (int sweep = 0; sweep < max_sweeps && k > 1; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < kp - 1; ++r) {
      for (int pi = w; pi < kp / 2; pi += nw) {
        const int pa = pi, pb = kp - 1 - pi;
        int a = (pa == 0) ? 0 : 1 + ((pa - 1 - r) % (kp - 1) + (kp - 1)) % (kp - 1);
        int b = (pb == 0) ? 0 : 1 + ((pb - 1 - r) % (kp - 1) + (kp - 1)) % (kp - 1);
        if (a >= k || b >= k) continue;
        if (a > b) { const int tt = a; a = b; b = tt; }
        TC* ga = B + (long)a * n;
        TC* gb = B + (long)b * n;
        TC al = 0, be = 0, gab = 0;
        for (int i = lane; i < n; i += 32) {
          const TC u = ga[i], v = gb[i];
          al += u * u;
          be += v * v;
          gab += u * v;
        }
        al = warp_sum_t<TC>(al);
        be = warp_sum_t<TC>(be);
        gab = warp_sum_t<TC>(gab);
        if (al < tiny || be < tiny) continue;
        if (fabs(gab) <= tol * sqrt(al) * sqrt(be)) continue;
        const TC zeta = (be - al) / ((TC)2 * gab);
        const TC t = (zeta >= (TC)0 ? (TC)1 : (TC)-1) / (fabs(zeta) + hypot((TC)1, zeta));
        const TC c = (TC)1 / sqrt((TC)1 + t * t), s = c * t;
        for (int i = lane; i < n; i += 32) {
          const TC u = ga[i], v = gb[i];
          ga[i] = c * u - s * v;
          gb[i] = s * u + c * v;
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    const int rotated = s_rot;
    __syncthreads();
    if (!rotated) break;
  }
  // column norms (the singular values times 2^sh) in the arithmetic type, the
  // descending order (NaN last), and the reciprocals once per column
  for (int j = w; j < k; j += nw) {
    const TC* g = B + (long)j * n;
    TC s2 = 0;
    for (int i = lane; i < n; i += 32) s2 += g[i] * g[i];
    s2 = warp_sum_t<TC>(s2);
    if (lane == 0) {
      const TC v = sqrt(s2);
      nrm[j] = v;
      rnv[j] = (v > (TC)0) ? (TC)1 / v : (TC)0;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    int rank = 0;
    const TC v = (nrm[j] == nrm[j]) ? nrm[j] : (TC)-1;
    for (int q = 0; q < k; ++q) {
      const TC u = (nrm[q] == nrm[q]) ? nrm[q] : (TC)-1;
      rank += (u > v) || (u == v && q < j);
    }
    ord[rank] = j;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) D.sig[j] = (j < k) ? st_tc<TC>(nrm[ord[j]], -sh) : 0.0;
  for (int j = w; j < n; j += nw) {
    double* vj = D.V + (long)j * D.ldv;
    if (j < k) {
      const int c = ord[j];
      const TC r = rnv[c];
      const TC* g = B + (long)c * n;
      for (int i = lane; i < n; i += 32) vj[i] = st_tc<TC>(g[i] * r);
    } else {
      for (int i = lane; i < n; i += 32) vj[i] = 0.0;
    }
  }
}

// ---------------------------------------------------------------- randomized range finder helpers
// Omega (m x s, ld m) of +-1 entries: bit 63 of SplitMix64(seed + 0x9E37..*(index+1)).
__global__ void k_sketch(const SketchDesc* __restrict__ d, int nd) {
  if ((int)blockIdx.x >= nd) return;
  const SketchDesc D = d[blockIdx.x];
  const long total = (long)D.m * D.s;
  for (long e = threadIdx.x; e < total; e += blockDim.x) {
    unsigned long long z = D.seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(e + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    D.omega[e] = (z >> 63) ? 1.0 : -1.0;
  }
}
// out[0] = Frobenius norm of the m x n block (ld)
__global__ void k_frob(const FrobDesc* __restrict__ d, int nd) {
  if ((int)blockIdx.x >= nd) return;
  const FrobDesc D = d[blockIdx.x];
  __shared__ double scratch[32];
  double s = 0.0;
  const long total = (long)D.m * D.n;
  for (long e = threadIdx.x; e < total; e += blockDim.x) {
    const double v = D.A[(e % D.m) + (e / D.m) * (long)D.ld];
    s += v * v;
  }
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) D.out[0] = sqrt(s);
}

// ---------------------------------------------------------------- GEMV
// 4 independent accumulators over the columns of a column-major block: row i,
// columns [0, n) of A (leading dimension lda) against x.
__device__ __forceinline__ double dot_row(const double* __restrict__ a, long lda, const double* __restrict__ x, int n) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int j = 0;
  for (; j + 3 < n; j += 4) {
    s0 += a[(long)j * lda] * x[j];
    s1 += a[(long)(j + 1) * lda] * x[j + 1];
    s2 += a[(long)(j + 2) * lda] * x[j + 2];
    s3 += a[(long)(j + 3) * lda] * x[j + 3];
  }
  for (; j < n; ++j) s0 += a[(long)j * lda] * x[j];
  return (s0 + s1) + (s2 + s3);
}

// y = alpha * op(A) x + beta * y.  Non-transposed: a thread per row walks the
// columns (consecutive threads read consecutive rows of a column).  Transposed:
// a warp per output reduces one contiguous column of A.
__global__ void k_gemv(const GemvDesc* __restrict__ d, int nd) {
  if ((int)blockIdx.x >= nd) return;
  const GemvDesc D = d[blockIdx.x];
  if (D.trans) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int i = w; i < D.n; i += nw) {
      const double* a = D.A + (long)i * D.lda;
      double s = 0.0;
      for (int j = lane; j < D.m; j += 32) s += a[j] * D.x[j];
      s = warp_sum(s);
      if (lane == 0) D.y[i] = (D.beta == 0.0) ? D.alpha * s : D.alpha * s + D.beta * D.y[i];
    }
  } else {
    for (int i = threadIdx.x; i < D.m; i += blockDim.x) {
      const double s = dot_row(D.A + i, D.lda, D.x, D.n);
      D.y[i] = (D.beta == 0.0) ? D.alpha * s : D.alpha * s + D.beta * D.y[i];
    }
  }
}

}  // namespace ifmm
