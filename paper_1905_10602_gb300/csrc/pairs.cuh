// Float-pair ("double-float") arithmetic: a value carried as an unevaluated
// sum of two floats (hi + lo, ~48-bit significand), combined with error-free
// transformations on the FP32 pipes (Knuth's two-sum, the FMA two-product,
// Dekker's renormalisation).  Used where GB300's narrow FP64 pipe would be the
// bottleneck but FP64-level accuracy is needed: the direct-summation matvecs and
// the reduced-precision solve.
#pragma once

#include <cuda_runtime.h>

namespace ifmm {

struct df {
  float h, l;
};
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df df_quick(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
// a - (bh + bl) with a two-sum of the high parts; the low part is left
// unnormalised (its consumer squares it)
__device__ __forceinline__ df df_diff(df a, float bh, float bl) {
  const df s = df_two_sum(a.h, -bh);
  return {s.h, s.l + (a.l - bl)};
}
// d^2 for d = h + l: h^2 exactly as a pair (FMA), plus 2 h l + l^2.  The
// difference of two close points is not renormalised (df_diff), so l can be
// ~1e-3 of h there and l^2 is not negligible.
__device__ __forceinline__ df df_sq(df d) {
  const float p = d.h * d.h;
  return {p, fmaf(d.h, d.h, -p) + fmaf(d.l, d.l, 2.f * d.h * d.l)};
}
__device__ __forceinline__ df df_sum3(df a, df b, df c) {
  const df s = df_two_sum(a.h, b.h);
  const df u = df_two_sum(s.h, c.h);
  return df_quick(u.h, u.l + (s.l + (a.l + b.l + c.l)));
}
// 1/sqrt(x) as a pair: y0 = rsqrtf(x.h), one Newton step y0 + y0 (1 - x y0^2)/2
// with the residual formed from the exact products (1 - x y0^2 is ~1e-7, so
// its rounding is far below the pair's precision)
__device__ __forceinline__ df df_rsqrt_fast(df x) {
  const float y0 = rsqrtf(x.h);
  const float th = y0 * y0;
  const float tl = fmaf(y0, y0, -th);
  const float uh = x.h * th;
  const float ul = fmaf(x.h, th, -uh) + fmaf(x.h, tl, x.l * th);
  const float e = (1.f - uh) - ul;
  return {y0, 0.5f * y0 * e};
}
// acc + (ph + pl): two-sum of the high parts, low parts added
__device__ __forceinline__ df df_acc(df acc, float ph, float pl) {
  const df s = df_two_sum(acc.h, ph);
  return df_quick(s.h, s.l + (acc.l + pl));
}

}  // namespace ifmm
