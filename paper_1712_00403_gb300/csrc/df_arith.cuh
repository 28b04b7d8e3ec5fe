// Double-float arithmetic on the FP32 units: a value is the unevaluated sum
// hi + lo of two floats (48-bit significand). Products use the exact FMA
// residual (p = a*b, e = fma(a, b, -p)), sums Knuth's branch-free TwoSum.
#pragma once
#include <cuda_runtime.h>

namespace fdst {

// (sh, sl) += a * b, a and b double-float; sl collects the rounding errors.
__device__ __forceinline__ void df_fma_acc(float2 a, float2 b, float &sh, float &sl) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float t = sh + p;
  const float z = t - sh;
  const float err = (sh - (t - z)) + (p - z);
  sh = t;
  sl = sl + (err + e);
}

// Renormalized pair (|lo| <= half an ulp of hi).
__device__ __forceinline__ float2 df_norm(float sh, float sl) {
  const float h = sh + sl;
  return make_float2(h, sl - (h - sh));
}

// (sh, sl) += (bh, bl).
__device__ __forceinline__ void df_add(float &sh, float &sl, float bh, float bl) {
  const float t = sh + bh;
  const float z = t - sh;
  const float err = (sh - (t - z)) + (bh - z);
  sh = t;
  sl = sl + (err + bl);
}

}  // namespace fdst
