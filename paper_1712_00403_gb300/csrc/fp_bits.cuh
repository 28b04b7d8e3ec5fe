// Conversions between binary64 and binary32 done on the integer units, from
// the IEEE 754 encodings (sign | biased exponent | fraction; biases 1023 and
// 127). GB300 runs FP64 instructions, conversions included, at a small
// fraction of its FP32/integer rate, so the streaming kernels that change
// precision (the double-float split and join, the FP64 -> FP32 operand
// conversion of the tensor-core path, the FP64 output of its epilogue) are
// bound by that unit when they use the conversion instructions. Values outside
// the ranges handled here (zero, subnormal, very small or very large, infinite,
// NaN) take the conversion instructions.
#pragma once
#include <cuda_runtime.h>

namespace fdst {

// Exact float -> double: rebias the exponent (+896 = 1023 - 127) and move the
// 23 fraction bits to the top of the 52-bit fraction.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ex = (b >> 23) & 0xFFu;
  if (ex - 1u < 254u) {
    const unsigned hi = (b & 0x80000000u) | (((b >> 3) & 0x0FFFFFFFu) + (896u << 20));
    return __hiloint2double((int)hi, (int)(b << 29));
  }
  return (double)f;
}

// double -> float, rounded to nearest (ties to even): the top 23 fraction bits
// with the exponent rebiased, plus one unit when the 29 dropped bits exceed
// half a unit (or equal it and the kept part is odd); a carry out of the
// fraction increments the exponent, and past the largest finite float gives
// infinity, as the rounding rule requires. Normal float range only.
__device__ __forceinline__ float f64_to_f32_rn(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned ex = (hi >> 20) & 0x7FFu;
  if (ex - 897u < 254u) {   // unbiased exponent in [-126, 127]
    unsigned bits = (hi & 0x80000000u) | ((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1FFFFFFFu;
    bits += (rem > 0x10000000u) || (rem == 0x10000000u && (bits & 1u));
    return __uint_as_float(bits);
  }
  return __double2float_rn(v);
}

// double -> double-float pair (hi, lo) with hi + lo = v to within 2^-48 |v|:
// hi keeps the top 24 significand bits (truncated), lo is the remaining 29-bit
// tail rounded to nearest as a normal float. Unbiased exponents in [-74, 127]
// (the tail's exponent is then at least -126).
__device__ __forceinline__ float2 f64_split(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned ex = (hi >> 20) & 0x7FFu;
  if (ex - 949u <= 201u) {
    const unsigned s = hi & 0x80000000u;
    const float fh = __uint_as_float(s | ((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
    const unsigned r = lo & 0x1FFFFFFFu;   // tail: r * 2^(e - 52)
    if (r == 0u) return make_float2(fh, 0.0f);
    const int msb = 31 - __clz((int)r);     // 0 .. 28
    int e2 = (int)ex - 1075 + msb;          // unbiased exponent of the tail's leading bit
    unsigned sig;
    if (msb <= 23) {
      sig = r << (23 - msb);
    } else {
      const int sh = msb - 23;               // 1 .. 5 bits dropped
      const unsigned q = r >> sh, rem = r & ((1u << sh) - 1u), half = 1u << (sh - 1);
      sig = q + ((rem > half) || (rem == half && (q & 1u)));
      if (sig >> 24) { sig >>= 1; ++e2; }
    }
    return make_float2(fh, __uint_as_float(s | ((unsigned)(e2 + 127) << 23) | (sig & 0x7FFFFFu)));
  }
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

// double-float pair -> double: both parts converted exactly, one FP64 add.
__device__ __forceinline__ double f64_join(float2 v) { return f32_to_f64(v.x) + f32_to_f64(v.y); }

}  // namespace fdst
