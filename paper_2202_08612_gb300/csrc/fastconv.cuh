// The hi/lo bfloat16 split of the split-precision path, kept off the FP64 pipe
// (on GB300 it retires about two FP64 operations per clock and SM, so an FP64
// subtraction or a double -> bf16 rounding per element bounds an otherwise
// memory-bound pass): one FP64 -> FP32 conversion, then FP32 work only.
#pragma once
#include <cuda_bf16.h>

namespace mlcc3 {

// x ~ hi + lo with hi = bf16(f), lo = bf16(f - hi), f = binary32(x); f - hi is
// exact in binary32 (it keeps the 16 low bits of f's significand).
__device__ __forceinline__ void split_hi_lo(double x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  const float f = __double2float_rn(x);
  hi = __float2bfloat16_rn(f);
  lo = __float2bfloat16_rn(f - __bfloat162float(hi));
}

// The same split of a binary32 value (no conversion from binary64).
__device__ __forceinline__ void split_hi_lo(float f, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(f);
  lo = __float2bfloat16_rn(f - __bfloat162float(hi));
}

// x scaled by +1 (mode 0), -1 (mode 1, a sign flip of the bit pattern) or s.
__device__ __forceinline__ double scaled(double x, int mode, double s) {
  if (mode == 0) return x;
  if (mode == 1) return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
  return s * x;
}

__device__ __forceinline__ float scaled(float x, int mode, double s) {
  if (mode == 0) return x;
  if (mode == 1) return -x;
  return (float)s * x;
}

}  // namespace mlcc3
