// Device helpers shared by the FP64 and split-precision kernels.
#pragma once
#include <cstdint>

namespace tk {

// s + e = a + b exactly (s = fl(a + b)); every operation is an explicit round-to-nearest add, so
// the compiler cannot contract or reassociate it.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Exact FP32 -> FP64 by assembling the bit pattern with integer operations (the FP64 pipe is
// scarce on this part); zeros and FP32 subnormals/non-finite values take the hardware path.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xFFu;
  if (ex == 0u) {
    if ((u << 1) == 0u) return __longlong_as_double((long long)(u & 0x80000000u) << 32);  // +-0
    return (double)f;
  }
  if (ex == 0xFFu) return (double)f;
  const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}


}  // namespace tk
