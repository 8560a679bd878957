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

// Exact FP32 -> FP64 by assembling the bit pattern with integer operations only (the FP64 pipe
// is scarce on this part): normal, subnormal (renormalised with a leading-zero count), zero,
// infinite and NaN inputs all take the same branch-free path.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xFFu, man = u & 0x7FFFFFu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  // normal numbers and infinities/NaNs (exponent 255 -> 2047)
  const unsigned long long e64 = ex == 0xFFu ? 0x7FFull : (unsigned long long)(ex + 896u);
  unsigned long long d = sign | (e64 << 52) | ((unsigned long long)man << 29);
  // subnormal: value man 2^-149 with its leading one at bit p
  const int p = 31 - __clz((int)(man | 1u));
  const unsigned long long dsub =
      sign | ((unsigned long long)(p + 874) << 52) | (((unsigned long long)man << (52 - p)) & 0xFFFFFFFFFFFFFull);
  d = ex != 0u ? d : (man != 0u ? dsub : sign);
  return __longlong_as_double((long long)d);
}

}  // namespace tk
