// Device helpers shared by the FP64 and split-precision kernels.
#pragma once
#include <cstdint>

namespace tk {

// s + e = a + b exactly (s = fl(a + b)); every operation is an explicit round-to-nearest add, so
// the compiler cannot contract or reassociate it.
static __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Packed FP32 pairs (one instruction per pair on this part).  y - x as fma(x, -1, y): the product
// is exact, so this rounds exactly like a subtraction.
static __device__ __forceinline__ float2 sub2(float2 y, float2 x) {
  return __ffma2_rn(x, make_float2(-1.f, -1.f), y);
}
// two_sum on both lanes of a pair.
static __device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = __fadd2_rn(a, b);
  const float2 bb = sub2(s, a);
  e = __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// Exact FP32 -> FP64 of a subnormal, infinite or NaN FP32 value, out of line (rare).
static __device__ __noinline__ double f32_to_f64_rare(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xFFu, man = u & 0x7FFFFFu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if (ex == 0xFFu) return __longlong_as_double((long long)(sign | (0x7FFull << 52) | ((unsigned long long)man << 29)));
  const int p = 31 - __clz((int)man);  // subnormal: value man 2^-149, leading one at bit p
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(p + 874) << 52) | (((unsigned long long)man << (52 - p)) & 0xFFFFFFFFFFFFFull)));
}

// Exact FP32 -> FP64 by assembling the bit pattern with 32-bit integer operations (the FP64 pipe
// is scarce on this part); zeros and normal numbers inline, everything else out of line.  For a
// normal value the high word is the sign, then exponent and fraction shifted right by 3 with the
// exponent bias raised by 1023 - 127 = 896; the low word holds the fraction's last 3 bits.
static __device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xFFu;
  if (ex - 1u >= 0xFEu) {  // exponent field 0 or 255
    if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);  // +-0
    return f32_to_f64_rare(f);
  }
  const uint32_t hi = (u & 0x80000000u) | (((u & 0x7FFFFFFFu) >> 3) + (896u << 20));
  return __hiloint2double((int)hi, (int)(u << 29));
}

}  // namespace tk
