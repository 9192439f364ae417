// Device helpers shared by the library's translation units (internal).
#pragma once

#include "hac_internal.cuh"

namespace hacg {

enum { LK_COMPLETE = 0, LK_AVERAGE = 1, LK_WARD = 2, LK_AVG2 = 3 };

// Square roots by the hardware approximation (sqrt.approx.f32): with it a
// distance's relative error stays within ((d+1)/2 + 4)u <= (d+16)u, the
// bound the search states for FP32 distances.
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The same with subnormal inputs flushed to zero (one instruction fewer
// paths); callers account for the flush: a squared distance below 2^-126
// yields 0 instead of at most 2^-63.
__device__ __forceinline__ float sqrt_approx_ftz(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Packed FP32 pairs (f32x2 in a 64-bit word): each half is rounded as the
// scalar instruction would round it.
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ float f2_hsum(unsigned long long v) {
  float a, b;
  f2_unpack(v, a, b);
  return a + b;
}

}  // namespace hacg
