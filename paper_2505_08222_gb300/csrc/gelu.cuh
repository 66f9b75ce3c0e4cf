// erf-GELU for the tensor-core networks' epilogues (transformer agent FFN,
// estimator hidden layers).
#pragma once

#include <cuda_runtime.h>

#include "f32x2.cuh"

namespace ut {

// GELU(x) = x Phi(x) = relu(x) - |x| Phi(-|x|), with Phi(-|x|) =
// erfc(|x| / sqrt 2) / 2 from the rational approximation of Abramowitz &
// Stegun, Handbook of Mathematical Functions, formula 7.1.26:
// erfc(z) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^(-z^2), t = 1 / (1 + p z),
// z >= 0, absolute error <= 1.5e-7.  The constants below fold the halving,
// the sign of the second term and z = |x| / sqrt 2 into the coefficients:
// t = 1 / (1 + (p / sqrt 2) |x|), e^(-z^2) = 2^(-x^2 log2(e) / 2).  In FP32 the
// GELU error stays below 5e-7 absolute, far inside the BF16 rounding its
// output receives.  Evaluated for two values at once on the packed FP32 pipe
// (the SFU reciprocal and exponential stay per lane).
__device__ __forceinline__ float ex2_sfu(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ void gelu2(float& x0, float& x1) {
  const float a0 = fabsf(x0), a1 = fabsf(x1);
  const unsigned long long A = f2pk(a0, a1);
  float d0, d1;
  f2upk(f2fma(A, f2pk(0.2316419f, 0.2316419f), f2pk(1.0f, 1.0f)), d0, d1);  // 0.3275911 / sqrt 2
  const unsigned long long t = f2pk(__fdividef(1.0f, d0), __fdividef(1.0f, d1));
  // -(a_k / 2), k = 5 .. 1
  unsigned long long c = f2fma(t, f2pk(-0.5307027145f, -0.5307027145f), f2pk(0.7265760135f, 0.7265760135f));
  c = f2fma(t, c, f2pk(-0.7107068705f, -0.7107068705f));
  c = f2fma(t, c, f2pk(0.1422483680f, 0.1422483680f));
  c = f2fma(t, c, f2pk(-0.1274147960f, -0.1274147960f));
  float s0, s1;
  f2upk(f2mul(f2mul(A, A), f2pk(-0.72134752044448170f, -0.72134752044448170f)), s0, s1);  // -log2(e) / 2
  c = f2mul(c, f2mul(t, f2pk(ex2_sfu(s0), ex2_sfu(s1))));  // -Phi(-|x|)
  f2upk(f2fma(A, c, f2pk(fmaxf(x0, 0.0f), fmaxf(x1, 0.0f))), x0, x1);
}

// The same value for one input (identical arithmetic in lane 0).
__device__ __forceinline__ float gelu1(float x) {
  float y = x, unused = 0.0f;
  gelu2(y, unused);
  return y;
}

}  // namespace ut
