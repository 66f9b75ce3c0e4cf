// erf-GELU for the tensor-core networks' epilogues (transformer agent FFN,
// estimator hidden layers).
#pragma once

#include <cuda_runtime.h>

namespace ut {

// GELU(x) = x Phi(x) with Phi(-|x|) = erfc(|x| / sqrt 2) / 2 from the rational
// approximation of Abramowitz & Stegun, Handbook of Mathematical Functions,
// formula 7.1.26: erfc(z) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^(-z^2),
// t = 1 / (1 + p z), z >= 0, absolute error <= 1.5e-7 (the coefficients below
// are that formula's, halved).  In FP32 the GELU error stays below 5e-7
// absolute, far inside the BF16 rounding its output receives.
// Evaluated for two values at once on the packed FP32 pipe (fma / mul
// .rn.f32x2, each lane rounded like the scalar operation; the SFU reciprocal
// and exponential stay per lane).
__device__ __forceinline__ unsigned long long f2pk(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2upk(unsigned long long r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ unsigned long long f2mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ void gelu2(float& x0, float& x1) {
  const unsigned long long x = f2pk(x0, x1);
  const unsigned long long z = f2mul(f2pk(fabsf(x0), fabsf(x1)), f2pk(0.70710678118654752f, 0.70710678118654752f));
  float d0, d1;
  f2upk(f2fma(f2pk(0.3275911f, 0.3275911f), z, f2pk(1.0f, 1.0f)), d0, d1);
  const unsigned long long t = f2pk(__fdividef(1.0f, d0), __fdividef(1.0f, d1));
  unsigned long long c = f2fma(t, f2pk(0.5307027145f, 0.5307027145f), f2pk(-0.7265760135f, -0.7265760135f));
  c = f2fma(t, c, f2pk(0.7107068705f, 0.7107068705f));
  c = f2fma(t, c, f2pk(-0.1422483680f, -0.1422483680f));
  c = f2fma(t, c, f2pk(0.1274147960f, 0.1274147960f));
  float z0, z1;
  f2upk(z, z0, z1);
  c = f2mul(c, f2mul(t, f2pk(__expf(-z0 * z0), __expf(-z1 * z1))));
  float c0, c1;
  f2upk(c, c0, c1);
  float y0, y1;
  f2upk(f2mul(x, f2pk(x0 >= 0.0f ? 1.0f - c0 : c0, x1 >= 0.0f ? 1.0f - c1 : c1)), y0, y1);
  x0 = y0;
  x1 = y1;
}

// The same value for one input (identical arithmetic in lane 0).
__device__ __forceinline__ float gelu1(float x) {
  float y = x, unused = 0.0f;
  gelu2(y, unused);
  return y;
}

}  // namespace ut
