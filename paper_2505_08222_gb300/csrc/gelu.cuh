// erf-GELU for the tensor-core networks' epilogues (transformer agent FFN,
// estimator hidden layers).
#pragma once

#include <cuda_runtime.h>

#include "f32x2.cuh"

namespace ut {

// GELU(x) = x Phi(x) = relu(x) - |x| Phi(-|x|), with
// Phi(-a) = e^(-a^2 / 2) Q(min(a, 4)): Q is a degree-8 polynomial fitted to
// Phi(-a) e^(a^2 / 2) = erfc(a / sqrt 2) e^(a^2 / 2) / 2 on [0, 4] (gelu_fit.py:
// least squares on the relative error, reweighted towards minimax; beyond 4
// the Gaussian factor makes the term negligible).  The largest absolute GELU
// error of this FP32 evaluation is 5.4e-6 over [-12, 12] (against FP64 erf),
// far inside the BF16 rounding its output receives.  One SFU operation per
// value (the exponential, 2^(-a^2 log2(e) / 2)); the rest runs two values at
// once on the packed FP32 pipe, relu and the subtraction included (one fma).
__device__ __forceinline__ float ex2_sfu(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ void gelu2(float& x0, float& x1) {
  const float a0 = fabsf(x0), a1 = fabsf(x1);
  const unsigned long long X = f2pk(x0, x1);
  const unsigned long long A = f2pk(a0, a1);
  const unsigned long long a = f2pk(fminf(a0, 4.0f), fminf(a1, 4.0f));
  // -Q(a) by Horner (the coefficients of Q negated: the same roundings)
  unsigned long long q = f2fma(a, f2pk(-1.348651040e-05f, -1.348651040e-05f), f2pk(2.779782226e-04f, 2.779782226e-04f));
  q = f2fma(a, q, f2pk(-2.518137917e-03f, -2.518137917e-03f));
  q = f2fma(a, q, f2pk(1.338012610e-02f, 1.338012610e-02f));
  q = f2fma(a, q, f2pk(-4.741621763e-02f, -4.741621763e-02f));
  q = f2fma(a, q, f2pk(1.223185360e-01f, 1.223185360e-01f));
  q = f2fma(a, q, f2pk(-2.459359616e-01f, -2.459359616e-01f));
  q = f2fma(a, q, f2pk(3.983022571e-01f, 3.983022571e-01f));
  q = f2fma(a, q, f2pk(-4.999814630e-01f, -4.999814630e-01f));
  float s0, s1;
  f2upk(f2mul(f2mul(A, A), f2pk(-0.72134752044448170f, -0.72134752044448170f)), s0, s1);  // -log2(e) / 2
  const unsigned long long ae = f2mul(A, f2pk(ex2_sfu(s0), ex2_sfu(s1)));
  // relu(x) - |x| e^(-x^2 / 2) Q as one rounding: (x + |x|) / 2 is relu(x)
  // exactly, and the fma adds the (exactly negated) product
  f2upk(f2fma(f2add(X, A), f2pk(0.5f, 0.5f), f2mul(ae, q)), x0, x1);
}

// The same value for one input (identical arithmetic in lane 0).
__device__ __forceinline__ float gelu1(float x) {
  float y = x, unused = 0.0f;
  gelu2(y, unused);
  return y;
}

}  // namespace ut
