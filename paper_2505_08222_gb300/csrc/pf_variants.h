// Launch variants of the particle-filter step: threads per filter (NT),
// particles per thread (PPT) and the minimum resident CTAs per SM the
// compiler must allow (MINB, which caps registers per thread).
#pragma once

#include "env.cuh"

namespace ut {
namespace pf {

struct Variant {
  int nt, ppt, minb;
  const char* name;
};

// X(index, NT, PPT, MINB); the first six are the defaults for P <= 128 .. 4096.
#define UT_PF_VARIANTS_A(X)             \
  X(0, 32, 4, 16, "nt32x4")            \
  X(1, 64, 4, 16, "nt64x4")            \
  X(2, 128, 4, 8, "nt128x4")           \
  X(3, 256, 4, 4, "nt256x4")           \
  X(4, 512, 4, 2, "nt512x4")           \
  X(5, 1024, 4, 1, "nt1024x4")         \
  X(6, 128, 4, 12, "nt128x4m12")       \
  X(7, 256, 4, 6, "nt256x4m6")
#define UT_PF_VARIANTS_B(X)             \
  X(8, 512, 4, 3, "nt512x4m3")         \
  X(9, 64, 8, 16, "nt64x8")            \
  X(10, 128, 8, 8, "nt128x8")          \
  X(11, 256, 8, 4, "nt256x8")          \
  X(12, 512, 8, 2, "nt512x8")          \
  X(13, 256, 8, 3, "nt256x8m3")        \
  X(14, 128, 8, 6, "nt128x8m6")

#define UT_PF_ENTRY(i, nt, ppt, minb, name) {nt, ppt, minb, name},
constexpr Variant kVariants[] = {UT_PF_VARIANTS_A(UT_PF_ENTRY) UT_PF_VARIANTS_B(UT_PF_ENTRY)};
#undef UT_PF_ENTRY
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

// Defined in pf_inst_a.cu / pf_inst_b.cu.
cudaError_t launch_variant_a(int v, const EnvDev& d, cudaStream_t s);
cudaError_t launch_variant_b(int v, const EnvDev& d, cudaStream_t s);

inline cudaError_t launch_variant(int v, const EnvDev& d, cudaStream_t s) {
  return v < 8 ? launch_variant_a(v, d, s) : launch_variant_b(v, d, s);
}

}  // namespace pf
}  // namespace ut
