// Instantiations of the particle-filter step, group A (see pf_variants.h).
#include "pf_kernel.cuh"
#include "pf_variants.h"

namespace ut {
namespace pf {

cudaError_t launch_variant_a(int v, const EnvDev& d, cudaStream_t s) {
  switch (v) {
#define UT_PF_CASE(i, nt, ppt, minb, name) \
  case i:                                  \
    return launch_step<nt, ppt, minb>(d, s);
    UT_PF_VARIANTS_A(UT_PF_CASE)
#undef UT_PF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace pf
}  // namespace ut
