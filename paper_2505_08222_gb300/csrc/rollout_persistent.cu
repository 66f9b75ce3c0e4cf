// Persistent rollout: the launcher (the kernel is in rollout_persistent.cuh;
// its instantiations are split over rollout_persistent_a.cu (4 particles per
// thread) and rollout_persistent_b.cu (8) so that they compile in parallel).
#include "pf_variants.h"
#include "rollout_persistent.cuh"

namespace ut {
namespace persist {
cudaError_t launch_ppt4(int nt, const EnvDev& d, int T, cudaStream_t s);
cudaError_t launch_ppt8(int nt, const EnvDev& d, int T, cudaStream_t s);
}  // namespace persist

namespace {

// T steps done: the step counters and the step count of the metrics, as
// advance_kernel does once per step.
__global__ void advance_by_kernel(EnvDev d, uint32_t T) {
  if (threadIdx.x == 0) {
    d.counters[0] += T;
    d.counters[1] += T;
    d.metrics_u[3] += T;
  }
}

}  // namespace

bool persistent_supported(const EnvDev& d, int variant) {
  if (variant < 0 || variant >= pf::kNumVariants) return false;
  return d.pw == nullptr && d.E > 0 && d.P <= pf::kVariants[variant].nt * pf::kVariants[variant].ppt;
}

cudaError_t launch_rollout_persistent(const EnvDev& d, int variant, int T, cudaStream_t s) {
  if (!persistent_supported(d, variant) || T < 1) return cudaErrorInvalidValue;
  const int nt = pf::kVariants[variant].nt, ppt = pf::kVariants[variant].ppt;
  cudaError_t e = ppt == 4 ? persist::launch_ppt4(nt, d, T, s)
                           : (ppt == 8 ? persist::launch_ppt8(nt, d, T, s) : cudaErrorInvalidValue);
  if (e != cudaSuccess) return e;
  advance_by_kernel<<<1, 32, 0, s>>>(d, (uint32_t)T);
  return cudaGetLastError();
}

}  // namespace ut
