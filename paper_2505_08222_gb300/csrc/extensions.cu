// Policy / estimator hooks (placeholder until those modules are linked in).
#include "runtime.cuh"

namespace ut {
ut_status extension_create(ut_env*) { return UT_OK; }
void extension_destroy(ut_env*) {}
cudaError_t extension_reset(ut_env*, cudaStream_t) { return cudaSuccess; }
cudaError_t extension_policy_actions(ut_env*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t extension_estimate(ut_env*, cudaStream_t) { return cudaErrorNotReady; }
const float* extension_logits(ut_env*) { return nullptr; }
int extension_policy_kernels(ut_env*) { return 0; }
uint16_t* extension_h(ut_env*) { return nullptr; }
}  // namespace ut
