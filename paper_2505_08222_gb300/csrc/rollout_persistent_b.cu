// Persistent rollout instantiations, 8 particles per thread.
#include "rollout_persistent.cuh"

namespace ut {
namespace persist {

cudaError_t launch_ppt8(int nt, const EnvDev& d, int T, cudaStream_t s) {
  switch (nt) {
    case 64: return launch_shape<64, 8>(d, T, s);
    case 128: return launch_shape<128, 8>(d, T, s);
    case 256: return launch_shape<256, 8>(d, T, s);
    case 512: return launch_shape<512, 8>(d, T, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace persist
}  // namespace ut
