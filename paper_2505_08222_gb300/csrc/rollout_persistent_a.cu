// Persistent rollout instantiations, 4 particles per thread.
#include "rollout_persistent.cuh"

namespace ut {
namespace persist {

cudaError_t launch_ppt4(int nt, const EnvDev& d, int T, cudaStream_t s) {
  switch (nt) {
    case 32: return launch_shape<32, 4>(d, T, s);
    case 64: return launch_shape<64, 4>(d, T, s);
    case 128: return launch_shape<128, 4>(d, T, s);
    case 256: return launch_shape<256, 4>(d, T, s);
    case 512: return launch_shape<512, 4>(d, T, s);
    case 1024: return launch_shape<1024, 4>(d, T, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace persist
}  // namespace ut
