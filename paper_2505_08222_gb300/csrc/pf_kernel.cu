// Particle-filter step: launch variants, the launcher and the stand-alone
// resample map.  The kernel itself is in pf_kernel.cuh; its instantiations are
// split over pf_inst_a.cu / pf_inst_b.cu so that they compile in parallel.
#include "pf_kernel.cuh"
#include "pf_variants.h"

namespace ut {

int pf_variant_count() { return pf::kNumVariants; }
const char* pf_variant_name(int v) { return (v >= 0 && v < pf::kNumVariants) ? pf::kVariants[v].name : "?"; }

bool pf_variant_valid(int v, int P) {
  if (v < 0 || v >= pf::kNumVariants) return false;
  const int cap = pf::kVariants[v].nt * pf::kVariants[v].ppt;
  // enough slots, and at most half of them idle (beyond the smallest block)
  return cap >= P && (2 * P > cap || pf::kVariants[v].nt == 32);
}

int pf_default_variant(int P) {
  // smallest 4-particles-per-thread block that covers P (variants 0..5)
  for (int v = 0; v < 6; ++v)
    if (pf::kVariants[v].nt * 4 >= P) return v;
  return 5;
}

cudaError_t launch_pf_step(const EnvDev& d, int variant, cudaStream_t s) {
  if (variant < 0 || variant >= pf::kNumVariants) return cudaErrorInvalidValue;
  return pf::launch_variant(variant, d, s);
}

namespace {
template <int NT, int PPT>
cudaError_t launch_resample_t(const float* w, const uint64_t* u, int64_t F, int P, int32_t* idx, cudaStream_t s) {
  static std::atomic<unsigned long long> ready{0};
  const size_t smem = pf::resample_smem_bytes(NT, PPT);
  auto k = pf::pf_resample_kernel<NT, PPT>;
  cudaError_t e = smem_optin(k, smem, ready);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)F, NT, smem, s>>>(w, u, P, idx);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_pf_resample(const float* wmax, const uint64_t* u64, int64_t n_filters, int P, int32_t* idx,
                               cudaStream_t s) {
  if (n_filters <= 0) return cudaSuccess;
  if (P <= 128) return launch_resample_t<32, 4>(wmax, u64, n_filters, P, idx, s);
  if (P <= 256) return launch_resample_t<64, 4>(wmax, u64, n_filters, P, idx, s);
  if (P <= 512) return launch_resample_t<128, 4>(wmax, u64, n_filters, P, idx, s);
  if (P <= 1024) return launch_resample_t<256, 4>(wmax, u64, n_filters, P, idx, s);
  if (P <= 2048) return launch_resample_t<512, 4>(wmax, u64, n_filters, P, idx, s);
  return launch_resample_t<1024, 4>(wmax, u64, n_filters, P, idx, s);
}

}  // namespace ut
