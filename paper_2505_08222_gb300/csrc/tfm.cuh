// Transformer training handle (tfm.cu): what other translation units of the
// library use of it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct ut_tfm;

namespace ut {

// Configuration of a handle.
struct TfmInfo {
  int d, n_layers, n_heads, n_out, n_slots, tokens_bf16;
  long long max_batch;
};
TfmInfo tfm_info(const ut_tfm* t);

// Forward of n samples (as tfm_forward, no row selection) enqueued on stream s
// instead of the handle's own stream (e.g. a stream being captured).
cudaError_t tfm_forward_on(ut_tfm* t, const void* tokens, const int32_t* n_ent, const float* h, long long n,
                           float* out, float* h_out, cudaStream_t s);

}  // namespace ut
