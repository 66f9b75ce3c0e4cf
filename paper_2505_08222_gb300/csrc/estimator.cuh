// Learned range-only estimator: device view and launchers (estimator.cu).
//
// MLP 96 -> 256 -> 256 -> 256 -> 2 with erf-GELU (reading C18).  Inputs are
// the 16 most recent pings of a filter's ring, newest first, each as
// [(qx - ax)/S, (qy - ay)/S, r/S, (g - g_m)/16, valid], zero padded to 96.
// The output is the target's position relative to the observer, in units of
// S.  FP32 master weights; BF16 operand images for the tensor cores (W for
// the forward pass, W^T for the input-gradient pass).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "env.cuh"

namespace ut {
namespace est {

constexpr int IN = 96;
constexpr int HID = 256;
constexpr int OUT = 2;
constexpr int NLIN = 4;
// parameter offsets in the canonical blob (floats)
constexpr int64_t W1_OFF = 0;
constexpr int64_t B1_OFF = W1_OFF + (int64_t)HID * IN;
constexpr int64_t W2_OFF = B1_OFF + HID;
constexpr int64_t B2_OFF = W2_OFF + (int64_t)HID * HID;
constexpr int64_t W3_OFF = B2_OFF + HID;
constexpr int64_t B3_OFF = W3_OFF + (int64_t)HID * HID;
constexpr int64_t W4_OFF = B3_OFF + HID;
constexpr int64_t B4_OFF = W4_OFF + (int64_t)OUT * HID;
constexpr int64_t NPARAM = B4_OFF + OUT;
// operand images (bytes): W1 [256 x 96], W2, W3 [256 x 256], and the
// transposes of W2, W3 for the backward pass
constexpr size_t IMG_W1 = (size_t)HID * IN * 2;
constexpr size_t IMG_W = (size_t)HID * HID * 2;
constexpr size_t IMG_W1_OFF = 0;
constexpr size_t IMG_W2_OFF = IMG_W1_OFF + IMG_W1;
constexpr size_t IMG_W3_OFF = IMG_W2_OFF + IMG_W;
constexpr size_t IMG_W2T_OFF = IMG_W3_OFF + IMG_W;
constexpr size_t IMG_W3T_OFF = IMG_W2T_OFF + IMG_W;
constexpr size_t IMG_BYTES = IMG_W3T_OFF + IMG_W;

// Partial-sum slabs of the backward pass: the bias / output-layer gradients
// (dW4 [2][256], db3, db2, db1 [256], db4 [2]) and the hidden weight
// gradients (dW1 [256][96], dW2, dW3 [256][256]); the batch is split over at
// most kWgradSplits weight-gradient CTAs per (layer, half).
constexpr int NB_PART = 2 * HID + 3 * HID + OUT;
constexpr int64_t NW_PART = (int64_t)HID * IN + 2 * (int64_t)HID * HID;
constexpr int kWgradSplits = 24;

struct Net {
  const unsigned char* img;  // operand images
  const float* master;       // FP32 parameters, canonical order (biases, W4)
};

// Training buffers for one batch of B rows.
struct TrainBufs {
  const float* X;        // [n_rows][96] features
  const float* Y;        // [n_rows][2] labels
  const int32_t* rows;   // [B] dataset rows of the batch (NULL: rows 0..B-1)
  float* z;              // [3][B][256] pre-activations
  uint16_t* a;           // [3][B][256] BF16 activations (GELU(z))
  float* out;            // [B][2]
  uint16_t* dz;          // [3][B][256] BF16 gradients w.r.t. z
  float* grad;           // [NPARAM] FP32 gradient
  double* loss;          // [1] loss of the batch
  // fixed-order partial sums (no atomics: the gradient is deterministic)
  float* part_b;         // [ceil(B/128)][NB_PART] per-CTA dW4, db3, db2, db1, db4
  double* part_loss;     // [ceil(B/128)] per-CTA loss sums
  float* part_w;         // [kWgradSplits][NW_PART] per-split dW1, dW2, dW3
  float huber;           // 0: squared error; > 0: Huber threshold (label units)
  int B;
};

cudaError_t launch_forward(const Net& net, const float* X, const int32_t* rows, int B, float* out, float* z,
                           uint16_t* a, cudaStream_t s);
cudaError_t launch_forward_env(const Net& net, const EnvDev& d, int stale, uint32_t test_wait_polls,
                               cudaStream_t s);
cudaError_t launch_record(const EnvDev& d, float* feat, float* label, cudaStream_t s);
cudaError_t launch_backward(const Net& net, const TrainBufs& t, cudaStream_t s);
cudaError_t launch_adam(float* master, float* m, float* v, const float* grad, int step, float lr, float beta1,
                        float beta2, float eps, unsigned char* img, cudaStream_t s);
cudaError_t launch_pack(const float* master, unsigned char* img, cudaStream_t s);
cudaError_t launch_batch_rows(int32_t* rows, int B, int64_t n_rows, uint64_t seed, uint32_t step, cudaStream_t s);

}  // namespace est
}  // namespace ut
