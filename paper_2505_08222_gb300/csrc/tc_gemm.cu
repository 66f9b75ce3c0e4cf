// Plain BF16 GEMM on the 5th-generation tensor cores: C = A * B^T with FP32
// accumulation in tensor memory.  It exposes, on its own, the operand layout,
// descriptors and TMEM read-back that the fused transformer and estimator
// kernels build on, so they can be checked against a host matmul.
#include "../../include/utrack.h"
#include "common.cuh"
#include "tc.cuh"

namespace ut {
namespace {

constexpr int kGemmThreads = 128;
constexpr int kMaxK = 256;
constexpr int kMaxN = 256;
// A [128 x K] + B [N x K] operand images, plus slack so that the operand
// regions are never the last bytes of the allocation.
constexpr size_t kGemmSmem = (size_t)128 * kMaxK * 2 + (size_t)kMaxN * kMaxK * 2 + 16384;

// One CTA per 128-row block of A; N <= 256, K <= 256 (multiples of 16).
__global__ void __launch_bounds__(kGemmThreads) tc_gemm_kernel(const uint16_t* __restrict__ A,
                                                               const uint16_t* __restrict__ B,
                                                               float* __restrict__ C, int M, int N, int K,
                                                               int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;
  unsigned char* sB = smem + (size_t)128 * kMaxK * 2;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * 128;

  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&mbar, 1);

  // stage operands in the K-major core-row layout (16-byte chunks)
  for (int c = tid; c < 128 * (K / 8); c += kGemmThreads) {
    const int row = c % 128, kc = c / 128;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (m0 + row < M) v = *reinterpret_cast<const uint4*>(A + (size_t)(m0 + row) * K + kc * 8);
    *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(row, kc * 8, 128)) = v;
  }
  for (int c = tid; c < N * (K / 8); c += kGemmThreads) {
    const int row = c % N, kc = c / N;
    *reinterpret_cast<uint4*>(sB + tc::kmajor_offset(row, kc * 8, N)) =
        *reinterpret_cast<const uint4*>(B + (size_t)row * K + kc * 8);
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (tid == 0) {
    const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
    const uint32_t idesc = tc::idesc_bf16(128, N);
    for (int k = 0; k < K / 16; ++k) {
      const uint64_t ad = tc::smem_desc(a0 + k * 2 * 128 * 16, 128 * 16, 128);
      const uint64_t bd = tc::smem_desc(b0 + k * 2 * N * 16, N * 16, 128);
      tc::mma_bf16(tmem, ad, bd, idesc, k > 0 ? 1u : 0u);
    }
    tc::mma_commit(&mbar);
  }
  const bool ok = tc::mbar_wait(&mbar, 0);
  if (!ok && tid == 0 && status) atomicExch(status, 4);
  tc::fence_after_sync();

  if (ok) {
    const int row = warp * 32 + (tid & 31);
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int n0 = 0; n0 < N; n0 += 16) {
      float v[16];
      tc::tmem_ld16(lane_addr + n0, v);
      if (m0 + row < M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) C[(size_t)(m0 + row) * N + n0 + i] = v[i];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

}  // namespace
}  // namespace ut

extern "C" ut_status tc_gemm_bf16(const uint16_t* A_dev, const uint16_t* B_dev, float* C_dev, int32_t M, int32_t N,
                                  int32_t K, int32_t* status_dev, void* cuda_stream) {
  if (M < 1 || N < 16 || N > 256 || N % 16 || K < 16 || K > 256 || K % 16) return UT_ERR_INVALID;
  if (!A_dev || !B_dev || !C_dev) return UT_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(A_dev) | reinterpret_cast<uintptr_t>(B_dev)) & 15) return UT_ERR_INVALID;
  static std::atomic<unsigned long long> ready{0};
  if (ut::smem_optin(ut::tc_gemm_kernel, ut::kGemmSmem, ready) != cudaSuccess) return UT_ERR_CUDA;
  ut::tc_gemm_kernel<<<(M + 127) / 128, ut::kGemmThreads, ut::kGemmSmem, (cudaStream_t)cuda_stream>>>(
      A_dev, B_dev, C_dev, M, N, K, status_dev);
  return cudaGetLastError() == cudaSuccess ? UT_OK : UT_ERR_CUDA;
}
