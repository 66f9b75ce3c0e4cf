// Device-side helpers shared by the tracking-environment kernels.
//
// Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11), keyed by the 64-bit
// seed, counter = (id0, id1, global step, stream tag).  Every random draw of
// the environment is addressed by what it belongs to (env, agent, target,
// filter, particle pair, step), so the sequence does not depend on the launch
// configuration and a CPU program can replay it.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace ut {

// Programmatic dependent launch between the kernels of one environment step:
// every step kernel waits for its predecessor's completion and memory before
// its first global access (pdl_wait); the small single-wave kernels also let
// the next kernel launch as soon as all of their own CTAs are running
// (pdl_trigger), the many-wave ones (filter, policy, estimator) let it launch
// as their CTAs exit, so that no waiting CTA holds an SM during their last
// wave.  Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with programmatic stream serialization: the kernel may start while
// the previous kernel in the stream is still running, so it must call
// pdl_wait() before touching memory that kernel writes.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Dynamic shared memory above the default limit is a per-device function
// attribute: opt each kernel in once on every device it runs on.  `mask`
// holds one bit per device index (devices >= 64 set the attribute on every
// call).
template <typename K>
inline cudaError_t smem_optin(K kernel, size_t bytes, std::atomic<unsigned long long>& mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit && (mask.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && bit) mask.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Stream tags (counter word 3).
enum : uint32_t {
  TAG_SPAWN = 1,
  TAG_AGENT_INIT = 2,
  TAG_TARGET_INIT = 3,
  TAG_PF_INIT = 4,
  TAG_PF_INIT2 = 5,
  TAG_ACTION = 6,
  TAG_AGENT_NOISE = 7,
  TAG_TARGET_MOVE = 8,
  TAG_PING = 9,
  TAG_COMM = 10,
  TAG_PF_PREDICT = 11,
  TAG_RESAMPLE = 12,
  TAG_GUMBEL = 13,
  TAG_RESET_PING = 15,
};

constexpr int kMaxAgents = 8;
constexpr int kMaxTargets = 8;
constexpr int kRing = 16;
constexpr int kFeat = 96;
constexpr float kPi = 3.14159265358979323846f;
// Smoothing of the estimate's motion: v <- kVelKeep v + (1 - kVelKeep) (e1 - e2)
// at every tracker update (learned estimator features, readings C18).
constexpr float kVelKeep = 0.85f;
constexpr float kTwoPi = 6.28318530717958647692f;

struct Rand4 {
  uint32_t x[4];
};

// Philox4x32-10.  Each round multiplies counter words 0 and 2 by the two
// published 32-bit multipliers; the high words are xored with words 1 / 3
// and the round key, the low words move to positions 1 / 3.  The key is
// bumped by the two Weyl constants between rounds.
__device__ __forceinline__ Rand4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    uint32_t lo_a = m0 * c0, hi_a = __umulhi(m0, c0);
    uint32_t lo_b = m1 * c2, hi_b = __umulhi(m1, c2);
    c0 = hi_b ^ c1 ^ k0;
    c1 = lo_b;
    c2 = hi_a ^ c3 ^ k1;
    c3 = lo_a;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  Rand4 r;
  r.x[0] = c0; r.x[1] = c1; r.x[2] = c2; r.x[3] = c3;
  return r;
}

// Uniform [0,1) from the top 24 bits: exact in fp32.
__device__ __forceinline__ float unif(uint32_t v) { return (float)(v >> 8) * 0x1p-24f; }
// Uniform (0,1].
__device__ __forceinline__ float unif_pos(uint32_t v) { return (float)((v >> 8) + 1u) * 0x1p-24f; }
// Uniform (0,1), cell midpoints.
__device__ __forceinline__ float unif_mid(uint32_t v) { return ((float)(v >> 8) + 0.5f) * 0x1p-24f; }

// Box-Muller transform: two standard normals from two uniforms.
__device__ __forceinline__ void box_muller(uint32_t va, uint32_t vb, float& n0, float& n1) {
  float rad = sqrtf(-2.0f * logf(unif_pos(va)));
  float s, c;
  sincospif(2.0f * unif(vb), &s, &c);
  n0 = rad * c;
  n1 = rad * s;
}

// Angle wrapped to [-pi, pi).
__device__ __forceinline__ float wrap_angle(float a) { return a - kTwoPi * floorf((a + kPi) / kTwoPi); }

__device__ __forceinline__ uint16_t f2bf_bits(float v) {
  __nv_bfloat16 b = __float2bfloat16_rn(v);
  return *reinterpret_cast<uint16_t*>(&b);
}
__device__ __forceinline__ float bf_bits2f(uint16_t v) { return __uint_as_float(((uint32_t)v) << 16); }
// Two FP32 values rounded to BF16 (nearest even, as f2bf_bits) and packed,
// lo in the low half: one cvt.rn.bf16x2.f32, whose first source goes to the
// upper half.
__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Warp reductions.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Device error word: first error code wins.  Codes: 1 an action outside
// [0, n_actions), 2 a bounded wait that gave up, 3 an index check of the
// checked build that failed.
__device__ __forceinline__ void raise_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Checked build (-DUT_CHECKED): the kernels test their data-dependent
// indexes (counts read from the CSR offsets and measurement headers, the
// resample map, shared-memory slots) before using them; a failed test records
// status 3 and the access is skipped, with no trap, so the context stays
// usable and the next synchronising call reports it.  In the normal build
// UT_IN_BOUNDS(cond, status) is the constant true and the test compiles away.
__device__ __forceinline__ bool check_bounds(bool ok, int* status) {
  if (!ok) raise_status(status, 3);
  return ok;
}
#ifdef UT_CHECKED
#define UT_IN_BOUNDS(cond, status) (::ut::check_bounds((cond), (status)))
#else
#define UT_IN_BOUNDS(cond, status) (true)
#endif

}  // namespace ut
