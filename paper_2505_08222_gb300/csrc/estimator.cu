// Learned range-only estimator kernels: forward (inference and training),
// input-gradient pass, weight-gradient pass, Adam, feature recording.
//
// All three hidden layers run on the tensor cores (tcgen05.mma, BF16 x BF16 ->
// FP32 in TMEM) with 128 rows per CTA: one thread per row in the epilogues of
// the training / stand-alone forward, four per row in the environment step's
// forward (fwd_env_kernel).  The first layer's inputs are FP32 features split into a BF16
// high part and a BF16 remainder that are multiplied by the same weights and
// accumulated together: ranges of hundreds of metres keep ~1e-5 relative
// precision instead of BF16's 4e-3, which matters for metre-level tracking.
// The 2-wide output layer runs on CUDA cores.
#include "estimator.cuh"
#include "gelu.cuh"
#include "tc.cuh"

#include <cmath>
#include <cstring>

namespace ut {
namespace est {
namespace {

constexpr int kT = 128;
constexpr uint32_t TAG_BATCH = 14;
constexpr float kMaxCorr = 3.0f;  // largest correction per step, in units of L
constexpr size_t kFwdSmem = 65536 + 65536;
constexpr size_t kWgradSmem = 32768 + 65536;

// Derivative of erf-GELU for the backward pass: Phi(x) + x phi(x).  (The
// forward passes evaluate GELU with gelu.cuh's form, within 5.4e-6 of the
// erf form.)
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

__device__ __forceinline__ void store8(unsigned char* img, int row, int k0, int rows, const float* v) {
  uint4 p;
  p.x = bf16x2_bits(v[0], v[1]);
  p.y = bf16x2_bits(v[2], v[3]);
  p.z = bf16x2_bits(v[4], v[5]);
  p.w = bf16x2_bits(v[6], v[7]);
  *reinterpret_cast<uint4*>(img + tc::kmajor_offset(row, k0, rows)) = p;
}

__device__ __forceinline__ void copy_img(unsigned char* dst, const unsigned char* __restrict__ src, size_t bytes) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* t = reinterpret_cast<uint4*>(dst);
  for (size_t i = threadIdx.x; i < bytes / 16; i += kT) t[i] = __ldg(s + i);
}

// Estimator features of filter f for its update at step g (reading C18):
// in the local frame of the filter's current estimate e1 (units of L), each
// of the 16 most recent pings, newest first, as [(q - e1) / L, range
// innovation (r - |q - e1|_3D) / L, (g - g_m) / 16, 1], then the last motion
// of the estimate (e1 - e2) / L and its smoothed motion v / L (the velocity
// EMA including this update's e1 - e2); zero padded to 96.  The network's
// output is the correction (x - e1) / L.
__device__ __forceinline__ void ring_features(const EnvDev& d, int f, uint32_t g, float e1x, float e1y, float e2x,
                                              float e2y, float vx, float vy, float (&x)[IN]) {
  const int it = d.filt_target[f];
  const float dz = UT_IN_BOUNDS(it >= 0 && it < d.NT, d.status) ? d.tz[it] : 0.0f;  // target depth; senders at the surface
  const float L = d.est_scale;
  const int head = d.ring_head[f], cnt = d.ring_count[f];
  const float4* ring = reinterpret_cast<const float4*>(d.ring) + (long long)f * kRing;
#pragma unroll
  for (int s = 0; s < kRing; ++s) {
    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool on = s < cnt;
    if (on) e = ring[(head - 1 - s) & (kRing - 1)];
    const float dx = e.x - e1x, dy = e.y - e1y;
    const float rho = sqrtf(dx * dx + dy * dy + dz * dz);
    x[5 * s + 0] = on ? dx / L : 0.0f;
    x[5 * s + 1] = on ? dy / L : 0.0f;
    x[5 * s + 2] = on ? (e.z - rho) / L : 0.0f;
    x[5 * s + 3] = on ? ((float)g - e.w) / 16.0f : 0.0f;
    x[5 * s + 4] = on ? 1.0f : 0.0f;
  }
  x[5 * kRing] = (e1x - e2x) / L;
  x[5 * kRing + 1] = (e1y - e2y) / L;
  x[5 * kRing + 2] = vx / L;
  x[5 * kRing + 3] = vy / L;
#pragma unroll
  for (int i = 5 * kRing + 4; i < IN; ++i) x[i] = 0.0f;
}

struct FwdArgs {
  Net net;
  const float* X;
  const int32_t* rows;
  int B;
  float* out;
  float* z;     // training: [3][B][256], else NULL
  uint16_t* a;  // training: [3][B][256], else NULL
  int* status;
};

__global__ void __launch_bounds__(kT, 1) fwd_kernel(FwdArgs p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;          // features hi | lo, then hidden activations [128 x 256]
  unsigned char* sB = smem + 65536;  // one weight chunk [128 x K]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long b = (long long)blockIdx.x * kT + tid;
  const long long n = (long long)p.B;
  const bool valid = b < n;

  if (warp == 0) {
    tc::tmem_alloc(&tbase, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&mbar, 1);

  float x[IN];
  {
    const long long src = valid ? (p.rows ? (long long)p.rows[b] : b) : 0;
#pragma unroll
    for (int i = 0; i < IN; i += 4) {
      float4 v = valid ? __ldg(reinterpret_cast<const float4*>(p.X + src * IN + i)) : make_float4(0.f, 0.f, 0.f, 0.f);
      x[i] = v.x; x[i + 1] = v.y; x[i + 2] = v.z; x[i + 3] = v.w;
    }
  }
#pragma unroll
  for (int c0 = 0; c0 < IN; c0 += 8) {
    float hi[8], lo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      hi[i] = bf_bits2f(f2bf_bits(x[c0 + i]));
      lo[i] = x[c0 + i] - hi[i];
    }
    store8(sA, tid, c0, 128, hi);
    store8(sA + 128 * IN * 2, tid, c0, 128, lo);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t aA = tc::smem_addr(sA), aB = tc::smem_addr(sB);
  uint32_t phase = 0;
  bool ok = true;
  const float* mst = p.net.master;

  // layer 1: K = 96, both halves of the features, two N-halves of 128
  {
    const uint32_t a2[2] = {aA, aA + 128 * IN * 2};
    for (int h = 0; h < 2; ++h) {
      copy_img(sB, p.net.img + IMG_W1_OFF + (size_t)h * 128 * IN * 2, (size_t)128 * IN * 2);
      ok &= tc::mma_group(tmem + 128 * h, a2, 2, aB, 128, IN, false, &mbar, phase);
    }
  }
  float o0 = 0.0f, o1 = 0.0f;
  for (int l = 0; l < 3; ++l) {
    // epilogue of hidden layer l: z = acc + b, a = GELU(z) -> next A operand
    const float* bias = mst + (l == 0 ? B1_OFF : (l == 1 ? B2_OFF : B3_OFF));
#pragma unroll 1
    for (int c0 = 0; c0 < HID; c0 += 16) {
      float v[16];
      tc::tmem_ld16(lane + c0, v);
      float av[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        v[i] += __ldg(bias + c0 + i);
        av[i] = v[i];
      }
#pragma unroll
      for (int i = 0; i < 16; i += 2) gelu2(av[i], av[i + 1]);  // same GELU as the environment step
      if (p.z && valid) {
        float* zr = p.z + ((long long)l * p.B + b) * HID + c0;
        uint16_t* ar = p.a + ((long long)l * p.B + b) * HID + c0;
#pragma unroll
        for (int i = 0; i < 16; i += 4) *reinterpret_cast<float4*>(zr + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
#pragma unroll
        for (int i = 0; i < 16; i += 2)
          *reinterpret_cast<uint32_t*>(ar + i) = bf16x2_bits(av[i], av[i + 1]);
      }
      if (l < 2) {
        store8(sA, tid, c0, 128, av);
        store8(sA, tid, c0 + 8, 128, av + 8);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          o0 = fmaf(__ldg(mst + W4_OFF + c0 + i), av[i], o0);
          o1 = fmaf(__ldg(mst + W4_OFF + HID + c0 + i), av[i], o1);
        }
      }
    }
    if (l < 2) {
      const size_t base = l == 0 ? IMG_W2_OFF : IMG_W3_OFF;
      for (int h = 0; h < 2; ++h) {
        copy_img(sB, p.net.img + base + (size_t)h * 128 * HID * 2, (size_t)128 * HID * 2);
        ok &= tc::mma_group(tmem + 128 * h, &aA, 1, aB, 128, HID, false, &mbar, phase);
      }
    }
  }
  o0 += __ldg(mst + B4_OFF);
  o1 += __ldg(mst + B4_OFF + 1);
  if (valid && ok) {
    p.out[b * OUT] = o0;
    p.out[b * OUT + 1] = o1;
  }
  if (!ok && tid == 0) raise_status(p.status, 2);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// ---------------------------------------------------------------------------
// Estimator step in the environment (learned form): one CTA of 512 threads
// per 128 filters, thread = filter row x one of 4 column parts.  Part 0
// builds the row's features; the hidden-layer epilogues (bias, erf-GELU of
// gelu.cuh in packed pairs, BF16 operand) split
// the 256 hidden units 4 ways; the weight images (N-halves
// of W1, W2, W3) stream through two shared-memory slots by the bulk-copy
// engine, so the next layer's weights arrive during the current epilogue.
// ---------------------------------------------------------------------------
constexpr int kTE = 512;
constexpr int kParts = kTE / 128;
constexpr int kEnvStages = 6;                               // W1, W2, W3, two N-halves each
constexpr size_t kEnvSlot = (size_t)128 * HID * 2;          // largest half image (64 KB)
constexpr size_t kEnvSmem = 65536 + 2 * kEnvSlot;           // A operand + two weight slots
constexpr uint32_t kEnvPolls = 1u << 22;

__device__ __forceinline__ void env_stage(int s, size_t& off, uint32_t& bytes) {
  if (s < 2) {
    off = IMG_W1_OFF + (size_t)s * 128 * IN * 2;
    bytes = (uint32_t)(128 * IN * 2);
  } else {
    const int l = (s - 2) >> 1, h = (s - 2) & 1;
    off = (l == 0 ? IMG_W2_OFF : IMG_W3_OFF) + (size_t)h * 128 * HID * 2;
    bytes = (uint32_t)(128 * HID * 2);
  }
}

// test_wait_polls > 0 (test hook, env_test_wait_timeout): first a bounded
// wait on a barrier that nothing signals, then the timed-out exit (status 2)
// before any copy or MMA is issued.
__global__ void __launch_bounds__(kTE, 1) fwd_env_kernel(Net net, EnvDev d, int stale, uint32_t test_wait_polls) {
  pdl_wait();  // (dependents launch as this grid's CTAs exit)
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;           // features hi | lo [2 x 128 x 96], then hidden activations [128 x 256]
  unsigned char* sW = smem + 65536;   // two weight slots
  __shared__ __align__(8) uint64_t full[2];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ __align__(8) uint64_t never;  // test hook: a barrier nothing signals
  __shared__ uint32_t tbase;
  __shared__ float sOut[kParts][2][128];
  __shared__ int bad;
  const int tid = threadIdx.x, warp = tid >> 5, row = tid & 127, part = tid >> 7;
  const long long f = (long long)blockIdx.x * 128 + row;
  const bool valid = f < d.F;

  if (warp == 0) {
    tc::tmem_alloc(&tbase, 256);
    tc::tmem_relinquish();
  }
  if (tid == 32) {
    tc::mbar_init(&full[0], 1);
    tc::mbar_init(&full[1], 1);
    tc::mbar_init(&mbar, 1);
    tc::mbar_init(&never, 1);
    bad = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  if (test_wait_polls) {
    if (tid == 32 && !tc::mbar_wait(&never, 0u, test_wait_polls)) bad = 1;
    __syncthreads();
    if (bad) {
      if (tid == 0) raise_status(d.status, 2);
      if (warp == 0) tc::tmem_dealloc(tmem, 256);
      return;
    }
  }
  const uint32_t tl = tmem + ((uint32_t)(warp & 3) << 21);  // this warp's lane quarter
  const uint32_t aA = tc::smem_addr(sA), aW = tc::smem_addr(sW);
  auto fetch = [&](int st) {  // thread 0: stage st into slot st % 2
    size_t off;
    uint32_t bytes;
    env_stage(st, off, bytes);
    tc::mbar_expect_tx(&full[st & 1], bytes);
    tc::bulk_g2s(sW + (st & 1) * kEnvSlot, net.img + off, bytes, &full[st & 1]);
  };
  if (tid == 0) {
    fetch(0);
    fetch(1);
  }

  // features of this row (part 0) -> A operand as BF16 high and low parts
  float x[IN];
  float e1x = 0.0f, e1y = 0.0f, vnx = 0.0f, vny = 0.0f;
  if (part == 0) {
    if (valid) {
      e1x = d.estx[f];
      e1y = d.esty[f];
      const float e2x = d.prev_estx[f], e2y = d.prev_esty[f];
      vnx = fmaf(kVelKeep, d.velx[f], (1.0f - kVelKeep) * (e1x - e2x));
      vny = fmaf(kVelKeep, d.vely[f], (1.0f - kVelKeep) * (e1y - e2y));
      ring_features(d, (int)f, d.counters[0] + 1u, e1x, e1y, e2x, e2y, vnx, vny, x);
    } else {
#pragma unroll
      for (int i = 0; i < IN; ++i) x[i] = 0.0f;
    }
#pragma unroll
    for (int c0 = 0; c0 < IN; c0 += 8) {
      float hi[8], lo[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        hi[i] = bf_bits2f(f2bf_bits(x[c0 + i]));
        lo[i] = x[c0 + i] - hi[i];
      }
      store8(sA, row, c0, 128, hi);
      store8(sA + 128 * IN * 2, row, c0, 128, lo);
    }
  }

  bool ok = true;
  uint32_t mphase = 0;
  int stage = 0;
  const float* mst = net.master;
  float o0 = 0.0f, o1 = 0.0f;
  for (int l = 0; l < 3; ++l) {
    // MMA group of layer l: both N-halves (and, for layer 1, both feature parts)
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const int K = l == 0 ? IN : HID;
      const uint32_t idesc = tc::idesc_bf16(128, 128);
      for (int h = 0; h < 2; ++h) {
        ok &= tc::mbar_wait(&full[(stage + h) & 1], (uint32_t)(((stage + h) >> 1) & 1), kEnvPolls);
        const uint32_t bB = aW + (uint32_t)(((stage + h) & 1) * kEnvSlot);
        const int nA = l == 0 ? 2 : 1;
        bool acc = false;
        for (int j = 0; j < nA; ++j) {
          const uint32_t a0 = aA + (uint32_t)(j * 128 * IN * 2);
          for (int k = 0; k < K / 16; ++k) {
            const uint64_t ad = tc::smem_desc(a0 + k * 2 * 128 * 16, 128 * 16, 128);
            const uint64_t bd = tc::smem_desc(bB + k * 2 * 128 * 16, 128 * 16, 128);
            tc::mma_bf16(tmem + 128 * h, ad, bd, idesc, acc ? 1u : 0u);
            acc = true;
          }
        }
      }
      tc::mma_commit(&mbar);
    }
    ok &= tc::mbar_wait(&mbar, mphase, kEnvPolls);
    mphase ^= 1u;
    tc::fence_after_sync();
    stage += 2;
    if (tid == 0 && stage < kEnvStages) {  // both slots are free again: next layer's weights
      fetch(stage);
      fetch(stage + 1);
    }
    // epilogue of hidden layer l on this thread's 64 hidden units
    const float* bias = mst + (l == 0 ? B1_OFF : (l == 1 ? B2_OFF : B3_OFF));
#pragma unroll 1
    for (int c0 = part * (HID / kParts); c0 < (part + 1) * (HID / kParts); c0 += 16) {
      float v[16];
      tc::tmem_ld16(tl + c0, v);
      float av[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) av[i] = v[i] + __ldg(bias + c0 + i);
#pragma unroll
      for (int i = 0; i < 16; i += 2) gelu2(av[i], av[i + 1]);  // erf-GELU, packed pairs
      if (l < 2) {
        store8(sA, row, c0, 128, av);
        store8(sA, row, c0 + 8, 128, av + 8);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          o0 = fmaf(__ldg(mst + W4_OFF + c0 + i), av[i], o0);
          o1 = fmaf(__ldg(mst + W4_OFF + HID + c0 + i), av[i], o1);
        }
      }
    }
  }
  sOut[part][0][row] = o0;
  sOut[part][1][row] = o1;
  if (!ok) atomicExch(&bad, 1);
  __syncthreads();
  if (part == 0 && valid && bad == 0) {
    o0 = __ldg(mst + B4_OFF);
    o1 = __ldg(mst + B4_OFF + 1);
#pragma unroll
    for (int k = 0; k < kParts; ++k) {
      o0 += sOut[k][0][row];
      o1 += sOut[k][1][row];
    }
    const int it0 = d.filt_target[f];
    const int it = UT_IN_BOUNDS(it0 >= 0 && it0 < d.NT, d.status) ? it0 : 0;
    // Bounded update (dropped if not finite): with a ping received this step
    // the estimate may move up to kMaxCorr L.  Without one, the rule chosen
    // by the mode applies: hold the estimate (stale inputs cannot drive the
    // closed loop away), apply the network all the same, or coast by the
    // estimate's smoothed motion v (constant velocity).
    const bool fresh = x[3] == 0.0f && x[4] == 1.0f;
    const float lim = (fresh || stale == 1) ? kMaxCorr : 0.0f;
    float c0 = isfinite(o0) ? fminf(fmaxf(o0, -lim), lim) : 0.0f;
    float c1 = isfinite(o1) ? fminf(fmaxf(o1, -lim), lim) : 0.0f;
    if (!fresh && stale == 2) {
      c0 = fminf(fmaxf(x[5 * kRing + 2], -kMaxCorr), kMaxCorr);
      c1 = fminf(fmaxf(x[5 * kRing + 3], -kMaxCorr), kMaxCorr);
    }
    const float ex = e1x + d.est_scale * c0, ey = e1y + d.est_scale * c1;
    d.prev2_estx[f] = d.prev_estx[f];
    d.prev2_esty[f] = d.prev_esty[f];
    d.prev_estx[f] = e1x;
    d.prev_esty[f] = e1y;
    d.velx[f] = vnx;
    d.vely[f] = vny;
    d.estx[f] = ex;
    d.esty[f] = ey;
    const float dx = ex - d.tx[it], dy = ey - d.ty[it];
    d.err[f] = sqrtf(dx * dx + dy * dy);
  }
  if (bad && tid == 0) {
    // no copy may still be landing in shared memory when the CTA exits
    for (int st = kEnvStages - 2; st < kEnvStages; ++st)
      tc::mbar_wait(&full[st & 1], (uint32_t)((st >> 1) & 1), kEnvPolls);
    raise_status(d.status, 2);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// ---------------------------------------------------------------------------
// Input-gradient pass: dz3, dz2, dz1 (BF16, for the weight gradients), bias
// gradients and the output layer's gradients; loss.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kT, 1) bwd_kernel(Net net, TrainBufs t, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;
  unsigned char* sB = smem + 65536;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  // per-warp sums, each entry written once by lane 0 of its warp and summed
  // over the warps in order after the last barrier: dW4, db3, db2, db1, db4
  __shared__ float s_red[kT / 32][NB_PART];
  __shared__ double s_loss[kT / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lanei = tid & 31;
  const long long b = (long long)blockIdx.x * kT + tid;
  const bool valid = b < t.B;
  const long long row = valid ? (t.rows ? (long long)t.rows[b] : b) : 0;
  const float* mst = net.master;

  if (warp == 0) {
    tc::tmem_alloc(&tbase, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t aA = tc::smem_addr(sA), aB = tc::smem_addr(sB);
  uint32_t phase = 0;
  bool ok = true;
  float* s_dW4 = s_red[warp];
  float* s_db3 = s_dW4 + 2 * HID;
  float* s_db2 = s_db3 + HID;
  float* s_db1 = s_db2 + HID;
  float* s_db4 = s_db1 + HID;

  // output layer: dL/dout = (out - y) / B
  // loss per row: sum over the two outputs of e^2 / 2 (Huber with delta > 0:
  // quadratic inside |e| <= delta, linear outside); gradient / B
  float d0 = 0.0f, d1 = 0.0f;
  double se = 0.0;
  if (valid) {
    const float e[2] = {t.out[b * OUT] - t.Y[row * OUT], t.out[b * OUT + 1] - t.Y[row * OUT + 1]};
    float g[2];
    for (int c = 0; c < 2; ++c) {
      const float ae = fabsf(e[c]);
      if (t.huber > 0.0f && ae > t.huber) {
        g[c] = copysignf(t.huber, e[c]);
        se += (double)t.huber * ((double)ae - 0.5 * t.huber);
      } else {
        g[c] = e[c];
        se += 0.5 * (double)e[c] * e[c];
      }
    }
    d0 = g[0] / (float)t.B;
    d1 = g[1] / (float)t.B;
  }
  se = warp_sum_d(se);
  if (lanei == 0) s_loss[warp] = se;
  {
    const float r0 = warp_sum(d0), r1 = warp_sum(d1);
    if (lanei == 0) {
      s_db4[0] = r0;
      s_db4[1] = r1;
    }
  }
  // dz3 = (W4^T dout) * GELU'(z3); dW4 += dout a3^T
#pragma unroll 1
  for (int c0 = 0; c0 < HID; c0 += 16) {
    float dz[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int k = c0 + i;
      const float z = valid ? t.z[((long long)2 * t.B + b) * HID + k] : 0.0f;
      const float a = valid ? gelu1(z) : 0.0f;  // the forward's GELU
      const float w0 = warp_sum(d0 * a), w1 = warp_sum(d1 * a);
      if (lanei == 0) {
        s_dW4[k] = w0;
        s_dW4[HID + k] = w1;
      }
      const float da = d0 * __ldg(mst + W4_OFF + k) + d1 * __ldg(mst + W4_OFF + HID + k);
      dz[i] = valid ? da * gelu_grad(z) : 0.0f;
      const float sdz = warp_sum(dz[i]);
      if (lanei == 0) s_db3[k] = sdz;
    }
    if (valid) {
      uint16_t* dr = t.dz + ((long long)2 * t.B + b) * HID + c0;
#pragma unroll
      for (int i = 0; i < 16; i += 2)
        *reinterpret_cast<uint32_t*>(dr + i) = bf16x2_bits(dz[i], dz[i + 1]);
    }
    store8(sA, tid, c0, 128, dz);
    store8(sA, tid, c0 + 8, 128, dz + 8);
  }
  // dz2, dz1 through the transposed weights on the tensor cores
  for (int l = 1; l >= 0; --l) {
    const size_t base = l == 1 ? IMG_W3T_OFF : IMG_W2T_OFF;
    for (int h = 0; h < 2; ++h) {
      copy_img(sB, net.img + base + (size_t)h * 128 * HID * 2, (size_t)128 * HID * 2);
      ok &= tc::mma_group(tmem + 128 * h, &aA, 1, aB, 128, HID, false, &mbar, phase);
    }
    float* s_db = l == 1 ? s_db2 : s_db1;
#pragma unroll 1
    for (int c0 = 0; c0 < HID; c0 += 16) {
      float v[16];
      tc::tmem_ld16(lane + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float z = valid ? t.z[((long long)l * t.B + b) * HID + c0 + i] : 0.0f;
        v[i] = valid ? v[i] * gelu_grad(z) : 0.0f;
        const float s = warp_sum(v[i]);
        if (lanei == 0) s_db[c0 + i] = s;
      }
      if (valid) {
        uint16_t* dr = t.dz + ((long long)l * t.B + b) * HID + c0;
#pragma unroll
        for (int i = 0; i < 16; i += 2)
          *reinterpret_cast<uint32_t*>(dr + i) = bf16x2_bits(v[i], v[i + 1]);
      }
      if (l == 1) {
        store8(sA, tid, c0, 128, v);
        store8(sA, tid, c0 + 8, 128, v + 8);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  // the CTA's partial sums: the four warps' values added in warp order
  float* pb = t.part_b + (long long)blockIdx.x * NB_PART;
  for (int i = tid; i < NB_PART; i += kT) {
    float acc = s_red[0][i];
#pragma unroll
    for (int w = 1; w < kT / 32; ++w) acc += s_red[w][i];
    pb[i] = acc;
  }
  if (tid == 0) {
    double acc = s_loss[0];
#pragma unroll
    for (int w = 1; w < kT / 32; ++w) acc += s_loss[w];
    t.part_loss[blockIdx.x] = acc;
  }
  if (!ok && tid == 0) raise_status(status, 2);
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// grad[dst(i)] = sum over p of part[p][i], i < len: block x sums entries
// 32x .. 32x+31, thread row g the parts p = g (mod 32) in increasing p, then
// the 32 row sums in order of g (a fixed association: deterministic).  dst
// maps a slab position to its canonical parameter offset: `which` 0 for the
// bias / output-layer slab, 1 for the hidden weight slab.
__device__ __forceinline__ long long part_dst(int which, long long i) {
  if (which == 0) {
    if (i < 2 * HID) return W4_OFF + i;
    if (i < 3 * HID) return B3_OFF + (i - 2 * HID);
    if (i < 4 * HID) return B2_OFF + (i - 3 * HID);
    if (i < 5 * HID) return B1_OFF + (i - 4 * HID);
    return B4_OFF + (i - 5 * HID);
  }
  if (i < (long long)HID * IN) return W1_OFF + i;
  if (i < (long long)HID * IN + (long long)HID * HID) return W2_OFF + (i - (long long)HID * IN);
  return W3_OFF + (i - (long long)HID * IN - (long long)HID * HID);
}

__global__ void __launch_bounds__(1024) part_reduce_kernel(const float* __restrict__ part, int nparts, long long len,
                                                           int which, float* __restrict__ grad) {
  __shared__ float red[32][33];
  const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
  const long long i = (long long)blockIdx.x * 32 + c;
  float s = 0.0f;
  if (i < len)
    for (int p = g; p < nparts; p += 32) s += part[(long long)p * len + i];
  red[g][c] = s;
  __syncthreads();
  if (g == 0 && i < len) {
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < 32; ++k) acc += red[k][c];
    grad[part_dst(which, i)] = acc;
  }
}

// Batch loss = (sum of the CTA partials, in order of p mod 256, then the 256
// sums in order) / B.
__global__ void __launch_bounds__(256) loss_reduce_kernel(const double* __restrict__ part, int nparts, int B,
                                                          double* __restrict__ loss) {
  __shared__ double red[256];
  double s = 0.0;
  for (int p = threadIdx.x; p < nparts; p += 256) s += part[p];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int k = 0; k < 256; ++k) acc += red[k];
    *loss = acc / B;
  }
}

// ---------------------------------------------------------------------------
// Weight gradients dW_l = dz_l^T a_{l-1} summed over the batch, on the tensor
// cores: M = 128 output features (one half), N = input features, K = 128
// batch rows per MMA group, accumulated in TMEM over the CTA's batch range
// and written to the split's partial slab (summed over the splits in a fixed
// order by part_reduce_kernel).  The transposed operands are written
// element-wise into K-major images.  grid = (batch splits, output half, layer).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kT, 2) wgrad_kernel(TrainBufs t, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;          // dz^T [128 x 128]
  unsigned char* sB = smem + 32768;  // a^T [N_in x 128]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int layer = blockIdx.z, half = blockIdx.y;
  const int n_in = layer == 0 ? IN : HID;
  const int n_chunks = (t.B + kT - 1) / kT;
  const int per = (n_chunks + gridDim.x - 1) / gridDim.x;
  const int c_begin = blockIdx.x * per, c_end = min(n_chunks, c_begin + per);

  if (warp == 0) {
    tc::tmem_alloc(&tbase, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const uint32_t aA = tc::smem_addr(sA), aB = tc::smem_addr(sB);
  uint32_t phase = 0;
  bool ok = true;
  uint16_t* sAh = reinterpret_cast<uint16_t*>(sA);
  uint16_t* sBh = reinterpret_cast<uint16_t*>(sB);
  for (int c = c_begin; c < c_end; ++c) {
    const long long b = (long long)c * kT + tid;
    const bool valid = b < t.B;
    // dz^T: element (o, b) of the [128 x 128] operand
    const uint16_t* dzr = t.dz + ((long long)layer * t.B + b) * HID + half * 128;
#pragma unroll 4
    for (int o = 0; o < 128; o += 8) {
      uint4 v = valid ? *reinterpret_cast<const uint4*>(dzr + o) : make_uint4(0, 0, 0, 0);
      const uint16_t* e = reinterpret_cast<const uint16_t*>(&v);
#pragma unroll
      for (int i = 0; i < 8; ++i) sAh[tc::kmajor_offset(o + i, tid, 128) / 2] = e[i];
    }
    // a^T: element (i, b) of the [n_in x 128] operand (layer 0: the features)
    if (layer == 0) {
      const long long row = valid ? (t.rows ? (long long)t.rows[b] : b) : 0;
      for (int i = 0; i < IN; ++i)
        sBh[tc::kmajor_offset(i, tid, IN) / 2] = valid ? f2bf_bits(t.X[row * IN + i]) : (uint16_t)0;
    } else {
      const uint16_t* ar = t.a + ((long long)(layer - 1) * t.B + b) * HID;
#pragma unroll 4
      for (int i = 0; i < HID; i += 8) {
        uint4 v = valid ? *reinterpret_cast<const uint4*>(ar + i) : make_uint4(0, 0, 0, 0);
        const uint16_t* e = reinterpret_cast<const uint16_t*>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) sBh[tc::kmajor_offset(i + j, tid, HID) / 2] = e[j];
      }
    }
    ok &= tc::mma_group(tmem, &aA, 1, aB, n_in, kT, c > c_begin, &mbar, phase);
  }
  if (c_end <= c_begin) {  // per = ceil(chunks / splits) can leave the last splits without rows: zero slab
    const int o = warp * 32 + (tid & 31);
    const long long w_off = layer == 0 ? 0 : (long long)HID * IN + (long long)(layer - 1) * HID * HID;
    float* pw = t.part_w + (long long)blockIdx.x * NW_PART + w_off;
    for (int c = 0; c < n_in; ++c) pw[(long long)(half * 128 + o) * n_in + c] = 0.0f;
  }
  if (c_end > c_begin && ok) {
    const int o = warp * 32 + (tid & 31);
    // this split's slab: dW1 [256][96], then dW2 and dW3 [256][256]
    const long long w_off = layer == 0 ? 0 : (long long)HID * IN + (long long)(layer - 1) * HID * HID;
    float* pw = t.part_w + (long long)blockIdx.x * NW_PART + w_off;
    const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < n_in; c0 += 16) {
      float v[16];
      tc::tmem_ld16(lane + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) pw[(long long)(half * 128 + o) * n_in + c0 + i] = v[i];
    }
  }
  if (!ok && tid == 0) raise_status(status, 2);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// Image position of weight element (layer, out, in) in the forward operand
// (chunks of 128 output rows) and, for layers 2 and 3, in the transposed one.
__device__ __forceinline__ void write_images(unsigned char* img, long long i, float w) {
  const uint16_t bits = f2bf_bits(w);
  if (i >= W1_OFF && i < B1_OFF) {
    const int o = (int)((i - W1_OFF) / IN), in = (int)((i - W1_OFF) % IN);
    *reinterpret_cast<uint16_t*>(img + IMG_W1_OFF + (size_t)(o / 128) * 128 * IN * 2 +
                                 tc::kmajor_offset(o % 128, in, 128)) = bits;
  } else if ((i >= W2_OFF && i < B2_OFF) || (i >= W3_OFF && i < B3_OFF)) {
    const bool l2 = i < B2_OFF;
    const long long r = i - (l2 ? W2_OFF : W3_OFF);
    const int o = (int)(r / HID), in = (int)(r % HID);
    const size_t fw = l2 ? IMG_W2_OFF : IMG_W3_OFF, bw = l2 ? IMG_W2T_OFF : IMG_W3T_OFF;
    *reinterpret_cast<uint16_t*>(img + fw + (size_t)(o / 128) * 128 * HID * 2 + tc::kmajor_offset(o % 128, in, 128)) =
        bits;
    *reinterpret_cast<uint16_t*>(img + bw + (size_t)(in / 128) * 128 * HID * 2 + tc::kmajor_offset(in % 128, o, 128)) =
        bits;
  }
}

__global__ void adam_kernel(float* master, float* m, float* v, const float* grad, float lr, float beta1, float beta2,
                            float eps, float c1, float c2, unsigned char* img) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float g = grad[i];
  const float mi = beta1 * m[i] + (1.0f - beta1) * g;
  const float vi = beta2 * v[i] + (1.0f - beta2) * g * g;
  const float th = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  m[i] = mi;
  v[i] = vi;
  master[i] = th;
  write_images(img, i, th);
}

__global__ void pack_kernel(const float* master, unsigned char* img) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NPARAM) write_images(img, i, master[i]);
}

__global__ void batch_rows_kernel(int32_t* rows, int B, uint32_t n_rows, uint64_t seed, uint32_t step) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  Rand4 r = philox((uint32_t)b, step, 0u, TAG_BATCH, seed);
  rows[b] = (int32_t)__umulhi(r.x[0], n_rows);
}

__global__ void record_kernel(EnvDev d, float* feat, float* label) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= d.F) return;
  // after the step: the update's inputs are the estimate history
  const float e1x = d.prev_estx[f], e1y = d.prev_esty[f];
  float x[IN];
  ring_features(d, f, d.counters[0], e1x, e1y, d.prev2_estx[f], d.prev2_esty[f], d.velx[f], d.vely[f], x);
#pragma unroll
  for (int i = 0; i < IN; i += 4)
    *reinterpret_cast<float4*>(feat + (long long)f * IN + i) = make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]);
  const int it = d.filt_target[f];
  label[(long long)f * 2] = (d.tx[it] - e1x) / d.est_scale;
  label[(long long)f * 2 + 1] = (d.ty[it] - e1y) / d.est_scale;
}

}  // namespace

cudaError_t launch_forward(const Net& net, const float* X, const int32_t* rows, int B, float* out, float* z,
                           uint16_t* a, cudaStream_t s) {
  static std::atomic<unsigned long long> ready{0};
  cudaError_t e = smem_optin(fwd_kernel, kFwdSmem, ready);
  if (e != cudaSuccess) return e;
  if (B <= 0) return cudaSuccess;
  FwdArgs p;
  memset(&p, 0, sizeof(p));
  p.net = net;
  p.X = X;
  p.rows = rows;
  p.B = B;
  p.out = out;
  p.z = z;
  p.a = a;
  fwd_kernel<<<(B + kT - 1) / kT, kT, kFwdSmem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_forward_env(const Net& net, const EnvDev& d, int stale, uint32_t test_wait_polls,
                               cudaStream_t s) {
  static std::atomic<unsigned long long> ready{0};
  cudaError_t e = smem_optin(fwd_env_kernel, kEnvSmem, ready);
  if (e != cudaSuccess) return e;
  if (d.F <= 0) return cudaSuccess;
  launch_pdl(fwd_env_kernel, dim3((d.F + 127) / 128), dim3(kTE), kEnvSmem, s, net, d, stale, test_wait_polls);
  return cudaGetLastError();
}

cudaError_t launch_record(const EnvDev& d, float* feat, float* label, cudaStream_t s) {
  if (d.F <= 0) return cudaSuccess;
  record_kernel<<<(d.F + 127) / 128, 128, 0, s>>>(d, feat, label);
  return cudaGetLastError();
}

cudaError_t launch_backward(const Net& net, const TrainBufs& t, cudaStream_t s) {
  static std::atomic<unsigned long long> ready_b{0}, ready_w{0};
  cudaError_t e = smem_optin(bwd_kernel, kFwdSmem, ready_b);
  if (e == cudaSuccess) e = smem_optin(wgrad_kernel, kWgradSmem, ready_w);
  if (e != cudaSuccess) return e;
  if (t.B <= 0) return cudaSuccess;
  const int n_chunks = (t.B + kT - 1) / kT;
  bwd_kernel<<<n_chunks, kT, kFwdSmem, s>>>(net, t, nullptr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int splits = n_chunks < kWgradSplits ? n_chunks : kWgradSplits;
  wgrad_kernel<<<dim3(splits, 2, 3), kT, kWgradSmem, s>>>(t, nullptr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // fixed-order sums of the partial slabs into the gradient and the loss
  part_reduce_kernel<<<(NB_PART + 31) / 32, 1024, 0, s>>>(t.part_b, n_chunks, NB_PART, 0, t.grad);
  part_reduce_kernel<<<(unsigned)((NW_PART + 31) / 32), 1024, 0, s>>>(t.part_w, splits, NW_PART, 1, t.grad);
  loss_reduce_kernel<<<1, 256, 0, s>>>(t.part_loss, n_chunks, t.B, t.loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* master, float* m, float* v, const float* grad, int step, float lr, float beta1,
                        float beta2, float eps, unsigned char* img, cudaStream_t s) {
  const double c1 = 1.0 - std::pow((double)beta1, step), c2 = 1.0 - std::pow((double)beta2, step);
  adam_kernel<<<(unsigned)((NPARAM + 255) / 256), 256, 0, s>>>(master, m, v, grad, lr, beta1, beta2, eps, (float)c1,
                                                              (float)c2, img);
  return cudaGetLastError();
}

cudaError_t launch_pack(const float* master, unsigned char* img, cudaStream_t s) {
  pack_kernel<<<(unsigned)((NPARAM + 255) / 256), 256, 0, s>>>(master, img);
  return cudaGetLastError();
}

cudaError_t launch_batch_rows(int32_t* rows, int B, int64_t n_rows, uint64_t seed, uint32_t step, cudaStream_t s) {
  batch_rows_kernel<<<(B + 255) / 256, 256, 0, s>>>(rows, B, (uint32_t)n_rows, seed, step);
  return cudaGetLastError();
}

}  // namespace est
}  // namespace ut
