// Transformer agent forward (Sec. III-B.1, Fig. 3) on the tensor cores.
//
// Each agent's tokens are its recurrent embedding h followed by its entity
// vectors (self, teammates, targets; observation tokens of Sec. III-A.2).
// Agents are packed R = 1 + max entities rows apart into 128-row tiles; one
// CTA of 128 threads owns a tile and thread r owns row r from start to end:
//
//   X = [h ; W_emb tok + b_emb]                         (CUDA cores, FP32)
//   per block l:   Y = LN1(X) -> BF16 operand A
//                  Q, K, V = Y Wq^T, Y Wk^T, Y Wv^T      (tcgen05.mma, TMEM)
//                  O = softmax(Q K^T / 4) V per head, within the agent's
//                      valid tokens                      (CUDA cores)
//                  X += O Wo^T + bo                      (tcgen05.mma)
//                  X += W2 GELU(W1 LN2(X) + b1) + b2      (tcgen05.mma, hidden
//                      units in chunks of 128 accumulated in TMEM)
//   logits = Wh LN_f(X[recurrent row]) + bh; next h = X[recurrent row];
//   action = argmax(logits + Gumbel noise)              (Actions Space: the
//                                                        agent's categorical
//                                                        policy, sampled)
// Readings (C16): pre-LN blocks, FFN width 4d with exact erf-GELU, LN eps
// 1e-5, head dimension 16.  Matrix operands are BF16, every accumulation is
// FP32.  Weights are packed once into the tensor cores' K-major operand
// layout (tc.cuh) so that each operand tile is one contiguous copy.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/utrack.h"
#include "policy.cuh"
#include "runtime.cuh"
#include "tc.cuh"

namespace ut {
namespace {

constexpr int kThreads = 128;
constexpr float kLnEps = 1e-5f;

template <int D>
struct Geo {
  static constexpr int H = D / 16;                 // heads of width 16
  static constexpr int XS = D + 1;                 // fp32 row stride of X (bank-conflict free)
  static constexpr int KVS = D + 8;                // bf16 row stride of K / V
  static constexpr int NC = (4 * D) / 128;         // FFN hidden chunks of 128
  static constexpr size_t X_BYTES = (size_t)128 * XS * 4;
  static constexpr size_t A_BYTES = (size_t)128 * D * 2;
  static constexpr size_t B_BYTES = (size_t)128 * D * 2;
  static constexpr size_t KV_BYTES = (size_t)2 * 128 * KVS * 2;
  static constexpr size_t X_OFF = 0;
  static constexpr size_t A_OFF = (X_OFF + X_BYTES + 127) & ~(size_t)127;
  static constexpr size_t B_OFF = A_OFF + A_BYTES;
  static constexpr size_t KV_OFF = B_OFF + B_BYTES;
  static constexpr size_t SMEM = KV_OFF + KV_BYTES;
  static constexpr uint32_t TMEM_COLS = D == 64 ? 256 : 512;
  static constexpr uint32_t COL_Q = 0;             // Q, later the FFN output accumulator
  static constexpr uint32_t COL_S = TMEM_COLS / 2; // scratch accumulator (<= 128 columns)
  // packed weight images of one layer (bytes)
  static constexpr size_t IMG_DD = (size_t)D * D * 2;
  static constexpr size_t IMG_W1 = (size_t)128 * D * 2;
  static constexpr size_t IMG_W2 = (size_t)D * 128 * 2;
  static constexpr size_t OFF_Q = 0, OFF_K = IMG_DD, OFF_V = 2 * IMG_DD, OFF_O = 3 * IMG_DD;
  static constexpr size_t OFF_W1 = 4 * IMG_DD;
  static constexpr size_t OFF_W2 = OFF_W1 + NC * IMG_W1;
  static constexpr size_t LAYER_BYTES = OFF_W2 + NC * IMG_W2;
  static_assert(KV_BYTES >= (size_t)128 * 128 * 2, "hidden chunk must fit in the K/V region");
};

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// Copy a contiguous operand image global -> shared (16 B per thread-step).
__device__ __forceinline__ void copy_image(unsigned char* dst, const unsigned char* __restrict__ src, size_t bytes) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* t = reinterpret_cast<uint4*>(dst);
  for (size_t i = threadIdx.x; i < bytes / 16; i += kThreads) t[i] = __ldg(s + i);
}

// Store 8 consecutive K values of `row` into a K-major operand image.
__device__ __forceinline__ void store8(unsigned char* img, int row, int k0, int rows, const float* v) {
  uint4 p;
  p.x = (uint32_t)f2bf_bits(v[0]) | ((uint32_t)f2bf_bits(v[1]) << 16);
  p.y = (uint32_t)f2bf_bits(v[2]) | ((uint32_t)f2bf_bits(v[3]) << 16);
  p.z = (uint32_t)f2bf_bits(v[4]) | ((uint32_t)f2bf_bits(v[5]) << 16);
  p.w = (uint32_t)f2bf_bits(v[6]) | ((uint32_t)f2bf_bits(v[7]) << 16);
  *reinterpret_cast<uint4*>(img + tc::kmajor_offset(row, k0, rows)) = p;
}

// LayerNorm of this thread's X row into the A operand (BF16).
template <int D>
__device__ __forceinline__ void ln_to_a(const float* xr, const float* __restrict__ g, const float* __restrict__ b,
                                        unsigned char* sA, int row) {
  float mu = 0.0f;
#pragma unroll 16
  for (int c = 0; c < D; ++c) mu += xr[c];
  mu *= (1.0f / D);
  float var = 0.0f;
#pragma unroll 16
  for (int c = 0; c < D; ++c) {
    const float t = xr[c] - mu;
    var = fmaf(t, t, var);
  }
  const float inv = rsqrtf(var * (1.0f / D) + kLnEps);
#pragma unroll
  for (int c0 = 0; c0 < D; c0 += 8) {
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = fmaf((xr[c0 + i] - mu) * inv, __ldg(g + c0 + i), __ldg(b + c0 + i));
    store8(sA, row, c0, 128, v);
  }
}

// One MMA stage: acc[tmem_col .. +N) (+)= A[128 x K] * B[N x K]^T.
// Publishes the operands written by every thread, issues from thread 0,
// waits for completion.  Returns false if the bounded wait gave up.
__device__ __forceinline__ bool mma_stage(uint32_t tmem, uint32_t a_addr, uint32_t b_addr, int N, int K,
                                          bool accumulate, uint64_t* mbar, uint32_t& phase) {
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x == 0) {
    const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)N);
    for (int k = 0; k < K / 16; ++k) {
      const uint64_t ad = tc::smem_desc(a_addr + k * 2 * 128 * 16, 128 * 16, 128);
      const uint64_t bd = tc::smem_desc(b_addr + k * 2 * N * 16, N * 16, 128);
      tc::mma_bf16(tmem, ad, bd, idesc, (accumulate || k > 0) ? 1u : 0u);
    }
    tc::mma_commit(mbar);
  }
  const bool ok = tc::mbar_wait(mbar, phase, 1u << 22);
  phase ^= 1u;
  tc::fence_after_sync();
  return ok;
}

template <int D>
__global__ void __launch_bounds__(kThreads, 1) policy_fwd_kernel(PolicyDev p) {
  using G = Geo<D>;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* sX = reinterpret_cast<float*>(smem + G::X_OFF);
  unsigned char* sA = smem + G::A_OFF;
  unsigned char* sB = smem + G::B_OFF;
  unsigned char* sKV = smem + G::KV_OFF;
  uint16_t* sK = reinterpret_cast<uint16_t*>(sKV);
  uint16_t* sV = sK + 128 * G::KVS;
  unsigned char* sH = sKV;  // FFN hidden chunk image [128 x 128] (K/V are dead by then)
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int bad;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid;
  const int slot = row / p.R, tok = row - slot * p.R;
  const long long ag = (long long)blockIdx.x * p.apt + slot;
  const bool agent_ok = slot < p.apt && ag < p.NA;
  const int n_tok = agent_ok ? 1 + p.n_ent[ag] : 0;
  const bool row_ok = tok < n_tok;
  const int row0 = slot * p.R;  // first row of this agent

  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_s, G::TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    bad = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base_s;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t tQ = tmem + lane_base + G::COL_Q, tS = tmem + lane_base + G::COL_S;
  const uint32_t aA = tc::smem_addr(sA), aB = tc::smem_addr(sB), aH = tc::smem_addr(sH);
  uint32_t phase = 0;
  bool ok = true;  // all bounded waits succeeded

  // ---- token rows ----------------------------------------------------------
  float* xr = sX + row * G::XS;
  if (row_ok && tok == 0) {
    const uint16_t* hp = p.h + ag * D;
#pragma unroll 8
    for (int c = 0; c < D; ++c) xr[c] = bf_bits2f(hp[c]);
  } else if (row_ok) {
    const uint4 t4 = *reinterpret_cast<const uint4*>(p.tokens + (ag * p.NS + (tok - 1)) * 8);
    float t[8] = {bf_bits2f(t4.x & 0xFFFF), bf_bits2f(t4.x >> 16), bf_bits2f(t4.y & 0xFFFF), bf_bits2f(t4.y >> 16),
                  bf_bits2f(t4.z & 0xFFFF), bf_bits2f(t4.z >> 16), bf_bits2f(t4.w & 0xFFFF), bf_bits2f(t4.w >> 16)};
#pragma unroll 4
    for (int c = 0; c < D; ++c) {
      float acc = __ldg(p.emb_b + c);
#pragma unroll
      for (int f = 0; f < 8; ++f) acc = fmaf(__ldg(p.emb_w + c * 8 + f), t[f], acc);
      xr[c] = acc;
    }
  } else {
#pragma unroll 8
    for (int c = 0; c < D; ++c) xr[c] = 0.0f;
  }

  // Every thread runs every stage (the barriers stay uniform); a wait that
  // gave up only marks the result invalid.
  for (int l = 0; l < p.L; ++l) {
    const unsigned char* img = p.wimg + (size_t)l * G::LAYER_BYTES;
    const float* vec = p.vec + (size_t)l * 13 * D;
    const float *ln1g = vec, *ln1b = vec + D, *bq = vec + 2 * D, *bk = vec + 3 * D, *bv = vec + 4 * D;
    const float *bo = vec + 5 * D, *ln2g = vec + 6 * D, *ln2b = vec + 7 * D, *b1 = vec + 8 * D, *b2 = vec + 12 * D;

    // ---- attention sub-block ----
    ln_to_a<D>(xr, ln1g, ln1b, sA, row);
    copy_image(sB, img + G::OFF_Q, G::IMG_DD);
    ok &= mma_stage(tmem + G::COL_Q, aA, aB, D, D, false, &mbar, phase);
    // K and V through the scratch accumulator into shared memory
    for (int kv = 0; kv < 2; ++kv) {
      copy_image(sB, img + (kv == 0 ? G::OFF_K : G::OFF_V), G::IMG_DD);
      ok &= mma_stage(tmem + G::COL_S, aA, aB, D, D, false, &mbar, phase);
      const float* bias = kv == 0 ? bk : bv;
      uint16_t* dst = (kv == 0 ? sK : sV) + row * G::KVS;
#pragma unroll 1
      for (int c0 = 0; c0 < D; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tS + c0, v);
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const uint32_t pk = (uint32_t)f2bf_bits(v[i] + __ldg(bias + c0 + i)) |
                              ((uint32_t)f2bf_bits(v[i + 1] + __ldg(bias + c0 + i + 1)) << 16);
          *reinterpret_cast<uint32_t*>(dst + c0 + i) = pk;
        }
      }
    }
    __syncthreads();  // K, V of every row visible
    // per-head softmax attention over the agent's valid tokens
#pragma unroll 1
    for (int h = 0; h < G::H; ++h) {
      float q[16];
      tc::tmem_ld16(tQ + h * 16, q);
      float o[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        q[i] = (q[i] + __ldg(bq + h * 16 + i)) * 0.25f;  // 1 / sqrt(16)
        o[i] = 0.0f;
      }
      if (row_ok) {
        float m = -INFINITY, den = 0.0f;
        for (int j = 0; j < n_tok; ++j) {
          const uint16_t* kr = sK + (row0 + j) * G::KVS + h * 16;
          const uint16_t* vr = sV + (row0 + j) * G::KVS + h * 16;
          float s = 0.0f;
#pragma unroll
          for (int i = 0; i < 16; ++i) s = fmaf(q[i], bf_bits2f(kr[i]), s);
          const float mn = fmaxf(m, s);
          const float corr = __expf(m - mn), e = __expf(s - mn);
          den = den * corr + e;
#pragma unroll
          for (int i = 0; i < 16; ++i) o[i] = fmaf(e, bf_bits2f(vr[i]), o[i] * corr);
          m = mn;
        }
        const float inv = 1.0f / den;
#pragma unroll
        for (int i = 0; i < 16; ++i) o[i] *= inv;
      }
      store8(sA, row, h * 16, 128, o);
      store8(sA, row, h * 16 + 8, 128, o + 8);
    }
    copy_image(sB, img + G::OFF_O, G::IMG_DD);
    ok &= mma_stage(tmem + G::COL_S, aA, aB, D, D, false, &mbar, phase);
#pragma unroll 1
    for (int c0 = 0; c0 < D; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tS + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) xr[c0 + i] += v[i] + __ldg(bo + c0 + i);
    }

    // ---- feed-forward sub-block ----
    ln_to_a<D>(xr, ln2g, ln2b, sA, row);
#pragma unroll 1
    for (int c = 0; c < G::NC; ++c) {
      copy_image(sB, img + G::OFF_W1 + c * G::IMG_W1, G::IMG_W1);
      ok &= mma_stage(tmem + G::COL_S, aA, aB, 128, D, false, &mbar, phase);
#pragma unroll 1
      for (int c0 = 0; c0 < 128; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tS + c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = gelu(v[i] + __ldg(b1 + c * 128 + c0 + i));
        store8(sH, row, c0, 128, v);
        store8(sH, row, c0 + 8, 128, v + 8);
      }
      copy_image(sB, img + G::OFF_W2 + c * G::IMG_W2, G::IMG_W2);
      ok &= mma_stage(tmem + G::COL_Q, aH, aB, D, 128, c > 0, &mbar, phase);
    }
#pragma unroll 1
    for (int c0 = 0; c0 < D; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tQ + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) xr[c0 + i] += v[i] + __ldg(b2 + c0 + i);
    }
  }

  // ---- head on the recurrent token ----------------------------------------
  if (!ok && tid == 0) atomicExch(&bad, 1);
  if (agent_ok && tok == 0 && ok) {
    uint16_t* hp = p.h + ag * D;
    float mu = 0.0f, var = 0.0f;
    for (int c = 0; c < D; ++c) {
      hp[c] = f2bf_bits(xr[c]);
      mu += xr[c];
    }
    mu *= (1.0f / D);
    for (int c = 0; c < D; ++c) var = fmaf(xr[c] - mu, xr[c] - mu, var);
    const float inv = rsqrtf(var * (1.0f / D) + kLnEps);
    float best = -INFINITY;
    int arg = 0;
    const uint32_t g = p.counters ? p.counters[0] + 1u : p.step;
    for (int j = 0; j < p.n_act; ++j) {
      float acc = __ldg(p.head_b + j);
      for (int c = 0; c < D; ++c)
        acc = fmaf(__ldg(p.head_w + j * D + c), fmaf((xr[c] - mu) * inv, __ldg(p.lnf_g + c), __ldg(p.lnf_b + c)),
                   acc);
      p.logits[ag * p.n_act + j] = acc;
      if (p.sample) {
        Rand4 r = philox((uint32_t)ag, (uint32_t)(j >> 2), g, TAG_GUMBEL, p.seed);
        const float gum = -logf(-logf(unif_mid(r.x[j & 3])));
        if (acc + gum > best) {
          best = acc + gum;
          arg = j;
        }
      }
    }
    if (p.sample) p.actions[ag] = arg;
  }

  tc::fence_before_sync();
  __syncthreads();
  if (bad && tid == 0) raise_status(p.status, 2);
  if (warp == 0) tc::tmem_dealloc(tmem, G::TMEM_COLS);
}

template <int D>
cudaError_t launch_policy_t(const PolicyDev& p, cudaStream_t s) {
  static int ready = 0;
  if (!ready) {
    cudaError_t e = cudaFuncSetAttribute(policy_fwd_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Geo<D>::SMEM);
    if (e != cudaSuccess) return e;
    ready = 1;
  }
  const long long tiles = (p.NA + p.apt - 1) / p.apt;
  if (tiles > 0) policy_fwd_kernel<D><<<(unsigned)tiles, kThreads, Geo<D>::SMEM, s>>>(p);
  return cudaGetLastError();
}

// Host-side packing of one [N x K] block (rows of a row-major matrix with
// leading dimension ld, starting at (r0, c0)) into the K-major operand image.
void pack_image(std::vector<unsigned char>& out, size_t off, const float* m, int ld, int r0, int c0, int N, int K) {
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < K; ++k) {
      const float v = m[(size_t)(r0 + n) * ld + c0 + k];
      uint32_t bits;
      std::memcpy(&bits, &v, 4);
      const uint32_t rnd = ((bits >> 16) & 1u) + 0x7FFFu;  // round to nearest even
      const uint16_t b = (uint16_t)((bits + rnd) >> 16);
      std::memcpy(&out[off + tc::kmajor_offset((uint32_t)n, (uint32_t)k, (uint32_t)N)], &b, 2);
    }
}

}  // namespace

int64_t policy_param_count(int d, int L, int n_act) {
  const int64_t D = d;
  const int64_t per = 2 * D + 3 * D * D + 3 * D + D * D + D + 2 * D + 4 * D * D + 4 * D + 4 * D * D + D;
  return D * 8 + D + L * per + 2 * D + (int64_t)n_act * D + n_act;
}

bool policy_supported(int d, int n_heads) { return (d == 64 || d == 128) && n_heads * 16 == d; }

size_t policy_layer_bytes(int d) { return d == 64 ? Geo<64>::LAYER_BYTES : Geo<128>::LAYER_BYTES; }

// Splits the canonical parameter blob into packed images and FP32 vectors.
void policy_pack(int d, int L, int n_act, const float* prm, std::vector<unsigned char>& img, std::vector<float>& vec,
                 std::vector<float>& emb, std::vector<float>& head) {
  const int D = d;
  const size_t LB = policy_layer_bytes(d);
  const size_t dd = (size_t)D * D * 2, w1 = (size_t)128 * D * 2, w2 = (size_t)D * 128 * 2;
  const int NC = 4 * D / 128;
  img.assign(LB * L, 0);
  vec.assign((size_t)13 * D * L, 0.0f);
  const float* q = prm;
  emb.assign(q, q + D * 8 + D);  // W_emb [D][8], b_emb [D]
  q += D * 8 + D;
  for (int l = 0; l < L; ++l) {
    const size_t base = LB * l;
    float* v = vec.data() + (size_t)13 * D * l;
    const float* ln1g = q; q += D;
    const float* ln1b = q; q += D;
    const float* Wqkv = q; q += (size_t)3 * D * D;
    const float* bqkv = q; q += 3 * D;
    const float* Wo = q; q += (size_t)D * D;
    const float* bo = q; q += D;
    const float* ln2g = q; q += D;
    const float* ln2b = q; q += D;
    const float* W1 = q; q += (size_t)4 * D * D;
    const float* b1 = q; q += 4 * D;
    const float* W2 = q; q += (size_t)4 * D * D;
    const float* b2 = q; q += D;
    pack_image(img, base + 0, Wqkv, D, 0, 0, D, D);
    pack_image(img, base + dd, Wqkv, D, D, 0, D, D);
    pack_image(img, base + 2 * dd, Wqkv, D, 2 * D, 0, D, D);
    pack_image(img, base + 3 * dd, Wo, D, 0, 0, D, D);
    for (int c = 0; c < NC; ++c) pack_image(img, base + 4 * dd + c * w1, W1, D, c * 128, 0, 128, D);
    for (int c = 0; c < NC; ++c) pack_image(img, base + 4 * dd + NC * w1 + c * w2, W2, 4 * D, 0, c * 128, D, 128);
    std::memcpy(v, ln1g, D * 4);
    std::memcpy(v + D, ln1b, D * 4);
    std::memcpy(v + 2 * D, bqkv, 3 * D * 4);
    std::memcpy(v + 5 * D, bo, D * 4);
    std::memcpy(v + 6 * D, ln2g, D * 4);
    std::memcpy(v + 7 * D, ln2b, D * 4);
    std::memcpy(v + 8 * D, b1, 4 * D * 4);
    std::memcpy(v + 12 * D, b2, D * 4);
  }
  head.assign(q, q + 2 * D + (size_t)n_act * D + n_act);  // lnf_g, lnf_b, Wh, bh
}

cudaError_t launch_policy(const PolicyDev& p, int d, cudaStream_t s) {
  if (d == 64) return launch_policy_t<64>(p, s);
  if (d == 128) return launch_policy_t<128>(p, s);
  return cudaErrorInvalidValue;
}

}  // namespace ut
