// Transformer actor and critic in FP32 for the TransfMAPPO update (Sec. II-B,
// Sec. III-B.1, Fig. 3): the forward pass with stored activations, the PPO
// clipped-surrogate and value losses, the backward pass, Adam, and
// generalized advantage estimation.
//
// Layout: sample s of a call occupies token rows s*T .. s*T+T-1 (T = 1 +
// n_slots, row 0 its recurrent embedding); every activation is row-major
// [rows][width].  Rows past a sample's entity count are computed (from the
// embedding bias alone) but no row attends to them, so they receive exactly
// zero gradient and add nothing to the weight gradients.
//
// The dense contractions run on CUDA cores in FP32 (a 64 x 64 register-tiled
// GEMM); the weight gradients are split along the token rows into partial
// slabs summed in a fixed order, so every result is deterministic.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/utrack.h"
#include "common.cuh"
#include "tc.cuh"
#include "tfm.cuh"

namespace ut {
namespace tfm {

constexpr int kMaxT = 1 + UT_MAX_AGENTS + UT_MAX_TARGETS;  // tokens per sample
constexpr int kRowBlocks = 304;                             // blocks of the head / embedding-gradient kernels
constexpr int kLnBlocks = 1216;                             // blocks of the LayerNorm kernels
constexpr int kRowWarps = kRowBlocks * 8;                   // warps writing partial sums
constexpr int kTcSplitsMax = 3 * 152;                       // row splits of a tensor-core weight gradient (at most)

enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_RES = 2, EPI_BIAS_GELU = 3, EPI_GELU_GRAD = 4, EPI_PARTIAL = 5 };

// C = op(A) op(B) with an epilogue.  A(m, k) is A[m * lda + k] when AK (k
// contiguous), else A[k * lda + m]; B(k, n) is B[n * ldb + k] when BK, else
// B[k * ldb + n].  blockIdx.z takes K range [z * kchunk, (z + 1) * kchunk).
struct Gemm {
  const float* A;
  long long lda;
  const float* B;
  long long ldb;
  float* C;
  long long ldc;
  long long M, K, kchunk;
  int N, epi;
  const float* bias;   // [N] (EPI_BIAS*)
  const float* R;      // residual added (EPI_BIAS_RES), ld = ldc
  float* C2;           // GELU of the output (EPI_BIAS_GELU), ld = ldc
  const float* aux;    // pre-activation whose GELU derivative scales the output (EPI_GELU_GRAD), ld = ldc
  const uint16_t* bimg;  // BF16 image of B for the tensor-core path (kinds 0, 1), or NULL: CUDA cores
  int* status;           // device status word (a tensor-core wait that gave up)
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// The epilogues of the GEMM kernels for output (m, n) with accumulator v.
__device__ __forceinline__ void epi_store(const Gemm& g, long long m, int n, float v) {
  const long long o = m * g.ldc + n;
  switch (g.epi) {
    case EPI_BIAS:
      g.C[o] = v + g.bias[n];
      break;
    case EPI_BIAS_RES:
      g.C[o] = v + g.bias[n] + g.R[o];
      break;
    case EPI_BIAS_GELU:
      v += g.bias[n];
      g.C[o] = v;
      g.C2[o] = gelu_f(v);
      break;
    case EPI_GELU_GRAD:
      g.C[o] = v * gelu_grad_f(g.aux[o]);
      break;
    case EPI_PARTIAL:
      g.C[((long long)blockIdx.z * g.M + m) * g.N + n] = v;
      break;
    default:
      g.C[o] = v;
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 64 x 64 output tile per CTA of 256 threads, 4 x 4 outputs per thread,
// K staged 16 at a time through shared memory.
template <bool AK, bool BK>
__global__ void __launch_bounds__(256) sgemm_kernel(Gemm g) {
  __shared__ __align__(16) float As[16][68];
  __shared__ __align__(16) float Bs[16][68];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long m0 = (long long)blockIdx.x * 64;
  const int n0 = blockIdx.y * 64;
  const long long kb = (long long)blockIdx.z * g.kchunk;
  const long long ke = kb + g.kchunk < g.K ? kb + g.kchunk : g.K;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  for (long long k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = tid + r * 256;
      const int mm = AK ? (i >> 4) : (i & 63), kk = AK ? (i & 15) : (i >> 6);
      const long long m = m0 + mm, k = k0 + kk;
      float v = 0.0f;
      if (m < g.M && k < ke) v = AK ? g.A[m * g.lda + k] : g.A[k * g.lda + m];
      As[kk][mm] = v;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = tid + r * 256;
      const int nn = BK ? (i >> 4) : (i & 63), kk = BK ? (i & 15) : (i >> 6);
      const long long k = k0 + kk;
      const int n = n0 + nn;
      float v = 0.0f;
      if (n < g.N && k < ke) v = BK ? g.B[(long long)n * g.ldb + k] : g.B[k * g.ldb + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= g.N) continue;
      epi_store(g, m, n, acc[i][j]);
    }
  }
}

// The same product with a 128 x 64 tile, 8 x 4 outputs per thread, float4
// global loads, K staged 32 at a time, the next K slice prefetched into
// registers while the current one is multiplied.  Preconditions (checked on
// the host): the contiguous dimension of each operand is read in aligned
// float4 (leading dimensions and base addresses multiples of 4 floats; M, N
// multiples of 4 where they are contiguous), and with k-contiguous operands
// the K range is a multiple of 32.
template <bool AK, bool BK>
__global__ void __launch_bounds__(256) sgemm128_kernel(Gemm g) {
  __shared__ __align__(16) float As[32][132];
  __shared__ __align__(16) float Bs[32][68];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long m0 = (long long)blockIdx.x * 128;
  const int n0 = blockIdx.y * 64;
  const long long kb = (long long)blockIdx.z * g.kchunk;
  const long long ke = kb + g.kchunk < g.K ? kb + g.kchunk : g.K;
  float4 ra[4], rb[2];
  // A slice: 128 (m) x 32 (k) as 1024 float4, four per thread
  auto load_a = [&](long long k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = tid + r * 256;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (AK) {
        const long long m = m0 + (i >> 3), k = k0 + (i & 7) * 4;
        if (m < g.M && k < ke) v = *reinterpret_cast<const float4*>(g.A + m * g.lda + k);
      } else {
        const long long k = k0 + (i >> 5), m = m0 + (i & 31) * 4;
        if (m < g.M && k < ke) v = *reinterpret_cast<const float4*>(g.A + k * g.lda + m);
      }
      ra[r] = v;
    }
  };
  // B slice: 32 (k) x 64 (n) as 512 float4, two per thread
  auto load_b = [&](long long k0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = tid + r * 256;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (BK) {
        const int n = n0 + (i >> 3);
        const long long k = k0 + (i & 7) * 4;
        if (n < g.N && k < ke) v = *reinterpret_cast<const float4*>(g.B + (long long)n * g.ldb + k);
      } else {
        const long long k = k0 + (i >> 4);
        const int n = n0 + (i & 15) * 4;
        if (n < g.N && k < ke) v = *reinterpret_cast<const float4*>(g.B + k * g.ldb + n);
      }
      rb[r] = v;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = tid + r * 256;
      if (AK) {
        const int mm = i >> 3, kk = (i & 7) * 4;
        As[kk][mm] = ra[r].x;
        As[kk + 1][mm] = ra[r].y;
        As[kk + 2][mm] = ra[r].z;
        As[kk + 3][mm] = ra[r].w;
      } else {
        *reinterpret_cast<float4*>(&As[i >> 5][(i & 31) * 4]) = ra[r];
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = tid + r * 256;
      if (BK) {
        const int nn = i >> 3, kk = (i & 7) * 4;
        Bs[kk][nn] = rb[r].x;
        Bs[kk + 1][nn] = rb[r].y;
        Bs[kk + 2][nn] = rb[r].z;
        Bs[kk + 3][nn] = rb[r].w;
      } else {
        *reinterpret_cast<float4*>(&Bs[i >> 4][(i & 15) * 4]) = rb[r];
      }
    }
  };
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  if (kb < ke) {
    load_a(kb);
    load_b(kb);
    store();
  }
  __syncthreads();
  for (long long k0 = kb; k0 < ke; k0 += 32) {
    const bool more = k0 + 32 < ke;
    if (more) {
      load_a(k0 + 32);
      load_b(k0 + 32);
    }
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();  // every thread is done with the slice before it is overwritten
    if (more) {
      store();
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long m = m0 + ty * 8 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= g.N) continue;
      epi_store(g, m, n, acc[i][j]);
    }
  }
}

// Embedding of the entity tokens; token 0 of each sample is its recurrent
// embedding.  Warps loop over token rows (lane: outputs lane + 32 i, its
// rows of W and its biases held in registers; a row's 8 token features read
// once).
template <typename TokT, int DJ>
__global__ void __launch_bounds__(256) embed_kernel(const TokT* __restrict__ tok, const int32_t* __restrict__ n_ent,
                                                    const float* __restrict__ h, const int32_t* __restrict__ sel,
                                                    const float* __restrict__ W, const float* __restrict__ b,
                                                    float* __restrict__ X, long long n, int T, int NS) {
  constexpr int d = 32 * DJ;
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  float wr[DJ][8], br[DJ];
#pragma unroll
  for (int i = 0; i < DJ; ++i) {
    br[i] = b[lane + 32 * i];
#pragma unroll
    for (int k = 0; k < 8; ++k) wr[i][k] = W[(lane + 32 * i) * 8 + k];
  }
  for (long long row = w0; row < n * T; row += nw) {
    const long long s = row / T;
    const int t = (int)(row - s * T);
    const long long bs = sel ? (long long)sel[s] : s;
    float* x = X + row * d;
    if (t == 0) {
#pragma unroll
      for (int i = 0; i < DJ; ++i) x[lane + 32 * i] = h[bs * d + lane + 32 * i];
      continue;
    }
    int ne = n_ent[bs];
    ne = ne < 0 ? 0 : (ne > NS ? NS : ne);
    float q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = 0.0f;
    if (t <= ne) {
      const TokT* qt = tok + (bs * NS + (t - 1)) * 8;
#pragma unroll
      for (int k = 0; k < 8; ++k) q[k] = (float)qt[k];
    }
#pragma unroll
    for (int i = 0; i < DJ; ++i) {
      float acc = br[i];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc = fmaf(wr[i][k], q[k], acc);
      x[lane + 32 * i] = acc;
    }
  }
}

// LayerNorm forward, one warp per row: Y = (X - mean) rstd g + b and the row's
// (mean, rstd).
template <int DJ>
__global__ void ln_fwd_kernel(const float* __restrict__ X, const float* __restrict__ gam,
                              const float* __restrict__ bet, float* __restrict__ Y, float* __restrict__ stat,
                              long long rows) {
  constexpr int d = 32 * DJ;
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  float gj[DJ], bj[DJ], xn[DJ];
#pragma unroll
  for (int i = 0; i < DJ; ++i) {
    gj[i] = gam[lane + 32 * i];
    bj[i] = bet[lane + 32 * i];
    xn[i] = w0 < rows ? X[w0 * d + lane + 32 * i] : 0.0f;
  }
  for (long long r = w0; r < rows; r += nw) {
    float x[DJ], s = 0.0f;
#pragma unroll
    for (int i = 0; i < DJ; ++i) {
      x[i] = xn[i];
      s += x[i];
    }
    if (r + nw < rows) {  // the warp's next row: in flight during this one
#pragma unroll
      for (int i = 0; i < DJ; ++i) xn[i] = X[(r + nw) * d + lane + 32 * i];
    }
    const float mean = warp_sum(s) * (1.0f / d);
    float v = 0.0f;
#pragma unroll
    for (int i = 0; i < DJ; ++i) v += (x[i] - mean) * (x[i] - mean);
    const float rstd = 1.0f / sqrtf(warp_sum(v) * (1.0f / d) + 1e-5f);
#pragma unroll
    for (int i = 0; i < DJ; ++i) Y[r * d + lane + 32 * i] = (x[i] - mean) * rstd * gj[i] + bj[i];
    if (lane == 0) {
      stat[2 * r] = mean;
      stat[2 * r + 1] = rstd;
    }
  }
}

// LayerNorm backward, one warp per row: out = base + dL/dX from dY (the
// gradient at the LayerNorm output), and per-block partial sums of dL/dg
// (sum dY xh) and dL/db (sum dY) into part[block][2d] (blocks of 256
// threads).  out may equal base.
template <int DJ>
__global__ void ln_bwd_kernel(const float* __restrict__ dY, const float* __restrict__ X,
                              const float* __restrict__ stat, const float* __restrict__ gam, const float* base,
                              float* out, float* __restrict__ part, long long rows) {
  constexpr int d = 32 * DJ;
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  float pg[DJ], pb[DJ], gj[DJ];
  // the warp's next row (dY, X, base, statistics): in flight during the
  // current one
  float dyn[DJ], xn[DJ], bn[DJ], mn = 0.0f, rn = 0.0f;
  auto fetch = [&](long long r) {
#pragma unroll
    for (int i = 0; i < DJ; ++i) {
      const long long o = r * d + lane + 32 * i;
      dyn[i] = dY[o];
      xn[i] = X[o];
      bn[i] = base[o];
    }
    mn = stat[2 * r];
    rn = stat[2 * r + 1];
  };
#pragma unroll
  for (int i = 0; i < DJ; ++i) {
    pg[i] = pb[i] = 0.0f;
    gj[i] = gam[lane + 32 * i];
  }
  if (w0 < rows) fetch(w0);
  for (long long r = w0; r < rows; r += nw) {
    const float mean = mn, rstd = rn;
    float xh[DJ], dxh[DJ], bs[DJ], m1 = 0.0f, m2 = 0.0f;
#pragma unroll
    for (int i = 0; i < DJ; ++i) {
      const float dy = dyn[i];
      xh[i] = (xn[i] - mean) * rstd;
      bs[i] = bn[i];
      dxh[i] = dy * gj[i];
      pg[i] = fmaf(dy, xh[i], pg[i]);
      pb[i] += dy;
      m1 += dxh[i];
      m2 = fmaf(dxh[i], xh[i], m2);
    }
    if (r + nw < rows) fetch(r + nw);
    m1 = warp_sum(m1) * (1.0f / d);
    m2 = warp_sum(m2) * (1.0f / d);
#pragma unroll
    for (int i = 0; i < DJ; ++i) out[r * d + lane + 32 * i] = bs[i] + rstd * (dxh[i] - m1 - xh[i] * m2);
  }
  // the block's 8 warps combined in warp order: one partial per block
  __shared__ float red[8][2 * d];
  const int wl = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < DJ; ++i) {
    red[wl][lane + 32 * i] = pg[i];
    red[wl][d + lane + 32 * i] = pb[i];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < 2 * d; j += blockDim.x) {
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += red[k][j];
    part[(long long)blockIdx.x * 2 * d + j] = t;
  }
}

// Attention work items: pair q = s * H + head.  A warp takes hp = 2 pairs
// when 2T <= 32 (lanes 0..T-1 the first, T..2T-1 the second), else one.
__host__ __device__ __forceinline__ int attn_pairs_per_warp(int T) { return 2 * T <= 32 ? 2 : 1; }
constexpr int kAttnStage = 32;  // staged rows per warp: hp * T <= 32

// Self-attention, lane (slot, t) = query token t of pair q0 + slot:
// P[s][head][t][u] (zero for masked keys u > n_ent) and O = P V.  The warp
// first copies its pairs' K and V rows to shared memory.  4 warps per block.
template <int DH>
__global__ void __launch_bounds__(128) attn_fwd_kernel(const float* __restrict__ QKV,
                                                       const int32_t* __restrict__ n_ent,
                                                       const int32_t* __restrict__ sel, float* __restrict__ P,
                                                       float* __restrict__ O, long long n, int T, int NS, int H,
                                                       float scale) {
  __shared__ float sk[4][kAttnStage * DH];
  __shared__ float sv[4][kAttnStage * DH];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int hp = attn_pairs_per_warp(T);
  const long long q0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * hp;
  const long long nq = n * H;
  if (q0 >= nq) return;  // whole warps leave together
  const int d = DH * H, ld = 3 * d;
  for (int i = lane; i < hp * T * DH; i += 32) {
    const int slot = i / (T * DH), r = i - slot * T * DH, u = r / DH, j = r - u * DH;
    const long long q = q0 + slot;
    if (q < nq) {
      const long long s = q / H;
      const float* base = QKV + s * T * ld + (q - s * H) * DH;
      sk[wl][i] = base[u * ld + d + j];
      sv[wl][i] = base[u * ld + 2 * d + j];
    }
  }
  __syncwarp();
  const int slot = lane / T, t = lane - slot * T;
  const long long q = q0 + slot;
  if (slot >= hp || q >= nq) return;
  const long long s = q / H;
  const int hh = (int)(q - s * H);
  int ne = n_ent[sel ? (long long)sel[s] : s];
  ne = ne < 0 ? 0 : (ne > NS ? NS : ne);
  const float* base = QKV + s * T * ld + hh * DH;
  const float* K = sk[wl] + slot * T * DH;
  const float* V = sv[wl] + slot * T * DH;
  float qv[DH];
#pragma unroll
  for (int j = 0; j < DH; ++j) qv[j] = base[t * ld + j];
  float sc[kMaxT];
  float mx = -INFINITY;
#pragma unroll
  for (int u = 0; u < kMaxT; ++u) {
    sc[u] = -INFINITY;
    if (u < T && u <= ne) {
      float acc = 0.0f;
#pragma unroll
      for (int j = 0; j < DH; ++j) acc = fmaf(qv[j], K[u * DH + j], acc);
      sc[u] = acc * scale;
      mx = fmaxf(mx, sc[u]);
    }
  }
  float z = 0.0f;
#pragma unroll
  for (int u = 0; u < kMaxT; ++u) {
    const float e = (u < T && u <= ne) ? expf(sc[u] - mx) : 0.0f;
    sc[u] = e;
    z += e;
  }
  const float iz = 1.0f / z;
  float o[DH];
#pragma unroll
  for (int j = 0; j < DH; ++j) o[j] = 0.0f;
  float* Pr = P + ((s * H + hh) * T + t) * T;
#pragma unroll
  for (int u = 0; u < kMaxT; ++u) {
    if (u < T) {
      const float p = sc[u] * iz;
      Pr[u] = p;
      if (u <= ne) {
#pragma unroll
        for (int j = 0; j < DH; ++j) o[j] = fmaf(p, V[u * DH + j], o[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < DH; ++j) O[(s * T + t) * d + hh * DH + j] = o[j];
}

// Attention backward of one (sample, head) per warp (4 warps per block): from
// dO and the stored P, dS = P (dP - rowsum(P dP)) scale with dP = dO V^T;
// lane t writes dQ_t, then lane u writes dK_u = sum_t dS_tu Q_t and
// dV_u = sum_t P_tu dO_t.  Q, K, V and dO rows are staged in shared memory.
template <int DH>
__global__ void __launch_bounds__(128) attn_bwd_kernel(const float* __restrict__ QKV, const float* __restrict__ P,
                                                       const float* __restrict__ dO, float* __restrict__ dQKV,
                                                       long long n, int T, int H, float scale) {
  __shared__ float sq[4][kMaxT * DH];
  __shared__ float sk[4][kMaxT * DH];
  __shared__ float sv[4][kMaxT * DH];
  __shared__ float sg[4][kMaxT * DH];
  __shared__ float sdS[4][kMaxT * kMaxT];
  __shared__ float sP[4][kMaxT * kMaxT];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= n * H) return;  // whole warps leave together
  const long long s = w / H;
  const int hh = (int)(w - s * H);
  const int d = DH * H, ld = 3 * d;
  const float* base = QKV + s * T * ld + hh * DH;
  const float* dOb = dO + s * T * d + hh * DH;
  float* out = dQKV + s * T * ld + hh * DH;
  const float* Pb = P + (s * H + hh) * T * T;
  for (int i = lane; i < T * DH; i += 32) {
    const int u = i / DH, j = i - u * DH;
    sq[wl][i] = base[u * ld + j];
    sk[wl][i] = base[u * ld + d + j];
    sv[wl][i] = base[u * ld + 2 * d + j];
    sg[wl][i] = dOb[u * d + j];
  }
  for (int i = lane; i < T * T; i += 32) sP[wl][i] = Pb[i];
  __syncwarp();
  if (lane < T) {
    float dp[kMaxT], dot = 0.0f;
#pragma unroll
    for (int u = 0; u < kMaxT; ++u) {
      dp[u] = 0.0f;
      if (u < T) {
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < DH; ++j) acc = fmaf(sg[wl][lane * DH + j], sv[wl][u * DH + j], acc);
        dp[u] = acc;
        dot = fmaf(sP[wl][lane * T + u], acc, dot);
      }
    }
    float dq[DH];
#pragma unroll
    for (int j = 0; j < DH; ++j) dq[j] = 0.0f;
#pragma unroll
    for (int u = 0; u < kMaxT; ++u) {
      if (u < T) {
        const float ds = sP[wl][lane * T + u] * (dp[u] - dot) * scale;
        sdS[wl][lane * T + u] = ds;
#pragma unroll
        for (int j = 0; j < DH; ++j) dq[j] = fmaf(ds, sk[wl][u * DH + j], dq[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < DH; ++j) out[lane * ld + j] = dq[j];
  }
  __syncwarp();
  if (lane < T) {
    float dk[DH], dv[DH];
#pragma unroll
    for (int j = 0; j < DH; ++j) dk[j] = dv[j] = 0.0f;
    for (int t = 0; t < T; ++t) {
      const float ds = sdS[wl][t * T + lane], p = sP[wl][t * T + lane];
#pragma unroll
      for (int j = 0; j < DH; ++j) {
        dk[j] = fmaf(ds, sq[wl][t * DH + j], dk[j]);
        dv[j] = fmaf(p, sg[wl][t * DH + j], dv[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < DH; ++j) {
      out[lane * ld + d + j] = dk[j];
      out[lane * ld + 2 * d + j] = dv[j];
    }
  }
}

// m16n8k8 TF32 MMA on FP32 registers (operands rounded to TF32 first, FP32
// accumulation).  Fragments (g = lane / 4, t = lane % 4): A a0 (g, t),
// a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4); B b0 (k t, n g),
// b1 (k t + 4, n g); C c0 (g, 2t), c1 (g, 2t + 1), c2 (g + 8, 2t),
// c3 (g + 8, 2t + 1).
__device__ __forceinline__ uint32_t tf32r(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
constexpr int kAttLd = 20;  // floats per staged 16-wide row (conflict-free fragment loads)

// C[16 x 16] (+)= A B over k = 16 from staged [16][kAttLd] tiles: A(r, k) =
// TA ? a[k][r] : a[r][k], B(k, n) = TB ? b[n][k] : b[k][n].  c[j] holds the
// n-tile of columns 8 j .. 8 j + 7.
template <bool TA, bool TB>
__device__ __forceinline__ void mma16x16(float (&c)[2][4], const float* a, const float* b, int g, int t) {
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const int k0 = 8 * kk + t, k1 = k0 + 4;
    const uint32_t a0 = tf32r(TA ? a[k0 * kAttLd + g] : a[g * kAttLd + k0]);
    const uint32_t a1 = tf32r(TA ? a[k0 * kAttLd + g + 8] : a[(g + 8) * kAttLd + k0]);
    const uint32_t a2 = tf32r(TA ? a[k1 * kAttLd + g] : a[g * kAttLd + k1]);
    const uint32_t a3 = tf32r(TA ? a[k1 * kAttLd + g + 8] : a[(g + 8) * kAttLd + k1]);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int nn = 8 * j + g;
      const uint32_t b0 = tf32r(TB ? b[nn * kAttLd + k0] : b[k0 * kAttLd + nn]);
      const uint32_t b1 = tf32r(TB ? b[nn * kAttLd + k1] : b[k1 * kAttLd + nn]);
      mma_tf32(c[j], a0, a1, a2, a3, b0, b1);
    }
  }
}

// Per-warp staging of one (sample, head) item: rows u = lane / 4 + 8 r
// (r = 0, 1) of the item's 16-wide Q, K, V slices (and dO in the backward),
// quarter lane % 4 of each row, as float4; rows u >= T are zero.  The warps
// are persistent: the next item's slices are loaded into registers while the
// current item is computed from shared memory.
struct AttRows {
  float4 q[2], k[2], v[2];
};
__device__ __forceinline__ void att_fetch(AttRows& r, const float* __restrict__ QKV, long long s, int hh, int T, int d,
                                          int lane) {
  const int u0 = lane >> 2, j4 = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int u = u0 + 8 * i;
    r.q[i] = r.k[i] = r.v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (u < T) {
      const float4* base = reinterpret_cast<const float4*>(QKV + (s * T + u) * 3 * d + hh * 16) + j4;
      r.q[i] = __ldg(base);
      r.k[i] = __ldg(base + d / 4);
      r.v[i] = __ldg(base + d / 2);
    }
  }
}
__device__ __forceinline__ void att_stage(const float4 (&x)[2], float* dst, int lane) {
  const int u0 = lane >> 2, j4 = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i) *reinterpret_cast<float4*>(dst + (u0 + 8 * i) * kAttLd + 4 * j4) = x[i];
}

// Blocks of `threads` threads of `kernel` resident on the device at once (at
// least one per SM), for the persistent and grid-stride kernels.
template <typename K>
inline long long resident_blocks(K kernel, int threads) {
  int dev = 0, b = 0, m = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    b = 1, m = 152;
  }
  return (long long)(b > 0 ? b : 1) * (m > 0 ? m : 152);
}

// Grid of a persistent attention kernel (4 items per block at a time): the
// resident blocks, or fewer when there are fewer items.
template <typename K>
inline long long att_grid(K kernel, long long items) {
  static const long long cap = resident_blocks(kernel, 128);  // (initialised once, thread-safe)
  const long long need = (items + 3) / 4;
  return need < cap ? need : cap;
}

// Attention forward on the tensor cores (tensor-core path; T <= 16, head
// dimension 16), one (sample, head) item per warp at a time, persistent warps
// (4 per block) over the items: S = Q K^T as m16n8k8 TF32 MMAs over the
// tokens padded to 16, the masked softmax on the accumulator fragments (keys
// u <= n_ent of the sample, a row in the 4 lanes of a quad), P written out
// (zero at masked keys) and staged, then O = P V.
__global__ void __launch_bounds__(128, 8)
    attn_fwd_mma_kernel(const float* __restrict__ QKV, const int32_t* __restrict__ n_ent,
                        const int32_t* __restrict__ sel, float* __restrict__ P, float* __restrict__ O, long long n,
                        int T, int NS, int H, float scale) {
  __shared__ __align__(16) float sm[4][4][16 * kAttLd];  // Q, K, V, P of each warp
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int d = 16 * H;
  const long long items = n * H, stride = (long long)gridDim.x * 4;
  float *sQ = sm[wl][0], *sK = sm[wl][1], *sV = sm[wl][2], *sP = sm[wl][3];
  long long w = (long long)blockIdx.x * 4 + wl;
  AttRows r;
  int ne_next = 0;
  auto fetch = [&](long long wi) {
    const long long s = wi / H;
    att_fetch(r, QKV, s, (int)(wi - s * H), T, d, lane);
    ne_next = __ldg(n_ent + (sel ? (long long)__ldg(sel + s) : s));
  };
  if (w < items) fetch(w);
  for (; w < items; w += stride) {
    const long long s = w / H;
    const int hh = (int)(w - s * H);
    att_stage(r.q, sQ, lane);
    att_stage(r.k, sK, lane);
    att_stage(r.v, sV, lane);
    const int ne = ne_next < 0 ? 0 : (ne_next > NS ? NS : ne_next);
    if (w + stride < items) fetch(w + stride);  // in flight during this item
    __syncwarp();
    float sc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    mma16x16<false, true>(sc, sQ, sK, g, t);  // S = Q K^T
    float* Pb = P + (s * H + hh) * T * T;
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int row = g + 8 * hr;
      float mx = -INFINITY;
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int col = 8 * j + 2 * t + e;
          const float v = (col < T && col <= ne) ? sc[j][2 * hr + e] * scale : -INFINITY;
          sc[j][2 * hr + e] = v;
          mx = fmaxf(mx, v);
        }
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      float z = 0.0f;
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float x = sc[j][2 * hr + e];
          const float ex = x == -INFINITY ? 0.0f : __expf(x - mx);
          sc[j][2 * hr + e] = ex;
          z += ex;
        }
      z += __shfl_xor_sync(0xffffffffu, z, 1);
      z += __shfl_xor_sync(0xffffffffu, z, 2);
      const float iz = 1.0f / z;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int col = 8 * j + 2 * t;
        const float p0 = sc[j][2 * hr] * iz, p1 = sc[j][2 * hr + 1] * iz;
        sP[row * kAttLd + col] = p0;
        sP[row * kAttLd + col + 1] = p1;
        if (row < T) {
          if (col < T) Pb[row * T + col] = p0;
          if (col + 1 < T) Pb[row * T + col + 1] = p1;
        }
      }
    }
    __syncwarp();
    float o[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    mma16x16<false, false>(o, sP, sV, g, t);  // O = P V
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int row = g + 8 * hr;
      if (row < T) {
#pragma unroll
        for (int j = 0; j < 2; ++j)
          *reinterpret_cast<float2*>(O + (s * T + row) * d + hh * 16 + 8 * j + 2 * t) =
              make_float2(o[j][2 * hr], o[j][2 * hr + 1]);
      }
    }
    __syncwarp();  // the staged tiles are read before the next item overwrites them
  }
}

// Attention backward on the tensor cores (tensor-core path; T <= 16, head
// dimension 16), one (sample, head) item per warp at a time, persistent warps
// (4 per block): the products of attn_bwd_kernel, dP = dO V^T, dQ = dS K,
// dK = dS^T Q, dV = P^T dO, as m16n8k8 TF32 MMAs over the tokens padded to
// 16 (padded rows and columns staged as zeros), and
// dS = P (dP - rowsum(P dP)) scale on the accumulator fragments (a row lives
// in the 4 lanes of a quad).  dS is staged over V (V is read only by dP).
__global__ void __launch_bounds__(128, 6)
    attn_bwd_mma_kernel(const float* __restrict__ QKV, const float* __restrict__ P, const float* __restrict__ dO,
                        float* __restrict__ dQKV, long long n, int T, int H, float scale) {
  __shared__ __align__(16) float sm[4][5][16 * kAttLd];  // Q, K, V then dS, dO, P of each warp
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int d = 16 * H, ld = 3 * d;
  const long long items = n * H, stride = (long long)gridDim.x * 4;
  float *sQ = sm[wl][0], *sK = sm[wl][1], *sV = sm[wl][2], *sS = sm[wl][2], *sG = sm[wl][3], *sP = sm[wl][4];
  // P of an item: T * T contiguous floats, element e = lane + 32 i at
  // (e / T, e % T) of the staged tile; the padding stays zero
  int pofs[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = lane + 32 * i;
    pofs[i] = e < T * T ? (e / T) * kAttLd + e % T : -1;
  }
  for (int i = lane; i < 16 * kAttLd; i += 32) sP[i] = 0.0f;
  long long w = (long long)blockIdx.x * 4 + wl;
  AttRows r;
  float4 rg[2];
  float rp[4];
  auto fetch = [&](long long wi) {
    const long long s = wi / H;
    const int hh = (int)(wi - s * H);
    att_fetch(r, QKV, s, hh, T, d, lane);
    const int u0 = lane >> 2, j4 = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int u = u0 + 8 * i;
      rg[i] = u < T ? __ldg(reinterpret_cast<const float4*>(dO + (s * T + u) * d + hh * 16) + j4)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float* Pb = P + (s * H + hh) * T * T;
#pragma unroll
    for (int i = 0; i < 4; ++i) rp[i] = pofs[i] >= 0 ? __ldg(Pb + lane + 32 * i) : 0.0f;
  };
  if (w < items) fetch(w);
  for (; w < items; w += stride) {
    const long long s = w / H;
    const int hh = (int)(w - s * H);
    att_stage(r.q, sQ, lane);
    att_stage(r.k, sK, lane);
    att_stage(r.v, sV, lane);
    att_stage(rg, sG, lane);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (pofs[i] >= 0) sP[pofs[i]] = rp[i];
    if (w + stride < items) fetch(w + stride);  // in flight during this item
    __syncwarp();
    // dP = dO V^T
    float dp[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    mma16x16<false, true>(dp, sG, sV, g, t);
    // dS = P (dP - rowsum(P dP)) scale (rows g and g + 8 of this quad)
    float pv[2][4], r0 = 0.0f, r1 = 0.0f;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int c = 8 * j + 2 * t;
      pv[j][0] = sP[g * kAttLd + c];
      pv[j][1] = sP[g * kAttLd + c + 1];
      pv[j][2] = sP[(g + 8) * kAttLd + c];
      pv[j][3] = sP[(g + 8) * kAttLd + c + 1];
      r0 = fmaf(pv[j][0], dp[j][0], fmaf(pv[j][1], dp[j][1], r0));
      r1 = fmaf(pv[j][2], dp[j][2], fmaf(pv[j][3], dp[j][3], r1));
    }
    r0 += __shfl_xor_sync(0xffffffffu, r0, 1);
    r0 += __shfl_xor_sync(0xffffffffu, r0, 2);
    r1 += __shfl_xor_sync(0xffffffffu, r1, 1);
    r1 += __shfl_xor_sync(0xffffffffu, r1, 2);
    __syncwarp();  // every lane's V fragments are read: dS goes over V
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int c = 8 * j + 2 * t;
      sS[g * kAttLd + c] = pv[j][0] * (dp[j][0] - r0) * scale;
      sS[g * kAttLd + c + 1] = pv[j][1] * (dp[j][1] - r0) * scale;
      sS[(g + 8) * kAttLd + c] = pv[j][2] * (dp[j][2] - r1) * scale;
      sS[(g + 8) * kAttLd + c + 1] = pv[j][3] * (dp[j][3] - r1) * scale;
    }
    __syncwarp();
    float dq[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    float dk[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    float dv[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    mma16x16<false, false>(dq, sS, sK, g, t);  // dQ = dS K
    mma16x16<true, false>(dk, sS, sQ, g, t);   // dK = dS^T Q
    mma16x16<true, false>(dv, sP, sG, g, t);   // dV = P^T dO
    float* out = dQKV + s * T * ld + hh * 16;
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int row = g + 8 * hr;
      if (row < T) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int c = 8 * j + 2 * t;
          *reinterpret_cast<float2*>(out + row * ld + c) = make_float2(dq[j][2 * hr], dq[j][2 * hr + 1]);
          *reinterpret_cast<float2*>(out + row * ld + d + c) = make_float2(dk[j][2 * hr], dk[j][2 * hr + 1]);
          *reinterpret_cast<float2*>(out + row * ld + 2 * d + c) = make_float2(dv[j][2 * hr], dv[j][2 * hr + 1]);
        }
      }
    }
    __syncwarp();  // the staged tiles are read before the next item overwrites them
  }
}

struct HeadArgs {
  const float* XL;  // [rows][d] residual stream after the last block
  long long n;
  int T, n_out, mode;  // mode 0: forward, 1: PPO actor loss, 2: value loss
  const float *lnf_g, *lnf_b, *Wh, *bh;
  float* out;        // [n][n_out] (mode 0)
  float* h_out;      // [n][d] (mode 0, optional)
  const int32_t* sel;
  const int32_t* actions;
  const float *logp_old, *adv, *ret;
  float clip_eps, ent_coef, inv_n;
  float* dXL;        // [rows][d] (modes 1, 2): token 0 gets the gradient, the other rows zero
  float* part;       // [warps][2d + n_out d + n_out]: lnf_g, lnf_b, Wh, bh partial gradients
  double* spart;     // [warps][4] partial sums of the per-sample statistics
};

// Final LayerNorm and head on token 0, one warp per sample; in the loss modes
// also the loss, dL/d(head output), the head's and final LayerNorm's
// backward, and per-warp partial sums of their parameter gradients.
template <int DJ, int NO>
__global__ void __launch_bounds__(256) head_kernel(HeadArgs a) {
  constexpr int d = 32 * DJ;
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const int no = a.n_out;
  float gW[NO][DJ], gB[NO], gg[DJ], gb[DJ];
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    gB[o] = 0.0f;
#pragma unroll
    for (int i = 0; i < DJ; ++i) gW[o][i] = 0.0f;
  }
#pragma unroll
  for (int i = 0; i < DJ; ++i) gg[i] = gb[i] = 0.0f;
  double st[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long s = w0; s < a.n; s += nw) {
    const float* x0 = a.XL + s * a.T * d;
    float x[DJ], xh[DJ], U[DJ], sum = 0.0f;
#pragma unroll
    for (int i = 0; i < DJ; ++i) {
      x[i] = x0[lane + 32 * i];
      sum += x[i];
    }
    const float mean = warp_sum(sum) * (1.0f / d);
    float v = 0.0f;
#pragma unroll
    for (int i = 0; i < DJ; ++i) v += (x[i] - mean) * (x[i] - mean);
    const float rstd = 1.0f / sqrtf(warp_sum(v) * (1.0f / d) + 1e-5f);
#pragma unroll
    for (int i = 0; i < DJ; ++i) {
      const int j = lane + 32 * i;
      xh[i] = (x[i] - mean) * rstd;
      U[i] = xh[i] * a.lnf_g[j] + a.lnf_b[j];
    }
    float z[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      z[o] = 0.0f;
      if (o < no) {
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < DJ; ++i) acc = fmaf(a.Wh[o * d + lane + 32 * i], U[i], acc);
        z[o] = warp_sum(acc) + a.bh[o];
      }
    }
    if (a.mode == 0) {
      if (lane < no) {
#pragma unroll
        for (int o = 0; o < NO; ++o)
          if (o == lane) a.out[s * no + o] = z[o];
      }
      if (a.h_out)
#pragma unroll
        for (int i = 0; i < DJ; ++i) a.h_out[s * d + lane + 32 * i] = x[i];
      continue;
    }
    const long long bs = a.sel ? (long long)a.sel[s] : s;
    float dz[NO];
    if (a.mode == 2) {
      const float e = z[0] - a.ret[bs];
#pragma unroll
      for (int o = 0; o < NO; ++o) dz[o] = 0.0f;
      dz[0] = 2.0f * e * a.inv_n;
      st[0] += (double)e * e;
      st[1] += (double)z[0];
    } else {
      float mx = -INFINITY;
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < no) mx = fmaxf(mx, z[o]);
      float zs = 0.0f;
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < no) zs += expf(z[o] - mx);
      const float lse = mx + logf(zs);
      const int act = a.actions[bs];
      float ent = 0.0f, lpa = 0.0f;
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < no) {
          const float lp = z[o] - lse;
          ent -= expf(lp) * lp;
          if (o == act) lpa = lp;
        }
      const float A = a.adv[bs], lo = a.logp_old[bs];
      const float r = expf(lpa - lo);
      const float rc = fminf(fmaxf(r, 1.0f - a.clip_eps), 1.0f + a.clip_eps);
      const float s1 = r * A, s2 = rc * A;
      const float gl = s1 <= s2 ? -A * r : 0.0f;  // ties: the unclipped term carries the gradient
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        dz[o] = 0.0f;
        if (o < no) {
          const float lp = z[o] - lse, p = expf(lp);
          dz[o] = (gl * ((o == act ? 1.0f : 0.0f) - p) + a.ent_coef * p * (lp + ent)) * a.inv_n;
        }
      }
      st[0] += (double)(-fminf(s1, s2) - a.ent_coef * ent);
      st[1] += (double)ent;
      st[2] += fabsf(r - 1.0f) > a.clip_eps ? 1.0 : 0.0;
      st[3] += (double)(lo - lpa);
    }
    float dU[DJ];
#pragma unroll
    for (int i = 0; i < DJ; ++i) dU[i] = 0.0f;
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < no) {
        gB[o] += dz[o];
#pragma unroll
        for (int i = 0; i < DJ; ++i) {
          gW[o][i] = fmaf(dz[o], U[i], gW[o][i]);
          dU[i] = fmaf(a.Wh[o * d + lane + 32 * i], dz[o], dU[i]);
        }
      }
    float dxh[DJ], m1 = 0.0f, m2 = 0.0f;
#pragma unroll
    for (int i = 0; i < DJ; ++i) {
      const int j = lane + 32 * i;
      dxh[i] = dU[i] * a.lnf_g[j];
      gg[i] = fmaf(dU[i], xh[i], gg[i]);
      gb[i] += dU[i];
      m1 += dxh[i];
      m2 = fmaf(dxh[i], xh[i], m2);
    }
    m1 = warp_sum(m1) * (1.0f / d);
    m2 = warp_sum(m2) * (1.0f / d);
    float* dx0 = a.dXL + s * a.T * d;
#pragma unroll
    for (int i = 0; i < DJ; ++i) dx0[lane + 32 * i] = rstd * (dxh[i] - m1 - xh[i] * m2);
    for (int t = 1; t < a.T; ++t)
#pragma unroll
      for (int i = 0; i < DJ; ++i) dx0[t * d + lane + 32 * i] = 0.0f;
  }
  if (a.mode == 0) return;
  const long long plen = 2 * d + (long long)no * d + no;
  float* pp = a.part + w0 * plen;
#pragma unroll
  for (int i = 0; i < DJ; ++i) {
    pp[lane + 32 * i] = gg[i];
    pp[d + lane + 32 * i] = gb[i];
  }
#pragma unroll
  for (int o = 0; o < NO; ++o)
    if (o < no) {
#pragma unroll
      for (int i = 0; i < DJ; ++i) pp[2 * d + o * d + lane + 32 * i] = gW[o][i];
      if (lane == 0) pp[2 * d + no * d + o] = gB[o];
    }
  if (lane == 0)
    for (int k = 0; k < 4; ++k) a.spart[w0 * 4 + k] = st[k];
}

// Embedding weight gradients, one warp per sample: per-warp partial sums of
// dW_emb[j][k] = sum dX[row][j] tok[row][k] and db_emb[j] over the sample's
// entity rows, into part[warp][9d] (W_emb then b_emb).
template <typename TokT, int DJ>
__global__ void __launch_bounds__(256) embed_grad_kernel(const TokT* __restrict__ tok,
                                                         const int32_t* __restrict__ n_ent,
                                                         const int32_t* __restrict__ sel,
                                                         const float* __restrict__ dX, float* __restrict__ part,
                                                         long long n, int T, int NS) {
  constexpr int d = 32 * DJ;
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  float gW[DJ][8], gb[DJ];
#pragma unroll
  for (int i = 0; i < DJ; ++i) {
    gb[i] = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) gW[i][k] = 0.0f;
  }
  for (long long s = w0; s < n; s += nw) {
    const long long bs = sel ? (long long)sel[s] : s;
    int ne = n_ent[bs];
    ne = ne < 0 ? 0 : (ne > NS ? NS : ne);
    for (int t = 1; t <= ne; ++t) {
      const TokT* q = tok + (bs * NS + (t - 1)) * 8;
      float tk[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) tk[k] = (float)q[k];
#pragma unroll
      for (int i = 0; i < DJ; ++i) {
        const float g = dX[(s * T + t) * d + lane + 32 * i];
        gb[i] += g;
#pragma unroll
        for (int k = 0; k < 8; ++k) gW[i][k] = fmaf(g, tk[k], gW[i][k]);
      }
    }
  }
  float* pp = part + w0 * 9 * d;
#pragma unroll
  for (int i = 0; i < DJ; ++i) {
    const int j = lane + 32 * i;
#pragma unroll
    for (int k = 0; k < 8; ++k) pp[j * 8 + k] = gW[i][k];
    pp[8 * d + j] = gb[i];
  }
}

// Column sums of A [rows][N] (leading dimension lda): block (x, y) sums
// columns 32x .. 32x+31 over its share of the rows into part[y][N].
__global__ void __launch_bounds__(256) colsum_kernel(const float* __restrict__ A, long long lda, long long rows,
                                                     int N, float* __restrict__ part) {
  __shared__ float red[8][33];
  const int c = blockIdx.x * 32 + (threadIdx.x & 31), rg = threadIdx.x >> 5;
  const long long chunk = (rows + gridDim.y - 1) / gridDim.y;
  const long long r0 = (long long)blockIdx.y * chunk;
  const long long r1 = r0 + chunk < rows ? r0 + chunk : rows;
  float acc = 0.0f;
  if (c < N)
    for (long long r = r0 + rg; r < r1; r += 8) acc += A[r * lda + c];
  red[rg][threadIdx.x & 31] = acc;
  __syncthreads();
  if (rg == 0 && c < N) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += red[k][threadIdx.x & 31];
    part[(long long)blockIdx.y * N + c] = s;
  }
}

// out[i] = sum over p of part[p * stride + i]: block x sums columns
// 32x .. 32x+31, thread row g the parts p = g (mod 32) in increasing p, then
// the 32 row sums in order of g (a fixed association: deterministic).
__global__ void __launch_bounds__(1024) reduce_kernel(const float* __restrict__ part, int nparts, long long len,
                                                      long long stride, float* __restrict__ out) {
  __shared__ float red[32][33];
  const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
  const long long i = (long long)blockIdx.x * 32 + c;
  float s = 0.0f;
  if (i < len)
    for (int p = g; p < nparts; p += 32) s += part[p * stride + i];
  red[g][c] = s;
  __syncthreads();
  if (g == 0 && i < len) {
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < 32; ++k) t += red[k][c];
    out[i] = t;
  }
}

// Statistics: sums of the per-warp partials times inv_n; thread j of 256
// sums parts p = j (mod 64) of statistic j / 64, then 64 partial sums are
// added in order.
__global__ void __launch_bounds__(256) reduce_stats_kernel(const double* __restrict__ spart, int nparts,
                                                           double inv_n, double* __restrict__ out) {
  __shared__ double red[4][64];
  const int k = threadIdx.x >> 6, j = threadIdx.x & 63;
  double s = 0.0;
  for (int p = j; p < nparts; p += 64) s += spart[p * 4 + k];
  red[k][j] = s;
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int q = 0; q < 64; ++q) t += red[threadIdx.x][q];
    out[threadIdx.x] = t * inv_n;
  }
}

// Adam with bias correction (Kingma & Ba 2015, Algorithm 1); bc1 = 1 -
// beta1^t and bc2 = 1 - beta2^t are computed on the host in double.
__global__ void adam_kernel(float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps,
                            float bc1, float bc2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// GAE by the backward recursion, one thread per env.
__global__ void gae_kernel(const float* __restrict__ r, const float* __restrict__ v, const int32_t* __restrict__ done,
                           int T, long long E, float gamma, float lam, float* __restrict__ adv,
                           float* __restrict__ ret) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  float a = 0.0f;
  for (int t = T - 1; t >= 0; --t) {
    const long long i = (long long)t * E + e;
    const float nd = done[i] ? 0.0f : 1.0f;
    const float delta = r[i] + gamma * nd * v[i + E] - v[i];
    a = delta + gamma * lam * nd * a;
    adv[i] = a;
    ret[i] = a + v[i];
  }
}

__global__ void gae_agents_kernel(const float* __restrict__ adv, const int32_t* __restrict__ agent_env, int T,
                                  long long E, long long NA, float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)T * NA) return;
  const long long t = i / NA, a = i - t * NA;
  out[i] = adv[t * E + agent_env[a]];
}

}  // namespace tfm
}  // namespace ut

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
#include "runtime.cuh"

struct ut_tfm {
  ut_tfm_config cfg{};
  cudaStream_t stream = nullptr;
  std::string err;
  int d = 0, L = 0, H = 0, dh = 0, n_out = 0, NS = 0, T = 0, f = 0;
  int64_t n_params = 0, max_rows = 0;
  std::vector<void*> allocs;
  float *prm = nullptr, *am = nullptr, *av = nullptr;
  int adam_t = 0;
  // activations: X [(L+1)][max_rows][d]; per block l: Y1, O, M, Y2 [rows][d],
  // S1, S2 [rows][2], QKV [rows][3d], P [samples][H][T][T], Z, G [rows][4d]
  float *X = nullptr, *Y1 = nullptr, *Y2 = nullptr, *S1 = nullptr, *S2 = nullptr, *QKV = nullptr, *P = nullptr,
        *O = nullptr, *M = nullptr, *Z = nullptr, *G = nullptr;
  // backward buffers
  float *dX = nullptr, *dM = nullptr, *dY = nullptr, *dO = nullptr, *dBig = nullptr;
  float* part = nullptr;  // partial sums of the parameter gradients
  double *spart = nullptr, *stats_d = nullptr;
  std::vector<int64_t> off;  // canonical tensor offsets
  // GEMM path: 1 BF16 tensor cores (FP32 accumulation), 0 FP32 CUDA cores
  int gemm_tc = 1;
  // BF16 images of the block weights for the tensor-core path, per block l:
  // Wqkv, Wo, W1, W2 as B of the forward, then their transposes as B of the
  // input gradient (ImgSpec table on the device, packed once per call)
  uint16_t* wimg = nullptr;
  std::vector<int64_t> img_off;  // [L][8] offsets into wimg (elements)
  int64_t* img_spec = nullptr;   // [L * 8][5] (weight offset, R, C, transpose, image offset)
  int n_img = 0, img_max = 0;
  int* status = nullptr;
};

namespace ut {
namespace tfm {
namespace {

// Tensor offsets in the canonical order: 0 W_emb, 1 b_emb, per block l at
// 2 + 12 l: ln1_g, ln1_b, Wqkv, bqkv, Wo, bo, ln2_g, ln2_b, W1, b1, W2, b2;
// then lnf_g, lnf_b, Wh, bh and the end.
enum { T_LN1G = 0, T_LN1B, T_WQKV, T_BQKV, T_WO, T_BO, T_LN2G, T_LN2B, T_W1, T_B1, T_W2, T_B2 };

std::vector<int64_t> offsets(int d, int L, int n_out) {
  std::vector<int64_t> o;
  int64_t p = 0;
  auto add = [&](int64_t n) {
    o.push_back(p);
    p += n;
  };
  const int64_t D = d, F = 4 * (int64_t)d;
  add(D * 8);
  add(D);
  for (int l = 0; l < L; ++l) {
    add(D); add(D); add(3 * D * D); add(3 * D); add(D * D); add(D);
    add(D); add(D); add(F * D); add(F); add(D * F); add(D);
  }
  add(D); add(D); add((int64_t)n_out * D); add(n_out);
  o.push_back(p);
  return o;
}

bool valid_config(const ut_tfm_config* c) {
  if (!c || c->abi_version != UT_ABI_VERSION) return false;
  const int d = c->d_model;
  if (d != 32 && d != 64 && d != 96 && d != 128) return false;
  if (c->n_layers < 1 || c->n_layers > 8 || c->n_heads < 1 || d % c->n_heads) return false;
  const int dh = d / c->n_heads;
  if (dh != 8 && dh != 16 && dh != 32) return false;
  if (c->n_out < 1 || c->n_out > 16) return false;
  if (c->n_slots < 1 || c->n_slots > UT_MAX_AGENTS + UT_MAX_TARGETS) return false;
  if (c->tokens_bf16 != 0 && c->tokens_bf16 != 1) return false;
  return c->max_batch >= 1 && c->max_batch <= (1ll << 22);
}

#include "tfm_tc.cuh"

// Every BF16 weight image of the handle: grid (elements, image).
__global__ void pack_images_kernel(const float* __restrict__ prm, const int64_t* __restrict__ spec,
                                   uint16_t* __restrict__ img) {
  const int64_t* sp = spec + 5 * blockIdx.y;
  const int R = (int)sp[1], C = (int)sp[2];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)R * C) return;
  const int r = (int)(i / C), c = (int)(i % C);
  const float* W = prm + sp[0];
  const float v = sp[3] ? W[(long long)c * R + r] : W[(long long)r * C + c];
  img[sp[4] + img_offset(r, c, R, C) / 2] = f2bf_bits(v);
}

inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// kind 0: forward (A row-major, B = W [N][K]); 1: input gradient (A
// row-major, B = W [K][N]); 2: weight gradient (A and B indexed [k][.]).
cudaError_t gemm(int kind, const Gemm& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
  if (kind != 2 && g.bimg && g.K % 32 == 0 && g.N % 32 == 0 && g.lda % 4 == 0 && g.ldc % 4 == 0 &&
      ((uintptr_t)g.A & 15) == 0 && ((uintptr_t)g.C & 15) == 0 && g.kchunk == g.K) {
    static std::atomic<unsigned long long> ready{0};
    cudaError_t e = smem_optin(tc_rows_kernel, kTcSmem, ready);
    if (e != cudaSuccess) return e;
    // CTAs loop over the row tiles: about as many per SM per column tile as
    // fit (three for N <= 128, two for the wider products)
    const size_t smem = tc_rows_smem(g.N);
    const int per_sm = smem <= 72 * 1024 ? 3 : 2;
    const long long tiles = (g.M + 127) / 128;
    const int n_tiles = (g.N + kTcMaxN - 1) / kTcMaxN;
    long long ctas = (per_sm * 152 + n_tiles - 1) / n_tiles;
    if (ctas > tiles) ctas = tiles;
    dim3 grid((unsigned)ctas, (unsigned)n_tiles);
    tc_rows_kernel<<<grid, kTcThreads, smem, s>>>(g, g.bimg, g.status);
    return cudaGetLastError();
  }
  const long long kc = g.kchunk > 0 ? g.kchunk : g.K;
  dim3 grid((unsigned)((g.M + 63) / 64), (unsigned)((g.N + 63) / 64), (unsigned)((g.K + kc - 1) / kc));
  Gemm a = g;
  a.kchunk = kc;
  // aligned float4 operands: the 128 x 64 kernel
  auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
  const bool ak = kind != 2, bk = kind == 0;
  bool fast = al(g.A) && al(g.B) && g.lda % 4 == 0 && g.ldb % 4 == 0;
  fast = fast && (ak ? (kc % 32 == 0 && g.K % 32 == 0) : g.M % 4 == 0);
  fast = fast && (bk ? (kc % 32 == 0 && g.K % 32 == 0) : g.N % 4 == 0);
  if (fast) {
    dim3 grid2((unsigned)((g.M + 127) / 128), (unsigned)((g.N + 63) / 64), (unsigned)((g.K + kc - 1) / kc));
    if (kind == 0)
      sgemm128_kernel<true, true><<<grid2, 256, 0, s>>>(a);
    else if (kind == 1)
      sgemm128_kernel<true, false><<<grid2, 256, 0, s>>>(a);
    else
      sgemm128_kernel<false, false><<<grid2, 256, 0, s>>>(a);
    return cudaGetLastError();
  }
  if (kind == 0)
    sgemm_kernel<true, true><<<grid, 256, 0, s>>>(a);
  else if (kind == 1)
    sgemm_kernel<true, false><<<grid, 256, 0, s>>>(a);
  else
    sgemm_kernel<false, false><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

Gemm mk(const float* A, long long lda, const float* B, long long ldb, float* C, long long ldc, long long M, int N,
        long long K, int epi) {
  Gemm g;
  std::memset(&g, 0, sizeof(g));
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
  g.M = M; g.N = N; g.K = K; g.kchunk = K; g.epi = epi;
  return g;
}

cudaError_t reduce(const float* part, int nparts, long long len, long long stride, float* out, cudaStream_t s) {
  reduce_kernel<<<blocks_for(len, 32), 1024, 0, s>>>(part, nparts, len, stride, out);
  return cudaGetLastError();
}

// dW[o][i] = sum_r dOut[r][o] In[r][i] and db[o] = sum_r dOut[r][o] over rows
// r, split along the rows into partial slabs summed in order.
cudaError_t wgrad(ut_tfm* t, const float* dOut, int n_o, const float* In, int n_i, long long rows, float* gW,
                  float* gb, cudaStream_t s) {
  if (t->gemm_tc && rows > 0) {
    // tensor cores: (n_o / 128) x (n_i / 256) tiles x row splits, about as
    // many CTAs per SM as fit (three for n_i <= 128, else two), each split a
    // multiple of 64 rows
    static std::atomic<unsigned long long> ready{0};
    cudaError_t e = smem_optin(tc_wgrad_kernel, kTcSmem, ready);
    if (e != cudaSuccess) return e;
    const size_t smem = tc_wgrad_smem(n_i);
    const int per_sm = smem <= 72 * 1024 ? 3 : 2;
    const long long tiles = (long long)((n_o + 127) / 128) * ((n_i + kTcMaxN - 1) / kTcMaxN);
    long long splits = (per_sm * 152 + tiles - 1) / tiles;
    const long long max_split = (rows + kTcChunk - 1) / kTcChunk;
    if (splits > max_split) splits = max_split;
    if (splits < 1) splits = 1;
    long long rc = (rows + splits - 1) / splits;
    rc = (rc + kTcChunk - 1) / kTcChunk * kTcChunk;
    splits = (rows + rc - 1) / rc;
    Gemm g = mk(dOut, n_o, In, n_i, t->part, n_i, n_o, n_i, rows, EPI_PARTIAL);
    g.kchunk = rc;
    g.status = t->status;
    dim3 grid((unsigned)((n_o + 127) / 128), (unsigned)((n_i + kTcMaxN - 1) / kTcMaxN), (unsigned)splits);
    float* bias_part = t->part + splits * n_o * n_i;
    tc_wgrad_kernel<<<grid, kTcThreads, smem, s>>>(g, bias_part, t->status);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = reduce(t->part, (int)splits, (long long)n_o * n_i, (long long)n_o * n_i, gW, s);
    if (e == cudaSuccess) e = reduce(bias_part, (int)splits, n_o, n_o, gb, s);
    return e;
  }
  Gemm g = mk(dOut, n_o, In, n_i, t->part, n_i, n_o, n_i, rows, EPI_PARTIAL);
  const long long tiles = (long long)((n_o + 63) / 64) * ((n_i + 63) / 64);
  long long splits = (608 + tiles - 1) / tiles;
  splits = splits < 1 ? 1 : (splits > 128 ? 128 : splits);
  const long long max_split = (rows + 63) / 64;
  if (splits > max_split) splits = max_split;
  long long kc = (rows + splits - 1) / splits;
  kc = (kc + 15) / 16 * 16;
  splits = (rows + kc - 1) / kc;
  g.kchunk = kc;
  cudaError_t e = gemm(2, g, s);
  if (e == cudaSuccess) e = reduce(t->part, (int)splits, (long long)n_o * n_i, (long long)n_o * n_i, gW, s);
  if (e != cudaSuccess) return e;
  long long nblk = (rows + 63) / 64;
  nblk = nblk < 1 ? 1 : (nblk > 256 ? 256 : nblk);
  colsum_kernel<<<dim3((unsigned)((n_o + 31) / 32), (unsigned)nblk), 256, 0, s>>>(dOut, n_o, rows, n_o, t->part);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = reduce(t->part, (int)nblk, n_o, n_o, gb, s);
  return e;
}

// The LayerNorm kernels loop over rows (grid stride): at most kLnBlocks
// blocks, no more than are resident at once.
template <int DJ>
cudaError_t ln_fwd(const float* X, const float* g, const float* b, float* Y, float* st, long long rows, cudaStream_t s) {
  static const int nblk = (int)std::min<long long>(kLnBlocks, resident_blocks(ln_fwd_kernel<DJ>, 256));
  ln_fwd_kernel<DJ><<<nblk, 256, 0, s>>>(X, g, b, Y, st, rows);
  return cudaGetLastError();
}

template <int DJ>
cudaError_t ln_bwd(ut_tfm* t, const float* dY, const float* X, const float* st, const float* g, const float* base,
                   float* out, float* grad_gb, long long rows, cudaStream_t s) {
  static const int nblk = (int)std::min<long long>(kLnBlocks, resident_blocks(ln_bwd_kernel<DJ>, 256));
  ln_bwd_kernel<DJ><<<nblk, 256, 0, s>>>(dY, X, st, g, base, out, t->part, rows);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = reduce(t->part, nblk, 2 * 32 * DJ, 2 * 32 * DJ, grad_gb, s);
  return e;
}

template <int DH>
cudaError_t attn_fwd(const float* QKV, const int32_t* ne, const int32_t* sel, float* P, float* O, long long n, int T,
                     int NS, int H, bool mma, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (mma && DH == 16 && T <= 16 && ((uintptr_t)QKV & 15) == 0) {
    const long long grid = att_grid(attn_fwd_mma_kernel, n * H);
    attn_fwd_mma_kernel<<<(unsigned)grid, 128, 0, s>>>(QKV, ne, sel, P, O, n, T, NS, H, 1.0f / sqrtf((float)DH));
    return cudaGetLastError();
  }
  const long long warps = (n * H + attn_pairs_per_warp(T) - 1) / attn_pairs_per_warp(T);
  attn_fwd_kernel<DH><<<blocks_for(warps * 32, 128), 128, 0, s>>>(QKV, ne, sel, P, O, n, T, NS, H,
                                                                   1.0f / sqrtf((float)DH));
  return cudaGetLastError();
}

template <int DH>
cudaError_t attn_bwd(const float* QKV, const float* P, const float* dO, float* dQKV, long long n, int T, int H,
                     bool mma, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (mma && DH == 16 && T <= 16 && ((uintptr_t)QKV & 15) == 0 && ((uintptr_t)dO & 15) == 0)
    attn_bwd_mma_kernel<<<(unsigned)att_grid(attn_bwd_mma_kernel, n * H), 128, 0, s>>>(QKV, P, dO, dQKV, n, T, H,
                                                                                       1.0f / sqrtf((float)DH));
  else
    attn_bwd_kernel<DH><<<blocks_for(n * H * 32, 128), 128, 0, s>>>(QKV, P, dO, dQKV, n, T, H, 1.0f / sqrtf((float)DH));
  return cudaGetLastError();
}

struct Call {
  const void* tok;
  const int32_t* ne;
  const float* h;
  const int32_t* sel;
  long long n;
};

template <int DJ, int DH, typename TokT>
cudaError_t forward(ut_tfm* t, const Call& c, cudaStream_t s) {
  constexpr int d = 32 * DJ;
  const long long rows = c.n * t->T, MR = t->max_rows;
  const float* w = t->prm;
  const auto& o = t->off;
  if (t->gemm_tc) {  // the weights' BF16 images for this call
    pack_images_kernel<<<dim3(blocks_for(t->img_max, 256), (unsigned)t->n_img), 256, 0, s>>>(t->prm, t->img_spec,
                                                                                            t->wimg);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
  }
  auto img = [&](int l, int which) -> const uint16_t* {
    return t->gemm_tc ? t->wimg + t->img_off[8 * l + which] : nullptr;
  };
  {
    const unsigned blocks = (unsigned)std::min<long long>((rows + 7) / 8, 152LL * 16);
    const TokT* tk = (const TokT*)c.tok;
    if (d == 32)
      embed_kernel<TokT, 1><<<blocks, 256, 0, s>>>(tk, c.ne, c.h, c.sel, w + o[0], w + o[1], t->X, c.n, t->T, t->NS);
    else if (d == 64)
      embed_kernel<TokT, 2><<<blocks, 256, 0, s>>>(tk, c.ne, c.h, c.sel, w + o[0], w + o[1], t->X, c.n, t->T, t->NS);
    else if (d == 96)
      embed_kernel<TokT, 3><<<blocks, 256, 0, s>>>(tk, c.ne, c.h, c.sel, w + o[0], w + o[1], t->X, c.n, t->T, t->NS);
    else
      embed_kernel<TokT, 4><<<blocks, 256, 0, s>>>(tk, c.ne, c.h, c.sel, w + o[0], w + o[1], t->X, c.n, t->T, t->NS);
  }
  cudaError_t e = cudaGetLastError();
  for (int l = 0; l < t->L && e == cudaSuccess; ++l) {
    const int64_t* ol = o.data() + 2 + 12 * l;
    float* Xl = t->X + l * MR * d;
    float* Xn = t->X + (l + 1) * MR * d;
    float* Y1 = t->Y1 + l * MR * d;
    float* Y2 = t->Y2 + l * MR * d;
    float* S1 = t->S1 + l * MR * 2;
    float* S2 = t->S2 + l * MR * 2;
    float* QKV = t->QKV + l * MR * 3 * d;
    float* P = t->P + (long long)l * t->cfg.max_batch * t->H * t->T * t->T;
    float* O = t->O + l * MR * d;
    float* M = t->M + l * MR * d;
    float* Z = t->Z + l * MR * 4 * d;
    float* G = t->G + l * MR * 4 * d;
    e = ln_fwd<DJ>(Xl, w + ol[T_LN1G], w + ol[T_LN1B], Y1, S1, rows, s);
    if (e != cudaSuccess) break;
    Gemm g = mk(Y1, d, w + ol[T_WQKV], d, QKV, 3 * d, rows, 3 * d, d, EPI_BIAS);
    g.bias = w + ol[T_BQKV];
    g.bimg = img(l, 0);
    g.status = t->status;
    e = gemm(0, g, s);
    if (e == cudaSuccess) e = attn_fwd<DH>(QKV, c.ne, c.sel, P, O, c.n, t->T, t->NS, t->H, t->gemm_tc != 0, s);
    if (e != cudaSuccess) break;
    g = mk(O, d, w + ol[T_WO], d, M, d, rows, d, d, EPI_BIAS_RES);
    g.bias = w + ol[T_BO];
    g.R = Xl;
    g.bimg = img(l, 1);
    g.status = t->status;
    e = gemm(0, g, s);
    if (e == cudaSuccess) e = ln_fwd<DJ>(M, w + ol[T_LN2G], w + ol[T_LN2B], Y2, S2, rows, s);
    if (e != cudaSuccess) break;
    g = mk(Y2, d, w + ol[T_W1], d, Z, 4 * d, rows, 4 * d, d, EPI_BIAS_GELU);
    g.bias = w + ol[T_B1];
    g.C2 = G;
    g.bimg = img(l, 2);
    g.status = t->status;
    e = gemm(0, g, s);
    if (e != cudaSuccess) break;
    g = mk(G, 4 * d, w + ol[T_W2], 4 * d, Xn, d, rows, d, 4 * d, EPI_BIAS_RES);
    g.bias = w + ol[T_B2];
    g.R = M;
    g.bimg = img(l, 3);
    g.status = t->status;
    e = gemm(0, g, s);
  }
  return e;
}

template <int DJ, int DH, typename TokT>
cudaError_t backward(ut_tfm* t, const Call& c, float* grad, cudaStream_t s) {
  constexpr int d = 32 * DJ;
  const long long rows = c.n * t->T, MR = t->max_rows;
  const float* w = t->prm;
  const auto& o = t->off;
  cudaError_t e = cudaSuccess;
  // input-gradient GEMM of block l with the transposed image `which` (4..7)
  auto dgemm = [&](int l, int which, Gemm g) {
    g.bimg = t->gemm_tc ? t->wimg + t->img_off[8 * l + which] : nullptr;
    g.status = t->status;
    return gemm(1, g, s);
  };
  for (int l = t->L - 1; l >= 0 && e == cudaSuccess; --l) {
    const int64_t* ol = o.data() + 2 + 12 * l;
    const float* Xl = t->X + l * MR * d;
    const float* Y1 = t->Y1 + l * MR * d;
    const float* Y2 = t->Y2 + l * MR * d;
    const float* S1 = t->S1 + l * MR * 2;
    const float* S2 = t->S2 + l * MR * 2;
    const float* QKV = t->QKV + l * MR * 3 * d;
    const float* P = t->P + (long long)l * t->cfg.max_batch * t->H * t->T * t->T;
    const float* O = t->O + l * MR * d;
    const float* M = t->M + l * MR * d;
    const float* Z = t->Z + l * MR * 4 * d;
    const float* G = t->G + l * MR * 4 * d;
    // feed-forward sub-block: X' = M + W2 gelu(W1 LN2(M) + b1) + b2
    Gemm g = mk(t->dX, d, w + ol[T_W2], 4 * d, t->dBig, 4 * d, rows, 4 * d, d, EPI_GELU_GRAD);
    g.aux = Z;
    e = dgemm(l, 7, g);
    if (e == cudaSuccess) e = wgrad(t, t->dX, d, G, 4 * d, rows, grad + ol[T_W2], grad + ol[T_B2], s);
    if (e == cudaSuccess) e = dgemm(l, 6, mk(t->dBig, 4 * d, w + ol[T_W1], d, t->dY, d, rows, d, 4 * d, EPI_STORE));
    if (e == cudaSuccess) e = wgrad(t, t->dBig, 4 * d, Y2, d, rows, grad + ol[T_W1], grad + ol[T_B1], s);
    if (e == cudaSuccess) e = ln_bwd<DJ>(t, t->dY, M, S2, w + ol[T_LN2G], t->dX, t->dM, grad + ol[T_LN2G], rows, s);
    // attention sub-block: M = X + Wo attn(LN1(X)) + bo
    if (e == cudaSuccess) e = dgemm(l, 5, mk(t->dM, d, w + ol[T_WO], d, t->dO, d, rows, d, d, EPI_STORE));
    if (e == cudaSuccess) e = wgrad(t, t->dM, d, O, d, rows, grad + ol[T_WO], grad + ol[T_BO], s);
    if (e == cudaSuccess) e = attn_bwd<DH>(QKV, P, t->dO, t->dBig, c.n, t->T, t->H, t->gemm_tc != 0, s);
    if (e == cudaSuccess) e = dgemm(l, 4, mk(t->dBig, 3 * d, w + ol[T_WQKV], d, t->dY, d, rows, d, 3 * d, EPI_STORE));
    if (e == cudaSuccess) e = wgrad(t, t->dBig, 3 * d, Y1, d, rows, grad + ol[T_WQKV], grad + ol[T_BQKV], s);
    if (e == cudaSuccess) e = ln_bwd<DJ>(t, t->dY, Xl, S1, w + ol[T_LN1G], t->dM, t->dX, grad + ol[T_LN1G], rows, s);
  }
  if (e != cudaSuccess) return e;
  embed_grad_kernel<TokT, DJ><<<kRowBlocks, 256, 0, s>>>((const TokT*)c.tok, c.ne, c.sel, t->dX, t->part, c.n, t->T,
                                                         t->NS);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = reduce(t->part, kRowWarps, 9 * d, 9 * d, grad + o[0], s);
  return e;
}

// mode 0: forward (out, h_out); 1: PPO actor loss + gradient; 2: value loss +
// gradient.
template <int DJ, int DH, typename TokT>
cudaError_t run(ut_tfm* t, const Call& c, int mode, const HeadArgs& ha_in, float* grad, cudaStream_t s) {
  constexpr int d = 32 * DJ;
  cudaError_t e = forward<DJ, DH, TokT>(t, c, s);
  if (e != cudaSuccess) return e;
  const auto& o = t->off;
  const int idx = 2 + 12 * t->L;
  HeadArgs ha = ha_in;
  ha.XL = t->X + (long long)t->L * t->max_rows * d;
  ha.n = c.n;
  ha.T = t->T;
  ha.n_out = t->n_out;
  ha.mode = mode;
  ha.lnf_g = t->prm + o[idx];
  ha.lnf_b = t->prm + o[idx + 1];
  ha.Wh = t->prm + o[idx + 2];
  ha.bh = t->prm + o[idx + 3];
  ha.sel = c.sel;
  ha.inv_n = 1.0f / (float)c.n;
  ha.dXL = t->dX;
  ha.part = t->part;
  ha.spart = t->spart;
  if (t->n_out == 1)
    head_kernel<DJ, 1><<<kRowBlocks, 256, 0, s>>>(ha);
  else
    head_kernel<DJ, 16><<<kRowBlocks, 256, 0, s>>>(ha);
  e = cudaGetLastError();
  if (e != cudaSuccess || mode == 0) return e;
  const long long plen = 2 * d + (long long)t->n_out * d + t->n_out;
  e = reduce(t->part, kRowWarps, plen, plen, grad + o[idx], s);
  if (e != cudaSuccess) return e;
  reduce_stats_kernel<<<1, 256, 0, s>>>(t->spart, kRowWarps, 1.0 / (double)c.n, t->stats_d);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return backward<DJ, DH, TokT>(t, c, grad, s);
}

template <int DJ, int DH>
cudaError_t run_tok(ut_tfm* t, const Call& c, int mode, const HeadArgs& ha, float* grad, cudaStream_t s) {
  return t->cfg.tokens_bf16 ? run<DJ, DH, __nv_bfloat16>(t, c, mode, ha, grad, s)
                            : run<DJ, DH, float>(t, c, mode, ha, grad, s);
}

template <int DJ>
cudaError_t run_dh(ut_tfm* t, const Call& c, int mode, const HeadArgs& ha, float* grad, cudaStream_t s) {
  switch (t->dh) {
    case 8: return run_tok<DJ, 8>(t, c, mode, ha, grad, s);
    case 16: return run_tok<DJ, 16>(t, c, mode, ha, grad, s);
    default: return run_tok<DJ, 32>(t, c, mode, ha, grad, s);
  }
}

cudaError_t dispatch(ut_tfm* t, const Call& c, int mode, const HeadArgs& ha, float* grad) {
  switch (t->d) {
    case 32: return run_dh<1>(t, c, mode, ha, grad, t->stream);
    case 64: return run_dh<2>(t, c, mode, ha, grad, t->stream);
    case 96: return run_dh<3>(t, c, mode, ha, grad, t->stream);
    default: return run_dh<4>(t, c, mode, ha, grad, t->stream);
  }
}

ut_status fail(ut_tfm* t, ut_status st, const std::string& msg) {
  t->err = msg;
  return st;
}

void* dalloc(ut_tfm* t, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
  t->allocs.push_back(p);
  return p;
}

bool call_ok(const ut_tfm* t, const void* tok, const int32_t* ne, const float* h, int64_t n) {
  return tok && ne && h && n >= 1 && n <= t->cfg.max_batch;
}

}  // namespace
}  // namespace tfm
}  // namespace ut

using namespace ut::tfm;

namespace ut {

TfmInfo tfm_info(const ut_tfm* t) {
  return TfmInfo{t->d, t->L, t->H, t->n_out, t->NS, t->cfg.tokens_bf16, (long long)t->cfg.max_batch};
}

cudaError_t tfm_forward_on(ut_tfm* t, const void* tokens, const int32_t* n_ent, const float* h, long long n,
                           float* out, float* h_out, cudaStream_t s) {
  HeadArgs ha;
  std::memset(&ha, 0, sizeof(ha));
  ha.out = out;
  ha.h_out = h_out;
  const cudaStream_t own = t->stream;
  t->stream = s;
  const cudaError_t e = dispatch(t, Call{tokens, n_ent, h, nullptr, n}, 0, ha, nullptr);
  t->stream = own;
  return e;
}

}  // namespace ut

extern "C" int64_t tfm_param_count(const ut_tfm_config* cfg) {
  if (!valid_config(cfg)) return -1;
  return offsets(cfg->d_model, cfg->n_layers, cfg->n_out).back();
}

extern "C" ut_status tfm_create(const ut_tfm_config* cfg, const float* params_host, int64_t n_params,
                                void* cuda_stream, ut_tfm** out) {
  if (!out) return UT_ERR_INVALID;
  *out = nullptr;
  if (!valid_config(cfg) || !params_host || n_params != tfm_param_count(cfg)) return UT_ERR_INVALID;
  ut_tfm* t = new ut_tfm();
  t->cfg = *cfg;
  t->stream = (cudaStream_t)cuda_stream;
  t->d = cfg->d_model;
  t->L = cfg->n_layers;
  t->H = cfg->n_heads;
  t->dh = t->d / t->H;
  t->n_out = cfg->n_out;
  t->NS = cfg->n_slots;
  t->T = 1 + cfg->n_slots;
  t->f = 4 * t->d;
  t->n_params = n_params;
  t->off = offsets(t->d, t->L, t->n_out);
  t->max_rows = cfg->max_batch * t->T;
  const size_t R = (size_t)t->max_rows, d = (size_t)t->d, L = (size_t)t->L;
  const size_t Pn = (size_t)cfg->max_batch * t->H * t->T * t->T;
  size_t part = (size_t)128 * 4 * d * d;
  part = std::max(part, (size_t)256 * 4 * d);
  part = std::max(part, (size_t)kRowWarps * (2 * d + (size_t)t->n_out * d + t->n_out));
  part = std::max(part, (size_t)kRowWarps * 9 * d);
  part = std::max(part, (size_t)kLnBlocks * 2 * d);
  part = std::max(part, (size_t)kTcSplitsMax * (4 * d * d + 4 * d));  // tensor-core weight- and bias-gradient slabs
  bool ok = true;
  auto A = [&](size_t n) -> float* {
    float* p = (float*)dalloc(t, n * 4);
    ok = ok && p;
    return p;
  };
  t->prm = A(n_params);
  t->am = A(n_params);
  t->av = A(n_params);
  t->X = A((L + 1) * R * d);
  t->Y1 = A(L * R * d);
  t->Y2 = A(L * R * d);
  t->S1 = A(L * R * 2);
  t->S2 = A(L * R * 2);
  t->QKV = A(L * R * 3 * d);
  t->P = A(L * Pn);
  t->O = A(L * R * d);
  t->M = A(L * R * d);
  t->Z = A(L * R * 4 * d);
  t->G = A(L * R * 4 * d);
  t->dX = A(R * d);
  t->dM = A(R * d);
  t->dY = A(R * d);
  t->dO = A(R * d);
  t->dBig = A(R * 4 * d);
  t->part = A(part);
  t->spart = (double*)dalloc(t, (size_t)kRowWarps * 4 * 8);
  t->stats_d = (double*)dalloc(t, 4 * 8);
  ok = ok && t->spart && t->stats_d;
  // weight images: per block, B of the forward for Wqkv [3d][d], Wo [d][d],
  // W1 [4d][d], W2 [d][4d], then B of the input gradient (their transposes)
  std::vector<int64_t> spec;
  int64_t img_total = 0;
  t->img_max = 0;
  for (int l = 0; l < t->L; ++l) {
    const int64_t* ol = t->off.data() + 2 + 12 * l;
    const int64_t woff[4] = {ol[T_WQKV], ol[T_WO], ol[T_W1], ol[T_W2]};
    const int rows_w[4] = {3 * t->d, t->d, 4 * t->d, t->d}, cols_w[4] = {t->d, t->d, t->d, 4 * t->d};
    for (int tr = 0; tr < 2; ++tr)
      for (int k = 0; k < 4; ++k) {
        const int R = tr ? cols_w[k] : rows_w[k], C = tr ? rows_w[k] : cols_w[k];
        // each 256-row block holds C columns of 256 rows (the last block padded)
        const int64_t n = (int64_t)((R + kTcMaxN - 1) / kTcMaxN) * kTcMaxN * C;
        t->img_off.push_back(img_total);
        spec.insert(spec.end(), {woff[k], (int64_t)R, (int64_t)C, (int64_t)tr, img_total});
        img_total += n;
        t->img_max = std::max(t->img_max, R * C);
      }
  }
  t->n_img = 8 * t->L;
  t->wimg = (uint16_t*)dalloc(t, (size_t)img_total * 2);
  t->img_spec = (int64_t*)dalloc(t, spec.size() * 8);
  t->status = (int*)dalloc(t, 4);
  ok = ok && t->wimg && t->img_spec && t->status;
  if (!ok) {
    tfm_destroy(t);
    return UT_ERR_NOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(t->prm, params_host, (size_t)n_params * 4, cudaMemcpyHostToDevice, t->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(t->img_spec, spec.data(), spec.size() * 8, cudaMemcpyHostToDevice, t->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->wimg, 0, (size_t)img_total * 2, t->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->status, 0, 4, t->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->am, 0, (size_t)n_params * 4, t->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->av, 0, (size_t)n_params * 4, t->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) {
    tfm_destroy(t);
    return UT_ERR_CUDA;
  }
  *out = t;
  return UT_OK;
}

extern "C" void tfm_destroy(ut_tfm* t) {
  if (!t) return;
  if (t->stream) cudaStreamSynchronize(t->stream);
  for (void* p : t->allocs) cudaFree(p);
  delete t;
}

extern "C" const char* tfm_last_error(const ut_tfm* t) { return t ? t->err.c_str() : "null handle"; }

extern "C" ut_status tfm_params(ut_tfm* t, float** params_dev) {
  if (!t || !params_dev) return UT_ERR_INVALID;
  *params_dev = t->prm;
  return UT_OK;
}

extern "C" ut_status tfm_forward(ut_tfm* t, const void* tokens_dev, const int32_t* n_ent_dev, const float* h_dev,
                                 const int32_t* sel_dev, int64_t n, float* out_dev, float* h_out_dev) {
  if (!t) return UT_ERR_INVALID;
  if (!call_ok(t, tokens_dev, n_ent_dev, h_dev, n) || !out_dev || (h_out_dev == h_dev && sel_dev))
    return fail(t, UT_ERR_INVALID, "tfm_forward: invalid arguments");
  HeadArgs ha;
  std::memset(&ha, 0, sizeof(ha));
  ha.out = out_dev;
  ha.h_out = h_out_dev;
  const cudaError_t e = dispatch(t, Call{tokens_dev, n_ent_dev, h_dev, sel_dev, n}, 0, ha, nullptr);
  return e == cudaSuccess ? UT_OK : fail(t, UT_ERR_CUDA, std::string("tfm_forward: ") + cudaGetErrorString(e));
}

static ut_status finish_stats(ut_tfm* t, double* stats_host, const char* name) {
  if (!stats_host) return UT_OK;
  int status = 0;
  cudaError_t e = cudaMemcpyAsync(stats_host, t->stats_d, 4 * 8, cudaMemcpyDeviceToHost, t->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, t->status, 4, cudaMemcpyDeviceToHost, t->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) return fail(t, UT_ERR_CUDA, std::string(name) + ": " + cudaGetErrorString(e));
  if (status == 2) return fail(t, UT_ERR_TIMEOUT, std::string(name) + ": a bounded tensor-core wait gave up");
  return UT_OK;
}

extern "C" ut_status tfm_set_gemm_path(ut_tfm* t, int32_t tensor_cores) {
  if (!t || (tensor_cores != 0 && tensor_cores != 1)) return UT_ERR_INVALID;
  t->gemm_tc = tensor_cores;
  return UT_OK;
}

extern "C" ut_status tfm_ppo_actor_grad(ut_tfm* t, const void* tokens_dev, const int32_t* n_ent_dev,
                                        const float* h_dev, const int32_t* sel_dev, int64_t n,
                                        const int32_t* actions_dev, const float* logp_old_dev, const float* adv_dev,
                                        float clip_eps, float ent_coef, float* grad_dev, double* stats_host) {
  if (!t) return UT_ERR_INVALID;
  if (!call_ok(t, tokens_dev, n_ent_dev, h_dev, n) || !actions_dev || !logp_old_dev || !adv_dev || !grad_dev ||
      !(clip_eps > 0.0f) || !(ent_coef >= 0.0f) || t->n_out < 2)
    return fail(t, UT_ERR_INVALID, "tfm_ppo_actor_grad: invalid arguments");
  HeadArgs ha;
  std::memset(&ha, 0, sizeof(ha));
  ha.actions = actions_dev;
  ha.logp_old = logp_old_dev;
  ha.adv = adv_dev;
  ha.clip_eps = clip_eps;
  ha.ent_coef = ent_coef;
  const cudaError_t e = dispatch(t, Call{tokens_dev, n_ent_dev, h_dev, sel_dev, n}, 1, ha, grad_dev);
  if (e != cudaSuccess) return fail(t, UT_ERR_CUDA, std::string("tfm_ppo_actor_grad: ") + cudaGetErrorString(e));
  return finish_stats(t, stats_host, "tfm_ppo_actor_grad");
}

extern "C" ut_status tfm_value_grad(ut_tfm* t, const void* tokens_dev, const int32_t* n_ent_dev, const float* h_dev,
                                    const int32_t* sel_dev, int64_t n, const float* returns_dev, float* grad_dev,
                                    double* stats_host) {
  if (!t) return UT_ERR_INVALID;
  if (!call_ok(t, tokens_dev, n_ent_dev, h_dev, n) || !returns_dev || !grad_dev || t->n_out != 1)
    return fail(t, UT_ERR_INVALID, "tfm_value_grad: invalid arguments");
  HeadArgs ha;
  std::memset(&ha, 0, sizeof(ha));
  ha.ret = returns_dev;
  const cudaError_t e = dispatch(t, Call{tokens_dev, n_ent_dev, h_dev, sel_dev, n}, 2, ha, grad_dev);
  if (e != cudaSuccess) return fail(t, UT_ERR_CUDA, std::string("tfm_value_grad: ") + cudaGetErrorString(e));
  return finish_stats(t, stats_host, "tfm_value_grad");
}

extern "C" ut_status tfm_adam_step(ut_tfm* t, const float* grad_dev, float lr, float beta1, float beta2, float eps) {
  if (!t) return UT_ERR_INVALID;
  if (!grad_dev || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
      !(eps > 0.0f))
    return fail(t, UT_ERR_INVALID, "tfm_adam_step: invalid arguments");
  t->adam_t += 1;
  const float bc1 = (float)(1.0 - std::pow((double)beta1, t->adam_t));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, t->adam_t));
  adam_kernel<<<blocks_for(t->n_params, 256), 256, 0, t->stream>>>(t->prm, t->am, t->av, grad_dev, t->n_params, lr,
                                                                   beta1, beta2, eps, bc1, bc2);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? UT_OK : fail(t, UT_ERR_CUDA, std::string("tfm_adam_step: ") + cudaGetErrorString(e));
}

extern "C" ut_status tfm_sync_policy(ut_tfm* t, ut_env* env) {
  if (!t || !env) return UT_ERR_INVALID;
  const ut_config& c = env->cfg;
  if (c.d_model != t->d || c.n_layers != t->L || c.n_heads != t->H || c.n_actions != t->n_out)
    return fail(t, UT_ERR_INVALID, "tfm_sync_policy: the env's transformer agent has another configuration");
  std::vector<float> host((size_t)t->n_params);
  cudaError_t e = cudaMemcpyAsync(host.data(), t->prm, host.size() * 4, cudaMemcpyDeviceToHost, t->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) return fail(t, UT_ERR_CUDA, std::string("tfm_sync_policy: ") + cudaGetErrorString(e));
  const ut_status st = env_set_policy(env, host.data(), t->n_params);
  if (st != UT_OK) t->err = std::string("tfm_sync_policy: ") + env_last_error(env);
  return st;
}

extern "C" ut_status ppo_gae(const float* reward_dev, const float* value_dev, const int32_t* done_dev, int32_t T,
                             int64_t E, float gamma, float lam, float* adv_dev, float* ret_dev,
                             const int32_t* agent_env_dev, int64_t NA, float* adv_agent_dev, void* cuda_stream) {
  if (!reward_dev || !value_dev || !done_dev || !adv_dev || !ret_dev || T < 1 || E < 1 || !(gamma >= 0.0f) ||
      !(gamma <= 1.0f) || !(lam >= 0.0f) || !(lam <= 1.0f))
    return UT_ERR_INVALID;
  if ((agent_env_dev == nullptr) != (adv_agent_dev == nullptr) || (adv_agent_dev && NA < 1)) return UT_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  gae_kernel<<<blocks_for(E, 256), 256, 0, s>>>(reward_dev, value_dev, done_dev, T, E, gamma, lam, adv_dev, ret_dev);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && adv_agent_dev) {
    gae_agents_kernel<<<blocks_for((long long)T * NA, 256), 256, 0, s>>>(adv_dev, agent_env_dev, T, E, NA,
                                                                        adv_agent_dev);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? UT_OK : UT_ERR_CUDA;
}
