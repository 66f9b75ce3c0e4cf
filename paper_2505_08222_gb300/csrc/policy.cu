// Transformer agent forward (Sec. III-B.1, Fig. 3) on the tensor cores.
//
// Each agent's tokens are its recurrent embedding h followed by its entity
// vectors (self, teammates, targets; observation tokens of Sec. III-A.2).
// A 128-row tile holds apt = 128 / R agents of R = 1 + S tokens (S entity
// slots): for R <= 16 agent a's tokens in rows R a .. R a + R - 1, recurrent
// token first; for R = 17 the entity tokens of agent a in rows S a ..
// S a + S - 1 and the recurrent tokens of all agents after them (rows
// S apt + a), so that each agent's entity queries fill one 16-row MMA tile.
// One CTA of 128 P threads owns a
// tile (P = 2 column parts for d = 64, 4 for d = 128): thread t works on row
// t % 128 and on column part t / 128 of that row, keeping its part of the
// residual stream X in registers from start to end:
//
//   X = [h ; W_emb tok + b_emb]                         (CUDA cores, FP32)
//   per block l:   Y = LN1(X) -> BF16 operand A
//                  Q, K, V = Y Wq^T, Y Wk^T, Y Wv^T      (three tcgen05.mma
//                      groups issued together, FP32 in TMEM)
//                  O = softmax(Q K^T / 4) V per head, within the agent's
//                      valid tokens                      (warp-level MMAs, a
//                      warp per (agent, head); with 17 tokens the recurrent
//                      queries per (head, 4 agents))
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
// layout (tc.cuh); each weight image is one contiguous bulk copy, streamed
// through a three-slot shared-memory ring by the bulk-copy engine while the
// CUDA cores work on the previous stage.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/utrack.h"
#include "policy.cuh"
#include "runtime.cuh"
#include "gelu.cuh"
#include "f32x2.cuh"
#include "tc.cuh"

namespace ut {
namespace {

constexpr int kSlots = 3;                                  // weight ring depth
static_assert(UT_MAX_AGENTS + UT_MAX_TARGETS <= 16, "an agent's entity queries fit one 16-row MMA tile");
constexpr float kLnEps = 1e-5f;
constexpr uint32_t kPolls = 1u << 22;                      // bounded mbarrier waits

template <int D>
struct Geo {
  static constexpr int H = D / 16;                 // heads of width 16
  static constexpr int NS = D == 64 ? 2 : 4;       // column parts per row
  static constexpr int THREADS = 128 * NS;
  static constexpr int COLS = D / NS;              // columns per thread
  static constexpr int HCOLS = 128 / NS;           // hidden units per thread in an FFN chunk
  static constexpr int NC = (4 * D) / 128;         // FFN hidden chunks of 128
  static constexpr int NSTG = 4 + 2 * NC;          // weight images per layer
  static constexpr int VEC = 13 * D;               // per-layer vector floats
  // packed weight images of one layer (bytes)
  static constexpr size_t IMG_DD = (size_t)D * D * 2;
  static constexpr size_t IMG_W1 = (size_t)128 * D * 2;
  static constexpr size_t IMG_W2 = (size_t)D * 128 * 2;
  // Wq, Wk, Wv, Wo at i * IMG_DD (i = 0 .. 3), then the FFN chunks
  static constexpr size_t OFF_W1 = 4 * IMG_DD;
  static constexpr size_t OFF_W2 = OFF_W1 + NC * IMG_W1;
  static constexpr size_t LAYER_BYTES = OFF_W2 + NC * IMG_W2;
  static constexpr size_t SLOT = IMG_W1 > IMG_DD ? IMG_W1 : IMG_DD;
  // shared memory
  static constexpr size_t A_OFF = 0;
  static constexpr size_t A_BYTES = (size_t)128 * D * 2;
  static constexpr size_t RING_OFF = A_OFF + A_BYTES;
  static constexpr size_t KV_OFF = RING_OFF + kSlots * SLOT;
  static constexpr size_t KV_BYTES = (size_t)2 * 128 * D * 2;   // K, V as K-major images
  static constexpr size_t VEC_OFF = KV_OFF + KV_BYTES;
  static constexpr size_t STAT_OFF = VEC_OFF + (size_t)2 * VEC * 4;
  static constexpr size_t SMEM = STAT_OFF + (size_t)NS * 128 * 8;
  // tensor memory columns
  static constexpr uint32_t TMEM_COLS = D == 64 ? 256 : 512;
  static constexpr uint32_t COL_Q = 0, COL_K = D, COL_V = 2 * D;
  static constexpr uint32_t COL_S = D;             // O-projection / W1 chunk (after K, V are drained)
  static constexpr uint32_t COL_ACC = 0;           // FFN output (after Q is consumed)
  // pipelined FFN (d = 128): the W1 MMA of chunk c + 1 runs while the CUDA
  // cores take GELU of chunk c, so the hidden chunk has two TMEM column
  // blocks (COL_S, COL_S + 128) and two BF16 images in the K/V region
  static constexpr bool PIPE = D == 128;
  // LayerNorm outputs (the A operand of the Q/K/V and W1 MMAs) in TMEM, two
  // BF16 per 32-bit column: D / 2 columns after V and after the hidden blocks
  static constexpr uint32_t COL_A = (3 * D > (int)COL_S + (PIPE ? 256 : 128)) ? 3 * D : COL_S + (PIPE ? 256 : 128);
  static_assert(COL_A + D / 2 <= TMEM_COLS, "TMEM plan: LayerNorm operand");
  static_assert(KV_BYTES >= (size_t)128 * 128 * 2, "hidden chunk must fit in the K/V region");
  static_assert(COL_S + 128 <= TMEM_COLS && 3 * D <= (int)TMEM_COLS, "TMEM plan");
  static_assert(!PIPE || (NC >= 2 && COL_S + 256 <= TMEM_COLS && KV_BYTES >= (size_t)2 * 128 * 128 * 2),
                "pipelined FFN plan");
  static_assert(SLOT % 16 == 0 && IMG_W2 <= SLOT, "bulk copies are 16-byte multiples");
  static_assert(VEC % 4 == 0 && VEC_OFF % 16 == 0, "16-byte copies of the per-layer vectors");
};

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

__device__ __forceinline__ uint32_t pack_bf2(float a, float b) { return bf16x2_bits(a, b); }

// Element-wise epilogue steps on packed FP32 pairs (each lane rounded like
// the scalar operation): v = (v + b) s over N values; v += b; x += v + b.
template <int N>
__device__ __forceinline__ void bias_scale2(float* v, const float* b, float s) {
  const unsigned long long S = f2pk(s, s);
#pragma unroll
  for (int i = 0; i < N; i += 2) f2upk(f2mul(f2add(f2pk(v[i], v[i + 1]), f2pk(b[i], b[i + 1])), S), v[i], v[i + 1]);
}
template <int N>
__device__ __forceinline__ void bias_add2(float* v, const float* b) {
#pragma unroll
  for (int i = 0; i < N; i += 2) f2upk(f2add(f2pk(v[i], v[i + 1]), f2pk(b[i], b[i + 1])), v[i], v[i + 1]);
}
template <int N>
__device__ __forceinline__ void residual_add2(float* x, const float* v, const float* b) {
#pragma unroll
  for (int i = 0; i < N; i += 2)
    f2upk(f2add(f2pk(x[i], x[i + 1]), f2add(f2pk(v[i], v[i + 1]), f2pk(b[i], b[i + 1]))), x[i], x[i + 1]);
}

// Store 8 consecutive K values of `row` into a K-major operand image.
__device__ __forceinline__ void store8(unsigned char* img, int row, int k0, int rows, const float* v) {
  uint4 q;
  q.x = pack_bf2(v[0], v[1]);
  q.y = pack_bf2(v[2], v[3]);
  q.z = pack_bf2(v[4], v[5]);
  q.w = pack_bf2(v[6], v[7]);
  *reinterpret_cast<uint4*>(img + tc::kmajor_offset(row, k0, rows)) = q;
}

// Weight image of global stage s (layer-major; within a layer: Wq, Wk, Wv,
// Wo, then W1 chunk c and W2 chunk c for c = 0 .. NC-1).
template <int D>
__device__ __forceinline__ void stage_image(int s, size_t& off, uint32_t& bytes) {
  using G = Geo<D>;
  const int l = s / G::NSTG, i = s - l * G::NSTG;
  if (i < 4) {
    off = (size_t)i * G::IMG_DD;
    bytes = (uint32_t)G::IMG_DD;
  } else {
    // FFN chunks in the order the MMAs consume them: W1_0, W2_0, W1_1, ...;
    // with the pipelined FFN (G::PIPE) W1 of the next chunk comes before W2
    // of the current one: W1_0, W1_1, W2_0, W1_2, W2_1, ..., W2_{NC-1}
    const int j = i - 4;
    bool w1;
    int c;
    if (!G::PIPE) {
      w1 = (j & 1) == 0;
      c = j >> 1;
    } else if (j == 0) {
      w1 = true;
      c = 0;
    } else if (j == 2 * G::NC - 1) {
      w1 = false;
      c = G::NC - 1;
    } else {
      w1 = (j & 1) == 1;
      c = w1 ? (j + 1) >> 1 : (j - 2) >> 1;
    }
    if (w1) {
      off = G::OFF_W1 + (size_t)c * G::IMG_W1;
      bytes = (uint32_t)G::IMG_W1;
    } else {
      off = G::OFF_W2 + (size_t)c * G::IMG_W2;
      bytes = (uint32_t)G::IMG_W2;
    }
  }
  off += (size_t)l * G::LAYER_BYTES;
}

// Loader state, meaningful in thread 0 (the only thread that issues copies
// and MMAs): stage `next` is the next image to fetch; slot s % kSlots may be
// refilled once the MMA that read stage s - kSlots has completed.
struct Loader {
  int next, done, total;
};

template <int D>
__device__ __forceinline__ void pump(Loader& ld, const unsigned char* __restrict__ wimg, unsigned char* ring,
                                     uint64_t* full) {
  while (ld.next < ld.total && ld.next < ld.done + kSlots) {
    size_t off;
    uint32_t bytes;
    stage_image<D>(ld.next, off, bytes);
    const int slot = ld.next % kSlots;
    tc::mbar_expect_tx(&full[slot], bytes);
    tc::bulk_g2s(ring + slot * Geo<D>::SLOT, wimg + off, bytes, &full[slot]);
    ++ld.next;
  }
}

// acc[128 x N] (+)= A[128 x K] * B[N x K]^T, issued by the calling thread.
__device__ __forceinline__ void issue_mma(uint32_t d_tmem, uint32_t a_addr, uint32_t b_addr, int N, int K,
                                          bool accumulate) {
  const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)N);
  for (int k = 0; k < K / 16; ++k) {
    const uint64_t ad = tc::smem_desc(a_addr + k * 2 * 128 * 16, 128 * 16, 128);
    const uint64_t bd = tc::smem_desc(b_addr + k * 2 * N * 16, N * 16, 128);
    tc::mma_bf16(d_tmem, ad, bd, idesc, (accumulate || k > 0) ? 1u : 0u);
  }
}

// acc[128 x N] (+)= A[128 x K] * B[N x K]^T with A in TMEM (columns a_tmem ..,
// K / 2 of them), issued by the calling thread.
__device__ __forceinline__ void issue_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint32_t b_addr, int N, int K,
                                             bool accumulate) {
  const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)N);
  for (int k = 0; k < K / 16; ++k) {
    const uint64_t bd = tc::smem_desc(b_addr + k * 2 * N * 16, N * 16, 128);
    tc::mma_bf16_ts(d_tmem, a_tmem + (uint32_t)(k * 8), bd, idesc, (accumulate || k > 0) ? 1u : 0u);
  }
}

// 16-byte asynchronous global -> shared copy; commit of the calling thread's
// copies as a group, and the wait for all of them.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_addr(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Make every thread's shared-memory operand writes (and TMEM reads) visible
// before thread 0 issues the next MMA group.
__device__ __forceinline__ void publish() {
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

// The per-row epilogue items of this thread: (part p, k) is the 16 columns
// p * W + 16 k .. + 15 of its row (W = the part's width, NIT = W / 16); f
// takes one item, f2 the pair k, k + 1 (the thread's own items).  Warp 0
// holds the thread that issues the MMAs, which blocks while the tensor pipe
// takes them, so with four column parts it takes no items: its items (part 0)
// go round-robin, from `rot` on, to the other warps of its TMEM lane quarter
// (4, 8, 12), which run on the same SM sub-partition; each sub-partition keeps
// the same work.
template <int NP, int NIT, typename F, typename F2>
__device__ __forceinline__ void for_items(int warp, int part, int rot, F&& f, F2&& f2) {
  static_assert(NIT % 2 == 0, "own items in pairs");
  constexpr bool kOffload = NP >= 4;  // (with one helper warp, its doubled items cost more than the issue)
  if (!kOffload || warp != 0) {  // own items two at a time
#pragma unroll 1
    for (int k = 0; k < NIT; k += 2) f2(part, k);
  }
  if (kOffload && warp != 0 && (warp & 3) == 0) {
    const int h = warp >> 2;  // 1 .. NP - 1
#pragma unroll 1
    for (int k = 0; k < NIT; ++k)
      if (1 + (k + rot) % (NP - 1) == h) f(0, k);
  }
}

// LayerNorm statistics of a row whose NS column parts live in NS threads
// (t, t + 128, ...): each part's mean and centred sum of squares are combined
// (pairwise update of Chan et al. for equal counts).  Contains a block
// barrier.
template <int D>
__device__ __forceinline__ void ln_part_stats(const float (&x)[Geo<D>::COLS], float2* sStat, int row, int part,
                                              float& mean_out, float& inv_out) {
  constexpr int NS = Geo<D>::NS, COLS = Geo<D>::COLS;
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < COLS; ++c) s += x[c];
  const float m = s * (1.0f / COLS);
  float q = 0.0f;
#pragma unroll
  for (int c = 0; c < COLS; ++c) {
    const float t = x[c] - m;
    q = fmaf(t, t, q);
  }
  sStat[part * 128 + row] = make_float2(m, q);
  __syncthreads();
  float2 st[NS];
  float mean = 0.0f;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    st[k] = sStat[k * 128 + row];
    mean += st[k].x;
  }
  mean *= (1.0f / NS);
  float m2 = 0.0f, dev = 0.0f;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const float dl = st[k].x - mean;
    m2 += st[k].y;
    dev = fmaf(dl, dl, dev);
  }
  m2 = fmaf(dev, (float)COLS, m2);
  mean_out = mean;
  inv_out = rsqrtf(m2 * (1.0f / D) + kLnEps);
}

// LayerNorm of the row (ln_part_stats), this thread's part of the normalised
// row written as BF16 pairs into the row's TMEM lane (the A operand of the
// next MMAs, columns taddr .. taddr + COLS / 2 - 1 of this warp's lane
// quarter), then the wait for the stores.  Contains a block barrier.
template <int D>
__device__ __forceinline__ void ln_part_to_tmem(const float (&x)[Geo<D>::COLS], const float* g, const float* b,
                                                uint32_t taddr, float2* sStat, int row, int part) {
  constexpr int COLS = Geo<D>::COLS;
  static_assert(COLS % 32 == 0, "whole 16-column TMEM stores");
  float mean, inv;
  ln_part_stats<D>(x, sStat, row, part, mean, inv);
  const int c_lo = part * COLS;
  const unsigned long long NM = f2pk(-mean, -mean), INV = f2pk(inv, inv);
#pragma unroll
  for (int c0 = 0; c0 < COLS; c0 += 32) {
    uint32_t w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {  // (x - mean) inv g + b on packed pairs
      const int c = c_lo + c0 + 2 * i;
      float y0, y1;
      f2upk(f2fma(f2mul(f2add(f2pk(x[c0 + 2 * i], x[c0 + 2 * i + 1]), NM), INV), f2pk(g[c], g[c + 1]),
                  f2pk(b[c], b[c + 1])),
            y0, y1);
      w[i] = pack_bf2(y0, y1);
    }
    tc::tmem_st16(taddr + (uint32_t)(c0 / 2), w);
  }
  tc::tmem_wait_st();
}

// 16 BF16 values (two 16-byte words) -> FP32.
__device__ __forceinline__ void load16_bf(const uint16_t* src, float (&v)[16]) {
  const uint4 a = *reinterpret_cast<const uint4*>(src);
  const uint4 b = *reinterpret_cast<const uint4*>(src + 8);
  const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    v[2 * i] = bf_lo(w[i]);
    v[2 * i + 1] = bf_hi(w[i]);
  }
}

// FP32 -> 16 BF16 values (two 16-byte words).
__device__ __forceinline__ void store16_bf(uint16_t* dst, const float (&v)[16]) {
  uint4 a, b;
  a.x = pack_bf2(v[0], v[1]);
  a.y = pack_bf2(v[2], v[3]);
  a.z = pack_bf2(v[4], v[5]);
  a.w = pack_bf2(v[6], v[7]);
  b.x = pack_bf2(v[8], v[9]);
  b.y = pack_bf2(v[10], v[11]);
  b.z = pack_bf2(v[12], v[13]);
  b.w = pack_bf2(v[14], v[15]);
  *reinterpret_cast<uint4*>(dst) = a;
  *reinterpret_cast<uint4*>(dst + 8) = b;
}

// ---- per-agent attention on warp-level MMAs ------------------------------
// Q (bias added, scaled by log2(e) / 4), K and V sit in shared memory as
// K-major BF16 operand images [128 rows x d] (tc.cuh layout: every 8 columns
// of a row form one 16-byte chunk), which ldmatrix reads directly.  One warp
// takes one (agent, head): S = Q_h K_h^T and O = softmax(S) V_h with
// mma.sync.m16n8k16 (BF16 inputs, FP32 accumulation) over the agent's rows
// padded to 16 (R <= 16) or 32; the softmax runs on the accumulator
// fragments (a row lives in the 4 lanes of a quad) and P is re-packed into A
// fragments in registers.
__device__ __forceinline__ uint32_t kmajor_row(uint32_t base, int row, int k0) {
  return base + (uint32_t)((k0 >> 3) * (128 * 16) + row * 16);
}
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
// D (16 x 8, FP32) += A (16 x 16, BF16, row) * B (16 x 8, BF16, col)
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Attention of one head within each agent's valid tokens, split row layout
// (agents of 17 tokens, one more than an MMA tile): the entity tokens of agent
// a are rows NS a .. NS a + NS - 1, its recurrent token is row RB + a
// (RB = NS apt: the recurrent rows of all agents follow the entity rows).  The valid keys of agent a are its recurrent row
// and the entity rows NS a + c, c < n_ent(a).  O overwrites Q in the query
// rows and the head's columns; the tasks of one head write disjoint rows and
// read other rows of Q only as queries whose results they discard.

// Entity queries of agent a, head h: one 16-row m-tile from NS a against the
// 16 entity-key rows from NS a and against the 8-key tile holding the
// agent's recurrent key (keys of other agents in those tiles masked).
__device__ __forceinline__ void attend_entity(uint32_t aQ, uint32_t aK, uint32_t aV, int a, int NS, int RB, int n_ent,
                                              int h) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3, mi = lane >> 3, rr = lane & 7;
  const int r0 = NS * a;
  const int kr0 = RB + (a & ~15);  // the 16 recurrent rows holding the agent's
  const bool hi = (a & 8) != 0;    // its 8-key tile within them
  const int kc = a & 7;            // its column within that tile
  uint32_t qa[4], kb[4], kr[4], vb[4], vr[4];
  ldsm_x4(kmajor_row(aQ, min(r0 + rr + (mi & 1) * 8, 127), 16 * h + (mi >> 1) * 8), qa);
  ldsm_x4(kmajor_row(aK, min(r0 + rr + (mi >> 1) * 8, 127), 16 * h + (mi & 1) * 8), kb);
  ldsm_x4(kmajor_row(aK, min(kr0 + rr + (mi >> 1) * 8, 127), 16 * h + (mi & 1) * 8), kr);
  ldsm_x4_t(kmajor_row(aV, min(r0 + rr + (mi & 1) * 8, 127), 16 * h + (mi >> 1) * 8), vb);
  ldsm_x4_t(kmajor_row(aV, min(kr0 + rr + (mi & 1) * 8, 127), 16 * h + (mi >> 1) * 8), vr);
  float s1[2][4], s2[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    s1[0][i] = 0.0f;
    s1[1][i] = 0.0f;
    s2[i] = 0.0f;
  }
  mma16816(s1[0], qa, kb[0], kb[1]);
  mma16816(s1[1], qa, kb[2], kb[3]);
  mma16816(s2, qa, hi ? kr[2] : kr[0], hi ? kr[3] : kr[1]);
  // softmax along each query row (base-2: Q carries the log2(e) factor);
  // the recurrent key is valid in every row, so each row max is finite
  float inv[2];
#pragma unroll
  for (int hr = 0; hr < 2; ++hr) {
    float mx = -INFINITY;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
#pragma unroll
      for (int n = 0; n < 2; ++n) {
        const float v = 8 * n + 2 * tig + j < n_ent ? s1[n][2 * hr + j] : -INFINITY;
        s1[n][2 * hr + j] = v;
        mx = fmaxf(mx, v);
      }
      const float v = 2 * tig + j == kc ? s2[2 * hr + j] : -INFINITY;
      s2[2 * hr + j] = v;
      mx = fmaxf(mx, v);
    }
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    float sum = 0.0f;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
#pragma unroll
      for (int n = 0; n < 2; ++n) {
        const float e = ex2_approx(s1[n][2 * hr + j] - mx);
        s1[n][2 * hr + j] = e;
        sum += e;
      }
      const float e = ex2_approx(s2[2 * hr + j] - mx);
      s2[2 * hr + j] = e;
      sum += e;
    }
    sum += __shfl_xor_sync(0xffffffffu, sum, 1);
    sum += __shfl_xor_sync(0xffffffffu, sum, 2);
    inv[hr] = 1.0f / sum;
  }
  // O = P V over the 16 entity keys, then over the 16 recurrent keys (P is
  // zero there but in the agent's column)
  float o[2][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    o[0][i] = 0.0f;
    o[1][i] = 0.0f;
  }
  const uint32_t pa[4] = {pack_bf2(s1[0][0], s1[0][1]), pack_bf2(s1[0][2], s1[0][3]), pack_bf2(s1[1][0], s1[1][1]),
                          pack_bf2(s1[1][2], s1[1][3])};
  mma16816(o[0], pa, vb[0], vb[1]);
  mma16816(o[1], pa, vb[2], vb[3]);
  const uint32_t p01 = pack_bf2(s2[0], s2[1]), p23 = pack_bf2(s2[2], s2[3]);
  const uint32_t pb[4] = {hi ? 0u : p01, hi ? 0u : p23, hi ? p01 : 0u, hi ? p23 : 0u};
  mma16816(o[0], pb, vr[0], vr[1]);
  mma16816(o[1], pb, vr[2], vr[3]);
  __syncwarp();
  // normalised O into the agent's entity rows (other rows of the m-tile
  // belong to the next agent or to the recurrent block)
#pragma unroll
  for (int hr = 0; hr < 2; ++hr) {
    const int rl = g + 8 * hr;
    if (rl < NS) {
#pragma unroll
      for (int dn = 0; dn < 2; ++dn) {
        const int k = 16 * h + 8 * dn + 2 * tig;
        const uint32_t w = pack_bf2(o[dn][2 * hr] * inv[hr], o[dn][2 * hr + 1] * inv[hr]);
        asm volatile("st.shared.b32 [%0], %1;" ::"r"(kmajor_row(aQ, r0 + rl, k) + (uint32_t)((k & 7) * 2)), "r"(w)
                     : "memory");
      }
    }
  }
}

// Recurrent queries of agents a0 .. a0 + na - 1 (na <= 4), head h (all within
// one block of 16 recurrent rows): the m-tile is that block of Q rows; each
// agent's 16 entity-key rows give a 16 x 16 score tile of which only the
// agent's own row is kept, and the block's 16 recurrent keys give one more
// tile of which only the diagonal is kept.  O = P V accumulates one product
// per agent (P nonzero in the agent's row only) plus the diagonal one.
__device__ __forceinline__ void attend_recurrent(uint32_t aQ, uint32_t aK, uint32_t aV, int a0, int na, int NS,
                                                 int RB, const int* nent, int h) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3, mi = lane >> 3, rr = lane & 7;
  const int base = a0 & ~15, rb16 = RB + base;
  uint32_t qa[4], kr[4], vr[4];
  ldsm_x4(kmajor_row(aQ, min(rb16 + rr + (mi & 1) * 8, 127), 16 * h + (mi >> 1) * 8), qa);
  ldsm_x4(kmajor_row(aK, min(rb16 + rr + (mi >> 1) * 8, 127), 16 * h + (mi & 1) * 8), kr);
  ldsm_x4_t(kmajor_row(aV, min(rb16 + rr + (mi & 1) * 8, 127), 16 * h + (mi >> 1) * 8), vr);
  // this thread's rows g + 8 hr are the recurrent rows of agents base + g + 8 hr
  bool mine[2];
  int ne[2];
#pragma unroll
  for (int hr = 0; hr < 2; ++hr) {
    const int a = base + g + 8 * hr;
    mine[hr] = a >= a0 && a < a0 + na;
    ne[hr] = mine[hr] ? nent[a] : 0;
  }
  // e[hr][2 n + j]: entity key 8 n + 2 tig + j of row hr's agent; er[hr]: its
  // recurrent key (column g of n-tile hr, held by the lane with 2 tig + j = g)
  float e[2][4], er[2];
  {
    float sr[2][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      sr[0][i] = 0.0f;
      sr[1][i] = 0.0f;
      e[0][i] = -INFINITY;
      e[1][i] = -INFINITY;
    }
    mma16816(sr[0], qa, kr[0], kr[1]);
    mma16816(sr[1], qa, kr[2], kr[3]);
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      er[hr] = -INFINITY;
#pragma unroll
      for (int j = 0; j < 2; ++j)
        if (2 * tig + j == g && mine[hr]) er[hr] = sr[hr][2 * hr + j];
    }
  }
#pragma unroll
  for (int al = 0; al < 4; ++al) {  // (na <= 4; unrolled so that the agents' loads and MMAs overlap)
    if (al >= na) break;
    const int a = a0 + al, ra = a - base, ha = ra >> 3, ga = ra & 7;
    uint32_t kb[4];
    ldsm_x4(kmajor_row(aK, min(NS * a + rr + (mi >> 1) * 8, 127), 16 * h + (mi & 1) * 8), kb);
    float sa[2][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      sa[0][i] = 0.0f;
      sa[1][i] = 0.0f;
    }
    mma16816(sa[0], qa, kb[0], kb[1]);
    mma16816(sa[1], qa, kb[2], kb[3]);
    if (g == ga) {
      if (ha == 0) {
        e[0][0] = sa[0][0];
        e[0][1] = sa[0][1];
        e[0][2] = sa[1][0];
        e[0][3] = sa[1][1];
      } else {
        e[1][0] = sa[0][2];
        e[1][1] = sa[0][3];
        e[1][2] = sa[1][2];
        e[1][3] = sa[1][3];
      }
    }
  }
  // softmax along each row (rows of agents outside the group get P = 0)
  float pr[2], inv[2];
#pragma unroll
  for (int hr = 0; hr < 2; ++hr) {
    float mx = er[hr];
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float v = 8 * n + 2 * tig + j < ne[hr] ? e[hr][2 * n + j] : -INFINITY;
        e[hr][2 * n + j] = v;
        mx = fmaxf(mx, v);
      }
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    if (!mine[hr]) mx = 0.0f;  // (every score of such a row is -inf)
    float sum = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      e[hr][i] = ex2_approx(e[hr][i] - mx);
      sum += e[hr][i];
    }
    pr[hr] = ex2_approx(er[hr] - mx);
    sum += pr[hr];
    sum += __shfl_xor_sync(0xffffffffu, sum, 1);
    sum += __shfl_xor_sync(0xffffffffu, sum, 2);
    inv[hr] = mine[hr] ? 1.0f / sum : 0.0f;
  }
  float o[2][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    o[0][i] = 0.0f;
    o[1][i] = 0.0f;
  }
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    if (al >= na) break;
    const int a = a0 + al, ra = a - base, ha = ra >> 3, ga = ra & 7;
    uint32_t vb[4];
    ldsm_x4_t(kmajor_row(aV, min(NS * a + rr + (mi & 1) * 8, 127), 16 * h + (mi >> 1) * 8), vb);
    const bool r_lo = g == ga && ha == 0, r_hi = g == ga && ha == 1;
    const uint32_t pa[4] = {r_lo ? pack_bf2(e[0][0], e[0][1]) : 0u, r_hi ? pack_bf2(e[1][0], e[1][1]) : 0u,
                            r_lo ? pack_bf2(e[0][2], e[0][3]) : 0u, r_hi ? pack_bf2(e[1][2], e[1][3]) : 0u};
    mma16816(o[0], pa, vb[0], vb[1]);
    mma16816(o[1], pa, vb[2], vb[3]);
  }
  {
    // the recurrent keys: row g's is column g (keys 0-7), row g + 8's is
    // column g + 8 (keys 8-15)
    const uint32_t pd[4] = {pack_bf2(2 * tig == g ? pr[0] : 0.0f, 2 * tig + 1 == g ? pr[0] : 0.0f), 0u, 0u,
                            pack_bf2(2 * tig == g ? pr[1] : 0.0f, 2 * tig + 1 == g ? pr[1] : 0.0f)};
    mma16816(o[0], pd, vr[0], vr[1]);
    mma16816(o[1], pd, vr[2], vr[3]);
  }
  __syncwarp();
#pragma unroll
  for (int hr = 0; hr < 2; ++hr) {
    if (mine[hr]) {
      const int row = rb16 + g + 8 * hr;
#pragma unroll
      for (int dn = 0; dn < 2; ++dn) {
        const int k = 16 * h + 8 * dn + 2 * tig;
        const uint32_t w = pack_bf2(o[dn][2 * hr] * inv[hr], o[dn][2 * hr + 1] * inv[hr]);
        asm volatile("st.shared.b32 [%0], %1;" ::"r"(kmajor_row(aQ, row, k) + (uint32_t)((k & 7) * 2)), "r"(w)
                     : "memory");
      }
    }
  }
}

// Contiguous row layout (agents of at most 16 tokens): agent a's tokens are
// rows r0 = R a .. r0 + R - 1, the recurrent token first.  One (agent, head)
// on the calling warp: keys r0 .. r0 + nt - 1 valid; writes O_h into the
// agent's rows of aO (the same K-major image as Q).  MT = 16-row tiles
// covering R.
template <int MT>
__device__ __forceinline__ void attend_warp(uint32_t aQ, uint32_t aK, uint32_t aV, int r0, int R, int nt, int h) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
  const int mi = lane >> 3, rr = lane & 7;
  uint32_t qa[MT][4];
#pragma unroll
  for (int m = 0; m < MT; ++m) {  // A: rows r0 + 16 m .., head columns 16 h ..
    const int row = min(r0 + 16 * m + rr + (mi & 1) * 8, 127);
    ldsm_x4(kmajor_row(aQ, row, 16 * h + (mi >> 1) * 8), qa[m]);
  }
  float sc[MT][2 * MT][4];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int n = 0; n < 2 * MT; ++n)
#pragma unroll
      for (int i = 0; i < 4; ++i) sc[m][n][i] = 0.0f;
#pragma unroll
  for (int kt = 0; kt < MT; ++kt) {  // keys 16 kt .. 16 kt + 15: B fragments of two 8-key tiles
    uint32_t kb[4];
    const int key = min(r0 + 16 * kt + rr + (mi >> 1) * 8, 127);
    ldsm_x4(kmajor_row(aK, key, 16 * h + (mi & 1) * 8), kb);
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      mma16816(sc[m][2 * kt], qa[m], kb[0], kb[1]);
      mma16816(sc[m][2 * kt + 1], qa[m], kb[2], kb[3]);
    }
  }
  // softmax along each query row (base-2: Q carries the log2(e) factor)
  float inv[MT][2];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      float mx = -INFINITY;
#pragma unroll
      for (int n = 0; n < 2 * MT; ++n)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int col = 8 * n + 2 * tig + j;
          const float v = col < nt ? sc[m][n][2 * hr + j] : -INFINITY;
          sc[m][n][2 * hr + j] = v;
          mx = fmaxf(mx, v);
        }
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      float sum = 0.0f;
#pragma unroll
      for (int n = 0; n < 2 * MT; ++n)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const float e = ex2_approx(sc[m][n][2 * hr + j] - mx);
          sc[m][n][2 * hr + j] = e;
          sum += e;
        }
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      sum += __shfl_xor_sync(0xffffffffu, sum, 2);
      inv[m][hr] = 1.0f / sum;
    }
  // O = P V: P from the score fragments, V through transposing loads
  float o[MT][2][4];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int dn = 0; dn < 2; ++dn)
#pragma unroll
      for (int i = 0; i < 4; ++i) o[m][dn][i] = 0.0f;
#pragma unroll
  for (int kk = 0; kk < MT; ++kk) {
    uint32_t vb[4];
    const int key = min(r0 + 16 * kk + rr + (mi & 1) * 8, 127);
    ldsm_x4_t(kmajor_row(aV, key, 16 * h + (mi >> 1) * 8), vb);
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      uint32_t pa[4];
      pa[0] = pack_bf2(sc[m][2 * kk][0], sc[m][2 * kk][1]);
      pa[1] = pack_bf2(sc[m][2 * kk][2], sc[m][2 * kk][3]);
      pa[2] = pack_bf2(sc[m][2 * kk + 1][0], sc[m][2 * kk + 1][1]);
      pa[3] = pack_bf2(sc[m][2 * kk + 1][2], sc[m][2 * kk + 1][3]);
      mma16816(o[m][0], pa, vb[0], vb[1]);
      mma16816(o[m][1], pa, vb[2], vb[3]);
    }
  }
  __syncwarp();
  // normalised O into the agent's own rows (other rows of the 16-row tiles
  // belong to the next agent or to padding)
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int row = r0 + 16 * m + g + 8 * hr;
      if (row < r0 + R && row < 128) {
#pragma unroll
        for (int dn = 0; dn < 2; ++dn) {
          const int k = 16 * h + 8 * dn + 2 * tig;
          const uint32_t w = pack_bf2(o[m][dn][2 * hr] * inv[m][hr], o[m][dn][2 * hr + 1] * inv[m][hr]);
          asm volatile("st.shared.b32 [%0], %1;" ::"r"(kmajor_row(aQ, row, k) + (uint32_t)((k & 7) * 2)), "r"(w)
                       : "memory");
        }
      }
    }
}

template <int D>
__global__ void __launch_bounds__(Geo<D>::THREADS, D == 64 ? 2 : 1) policy_fwd_kernel(PolicyDev p) {
  pdl_wait();  // (dependents launch as this grid's CTAs exit: no early trigger in a many-wave kernel)
  using G = Geo<D>;
  constexpr int COLS = G::COLS, kThreads = G::THREADS;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem + G::A_OFF;
  unsigned char* ring = smem + G::RING_OFF;
  unsigned char* sK = smem + G::KV_OFF;             // K-major image [128 x D]
  unsigned char* sV = sK + (size_t)128 * D * 2;      // K-major image [128 x D]
  unsigned char* sH = smem + G::KV_OFF;  // FFN hidden chunk image [128 x 128] (K/V are dead by then)
  float* sVec = reinterpret_cast<float*>(smem + G::VEC_OFF);
  float2* sStat = reinterpret_cast<float2*>(smem + G::STAT_OFF);
  __shared__ __align__(8) uint64_t full[kSlots];
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ __align__(8) uint64_t bar[4];  // further MMA groups in flight at the same time
  __shared__ __align__(8) uint64_t never;  // test hook: a barrier nothing signals
  __shared__ uint32_t tmem_base_s;
  __shared__ int bad;
  __shared__ int s_nent[64];  // entity tokens in use per agent of the tile

  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & 127, part = tid >> 7;
  const int c_lo = part * COLS;
  // row layout: agents of at most 16 tokens contiguous (slot * R + tok);
  // longer ones split: entity rows slot * NS + (tok - 1), then the recurrent
  // rows (tok 0) at NS * apt + slot; rows past those are padding (slot >= apt)
  const bool split = p.R > 16;
  const int rb = p.NS * p.apt;
  const int slot = split ? (row < rb ? row / p.NS : row - rb) : row / p.R;
  const int tok = split ? (row < rb ? 1 + row - slot * p.NS : 0) : row - slot * p.R;
  const long long ag = (long long)blockIdx.x * p.apt + slot;
  const bool agent_ok = slot < p.apt && ag < p.NA;
  const int n_tok = agent_ok ? 1 + min(max(p.n_ent[ag], 0), p.NS) : 0;
  const bool row_ok = tok < n_tok;
  if (tid < p.apt) {
    const long long a2 = (long long)blockIdx.x * p.apt + tid;
    s_nent[tid] = a2 < p.NA ? min(max(p.n_ent[a2], 0), p.NS) : 0;
  }

  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_s, G::TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 32) {
    for (int k = 0; k < kSlots; ++k) tc::mbar_init(&full[k], 1);
    tc::mbar_init(&mma_bar, 1);
    for (int k = 0; k < 4; ++k) tc::mbar_init(&bar[k], 1);
    tc::mbar_init(&never, 1);
    bad = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base_s;
  if (p.test_wait_polls) {
    // test hook: a bounded wait that runs out, then the timed-out exit (no
    // copy or MMA has been issued, so nothing is in flight)
    if (tid == 32 && !tc::mbar_wait(&never, 0u, p.test_wait_polls)) bad = 1;
    __syncthreads();
    if (bad) {
      if (tid == 0) raise_status(p.status, 2);
      if (warp == 0) tc::tmem_dealloc(tmem, G::TMEM_COLS);
      return;
    }
  }
  const uint32_t tl = tmem + ((uint32_t)(warp & 3) << 21);  // this warp's lane quarter (lane 32 (w % 4))
  const uint32_t aA = tc::smem_addr(sA), aH = tc::smem_addr(sH), aRing = tc::smem_addr(ring);
  Loader ld{0, 0, p.L * G::NSTG};
  if (tid == 0) pump<D>(ld, p.wimg, ring, full);
  uint32_t mphase = 0, phases = 0;  // bit k: parity of bar[k]
  bool ok = true;  // every bounded wait of this thread succeeded
  int s = 0;       // global weight stage

  // Thread 0: wait for the images of stages s .. s + n - 1 (bounded).
  auto wait_images = [&](int n) {
    for (int j = 0; j < n; ++j) ok &= tc::mbar_wait(&full[(s + j) % kSlots], (uint32_t)(((s + j) / kSlots) & 1), kPolls);
  };
  // Every thread: wait for the MMA group just committed, then refill the ring.
  auto wait_mma = [&](int n) {
    ok &= tc::mbar_wait(&mma_bar, mphase, kPolls);
    mphase ^= 1u;
    tc::fence_after_sync();
    s += n;
    if (tid == 0) {
      ld.done = s;
      pump<D>(ld, p.wimg, ring, full);
    }
  };
  auto slot_addr = [&](int stage) { return aRing + (uint32_t)((stage % kSlots) * G::SLOT); };
  // Every thread: wait for the group committed to bar[k].  A barrier gets
  // its next commit only after a block barrier that follows every thread's
  // wait, so that no thread can miss a phase.
  auto wait_bar = [&](int k) {
    ok &= tc::mbar_wait(&bar[k], (phases >> k) & 1u, kPolls);
    phases ^= 1u << k;
  };
  // Thread 0: every stage issued so far has completed; refill the ring.
  auto release = [&]() {
    tc::fence_after_sync();
    if (tid == 0) {
      ld.done = s;
      pump<D>(ld, p.wimg, ring, full);
    }
  };

  // The per-layer vectors (LayerNorm gains and offsets, biases) arrive by
  // asynchronous copies into the double buffer, layer 0's now and layer
  // l + 1's during layer l's attention; each thread waits for its own copies
  // at the top of the layer, and the LayerNorm's barrier publishes them.
  auto prefetch_vec = [&](int l) {
    float* dst = sVec + (l & 1) * G::VEC;
    const float* src = p.vec + (size_t)l * G::VEC;
    for (int i = tid; i < G::VEC / 4; i += kThreads) cp_async16(dst + 4 * i, src + 4 * i);
    cp_async_commit();
  };
  prefetch_vec(0);

  // ---- token rows ----------------------------------------------------------
  float x[COLS];
  if (row_ok && tok == 0) {
    const uint16_t* hp = p.h + ag * D + c_lo;
#pragma unroll
    for (int c0 = 0; c0 < COLS; c0 += 16) {
      float v[16];
      load16_bf(hp + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) x[c0 + i] = v[i];
    }
  } else if (row_ok) {
    const uint4 t4 = *reinterpret_cast<const uint4*>(p.tokens + (ag * p.NS + (tok - 1)) * 8);
    const float t[8] = {bf_lo(t4.x), bf_hi(t4.x), bf_lo(t4.y), bf_hi(t4.y),
                        bf_lo(t4.z), bf_hi(t4.z), bf_lo(t4.w), bf_hi(t4.w)};
    const float4* w4 = reinterpret_cast<const float4*>(p.emb_w) + c_lo * 2;
#pragma unroll
    for (int c = 0; c < COLS; ++c) {
      const float4 wa = __ldg(w4 + 2 * c), wb = __ldg(w4 + 2 * c + 1);
      float acc = __ldg(p.emb_b + c_lo + c);
      acc = fmaf(wa.x, t[0], acc);
      acc = fmaf(wa.y, t[1], acc);
      acc = fmaf(wa.z, t[2], acc);
      acc = fmaf(wa.w, t[3], acc);
      acc = fmaf(wb.x, t[4], acc);
      acc = fmaf(wb.y, t[5], acc);
      acc = fmaf(wb.z, t[6], acc);
      acc = fmaf(wb.w, t[7], acc);
      x[c] = acc;
    }
  } else {
#pragma unroll
    for (int c = 0; c < COLS; ++c) x[c] = 0.0f;
  }

  // Every thread runs every stage (the barriers stay uniform); a wait that
  // gave up only marks the result invalid.
  for (int l = 0; l < p.L; ++l) {
    float* vec = sVec + (l & 1) * G::VEC;  // double-buffered: the previous layer may still read its copy
    cp_async_wait_all();
    const float *ln1g = vec, *ln1b = vec + D, *bq = vec + 2 * D, *bk = vec + 3 * D, *bv = vec + 4 * D;
    const float *bo = vec + 5 * D, *ln2g = vec + 6 * D, *ln2b = vec + 7 * D, *b1 = vec + 8 * D, *b2 = vec + 12 * D;

    // ---- attention sub-block: the LayerNorm output in TMEM is the A
    // operand of Q, K and V (three MMA groups, each drained as it completes
    // while the later ones run) ----
    ln_part_to_tmem<D>(x, ln1g, ln1b, tl + G::COL_A + (uint32_t)(c_lo / 2), sStat, row, part);  // (publishes `vec`)
    publish();
    if (tid == 0) {
      wait_images(3);
      issue_mma_ts(tmem + G::COL_Q, tmem + G::COL_A, slot_addr(s), D, D, false);
      tc::mma_commit(&bar[0]);
      issue_mma_ts(tmem + G::COL_K, tmem + G::COL_A, slot_addr(s + 1), D, D, false);
      tc::mma_commit(&bar[1]);
      issue_mma_ts(tmem + G::COL_V, tmem + G::COL_A, slot_addr(s + 2), D, D, false);
      tc::mma_commit(&mma_bar);
    }
    // Q (+ bias, times log2(e) / 4 for a base-2 softmax), K and V (+ bias) ->
    // K-major BF16 images, this thread's part of the columns
#pragma unroll 1
    for (int qkv = 0; qkv < 3; ++qkv) {
      if (qkv < 2) wait_bar(qkv);
      if (qkv == 2) wait_mma(3);  // (releases the three weight images)
      tc::fence_after_sync();
      const float* bias = qkv == 0 ? bq : (qkv == 1 ? bk : bv);
      const float scale = qkv == 0 ? 0.25f * 1.44269504088896341f : 1.0f;  // 1 / sqrt(16), log2(e)
      unsigned char* dst = qkv == 0 ? sA : (qkv == 1 ? sK : sV);
      const uint32_t col = qkv == 0 ? G::COL_Q : (qkv == 1 ? G::COL_K : G::COL_V);
      for_items<G::NS, COLS / 16>(
          warp, part, qkv * (COLS / 16),
          [&](int pp, int k) {
            const int cc = pp * COLS + 16 * k;
            float v[16];
            tc::tmem_ld16(tl + col + cc, v);
            bias_scale2<16>(v, bias + cc, scale);
            store8(dst, row, cc, 128, v);
            store8(dst, row, cc + 8, 128, v + 8);
          },
          [&](int pp, int k) {
            const int cc = pp * COLS + 16 * k;
            float v[32];
            tc::tmem_ld32(tl + col + cc, v);
            bias_scale2<32>(v, bias + cc, scale);
#pragma unroll
            for (int i = 0; i < 32; i += 8) store8(dst, row, cc + i, 128, v + i);
          });
    }
    __syncthreads();  // Q, K, V of every row visible
    // softmax attention on warp-level MMAs, one task per warp at a time:
    // contiguous layout: (agent, head); split layout: (head, group of 4
    // agents) for the recurrent queries, then (agent, head) for the entity
    // queries; O overwrites Q in the query rows
    {
      const uint32_t aK = tc::smem_addr(sK), aV = tc::smem_addr(sV);
      // (split layout, last block: only the recurrent rows reach the head and
      // the next h, so the entity queries' outputs are never read and their
      // tasks are skipped; the keys and values of every token still enter)
      const int n_rec = split ? ((p.apt + 3) >> 2) * G::H : 0;
      const int n_tasks = n_rec + (split && l == p.L - 1 ? 0 : p.apt * G::H);
      const long long left = p.NA - (long long)blockIdx.x * p.apt;  // agents of this tile and beyond
#pragma unroll 1
      for (int task = warp; task < n_tasks; task += kThreads / 32) {  // (warp-uniform)
        if (task < n_rec) {
          const int gi = task / G::H, h = task - gi * G::H, a0 = 4 * gi;
          const int na = (int)min((long long)min(4, p.apt - a0), left - a0);
          if (na > 0) attend_recurrent(aA, aK, aV, a0, na, p.NS, rb, s_nent, h);
        } else {
          const int t2 = task - n_rec, a = t2 / G::H, h = t2 - a * G::H;
          if (a >= left) continue;
          if (split)
            attend_entity(aA, aK, aV, a, p.NS, rb, s_nent[a], h);
          else
            attend_warp<1>(aA, aK, aV, a * p.R, p.R, 1 + s_nent[a], h);
        }
      }
    }
    if (l + 1 < p.L) prefetch_vec(l + 1);  // (buffer (l + 1) & 1 was last read in layer l - 1)
    publish();
    if (tid == 0) {
      wait_images(1);
      issue_mma(tmem + G::COL_S, aA, slot_addr(s), D, D, false);
      tc::mma_commit(&mma_bar);
    }
    wait_mma(1);
#pragma unroll
    for (int c0 = 0; c0 < COLS; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tl + G::COL_S + c_lo + c0, v);
      residual_add2<16>(x + c0, v, bo + c_lo + c0);
    }

    // ---- feed-forward sub-block ----
    ln_part_to_tmem<D>(x, ln2g, ln2b, tl + G::COL_A + (uint32_t)(c_lo / 2), sStat, row, part);
    if constexpr (G::PIPE) {
      // Software-pipelined over the hidden chunks: the tensor cores run W2 of
      // chunk c - 1 and W1 of chunk c + 1 during GELU_c.  The chunk's pre-activations alternate
      // between two TMEM column blocks and its GELU output between two BF16
      // images; W1_c commits to bar[c & 1], W2_c to bar[2 + (c & 1)], and both
      // are waited for at the top of a later chunk, when the MMAs have long
      // completed.
      publish();
      if (tid == 0) {
        wait_images(1);
        issue_mma_ts(tmem + G::COL_S, tmem + G::COL_A, slot_addr(s), 128, D, false);
        tc::mma_commit(&bar[0]);
      }
      ++s;
#pragma unroll 1
      for (int c = 0; c < G::NC; ++c) {
        const uint32_t col_cur = G::COL_S + (uint32_t)(c & 1) * 128u, col_nxt = G::COL_S + (uint32_t)((c + 1) & 1) * 128u;
        unsigned char* hcur = sH + (size_t)(c & 1) * 128 * 128 * 2;
        // W1_c complete (block c & 1 holds its output) and W2_{c-2} complete
        // (its operand image c & 1 is free)
        wait_bar(c & 1);
        if (c >= 2) wait_bar(2 + (c & 1));
        release();
        if (c > 0) {
          if (tid == 0) {
            wait_images(1);
            issue_mma(tmem + G::COL_ACC, tc::smem_addr(sH + (size_t)((c - 1) & 1) * 128 * 128 * 2), slot_addr(s), D,
                      128, c > 1);
            tc::mma_commit(&bar[2 + ((c - 1) & 1)]);
          }
          ++s;
        }
        if (c + 1 < G::NC) {  // (warp 0 takes no GELU items: its thread 0 issues W1_{c+1} now)
          if (tid == 0) {
            wait_images(1);
            issue_mma_ts(tmem + col_nxt, tmem + G::COL_A, slot_addr(s), 128, D, false);
            tc::mma_commit(&bar[(c + 1) & 1]);
          }
          ++s;
        }
        // GELU of this thread's hidden units of chunk c -> BF16 operand
        for_items<G::NS, G::HCOLS / 16>(
            warp, part, c * (G::HCOLS / 16),
            [&](int pp, int k) {
              const int hc = pp * G::HCOLS + 16 * k;
              float v[16];
              tc::tmem_ld16(tl + col_cur + hc, v);
              bias_add2<16>(v, b1 + c * 128 + hc);
#pragma unroll
              for (int i = 0; i < 16; i += 2) gelu2(v[i], v[i + 1]);
              store8(hcur, row, hc, 128, v);
              store8(hcur, row, hc + 8, 128, v + 8);
            },
            [&](int pp, int k) {  // (one item at a time: 32 live values cost more than the second wait)
#pragma unroll 1
              for (int kk = k; kk < k + 2; ++kk) {
                const int hc = pp * G::HCOLS + 16 * kk;
                float v[16];
                tc::tmem_ld16(tl + col_cur + hc, v);
                bias_add2<16>(v, b1 + c * 128 + hc);
#pragma unroll
                for (int i = 0; i < 16; i += 2) gelu2(v[i], v[i + 1]);
                store8(hcur, row, hc, 128, v);
                store8(hcur, row, hc + 8, 128, v + 8);
              }
            });
        publish();  // H_c visible to the tensor cores, block c & 1 read
      }
      // W2 of the last chunk; then W2_{NC-2} and W2_{NC-1} complete
      if (tid == 0) {
        wait_images(1);
        issue_mma(tmem + G::COL_ACC, tc::smem_addr(sH + (size_t)((G::NC - 1) & 1) * 128 * 128 * 2), slot_addr(s), D,
                  128, true);
        tc::mma_commit(&bar[2 + ((G::NC - 1) & 1)]);
      }
      ++s;
      wait_bar(2 + ((G::NC - 2) & 1));
      wait_bar(2 + ((G::NC - 1) & 1));
      release();
    } else {
#pragma unroll 1
    for (int c = 0; c < G::NC; ++c) {
      publish();
      if (tid == 0) {
        wait_images(1);
        issue_mma_ts(tmem + G::COL_S, tmem + G::COL_A, slot_addr(s), 128, D, false);
        tc::mma_commit(&mma_bar);
      }
      wait_mma(1);
      // GELU of this thread's hidden units of the chunk -> BF16 operand
      for_items<G::NS, G::HCOLS / 16>(
          warp, part, c * (G::HCOLS / 16),
          [&](int pp, int k) {
            const int hc = pp * G::HCOLS + 16 * k;
            float v[16];
            tc::tmem_ld16(tl + G::COL_S + hc, v);
            bias_add2<16>(v, b1 + c * 128 + hc);
#pragma unroll
            for (int i = 0; i < 16; i += 2) gelu2(v[i], v[i + 1]);
            store8(sH, row, hc, 128, v);
            store8(sH, row, hc + 8, 128, v + 8);
          },
          [&](int pp, int k) {
#pragma unroll 1
            for (int kk = k; kk < k + 2; ++kk) {
              const int hc = pp * G::HCOLS + 16 * kk;
              float v[16];
              tc::tmem_ld16(tl + G::COL_S + hc, v);
              bias_add2<16>(v, b1 + c * 128 + hc);
#pragma unroll
              for (int i = 0; i < 16; i += 2) gelu2(v[i], v[i + 1]);
              store8(sH, row, hc, 128, v);
              store8(sH, row, hc + 8, 128, v + 8);
            }
          });
      publish();
      if (tid == 0) {
        wait_images(1);
        issue_mma(tmem + G::COL_ACC, aH, slot_addr(s), D, 128, c > 0);
        tc::mma_commit(&mma_bar);
      }
      wait_mma(1);
    }
    }
#pragma unroll
    for (int c0 = 0; c0 < COLS; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tl + G::COL_ACC + c_lo + c0, v);
      residual_add2<16>(x + c0, v, b2 + c_lo + c0);
    }
  }

  // ---- head on the recurrent token ----------------------------------------
  // LN_f of the recurrent rows (statistics combined across the row's column
  // parts) goes to shared memory (the K/V region is free once the last MMA
  // has completed); then one warp per agent forms the logits (lanes split the
  // columns, warp sums) and draws the action (one lane per action, warp
  // argmax with the lowest index among equal maxima).
  float* sY = reinterpret_cast<float*>(smem + G::KV_OFF);  // [apt][D]
  if (!ok) atomicExch(&bad, 1);
  {
    float mean, inv;
    ln_part_stats<D>(x, sStat, row, part, mean, inv);
    if (agent_ok && tok == 0) {
      uint16_t* hp = p.h + ag * D + c_lo;
#pragma unroll
      for (int c0 = 0; c0 < COLS; c0 += 16) {
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          v[i] = x[c0 + i];
          sY[slot * D + c_lo + c0 + i] =
              fmaf((x[c0 + i] - mean) * inv, __ldg(p.lnf_g + c_lo + c0 + i), __ldg(p.lnf_b + c_lo + c0 + i));
        }
        store16_bf(hp + c0, v);
      }
    }
  }
  __syncthreads();
  const bool good = bad == 0;
#pragma unroll 1
  for (int sl = warp; sl < p.apt && good; sl += kThreads / 32) {
    const int lane = tid & 31, n_act = p.n_act;
    const long long a2 = (long long)blockIdx.x * p.apt + sl;
    if (a2 < p.NA) {  // (warp-uniform)
      float y[D / 32];
#pragma unroll
      for (int i = 0; i < D / 32; ++i) y[i] = sY[sl * D + lane + 32 * i];
      float mine = 0.0f;  // lane j: logit of action j
      for (int j0 = 0; j0 < n_act; j0 += 8) {
        float acc[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          acc[jj] = 0.0f;
          if (j0 + jj < n_act) {
            const float* w = p.head_w + (size_t)(j0 + jj) * D + lane;
#pragma unroll
            for (int i = 0; i < D / 32; ++i) acc[jj] = fmaf(__ldg(w + 32 * i), y[i], acc[jj]);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) acc[jj] += __shfl_xor_sync(0xffffffffu, acc[jj], o);
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          if (lane == j0 + jj) mine = acc[jj];
      }
      if (lane < n_act) {
        mine += __ldg(p.head_b + lane);
        p.logits[a2 * n_act + lane] = mine;
      }
      if (p.sample) {
        float z = -INFINITY;
        int arg = lane;
        if (lane < n_act) {
          const uint32_t g = p.counters ? p.counters[0] + 1u : p.step;
          const Rand4 r = philox(p.gid_agent + (uint32_t)a2, (uint32_t)(lane >> 2), g, TAG_GUMBEL, p.seed);
          const int q = lane & 3;
          const uint32_t u = q == 0 ? r.x[0] : (q == 1 ? r.x[1] : (q == 2 ? r.x[2] : r.x[3]));
          z = mine - logf(-logf(unif_mid(u)));
          if (!(z == z)) z = -INFINITY;  // a NaN never wins
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float oz = __shfl_xor_sync(0xffffffffu, z, o);
          const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
          if (oz > z || (oz == z && oa < arg)) {
            z = oz;
            arg = oa;
          }
        }
        if (lane == 0) p.actions[a2] = arg;
      }
    }
  }

  // no copy may still be landing in shared memory when the CTA exits
  if (tid == 0 && !good)
    for (int k = 0; k < kSlots && k < ld.next; ++k) {
      const int last = ld.next - 1 - ((ld.next - 1 - k) % kSlots);  // last stage fetched into slot k
      tc::mbar_wait(&full[k], (uint32_t)((last / kSlots) & 1), kPolls);
    }
  tc::fence_before_sync();
  __syncthreads();
  if (good == false && tid == 0) raise_status(p.status, 2);
  if (warp == 0) tc::tmem_dealloc(tmem, G::TMEM_COLS);
}

template <int D>
cudaError_t launch_policy_t(const PolicyDev& p, cudaStream_t s) {
  static std::atomic<unsigned long long> ready{0};
  {
    const cudaError_t e = smem_optin(policy_fwd_kernel<D>, Geo<D>::SMEM, ready);
    if (e != cudaSuccess) return e;
  }
  // (a lane per action; the row layouts need R = 1 + NS and R apt <= 128)
  if (p.n_act < 1 || p.n_act > 32 || p.NS < 1 || p.NS > 16 || p.R != 1 + p.NS || p.apt < 1 || p.apt > 64 ||
      p.R * p.apt > 128)
    return cudaErrorInvalidValue;
  const long long tiles = (p.NA + p.apt - 1) / p.apt;
  if (tiles > 0) {
    const cudaError_t e =
        launch_pdl(policy_fwd_kernel<D>, dim3((unsigned)tiles), dim3(Geo<D>::THREADS), Geo<D>::SMEM, s, p);
    if (e != cudaSuccess) return e;
  }
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
