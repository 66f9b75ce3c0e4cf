// Tensor-core GEMMs of the transformer training path (included by tfm.cu,
// inside namespace ut::tfm after the Gemm descriptor and its epilogues).
//
// The three products of a linear layer y = W x + b over the token rows:
//   forward          C[m][n] = sum_k A[m][k] W[n][k]        (kind 0)
//   input gradient   C[m][k] = sum_n A[m][n] W[n][k]        (kind 1)
//   weight gradient  dW[n][k] = sum_m dOut[m][n] In[m][k]   (kind 2)
// run on tcgen05.mma (kind::f16): BF16 operands, FP32 accumulation in
// tensor memory.  Activations stay FP32 in HBM; each CTA converts its
// operand tiles to BF16 while it stages them in shared memory (K-major, no
// swizzle, tc.cuh's layout), two stages deep, so that the conversion of one
// K chunk overlaps the MMAs of the previous one.  The weights' BF16 images
// (W for the forward, W^T for the input gradient) are packed once per call
// (pack_images_kernel in tfm.cu).
//
// Tiles: kinds 0 / 1 take 128 token rows x up to 256 outputs per CTA, K in
// chunks of 64; kind 2 takes 128 output features x up to 256 input features
// per CTA and a range of token rows in chunks of 64 (the K of the MMA),
// written as a partial slab that the caller sums over the row splits in a
// fixed order.  The epilogues (bias, residual, erf-GELU and its derivative)
// are the SIMT kernels' epi_store.
// (tc.cuh is included by tfm.cu at file scope.)
#pragma once

constexpr int kTcThreads = 256;
constexpr int kTcChunk = 64;        // K per stage
constexpr int kTcMaxN = 256;        // N per CTA (tensor-memory columns)
constexpr size_t kTcStageA = (size_t)128 * kTcChunk * 2;      // 16 KB
constexpr size_t kTcStageB = (size_t)kTcMaxN * kTcChunk * 2;  // 32 KB
constexpr size_t kTcSmem = 2 * (kTcStageA + kTcStageB);       // 96 KB
constexpr uint32_t kTcPolls = 1u << 22;

// Columns of tensor memory for an N-wide accumulator (a power of two >= 32).
__host__ __device__ constexpr uint32_t tc_cols(int n) {
  return n <= 32 ? 32u : (n <= 64 ? 64u : (n <= 128 ? 128u : 256u));
}

// BF16 image of a weight matrix for the B operand: rows r of the product's
// B (r < R) by contraction index c (c < C), K-major no-swizzle, in blocks of
// 256 rows, each block [C / 8][rows in block][8]; so the 64-wide chunk j of a
// block is the contiguous range of 8 * rows * 16 bytes at j * 8 * rows * 16.
// transpose = 0: B(r, c) = W[r][c] (W [R][C] row-major: the forward);
// transpose = 1: B(r, c) = W[c][r] (W [C][R] row-major: the input gradient).
__host__ __device__ inline size_t img_offset(int r, int c, int R, int C) {
  const int blk = r / kTcMaxN, rr = r % kTcMaxN;
  const int rows = min(kTcMaxN, R - blk * kTcMaxN);
  return (size_t)blk * kTcMaxN * C * 2 + (size_t)(c >> 3) * rows * 16 + (size_t)rr * 16 + (size_t)(c & 7) * 2;
}

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) { return bf16x2_bits(lo, hi); }

// The epilogue of four consecutive outputs (m, n .. n + 3) (float4 form of
// epi_store; ldc, n multiples of 4).
__device__ __forceinline__ void epi_store4(const Gemm& g, long long m, int n, float4 v) {
  const long long o = m * g.ldc + n;
  float4 r;
  switch (g.epi) {
    case EPI_BIAS: {
      const float4 b = *reinterpret_cast<const float4*>(g.bias + n);
      r = make_float4(v.x + b.x, v.y + b.y, v.z + b.z, v.w + b.w);
      break;
    }
    case EPI_BIAS_RES: {
      const float4 b = *reinterpret_cast<const float4*>(g.bias + n);
      const float4 q = *reinterpret_cast<const float4*>(g.R + o);
      r = make_float4(v.x + b.x + q.x, v.y + b.y + q.y, v.z + b.z + q.z, v.w + b.w + q.w);
      break;
    }
    case EPI_BIAS_GELU: {
      const float4 b = *reinterpret_cast<const float4*>(g.bias + n);
      r = make_float4(v.x + b.x, v.y + b.y, v.z + b.z, v.w + b.w);
      *reinterpret_cast<float4*>(g.C2 + o) = make_float4(gelu_f(r.x), gelu_f(r.y), gelu_f(r.z), gelu_f(r.w));
      break;
    }
    case EPI_GELU_GRAD: {
      const float4 z = *reinterpret_cast<const float4*>(g.aux + o);
      r = make_float4(v.x * gelu_grad_f(z.x), v.y * gelu_grad_f(z.y), v.z * gelu_grad_f(z.z), v.w * gelu_grad_f(z.w));
      break;
    }
    default:
      r = v;
  }
  *reinterpret_cast<float4*>(g.C + o) = r;
}

// Shared memory of tc_wgrad_kernel for inputs n_i wide: two A stages and two
// B stages of min(n_i rounded up to 32, 256) rows.
inline size_t tc_wgrad_smem(int n_i) {
  return 2 * kTcStageA + 2 * (size_t)std::min(kTcMaxN, (n_i + 31) / 32 * 32) * kTcChunk * 2;
}

// Shared memory of tc_rows_kernel for outputs N wide: two A stages (the
// epilogue's staging tile overlays them) and two B stages sized for
// min(N, 256) rows; narrow products fit three CTAs per SM.
inline size_t tc_rows_smem(int N) {
  return 2 * kTcStageA + 2 * (size_t)std::min(kTcMaxN, N) * kTcChunk * 2;
}

// Kinds 0 / 1: C[m][n] = sum_k A[m][k] B(n, k) + epilogue, A FP32 row-major
// (lda), B the image of `R` = g.N rows by `C` = g.K columns.  Grid (CTAs
// looping over the row tiles of 128, column tiles of 256): each CTA keeps
// its tensor memory and barriers across its row tiles.  The K chunks are
// staged two deep.  A chunk's B (a contiguous range of the image) arrives by
// one bulk copy; with K <= 128 the B chunks stay resident across row tiles.
// A is loaded into registers a chunk ahead (the next chunk's loads, of this
// tile or the next, are issued as soon as the current chunk is converted,
// so they are in flight during its MMAs and the epilogue), rounded to BF16
// and written K-major.  The accumulator goes through a staging tile over the
// A stages (rows of 64 floats, 16-byte chunks XOR-swizzled by row) so that
// the epilogue reads and writes whole rows (coalesced float4 accesses).
__device__ __forceinline__ int epi_pos(int row, int c4) { return row * 64 + ((c4 ^ (row & 15)) << 2); }

__global__ void __launch_bounds__(kTcThreads, 3) tc_rows_kernel(Gemm g, const uint16_t* __restrict__ bimg,
                                                                int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                    // [2][128 x 64] BF16
  unsigned char* sB = smem + 2 * kTcStageA;    // [2][min(N, 256) x 64] BF16
  float* sE = reinterpret_cast<float*>(smem);  // epilogue staging [128][64] over the A stages
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t bfull[2];
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.y * kTcMaxN;
  const int Nt = min(kTcMaxN, g.N - n0);
  const int K = (int)g.K;
  const uint32_t ncols = tc_cols(Nt);
  if (warp == 0) {
    tc::tmem_alloc(&tbase, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 32) {
    for (int k = 0; k < 2; ++k) {
      tc::mbar_init(&mbar[k], 1);
      tc::mbar_init(&bfull[k], 1);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const uint16_t* bblk = bimg + (size_t)blockIdx.y * kTcMaxN * K;  // this column tile's image block
  const int nchunks = (K + kTcChunk - 1) / kTcChunk;
  const bool b_resident = nchunks <= 2;  // chunk c of every tile uses stage c (or both, for one chunk)
  const size_t b_stage = (size_t)min(kTcMaxN, g.N) * kTcChunk * 2;  // B stage bytes (tc_rows_smem)
  const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)Nt);
  const long long tiles = (g.M + 127) / 128;
  uint32_t phase = 0u, bphase = 0u, bpend = 0u;  // per stage s: bit s
  bool ok = true;
  int q_used = 0;  // chunks committed so far (the stage ring runs across tiles)

  // A of (row tile m0, chunk at k0): unit = (row, 8-column group), 2 or 4 per
  // thread, in registers until stage_a
  float4 xa[4][2];
  auto load_a = [&](long long m0, int k0) {
    const int units = 128 * (min(kTcChunk, K - k0) >> 3);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int u = tid + i * kTcThreads;
      const int row = u & 127, grp = u >> 7;
      xa[i][0] = xa[i][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (u < units && m0 + row < g.M) {
        const float4* src = reinterpret_cast<const float4*>(g.A + (m0 + row) * g.lda + k0 + grp * 8);
        xa[i][0] = __ldg(src);
        xa[i][1] = __ldg(src + 1);
      }
    }
  };
  // consecutive threads on consecutive rows of one group: conflict-free
  // 16-byte stores
  auto stage_a = [&](unsigned char* a, int kc) {
    const int units = 128 * (kc >> 3);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int u = tid + i * kTcThreads;
      if (u < units) {
        const int row = u & 127, grp = u >> 7;
        const uint4 p = make_uint4(pack_bf2(xa[i][0].x, xa[i][0].y), pack_bf2(xa[i][0].z, xa[i][0].w),
                                   pack_bf2(xa[i][1].x, xa[i][1].y), pack_bf2(xa[i][1].z, xa[i][1].w));
        *reinterpret_cast<uint4*>(a + tc::kmajor_offset(row, grp * 8, 128)) = p;
      }
    }
  };

  if ((long long)blockIdx.x < tiles) load_a((long long)blockIdx.x * 128, 0);
  for (long long mt = blockIdx.x; mt < tiles; mt += gridDim.x) {
    const long long m0 = mt * 128;
    for (int c = 0; c < nchunks; ++c, ++q_used) {
      const int s = q_used & 1;
      const int k0 = c * kTcChunk, kc = min(kTcChunk, K - k0);
      if (q_used >= 2 && c >= 2) {  // this tile's MMAs two chunks back read this stage
        ok &= tc::mbar_wait(&mbar[s], (phase >> s) & 1u, kTcPolls);
        phase ^= 1u << s;
        tc::fence_after_sync();
      }
      unsigned char* a = sA + s * kTcStageA;
      unsigned char* b = sB + (size_t)s * b_stage;
      const bool b_new = !b_resident || q_used < 2;
      if (b_new && tid == 0) {  // the stage is free: its last MMA has completed
        const uint32_t bytes = (uint32_t)(Nt * kc * 2);
        tc::mbar_expect_tx(&bfull[s], bytes);
        tc::bulk_g2s(b, bblk + (size_t)k0 * Nt, bytes, &bfull[s]);
      }
      stage_a(a, kc);
      // the next chunk's A: in flight during this chunk's MMAs (and epilogue)
      if (c + 1 < nchunks)
        load_a(m0, k0 + kTcChunk);
      else if (mt + gridDim.x < tiles)
        load_a(m0 + (long long)gridDim.x * 128, 0);
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (tid == 0) {
        if (b_new) {
          if (tc::mbar_wait(&bfull[s], (bphase >> s) & 1u, kTcPolls))
            bphase ^= 1u << s;
          else
            ok = false, bpend |= 1u << s;
        }
        const uint32_t aa = tc::smem_addr(a), bb = tc::smem_addr(b);
        for (int j = 0; j < kc / 16; ++j) {
          const uint64_t ad = tc::smem_desc(aa + j * 2 * 128 * 16, 128 * 16, 128);
          const uint64_t bd = tc::smem_desc(bb + j * 2 * Nt * 16, Nt * 16, 128);
          tc::mma_bf16(tmem, ad, bd, idesc, (c > 0 || j > 0) ? 1u : 0u);
        }
        tc::mma_commit(&mbar[s]);
      }
    }
    // this tile's last (up to two) chunks: their MMAs are done
    for (int c = max(0, nchunks - 2); c < nchunks; ++c) {
      const int s = (q_used - nchunks + c) & 1;
      ok &= tc::mbar_wait(&mbar[s], (phase >> s) & 1u, kTcPolls);
      phase ^= 1u << s;
    }
    tc::fence_after_sync();
    ok = __syncthreads_and(ok);  // (the tensor-memory loads below are warp-collective)
    if (!ok) break;
    // epilogue, 64 columns per round: warps 0-3 move columns [c0, c0 + 32),
    // warps 4-7 [c0 + 32, c0 + 64) of lane quarter w % 4 into the staging
    // tile; then each row's columns are read, finished and stored as float4
    const int q = warp & 3, half = warp >> 2;
    const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
    for (int c0 = 0; c0 < Nt; c0 += 64) {
      const int cw = min(64, Nt - c0);  // 32 or 64
      if (half * 32 < cw) {
        const int row = q * 32 + lane;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v[16];
          tc::tmem_ld16(lane_addr + c0 + half * 32 + h * 16, v);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            *reinterpret_cast<float4*>(sE + epi_pos(row, half * 8 + h * 4 + j)) =
                make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      const int per_row = cw / 4;  // float4 per row: 8 or 16
      for (int u = tid; u < 128 * per_row; u += kTcThreads) {
        const int row = u / per_row, c4 = u - row * per_row;
        const long long m = m0 + row;
        if (m < g.M) {
          const float4 v = *reinterpret_cast<const float4*>(sE + epi_pos(row, c4));
          epi_store4(g, m, n0 + c0 + c4 * 4, v);
        }
      }
      __syncthreads();  // the staging tile (the A stages) is free again
    }
  }
  // (a B copy whose wait gave up may still be landing: wait for it, bounded,
  // before the CTA exits)
  if (bpend != 0u)
    for (int k = 0; k < 2; ++k)
      if ((bpend >> k) & 1u) tc::mbar_wait(&bfull[k], (bphase >> k) & 1u, kTcPolls);
  if (!ok && tid == 0) raise_status(status, 2);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// Kind 2: part[z][n][k] = sum over this CTA's token rows m of
// dOut[m][n] In[m][k], n in a tile of 128 (grid.x), k in a tile of up to 256
// (grid.y), rows [z * rchunk, (z + 1) * rchunk) (grid.z).  g.A = dOut
// (lda = its width n_o = g.M), g.B = In (ldb = its width n_i = g.N),
// g.K = rows, g.kchunk = rows per split; part is g.C [splits][n_o][n_i].
// The bias gradient's partial sums sum_m dOut[m][n] (FP32, fixed order) go to
// bias_part [splits][n_o].
__global__ void __launch_bounds__(kTcThreads, 3) tc_wgrad_kernel(Gemm g, float* __restrict__ bias_part, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                   // [2][128 x 64] BF16: (n, m)
  unsigned char* sB = smem + 2 * kTcStageA;   // [2][256 x 64] BF16: (k, m)
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_o = (int)g.M, n_i = g.N;
  const int nb0 = blockIdx.x * 128, kb0 = blockIdx.y * kTcMaxN;
  const int Nt = min(kTcMaxN, n_i - kb0);
  const int Ntp = (Nt + 31) / 32 * 32;  // B rows staged (a multiple of 32; rows past n_i are zero)
  const size_t b_stage = (size_t)min(kTcMaxN, (n_i + 31) / 32 * 32) * kTcChunk * 2;  // (tc_wgrad_smem)
  const long long r0 = (long long)blockIdx.z * g.kchunk;
  const long long r1 = min(g.K, r0 + g.kchunk);
  const uint32_t ncols = tc_cols(Ntp);
  if (warp == 0) {
    tc::tmem_alloc(&tbase, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const long long nrows = r1 > r0 ? r1 - r0 : 0;
  const int nchunks = (int)((nrows + kTcChunk - 1) / kTcChunk);
  const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)Ntp);
  uint32_t phase[2] = {0u, 0u};
  bool ok = true;
  float bsum[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // this thread's rows of columns nb0 + 32 j + lane of dOut
  for (int c = 0; c < nchunks; ++c) {
    const int s = c & 1;
    const long long m0 = r0 + (long long)c * kTcChunk;
    if (c >= 2) {
      ok &= tc::mbar_wait(&mbar[s], phase[s], kTcPolls);
      phase[s] ^= 1u;
      tc::fence_after_sync();
    }
    unsigned char* a = sA + s * kTcStageA;
    unsigned char* b = sB + (size_t)s * b_stage;
    // transposed staging: warp w takes rows m0 + 8 w .. + 7 of the chunk, in
    // blocks of 32 consecutive columns (row loads coalesced across the warp);
    // each lane packs its column's 8 rows into one 16-byte core row.  A
    // (dOut): 4 column blocks, all 32 loads issued first; the lanes also sum
    // their FP32 values for the bias gradient.  B (In): Ntp / 32 blocks, two
    // at a time.
    {
      const long long mrow = m0 + warp * 8;
      float va[4][8];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gcol = nb0 + j * 32 + lane;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          va[j][i] = (mrow + i < r1 && gcol < n_o) ? __ldg(g.A + (mrow + i) * g.lda + gcol) : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float cs = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) cs += va[j][i];
        bsum[j] += cs;
        const uint4 p = make_uint4(pack_bf2(va[j][0], va[j][1]), pack_bf2(va[j][2], va[j][3]),
                                   pack_bf2(va[j][4], va[j][5]), pack_bf2(va[j][6], va[j][7]));
        *reinterpret_cast<uint4*>(a + tc::kmajor_offset(j * 32 + lane, warp * 8, 128)) = p;
      }
      for (int j0 = 0; j0 < Ntp / 32; j0 += 2) {
        float vb[2][8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int gcol = kb0 + (j0 + h) * 32 + lane;
          const bool on = j0 + h < Ntp / 32 && gcol < n_i;
#pragma unroll
          for (int i = 0; i < 8; ++i) vb[h][i] = (on && mrow + i < r1) ? __ldg(g.B + (mrow + i) * g.ldb + gcol) : 0.0f;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (j0 + h < Ntp / 32) {
            const uint4 p = make_uint4(pack_bf2(vb[h][0], vb[h][1]), pack_bf2(vb[h][2], vb[h][3]),
                                       pack_bf2(vb[h][4], vb[h][5]), pack_bf2(vb[h][6], vb[h][7]));
            *reinterpret_cast<uint4*>(b + tc::kmajor_offset((j0 + h) * 32 + lane, warp * 8, Ntp)) = p;
          }
        }
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t aa = tc::smem_addr(a), bb = tc::smem_addr(b);
      for (int j = 0; j < kTcChunk / 16; ++j) {
        const uint64_t ad = tc::smem_desc(aa + j * 2 * 128 * 16, 128 * 16, 128);
        const uint64_t bd = tc::smem_desc(bb + j * 2 * Ntp * 16, Ntp * 16, 128);
        tc::mma_bf16(tmem, ad, bd, idesc, (c > 0 || j > 0) ? 1u : 0u);
      }
      tc::mma_commit(&mbar[s]);
    }
  }
  for (int c = max(0, nchunks - 2); c < nchunks; ++c) {
    const int s = c & 1;
    ok &= tc::mbar_wait(&mbar[s], phase[s], kTcPolls);
    phase[s] ^= 1u;
  }
  tc::fence_after_sync();
  ok = __syncthreads_and(ok);  // (the tensor-memory loads below are warp-collective)
  if (ok) {
    const int q = warp & 3, half = warp >> 2;
    const int n = nb0 + q * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
    const int hw = Ntp / 2;
    float* out = g.C + ((long long)blockIdx.z * n_o + n) * n_i;
    for (int c0 = half * hw; c0 < (half + 1) * hw; c0 += 16) {
      float v[16];
      if (nchunks > 0) {
        tc::tmem_ld16(lane_addr + c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.0f;
      }
      if (n < n_o) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (kb0 + c0 + i < n_i) out[kb0 + c0 + i] = v[i];
      }
    }
  } else if (tid == 0) {
    raise_status(status, 2);
  }
  // bias gradient of this split: the eight warps' row sums added in warp
  // order (the first column tile only; the other tiles see the same dOut)
  __shared__ float s_bias[kTcThreads / 32][128];
  if (blockIdx.y == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) s_bias[warp][j * 32 + lane] = bsum[j];
  }
  __syncthreads();
  if (blockIdx.y == 0 && tid < 128 && nb0 + tid < n_o) {
    float acc = s_bias[0][tid];
#pragma unroll
    for (int w = 1; w < kTcThreads / 32; ++w) acc += s_bias[w][tid];
    bias_part[(long long)blockIdx.z * n_o + nb0 + tid] = acc;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}
