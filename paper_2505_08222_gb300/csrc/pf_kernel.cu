// Particle-filter step: predict, weight, estimate, systematic resample.
//
// One CTA per filter (one filter per (env, observer agent, target),
// Sec. III-A.2), NT threads x PPT consecutive particles each.  The filter's
// particles make exactly one round trip through HBM per step: 16 B read
// (x, y, vx, vy as four coalesced float4 streams) and 16 B written.  Weights,
// the CDF, the resample map and the gather stay on chip:
//   predict   v += sigma_a N(0, I) (one Philox call per particle pair),
//             |v| capped, p += dt v                                (reading C2)
//   weight    l_i = -sum_m (r_m - |p_i - q_m|)^2 / (2 sigma_r^2),  max by warp
//             shuffles, w_i = exp(l_i - max l), sums by warp shuffles (C3)
//   estimate  weighted mean before resampling                      (C6)
//   resample  q_i = floor(w_i 2^38) (exact), int64 block scan -> Q, W;
//             U0 = mulhi(u64, W); particle i owns the outputs
//             [count(P Q_{i-1}), count(P Q_i)) with
//             count(X) = #{j : j W + U0 < X}; its index is written at the
//             first owned output and a block prefix-max fills the rest;
//             gather from shared memory.                           (C4, C5)
// Integer arithmetic makes the resample map independent of summation order:
// with identical weights and offset it is bit-identical to the definition
// idx_j = min{i : P Q_i > j W + U0}.
#include "env.cuh"

namespace ut {

namespace {

template <int NT>
__device__ __forceinline__ float block_max(float v, float* s_tmp) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_max(v);
  if (lane == 0) s_tmp[wid] = v;
  __syncthreads();
  float r = lane < NW ? s_tmp[lane] : -INFINITY;
  r = warp_max(r);
  __syncthreads();
  return r;
}

template <int NT>
__device__ __forceinline__ void block_sum3(float& a, float& b, float& c, float* s_tmp) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  if (lane == 0) {
    s_tmp[wid] = a;
    s_tmp[NW + wid] = b;
    s_tmp[2 * NW + wid] = c;
  }
  __syncthreads();
  float ra = lane < NW ? s_tmp[lane] : 0.0f;
  float rb = lane < NW ? s_tmp[NW + lane] : 0.0f;
  float rc = lane < NW ? s_tmp[2 * NW + lane] : 0.0f;
  a = warp_sum(ra);
  b = warp_sum(rb);
  c = warp_sum(rc);
  __syncthreads();
}

// Exclusive block scan of int64 values; also returns the block total.
template <int NT>
__device__ __forceinline__ long long block_excl_scan(long long v, long long* s_tmp, long long& total) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_tmp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    long long w = lane < NW ? s_tmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < NW) s_tmp[lane] = w;
  }
  __syncthreads();
  const long long before = wid > 0 ? s_tmp[wid - 1] : 0;
  total = s_tmp[NW - 1];
  __syncthreads();
  return before + incl - v;
}

// Inclusive block prefix-max of int values (identity -1), given each
// thread's local maximum; returns the maximum over all earlier threads.
template <int NT>
__device__ __forceinline__ int block_excl_max(int v, int* s_tmp) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl = max(incl, t);
  }
  int excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = -1;
  if (lane == 31) s_tmp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < NW ? s_tmp[lane] : -1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w = max(w, t);
    }
    if (lane < NW) s_tmp[lane] = w;
  }
  __syncthreads();
  const int before = wid > 0 ? s_tmp[wid - 1] : -1;
  __syncthreads();
  return max(before, excl);
}

// count(X) = #{ j in [0, P) : j W + U0 < X }, exact.
__device__ __forceinline__ int resample_count(long long X, long long W, long long U0, int P) {
  if (X <= U0) return 0;
  int n = (int)ceilf(__ll2float_rn(X - U0) / __ll2float_rn(W));
  n = n < 0 ? 0 : (n > P ? P : n);
  while (n > 0 && (long long)(n - 1) * W + U0 >= X) --n;
  while (n < P && (long long)n * W + U0 < X) ++n;
  return n;
}

// Resample map of one filter.  w[q] = max-normalised weight of particle
// base + q (0 for slots >= P).  Writes idx[q] for outputs base + q.
template <int NT, int PPT>
__device__ __forceinline__ void resample_map(const float (&w)[PPT], int base, int P, uint64_t u64, int* s_mark,
                                             long long* s_ll, int* s_int, int (&idx)[PPT]) {
  long long incl[PPT];
  long long acc = 0;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    acc += __float2ll_rd(w[q] * 274877906944.0f);  // floor(w 2^38), exact
    incl[q] = acc;
  }
  long long W;
  const long long excl = block_excl_scan<NT>(acc, s_ll, W);
  const long long U0 = (long long)__umul64hi(u64, (unsigned long long)W);
#pragma unroll
  for (int q = 0; q < PPT; ++q)
    if (base + q < P) s_mark[base + q] = -1;
  __syncthreads();
  int lo = resample_count((long long)P * excl, W, U0, P);
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    if (base + q < P) {
      const int hi = resample_count((long long)P * (excl + incl[q]), W, U0, P);
      if (hi > lo) s_mark[lo] = base + q;
      lo = hi;
    }
  }
  __syncthreads();
  int run = -1;
  int m[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    m[q] = base + q < P ? s_mark[base + q] : -1;
    run = max(run, m[q]);
  }
  int before = block_excl_max<NT>(run, s_int);
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    before = max(before, m[q]);
    // Only non-finite weights can leave an output unowned; keep the particle.
    idx[q] = (before >= 0 && before < P) ? before : min(base + q, P - 1);
  }
}

struct PfShared {
  float red[3 * 32];
  long long ll[32];
  int in[32];
  float4 meas[kMaxAgents];
  float tgt[3];
  int nm;
  unsigned long long u64;
};

template <int NT, int PPT, bool VEC>
__global__ void __launch_bounds__(NT) pf_step_kernel(EnvDev d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s_part = reinterpret_cast<float4*>(smem_raw);   // [NT*PPT]
  int* s_mark = reinterpret_cast<int*>(s_part + NT * PPT);  // [NT*PPT]
  __shared__ PfShared sh;

  const int tid = threadIdx.x;
  const int f = blockIdx.x;
  const int P = d.P;
  const uint32_t g = d.counters[0] + 1u;
  const int base = tid * PPT;
  const long long off = (long long)f * P;

  if (tid == 0) {
    sh.nm = d.meas_n[f];
    const int it = d.filt_target[f];
    sh.tgt[0] = d.tx[it];
    sh.tgt[1] = d.ty[it];
    sh.tgt[2] = d.tz[it];
    Rand4 r = philox((uint32_t)f, 0u, g, TAG_RESAMPLE, d.seed);
    sh.u64 = (unsigned long long)r.x[0] | ((unsigned long long)r.x[1] << 32);
  }
  if (tid < d.AM) sh.meas[tid] = d.meas[(long long)f * d.AM + tid];

  float x[PPT], y[PPT], vx[PPT], vy[PPT];
  if (VEC) {
#pragma unroll
    for (int q = 0; q < PPT; q += 4) {
      if (base + q < P) {
        const float4 a = *reinterpret_cast<const float4*>(d.px + off + base + q);
        const float4 b = *reinterpret_cast<const float4*>(d.py + off + base + q);
        const float4 c = *reinterpret_cast<const float4*>(d.pvx + off + base + q);
        const float4 e = *reinterpret_cast<const float4*>(d.pvy + off + base + q);
        x[q] = a.x; x[q + 1] = a.y; x[q + 2] = a.z; x[q + 3] = a.w;
        y[q] = b.x; y[q + 1] = b.y; y[q + 2] = b.z; y[q + 3] = b.w;
        vx[q] = c.x; vx[q + 1] = c.y; vx[q + 2] = c.z; vx[q + 3] = c.w;
        vy[q] = e.x; vy[q + 1] = e.y; vy[q + 2] = e.z; vy[q + 3] = e.w;
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t) x[q + t] = y[q + t] = vx[q + t] = vy[q + t] = 0.0f;
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const bool in = base + q < P;
      x[q] = in ? d.px[off + base + q] : 0.0f;
      y[q] = in ? d.py[off + base + q] : 0.0f;
      vx[q] = in ? d.pvx[off + base + q] : 0.0f;
      vy[q] = in ? d.pvy[off + base + q] : 0.0f;
    }
  }

  // predict: particles 2m and 2m+1 share one Philox call
#pragma unroll
  for (int q = 0; q < PPT; q += 2) {
    const int i = base + q;
    float n[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (i < P) {
      Rand4 r = philox((uint32_t)f, (uint32_t)(i >> 1), g, TAG_PF_PREDICT, d.seed);
      box_muller(r.x[0], r.x[1], n[0], n[1]);
      box_muller(r.x[2], r.x[3], n[2], n[3]);
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int qq = q + t;
      float ux = vx[qq] + d.pf_accel_sigma * n[2 * t];
      float uy = vy[qq] + d.pf_accel_sigma * n[2 * t + 1];
      const float sp = sqrtf(ux * ux + uy * uy);
      if (sp > d.pf_vcap) {
        const float sc = d.pf_vcap / sp;
        ux *= sc;
        uy *= sc;
      }
      vx[qq] = ux;
      vy[qq] = uy;
      x[qq] += d.dt * ux;
      y[qq] += d.dt * uy;
    }
  }
  __syncthreads();  // sh.* visible

  // weight (log domain)
  const int nm = sh.nm;
  const float zt = sh.tgt[2];
  float l[PPT];
  float lmax = -INFINITY;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    float acc = 0.0f;
    for (int m = 0; m < nm; ++m) {
      const float4 mm = sh.meas[m];
      const float dx = x[q] - mm.x, dy = y[q] - mm.y, dz = zt - mm.z;
      const float res = mm.w - sqrtf(dx * dx + dy * dy + dz * dz);
      acc += res * res;
    }
    l[q] = -acc * d.inv_two_s2;
    if (base + q < P) lmax = fmaxf(lmax, l[q]);
  }
  lmax = block_max<NT>(lmax, sh.red);
  float w[PPT];
  float sw = 0.0f, swx = 0.0f, swy = 0.0f;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    w[q] = base + q < P ? expf(l[q] - lmax) : 0.0f;
    sw += w[q];
    swx += w[q] * x[q];
    swy += w[q] * y[q];
  }
  block_sum3<NT>(sw, swx, swy, sh.red);

  // estimate
  if (tid == 0) {
    const float ex = swx / sw, ey = swy / sw;
    d.estx[f] = ex;
    d.esty[f] = ey;
    const float dx = ex - sh.tgt[0], dy = ey - sh.tgt[1];
    d.err[f] = sqrtf(dx * dx + dy * dy);
  }
  if (d.debug_on) {
    const float inv = 1.0f / sw;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      if (base + q < P) {
        d.dbg_px[off + base + q] = x[q];
        d.dbg_py[off + base + q] = y[q];
        d.dbg_pvx[off + base + q] = vx[q];
        d.dbg_pvy[off + base + q] = vy[q];
        d.dbg_w[off + base + q] = w[q] * inv;
        d.dbg_wmax[off + base + q] = w[q];
      }
    }
  }

  int idx[PPT];
  if (nm > 0) {
#pragma unroll
    for (int q = 0; q < PPT; ++q)
      if (base + q < P) s_part[base + q] = make_float4(x[q], y[q], vx[q], vy[q]);
    resample_map<NT, PPT>(w, base, P, sh.u64, s_mark, sh.ll, sh.in, idx);
    // (resample_map ends with barriers, so s_part is complete here)
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      if (base + q < P) {
        const float4 pnew = s_part[idx[q]];
        x[q] = pnew.x;
        y[q] = pnew.y;
        vx[q] = pnew.z;
        vy[q] = pnew.w;
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < PPT; ++q) idx[q] = base + q;
  }
  if (d.debug_on) {
#pragma unroll
    for (int q = 0; q < PPT; ++q)
      if (base + q < P) d.dbg_idx[off + base + q] = idx[q];
  }

  // write back
  if (VEC) {
#pragma unroll
    for (int q = 0; q < PPT; q += 4) {
      if (base + q < P) {
        *reinterpret_cast<float4*>(d.px + off + base + q) = make_float4(x[q], x[q + 1], x[q + 2], x[q + 3]);
        *reinterpret_cast<float4*>(d.py + off + base + q) = make_float4(y[q], y[q + 1], y[q + 2], y[q + 3]);
        *reinterpret_cast<float4*>(d.pvx + off + base + q) = make_float4(vx[q], vx[q + 1], vx[q + 2], vx[q + 3]);
        *reinterpret_cast<float4*>(d.pvy + off + base + q) = make_float4(vy[q], vy[q + 1], vy[q + 2], vy[q + 3]);
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      if (base + q < P) {
        d.px[off + base + q] = x[q];
        d.py[off + base + q] = y[q];
        d.pvx[off + base + q] = vx[q];
        d.pvy[off + base + q] = vy[q];
      }
    }
  }
}

// Stand-alone resample map (same device code as the fused step).
template <int NT, int PPT>
__global__ void __launch_bounds__(NT) pf_resample_kernel(const float* __restrict__ wmax,
                                                          const uint64_t* __restrict__ u64, int P,
                                                          int32_t* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* s_mark = reinterpret_cast<int*>(smem_raw);
  __shared__ long long s_ll[32];
  __shared__ int s_in[32];
  const long long f = blockIdx.x;
  const int base = threadIdx.x * PPT;
  float w[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) w[q] = base + q < P ? wmax[f * P + base + q] : 0.0f;
  int idx[PPT];
  resample_map<NT, PPT>(w, base, P, u64[f], s_mark, s_ll, s_in, idx);
#pragma unroll
  for (int q = 0; q < PPT; ++q)
    if (base + q < P) out[f * P + base + q] = idx[q];
}

// ---------------------------------------------------------------------------
// Variants: (threads per filter, particles per thread).
// ---------------------------------------------------------------------------
struct Variant {
  int nt, ppt;
  const char* name;
};
constexpr Variant kVariants[] = {
    {32, 4, "nt32x4"},   {64, 4, "nt64x4"},   {128, 4, "nt128x4"}, {256, 4, "nt256x4"},
    {512, 4, "nt512x4"}, {1024, 4, "nt1024x4"}, {64, 8, "nt64x8"}, {128, 8, "nt128x8"},
    {256, 8, "nt256x8"}, {512, 8, "nt512x8"},
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

// Opt in to the dynamic shared memory a kernel needs (once per process; the
// first call happens outside any graph capture, at handle creation).
template <typename K>
cudaError_t ensure_smem(K k, size_t smem, int& done) {
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done = 1;
  return e;
}

template <int NT, int PPT>
cudaError_t launch_t(const EnvDev& d, cudaStream_t s) {
  static int ready_vec = 0, ready_scalar = 0;
  const size_t smem = (size_t)NT * PPT * (sizeof(float4) + sizeof(int));
  if (d.P % 4 == 0) {
    auto k = pf_step_kernel<NT, PPT, true>;
    cudaError_t e = ensure_smem(k, smem, ready_vec);
    if (e != cudaSuccess) return e;
    if (d.F > 0) k<<<d.F, NT, smem, s>>>(d);
  } else {
    auto k = pf_step_kernel<NT, PPT, false>;
    cudaError_t e = ensure_smem(k, smem, ready_scalar);
    if (e != cudaSuccess) return e;
    if (d.F > 0) k<<<d.F, NT, smem, s>>>(d);
  }
  return cudaGetLastError();
}

template <int NT, int PPT>
cudaError_t launch_resample_t(const float* w, const uint64_t* u, int64_t F, int P, int32_t* idx, cudaStream_t s) {
  static int ready = 0;
  const size_t smem = (size_t)NT * PPT * sizeof(int);
  auto k = pf_resample_kernel<NT, PPT>;
  cudaError_t e = ensure_smem(k, smem, ready);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)F, NT, smem, s>>>(w, u, P, idx);
  return cudaGetLastError();
}

}  // namespace

int pf_variant_count() { return kNumVariants; }
const char* pf_variant_name(int v) { return (v >= 0 && v < kNumVariants) ? kVariants[v].name : "?"; }
bool pf_variant_valid(int v, int P) {
  if (v < 0 || v >= kNumVariants) return false;
  const int cap = kVariants[v].nt * kVariants[v].ppt;
  // enough slots, and no thread entirely idle beyond one partial warp
  return cap >= P && cap - P < kVariants[v].ppt * 32 + kVariants[v].ppt * (kVariants[v].nt / 2);
}
int pf_default_variant(int P) {
  // smallest PPT=4 block that covers P
  for (int v = 0; v < 6; ++v)
    if (kVariants[v].nt * 4 >= P) return v;
  return 5;
}

cudaError_t launch_pf_step(const EnvDev& d, int variant, cudaStream_t s) {
  switch (variant) {
    case 0: return launch_t<32, 4>(d, s);
    case 1: return launch_t<64, 4>(d, s);
    case 2: return launch_t<128, 4>(d, s);
    case 3: return launch_t<256, 4>(d, s);
    case 4: return launch_t<512, 4>(d, s);
    case 5: return launch_t<1024, 4>(d, s);
    case 6: return launch_t<64, 8>(d, s);
    case 7: return launch_t<128, 8>(d, s);
    case 8: return launch_t<256, 8>(d, s);
    case 9: return launch_t<512, 8>(d, s);
    default: return cudaErrorInvalidValue;
  }
}

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
