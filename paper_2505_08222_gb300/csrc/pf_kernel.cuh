// Particle-filter step kernel (template), shared by the instantiation units.
//
// One CTA per filter (one filter per (env, observer agent, target),
// Sec. III-A.2), NT threads x PPT consecutive particles each.  The filter's
// particles make exactly one round trip through HBM per step: 16 B read
// (x, y, vx, vy as four coalesced float4 streams) and 16 B written.  Weights,
// the CDF, the resample map and the gather stay on chip:
//   predict   v += sigma_a N(0, I) (one Philox call per particle pair),
//             |v| capped, p += dt v                                 (reading C2)
//   weight    l_i = -sum_m (r_m - |p_i - q_m|)^2 / (2 sigma_r^2); max by warp
//             shuffles, w_i = exp(l_i - max l), sums by warp shuffles (C3)
//   estimate  weighted mean before resampling                       (C6)
//   resample  q_i = floor(w_i 2^38) (exact), int64 block scan -> Q, W;
//             U0 = mulhi(u64, W); particle i owns the outputs
//             [count(P Q_{i-1}), count(P Q_i)) with
//             count(X) = #{j : j W + U0 < X}; its index is written at the
//             first owned output and a block prefix-max fills the rest;
//             gather from shared memory.                            (C4, C5)
// Integer arithmetic makes the resample map independent of summation order:
// given the weights and the offset it is bit-identical to the definition
// idx_j = min{i : P Q_i > j W + U0}.
//
// Transcendentals in the per-particle loop use the SFU approximations
// (lg2 / ex2 / sin / cos / sqrt .approx): their relative errors (~1e-7) are
// far inside the parity tolerances, and they cut the instruction count of the
// step, which is what bounds it.
#pragma once

#include "env.cuh"

namespace ut {
namespace pf {

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Box-Muller on the SFU: sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2), with the
// angle shifted into [-pi, pi) where the fast sine / cosine are accurate
// (cos t = -cos(t - pi), sin t = -sin(t - pi)).
__device__ __forceinline__ void box_muller_fast(uint32_t va, uint32_t vb, float& n0, float& n1) {
  const float rad = sqrt_approx(-2.0f * __logf(unif_pos(va)));
  float s, c;
  __sincosf(fmaf(kTwoPi, unif(vb), -kPi), &s, &c);
  n0 = -rad * c;
  n1 = -rad * s;
}

template <int NT>
__device__ __forceinline__ float block_max(float v, float* s_tmp) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_max(v);
  if (NW == 1) return v;
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
  if (NW == 1) return;
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
// s_tot / s_pre [32] are used once per CTA (no trailing barrier).
template <int NT>
__device__ __forceinline__ long long block_excl_scan(long long v, long long* s_tot, long long* s_pre,
                                                     long long& total) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (NW == 1) {
    total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - v;
  }
  if (lane == 31) s_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    long long w = lane < NW ? s_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < NW) s_pre[lane] = w;
  }
  __syncthreads();
  total = s_pre[NW - 1];
  return (wid > 0 ? s_pre[wid - 1] : 0) + incl - v;
}

// Maximum over all earlier threads of each thread's value (identity -1).
// s_tot / s_pre [32] are used once per CTA (no trailing barrier).
template <int NT>
__device__ __forceinline__ int block_excl_max(int v, int* s_tot, int* s_pre) {
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
  if (NW == 1) return excl;
  if (lane == 31) s_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < NW ? s_tot[lane] : -1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w = max(w, t);
    }
    if (lane < NW) s_pre[lane] = w;
  }
  __syncthreads();
  return max(wid > 0 ? s_pre[wid - 1] : -1, excl);
}

// Cross-warp scratch of the resample map (each array used once per CTA).
struct ScanScratch {
  long long tot[32], pre[32];
  int mtot[32], mpre[32];
};

// count(X) = #{ j in [0, P) : j W + U0 < X } = clamp(ceil((X - U0) / W), 0, P),
// exact.  A float estimate v = (X - U0) * (1/W) has absolute error below 2e-3
// for v <= 4096; ceil(v) is taken directly unless v lies within 4e-3 of an
// integer, where one int64 comparison decides.
__device__ __forceinline__ int resample_count(long long X, long long W, long long U0, float invW, int P) {
  if (X <= U0) return 0;
  const long long D = X - U0;
  const float v = __ll2float_rn(D) * invW;
  const float r = rintf(v);
  int n;
  if (fabsf(v - r) < 4e-3f) {
    const int m = (int)r;
    n = ((long long)m * W >= D) ? m : m + 1;
  } else {
    n = (int)ceilf(v);
  }
  return n < 0 ? 0 : (n > P ? P : n);
}

// Shared-memory slot of particle i: thread t's PPT particles are spread NT
// apart so that a warp's stores of "its q-th particle" are consecutive.
template <int NT, int PPT>
__device__ __forceinline__ int slot_of(int i) {
  return (i % PPT) * NT + i / PPT;
}

// Resample map of one filter.  w[q] = max-normalised weight of particle
// base + q (0 for slots >= P).  Writes idx[q] for outputs base + q.
template <int NT, int PPT>
__device__ __forceinline__ void resample_map(const float (&w)[PPT], int base, int P, uint64_t u64, int* s_mark,
                                             ScanScratch* sc, int (&idx)[PPT]) {
  long long incl[PPT];
  long long acc = 0;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    acc += __float2ll_rd(w[q] * 274877906944.0f);  // floor(w 2^38), exact
    incl[q] = acc;
  }
  // markers start at -1 (vector stores; slots >= P are never read)
#pragma unroll
  for (int q = 0; q < PPT; q += 4)
    *reinterpret_cast<int4*>(s_mark + base + q) = make_int4(-1, -1, -1, -1);
  long long W;
  const long long excl = block_excl_scan<NT>(acc, sc->tot, sc->pre, W);  // contains barriers
  if (NT == 32) __syncwarp();  // single-warp blocks: order the marker initialisation
  const long long U0 = (long long)__umul64hi(u64, (unsigned long long)W);
  const float invW = 1.0f / __ll2float_rn(W);
  int lo = resample_count((long long)P * excl, W, U0, invW, P);
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    if (base + q < P) {
      const int hi = resample_count((long long)P * (excl + incl[q]), W, U0, invW, P);
      if (hi > lo) s_mark[lo] = base + q;
      lo = hi;
    }
  }
  __syncthreads();
  int m[PPT];
  int run = -1;
#pragma unroll
  for (int q = 0; q < PPT; q += 4) {
    const int4 v = *reinterpret_cast<const int4*>(s_mark + base + q);
    m[q] = v.x; m[q + 1] = v.y; m[q + 2] = v.z; m[q + 3] = v.w;
  }
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    if (base + q >= P) m[q] = -1;
    run = max(run, m[q]);
  }
  int before = block_excl_max<NT>(run, sc->mtot, sc->mpre);
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    before = max(before, m[q]);
    // Only non-finite weights can leave an output unowned; keep the particle.
    idx[q] = (before >= 0 && before < P) ? before : min(base + q, P - 1);
  }
}

struct Shared {
  float red[3 * 32];
  ScanScratch scan;
  float4 meas[kMaxAgents];  // (qx, qy, (z_target - qz)^2, r)
  float tgt[2];
  float dz2;
  int nm;
  unsigned long long u64;
};

template <int NT, int PPT, int MINB, bool VEC>
__global__ void __launch_bounds__(NT, MINB) pf_step_kernel(EnvDev d) {
  static_assert(PPT % 4 == 0, "PPT must be a multiple of 4");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s_part = reinterpret_cast<float4*>(smem_raw);      // [NT*PPT], slot_of layout
  int* s_mark = reinterpret_cast<int*>(s_part + NT * PPT);   // [NT*PPT]
  __shared__ Shared sh;

  const int tid = threadIdx.x;
  const int f = blockIdx.x;
  const int P = d.P;
  const uint32_t g = d.counters[0] + 1u;
  const int base = tid * PPT;
  const long long off = (long long)f * P;

  // estimate history, fetched early so that its latency hides behind the
  // particle loads (thread 0 writes it back before a block barrier)
  float hist[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  if (tid == 0 && d.prev_estx) {
    hist[0] = d.estx[f];
    hist[1] = d.esty[f];
    hist[2] = d.prev_estx[f];
    hist[3] = d.prev_esty[f];
    if (d.velx) {
      hist[4] = d.velx[f];
      hist[5] = d.vely[f];
    }
  }
  // measurement list and the filter's header (senders are at the surface:
  // the vertical offset of every range is the target depth)
  if (tid < d.AM) sh.meas[tid] = d.meas[(long long)f * d.AM + tid];
  if (tid == 0) {
    const float4 hd = d.meas_hdr[f];
    sh.tgt[0] = hd.x;
    sh.tgt[1] = hd.y;
    sh.dz2 = hd.z;
    sh.nm = (int)hd.w;
    Rand4 r = philox(d.gid_filter + (uint32_t)f, 0u, g, TAG_RESAMPLE, d.seed);
    sh.u64 = (unsigned long long)r.x[0] | ((unsigned long long)r.x[1] << 32);
  }

  float x[PPT], y[PPT], vx[PPT], vy[PPT];
  if (VEC) {
#pragma unroll
    for (int q = 0; q < PPT; q += 4) {
      if (base + q < P) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(d.px + off + base + q));
        const float4 b = __ldcs(reinterpret_cast<const float4*>(d.py + off + base + q));
        const float4 c = __ldcs(reinterpret_cast<const float4*>(d.pvx + off + base + q));
        const float4 e = __ldcs(reinterpret_cast<const float4*>(d.pvy + off + base + q));
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
  const float vcap2 = d.pf_vcap * d.pf_vcap;
#pragma unroll
  for (int q = 0; q < PPT; q += 2) {
    const int i = base + q;
    float n[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (i < P) {
      Rand4 r = philox(d.gid_filter + (uint32_t)f, (uint32_t)(i >> 1), g, TAG_PF_PREDICT, d.seed);
      box_muller_fast(r.x[0], r.x[1], n[0], n[1]);
      box_muller_fast(r.x[2], r.x[3], n[2], n[3]);
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int qq = q + t;
      float ux = fmaf(d.pf_accel_sigma, n[2 * t], vx[qq]);
      float uy = fmaf(d.pf_accel_sigma, n[2 * t + 1], vy[qq]);
      const float sp2 = ux * ux + uy * uy;
      if (sp2 > vcap2) {
        const float sc = d.pf_vcap * rsqrtf(sp2);
        ux *= sc;
        uy *= sc;
      }
      vx[qq] = ux;
      vy[qq] = uy;
      x[qq] = fmaf(d.dt, ux, x[qq]);
      y[qq] = fmaf(d.dt, uy, y[qq]);
    }
  }
  __syncthreads();  // sh.* visible

  // weight (log domain); measurements outer, particles inner
  const int nm = sh.nm;
  const float dz2 = sh.dz2;
  float acc[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) acc[q] = 0.0f;
  for (int m = 0; m < nm; ++m) {
    const float4 mm = sh.meas[m];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const float dx = x[q] - mm.x, dy = y[q] - mm.y;
      const float res = mm.w - sqrt_approx(fmaf(dx, dx, fmaf(dy, dy, dz2)));
      acc[q] = fmaf(res, res, acc[q]);
    }
  }
  float lmax = -INFINITY;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    acc[q] = -acc[q] * d.inv_two_s2;  // log-likelihood
    if (base + q < P) lmax = fmaxf(lmax, acc[q]);
  }
  lmax = block_max<NT>(lmax, sh.red);
  float w[PPT];
  float sw = 0.0f, swx = 0.0f, swy = 0.0f;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    w[q] = base + q < P ? __expf(acc[q] - lmax) : 0.0f;
    sw += w[q];
    swx = fmaf(w[q], x[q], swx);
    swy = fmaf(w[q], y[q], swy);
  }
  block_sum3<NT>(sw, swx, swy, sh.red);

  // estimate
  if (tid == 0) {
    const float ex = swx / sw, ey = swy / sw;
    if (d.prev_estx) {  // estimate history: the update's inputs
      d.prev2_estx[f] = hist[2];
      d.prev2_esty[f] = hist[3];
      d.prev_estx[f] = hist[0];
      d.prev_esty[f] = hist[1];
      if (d.velx) {  // motion of the previous update folded into the smoothed velocity
        d.velx[f] = fmaf(kVelKeep, hist[4], (1.0f - kVelKeep) * (hist[0] - hist[2]));
        d.vely[f] = fmaf(kVelKeep, hist[5], (1.0f - kVelKeep) * (hist[1] - hist[3]));
      }
    }
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
    for (int q = 0; q < PPT; ++q) s_part[q * NT + tid] = make_float4(x[q], y[q], vx[q], vy[q]);
    resample_map<NT, PPT>(w, base, P, sh.u64, s_mark, &sh.scan, idx);
    // (resample_map contains barriers after the s_part stores)
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const float4 pnew = s_part[slot_of<NT, PPT>(idx[q])];
      x[q] = pnew.x;
      y[q] = pnew.y;
      vx[q] = pnew.z;
      vy[q] = pnew.w;
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

  // write back (streaming stores: the state is not reread this step)
  if (VEC) {
#pragma unroll
    for (int q = 0; q < PPT; q += 4) {
      if (base + q < P) {
        __stcs(reinterpret_cast<float4*>(d.px + off + base + q), make_float4(x[q], x[q + 1], x[q + 2], x[q + 3]));
        __stcs(reinterpret_cast<float4*>(d.py + off + base + q), make_float4(y[q], y[q + 1], y[q + 2], y[q + 3]));
        __stcs(reinterpret_cast<float4*>(d.pvx + off + base + q),
               make_float4(vx[q], vx[q + 1], vx[q + 2], vx[q + 3]));
        __stcs(reinterpret_cast<float4*>(d.pvy + off + base + q),
               make_float4(vy[q], vy[q + 1], vy[q + 2], vy[q + 3]));
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
  __shared__ ScanScratch s_scan;
  const long long f = blockIdx.x;
  const int base = threadIdx.x * PPT;
  float w[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) w[q] = base + q < P ? wmax[f * P + base + q] : 0.0f;
  int idx[PPT];
  resample_map<NT, PPT>(w, base, P, u64[f], s_mark, &s_scan, idx);
#pragma unroll
  for (int q = 0; q < PPT; ++q)
    if (base + q < P) out[f * P + base + q] = idx[q];
}

// Opt in to the dynamic shared memory a kernel needs (once per process).
template <typename K>
cudaError_t ensure_smem(K k, size_t smem, int& done) {
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done = 1;
  return e;
}

template <int NT, int PPT, int MINB>
cudaError_t launch_step(const EnvDev& d, cudaStream_t s) {
  static int ready_vec = 0, ready_scalar = 0;
  const size_t smem = (size_t)NT * PPT * (sizeof(float4) + sizeof(int));
  if (d.P % 4 == 0) {
    auto k = pf_step_kernel<NT, PPT, MINB, true>;
    cudaError_t e = ensure_smem(k, smem, ready_vec);
    if (e != cudaSuccess) return e;
    if (d.F > 0) k<<<d.F, NT, smem, s>>>(d);
  } else {
    auto k = pf_step_kernel<NT, PPT, MINB, false>;
    cudaError_t e = ensure_smem(k, smem, ready_scalar);
    if (e != cudaSuccess) return e;
    if (d.F > 0) k<<<d.F, NT, smem, s>>>(d);
  }
  return cudaGetLastError();
}

}  // namespace pf
}  // namespace ut
