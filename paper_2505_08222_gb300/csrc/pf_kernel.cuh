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
//   estimate  weighted mean before resampling, the weight total taken as
//             the exact integer total W below times 2^-38          (C6)
//   resample  q_i = floor(w_i 2^38) (exact), int64 block scan -> Q, W (the
//             scan also carries the estimate's sums); U0 = mulhi(u64, W);
//             particle i owns the outputs [count(P Q_{i-1}), count(P Q_i))
//             with count(X) = #{j : j W + U0 < X}; its index is written at
//             the first owned output and a block prefix-max fills the rest;
//             gather from shared memory.                            (C4, C5)
// The resample map is independent of summation order: given the weights and
// the offset it is bit-identical to the definition
// idx_j = min{i : P Q_i > j W + U0}.  count is evaluated in FP32 from a
// running FP32 weight sum whose error is bounded (resample_map); where the
// FP32 value lies within that bound of an integer, int64 arithmetic decides.
//
// Transcendentals in the per-particle loop use the SFU approximations
// (lg2 / ex2 / sin / cos / sqrt .approx): their relative errors (~1e-7) are
// far inside the parity tolerances, and they cut the instruction count of the
// step, which is what bounds it.
#pragma once

#include "env.cuh"
#include "f32x2.cuh"

namespace ut {
namespace pf {

// 4-byte asynchronous global -> shared copy, and the wait for all of the
// calling thread's copies.
__device__ __forceinline__ void cp_async4(float* dst_smem, const float* src) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(dst_smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(a), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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

// Cross-warp scratch of the block-wide reductions (each array used once per
// CTA, so no reduction needs a trailing barrier).
struct ScanScratch {
  float max[32];
  long long tot[32], pre[32];  // pre[NW - 1] = the block total W after the scan
  float fx[32], fy[32], fsum[2];
  int mtot[32];
  unsigned long long u64;  // the filter's resampling draw
  unsigned long long e1[32], e2[32];  // per-warp ESS sums (resampling trigger)
};

// Warp maximum on the warp reduction unit (NaN inputs ignored, as by fmaxf).
__device__ __forceinline__ float warp_max_redux(float v) {
  float r;
  asm("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}

// Block maximum.
template <int NT>
__device__ __forceinline__ float block_max(float v, ScanScratch* sc) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_max_redux(v);
  if (NW == 1) return v;
  if (lane == 0) sc->max[wid] = v;
  __syncthreads();
  return warp_max_redux(lane < NW ? sc->max[lane] : -INFINITY);
}

// Resampling trigger (pf_ess_num = k > 0): with r = floor(w 2^15) of the
// max-normalised weights (the integer weight floor(w 2^38) shifted right by
// 23), resample iff 16 (sum r)^2 < k P sum r^2, i.e. the effective sample
// size (sum r)^2 / sum r^2 is below k/16 of P.  Exact integers: sum r <=
// 2^27, sum r^2 <= 2^42, both sides below 2^59.  One exchange through shared
// memory; every warp reduces the warp sums itself, so the decision is the
// same in all of them.  sc->e1 / e2 are used once per CTA.
template <int NT>
__device__ __forceinline__ bool block_ess_trigger(unsigned long long s1, unsigned long long s2, int k, int P,
                                                  ScanScratch* sc) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (NW > 1) {
    if (lane == 0) {
      sc->e1[wid] = s1;
      sc->e2[wid] = s2;
    }
    __syncthreads();
    s1 = lane < NW ? sc->e1[lane] : 0ull;
    s2 = lane < NW ? sc->e2[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
  }
  return 16ull * s1 * s1 < (unsigned long long)k * (unsigned long long)P * s2;
}

// Exclusive block scan of the int64 v (returned; the block total in W),
// fused with the block sums of fx and fy (returned in place, and kept in
// sc->fsum): one exchange through shared memory; the cross-warp scan and the
// two sums run on three different warps.
template <int NT>
__device__ __forceinline__ long long block_scan_sums(long long v, float& fx, float& fy, ScanScratch* sc,
                                                     long long& W) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  fx = warp_sum(fx);
  fy = warp_sum(fy);
  if (NW == 1) {
    W = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 0) {  // ordered by the caller's __syncwarp
      sc->pre[0] = W;
      sc->fsum[0] = fx;
      sc->fsum[1] = fy;
    }
    return incl - v;
  }
  if (lane == 31) {
    sc->tot[wid] = incl;
    sc->fx[wid] = fx;
    sc->fy[wid] = fy;
  }
  __syncthreads();
  constexpr int WX = NW >= 2 ? 1 : 0, WY = NW >= 3 ? 2 : WX;
  if (wid == 0) {
    long long t = lane < NW ? sc->tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    if (lane < NW) sc->pre[lane] = t;
  }
  if (wid == WX) {
    const float a = warp_sum(lane < NW ? sc->fx[lane] : 0.0f);
    if (lane == 0) sc->fsum[0] = a;
  }
  if (wid == WY) {
    const float b = warp_sum(lane < NW ? sc->fy[lane] : 0.0f);
    if (lane == 0) sc->fsum[1] = b;
  }
  __syncthreads();
  W = sc->pre[NW - 1];
  fx = sc->fsum[0];
  fy = sc->fsum[1];
  return (wid > 0 ? sc->pre[wid - 1] : 0) + incl - v;
}

// The nearest marker before each thread's outputs (-1 if none), given the
// last marker among the thread's own outputs (run, -1 if none).  Markers are
// particle indices placed at increasing output positions in increasing
// particle order, so the nearest earlier marker is also the largest: within
// the warp it comes from the nearest lower lane that holds one (a ballot and
// one shuffle), across warps from the maximum of the earlier warps' last
// markers (warp reductions).  sc->mtot is used once per CTA.
template <int NT>
__device__ __forceinline__ int block_prev_marker(int run, ScanScratch* sc) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned below = __ballot_sync(0xffffffffu, run >= 0) & ((1u << lane) - 1u);
  const int from = __shfl_sync(0xffffffffu, run, (31 - __clz(below)) & 31);
  const int excl = below ? from : -1;
  if (NW == 1) return excl;
  const int last = __reduce_max_sync(0xffffffffu, run);
  if (lane == 0) sc->mtot[wid] = last;
  __syncthreads();
  const int prev = __reduce_max_sync(0xffffffffu, lane < wid ? sc->mtot[lane] : -1);
  return max(prev, excl);
}

// Shared-memory slot of particle i: thread t's PPT particles are spread NT
// apart so that a warp's stores of "its q-th particle" are consecutive.
template <int NT, int PPT>
__device__ __forceinline__ int slot_of(int i) {
  return (i % PPT) * NT + i / PPT;
}

// Markers of the thread's PPT outputs set to -1 (vector stores; slots >= P
// are never read).  Must precede the block barrier of the scan.
template <int PPT>
__device__ __forceinline__ void init_markers(int* s_mark, int base) {
#pragma unroll
  for (int q = 0; q < PPT; q += 4) *reinterpret_cast<int4*>(s_mark + base + q) = make_int4(-1, -1, -1, -1);
}

// Exact integer weight floor(w 2^38) (w in [0, 1]).
__device__ __forceinline__ long long qweight(float w) { return __float2ll_rd(w * 274877906944.0f); }

// count at the boundary after the thread's first nq particles, from its FP32
// estimate v of D / W with D = P C - U0, U0 = mulhi(u64, W), C = excl + the
// integer weights of those particles: count = clamp(ceil(D / W), 0, P).
// If v lies within eps of an integer m, |D / W - m| < 2 eps < 1/2 and
// D <= m W decides between m and m + 1 exactly; otherwise
// ceil(v) = ceil(D / W).  The exact branch is rare: it reads the thread's
// excl and weights (s_w [PPT]), W and u64 from shared memory and rebuilds C,
// so that none of them holds a register through the common path.
template <int PPT>
__device__ __forceinline__ int count_at(float v, float eps, const float* s_w, int nq, const long long* s_excl,
                                        const ScanScratch* sc, int NW, int P) {
  const float r = rintf(v);
  int n;
  if (fabsf(v - r) < eps) {
    const long long W = sc->pre[NW - 1];
    const long long U0 = (long long)__umul64hi(sc->u64, (unsigned long long)W);
    long long C = *s_excl;
#pragma unroll
    for (int t = 0; t < PPT; ++t)
      if (t < nq) C += qweight(s_w[t]);
    const long long D = (long long)P * C - U0;
    const int m = (int)r;
    n = (D <= (long long)m * W) ? m : m + 1;
  } else {
    n = __float2int_ru(v);
  }
  return min(max(n, 0), P);
}

// Resample map of one filter.  w[q] = max-normalised weight of particle
// base + q (0 for slots >= P); excl = the sum of the integer weights
// floor(w 2^38) over all earlier threads, W = their total (block_scan_sums,
// which also left W in sc->pre[NW - 1]); sc->u64 holds the filter's draw;
// s_excl [NT] and s_w [NT*PPT] are scratch; the markers are -1
// (init_markers) and the scan's barrier has passed.  Writes idx[q] for
// outputs base + q.
//
// FP32 bound of v = fma(a, cw, b) against D / W, with u = 2^-24, W >= 2^38
// (the heaviest particle has w = 1) so that a = P 2^38 / W <= P:
// a carries 3u relative error, the running sum cw of PPT weights in [0, 1]
// (PPT - 1)u, the product 1u, so a cw is within (PPT + 3) u P; b = (P excl -
// U0) / W (|b| <= P + 1) within 4u (P + 1); the fma rounds by u (P + 1);
// cw replaces the floored q's by w 2^-38 2^38, which moves v by at most
// P PPT 2^-38.  Total below (PPT + 9) u (P + 1); eps is twice that.
template <int NT, int PPT, bool FULL>
__device__ __forceinline__ void resample_map(const float (&w)[PPT], long long excl, long long W, int base, int P,
                                             long long* s_excl, float* s_w, int* s_mark, ScanScratch* sc,
                                             int (&idx)[PPT], int* status) {
  constexpr int NW = NT / 32;
  const long long U0 = (long long)__umul64hi(sc->u64, (unsigned long long)W);
  const float invW = 1.0f / __ll2float_rn(W);
  const float a = (float)P * 274877906944.0f * invW;
  const float b = __ll2float_rn((long long)P * excl - U0) * invW;
  const float eps = (float)(2 * (PPT + 9)) * 0x1p-24f * (float)(P + 1);
  long long* my_excl = s_excl + threadIdx.x;
  float* my_w = s_w + base;
  *my_excl = excl;  // both read back by this thread only
#pragma unroll
  for (int q = 0; q < PPT; q += 4)
    *reinterpret_cast<float4*>(my_w + q) = make_float4(w[q], w[q + 1], w[q + 2], w[q + 3]);
  int lo = count_at<PPT>(b, eps, my_w, 0, my_excl, sc, NW, P);
  float cw = 0.0f;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    if (FULL || base + q < P) {
      cw += w[q];
      const int hi = count_at<PPT>(fmaf(a, cw, b), eps, my_w, q + 1, my_excl, sc, NW, P);
      if (hi > lo && UT_IN_BOUNDS(lo >= 0 && lo < NT * PPT, status)) s_mark[lo] = base + q;
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
    if (!FULL && base + q >= P) m[q] = -1;
    run = max(run, m[q]);
  }
  int before = block_prev_marker<NT>(run, sc);
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    before = max(before, m[q]);
    // Only non-finite weights can leave an output unowned; keep the particle.
    idx[q] = (before >= 0 && before < P) ? before : min(base + q, P - 1);
  }
}

struct Shared {
  ScanScratch scan;
  float hist[6];  // estx, esty, prev_estx, prev_esty, velx, vely of the filter
  float4 meas[kMaxAgents];  // (qx, qy, (z_target - qz)^2, r)
  float tgt[2];
  float dz2;
  int nm;
};

// One filter's step by the whole CTA (filter f, global step g): stage the
// inputs, load the particles (unless RES), predict, weight, estimate sums,
// resample map and gather, store (unless RES), then thread 0's estimate and
// history writes.  RES: the particles stay in the registers x, y, vx, vy
// across calls (thread t holds particles t * PPT .. t * PPT + PPT - 1), as in
// the persistent rollout; otherwise those arrays are scratch.  MODE 0: any P
// (scalar loads); 1: P % 4 == 0 (float4 streams); 2: P equal to NT * PPT
// (float4 streams, no slot is out of range).  ESS: weights carried across
// steps as log-weights d.pw, resampling only when triggered.  The shared
// memory is the kernel's: a caller that calls it again must put a block
// barrier between the calls.
template <int NT, int PPT, int MODE, bool ESS, bool RES>
__device__ __forceinline__ void pf_step_body(const EnvDev& d, const int f, const uint32_t g, float (&x)[PPT],
                                             float (&y)[PPT], float (&vx)[PPT], float (&vy)[PPT]) {
  static_assert(PPT % 4 == 0, "PPT must be a multiple of 4");
  constexpr bool VEC = MODE >= 1, FULL = MODE == 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s_part = reinterpret_cast<float4*>(smem_raw);                 // [NT*PPT], slot_of layout
  int* s_mark = reinterpret_cast<int*>(s_part + NT * PPT);              // [NT*PPT]
  long long* s_excl = reinterpret_cast<long long*>(s_mark + NT * PPT);  // [NT]
  float* s_w = reinterpret_cast<float*>(s_excl + NT);                  // [NT*PPT]
  __shared__ Shared sh;

  const int tid = threadIdx.x;
  const int P = d.P;
  const int base = tid * PPT;
  const long long off = (long long)f * P;

  // estimate history: thread 0 copies it to shared memory asynchronously
  // and shifts it after the particles are written
  const bool has_hist = d.prev_estx != nullptr, has_vel = d.velx != nullptr;
  if (tid == 0 && has_hist) {
    cp_async4(&sh.hist[0], d.estx + f);
    cp_async4(&sh.hist[1], d.esty + f);
    cp_async4(&sh.hist[2], d.prev_estx + f);
    cp_async4(&sh.hist[3], d.prev_esty + f);
    if (has_vel) {
      cp_async4(&sh.hist[4], d.velx + f);
      cp_async4(&sh.hist[5], d.vely + f);
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
  }
  if (tid == NT - 1) {  // the resampling draw, on the warp with no other extra duty
    Rand4 r = philox(d.gid_filter + (uint32_t)f, 0u, g, TAG_RESAMPLE, d.seed);
    sh.scan.u64 = (unsigned long long)r.x[0] | ((unsigned long long)r.x[1] << 32);
  }

  if (RES) {
  } else if (VEC) {
#pragma unroll
    for (int q = 0; q < PPT; q += 4) {
      if (FULL || base + q < P) {
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
    if (FULL || i < P) {
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
  const int nm = UT_IN_BOUNDS(sh.nm >= 0 && sh.nm <= d.AM && d.AM <= kMaxAgents, d.status) ? sh.nm : 0;
  const float dz2 = sh.dz2;
  float pwv[PPT];  // carried log-weights (ESS form)
  if (ESS) {
#pragma unroll
    for (int q = 0; q < PPT; ++q) pwv[q] = (FULL || base + q < P) ? d.pw[off + base + q] : 0.0f;
  }
  float acc[PPT];
  {
    // particle pairs on the packed FP32 pipe: each lane rounds like the scalar
    // operation, in the same order; (sqrt - r)^2 equals (r - sqrt)^2 bit for
    // bit because rounding is symmetric.  Positions live only in packed form
    // through the loop.
    unsigned long long X[PPT / 2], Y[PPT / 2], A[PPT / 2];
#pragma unroll
    for (int h = 0; h < PPT / 2; ++h) {
      X[h] = f2pk(x[2 * h], x[2 * h + 1]);
      Y[h] = f2pk(y[2 * h], y[2 * h + 1]);
      A[h] = 0ull;
    }
    const unsigned long long DZ2 = f2pk(dz2, dz2);
    for (int m = 0; m < nm; ++m) {
      const float4 mm = sh.meas[m];
      const unsigned long long MX = f2pk(-mm.x, -mm.x), MY = f2pk(-mm.y, -mm.y), NR = f2pk(-mm.w, -mm.w);
#pragma unroll
      for (int h = 0; h < PPT / 2; ++h) {
        const unsigned long long dx = f2add(X[h], MX), dy = f2add(Y[h], MY);
        float s0, s1;
        f2upk(f2fma(dx, dx, f2fma(dy, dy, DZ2)), s0, s1);
        const unsigned long long res = f2add(f2pk(sqrt_approx(s0), sqrt_approx(s1)), NR);
        A[h] = f2fma(res, res, A[h]);
      }
    }
#pragma unroll
    for (int h = 0; h < PPT / 2; ++h) {
      f2upk(A[h], acc[2 * h], acc[2 * h + 1]);
      f2upk(X[h], x[2 * h], x[2 * h + 1]);
      f2upk(Y[h], y[2 * h], y[2 * h + 1]);
    }
  }
  float lmax = -INFINITY;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    // log-likelihood (plus the carried log-weight in the ESS form)
    acc[q] = ESS ? fmaf(-acc[q], d.inv_two_s2, pwv[q]) : -acc[q] * d.inv_two_s2;
    if (FULL || base + q < P) lmax = fmaxf(lmax, acc[q]);
  }
  lmax = block_max<NT>(lmax, &sh.scan);
  // max-normalised weights, their exact integer images floor(w 2^38) summed
  // per thread, and the estimate's weighted sums
  float w[PPT];
  long long qsum = 0;
  float swx = 0.0f, swy = 0.0f;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    w[q] = (FULL || base + q < P) ? __expf(acc[q] - lmax) : 0.0f;
    swx = fmaf(w[q], x[q], swx);
    swy = fmaf(w[q], y[q], swy);
    qsum += qweight(w[q]);
  }
  if (d.debug_on) {  // pre-resample state and weights (normalised below)
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      if (FULL || base + q < P) {
        d.dbg_px[off + base + q] = x[q];
        d.dbg_py[off + base + q] = y[q];
        d.dbg_pvx[off + base + q] = vx[q];
        d.dbg_pvy[off + base + q] = vy[q];
        d.dbg_wmax[off + base + q] = w[q];
      }
    }
  }
  // ESS form: the trigger, then the new log-weights (0 after a resample,
  // log w - max log w otherwise)
  bool resample = nm > 0;
  if (ESS) {
    unsigned long long s1 = 0ull, s2 = 0ull;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const unsigned long long r = (unsigned long long)(qweight(w[q]) >> 23);
      s1 += r;
      s2 += r * r;
    }
    resample = block_ess_trigger<NT>(s1, s2, d.pf_ess_num, P, &sh.scan) && nm > 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q)
      if (FULL || base + q < P) d.pw[off + base + q] = resample ? 0.0f : acc[q] - lmax;
  }
  // the branch condition is the same for the whole CTA, so both branches
  // keep their barriers uniform; the particles are dead across the scan in
  // the resampling branch
  long long W;
  int idx[PPT];
  if (resample) {
#pragma unroll
    for (int q = 0; q < PPT; ++q) s_part[q * NT + tid] = make_float4(x[q], y[q], vx[q], vy[q]);
    init_markers<PPT>(s_mark, base);
    const long long excl = block_scan_sums<NT>(qsum, swx, swy, &sh.scan, W);  // contains barriers
    if (NT == 32) __syncwarp();  // single-warp blocks: order the shared-memory stores
    resample_map<NT, PPT, FULL>(w, excl, W, base, P, s_excl, s_w, s_mark, &sh.scan, idx, d.status);
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int sl = slot_of<NT, PPT>(idx[q]);
      const float4 pnew = UT_IN_BOUNDS(sl >= 0 && sl < NT * PPT, d.status) ? s_part[sl] : make_float4(0.f, 0.f, 0.f, 0.f);
      x[q] = pnew.x;
      y[q] = pnew.y;
      vx[q] = pnew.z;
      vy[q] = pnew.w;
    }
  } else {
    block_scan_sums<NT>(qsum, swx, swy, &sh.scan, W);
    if (NT == 32) __syncwarp();
#pragma unroll
    for (int q = 0; q < PPT; ++q) idx[q] = base + q;
  }
  if (d.debug_on) {
    const float inv = 1.0f / (__ll2float_rn(W) * 0x1p-38f);
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      if (FULL || base + q < P) {
        d.dbg_w[off + base + q] = w[q] * inv;
        d.dbg_idx[off + base + q] = idx[q];
      }
    }
  }

  // write back (streaming stores: the state is not reread this step)
  if (RES) {
  } else if (VEC) {
#pragma unroll
    for (int q = 0; q < PPT; q += 4) {
      if (FULL || base + q < P) {
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
  // estimate (from the block sums and the integer weight total, both left in
  // shared memory by the scan) and the history shift by one update, after
  // the particles: no barrier waits for thread 0 here
  if (tid == 0) {
    if (has_hist) {
      cp_async_wait_all();  // thread 0's own copies
      const float* h = sh.hist;
      d.prev2_estx[f] = h[2];
      d.prev2_esty[f] = h[3];
      d.prev_estx[f] = h[0];
      d.prev_esty[f] = h[1];
      if (has_vel) {  // motion of the previous update folded into the smoothed velocity
        d.velx[f] = fmaf(kVelKeep, h[4], (1.0f - kVelKeep) * (h[0] - h[2]));
        d.vely[f] = fmaf(kVelKeep, h[5], (1.0f - kVelKeep) * (h[1] - h[3]));
      }
    }
    const float sw = __ll2float_rn(sh.scan.pre[NT / 32 - 1]) * 0x1p-38f;
    const float ex = sh.scan.fsum[0] / sw, ey = sh.scan.fsum[1] / sw;
    d.estx[f] = ex;
    d.esty[f] = ey;
    const float dx = ex - sh.tgt[0], dy = ey - sh.tgt[1];
    d.err[f] = sqrtf(dx * dx + dy * dy);
  }
}

// Particles of filter f into / out of registers (the persistent rollout's
// resident form; the same accesses as pf_step_body's).
template <int NT, int PPT, int MODE>
__device__ __forceinline__ void load_particles(const EnvDev& d, int f, float (&x)[PPT], float (&y)[PPT],
                                               float (&vx)[PPT], float (&vy)[PPT]) {
  constexpr bool VEC = MODE >= 1, FULL = MODE == 2;
  const int P = d.P;
  const int base = threadIdx.x * PPT;
  const long long off = (long long)f * P;
  if (VEC) {
#pragma unroll
    for (int q = 0; q < PPT; q += 4) {
      if (FULL || base + q < P) {
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
}

template <int NT, int PPT, int MODE>
__device__ __forceinline__ void store_particles(const EnvDev& d, int f, const float (&x)[PPT], const float (&y)[PPT],
                                                const float (&vx)[PPT], const float (&vy)[PPT]) {
  constexpr bool VEC = MODE >= 1, FULL = MODE == 2;
  const int P = d.P;
  const int base = threadIdx.x * PPT;
  const long long off = (long long)f * P;
  if constexpr (VEC) {
#pragma unroll
    for (int q = 0; q < PPT; q += 4) {
      if (FULL || base + q < P) {
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

template <int NT, int PPT, int MINB, int MODE, bool ESS>
__global__ void __launch_bounds__(NT, MINB) pf_step_kernel(EnvDev d) {
  pdl_wait();  // (dependents launch as this grid's CTAs exit: no early trigger in a many-wave kernel)
  float x[PPT], y[PPT], vx[PPT], vy[PPT];
  pf_step_body<NT, PPT, MODE, ESS, false>(d, (int)blockIdx.x, d.counters[0] + 1u, x, y, vx, vy);
}

// Stand-alone resample map (same device code as the fused step).
template <int NT, int PPT>
__global__ void __launch_bounds__(NT) pf_resample_kernel(const float* __restrict__ wmax,
                                                          const uint64_t* __restrict__ u64, int P,
                                                          int32_t* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* s_mark = reinterpret_cast<int*>(smem_raw);                       // [NT*PPT]
  long long* s_excl = reinterpret_cast<long long*>(s_mark + NT * PPT);  // [NT]
  float* s_w = reinterpret_cast<float*>(s_excl + NT);                  // [NT*PPT]
  __shared__ ScanScratch s_scan;
  const long long f = blockIdx.x;
  if (threadIdx.x == 0) s_scan.u64 = u64[f];  // ordered by the scan's barriers
  const int base = threadIdx.x * PPT;
  float w[PPT];
  long long qsum = 0;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    w[q] = base + q < P ? wmax[f * P + base + q] : 0.0f;
    qsum += qweight(w[q]);
  }
  init_markers<PPT>(s_mark, base);
  float fx = 0.0f, fy = 0.0f;
  long long W;
  const long long excl = block_scan_sums<NT>(qsum, fx, fy, &s_scan, W);
  if (NT == 32) __syncwarp();
  int idx[PPT];
  resample_map<NT, PPT, false>(w, excl, W, base, P, s_excl, s_w, s_mark, &s_scan, idx, nullptr);
#pragma unroll
  for (int q = 0; q < PPT; ++q)
    if (base + q < P) out[f * P + base + q] = idx[q];
}

// Dynamic shared memory of the step (particles, markers, per-thread excl,
// weights) and of the stand-alone resample map (markers, excl, weights).
constexpr size_t step_smem_bytes(int NT, int PPT) {
  return (size_t)NT * PPT * (sizeof(float4) + 2 * sizeof(int)) + (size_t)NT * sizeof(long long);
}
constexpr size_t resample_smem_bytes(int NT, int PPT) {
  return (size_t)NT * PPT * 2 * sizeof(int) + (size_t)NT * sizeof(long long);
}

template <int NT, int PPT, int MINB, int MODE, bool ESS>
cudaError_t launch_mode(const EnvDev& d, cudaStream_t s) {
  static std::atomic<unsigned long long> ready{0};
  const size_t smem = step_smem_bytes(NT, PPT);
  auto k = pf_step_kernel<NT, PPT, MINB, MODE, ESS>;
  cudaError_t e = smem_optin(k, smem, ready);
  if (e != cudaSuccess) return e;
  if (d.F > 0) return launch_pdl(k, dim3(d.F), dim3(NT), smem, s, d);
  return cudaSuccess;
}

// Requires NT * PPT >= P (the variant check).
template <int NT, int PPT, int MINB>
cudaError_t launch_step(const EnvDev& d, cudaStream_t s) {
  if (d.P > NT * PPT) return cudaErrorInvalidValue;
  if (d.pw) {
    if (d.P == NT * PPT) return launch_mode<NT, PPT, MINB, 2, true>(d, s);
    if (d.P % 4 == 0) return launch_mode<NT, PPT, MINB, 1, true>(d, s);
    return launch_mode<NT, PPT, MINB, 0, true>(d, s);
  }
  if (d.P == NT * PPT) return launch_mode<NT, PPT, MINB, 2, false>(d, s);
  if (d.P % 4 == 0) return launch_mode<NT, PPT, MINB, 1, false>(d, s);
  return launch_mode<NT, PPT, MINB, 0, false>(d, s);
}

}  // namespace pf
}  // namespace ut
