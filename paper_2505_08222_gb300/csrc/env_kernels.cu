// Environment kernels: reset, move/ping/communicate, observation/reward.
//
// These stages are tiny next to the particle filter (bytes per env-step are
// O(A*T) against O(A*T*P)), so they favour simplicity: one warp per
// environment, entity state staged in shared memory, struct-of-arrays in HBM.
#include "env.cuh"
#include "env_step.cuh"

namespace ut {

namespace {

constexpr int kWarpsPerBlock = 4;

// -------------------------------------------------------------------------
// Reset, part 1: spawn (Sec. III-A.2).  One thread per environment.
// Entities (agents then targets) are placed one after the other by bounded
// rejection on a 2^-16 m integer lattice inside the spawn disk, keeping a
// candidate whose squared distance to every placed entity is at least
// spawn_min^2 (exact integer test); after spawn_tries failures the last
// in-disk candidate is kept.
// -------------------------------------------------------------------------
__global__ void reset_spawn_kernel(EnvDev d, uint32_t g) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  const int a0 = d.agent_off[e], A = d.agent_off[e + 1] - a0;
  const int t0 = d.target_off[e], T = d.target_off[e + 1] - t0;
  long long X[kMaxAgents + kMaxTargets], Y[kMaxAgents + kMaxTargets];
  const long long r2 = d.spawn_r_int * d.spawn_r_int;
  const long long m2 = d.spawn_dmin_int * d.spawn_dmin_int;
  for (int n = 0; n < A + T; ++n) {
    long long cx = 0, cy = 0;
    for (int t = 0; t < d.spawn_tries; ++t) {
      Rand4 r = philox(d.gid_env + (uint32_t)e, (uint32_t)(n * 64 + t), g, TAG_SPAWN, d.seed);
      long long ux = (long long)(r.x[0] >> 8) - 8388608LL;
      long long uy = (long long)(r.x[1] >> 8) - 8388608LL;
      if (ux * ux + uy * uy > r2) continue;
      cx = ux;
      cy = uy;
      bool ok = true;
      for (int m = 0; m < n; ++m) {
        long long dx = cx - X[m], dy = cy - Y[m];
        if (dx * dx + dy * dy < m2) { ok = false; break; }
      }
      if (ok) break;
    }
    X[n] = cx;
    Y[n] = cy;
  }
  for (int a = 0; a < A; ++a) {
    const int i = a0 + a;
    Rand4 r = philox(d.gid_agent + (uint32_t)i, 0u, g, TAG_AGENT_INIT, d.seed);
    d.ax[i] = (float)X[a] * 0x1p-16f;
    d.ay[i] = (float)Y[a] * 0x1p-16f;
    d.apsi[i] = (2.0f * unif(r.x[0]) - 1.0f) * kPi;
    d.rudder[i] = (d.n_rudder - 1) / 2;  // straight (action_mode 2)
  }
  for (int k = 0; k < T; ++k) {
    const int j = t0 + k;
    Rand4 r = philox(d.gid_target + (uint32_t)j, 0u, g, TAG_TARGET_INIT, d.seed);
    d.tx[j] = (float)X[A + k] * 0x1p-16f;
    d.ty[j] = (float)Y[A + k] * 0x1p-16f;
    d.tpsi[j] = (2.0f * unif(r.x[0]) - 1.0f) * kPi;
    d.tspeed[j] = d.ts_min + (d.ts_max - d.ts_min) * unif(r.x[1]);
    d.tz[j] = d.depth_max * unif(r.x[2]);
  }
  // at spawn every teammate is in range: all poses known, age 0
  for (int a = 0; a < A; ++a)
    for (int b = 0; b < d.AM; ++b) {
      const long long o = (long long)(a0 + a) * d.AM + b;
      d.lpx[o] = b < A ? (float)X[b] * 0x1p-16f : 0.0f;
      d.lpy[o] = b < A ? (float)Y[b] * 0x1p-16f : 0.0f;
      d.lpage[o] = 0;
    }
}

// -------------------------------------------------------------------------
// Reset, part 2: first ping of each filter and particle initialisation
// around the observer at the heard horizontal range (uniform in the
// detection disk if nothing was heard).  One block per filter.
// -------------------------------------------------------------------------
constexpr int kInitThreads = 256;

__global__ void __launch_bounds__(kInitThreads) reset_pf_kernel(EnvDev d, uint32_t g) {
  const int f = blockIdx.x;
  const int ia = d.filt_agent[f], it = d.filt_target[f];
  if (!UT_IN_BOUNDS(ia >= 0 && ia < d.NA && it >= 0 && it < d.NT, d.status)) return;  // (CTA-uniform)
  const float axv = d.ax[ia], ayv = d.ay[ia];
  const float dx = axv - d.tx[it], dy = ayv - d.ty[it], dz = 0.0f - d.tz[it];
  const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
  const bool heard = dist <= d.det_radius;
  Rand4 rp = philox(d.gid_filter + (uint32_t)f, 0u, g, TAG_RESET_PING, d.seed);
  float n0, n1;
  box_muller(rp.x[0], rp.x[1], n0, n1);
  const float r0 = dist + d.range_sigma * n0;
  const float zk = d.tz[it];
  const float horiz = sqrtf(fmaxf(r0 * r0 - zk * zk, 0.0f));
  float sx = 0.0f, sy = 0.0f;
  const long long base = (long long)f * d.P;
  for (int i = threadIdx.x; i < d.P; i += kInitThreads) {
    Rand4 r = philox(d.gid_filter + (uint32_t)f, (uint32_t)i, g, TAG_PF_INIT, d.seed);
    Rand4 q = philox(d.gid_filter + (uint32_t)f, (uint32_t)i, g, TAG_PF_INIT2, d.seed);
    float rho;
    if (heard) {
      float m0, m1;
      box_muller(r.x[0], r.x[1], m0, m1);
      rho = horiz + d.range_sigma * m0;
    } else {
      rho = d.det_radius * sqrtf(unif(r.x[0]));
    }
    float sphi, cphi, schi, cchi;
    sincospif(2.0f * unif(r.x[2]), &sphi, &cphi);
    sincospif(2.0f * unif(q.x[0]), &schi, &cchi);
    const float spd = d.pf_vcap * unif(r.x[3]);
    const float x = axv + rho * cphi, y = ayv + rho * sphi;
    d.px[base + i] = x;
    d.py[base + i] = y;
    d.pvx[base + i] = spd * cchi;
    d.pvy[base + i] = spd * schi;
    if (d.pw) d.pw[base + i] = 0.0f;  // equal weights
    sx += x;
    sy += y;
  }
  __shared__ float s_x[kInitThreads / 32], s_y[kInitThreads / 32];
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  if ((threadIdx.x & 31) == 0) {
    s_x[threadIdx.x >> 5] = sx;
    s_y[threadIdx.x >> 5] = sy;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float tx = 0.0f, ty = 0.0f;
    for (int w = 0; w < kInitThreads / 32; ++w) { tx += s_x[w]; ty += s_y[w]; }
    d.estx[f] = tx / (float)d.P;
    d.esty[f] = ty / (float)d.P;
    d.prev_estx[f] = d.prev2_estx[f] = d.estx[f];
    d.prev_esty[f] = d.prev2_esty[f] = d.esty[f];
    d.velx[f] = 0.0f;
    d.vely[f] = 0.0f;
    d.ring_head[f] = 0;
    d.ring_count[f] = 0;
  }
  if (d.ring_on)
    for (int j = threadIdx.x; j < kRing * 4; j += kInitThreads) d.ring[(long long)f * kRing * 4 + j] = 0.0f;
}

__global__ void reset_counters_kernel(EnvDev d) {
  if (threadIdx.x == 0) {
    d.counters[0] = 0;
    d.counters[1] = 0;
    d.metrics_d[0] = 0.0;
    d.metrics_d[1] = 0.0;
    for (int i = 0; i < 4; ++i) d.metrics_u[i] = 0ull;
  }
}

// -------------------------------------------------------------------------
// Step, part 1 (env_step.cuh: step_env_warp): one warp per environment.
// -------------------------------------------------------------------------
__global__ void __launch_bounds__(kWarpsPerBlock * 32) step_env_kernel(EnvDev d, const int32_t* __restrict__ act_in) {
  pdl_wait();
  pdl_trigger();
  const int wid = threadIdx.x >> 5;
  const int e = blockIdx.x * kWarpsPerBlock + wid;
  __shared__ EnvWarpSmem sw[kWarpsPerBlock];
  if (e >= d.E) return;  // warp-uniform
  step_env_warp(d, e, act_in, d.counters[0] + 1u, sw[wid]);
}

// -------------------------------------------------------------------------
// Step, part 3 (env_step.cuh: obs_reward_warp): one warp per environment;
// the block's four warps' metrics are added to the device sums.
// -------------------------------------------------------------------------
__global__ void __launch_bounds__(kWarpsPerBlock * 32) obs_reward_kernel(EnvDev d, int after_reset) {
  pdl_wait();
  pdl_trigger();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * kWarpsPerBlock + wid;
  __shared__ double s_sq[kWarpsPerBlock], s_rw[kWarpsPerBlock];
  __shared__ unsigned long long s_cnt[kWarpsPerBlock][3];
  StepMetrics m;
  if (e < d.E) obs_reward_warp(d, e, after_reset, d.counters[1] + 1u, m);
  if (!after_reset) {
    if (lane == 0) {
      s_sq[wid] = m.sq;
      s_rw[wid] = m.rw;
      s_cnt[wid][0] = m.n_err;
      s_cnt[wid][1] = m.n_crash;
      s_cnt[wid][2] = m.n_agents;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      unsigned long long c0 = 0, c1 = 0, c2 = 0;
      for (int w = 0; w < kWarpsPerBlock; ++w) {
        a += s_sq[w]; b += s_rw[w]; c0 += s_cnt[w][0]; c1 += s_cnt[w][1]; c2 += s_cnt[w][2];
      }
      atomicAdd(&d.metrics_d[0], a);
      atomicAdd(&d.metrics_d[1], b);
      atomicAdd(&d.metrics_u[0], c0);
      atomicAdd(&d.metrics_u[1], c1);
      atomicAdd(&d.metrics_u[2], c2);
    }
  }
}

__global__ void advance_kernel(EnvDev d) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x == 0) {
    d.counters[0] += 1u;
    d.counters[1] += 1u;
    d.metrics_u[3] += 1ull;
  }
}

// Stand-alone Philox: one thread per counter.
__global__ void philox_kernel(const uint4* __restrict__ ctr, uint64_t seed, uint4* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = ctr[i];
  Rand4 r = philox(c.x, c.y, c.z, c.w, seed);
  out[i] = make_uint4(r.x[0], r.x[1], r.x[2], r.x[3]);
}

}  // namespace

cudaError_t launch_reset(const EnvDev& d, cudaStream_t s) {
  reset_counters_kernel<<<1, 32, 0, s>>>(d);
  reset_spawn_kernel<<<(d.E + 127) / 128, 128, 0, s>>>(d, 0u);
  if (d.F > 0) reset_pf_kernel<<<d.F, kInitThreads, 0, s>>>(d, 0u);
  return cudaGetLastError();
}

cudaError_t launch_step_env(const EnvDev& d, const int32_t* act_in, cudaStream_t s) {
  return launch_pdl(step_env_kernel, dim3((d.E + kWarpsPerBlock - 1) / kWarpsPerBlock), dim3(kWarpsPerBlock * 32), 0,
                    s, d, act_in);
}

cudaError_t launch_obs_reward(const EnvDev& d, int after_reset, cudaStream_t s) {
  return launch_pdl(obs_reward_kernel, dim3((d.E + kWarpsPerBlock - 1) / kWarpsPerBlock), dim3(kWarpsPerBlock * 32), 0,
                    s, d, after_reset);
}

cudaError_t launch_advance(const EnvDev& d, cudaStream_t s) {
  return launch_pdl(advance_kernel, dim3(1), dim3(32), 0, s, d);
}

cudaError_t launch_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(reinterpret_cast<const uint4*>(ctr), seed,
                                                           reinterpret_cast<uint4*>(out), n);
  return cudaGetLastError();
}

}  // namespace ut
