// Environment kernels: reset, move/ping/communicate, observation/reward.
//
// These stages are tiny next to the particle filter (bytes per env-step are
// O(A*T) against O(A*T*P)), so they favour simplicity: one warp per
// environment, entity state staged in shared memory, struct-of-arrays in HBM.
#include "env.cuh"

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
// Step, part 1: actions, agent kinematics (Sec. III-A.3), target motion,
// pings, communication and per-filter measurement lists (Sec. III-A.2).
// One warp per environment.
// -------------------------------------------------------------------------
__global__ void __launch_bounds__(kWarpsPerBlock * 32) step_env_kernel(EnvDev d, const int32_t* __restrict__ act_in) {
  pdl_wait();
  pdl_trigger();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * kWarpsPerBlock + wid;
  __shared__ float s_ax[kWarpsPerBlock][kMaxAgents], s_ay[kWarpsPerBlock][kMaxAgents];
  __shared__ float s_tx[kWarpsPerBlock][kMaxTargets], s_ty[kWarpsPerBlock][kMaxTargets];
  __shared__ float s_tz[kWarpsPerBlock][kMaxTargets];
  __shared__ float s_rng[kWarpsPerBlock][kMaxAgents * kMaxTargets];
  __shared__ int s_valid[kWarpsPerBlock][kMaxAgents * kMaxTargets];
  __shared__ int s_recv[kWarpsPerBlock][kMaxAgents * kMaxAgents];
  if (e >= d.E) return;  // warp-uniform
  const uint32_t g = d.counters[0] + 1u;
  const int a0 = d.agent_off[e], A = d.agent_off[e + 1] - a0;
  const int t0 = d.target_off[e], T = d.target_off[e + 1] - t0;
  const int f0 = d.filter_off[e], q0 = d.pair_off[e];
  if (!UT_IN_BOUNDS(A >= 1 && A <= d.AM && d.AM <= kMaxAgents && T >= 1 && T <= d.TM && d.TM <= kMaxTargets &&
                        a0 >= 0 && a0 + A <= d.NA && t0 >= 0 && t0 + T <= d.NT && f0 >= 0 &&
                        f0 + (d.shared_filter ? T : A * T) <= d.F,
                    d.status))
    return;  // (warp-uniform)

  if (lane < A) {
    const int i = a0 + lane;
    int act;
    if (act_in) {
      act = act_in[i];
      if (act < 0 || act >= d.n_act) {
        raise_status(d.status, 1);
        act = act < 0 ? 0 : d.n_act - 1;
      }
    } else {
      Rand4 r = philox(d.gid_agent + (uint32_t)i, 0u, g, TAG_ACTION, d.seed);
      act = (int)__umulhi(r.x[0], (uint32_t)d.n_act);
    }
    d.actions[i] = act;
    int ang = act;  // index into the heading-change table
    if (d.rudder_mode) {  // the action moves the rudder down / keeps it / moves it up
      ang = min(max(d.rudder[i] + act - 1, 0), d.n_rudder - 1);
      d.rudder[i] = ang;
    }
    Rand4 r = philox(d.gid_agent + (uint32_t)i, 0u, g, TAG_AGENT_NOISE, d.seed);
    float n0, n1;
    box_muller(r.x[0], r.x[1], n0, n1);
    const float psi = wrap_angle(d.apsi[i] + d.dpsi[ang] + d.heading_noise * n0);
    float s, c;
    sincosf(psi, &s, &c);
    const float step_len = d.agent_speed * d.dt;
    const float x = d.ax[i] + step_len * c, y = d.ay[i] + step_len * s;
    d.apsi[i] = psi;
    d.ax[i] = x;
    d.ay[i] = y;
    s_ax[wid][lane] = x;
    s_ay[wid][lane] = y;
  } else if (lane >= 8 && lane - 8 < T) {
    const int k = lane - 8, j = t0 + k;
    Rand4 r = philox(d.gid_target + (uint32_t)j, 0u, g, TAG_TARGET_MOVE, d.seed);
    float psi;
    if (d.target_model == 0) {
      psi = wrap_angle(kTwoPi * unif(r.x[0]));
    } else {
      float n0, n1;
      box_muller(r.x[0], r.x[1], n0, n1);
      psi = wrap_angle(d.tpsi[j] + d.drift * n0);
    }
    float s, c;
    sincosf(psi, &s, &c);
    const float step_len = d.tspeed[j] * d.dt;
    const float x = d.tx[j] + step_len * c, y = d.ty[j] + step_len * s;
    d.tpsi[j] = psi;
    d.tx[j] = x;
    d.ty[j] = y;
    s_tx[wid][k] = x;
    s_ty[wid][k] = y;
    s_tz[wid][k] = d.tz[j];
  }
  __syncwarp();

  // pings of pair p = a * T + k (pair index q0 + p; the filter index with
  // per-agent filters)
  for (int p = lane; p < A * T; p += 32) {
    const int a = p / T, k = p - a * T;
    const float dx = s_ax[wid][a] - s_tx[wid][k], dy = s_ay[wid][a] - s_ty[wid][k], dz = 0.0f - s_tz[wid][k];
    const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
    Rand4 r = philox(d.gid_pair + (uint32_t)(q0 + p), 0u, g, TAG_PING, d.seed);
    float n0, n1;
    box_muller(r.x[0], r.x[1], n0, n1);
    const int v = dist <= d.det_radius;
    const float rg = v ? dist + d.range_sigma * n0 : 0.0f;
    s_rng[wid][p] = rg;
    s_valid[wid][p] = v;
    if (d.debug_on) {
      d.range[q0 + p] = rg;
      d.valid[q0 + p] = v;
    }
  }
  // communication: agent a hears agent b
  for (int p = lane; p < A * d.AM; p += 32) {
    const int a = p / d.AM, b = p - a * d.AM;
    const int ia = a0 + a;
    int rcv = 0;
    if (b < A) {
      if (a == b) {
        rcv = 1;
      } else {
        const float dx = s_ax[wid][a] - s_ax[wid][b], dy = s_ay[wid][a] - s_ay[wid][b];
        Rand4 r = philox(d.gid_agent + (uint32_t)ia, (uint32_t)b, g, TAG_COMM, d.seed);
        rcv = (sqrtf(dx * dx + dy * dy) <= d.comm_radius) && !(unif(r.x[0]) < d.comm_drop);
        const long long o = (long long)ia * d.AM + b;
        if (rcv) {
          d.lpx[o] = s_ax[wid][b];
          d.lpy[o] = s_ay[wid][b];
          d.lpage[o] = 0;
        } else {
          d.lpage[o] += 1;
        }
      }
      s_recv[wid][a * kMaxAgents + b] = rcv;
    }
    if (d.debug_on) d.recv[(long long)ia * d.AM + b] = rcv;
  }
  __syncwarp();

  // measurement list of each filter: the received senders that heard target
  // k (per-agent filter a T + k), or every agent that heard k (shared filter k)
  const int nfe = d.shared_filter ? T : A * T;
  for (int p = lane; p < nfe; p += 32) {
    const int a = d.shared_filter ? 0 : p / T, k = d.shared_filter ? p : p - a * T;
    const int f = f0 + p;
    int n = 0;
    int head = 0, cnt = 0;
    if (d.ring_on) {
      head = d.ring_head[f];
      cnt = d.ring_count[f];
    }
    for (int b = 0; b < A; ++b) {
      if ((d.shared_filter || s_recv[wid][a * kMaxAgents + b]) && s_valid[wid][b * T + k]) {
        const float qx = s_ax[wid][b], qy = s_ay[wid][b], r = s_rng[wid][b * T + k];
        if (UT_IN_BOUNDS(n < d.AM, d.status)) d.meas[(long long)f * d.AM + n] = make_float4(qx, qy, 0.0f, r);
        ++n;
        if (d.ring_on) {
          reinterpret_cast<float4*>(d.ring)[(long long)f * kRing + head] = make_float4(qx, qy, r, (float)g);
          head = (head + 1) & (kRing - 1);
          cnt = cnt < kRing ? cnt + 1 : kRing;
        }
      }
    }
    d.meas_n[f] = n;
    // per-filter header read by the filter step (no dependent loads there)
    d.meas_hdr[f] = make_float4(s_tx[wid][k], s_ty[wid][k], s_tz[wid][k] * s_tz[wid][k], (float)n);
    if (d.ring_on) {
      d.ring_head[f] = head;
      d.ring_count[f] = cnt;
    }
  }
}

// Tracking reward Eq. (1) of one error.
__device__ __forceinline__ float tracking_reward(float err, float emin, float emax) {
  if (err < emin) return 1.0f;
  if (err > emax) return 0.0f;
  const float t = (err - emin) / (emax - emin);
  if (t >= 1.0f) return 0.0f;
  return expf(-2.0f * t / (1.0f - t));
}

// -------------------------------------------------------------------------
// Step, part 3: observation tokens (Sec. III-A.2 Observation Space, Fig. 3)
// and reward (Eq. 1 / Eq. 2, normalised by targets, crash penalty), device
// metrics.  One warp per environment.
// -------------------------------------------------------------------------
__global__ void __launch_bounds__(kWarpsPerBlock * 32) obs_reward_kernel(EnvDev d, int after_reset) {
  pdl_wait();
  pdl_trigger();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * kWarpsPerBlock + wid;
  __shared__ double s_sq[kWarpsPerBlock], s_rw[kWarpsPerBlock];
  __shared__ unsigned long long s_cnt[kWarpsPerBlock][3];
  double sq = 0.0, rw = 0.0;
  unsigned long long n_err = 0, n_crash = 0, n_agents = 0;
  if (e < d.E) {
    const int a0 = d.agent_off[e], A0 = d.agent_off[e + 1] - a0;
    const int t0 = d.target_off[e], T0 = d.target_off[e + 1] - t0;
    const int f0 = d.filter_off[e];
    // (checked build: an env whose counts fall outside the handle's maxima is skipped)
    const bool counts_ok = UT_IN_BOUNDS(A0 >= 1 && A0 <= d.AM && T0 >= 1 && T0 <= d.TM && A0 + T0 <= d.NS &&
                                            a0 >= 0 && a0 + A0 <= d.NA && f0 >= 0 &&
                                            f0 + (d.shared_filter ? T0 : A0 * T0) <= d.F,
                                        d.status);
    const int A = counts_ok ? A0 : 0, T = counts_ok ? T0 : 1;
    for (int p = lane; p < A * d.NS; p += 32) {
      const int a = p / d.NS, slot = p - a * d.NS;
      const int ia = a0 + a;
      float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (slot == 0) {
        v[3] = 1.0f;
      } else if (slot < A) {
        const int b = (slot - 1) < a ? slot - 1 : slot;
        const long long o = (long long)ia * d.AM + b;
        const int age = d.lpage[o];
        v[0] = (d.lpx[o] - d.ax[ia]) / d.S;
        v[1] = (d.lpy[o] - d.ay[ia]) / d.S;
        v[4] = 1.0f;
        v[6] = age > 0 ? 1.0f : 0.0f;
        v[7] = (float)(age < 16 ? age : 16) / 16.0f;
      } else if (slot < A + T) {
        const int k = slot - A;
        const int f = f0 + (d.shared_filter ? k : a * T + k);
        v[0] = (d.estx[f] - d.ax[ia]) / d.S;
        v[1] = (d.esty[f] - d.ay[ia]) / d.S;
        v[2] = d.tz[t0 + k] / d.S;
        v[5] = 1.0f;
      }
      uint4 packed;
      packed.x = (uint32_t)f2bf_bits(v[0]) | ((uint32_t)f2bf_bits(v[1]) << 16);
      packed.y = (uint32_t)f2bf_bits(v[2]) | ((uint32_t)f2bf_bits(v[3]) << 16);
      packed.z = (uint32_t)f2bf_bits(v[4]) | ((uint32_t)f2bf_bits(v[5]) << 16);
      packed.w = (uint32_t)f2bf_bits(v[6]) | ((uint32_t)f2bf_bits(v[7]) << 16);
      reinterpret_cast<uint4*>(d.obs)[(long long)ia * d.NS + slot] = packed;
    }
    if (!after_reset) {
      float rk = 0.0f;
      if (lane < T) {
        const int k = lane;
        if (d.reward_type == 0) {
          // agent-averaged error; a shared filter's error is every agent's
          float ek = 0.0f;
          if (d.shared_filter) {
            ek = d.err[f0 + k];
          } else {
            for (int a = 0; a < A; ++a) ek += d.err[f0 + a * T + k];
            ek /= (float)A;
          }
          rk = tracking_reward(ek, d.eps_min, d.eps_max);
        } else {
          float dk = INFINITY;
          for (int a = 0; a < A; ++a) {
            const float dx = d.ax[a0 + a] - d.tx[t0 + k], dy = d.ay[a0 + a] - d.ty[t0 + k];
            dk = fminf(dk, sqrtf(dx * dx + dy * dy));
          }
          rk = dk <= d.follow_dmin ? 1.0f : 0.0f;
        }
      }
      rk = warp_sum(rk);
      int cr = 0;
      for (int p = lane; p < A * A; p += 32) {
        const int a = p / A, b = p - a * A;
        if (b > a) {
          const float dx = d.ax[a0 + a] - d.ax[a0 + b], dy = d.ay[a0 + a] - d.ay[a0 + b];
          if (sqrtf(dx * dx + dy * dy) < d.d_safe) cr = 1;
        }
      }
      cr = __any_sync(0xffffffffu, cr);
      double se = 0.0;
      const int nfe = d.filter_off[e + 1] - f0;
      for (int p = lane; p < nfe; p += 32) {
        const double v = (double)d.err[f0 + p];
        se += v * v;
      }
      se = warp_sum_d(se);
      const float r = cr ? -1.0f : rk / (float)T;
      if (lane == 0) {
        d.reward[e] = r;
        d.crash[e] = cr;
        d.done[e] = (d.counters[1] + 1u) >= (uint32_t)d.horizon;
      }
      sq = se;
      rw = (double)r;
      n_err = (unsigned long long)nfe;
      n_crash = (unsigned long long)cr;
      n_agents = (unsigned long long)A;
    } else if (lane == 0) {
      d.reward[e] = 0.0f;
      d.crash[e] = 0;
      d.done[e] = 0;
    }
  }
  if (!after_reset) {
    if (lane == 0) {
      s_sq[wid] = sq;
      s_rw[wid] = rw;
      s_cnt[wid][0] = n_err;
      s_cnt[wid][1] = n_crash;
      s_cnt[wid][2] = n_agents;
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
