// Per-environment step stages as warp-level device functions, shared by the
// step kernels (env_kernels.cu) and the persistent rollout kernel
// (rollout_persistent.cu): one warp owns one environment.
#pragma once

#include "env.cuh"

namespace ut {

// Shared-memory staging of one environment (one warp).
struct EnvWarpSmem {
  float ax[kMaxAgents], ay[kMaxAgents];
  float tx[kMaxTargets], ty[kMaxTargets], tz[kMaxTargets];
  float rng[kMaxAgents * kMaxTargets];
  int valid[kMaxAgents * kMaxTargets];
  int recv[kMaxAgents * kMaxAgents];
};

// Per-warp metric contributions of one step (lane 0's values are the warp's).
struct StepMetrics {
  double sq = 0.0, rw = 0.0;
  unsigned long long n_err = 0, n_crash = 0, n_agents = 0;
};

// -------------------------------------------------------------------------
// Step, part 1: actions, agent kinematics (Sec. III-A.3), target motion,
// pings, communication and per-filter measurement lists (Sec. III-A.2).
// Called by the whole warp that owns environment e, at global step g.
// -------------------------------------------------------------------------
__device__ __forceinline__ void step_env_warp(const EnvDev& d, int e, const int32_t* __restrict__ act_in, uint32_t g,
                                              EnvWarpSmem& w) {
  const int lane = threadIdx.x & 31;
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
    w.ax[lane] = x;
    w.ay[lane] = y;
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
    w.tx[k] = x;
    w.ty[k] = y;
    w.tz[k] = d.tz[j];
  }
  __syncwarp();

  // pings of pair p = a * T + k (pair index q0 + p; the filter index with
  // per-agent filters)
  for (int p = lane; p < A * T; p += 32) {
    const int a = p / T, k = p - a * T;
    const float dx = w.ax[a] - w.tx[k], dy = w.ay[a] - w.ty[k], dz = 0.0f - w.tz[k];
    const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
    Rand4 r = philox(d.gid_pair + (uint32_t)(q0 + p), 0u, g, TAG_PING, d.seed);
    float n0, n1;
    box_muller(r.x[0], r.x[1], n0, n1);
    const int v = dist <= d.det_radius;
    const float rg = v ? dist + d.range_sigma * n0 : 0.0f;
    w.rng[p] = rg;
    w.valid[p] = v;
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
        const float dx = w.ax[a] - w.ax[b], dy = w.ay[a] - w.ay[b];
        Rand4 r = philox(d.gid_agent + (uint32_t)ia, (uint32_t)b, g, TAG_COMM, d.seed);
        rcv = (sqrtf(dx * dx + dy * dy) <= d.comm_radius) && !(unif(r.x[0]) < d.comm_drop);
        const long long o = (long long)ia * d.AM + b;
        if (rcv) {
          d.lpx[o] = w.ax[b];
          d.lpy[o] = w.ay[b];
          d.lpage[o] = 0;
        } else {
          d.lpage[o] += 1;
        }
      }
      w.recv[a * kMaxAgents + b] = rcv;
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
      if ((d.shared_filter || w.recv[a * kMaxAgents + b]) && w.valid[b * T + k]) {
        const float qx = w.ax[b], qy = w.ay[b], r = w.rng[b * T + k];
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
    d.meas_hdr[f] = make_float4(w.tx[k], w.ty[k], w.tz[k] * w.tz[k], (float)n);
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
// metrics.  Called by the whole warp that owns environment e; t_next = steps
// since the reset after this step (the episode ends at the horizon); the
// warp's metric contributions are returned in `out` (lane 0's are the sums).
// -------------------------------------------------------------------------
__device__ __forceinline__ void obs_reward_warp(const EnvDev& d, int e, int after_reset, uint32_t t_next,
                                                StepMetrics& out) {
  const int lane = threadIdx.x & 31;
  double sq = 0.0, rw = 0.0;
  unsigned long long n_err = 0, n_crash = 0, n_agents = 0;
  {
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
      packed.x = bf16x2_bits(v[0], v[1]);
      packed.y = bf16x2_bits(v[2], v[3]);
      packed.z = bf16x2_bits(v[4], v[5]);
      packed.w = bf16x2_bits(v[6], v[7]);
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
        d.done[e] = t_next >= (uint32_t)d.horizon;
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
  out.sq = sq;
  out.rw = rw;
  out.n_err = n_err;
  out.n_crash = n_crash;
  out.n_agents = n_agents;
}

}  // namespace ut
