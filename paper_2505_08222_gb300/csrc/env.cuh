// Internal device view of one environment batch and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace ut {

// Everything a kernel needs, passed by value.  Sizes, constants (already
// converted to float on the host), and device pointers into the handle's
// buffers.  Layouts are documented in include/utrack.h.
struct EnvDev {
  // sizes
  int E, AM, TM, NS, P, NA, NT, F;
  int n_act, horizon;
  const int32_t* agent_off;   // [E+1]
  const int32_t* target_off;  // [E+1]
  const int32_t* filter_off;  // [E+1]
  const int32_t* pair_off;    // [E+1] first (agent, target) pair of each env (= filter_off per agent)
  int shared_filter;          // 1: one filter per (env, target), filter_off[e] + k
  int NPAIR;                  // sum of A_e T_e
  const int32_t* filt_agent;  // [F] global agent index of filter f (the env's first agent if shared)
  const int32_t* filt_target; // [F] global target index of filter f
  // constants
  uint64_t seed;
  uint32_t gid_env, gid_agent, gid_target, gid_filter, gid_pair;  // global id offsets
  float dt, agent_speed, heading_noise;
  float dpsi[8];              // heading change of each action (action_mode 2: of each rudder position)
  int rudder_mode;            // action_mode 2: actions move the rudder position
  int n_rudder;
  int target_model;
  float ts_min, ts_max, drift, depth_max;
  float range_sigma, inv_two_s2, det_radius, comm_radius, comm_drop;
  float pf_accel_sigma, pf_vcap;
  int reward_type;
  float eps_min, eps_max, follow_dmin, d_safe;
  long long spawn_r_int, spawn_dmin_int;  // on the 2^-16 m lattice
  int spawn_tries;
  float S;
  int ring_on, debug_on;
  // state
  float *ax, *ay, *apsi;
  float *tx, *ty, *tz, *tpsi, *tspeed;
  float *px, *py, *pvx, *pvy;
  float* pw;        // particle log-weights [F*P] (pf_ess_num > 0), else null
  int pf_ess_num;   // resample when 16 (sum r)^2 < pf_ess_num P sum r^2; 0: every step
  float *lpx, *lpy;
  int32_t* lpage;
  float *estx, *esty, *err;
  // the two previous estimates of each filter (estimate history of the
  // learned estimator's features; NULL where not kept)
  float *prev_estx, *prev_esty, *prev2_estx, *prev2_esty;
  int32_t* rudder;            // [NA] rudder position (action_mode 2)
  // smoothed motion of the estimate per step (EMA over the updates' e1 - e2)
  float *velx, *vely;
  float est_scale;  // L: metres per unit of the learned estimator's local frame
  float* ring;
  int32_t *ring_head, *ring_count;
  // per-step buffers
  float4* meas;               // [F][AM]
  int32_t* meas_n;            // [F]
  float4* meas_hdr;           // [F] (target x, target y, target depth^2, list length)
  float* range;               // [F] (debug)
  int32_t* valid;             // [F] (debug)
  int32_t* recv;              // [NA][AM] (debug)
  int32_t* actions;           // [NA]
  uint16_t* obs;              // [NA][NS][8]
  float* reward;              // [E]
  int32_t* crash;             // [E]
  int32_t* done;              // [E]
  uint32_t* counters;         // [0] global step g, [1] steps since reset
  double* metrics_d;          // [0] sum sq err, [1] reward sum
  unsigned long long* metrics_u;  // [0] n_err, [1] crashes, [2] agent steps, [3] steps
  int* status;
  // debug intermediates
  float *dbg_px, *dbg_py, *dbg_pvx, *dbg_pvy, *dbg_w, *dbg_wmax;
  int32_t* dbg_idx;
};

// Launchers (env_kernels.cu, pf_kernel.cu).
cudaError_t launch_reset(const EnvDev& d, cudaStream_t s);
cudaError_t launch_step_env(const EnvDev& d, const int32_t* act_in, cudaStream_t s);
cudaError_t launch_obs_reward(const EnvDev& d, int after_reset, cudaStream_t s);
cudaError_t launch_advance(const EnvDev& d, cudaStream_t s);
cudaError_t launch_pf_step(const EnvDev& d, int variant, cudaStream_t s);
cudaError_t launch_ls_update(const EnvDev& d, cudaStream_t s);
int pf_default_variant(int P);
int pf_variant_count();
const char* pf_variant_name(int v);
bool pf_variant_valid(int v, int P);
cudaError_t launch_pf_resample(const float* wmax, const uint64_t* u64, int64_t n_filters, int P, int32_t* idx,
                               cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n, cudaStream_t s);
// Persistent rollout (rollout_persistent.cu): T steps in one launch, one CTA
// per environment, random actions, the filter launch shape of `variant`.
bool persistent_supported(const EnvDev& d, int variant);
cudaError_t launch_rollout_persistent(const EnvDev& d, int variant, int T, cudaStream_t s);

}  // namespace ut
