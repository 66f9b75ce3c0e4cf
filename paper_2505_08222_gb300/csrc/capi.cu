// C ABI runtime: handle creation, buffer allocation, step sequencing,
// CUDA-graph rollout, state import/export.  Declarations and contracts are
// in include/utrack.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/utrack.h"
#include "env.cuh"
#include "runtime.cuh"

using namespace ut;

namespace {

ut_status fail(ut_env* h, ut_status code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

ut_status cuda_fail(ut_env* h, cudaError_t e, const char* where) {
  return fail(h, UT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define UT_CUDA(h, call)                                       \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);   \
  } while (0)

}  // namespace

namespace ut {

void* env_alloc(ut_env* h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (h->has_alloc) {
    p = h->alloc.alloc(bytes, (void*)h->stream, h->alloc.ctx);
  } else {
    if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) p = nullptr;
  }
  if (!p) return nullptr;
  h->allocations.push_back(p);
  if (cudaMemsetAsync(p, 0, bytes, h->stream) != cudaSuccess) return nullptr;
  return p;
}

void env_free_all(ut_env* h) {
  for (void* p : h->allocations) {
    if (h->has_alloc) h->alloc.free(p, (void*)h->stream, h->alloc.ctx);
    else cudaFreeAsync(p, h->stream);
  }
  h->allocations.clear();
}

}  // namespace ut

namespace {

template <typename T>
T* alloc_n(ut_env* h, size_t n, bool& ok) {
  T* p = (T*)env_alloc(h, n * sizeof(T));
  if (!p) ok = false;
  return p;
}

ut_status validate(const ut_config* c, std::string& why) {
  auto bad = [&](const char* m) { why = m; return UT_ERR_INVALID; };
  if (!c) return bad("config is NULL");
  if (c->abi_version != UT_ABI_VERSION) return bad("abi_version mismatch");
  if (c->n_envs < 1) return bad("n_envs must be >= 1");
  if (c->max_agents < 1 || c->max_agents > UT_MAX_AGENTS) return bad("max_agents out of range");
  if (c->max_targets < 1 || c->max_targets > UT_MAX_TARGETS) return bad("max_targets out of range");
  if (c->n_particles < 1 || c->n_particles > UT_MAX_PARTICLES) return bad("n_particles out of range");
  if (c->horizon < 1) return bad("horizon must be >= 1");
  if (c->action_mode == 0 && c->n_actions != 3) return bad("action_mode 0 needs n_actions == 3");
  if (c->action_mode == 1 && (c->n_actions < 2 || c->n_actions > 8)) return bad("n_actions must be in 2..8");
  if (c->action_mode == 2 && c->n_actions != 3) return bad("action_mode 2 needs n_actions == 3 (down, keep, up)");
  if (c->action_mode == 2 && (c->n_rudder < 2 || c->n_rudder > 8)) return bad("n_rudder must be in 2..8");
  if (c->action_mode < 0 || c->action_mode > 2) return bad("action_mode must be 0, 1 or 2");
  if (!(c->range_sigma > 0.0f)) return bad("range_sigma must be > 0");
  if (!(c->dt > 0.0f)) return bad("dt must be > 0");
  if (c->spawn_tries < 1 || c->spawn_tries > 64) return bad("spawn_tries must be in 1..64");
  if (!(c->spawn_radius > 0.0f) || c->spawn_radius * 65536.0 > 8388607.0) return bad("spawn_radius out of range");
  if (!(c->feature_scale > 0.0f)) return bad("feature_scale must be > 0");
  if (!(c->est_scale > 0.0f)) return bad("est_scale must be > 0");
  if (c->reward_type != 0 && c->reward_type != 1) return bad("reward_type must be 0 or 1");
  if (c->shared_filter != 0 && c->shared_filter != 1) return bad("shared_filter must be 0 or 1");
  if (c->pf_ess_num < 0 || c->pf_ess_num > 16) return bad("pf_ess_num must be in 0..16");
  if (c->d_model < 0) return bad("d_model must be >= 0");
  if (c->d_model > 0) {
    if (c->n_heads < 1 || c->d_model % c->n_heads != 0) return bad("d_model % n_heads != 0");
    if (c->n_layers < 1) return bad("n_layers must be >= 1");
  }
  return UT_OK;
}

// Host copy of the per-env counts and CSR offsets.
struct Layout {
  std::vector<int32_t> a, t, aoff, toff, foff, poff, fagent, ftarget;
  int64_t NA = 0, NT = 0, F = 0, NPAIR = 0;
};

ut_status make_layout(const ut_config* c, Layout& L, std::string& why) {
  const int E = c->n_envs;
  L.a.resize(E);
  L.t.resize(E);
  for (int e = 0; e < E; ++e) {
    L.a[e] = c->agents_per_env_host ? c->agents_per_env_host[e] : c->max_agents;
    L.t[e] = c->targets_per_env_host ? c->targets_per_env_host[e] : c->max_targets;
    if (L.a[e] < 1 || L.a[e] > c->max_agents || L.t[e] < 1 || L.t[e] > c->max_targets) {
      why = "per-env agent/target count out of range";
      return UT_ERR_INVALID;
    }
  }
  L.aoff.assign(E + 1, 0);
  L.toff.assign(E + 1, 0);
  L.foff.assign(E + 1, 0);
  L.poff.assign(E + 1, 0);
  const bool shared = c->shared_filter != 0;
  int64_t na = 0, nt = 0, nf = 0, np = 0;
  for (int e = 0; e < E; ++e) {
    L.aoff[e] = (int32_t)na;
    L.toff[e] = (int32_t)nt;
    L.foff[e] = (int32_t)nf;
    L.poff[e] = (int32_t)np;
    na += L.a[e];
    nt += L.t[e];
    np += (int64_t)L.a[e] * L.t[e];
    nf += shared ? L.t[e] : (int64_t)L.a[e] * L.t[e];
  }
  if (np >= (1ll << 31) - 1) {
    why = "too many filters";
    return UT_ERR_INVALID;
  }
  L.aoff[E] = (int32_t)na;
  L.toff[E] = (int32_t)nt;
  L.foff[E] = (int32_t)nf;
  L.poff[E] = (int32_t)np;
  L.NA = na;
  L.NT = nt;
  L.F = nf;
  L.NPAIR = np;
  L.fagent.resize(nf);
  L.ftarget.resize(nf);
  for (int e = 0; e < E; ++e) {
    const int nfe = L.foff[e + 1] - L.foff[e];
    for (int j = 0; j < nfe; ++j) {
      const int64_t f = L.foff[e] + j;
      // per agent: filter j = a T + k; shared: filter j = k, anchored at agent 0
      L.fagent[f] = L.aoff[e] + (shared ? 0 : j / L.t[e]);
      L.ftarget[f] = L.toff[e] + (shared ? j : j % L.t[e]);
    }
  }
  return UT_OK;
}

}  // namespace

extern "C" {

ut_status env_create(const ut_config* cfg, const ut_allocator* allocator, void* cuda_stream, ut_env** out) {
  if (!out) return UT_ERR_INVALID;
  *out = nullptr;
  std::string why;
  ut_status st = validate(cfg, why);
  if (st != UT_OK) {
    std::fprintf(stderr, "env_create: %s\n", why.c_str());
    return st;
  }
  Layout L;
  st = make_layout(cfg, L, why);
  if (st != UT_OK) {
    std::fprintf(stderr, "env_create: %s\n", why.c_str());
    return st;
  }
  ut_env* h = new ut_env();
  h->cfg = *cfg;
  h->cfg.agents_per_env_host = nullptr;
  h->cfg.targets_per_env_host = nullptr;
  h->stream = (cudaStream_t)cuda_stream;
  if (allocator && allocator->alloc && allocator->free) {
    h->has_alloc = true;
    h->alloc = *allocator;
  }
  cudaGetDevice(&h->device);
  h->NA = L.NA;
  h->NT = L.NT;
  h->F = L.F;
  h->agents_per_env = L.a;
  h->targets_per_env = L.t;

  EnvDev& d = h->d;
  std::memset(&d, 0, sizeof(d));
  const int E = cfg->n_envs, AM = cfg->max_agents, P = cfg->n_particles;
  d.E = E;
  d.AM = AM;
  d.TM = cfg->max_targets;
  d.NS = cfg->max_agents + cfg->max_targets;
  d.P = P;
  d.NA = (int)L.NA;
  d.NT = (int)L.NT;
  d.F = (int)L.F;
  d.n_act = cfg->n_actions;
  d.horizon = cfg->horizon;
  d.dt = cfg->dt;
  d.agent_speed = cfg->agent_speed;
  d.heading_noise = cfg->heading_noise;
  d.rudder_mode = cfg->action_mode == 2 ? 1 : 0;
  d.n_rudder = cfg->action_mode == 2 ? cfg->n_rudder : 0;
  const int n_ang = cfg->action_mode == 2 ? cfg->n_rudder : cfg->n_actions;  // rudder angles in the table
  for (int j = 0; j < 8; ++j) {
    double v = 0.0;
    if (j < n_ang) {
      if (cfg->action_mode == 0) {
        v = (double)(j - 1) * (double)cfg->turn_angle;
      } else {
        const double gam = -(double)cfg->rudder_max + 2.0 * cfg->rudder_max * j / (double)(n_ang - 1);
        v = (double)cfg->rudder_gain * gam;
      }
    }
    d.dpsi[j] = (float)v;
  }
  d.target_model = cfg->target_model;
  d.ts_min = cfg->target_speed_min;
  d.ts_max = cfg->target_speed_max;
  d.drift = cfg->target_drift_sigma;
  d.depth_max = cfg->target_depth_max;
  d.range_sigma = cfg->range_sigma;
  d.inv_two_s2 = (float)(1.0 / (2.0 * (double)cfg->range_sigma * (double)cfg->range_sigma));
  d.det_radius = cfg->det_radius;
  d.comm_radius = cfg->comm_radius;
  d.comm_drop = cfg->comm_drop;
  d.pf_accel_sigma = cfg->pf_accel_sigma;
  d.pf_vcap = cfg->pf_vcap;
  d.reward_type = cfg->reward_type;
  d.eps_min = cfg->eps_min;
  d.eps_max = cfg->eps_max;
  d.follow_dmin = cfg->follow_dmin;
  d.d_safe = cfg->d_safe;
  d.spawn_r_int = (long long)std::floor((double)cfg->spawn_radius * 65536.0);
  d.spawn_dmin_int = (long long)std::floor((double)cfg->spawn_min * 65536.0);
  d.spawn_tries = cfg->spawn_tries;
  d.S = cfg->feature_scale;
  d.gid_env = cfg->id_env0;
  d.gid_agent = cfg->id_agent0;
  d.gid_target = cfg->id_target0;
  d.gid_filter = cfg->id_filter0;
  // pings are keyed by (agent, target) pair: per-agent filters are their pairs
  d.gid_pair = cfg->shared_filter ? cfg->id_pair0 : cfg->id_filter0;
  d.shared_filter = cfg->shared_filter ? 1 : 0;
  d.NPAIR = (int)L.NPAIR;
  d.est_scale = cfg->est_scale;
  d.ring_on = (cfg->flags & UT_FLAG_RING) ? 1 : 0;
  d.debug_on = (cfg->flags & UT_FLAG_DEBUG) ? 1 : 0;

  bool ok = true;
  const size_t NA = L.NA, NT = L.NT, F = L.F, FP = (size_t)L.F * P;
  int32_t* aoff = alloc_n<int32_t>(h, E + 1, ok);
  int32_t* toff = alloc_n<int32_t>(h, E + 1, ok);
  int32_t* foff = alloc_n<int32_t>(h, E + 1, ok);
  int32_t* poff = alloc_n<int32_t>(h, E + 1, ok);
  const size_t NPAIR = L.NPAIR;
  int32_t* fag = alloc_n<int32_t>(h, F, ok);
  int32_t* ftg = alloc_n<int32_t>(h, F, ok);
  d.ax = alloc_n<float>(h, NA, ok);
  d.ay = alloc_n<float>(h, NA, ok);
  d.apsi = alloc_n<float>(h, NA, ok);
  d.tx = alloc_n<float>(h, NT, ok);
  d.ty = alloc_n<float>(h, NT, ok);
  d.tz = alloc_n<float>(h, NT, ok);
  d.tpsi = alloc_n<float>(h, NT, ok);
  d.tspeed = alloc_n<float>(h, NT, ok);
  d.px = alloc_n<float>(h, FP, ok);
  d.py = alloc_n<float>(h, FP, ok);
  d.pvx = alloc_n<float>(h, FP, ok);
  d.pvy = alloc_n<float>(h, FP, ok);
  d.pf_ess_num = cfg->pf_ess_num;
  d.pw = cfg->pf_ess_num > 0 ? alloc_n<float>(h, FP, ok) : nullptr;
  d.lpx = alloc_n<float>(h, NA * AM, ok);
  d.lpy = alloc_n<float>(h, NA * AM, ok);
  d.lpage = alloc_n<int32_t>(h, NA * AM, ok);
  d.estx = alloc_n<float>(h, F, ok);
  d.esty = alloc_n<float>(h, F, ok);
  d.prev_estx = alloc_n<float>(h, F, ok);
  d.prev_esty = alloc_n<float>(h, F, ok);
  d.prev2_estx = alloc_n<float>(h, F, ok);
  d.prev2_esty = alloc_n<float>(h, F, ok);
  d.rudder = alloc_n<int32_t>(h, NA, ok);
  d.velx = alloc_n<float>(h, F, ok);
  d.vely = alloc_n<float>(h, F, ok);
  d.err = alloc_n<float>(h, F, ok);
  d.ring = alloc_n<float>(h, d.ring_on ? F * kRing * 4 : 4, ok);
  d.ring_head = alloc_n<int32_t>(h, F, ok);
  d.ring_count = alloc_n<int32_t>(h, F, ok);
  d.meas = alloc_n<float4>(h, F * AM, ok);
  d.meas_n = alloc_n<int32_t>(h, F, ok);
  d.meas_hdr = alloc_n<float4>(h, F, ok);
  d.actions = alloc_n<int32_t>(h, NA, ok);
  d.obs = alloc_n<uint16_t>(h, NA * d.NS * 8, ok);
  d.reward = alloc_n<float>(h, E, ok);
  d.crash = alloc_n<int32_t>(h, E, ok);
  d.done = alloc_n<int32_t>(h, E, ok);
  d.counters = alloc_n<uint32_t>(h, 4, ok);
  d.metrics_d = alloc_n<double>(h, 2, ok);
  d.metrics_u = alloc_n<unsigned long long>(h, 4, ok);
  d.status = alloc_n<int>(h, 1, ok);
  if (d.debug_on) {
    d.range = alloc_n<float>(h, NPAIR, ok);
    d.valid = alloc_n<int32_t>(h, NPAIR, ok);
    d.recv = alloc_n<int32_t>(h, NA * AM, ok);
    d.dbg_px = alloc_n<float>(h, FP, ok);
    d.dbg_py = alloc_n<float>(h, FP, ok);
    d.dbg_pvx = alloc_n<float>(h, FP, ok);
    d.dbg_pvy = alloc_n<float>(h, FP, ok);
    d.dbg_w = alloc_n<float>(h, FP, ok);
    d.dbg_wmax = alloc_n<float>(h, FP, ok);
    d.dbg_idx = alloc_n<int32_t>(h, FP, ok);
  }
  if (!ok) {
    env_free_all(h);
    cudaStreamSynchronize(h->stream);
    delete h;
    return UT_ERR_NOMEM;
  }
  d.agent_off = aoff;
  d.target_off = toff;
  d.filter_off = foff;
  d.pair_off = poff;
  d.filt_agent = fag;
  d.filt_target = ftg;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpyAsync(aoff, L.aoff.data(), (E + 1) * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(toff, L.toff.data(), (E + 1) * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(foff, L.foff.data(), (E + 1) * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(poff, L.poff.data(), (E + 1) * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && F) e = cudaMemcpyAsync(fag, L.fagent.data(), F * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && F) e = cudaMemcpyAsync(ftg, L.ftarget.data(), F * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "env_create: %s\n", cudaGetErrorString(e));
    env_free_all(h);
    delete h;
    return UT_ERR_CUDA;
  }
  h->pf_variant = pf_default_variant(P);
  st = extension_create(h);
  if (st != UT_OK) {
    std::fprintf(stderr, "env_create: %s\n", h->err.c_str());
    extension_destroy(h);
    env_free_all(h);
    cudaStreamSynchronize(h->stream);
    delete h;
    return st;
  }
  *out = h;
  return UT_OK;
}

void env_destroy(ut_env* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->ppo_exec) cudaGraphExecDestroy(h->ppo_exec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (cudaEvent_t ev : h->eager_ev) cudaEventDestroy(ev);
  extension_destroy(h);
  env_free_all(h);
  cudaStreamSynchronize(h->stream);
  delete h;
}

const char* env_last_error(const ut_env* h) { return h ? h->err.c_str() : "null handle"; }

ut_status env_reset(ut_env* h, uint64_t seed) {
  if (!h) return UT_ERR_INVALID;
  h->d.seed = seed;
  UT_CUDA(h, launch_reset(h->d, h->stream));
  UT_CUDA(h, extension_reset(h, h->stream));
  UT_CUDA(h, launch_obs_reward(h->d, 1, h->stream));
  h->reset_done = true;
  return UT_OK;
}

}  // extern "C"

namespace ut {

// Timing-event pair for the tracker stage of this step (nullptr: off).
static cudaError_t stage_events(ut_env* h, cudaEvent_t* ev0, cudaEvent_t* ev1) {
  *ev0 = *ev1 = nullptr;
  // CUDA cannot time events recorded by graph nodes: eager steps only
  if (!h->prof_on || h->capturing) return cudaSuccess;
  if (2 * (h->eager_used + 1) > h->eager_ev.size()) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t ev;
      cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return e;
      h->eager_ev.push_back(ev);
    }
  }
  *ev0 = h->eager_ev[2 * h->eager_used];
  *ev1 = h->eager_ev[2 * h->eager_used + 1];
  h->eager_used++;
  return cudaSuccess;
}

int count_step_kernels(ut_env* h) {
  // policy (when it picks the actions) + env + tracker + obs/reward + advance
  return 4 + (h->policy_ready ? extension_policy_kernels(h) : 0);
}

// The kernels of one step, in order, on stream s.
cudaError_t enqueue_step(ut_env* h, const int32_t* act, cudaStream_t s) {
  cudaError_t e;
  const int32_t* a = act;
  int n = 4;
  if (!a && h->policy_ready) {
    e = extension_policy_actions(h, s);
    if (e != cudaSuccess) return e;
    a = h->d.actions;
    n += extension_policy_kernels(h);
  }
  e = launch_step_env(h->d, a, s);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev0, ev1;
  e = stage_events(h, &ev0, &ev1);
  if (e != cudaSuccess) return e;
  if (ev0 && (e = cudaEventRecord(ev0, s)) != cudaSuccess) return e;
  e = extension_estimate(h, s);  // learned estimator replaces the filter when enabled
  if (e == cudaErrorNotReady) e = launch_pf_step(h->d, h->pf_variant, s);
  if (e != cudaSuccess) return e;
  if (ev1 && (e = cudaEventRecord(ev1, s)) != cudaSuccess) return e;
  e = launch_obs_reward(h->d, 0, s);
  if (e != cudaSuccess) return e;
  h->launches += n;
  return launch_advance(h->d, s);
}


// The capture stream and fork/join events of a handle, created on first use.
cudaError_t capture_stream_ensure(ut_env* h) {
  cudaError_t e = cudaSuccess;
  if (!h->cap_stream) {
    e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  }
  return e;
}
}  // namespace ut

extern "C" {

ut_status env_step(ut_env* h, const int32_t* actions_dev, ut_step_out* out) {
  if (!h) return UT_ERR_INVALID;
  if (!h->reset_done) return fail(h, UT_ERR_STATE, "env_step before env_reset");
  UT_CUDA(h, enqueue_step(h, actions_dev, h->stream));
  if (out) {
    out->reward = h->d.reward;
    out->done = h->d.done;
    out->obs = h->d.obs;
    out->estx = h->d.estx;
    out->esty = h->d.esty;
    out->err = h->d.err;
    out->actions = h->d.actions;
    out->logits = h->policy_ready ? extension_logits(h) : nullptr;
  }
  return UT_OK;
}

ut_status env_metrics_reset(ut_env* h) {
  if (!h) return UT_ERR_INVALID;
  h->launches = 0;
  UT_CUDA(h, cudaMemsetAsync(h->d.metrics_d, 0, 2 * sizeof(double), h->stream));
  UT_CUDA(h, cudaMemsetAsync(h->d.metrics_u, 0, 4 * sizeof(unsigned long long), h->stream));
  UT_CUDA(h, cudaMemsetAsync(h->d.status, 0, sizeof(int), h->stream));
  return UT_OK;
}

ut_status env_test_wait_timeout(ut_env* h, uint32_t polls) {
  if (!h) return UT_ERR_INVALID;
  if (h->test_wait_polls == polls) return UT_OK;
  h->test_wait_polls = polls;
  // captured graphs hold the kernels' arguments: capture again with the new value
  if (h->graph_exec) {
    cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
  }
  if (h->ppo_exec) {
    cudaGraphExecDestroy(h->ppo_exec);
    h->ppo_exec = nullptr;
    h->ppo_key.clear();
  }
  return UT_OK;
}

ut_status env_metrics(ut_env* h, ut_rollout_stats* out) {
  if (!h || !out) return UT_ERR_INVALID;
  double md[2];
  unsigned long long mu[4];
  int status = 0;
  UT_CUDA(h, cudaMemcpyAsync(md, h->d.metrics_d, sizeof(md), cudaMemcpyDeviceToHost, h->stream));
  UT_CUDA(h, cudaMemcpyAsync(mu, h->d.metrics_u, sizeof(mu), cudaMemcpyDeviceToHost, h->stream));
  UT_CUDA(h, cudaMemcpyAsync(&status, h->d.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  UT_CUDA(h, cudaStreamSynchronize(h->stream));
  out->sum_sq_err = md[0];
  out->n_err = (int64_t)mu[0];
  out->rmse = mu[0] ? std::sqrt(md[0] / (double)mu[0]) : 0.0;
  out->reward_sum = md[1];
  out->crash_count = (int64_t)mu[1];
  out->agent_steps = (int64_t)mu[2];
  out->steps = (int64_t)mu[3];
  out->device_status = status;
  out->kernel_launches = h->launches;
  if (status == 2) return fail(h, UT_ERR_TIMEOUT, "a bounded device wait gave up");
  if (status == 3) return fail(h, UT_ERR_INVALID, "an index check of the checked build failed");
  return UT_OK;
}

static ut_status graph_ensure(ut_env* h, int32_t T) {
  UT_CUDA(h, ut::capture_stream_ensure(h));
  const int key = T * 16 + (h->policy_ready ? 1 : 0) + 2 * h->est_mode;  // est_mode 0..4
  if (!h->graph_exec || h->graph_key != key || h->graph_variant != h->pf_variant) {
    if (h->graph_exec) {
      cudaGraphExecDestroy(h->graph_exec);
      h->graph_exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    const int64_t launches_before = h->launches;
    h->capturing = true;
    UT_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < T && e == cudaSuccess; ++t) e = enqueue_step(h, nullptr, h->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
    h->capturing = false;
    h->launches_per_graph = (int)(h->launches - launches_before);
    h->launches = launches_before;
    if (e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(h, e, "rollout capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    h->graph_key = key;
    h->graph_variant = h->pf_variant;
    UT_CUDA(h, cudaGraphUpload(h->graph_exec, h->cap_stream));
  }
  return UT_OK;
}

ut_status rollout_prepare(ut_env* h, int32_t T) {
  if (!h || T < 1) return UT_ERR_INVALID;
  if (!h->reset_done) return fail(h, UT_ERR_STATE, "rollout_prepare before env_reset");
  return graph_ensure(h, T);
}

// The persistent kernel runs the step with the environment's random actions
// and the particle filter: no transformer agent, no learned or LS tracker,
// every-step resampling, and a filter launch shape that covers P.
static bool persistent_ok(const ut_env* h) {
  return !h->policy_ready && h->est_mode == 0 && ut::persistent_supported(h->d, h->pf_variant);
}

ut_status rollout(ut_env* h, int32_t T, ut_rollout_stats* stats) {
  if (!h || T < 1) return UT_ERR_INVALID;
  if (!h->reset_done) return fail(h, UT_ERR_STATE, "rollout before env_reset");
  if (h->rollout_form == 1 && persistent_ok(h)) {
    UT_CUDA(h, env_metrics_reset(h) == UT_OK ? cudaSuccess : cudaErrorUnknown);
    UT_CUDA(h, ut::launch_rollout_persistent(h->d, h->pf_variant, T, h->stream));
    h->launches += 2;
    if (stats) return env_metrics(h, stats);
    return UT_OK;
  }
  ut_status st = graph_ensure(h, T);
  if (st != UT_OK) return st;
  UT_CUDA(h, env_metrics_reset(h) == UT_OK ? cudaSuccess : cudaErrorUnknown);
  h->launches += h->launches_per_graph;
  UT_CUDA(h, cudaEventRecord(h->ev_fork, h->stream));
  UT_CUDA(h, cudaStreamWaitEvent(h->cap_stream, h->ev_fork, 0));
  UT_CUDA(h, cudaGraphLaunch(h->graph_exec, h->cap_stream));
  UT_CUDA(h, cudaEventRecord(h->ev_join, h->cap_stream));
  UT_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  if (stats) return env_metrics(h, stats);
  return UT_OK;
}

int32_t pf_variant_count(void) { return ut::pf_variant_count(); }
int32_t pf_variant_usable(int32_t v, int32_t P) { return ut::pf_variant_valid(v, P) ? 1 : 0; }
const char* pf_variant_label(int32_t v) { return ut::pf_variant_name(v); }

ut_status env_set_pf_variant(ut_env* h, int32_t v) {
  if (!h) return UT_ERR_INVALID;
  if (!ut::pf_variant_valid(v, h->d.P)) return fail(h, UT_ERR_INVALID, "particle-filter variant not usable for this P");
  h->pf_variant = v;
  return UT_OK;
}

ut_status env_get_pf_variant(const ut_env* h, int32_t* v) {
  if (!h || !v) return UT_ERR_INVALID;
  *v = h->pf_variant;
  return UT_OK;
}

ut_status env_set_rollout_form(ut_env* h, int32_t form) {
  if (!h || form < 0 || form > 1) return UT_ERR_INVALID;
  if (form == 1 && !persistent_ok(h))
    return fail(h, UT_ERR_UNSUPPORTED,
                "persistent rollout: needs random actions (no policy), the particle filter (est_mode 0), "
                "every-step resampling and a filter launch shape covering P");
  h->rollout_form = form;
  return UT_OK;
}

ut_status env_get_rollout_form(const ut_env* h, int32_t* form) {
  if (!h || !form) return UT_ERR_INVALID;
  *form = (h->rollout_form == 1 && persistent_ok(h)) ? 1 : 0;
  return UT_OK;
}

namespace {
std::mutex g_tune_mutex;
// (E, A_max, T_max, P, filters) -> (filter variant, rollout form)
std::map<std::tuple<int, int, int, int, int64_t>, std::pair<int, int>> g_tune_cache;

// Device time (ms) of one rollout(T) of the handle in its current form.
ut_status time_rollout(ut_env* h, int32_t T, float* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  UT_CUDA(h, cudaEventCreate(&a));
  UT_CUDA(h, cudaEventCreate(&b));
  UT_CUDA(h, cudaEventRecord(a, h->stream));
  ut_status st = rollout(h, T, nullptr);
  if (st == UT_OK) {
    UT_CUDA(h, cudaEventRecord(b, h->stream));
    UT_CUDA(h, cudaEventSynchronize(b));
    UT_CUDA(h, cudaEventElapsedTime(ms, a, b));
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return st;
}
}  // namespace

ut_status env_autotune(ut_env* h, int32_t reps, int32_t* chosen) {
  if (!h || reps < 1) return UT_ERR_INVALID;
  if (!h->reset_done) return fail(h, UT_ERR_STATE, "env_autotune before env_reset");
  const auto key = std::make_tuple(h->d.E, h->d.AM, h->d.TM, h->d.P, h->F);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      h->pf_variant = it->second.first;
      h->rollout_form = it->second.second;
      if (chosen) *chosen = it->second.first;
      return UT_OK;
    }
  }
  const bool prof_before = h->prof_on;
  double best = 1e30;
  int best_v = h->pf_variant;
  for (int v = 0; v < ut::pf_variant_count(); ++v) {
    if (!ut::pf_variant_valid(v, h->d.P)) continue;
    h->pf_variant = v;
    h->prof_on = false;
    UT_CUDA(h, enqueue_step(h, nullptr, h->stream));  // warm-up (also the smem opt-in)
    h->prof_on = true;
    h->eager_used = 0;
    for (int r = 0; r < reps; ++r) UT_CUDA(h, enqueue_step(h, nullptr, h->stream));
    double ms = 0.0;
    int64_t n = 0;
    ut_status st = env_stage_time(h, &ms, &n);
    if (st != UT_OK) return st;
    const double avg = ms / (double)(n > 0 ? n : 1);
    if (avg < best) {
      best = avg;
      best_v = v;
    }
  }
  h->prof_on = prof_before;
  h->eager_used = 0;
  h->pf_variant = best_v;
  // the rollout form: the captured graph against the persistent kernel (when
  // the handle qualifies), each timed over `reps` steps after one warm-up
  // rollout, with the chosen filter variant
  int form = 0;
  if (persistent_ok(h)) {
    float ms_form[2] = {0.0f, 0.0f};
    for (int f = 0; f < 2; ++f) {
      h->rollout_form = f;
      float warm = 0.0f;
      ut_status st = time_rollout(h, reps, &warm);
      if (st == UT_OK) st = time_rollout(h, reps, &ms_form[f]);
      if (st != UT_OK) return st;
    }
    form = ms_form[1] < ms_form[0] ? 1 : 0;
  }
  h->rollout_form = form;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = std::make_pair(best_v, form);
  }
  if (chosen) *chosen = best_v;
  return UT_OK;
}

ut_status env_profile(ut_env* h, int32_t enable) {
  if (!h) return UT_ERR_INVALID;
  h->prof_on = enable != 0;
  h->eager_used = 0;
  return UT_OK;
}

ut_status env_stage_time(ut_env* h, double* total_ms, int64_t* launches) {
  if (!h || !total_ms || !launches) return UT_ERR_INVALID;
  UT_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->cap_stream) UT_CUDA(h, cudaStreamSynchronize(h->cap_stream));
  double sum = 0.0;
  int64_t n = 0;
  for (size_t k = 0; k < h->eager_used; ++k) {
    float ms = 0.0f;
    UT_CUDA(h, cudaEventElapsedTime(&ms, h->eager_ev[2 * k], h->eager_ev[2 * k + 1]));
    sum += ms;
    ++n;
  }
  h->eager_used = 0;
  *total_ms = sum;
  *launches = n;
  return UT_OK;
}

ut_status env_get_state(const ut_env* hc, ut_state_view* out) {
  ut_env* h = const_cast<ut_env*>(hc);
  if (!h || !out) return UT_ERR_INVALID;
  const EnvDev& d = h->d;
  out->ax = d.ax; out->ay = d.ay; out->apsi = d.apsi;
  out->tx = d.tx; out->ty = d.ty; out->tz = d.tz; out->tpsi = d.tpsi; out->tspeed = d.tspeed;
  out->px = d.px; out->py = d.py; out->pvx = d.pvx; out->pvy = d.pvy;
  out->lpx = d.lpx; out->lpy = d.lpy; out->lpage = d.lpage;
  out->estx = d.estx; out->esty = d.esty;
  out->prev_estx = d.prev_estx; out->prev_esty = d.prev_esty;
  out->prev2_estx = d.prev2_estx; out->prev2_esty = d.prev2_esty;
  out->rudder = d.rudder;
  out->velx = d.velx; out->vely = d.vely;
  out->ring = d.ring_on ? d.ring : nullptr;
  out->ring_head = d.ring_head; out->ring_count = d.ring_count;
  out->h = extension_h(h);
  out->pw = d.pw;
  uint32_t c[2];
  UT_CUDA(h, cudaMemcpyAsync(c, d.counters, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
  UT_CUDA(h, cudaStreamSynchronize(h->stream));
  out->step = c[0];
  out->t_ep = (int32_t)c[1];
  out->n_agents = h->NA;
  out->n_targets = h->NT;
  out->n_filters = h->F;
  return UT_OK;
}

ut_status env_set_state(ut_env* h, const ut_state_view* in) {
  if (!h || !in) return UT_ERR_INVALID;
  const EnvDev& d = h->d;
  const size_t NA = h->NA, NT = h->NT, F = h->F, FP = (size_t)h->F * d.P, AM = d.AM;
  auto cp = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (!src) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, h->stream);
  };
  UT_CUDA(h, cp(d.ax, in->ax, NA * 4));
  UT_CUDA(h, cp(d.ay, in->ay, NA * 4));
  UT_CUDA(h, cp(d.apsi, in->apsi, NA * 4));
  UT_CUDA(h, cp(d.tx, in->tx, NT * 4));
  UT_CUDA(h, cp(d.ty, in->ty, NT * 4));
  UT_CUDA(h, cp(d.tz, in->tz, NT * 4));
  UT_CUDA(h, cp(d.tpsi, in->tpsi, NT * 4));
  UT_CUDA(h, cp(d.tspeed, in->tspeed, NT * 4));
  UT_CUDA(h, cp(d.px, in->px, FP * 4));
  UT_CUDA(h, cp(d.py, in->py, FP * 4));
  UT_CUDA(h, cp(d.pvx, in->pvx, FP * 4));
  UT_CUDA(h, cp(d.pvy, in->pvy, FP * 4));
  if (d.pw) UT_CUDA(h, cp(d.pw, in->pw, FP * 4));
  UT_CUDA(h, cp(d.lpx, in->lpx, NA * AM * 4));
  UT_CUDA(h, cp(d.lpy, in->lpy, NA * AM * 4));
  UT_CUDA(h, cp(d.lpage, in->lpage, NA * AM * 4));
  UT_CUDA(h, cp(d.estx, in->estx, F * 4));
  UT_CUDA(h, cp(d.esty, in->esty, F * 4));
  UT_CUDA(h, cp(d.prev_estx, in->prev_estx, F * 4));
  UT_CUDA(h, cp(d.prev_esty, in->prev_esty, F * 4));
  UT_CUDA(h, cp(d.prev2_estx, in->prev2_estx, F * 4));
  UT_CUDA(h, cp(d.prev2_esty, in->prev2_esty, F * 4));
  UT_CUDA(h, cp(d.rudder, in->rudder, NA * 4));
  UT_CUDA(h, cp(d.velx, in->velx, F * 4));
  UT_CUDA(h, cp(d.vely, in->vely, F * 4));
  if (d.ring_on) UT_CUDA(h, cp(d.ring, in->ring, F * kRing * 16));
  UT_CUDA(h, cp(d.ring_head, in->ring_head, F * 4));
  UT_CUDA(h, cp(d.ring_count, in->ring_count, F * 4));
  uint16_t* hd = extension_h(h);
  if (hd && in->h) UT_CUDA(h, cp(hd, in->h, NA * (size_t)h->cfg.d_model * 2));
  uint32_t c[4] = {in->step, (uint32_t)in->t_ep, 0, 0};
  UT_CUDA(h, cudaMemcpyAsync(d.counters, c, sizeof(c), cudaMemcpyHostToDevice, h->stream));
  UT_CUDA(h, cudaStreamSynchronize(h->stream));
  h->reset_done = true;
  return UT_OK;
}

ut_status env_debug(const ut_env* hc, ut_debug_view* out) {
  ut_env* h = const_cast<ut_env*>(hc);
  if (!h || !out) return UT_ERR_INVALID;
  if (!h->d.debug_on) return fail(h, UT_ERR_STATE, "handle created without UT_FLAG_DEBUG");
  const EnvDev& d = h->d;
  out->range = d.range;
  out->valid = d.valid;
  out->recv = d.recv;
  out->meas = reinterpret_cast<float*>(d.meas);
  out->meas_n = d.meas_n;
  out->pred_px = d.dbg_px;
  out->pred_py = d.dbg_py;
  out->pred_pvx = d.dbg_pvx;
  out->pred_pvy = d.dbg_pvy;
  out->weight = d.dbg_w;
  out->wmax = d.dbg_wmax;
  out->idx = d.dbg_idx;
  return UT_OK;
}

ut_status ut_philox(const uint32_t* ctr_dev, uint64_t seed, uint32_t* out_dev, int64_t n, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!ctr_dev || !out_dev))) return UT_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(ctr_dev) | reinterpret_cast<uintptr_t>(out_dev)) & 15) return UT_ERR_INVALID;
  return launch_philox(ctr_dev, seed, out_dev, n, (cudaStream_t)cuda_stream) == cudaSuccess ? UT_OK : UT_ERR_CUDA;
}

ut_status pf_resample(const float* wmax_dev, const uint64_t* u64_dev, int64_t n_filters, int32_t P, int32_t* idx_dev,
                      void* cuda_stream) {
  if (n_filters < 0 || P < 1 || P > UT_MAX_PARTICLES || n_filters > 0x7fffffff) return UT_ERR_INVALID;
  if (n_filters > 0 && (!wmax_dev || !u64_dev || !idx_dev)) return UT_ERR_INVALID;
  return launch_pf_resample(wmax_dev, u64_dev, n_filters, P, idx_dev, (cudaStream_t)cuda_stream) == cudaSuccess
             ? UT_OK
             : UT_ERR_CUDA;
}

}  // extern "C"
