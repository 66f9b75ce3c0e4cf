// Rollout recording for the TransfMAPPO update (Sec. II-B, Sec. III-B.1):
// the critic's global-state tokens (Sec. III-A: the true 3-D position,
// velocity and direction of every entity), and the per-step snapshot and
// record of the actors' inputs, actions, behaviour log-probabilities,
// rewards and episode ends.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/utrack.h"
#include "env.cuh"
#include "runtime.cuh"
#include "tfm.cuh"

#include <vector>

namespace ut {
namespace {

// One thread per (env, slot): agents then targets packed from slot 0, each
// [x/S, y/S, z/S, vx, vy, cos psi, sin psi, kind]; zero padding.
__global__ void state_tokens_kernel(EnvDev d, float* __restrict__ tok, int32_t* __restrict__ n_ent) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)d.E * d.NS) return;
  const int e = (int)(i / d.NS), s = (int)(i - (long long)e * d.NS);
  const int a0 = d.agent_off[e], A = d.agent_off[e + 1] - a0;
  const int k0 = d.target_off[e], T = d.target_off[e + 1] - k0;
  float q[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const float invS = 1.0f / d.S;
  if (s < A) {
    const int a = a0 + s;
    float sn, cs;
    sincosf(d.apsi[a], &sn, &cs);
    q[0] = d.ax[a] * invS;
    q[1] = d.ay[a] * invS;
    q[3] = d.agent_speed * cs;
    q[4] = d.agent_speed * sn;
    q[5] = cs;
    q[6] = sn;
    q[7] = 1.0f;
  } else if (s < A + T) {
    const int k = k0 + s - A;
    float sn, cs;
    sincosf(d.tpsi[k], &sn, &cs);
    q[0] = d.tx[k] * invS;
    q[1] = d.ty[k] * invS;
    q[2] = d.tz[k] * invS;
    q[3] = d.tspeed[k] * cs;
    q[4] = d.tspeed[k] * sn;
    q[5] = cs;
    q[6] = sn;
  }
  float4* o = reinterpret_cast<float4*>(tok + i * 8);
  o[0] = make_float4(q[0], q[1], q[2], q[3]);
  o[1] = make_float4(q[4], q[5], q[6], q[7]);
  if (s == 0) n_ent[e] = A + T;
}

// Entity counts of the agents (A_e + T_e), one thread per env.
__global__ void snapshot_nent_kernel(EnvDev d, int32_t* __restrict__ n_ent) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  const int a0 = d.agent_off[e], a1 = d.agent_off[e + 1];
  const int ne = (a1 - a0) + (d.target_off[e + 1] - d.target_off[e]);
  for (int a = a0; a < a1; ++a) n_ent[a] = ne;
}

// The agents' recurrent embedding (BF16) widened to FP32, one thread per value.
__global__ void snapshot_h_kernel(const uint16_t* __restrict__ h_bf16, long long n, float* __restrict__ h_out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) h_out[i] = __uint_as_float((uint32_t)h_bf16[i] << 16);
}

// Log-probability of each agent's action under its logits (log-softmax in
// FP32), one thread per agent.
__global__ void logp_kernel(const float* __restrict__ logits, const int32_t* __restrict__ act, int n_act,
                            long long NA, float* __restrict__ logp) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NA) return;
  const float* z = logits + i * n_act;
  float mx = -INFINITY;
  for (int k = 0; k < n_act; ++k) mx = fmaxf(mx, z[k]);
  float s = 0.0f;
  for (int k = 0; k < n_act; ++k) s += expf(z[k] - mx);
  int a = act[i];
  a = a < 0 ? 0 : (a >= n_act ? n_act - 1 : a);
  logp[i] = z[a] - mx - logf(s);
}

inline unsigned blocks(long long n) { return (unsigned)((n + 255) / 256); }

// One collection step t of env_ppo_collect on stream s (t == T: the last
// critic forward only).
cudaError_t collect_step(ut_env* h, ut_tfm* critic, const ut_ppo_buffers& b, int t, int T, cudaStream_t s) {
  const long long E = h->d.E, NA = h->NA, NS = h->d.NS, dm = h->cfg.d_model;
  const long long dc = tfm_info(critic).d;
  float* ctok = b.ctokens + t * E * NS * 8;
  int32_t* cne = b.cn_ent + t * E;
  state_tokens_kernel<<<blocks(E * NS), 256, 0, s>>>(h->d, ctok, cne);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = tfm_forward_on(critic, ctok, cne, b.ch + t * E * dc, E, b.value + t * E, b.ch + (t + 1) * E * dc, s);
  if (e != cudaSuccess || t == T) return e;
  e = cudaMemcpyAsync(b.tokens + t * NA * NS * 8, h->d.obs, (size_t)NA * NS * 8 * 2, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  snapshot_nent_kernel<<<blocks(E), 256, 0, s>>>(h->d, b.n_ent + t * NA);
  snapshot_h_kernel<<<blocks(NA * dm), 256, 0, s>>>(extension_h(h), NA * dm, b.h + t * NA * dm);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = enqueue_step(h, nullptr, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.actions + t * NA, h->d.actions, (size_t)NA * 4, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  logp_kernel<<<blocks(NA), 256, 0, s>>>(extension_logits(h), h->d.actions, h->cfg.n_actions, NA, b.logp + t * NA);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.reward + t * E, h->d.reward, (size_t)E * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b.done + t * E, h->d.done, (size_t)E * 4, cudaMemcpyDeviceToDevice, s);
  return e;
}

ut_status cuda_fail(ut_env* h, const char* what, cudaError_t e) {
  h->err = std::string(what) + ": " + cudaGetErrorString(e);
  return UT_ERR_CUDA;
}

}  // namespace
}  // namespace ut

using namespace ut;

extern "C" ut_status env_state_tokens(ut_env* h, float* tokens_dev, int32_t* n_ent_dev) {
  if (!h || !tokens_dev || !n_ent_dev) return UT_ERR_INVALID;
  state_tokens_kernel<<<blocks((long long)h->d.E * h->d.NS), 256, 0, h->stream>>>(h->d, tokens_dev, n_ent_dev);
  h->launches += 1;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? UT_OK : cuda_fail(h, "env_state_tokens", e);
}

extern "C" ut_status env_ppo_snapshot(ut_env* h, uint16_t* tokens_dev, int32_t* n_ent_dev, float* h_dev) {
  if (!h) return UT_ERR_INVALID;
  const uint16_t* hb = extension_h(h);
  if (!hb) {
    h->err = "env_ppo_snapshot: handle created with d_model == 0";
    return UT_ERR_STATE;
  }
  cudaError_t e = cudaSuccess;
  if (tokens_dev)
    e = cudaMemcpyAsync(tokens_dev, h->d.obs, (size_t)h->NA * h->d.NS * 8 * 2, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess && n_ent_dev) {
    snapshot_nent_kernel<<<blocks(h->d.E), 256, 0, h->stream>>>(h->d, n_ent_dev);
    h->launches += 1;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && h_dev) {
    const long long n = (long long)h->NA * h->cfg.d_model;
    snapshot_h_kernel<<<blocks(n), 256, 0, h->stream>>>(hb, n, h_dev);
    h->launches += 1;
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? UT_OK : cuda_fail(h, "env_ppo_snapshot", e);
}

extern "C" ut_status env_ppo_record(ut_env* h, int32_t* actions_dev, float* logp_dev, float* reward_dev,
                                    int32_t* done_dev) {
  if (!h) return UT_ERR_INVALID;
  const float* logits = extension_logits(h);
  if (!logits || !h->policy_ready) {
    h->err = "env_ppo_record: no transformer agent weights";
    return UT_ERR_STATE;
  }
  cudaError_t e = cudaSuccess;
  if (actions_dev)
    e = cudaMemcpyAsync(actions_dev, h->d.actions, (size_t)h->NA * 4, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess && logp_dev) {
    logp_kernel<<<blocks(h->NA), 256, 0, h->stream>>>(logits, h->d.actions, h->cfg.n_actions, h->NA, logp_dev);
    h->launches += 1;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && reward_dev)
    e = cudaMemcpyAsync(reward_dev, h->d.reward, (size_t)h->d.E * 4, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess && done_dev)
    e = cudaMemcpyAsync(done_dev, h->d.done, (size_t)h->d.E * 4, cudaMemcpyDeviceToDevice, h->stream);
  return e == cudaSuccess ? UT_OK : cuda_fail(h, "env_ppo_record", e);
}

extern "C" ut_status env_ppo_collect(ut_env* h, ut_tfm* critic, int32_t T, const ut_ppo_buffers* b) {
  if (!h || !critic || !b || T < 1) return UT_ERR_INVALID;
  if (!b->tokens || !b->n_ent || !b->h || !b->actions || !b->logp || !b->reward || !b->done || !b->ctokens ||
      !b->cn_ent || !b->ch || !b->value)
    return UT_ERR_INVALID;
  if (!h->reset_done || !h->policy_ready || !extension_h(h)) {
    h->err = "env_ppo_collect: needs env_reset and the transformer agent's weights";
    return UT_ERR_STATE;
  }
  const TfmInfo ci = tfm_info(critic);
  if (ci.n_out != 1 || ci.tokens_bf16 != 0 || ci.n_slots != h->d.NS || ci.max_batch < h->d.E) {
    h->err = "env_ppo_collect: the critic needs n_out 1, FP32 tokens, the env's slots and max_batch >= n_envs";
    return UT_ERR_INVALID;
  }
  cudaError_t e = capture_stream_ensure(h);
  if (e != cudaSuccess) return cuda_fail(h, "env_ppo_collect", e);
  // the graph is rebuilt when any argument or the step's configuration changes
  std::vector<uintptr_t> key = {(uintptr_t)critic, (uintptr_t)T, (uintptr_t)h->pf_variant, (uintptr_t)h->est_mode};
  for (const void* p : {(const void*)b->tokens, (const void*)b->n_ent, (const void*)b->h, (const void*)b->actions,
                        (const void*)b->logp, (const void*)b->reward, (const void*)b->done, (const void*)b->ctokens,
                        (const void*)b->cn_ent, (const void*)b->ch, (const void*)b->value})
    key.push_back((uintptr_t)p);
  if (!h->ppo_exec || h->ppo_key != key) {
    if (h->ppo_exec) {
      cudaGraphExecDestroy(h->ppo_exec);
      h->ppo_exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    const int64_t launches_before = h->launches;
    h->capturing = true;
    e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    cudaError_t ec = cudaSuccess;
    for (int t = 0; t <= T && e == cudaSuccess && ec == cudaSuccess; ++t) ec = collect_step(h, critic, *b, t, T, h->cap_stream);
    const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(h->cap_stream, &graph) : e;
    h->capturing = false;
    h->launches = launches_before;
    if (ec != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(h, "env_ppo_collect capture", ec != cudaSuccess ? ec : e2);
    }
    e = cudaGraphInstantiate(&h->ppo_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, "env_ppo_collect instantiate", e);
    h->ppo_key = key;
  }
  e = cudaEventRecord(h->ev_fork, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->cap_stream, h->ev_fork, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(h->ppo_exec, h->cap_stream);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->cap_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_join, 0);
  return e == cudaSuccess ? UT_OK : cuda_fail(h, "env_ppo_collect", e);
}
