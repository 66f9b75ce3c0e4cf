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

// Entity counts of the agents (A_e + T_e) and their recurrent embedding
// (BF16) widened to FP32; one thread per agent.
__global__ void snapshot_kernel(EnvDev d, const uint16_t* __restrict__ h_bf16, int dm, int32_t* __restrict__ n_ent,
                                float* __restrict__ h_out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.E) return;
  const int e = (int)i;
  const int a0 = d.agent_off[e], a1 = d.agent_off[e + 1];
  const int ne = (a1 - a0) + (d.target_off[e + 1] - d.target_off[e]);
  for (int a = a0; a < a1; ++a) {
    if (n_ent) n_ent[a] = ne;
    if (h_out)
      for (int j = 0; j < dm; ++j)
        h_out[(long long)a * dm + j] = __uint_as_float((uint32_t)h_bf16[(long long)a * dm + j] << 16);
  }
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
  if (e == cudaSuccess && (n_ent_dev || h_dev)) {
    snapshot_kernel<<<blocks(h->d.E), 256, 0, h->stream>>>(h->d, hb, h->cfg.d_model, n_ent_dev, h_dev);
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
