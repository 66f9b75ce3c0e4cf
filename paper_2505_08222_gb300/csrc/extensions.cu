// Hooks through which the transformer agent (and the learned estimator) plug
// into the environment step, and their C-ABI entry points.
#include <cstring>
#include <vector>

#include "../../include/utrack.h"
#include "policy.cuh"
#include "runtime.cuh"

struct PolicyState {
  int d = 0, L = 0, H = 0, n_act = 0;
  bool supported = false;
  unsigned char* wimg = nullptr;
  float* vec = nullptr;
  float* emb = nullptr;
  float* head = nullptr;
  uint16_t* h = nullptr;
  float* logits = nullptr;
  int32_t* n_ent = nullptr;
};

namespace ut {

static PolicyDev policy_dev(ut_env* h) {
  PolicyState* ps = h->policy;
  PolicyDev p;
  std::memset(&p, 0, sizeof(p));
  p.NA = h->NA;
  p.NS = h->d.NS;
  p.R = 1 + h->d.NS;
  p.apt = 128 / p.R;
  p.n_act = ps->n_act;
  p.L = ps->L;
  p.tokens = h->d.obs;
  p.n_ent = ps->n_ent;
  p.h = ps->h;
  p.logits = ps->logits;
  p.actions = h->d.actions;
  p.emb_w = ps->emb;
  p.emb_b = ps->emb + (size_t)ps->d * 8;
  p.wimg = ps->wimg;
  p.vec = ps->vec;
  p.lnf_g = ps->head;
  p.lnf_b = ps->head + ps->d;
  p.head_w = ps->head + 2 * ps->d;
  p.head_b = ps->head + 2 * ps->d + (size_t)ps->n_act * ps->d;
  p.seed = h->d.seed;
  p.counters = h->d.counters;
  p.sample = 1;
  p.status = h->d.status;
  return p;
}

ut_status extension_create(ut_env* h) {
  const ut_config& c = h->cfg;
  if (c.d_model <= 0) return UT_OK;
  PolicyState* ps = new PolicyState();
  h->policy = ps;
  ps->d = c.d_model;
  ps->L = c.n_layers;
  ps->H = c.n_heads;
  ps->n_act = c.n_actions;
  ps->supported = policy_supported(c.d_model, c.n_heads);
  ps->h = (uint16_t*)env_alloc(h, (size_t)h->NA * c.d_model * 2);
  ps->logits = (float*)env_alloc(h, (size_t)h->NA * c.n_actions * 4);
  ps->n_ent = (int32_t*)env_alloc(h, (size_t)h->NA * 4);
  if (!ps->h || !ps->logits || !ps->n_ent) {
    h->err = "policy buffers: allocation failed";
    return UT_ERR_NOMEM;
  }
  std::vector<int32_t> ne;
  ne.reserve(h->NA);
  for (size_t e = 0; e < h->agents_per_env.size(); ++e)
    for (int a = 0; a < h->agents_per_env[e]; ++a) ne.push_back(h->agents_per_env[e] + h->targets_per_env[e]);
  if (cudaMemcpyAsync(ps->n_ent, ne.data(), ne.size() * 4, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    h->err = "policy buffers: copy failed";
    return UT_ERR_CUDA;
  }
  return UT_OK;
}

void extension_destroy(ut_env* h) {
  delete h->policy;
  h->policy = nullptr;
}

cudaError_t extension_reset(ut_env* h, cudaStream_t s) {
  if (!h->policy) return cudaSuccess;
  return cudaMemsetAsync(h->policy->h, 0, (size_t)h->NA * h->policy->d * 2, s);
}

cudaError_t extension_policy_actions(ut_env* h, cudaStream_t s) {
  if (!h->policy_ready) return cudaErrorNotSupported;
  return launch_policy(policy_dev(h), h->policy->d, s);
}

int extension_policy_kernels(ut_env*) { return 1; }
cudaError_t extension_estimate(ut_env*, cudaStream_t) { return cudaErrorNotReady; }
const float* extension_logits(ut_env* h) { return h->policy ? h->policy->logits : nullptr; }
uint16_t* extension_h(ut_env* h) { return h->policy ? h->policy->h : nullptr; }

}  // namespace ut

using namespace ut;

extern "C" ut_status env_set_policy(ut_env* h, const float* params_host, int64_t n_params) {
  if (!h || !params_host) return UT_ERR_INVALID;
  PolicyState* ps = h->policy;
  if (!ps) {
    h->err = "env_set_policy: handle created with d_model == 0";
    return UT_ERR_STATE;
  }
  if (!ps->supported) {
    h->err = "env_set_policy: only d_model 64 or 128 with 16-wide heads are built";
    return UT_ERR_UNSUPPORTED;
  }
  if (n_params != policy_param_count(ps->d, ps->L, ps->n_act)) {
    h->err = "env_set_policy: parameter count does not match (d_model, n_layers, n_actions)";
    return UT_ERR_INVALID;
  }
  std::vector<unsigned char> img;
  std::vector<float> vec, emb, head;
  policy_pack(ps->d, ps->L, ps->n_act, params_host, img, vec, emb, head);
  if (!ps->wimg) {
    ps->wimg = (unsigned char*)env_alloc(h, img.size());
    ps->vec = (float*)env_alloc(h, vec.size() * 4);
    ps->emb = (float*)env_alloc(h, emb.size() * 4);
    ps->head = (float*)env_alloc(h, head.size() * 4);
    if (!ps->wimg || !ps->vec || !ps->emb || !ps->head) {
      h->err = "env_set_policy: allocation failed";
      return UT_ERR_NOMEM;
    }
  }
  cudaError_t e = cudaMemcpyAsync(ps->wimg, img.data(), img.size(), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ps->vec, vec.data(), vec.size() * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ps->emb, emb.data(), emb.size() * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ps->head, head.data(), head.size() * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    h->err = std::string("env_set_policy: ") + cudaGetErrorString(e);
    return UT_ERR_CUDA;
  }
  h->policy_ready = true;
  return UT_OK;
}

extern "C" ut_status policy_forward(ut_env* h, const uint16_t* tokens_dev, const int32_t* n_ent_dev, uint16_t* h_dev,
                                    float* logits_dev, int32_t* actions_dev, int64_t n_agents, int32_t n_slots,
                                    uint32_t step, void* cuda_stream) {
  if (!h) return UT_ERR_INVALID;
  if (!h->policy_ready) {
    h->err = "policy_forward: no policy weights set";
    return UT_ERR_STATE;
  }
  if (n_agents < 0 || n_slots < 1 || n_slots > 127 || !tokens_dev || !n_ent_dev || !h_dev || !logits_dev) {
    h->err = "policy_forward: invalid arguments";
    return UT_ERR_INVALID;
  }
  if (reinterpret_cast<uintptr_t>(tokens_dev) & 15) {
    h->err = "policy_forward: tokens must be 16-byte aligned";
    return UT_ERR_INVALID;
  }
  PolicyDev p = policy_dev(h);
  p.NA = n_agents;
  p.NS = n_slots;
  p.R = 1 + n_slots;
  p.apt = 128 / p.R;
  p.tokens = tokens_dev;
  p.n_ent = n_ent_dev;
  p.h = h_dev;
  p.logits = logits_dev;
  p.actions = actions_dev;
  p.sample = actions_dev ? 1 : 0;
  p.counters = nullptr;
  p.step = step;
  cudaError_t e = launch_policy(p, h->policy->d, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) {
    h->err = std::string("policy_forward: ") + cudaGetErrorString(e);
    return UT_ERR_CUDA;
  }
  return UT_OK;
}
