// Hooks through which the transformer agent (and the learned estimator) plug
// into the environment step, and their C-ABI entry points.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/utrack.h"
#include "estimator.cuh"
#include "policy.cuh"
#include "runtime.cuh"

struct EstimatorState {
  bool weights_set = false;
  float* master = nullptr;  // [NPARAM]
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  unsigned char* img = nullptr;
  int adam_t = 0;
  // training buffers (sized for batch_cap rows)
  int batch_cap = 0;
  float* z = nullptr;
  uint16_t* a = nullptr;
  uint16_t* dz = nullptr;
  float* out = nullptr;
  int32_t* rows = nullptr;
  double* loss = nullptr;
  // fixed-order partial sums of the backward pass
  float* part_b = nullptr;
  double* part_loss = nullptr;
  float* part_w = nullptr;
};

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
  p.gid_agent = h->d.gid_agent;
  p.counters = h->d.counters;
  p.sample = 1;
  p.status = h->d.status;
  p.test_wait_polls = h->test_wait_polls;
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
  delete h->est;
  h->est = nullptr;
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
cudaError_t extension_estimate_impl(ut_env* h, cudaStream_t s);
cudaError_t extension_estimate(ut_env* h, cudaStream_t s) { return extension_estimate_impl(h, s); }
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
  if (!ps->wimg) {  // all or nothing (a failed attempt's buffers stay owned by the handle)
    unsigned char* wimg = (unsigned char*)env_alloc(h, img.size());
    float* vec_d = (float*)env_alloc(h, vec.size() * 4);
    float* emb_d = (float*)env_alloc(h, emb.size() * 4);
    float* head_d = (float*)env_alloc(h, head.size() * 4);
    if (!wimg || !vec_d || !emb_d || !head_d) {
      h->err = "env_set_policy: allocation failed";
      return UT_ERR_NOMEM;
    }
    ps->vec = vec_d;
    ps->emb = emb_d;
    ps->head = head_d;
    ps->wimg = wimg;
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
  if (n_agents < 0 || n_slots < 1 || n_slots > UT_MAX_AGENTS + UT_MAX_TARGETS || !tokens_dev || !n_ent_dev ||
      !h_dev || !logits_dev) {
    h->err = "policy_forward: invalid arguments";
    return UT_ERR_INVALID;
  }
  if ((reinterpret_cast<uintptr_t>(tokens_dev) | reinterpret_cast<uintptr_t>(h_dev)) & 15) {
    h->err = "policy_forward: tokens and h must be 16-byte aligned";
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

// ---------------------------------------------------------------------------
// Learned range-only estimator
// ---------------------------------------------------------------------------



namespace {

EstimatorState* est_state(ut_env* h) {
  if (!h->est) h->est = new EstimatorState();
  return h->est;
}

ut_status est_fail(ut_env* h, ut_status st, const char* msg) {
  h->err = msg;
  return st;
}

ut_status est_alloc_weights(ut_env* h) {
  EstimatorState* es = est_state(h);
  if (es->master) return UT_OK;
  // all or nothing: a failed attempt leaves the state unset (its partial
  // buffers stay owned by the handle until env_destroy), so a later call
  // allocates again instead of finding half a set
  float* master = (float*)env_alloc(h, est::NPARAM * 4);
  float* m = (float*)env_alloc(h, est::NPARAM * 4);
  float* v = (float*)env_alloc(h, est::NPARAM * 4);
  float* grad = (float*)env_alloc(h, est::NPARAM * 4);
  unsigned char* img = (unsigned char*)env_alloc(h, est::IMG_BYTES);
  double* loss = (double*)env_alloc(h, 8);
  if (!master || !m || !v || !grad || !img || !loss) return est_fail(h, UT_ERR_NOMEM, "estimator: allocation failed");
  es->m = m;
  es->v = v;
  es->grad = grad;
  es->img = img;
  es->loss = loss;
  es->master = master;
  return UT_OK;
}

ut_status est_alloc_batch(ut_env* h, int B) {
  EstimatorState* es = est_state(h);
  if (es->batch_cap >= B) return UT_OK;
  // earlier (smaller) buffers stay owned by the handle until destroy
  es->z = (float*)env_alloc(h, (size_t)3 * B * est::HID * 4);
  es->a = (uint16_t*)env_alloc(h, (size_t)3 * B * est::HID * 2);
  es->dz = (uint16_t*)env_alloc(h, (size_t)3 * B * est::HID * 2);
  es->out = (float*)env_alloc(h, (size_t)B * 2 * 4);
  es->rows = (int32_t*)env_alloc(h, (size_t)B * 4);
  const size_t n_cta = ((size_t)B + 127) / 128;
  es->part_b = (float*)env_alloc(h, n_cta * est::NB_PART * 4);
  es->part_loss = (double*)env_alloc(h, n_cta * 8);
  if (!es->part_w) es->part_w = (float*)env_alloc(h, (size_t)est::kWgradSplits * est::NW_PART * 4);
  if (!es->z || !es->a || !es->dz || !es->out || !es->rows || !es->part_b || !es->part_loss || !es->part_w)
    return est_fail(h, UT_ERR_NOMEM, "estimator: batch allocation failed");
  es->batch_cap = B;
  return UT_OK;
}

est::Net est_net(ut_env* h) {
  est::Net n;
  n.img = h->est->img;
  n.master = h->est->master;
  return n;
}

// Forward + backward of one batch into es->grad (cleared first) and es->loss.
cudaError_t est_grad_batch(ut_env* h, const float* X, const float* Y, const int32_t* rows, int B, float huber) {
  EstimatorState* es = h->est;
  cudaStream_t s = h->stream;
  cudaError_t e = cudaMemsetAsync(es->grad, 0, est::NPARAM * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(es->loss, 0, 8, s);
  if (e == cudaSuccess) e = est::launch_forward(est_net(h), X, rows, B, es->out, es->z, es->a, s);
  if (e != cudaSuccess) return e;
  est::TrainBufs t;
  t.X = X;
  t.Y = Y;
  t.rows = rows;
  t.z = es->z;
  t.a = es->a;
  t.out = es->out;
  t.dz = es->dz;
  t.grad = es->grad;
  t.loss = es->loss;
  t.part_b = es->part_b;
  t.part_loss = es->part_loss;
  t.part_w = es->part_w;
  t.huber = huber;
  t.B = B;
  return est::launch_backward(est_net(h), t, s);
}

}  // namespace

namespace ut {
cudaError_t extension_estimate_impl(ut_env* h, cudaStream_t s) {
  if (h->est_mode == 4) return launch_ls_update(h->d, s);
  if (h->est_mode < 1 || !h->est || !h->est->weights_set) return cudaErrorNotReady;
  return est::launch_forward_env(est_net(h), h->d, h->est_mode - 1, h->test_wait_polls, s);
}
}  // namespace ut

extern "C" ut_status est_set_weights(ut_env* h, const float* params_host, int64_t n_params) {
  if (!h || !params_host) return UT_ERR_INVALID;
  if (n_params != est::NPARAM) return est_fail(h, UT_ERR_INVALID, "est_set_weights: parameter count mismatch");
  ut_status st = est_alloc_weights(h);
  if (st != UT_OK) return st;
  EstimatorState* es = h->est;
  cudaError_t e = cudaMemcpyAsync(es->master, params_host, est::NPARAM * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(es->m, 0, est::NPARAM * 4, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(es->v, 0, est::NPARAM * 4, h->stream);
  if (e == cudaSuccess) e = est::launch_pack(es->master, es->img, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return est_fail(h, UT_ERR_CUDA, cudaGetErrorString(e));
  es->adam_t = 0;
  es->weights_set = true;
  return UT_OK;
}

extern "C" ut_status est_get_weights(ut_env* h, float* params_host, int64_t n_params) {
  if (!h || !params_host) return UT_ERR_INVALID;
  if (!h->est || !h->est->weights_set) return est_fail(h, UT_ERR_STATE, "est_get_weights: no weights");
  if (n_params != est::NPARAM) return est_fail(h, UT_ERR_INVALID, "est_get_weights: parameter count mismatch");
  cudaError_t e = cudaMemcpyAsync(params_host, h->est->master, est::NPARAM * 4, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? UT_OK : est_fail(h, UT_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" ut_status est_set_mode(ut_env* h, int32_t mode) {
  if (!h || mode < 0 || mode > 4) return UT_ERR_INVALID;
  if (mode == 4 && !h->d.ring_on) return est_fail(h, UT_ERR_STATE, "est_set_mode: handle created without UT_FLAG_RING");
  if (mode >= 1 && mode <= 3) {
    if (!h->est || !h->est->weights_set) return est_fail(h, UT_ERR_STATE, "est_set_mode: no estimator weights");
    if (!h->d.ring_on) return est_fail(h, UT_ERR_STATE, "est_set_mode: handle created without UT_FLAG_RING");
  }
  h->est_mode = mode;
  return UT_OK;
}

extern "C" ut_status est_forward(ut_env* h, const float* X_dev, float* out_dev, int64_t n_rows) {
  if (!h || n_rows < 0 || n_rows > 0x7fffffff || (n_rows && (!X_dev || !out_dev))) return UT_ERR_INVALID;
  if (!h->est || !h->est->weights_set) return est_fail(h, UT_ERR_STATE, "est_forward: no weights");
  if (reinterpret_cast<uintptr_t>(X_dev) & 15) return est_fail(h, UT_ERR_INVALID, "est_forward: X not 16-byte aligned");
  cudaError_t e = est::launch_forward(est_net(h), X_dev, nullptr, (int)n_rows, out_dev, nullptr, nullptr, h->stream);
  return e == cudaSuccess ? UT_OK : est_fail(h, UT_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" ut_status est_record(ut_env* h, float* feat_dev, float* label_dev) {
  if (!h || !feat_dev || !label_dev) return UT_ERR_INVALID;
  if (!h->d.ring_on) return est_fail(h, UT_ERR_STATE, "est_record: handle created without UT_FLAG_RING");
  if (reinterpret_cast<uintptr_t>(feat_dev) & 15) return est_fail(h, UT_ERR_INVALID, "est_record: misaligned");
  cudaError_t e = est::launch_record(h->d, feat_dev, label_dev, h->stream);
  return e == cudaSuccess ? UT_OK : est_fail(h, UT_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" ut_status est_loss_grad(ut_env* h, const float* X_dev, const float* Y_dev, int64_t n_rows, int32_t B,
                                   uint64_t seed, uint32_t step, float huber_delta, float* grad_dev,
                                   double* loss_host) {
  if (!h || !X_dev || !Y_dev || n_rows < 1 || n_rows >= (1ll << 32) || B < 1 || B > (1 << 22) || !grad_dev ||
      !(huber_delta >= 0.0f))
    return UT_ERR_INVALID;
  if (!h->est || !h->est->weights_set) return est_fail(h, UT_ERR_STATE, "est_loss_grad: no weights");
  ut_status st = est_alloc_batch(h, B);
  if (st != UT_OK) return st;
  const int32_t* rows = nullptr;
  if (B != n_rows) {
    const cudaError_t er = est::launch_batch_rows(h->est->rows, B, n_rows, seed, step, h->stream);
    if (er != cudaSuccess) return est_fail(h, UT_ERR_CUDA, cudaGetErrorString(er));
    rows = h->est->rows;
  }
  cudaError_t e = est_grad_batch(h, X_dev, Y_dev, rows, B, huber_delta);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(grad_dev, h->est->grad, est::NPARAM * 4, cudaMemcpyDeviceToDevice, h->stream);
  double loss = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&loss, h->est->loss, 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return est_fail(h, UT_ERR_CUDA, cudaGetErrorString(e));
  if (loss_host) *loss_host = loss;
  return UT_OK;
}

extern "C" ut_status est_adam_step(ut_env* h, const float* grad_dev, float lr, float beta1, float beta2, float eps) {
  if (!h || !grad_dev || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
      !(eps > 0.0f))
    return UT_ERR_INVALID;
  if (!h->est || !h->est->weights_set) return est_fail(h, UT_ERR_STATE, "est_adam_step: no weights");
  EstimatorState* es = h->est;
  es->adam_t += 1;
  cudaError_t e = est::launch_adam(es->master, es->m, es->v, grad_dev, es->adam_t, lr, beta1, beta2, eps, es->img,
                                   h->stream);
  return e == cudaSuccess ? UT_OK : est_fail(h, UT_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" ut_status est_train(ut_env* h, const float* X_dev, const float* Y_dev, int64_t n_rows,
                               const ut_est_train_config* cfg, ut_est_train_stats* out) {
  if (!h || !X_dev || !Y_dev || !cfg || n_rows < 1 || n_rows >= (1ll << 32)) return UT_ERR_INVALID;
  if (cfg->steps < 1 || cfg->batch < 1 || cfg->batch > (1 << 22) || !(cfg->lr > 0.0f)) return UT_ERR_INVALID;
  if (!h->est || !h->est->weights_set) return est_fail(h, UT_ERR_STATE, "est_train: no initial weights");
  const int B = cfg->batch;
  ut_status st = est_alloc_batch(h, B);
  if (st != UT_OK) return st;
  EstimatorState* es = h->est;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, h->stream);
  double first = -1.0, last = 0.0;
  const bool full = (B == n_rows);  // the whole dataset as one batch, in order
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < cfg->steps && e == cudaSuccess; ++s) {
    const int32_t* rows = nullptr;
    if (!full) {
      e = est::launch_batch_rows(es->rows, B, n_rows, cfg->seed, (uint32_t)s, h->stream);
      rows = es->rows;
    }
    if (e == cudaSuccess) e = est_grad_batch(h, X_dev, Y_dev, rows, B, cfg->huber_delta);
    // cosine decay of the learning rate over the run (reading C18)
    const double frac = cfg->steps > 1 ? (double)s / (double)(cfg->steps - 1) : 0.0;
    const float lr = cfg->cosine ? (float)(cfg->lr * 0.5 * (1.0 + std::cos(3.141592653589793 * frac))) : cfg->lr;
    es->adam_t += 1;
    if (e == cudaSuccess)
      e = est::launch_adam(es->master, es->m, es->v, es->grad, es->adam_t, lr, cfg->beta1, cfg->beta2, cfg->eps,
                           es->img, h->stream);
    if (e == cudaSuccess && (s == 0 || s == cfg->steps - 1)) {
      double l = 0.0;
      e = cudaMemcpyAsync(&l, es->loss, 8, cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (s == 0) first = l;
      last = l;
    }
  }
  cudaEventRecord(e1, h->stream);
  cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return est_fail(h, UT_ERR_CUDA, cudaGetErrorString(e));
  if (out) {
    out->loss_first = first;
    out->loss_last = last;
    out->ms = ms;
    out->rows_seen = (int64_t)cfg->steps * B;
  }
  return UT_OK;
}

extern "C" ut_status est_save(ut_env* h, const char* path) {
  if (!h || !path) return UT_ERR_INVALID;
  if (!h->est || !h->est->weights_set) return est_fail(h, UT_ERR_STATE, "est_save: no weights");
  std::vector<float> buf(3 * est::NPARAM);
  EstimatorState* es = h->est;
  cudaError_t e = cudaMemcpyAsync(buf.data(), es->master, est::NPARAM * 4, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(buf.data() + est::NPARAM, es->m, est::NPARAM * 4, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(buf.data() + 2 * est::NPARAM, es->v, est::NPARAM * 4, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return est_fail(h, UT_ERR_CUDA, cudaGetErrorString(e));
  FILE* f = std::fopen(path, "wb");
  if (!f) return est_fail(h, UT_ERR_INVALID, "est_save: cannot open file");
  const uint32_t hdr[4] = {0x55545245u /* "UTRE" */, 1u, (uint32_t)est::NPARAM, (uint32_t)es->adam_t};
  bool ok = std::fwrite(hdr, 4, 4, f) == 4 && std::fwrite(buf.data(), 4, buf.size(), f) == buf.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? UT_OK : est_fail(h, UT_ERR_INVALID, "est_save: write failed");
}

extern "C" ut_status est_load(ut_env* h, const char* path) {
  if (!h || !path) return UT_ERR_INVALID;
  FILE* f = std::fopen(path, "rb");
  if (!f) return est_fail(h, UT_ERR_INVALID, "est_load: cannot open file");
  uint32_t hdr[4] = {0, 0, 0, 0};
  std::vector<float> buf(3 * est::NPARAM);
  bool ok = std::fread(hdr, 4, 4, f) == 4 && hdr[0] == 0x55545245u && hdr[1] == 1u && hdr[2] == (uint32_t)est::NPARAM &&
            std::fread(buf.data(), 4, buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok) return est_fail(h, UT_ERR_INVALID, "est_load: not an estimator file of this layout");
  ut_status st = est_set_weights(h, buf.data(), est::NPARAM);
  if (st != UT_OK) return st;
  EstimatorState* es = h->est;
  cudaError_t e = cudaMemcpyAsync(es->m, buf.data() + est::NPARAM, est::NPARAM * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(es->v, buf.data() + 2 * est::NPARAM, est::NPARAM * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return est_fail(h, UT_ERR_CUDA, cudaGetErrorString(e));
  es->adam_t = (int)hdr[3];
  return UT_OK;
}
