// Host-side handle of one environment batch (the opaque ut_env of the C ABI)
// and the hooks through which the policy and the learned estimator plug into
// the step.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/utrack.h"
#include "env.cuh"

struct PolicyState;
struct EstimatorState;

struct ut_env {
  ut_config cfg{};
  bool has_alloc = false;
  ut_allocator alloc{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::vector<void*> allocations;
  ut::EnvDev d{};
  std::string err;
  int64_t NA = 0, NT = 0, F = 0;
  std::vector<int32_t> agents_per_env, targets_per_env;
  int pf_variant = 0;
  bool reset_done = false;
  // graph-captured rollout
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_key = -1, graph_variant = -1;
  // graph-captured PPO collection (env_ppo_collect), keyed by its arguments
  cudaGraphExec_t ppo_exec = nullptr;
  std::vector<uintptr_t> ppo_key;
  // host count of kernels enqueued since the metrics were cleared
  int64_t launches = 0;
  int launches_per_graph = 0;
  // stage timing events
  bool prof_on = false;
  std::vector<cudaEvent_t> eager_ev;   // pairs for eager steps
  size_t eager_used = 0;               // pairs recorded since the last read
  bool capturing = false;              // inside rollout graph capture
  // transformer agent and learned estimator
  bool policy_ready = false;
  PolicyState* policy = nullptr;
  int est_mode = 0;
  EstimatorState* est = nullptr;
  // test hook (env_test_wait_timeout): poll bound of a wait that runs out
  uint32_t test_wait_polls = 0;
  // rollout(): 0 the captured CUDA graph of T steps, 1 the persistent kernel
  // (when the handle qualifies: random actions, the filter tracker)
  int rollout_form = 0;
};

namespace ut {

void* env_alloc(ut_env* h, size_t bytes);
void env_free_all(ut_env* h);
cudaError_t enqueue_step(ut_env* h, const int32_t* act, cudaStream_t s);
cudaError_t capture_stream_ensure(ut_env* h);
int count_step_kernels(ut_env* h);

// Hooks implemented by the policy / estimator modules.
ut_status extension_create(ut_env* h);
void extension_destroy(ut_env* h);
cudaError_t extension_reset(ut_env* h, cudaStream_t s);
// Writes actions for this step into h->d.actions.
cudaError_t extension_policy_actions(ut_env* h, cudaStream_t s);
// Learned estimate in place of the filter; cudaErrorNotReady = run the filter.
cudaError_t extension_estimate(ut_env* h, cudaStream_t s);
const float* extension_logits(ut_env* h);
int extension_policy_kernels(ut_env* h);
uint16_t* extension_h(ut_env* h);

}  // namespace ut
