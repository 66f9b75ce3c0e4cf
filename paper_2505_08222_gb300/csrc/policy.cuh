// Transformer agent: device view and host helpers (policy.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace ut {

struct PolicyDev {
  long long NA;               // agents
  int NS;                     // entity slots per agent
  int R;                      // rows per agent in a tile (1 + NS)
  int apt;                    // agents per 128-row tile
  int n_act, L;
  const uint16_t* tokens;     // [NA][NS][8] bf16
  const int32_t* n_ent;       // [NA] entity tokens in use
  uint16_t* h;                // [NA][d] bf16, read then overwritten
  float* logits;              // [NA][n_act]
  int32_t* actions;           // [NA] (written when sample != 0)
  const float* emb_w;         // [d][8]
  const float* emb_b;         // [d]
  const unsigned char* wimg;  // packed BF16 operand images, layer-major
  const float* vec;           // per layer: ln1 g/b, bq, bk, bv, bo, ln2 g/b, b1 (4d), b2
  const float* lnf_g;
  const float* lnf_b;
  const float* head_w;        // [n_act][d]
  const float* head_b;        // [n_act]
  uint64_t seed;
  uint32_t gid_agent;         // global id of agent 0 (sharded batches)
  const uint32_t* counters;   // step counter (g = counters[0] + 1), or NULL: use `step`
  uint32_t step;
  int sample;                 // draw Gumbel-max actions
  int* status;
  // test hook (env_test_wait_timeout): > 0 makes the kernel first wait on a
  // barrier that nothing signals, for this many polls, and take the
  // timed-out path (status 2) before it issues any copy or MMA
  uint32_t test_wait_polls;
};

int64_t policy_param_count(int d, int L, int n_act);
bool policy_supported(int d, int n_heads);
size_t policy_layer_bytes(int d);
void policy_pack(int d, int L, int n_act, const float* prm, std::vector<unsigned char>& img, std::vector<float>& vec,
                 std::vector<float>& emb, std::vector<float>& head);
cudaError_t launch_policy(const PolicyDev& p, int d, cudaStream_t s);

}  // namespace ut
