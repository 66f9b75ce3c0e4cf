// Persistent rollout: T environment steps in one launch, one CTA per
// environment.
//
// Environments are independent (the step vectorises over them, Sec.
// III-A.3), so a CTA can advance its own environment through all T steps
// with block barriers only, no grid-wide synchronisation: each step is the
// warp-level env stage (actions, kinematics, targets, pings, communication,
// measurement lists; warp 0), the particle-filter step of each of the
// environment's filters (the whole CTA, the same device code as
// pf_step_kernel), then observation tokens and reward (warp 0).  An
// environment with a single filter keeps that filter's particles in
// registers for the whole rollout: they are read from HBM once before the
// first step and written once after the last.  The counters and the
// episode-end flag follow the step-by-step rollout exactly (global step
// g = counters[0] + 1 + t), so the results equal the graph rollout's bit for
// bit when both use the same filter launch shape (NT, PPT); the device
// metrics are the same sums added in another order.
//
// Actions are the environment's uniform random actions: the transformer
// agent and the learned estimator run as their own kernels and keep the
// graph rollout.
#pragma once

#include "env_step.cuh"
#include "pf_kernel.cuh"

namespace ut {
namespace persist {

template <int NT, int PPT, int MODE>
__global__ void __launch_bounds__(NT, 1) rollout_kernel(EnvDev d, int T) {
  __shared__ EnvWarpSmem ew;
  const int e = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t g0 = d.counters[0], t0 = d.counters[1];
  const int f0 = d.filter_off[e], nf = d.filter_off[e + 1] - f0;
  const bool resident = nf == 1;  // (CTA-uniform)
  float x[PPT], y[PPT], vx[PPT], vy[PPT];
  if (resident) pf::load_particles<NT, PPT, MODE>(d, f0, x, y, vx, vy);
  StepMetrics acc;
  for (int t = 0; t < T; ++t) {
    const uint32_t g = g0 + 1u + (uint32_t)t;
    if (warp == 0) step_env_warp(d, e, nullptr, g, ew);
    __syncthreads();  // measurement lists and headers of this step
    if (resident) {
      pf::pf_step_body<NT, PPT, MODE, false, true>(d, f0, g, x, y, vx, vy);
      __syncthreads();  // estimates visible; the filter's shared memory free again
    } else {
      for (int k = 0; k < nf; ++k) {
        pf::pf_step_body<NT, PPT, MODE, false, false>(d, f0 + k, g, x, y, vx, vy);
        __syncthreads();
      }
    }
    if (warp == 0) {
      StepMetrics m;
      obs_reward_warp(d, e, 0, t0 + (uint32_t)t + 1u, m);
      acc.sq += m.sq;
      acc.rw += m.rw;
      acc.n_err += m.n_err;
      acc.n_crash += m.n_crash;
      acc.n_agents += m.n_agents;
    }
    // (warp 0 alone touches the environment state between the barriers: the
    // next step's env stage follows its own observation stage)
  }
  if (resident) pf::store_particles<NT, PPT, MODE>(d, f0, x, y, vx, vy);
  if (warp == 0 && lane == 0) {
    atomicAdd(&d.metrics_d[0], acc.sq);
    atomicAdd(&d.metrics_d[1], acc.rw);
    atomicAdd(&d.metrics_u[0], acc.n_err);
    atomicAdd(&d.metrics_u[1], acc.n_crash);
    atomicAdd(&d.metrics_u[2], acc.n_agents);
  }
}

template <int NT, int PPT>
cudaError_t launch_shape(const EnvDev& d, int T, cudaStream_t s) {
  const size_t smem = pf::step_smem_bytes(NT, PPT);
  if (d.P > NT * PPT) return cudaErrorInvalidValue;
  cudaError_t e;
  if (d.P == NT * PPT) {
    static std::atomic<unsigned long long> ready{0};
    auto k = rollout_kernel<NT, PPT, 2>;
    if ((e = smem_optin(k, smem, ready)) != cudaSuccess) return e;
    k<<<d.E, NT, smem, s>>>(d, T);
  } else if (d.P % 4 == 0) {
    static std::atomic<unsigned long long> ready{0};
    auto k = rollout_kernel<NT, PPT, 1>;
    if ((e = smem_optin(k, smem, ready)) != cudaSuccess) return e;
    k<<<d.E, NT, smem, s>>>(d, T);
  } else {
    static std::atomic<unsigned long long> ready{0};
    auto k = rollout_kernel<NT, PPT, 0>;
    if ((e = smem_optin(k, smem, ready)) != cudaSuccess) return e;
    k<<<d.E, NT, smem, s>>>(d, T);
  }
  return cudaGetLastError();
}

}  // namespace persist
}  // namespace ut
