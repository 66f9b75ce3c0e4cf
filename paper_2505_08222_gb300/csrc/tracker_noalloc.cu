// Allocation-free tracker update: pings, communication and the particle-filter
// step for caller-owned state, with all scratch in a static device array.
//
// Some callers cannot allocate device memory: a host thread with real-time
// guarantees that forbid allocator calls (cudaMalloc may synchronise the
// device and take unbounded time), a vehicle simulator that hands us its own
// buffers and owns the memory budget of the GPU, or a plug-in whose host
// process has given every byte of device memory to another framework's pool.
// For them tracker_update_noalloc() performs the tracking part of one step —
// the same device code as env_step's ping / communication / particle-filter
// stages — on buffers the caller passes in, and keeps its own intermediates
// (the layout tables and each filter's measurement list) in the file-scope
// array below instead of in memory it would have to allocate.
//
// The array is part of the library image: every GPU that loads the library
// holds its kScratchBytes until the process exits.  All calls share it and it
// keeps the last call's contents, so calls that overlap on the GPU (different
// streams, or different host threads without ordering) race on it.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/utrack.h"
#include "env.cuh"

namespace ut {
namespace {

constexpr int kNoallocMaxEnvs = 8192;
constexpr int kNoallocMaxFilters = 32768;

// Scratch layout (bytes, each region 256-byte aligned):
//   meas      [kNoallocMaxFilters][kMaxAgents] float4   measurement lists
//   meas_n    [kNoallocMaxFilters] int32
//   meas_hdr  [kNoallocMaxFilters] float4 (target x, y, depth^2, list length)
//   filt_agent, filt_target [kNoallocMaxFilters] int32
//   agent_off, target_off, filter_off [kNoallocMaxEnvs + 1] int32
//   counters  [4] uint32
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kMeasOff = 0;
constexpr size_t kMeasNOff = kMeasOff + align256((size_t)kNoallocMaxFilters * kMaxAgents * sizeof(float4));
constexpr size_t kMeasHdrOff = kMeasNOff + align256((size_t)kNoallocMaxFilters * 4);
constexpr size_t kFiltAgentOff = kMeasHdrOff + align256((size_t)kNoallocMaxFilters * sizeof(float4));
constexpr size_t kFiltTargetOff = kFiltAgentOff + align256((size_t)kNoallocMaxFilters * 4);
constexpr size_t kAgentOffOff = kFiltTargetOff + align256((size_t)kNoallocMaxFilters * 4);
constexpr size_t kTargetOffOff = kAgentOffOff + align256((size_t)(kNoallocMaxEnvs + 1) * 4);
constexpr size_t kFilterOffOff = kTargetOffOff + align256((size_t)(kNoallocMaxEnvs + 1) * 4);
constexpr size_t kCountersOff = kFilterOffOff + align256((size_t)(kNoallocMaxEnvs + 1) * 4);
constexpr size_t kScratchBytes = kCountersOff + 256;  // about 5.1 MB

static __device__ __align__(256) unsigned char g_tracker_scratch[kScratchBytes];

// Layout tables of a uniform fleet and the random-stream position.
__global__ void noalloc_layout_kernel(EnvDev d, int A, int T, uint32_t step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int32_t* aoff = const_cast<int32_t*>(d.agent_off);
  int32_t* toff = const_cast<int32_t*>(d.target_off);
  int32_t* foff = const_cast<int32_t*>(d.filter_off);
  int32_t* fag = const_cast<int32_t*>(d.filt_agent);
  int32_t* ftg = const_cast<int32_t*>(d.filt_target);
  if (i <= d.E) {
    aoff[i] = i * A;
    toff[i] = i * T;
    foff[i] = i * A * T;
  }
  if (i < d.F) {
    const int e = i / (A * T), r = i - e * A * T;
    fag[i] = e * A + r / T;
    ftg[i] = e * T + r % T;
  }
  if (i == 0) {
    d.counters[0] = step - 1u;  // the filter kernel draws at counters[0] + 1
    d.counters[1] = 0u;
  }
}

// Pings and per-filter measurement lists for positions the caller has
// already moved: the ping and communication rules of env_step (range within
// det_radius with Gaussian noise; agent b heard by agent a within
// comm_radius unless dropped), one warp per environment.
constexpr int kNoallocWarps = 4;

__global__ void __launch_bounds__(kNoallocWarps * 32) noalloc_lists_kernel(EnvDev d, int A, int T, uint32_t g) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * kNoallocWarps + wid;
  __shared__ float s_ax[kNoallocWarps][kMaxAgents], s_ay[kNoallocWarps][kMaxAgents];
  __shared__ float s_tx[kNoallocWarps][kMaxTargets], s_ty[kNoallocWarps][kMaxTargets];
  __shared__ float s_tz[kNoallocWarps][kMaxTargets];
  __shared__ float s_rng[kNoallocWarps][kMaxAgents * kMaxTargets];
  __shared__ int s_valid[kNoallocWarps][kMaxAgents * kMaxTargets];
  __shared__ int s_recv[kNoallocWarps][kMaxAgents * kMaxAgents];
  if (e >= d.E) return;  // warp-uniform
  const int a0 = e * A, t0 = e * T, f0 = e * A * T;
  if (lane < A) {
    s_ax[wid][lane] = d.ax[a0 + lane];
    s_ay[wid][lane] = d.ay[a0 + lane];
  } else if (lane >= 8 && lane - 8 < T) {
    const int k = lane - 8;
    s_tx[wid][k] = d.tx[t0 + k];
    s_ty[wid][k] = d.ty[t0 + k];
    s_tz[wid][k] = d.tz[t0 + k];
  }
  __syncwarp();
  for (int p = lane; p < A * T; p += 32) {
    const int a = p / T, k = p - a * T;
    const float dx = s_ax[wid][a] - s_tx[wid][k], dy = s_ay[wid][a] - s_ty[wid][k], dz = 0.0f - s_tz[wid][k];
    const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
    Rand4 r = philox(d.gid_pair + (uint32_t)(f0 + p), 0u, g, TAG_PING, d.seed);
    float n0, n1;
    box_muller(r.x[0], r.x[1], n0, n1);
    const int v = dist <= d.det_radius;
    s_rng[wid][p] = v ? dist + d.range_sigma * n0 : 0.0f;
    s_valid[wid][p] = v;
  }
  for (int p = lane; p < A * A; p += 32) {
    const int a = p / A, b = p - a * A;
    int rcv = 1;
    if (a != b) {
      const float dx = s_ax[wid][a] - s_ax[wid][b], dy = s_ay[wid][a] - s_ay[wid][b];
      Rand4 r = philox(d.gid_agent + (uint32_t)(a0 + a), (uint32_t)b, g, TAG_COMM, d.seed);
      rcv = (sqrtf(dx * dx + dy * dy) <= d.comm_radius) && !(unif(r.x[0]) < d.comm_drop);
    }
    s_recv[wid][a * kMaxAgents + b] = rcv;
  }
  __syncwarp();
  for (int p = lane; p < A * T; p += 32) {
    const int a = p / T, k = p - a * T;
    int n = 0;
    for (int b = 0; b < A; ++b) {
      if (s_recv[wid][a * kMaxAgents + b] && s_valid[wid][b * T + k]) {
        d.meas[(long long)(f0 + p) * d.AM + n] = make_float4(s_ax[wid][b], s_ay[wid][b], 0.0f, s_rng[wid][b * T + k]);
        ++n;
      }
    }
    d.meas_n[f0 + p] = n;
    d.meas_hdr[f0 + p] = make_float4(s_tx[wid][k], s_ty[wid][k], s_tz[wid][k] * s_tz[wid][k], (float)n);
  }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_scratch_mutex;
unsigned char* g_scratch_ptr[64] = {nullptr};

cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_tracker_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace ut

extern "C" ut_status tracker_update_noalloc(const ut_config* cfg, uint64_t seed, uint32_t step, const float* ax_dev,
                                            const float* ay_dev, const float* tx_dev, const float* ty_dev,
                                            const float* tz_dev, float* px_dev, float* py_dev, float* pvx_dev,
                                            float* pvy_dev, float* estx_dev, float* esty_dev, float* err_dev,
                                            void* cuda_stream) {
  using namespace ut;
  if (!cfg || cfg->abi_version != UT_ABI_VERSION) return UT_ERR_INVALID;
  const int E = cfg->n_envs, A = cfg->max_agents, T = cfg->max_targets, P = cfg->n_particles;
  if (E < 1 || A < 1 || A > UT_MAX_AGENTS || T < 1 || T > UT_MAX_TARGETS || P < 1 || P > UT_MAX_PARTICLES ||
      cfg->agents_per_env_host || cfg->targets_per_env_host || !(cfg->range_sigma > 0.0f) || step < 1u ||
      cfg->shared_filter != 0 || cfg->pf_ess_num != 0) {
    std::fprintf(stderr,
                 "tracker_update_noalloc: invalid configuration (uniform fleets, per-agent filters resampled "
                 "every step, step >= 1)\n");
    return UT_ERR_INVALID;
  }
  const long long F = (long long)E * A * T;
  if (E > kNoallocMaxEnvs || F > kNoallocMaxFilters) {
    std::fprintf(stderr,
                 "tracker_update_noalloc: %d envs / %lld filters exceed the static scratch limit of %d envs / "
                 "%d filters\n",
                 E, F, kNoallocMaxEnvs, kNoallocMaxFilters);
    return UT_ERR_INVALID;
  }
  if (!ax_dev || !ay_dev || !tx_dev || !ty_dev || !tz_dev || !px_dev || !py_dev || !pvx_dev || !pvy_dev ||
      !estx_dev || !esty_dev || !err_dev)
    return UT_ERR_INVALID;
  // the filter kernel reads and writes the particles as float4 when P % 4 == 0
  if (P % 4 == 0) {
    const float* parts[4] = {px_dev, py_dev, pvx_dev, pvy_dev};
    for (const float* q : parts) {
      if (reinterpret_cast<uintptr_t>(q) % 16 != 0) {
        std::fprintf(stderr,
                     "tracker_update_noalloc: particle arrays must be 16-byte aligned when n_particles %% 4 == 0\n");
        return UT_ERR_INVALID;
      }
    }
  }
  // an error left by earlier, unrelated work is not this call's
  const cudaError_t stale = cudaGetLastError();
  if (stale != cudaSuccess)
    std::fprintf(stderr, "tracker_update_noalloc: cleared an earlier CUDA error: %s\n", cudaGetErrorString(stale));
  unsigned char* s = nullptr;
  if (scratch_address(&s) != cudaSuccess) return UT_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  EnvDev d;
  memset(&d, 0, sizeof(d));
  d.E = E;
  d.AM = A;
  d.TM = T;
  d.NS = A + T;
  d.P = P;
  d.NA = E * A;
  d.NT = E * T;
  d.F = (int)F;
  d.seed = seed;
  // global ids of a shard's first env / agent / target / filter, as env_step
  // takes them: per-agent filters are their (agent, target) pairs
  d.gid_env = cfg->id_env0;
  d.gid_agent = cfg->id_agent0;
  d.gid_target = cfg->id_target0;
  d.gid_filter = cfg->id_filter0;
  d.gid_pair = cfg->id_filter0;
  d.dt = cfg->dt;
  d.range_sigma = cfg->range_sigma;
  d.inv_two_s2 = (float)(1.0 / (2.0 * (double)cfg->range_sigma * (double)cfg->range_sigma));
  d.det_radius = cfg->det_radius;
  d.comm_radius = cfg->comm_radius;
  d.comm_drop = cfg->comm_drop;
  d.pf_accel_sigma = cfg->pf_accel_sigma;
  d.pf_vcap = cfg->pf_vcap;
  d.ax = const_cast<float*>(ax_dev);
  d.ay = const_cast<float*>(ay_dev);
  d.tx = const_cast<float*>(tx_dev);
  d.ty = const_cast<float*>(ty_dev);
  d.tz = const_cast<float*>(tz_dev);
  d.px = px_dev;
  d.py = py_dev;
  d.pvx = pvx_dev;
  d.pvy = pvy_dev;
  d.estx = estx_dev;
  d.esty = esty_dev;
  d.err = err_dev;
  d.meas = reinterpret_cast<float4*>(s + kMeasOff);
  d.meas_n = reinterpret_cast<int32_t*>(s + kMeasNOff);
  d.meas_hdr = reinterpret_cast<float4*>(s + kMeasHdrOff);
  d.filt_agent = reinterpret_cast<int32_t*>(s + kFiltAgentOff);
  d.filt_target = reinterpret_cast<int32_t*>(s + kFiltTargetOff);
  d.agent_off = reinterpret_cast<int32_t*>(s + kAgentOffOff);
  d.target_off = reinterpret_cast<int32_t*>(s + kTargetOffOff);
  d.filter_off = reinterpret_cast<int32_t*>(s + kFilterOffOff);
  d.counters = reinterpret_cast<uint32_t*>(s + kCountersOff);

  const int n_layout = (int)(F > E + 1 ? F : E + 1);
  noalloc_layout_kernel<<<(n_layout + 255) / 256, 256, 0, st>>>(d, A, T, step);
  noalloc_lists_kernel<<<(E + kNoallocWarps - 1) / kNoallocWarps, kNoallocWarps * 32, 0, st>>>(d, A, T, step);
  if (cudaGetLastError() != cudaSuccess) return UT_ERR_CUDA;
  if (launch_pf_step(d, pf_default_variant(P), st) != cudaSuccess) return UT_ERR_CUDA;
  return UT_OK;
}
