// Least-squares trilateration tracker (Sec. II-A; Sec. III-A.2: each agent
// keeps an LS or a PF tracking model per target), reading C21.
//
// Per filter, the pings it holds in its 16-entry ring (sender q, range r),
// with the target depth known (the plane is tracked): horizontal ranges
// rho = sqrt(max(r^2 - dz^2, 0)).  The target is taken as static over the
// window; each ping gives |x - q|^2 = rho^2, i.e. 2 q.x = |x|^2 + a with
// a = |q|^2 - rho^2, and subtracting the mean over the pings removes |x|^2:
//   2 (q_m - qbar) . x = a_m - abar      (linear least squares),
// solved by the 2 x 2 normal equations A x = b, A = sum (q - qbar)(q - qbar)^T,
// b = 1/2 sum (q - qbar)(a - abar).  Positions are taken relative to the
// previous estimate e1 (the solution does not depend on the origin; the
// smaller numbers keep FP32 accurate).  With fewer than 3 pings or a
// near-degenerate geometry (det A <= 1e-3 (tr A)^2, collinear senders) the
// estimate is held.  The estimate history and smoothed motion advance as for
// every tracker.
#include "env.cuh"

namespace ut {
namespace {

constexpr float kLsMinDetRatio = 1e-3f;

__global__ void ls_update_kernel(EnvDev d) {
  pdl_wait();  // (dependents launch as this grid's CTAs exit)
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= d.F) return;
  const int it = d.filt_target[f];
  if (!UT_IN_BOUNDS(it >= 0 && it < d.NT, d.status)) return;
  const float dz = d.tz[it];
  const float e1x = d.estx[f], e1y = d.esty[f];
  const float e2x = d.prev_estx[f], e2y = d.prev_esty[f];
  const int n = d.ring_count[f], head = d.ring_head[f];
  const float4* ring = reinterpret_cast<const float4*>(d.ring) + (long long)f * kRing;
  float qx[kRing], qy[kRing], a[kRing];
  float sx = 0.0f, sy = 0.0f, sa = 0.0f;
#pragma unroll
  for (int s = 0; s < kRing; ++s) {
    qx[s] = qy[s] = a[s] = 0.0f;
    if (s < n) {
      const float4 e = ring[(head - 1 - s) & (kRing - 1)];  // the s-th newest ping
      const float x = e.x - e1x, y = e.y - e1y;
      const float rho2 = fmaxf(fmaf(e.z, e.z, -dz * dz), 0.0f);
      qx[s] = x;
      qy[s] = y;
      a[s] = fmaf(x, x, fmaf(y, y, -rho2));
      sx += x;
      sy += y;
      sa += a[s];
    }
  }
  float ex = e1x, ey = e1y;
  if (n >= 3) {
    const float inv_n = 1.0f / (float)n;
    const float mx = sx * inv_n, my = sy * inv_n, ma = sa * inv_n;
    float a00 = 0.0f, a01 = 0.0f, a11 = 0.0f, b0 = 0.0f, b1 = 0.0f;
#pragma unroll
    for (int s = 0; s < kRing; ++s) {
      if (s < n) {
        const float dx = qx[s] - mx, dy = qy[s] - my, da = a[s] - ma;
        a00 = fmaf(dx, dx, a00);
        a01 = fmaf(dx, dy, a01);
        a11 = fmaf(dy, dy, a11);
        b0 = fmaf(dx, da, b0);
        b1 = fmaf(dy, da, b1);
      }
    }
    b0 *= 0.5f;
    b1 *= 0.5f;
    const float det = a00 * a11 - a01 * a01, tr = a00 + a11;
    if (det > kLsMinDetRatio * tr * tr) {
      ex = e1x + (a11 * b0 - a01 * b1) / det;
      ey = e1y + (a00 * b1 - a01 * b0) / det;
    }
  }
  d.prev2_estx[f] = e2x;
  d.prev2_esty[f] = e2y;
  d.prev_estx[f] = e1x;
  d.prev_esty[f] = e1y;
  d.velx[f] = fmaf(kVelKeep, d.velx[f], (1.0f - kVelKeep) * (e1x - e2x));
  d.vely[f] = fmaf(kVelKeep, d.vely[f], (1.0f - kVelKeep) * (e1y - e2y));
  d.estx[f] = ex;
  d.esty[f] = ey;
  const float dx = ex - d.tx[it], dy = ey - d.ty[it];
  d.err[f] = sqrtf(dx * dx + dy * dy);
}

}  // namespace

cudaError_t launch_ls_update(const EnvDev& d, cudaStream_t s) {
  if (d.F <= 0) return cudaSuccess;
  return launch_pdl(ls_update_kernel, dim3((d.F + 127) / 128), dim3(128), 0, s, d);
}

}  // namespace ut
