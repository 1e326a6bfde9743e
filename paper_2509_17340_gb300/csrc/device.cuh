// Device-side building blocks of the planning step: Philox noise, quadrotor
// RK4, cost terms, nearest-point query on the collision grid, warp reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace aero {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 multiplies;
// the key is bumped by the Weyl constants before every round but the first.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// (2 (w >> 9) + 1) 2^-24: exact in binary32, in (0, 1).
__device__ __forceinline__ float uniform01(uint32_t w) {
  return static_cast<float>(2u * (w >> 9) + 1u) * 5.9604644775390625e-8f;
}

// Four standard normals from one Philox block (Box-Muller on (u0,u1), (u2,u3)).
__device__ __forceinline__ float4 normals4(uint4 w) {
  const float ra = sqrtf(-2.0f * logf(uniform01(w.x)));
  const float rb = sqrtf(-2.0f * logf(uniform01(w.z)));
  float sa, ca, sb, cb;
  sincospif(2.0f * uniform01(w.y), &sa, &ca);
  sincospif(2.0f * uniform01(w.w), &sb, &cb);
  return make_float4(ra * ca, ra * sa, rb * cb, rb * sb);
}

// Perturbation delta for sample k, step j, instance e (Sec. III-B).
__device__ __forceinline__ float4 noise_delta(uint32_t k, uint32_t j, uint32_t e, uint32_t c3,
                                              uint32_t k0, uint32_t k1, const float* sigma) {
  const float4 n = normals4(philox4x32_10(make_uint4(k, j, e, c3), k0, k1));
  return make_float4(sigma[0] * n.x, sigma[1] * n.y, sigma[2] * n.z, sigma[3] * n.w);
}

// ---------------------------------------------------------------------------
// Quadrotor model (Eq. dynamics) and one RK4 step with renormalisation.
// ---------------------------------------------------------------------------
struct State {
  float p[3], q[4], v[3];
};

__device__ __forceinline__ void dynamics(const State& x, float F, float wx, float wy, float wz,
                                         const DynParams& dp, State& d) {
  d.p[0] = x.v[0];
  d.p[1] = x.v[1];
  d.p[2] = x.v[2];
  // q' = 1/2 q (x) [0, w]
  d.q[0] = 0.5f * (-x.q[1] * wx - x.q[2] * wy - x.q[3] * wz);
  d.q[1] = 0.5f * (x.q[0] * wx + x.q[2] * wz - x.q[3] * wy);
  d.q[2] = 0.5f * (x.q[0] * wy - x.q[1] * wz + x.q[3] * wx);
  d.q[3] = 0.5f * (x.q[0] * wz + x.q[1] * wy - x.q[2] * wx);
  // v' = (F/m) R(q) e3 + g
  const float a = F * dp.inv_mass;
  d.v[0] = a * (2.0f * (x.q[1] * x.q[3] + x.q[0] * x.q[2]));
  d.v[1] = a * (2.0f * (x.q[2] * x.q[3] - x.q[0] * x.q[1]));
  d.v[2] = a * (1.0f - 2.0f * (x.q[1] * x.q[1] + x.q[2] * x.q[2])) - dp.g;
}

__device__ __forceinline__ void axpy_state(const State& x, float h, const State& k, State& o) {
#pragma unroll
  for (int i = 0; i < 3; ++i) o.p[i] = x.p[i] + h * k.p[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) o.q[i] = x.q[i] + h * k.q[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) o.v[i] = x.v[i] + h * k.v[i];
}

__device__ __forceinline__ void rk4_step(State& x, float4 u, const DynParams& dp) {
  State k1, k2, k3, k4, t;
  const float h = dp.dt, hh = 0.5f * dp.dt, h6 = dp.dt * (1.0f / 6.0f);
  dynamics(x, u.x, u.y, u.z, u.w, dp, k1);
  axpy_state(x, hh, k1, t);
  dynamics(t, u.x, u.y, u.z, u.w, dp, k2);
  axpy_state(x, hh, k2, t);
  dynamics(t, u.x, u.y, u.z, u.w, dp, k3);
  axpy_state(x, h, k3, t);
  dynamics(t, u.x, u.y, u.z, u.w, dp, k4);
#pragma unroll
  for (int i = 0; i < 3; ++i) x.p[i] += h6 * (k1.p[i] + 2.0f * (k2.p[i] + k3.p[i]) + k4.p[i]);
#pragma unroll
  for (int i = 0; i < 4; ++i) x.q[i] += h6 * (k1.q[i] + 2.0f * (k2.q[i] + k3.q[i]) + k4.q[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) x.v[i] += h6 * (k1.v[i] + 2.0f * (k2.v[i] + k3.v[i]) + k4.v[i]);
  const float inv = rsqrtf(x.q[0] * x.q[0] + x.q[1] * x.q[1] + x.q[2] * x.q[2] + x.q[3] * x.q[3]);
#pragma unroll
  for (int i = 0; i < 4; ++i) x.q[i] *= inv;
}

// ---------------------------------------------------------------------------
// Collision grid query: squared distance to the nearest collision point if it
// is below d_max^2, else d_max^2.  Cells have edge h >= d_max (1 + 1/16), so
// every point within d_max lies in the 3x3x3 block around the query's cell.
// Rows of the block whose slab is farther than d_max are skipped; along x the
// neighbours are taken only when they can be within d_max.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float nn_dist2(float px, float py, float pz, const GridView& g,
                                          float dmax, float dmax2) {
  const float fx = (px - g.origin) * g.inv_h;
  const float fy = (py - g.origin) * g.inv_h;
  const float fz = (pz - g.origin) * g.inv_h;
  float best = dmax2;
  if (!(fx > -1.0f && fy > -1.0f && fz > -1.0f && fx < g.G + 1.0f && fy < g.G + 1.0f &&
        fz < g.G + 1.0f))
    return best;  // farther than one cell from every point (or not finite)
  const int cx = __float2int_rd(fx), cy = __float2int_rd(fy), cz = __float2int_rd(fz);
  const float h = 1.0f / g.inv_h;
  // distances from the query to the lower / upper faces of its cell
  const float lx = (fx - cx) * h, ux = h - lx;
  const float ly = (fy - cy) * h, uy = h - ly;
  const float lz = (fz - cz) * h, uz = h - lz;
  const int x0 = max(lx < dmax ? cx - 1 : cx, 0);
  const int x1 = min(ux < dmax ? cx + 1 : cx, g.G - 1);
  if (x0 > x1) return best;
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = cz + dz;
    if (z < 0 || z >= g.G) continue;
    const float ez = dz < 0 ? lz : (dz > 0 ? uz : 0.0f);
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = cy + dy;
      if (y < 0 || y >= g.G) continue;
      const float ey = dy < 0 ? ly : (dy > 0 ? uy : 0.0f);
      if (ey * ey + ez * ez >= dmax2) continue;
      const int row = (z * g.G + y) * g.G;
      const int s = __ldg(g.start + row + x0), e = __ldg(g.start + row + x1 + 1);
      for (int i = s; i < e; ++i) {
        const float4 q = __ldg(g.pts + i);
        const float ax = px - q.x, ay = py - q.y, az = pz - q.z;
        best = fminf(best, ax * ax + ay * ay + az * az);
      }
    }
  }
  return best;
}

// Piecewise collision penalty from a squared distance (d >= d_max -> 0).
__device__ __forceinline__ float jcol_from_d2(float d2, const CostParams& c, float dmax2) {
  if (!(d2 < dmax2)) return 0.0f;
  const float d = sqrtf(d2);
  return d < c.d_min ? c.C_col : c.C_col * expf(-c.a_col * (d - c.d_min));
}

// ||R(q) R(q_g)^T - I||_F = 2 sqrt(2) |vec(q (x) conj(q_g))| for unit quaternions.
__device__ __forceinline__ float attitude_err(const float* q, const float* g) {
  const float r1 = -q[0] * g[1] + q[1] * g[0] - q[2] * g[3] + q[3] * g[2];
  const float r2 = -q[0] * g[2] + q[1] * g[3] + q[2] * g[0] - q[3] * g[1];
  const float r3 = -q[0] * g[3] - q[1] * g[2] + q[2] * g[1] + q[3] * g[0];
  return 2.8284271247461903f * sqrtf(r1 * r1 + r2 * r2 + r3 * r3);
}

__device__ __forceinline__ float norm3f(float a, float b, float c) {
  return sqrtf(a * a + b * b + c * c);
}

// Goal term of one step: Q_p |p - p_goal| + Q_v |v - v_goal| + Q_q ||R R_g^T - I||_F.
__device__ __forceinline__ float goal_term(const State& x, const CostParams& c) {
  return c.Q_p * norm3f(x.p[0] - c.goal_rel[0], x.p[1] - c.goal_rel[1], x.p[2] - c.goal_rel[2]) +
         c.Q_v * norm3f(x.v[0] - c.v_goal[0], x.v[1] - c.v_goal[1], x.v[2] - c.v_goal[2]) +
         c.Q_q * attitude_err(x.q, c.q_goal);
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum four values over the warp with six shuffles: after the call, lane
// 8*c holds the warp total of component c (lanes 0, 8, 16, 24).
__device__ __forceinline__ float warp_sum4(float a0, float a1, float a2, float a3, int lane) {
  const bool hi16 = lane & 16;
  const float s0 = hi16 ? a0 : a2, s1 = hi16 ? a1 : a3;
  const float r0 = __shfl_xor_sync(0xffffffffu, s0, 16);
  const float r1 = __shfl_xor_sync(0xffffffffu, s1, 16);
  const float b0 = (hi16 ? a2 : a0) + r0;
  const float b1 = (hi16 ? a3 : a1) + r1;
  const bool hi8 = lane & 8;
  const float s = hi8 ? b0 : b1;
  const float r = __shfl_xor_sync(0xffffffffu, s, 8);
  float c = (hi8 ? b1 : b0) + r;
  c += __shfl_xor_sync(0xffffffffu, c, 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

}  // namespace aero
