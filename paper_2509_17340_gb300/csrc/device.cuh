// Device-side building blocks of the planning step: Philox noise, quadrotor
// RK4, cost terms, nearest-point query on the collision grid, warp reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace aero {

// ---------------------------------------------------------------------------
// Programmatic dependent launch (sm_90 and later).  pdl_start lets the next
// kernel of the stream be scheduled now, then waits until this kernel's
// predecessor has completed and its writes are visible.  Both instructions are
// no-ops for a kernel launched without programmatic stream serialization.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_start() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// The first half of pdl_start alone: let the next kernel be scheduled, without
// waiting for the predecessor.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The second half alone: wait until the predecessor has completed and its
// writes are visible (immediate once waited for).
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

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
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;  // one 32x32->64 multiply each
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1,
                   (uint32_t)p0);
  }
  return c;
}

// The same rounds with the key schedule given: rk[2r], rk[2r + 1] are the
// key words of round r (the key plus r times the Weyl constants).  Kernels
// whose arguments live in the parameter space read them as constant operands.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1], (uint32_t)p0);
  }
  return c;
}

// (2 (w >> 9) + 1) 2^-24: exact in binary32, in (0, 1).  Built from the bits:
// 1 + (w >> 9) 2^-23 has those mantissa bits, and subtracting 1 - 2^-24 is
// exact (Sterbenz), leaving (w >> 9) 2^-23 + 2^-24 with no integer conversion.
__device__ __forceinline__ float uniform01(uint32_t w) {
  return __uint_as_float(0x3F800000u | (w >> 9)) - 0.99999994039535522f;
}

// sqrt(x) for x >= 0 by the hardware's approximate square root, subnormal
// inputs flushed to zero (sqrt.approx.ftz.f32: 0 at 0; a subnormal squared
// norm is a length below 1e-19, taken as 0).  Its error is far below the
// tolerances, which the GPU tests check on the normals and on the costs.
__device__ __forceinline__ float fast_sqrt(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/sqrt(x) by the hardware's approximation with subnormals flushed
// (rsqrt.approx.ftz.f32), for the renormalisation of a quaternion whose
// squared norm is close to 1.
__device__ __forceinline__ float fast_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Four standard normals from one Philox block (Box-Muller on (u0,u1), (u2,u3)).
// ln u for u in (0, 1): CUDA's hardware base-2 logarithm (absolute error
// about 2^-22 on [0.5, 2]) times ln 2; near 1, where that absolute error would
// dominate the small Box-Muller radius, the series -(v + v^2/2 + v^3/3 + v^4/4)
// of ln(1 - v) with v = 1 - u exact (remainder below v^5/5 < 2e-13).
__device__ __forceinline__ float log_unit(float u) {
  const float v = 1.0f - u;
  if (v < 4e-3f) return -v * fmaf(v, fmaf(v, fmaf(v, 0.25f, 1.0f / 3.0f), 0.5f), 1.0f);
  return __log2f(u) * 0.693147180559945309f;
}

// Box-Muller on two uniforms: r (cos 2 pi u2, sin 2 pi u2), r = sqrt(-2 ln u1).
// The angle is taken as 2 pi (u2 - 1/2) in [-pi, pi], where CUDA's hardware
// sine and cosine have an absolute error of about 2^-21.4; with |r| <= 5.8 and
// the radius error of log_unit the normals are within 5e-6 of their
// correctly rounded values.
__device__ __forceinline__ float2 box_muller(uint32_t w1, uint32_t w2) {
  const float r = fast_sqrt(-2.0f * log_unit(uniform01(w1)));
  float s, c;
  __sincosf((uniform01(w2) - 0.5f) * 6.28318530717958648f, &s, &c);
  return make_float2(-r * c, -r * s);  // cos(t + pi) = -cos t, sin(t + pi) = -sin t
}

__device__ __forceinline__ float4 normals4(uint4 w) {
  const float2 a = box_muller(w.x, w.y), b = box_muller(w.z, w.w);
  return make_float4(a.x, a.y, b.x, b.y);
}

// Perturbation delta for sample k, step j, instance e (Sec. III-B).
__device__ __forceinline__ float4 noise_delta(uint32_t k, uint32_t j, uint32_t e, uint32_t c3,
                                              uint32_t k0, uint32_t k1, float4 sigma) {
  const float4 n = normals4(philox4x32_10(make_uint4(k, j, e, c3), k0, k1));
  return make_float4(sigma.x * n.x, sigma.y * n.y, sigma.z * n.z, sigma.w * n.w);
}

// The same from the round keys (see philox4x32_10_rk).
__device__ __forceinline__ float4 noise_delta_rk(uint32_t k, uint32_t j, uint32_t e, uint32_t c3,
                                                 const uint32_t* rk, float4 sigma) {
  const float4 n = normals4(philox4x32_10_rk(make_uint4(k, j, e, c3), rk));
  return make_float4(sigma.x * n.x, sigma.y * n.y, sigma.z * n.z, sigma.w * n.w);
}

// ---------------------------------------------------------------------------
// Quadrotor model (Eq. dynamics) integrated by one classical RK4 step with the
// control held over the step (Eq. mppi_rollout_simplified), then the
// quaternion renormalised.
//
// The RK4 stages are evaluated in closed form.  With the body rate w held,
// q' = A q with A q = 1/2 q (x) [0, w] and A^2 = -s I, s = |w|^2 / 4, so every
// stage quaternion is a combination of q and A q:
//   q1 = q,  q2 = q + h/2 Aq,  q3 = (1 - h^2 s/4) q + h/2 Aq,
//   q4 = (1 - h^2 s/2) q + h (1 - h^2 s/4) Aq,
//   q+ = (1 - h^2 s/2 + h^4 s^2/24) q + (h - h^3 s/6) Aq.
// v' = a(q) = (F/m) R(q) e3 - g e3 does not depend on p or v, so with
// a_i = a(q_i):  p+ = p + h v + h^2/6 (a1 + a2 + a3),
//                v+ = v + h/6 (a1 + 2 a2 + 2 a3 + a4).
// These are the RK4 stage sums of the textbook scheme, regrouped.
// ---------------------------------------------------------------------------
struct State {
  float p[3], q[4], v[3];
};

// Third column of R(q) (unit-quaternion formula), i.e. R(q) e3.
__device__ __forceinline__ void r_e3(float w, float x, float y, float z, float& rx, float& ry,
                                     float& rz) {
  rx = 2.0f * (x * z + w * y);
  ry = 2.0f * (y * z - w * x);
  rz = 1.0f - 2.0f * (x * x + y * y);
}

// Half of R(q) e3: (xz + wy, yz - wx, 1/2 - x^2 - y^2); rk4_step folds the
// factor 2 into its thrust coefficients.
__device__ __forceinline__ void r_e3_half(float w, float x, float y, float z, float& rx, float& ry,
                                          float& rz) {
  rx = x * z + w * y;
  ry = y * z - w * x;
  rz = 0.5f - x * x - y * y;
}

__device__ __forceinline__ void rk4_step(State& x, float4 u, const DynParams& dp) {
  const float h = dp.dt;
  // half rates: A q = 1/2 q (x) [0, w] = q (x) [0, w/2]
  const float hx = 0.5f * u.y, hy = 0.5f * u.z, hz = 0.5f * u.w;
  const float* q = x.q;
  const float a0 = -q[1] * hx - q[2] * hy - q[3] * hz;
  const float a1 = q[0] * hx + q[2] * hz - q[3] * hy;
  const float a2 = q[0] * hy - q[1] * hz + q[3] * hx;
  const float a3 = q[0] * hz + q[1] * hy - q[2] * hx;
  const float s = hx * hx + hy * hy + hz * hz;  // |w|^2 / 4
  const float hh = h * h * s;
  const float c3 = 1.0f - 0.25f * hh, c4 = 1.0f - 0.5f * hh;
  const float hb = 0.5f * h, h4 = h * c3;
  const float b0 = hb * a0, b1 = hb * a1, b2 = hb * a2, b3 = hb * a3;
  float r1x, r1y, r1z, r2x, r2y, r2z, r3x, r3y, r3z, r4x, r4y, r4z;
  r_e3_half(q[0], q[1], q[2], q[3], r1x, r1y, r1z);
  r_e3_half(q[0] + b0, q[1] + b1, q[2] + b2, q[3] + b3, r2x, r2y, r2z);
  r_e3_half(c3 * q[0] + b0, c3 * q[1] + b1, c3 * q[2] + b2, c3 * q[3] + b3, r3x, r3y, r3z);
  r_e3_half(c4 * q[0] + h4 * a0, c4 * q[1] + h4 * a1, c4 * q[2] + h4 * a2, c4 * q[3] + h4 * a3, r4x,
            r4y, r4z);
  const float f = u.x * dp.inv_mass;
  // h^2/6 f and h/6 f times R e3 = 2 (the half above)
  const float fp = h * h * (1.0f / 3.0f) * f, fv = h * (1.0f / 3.0f) * f;
  const float gp = 0.5f * h * h * dp.g, gv = h * dp.g;
  x.p[0] += h * x.v[0] + fp * (r1x + r2x + r3x);
  x.p[1] += h * x.v[1] + fp * (r1y + r2y + r3y);
  x.p[2] += h * x.v[2] + fp * (r1z + r2z + r3z) - gp;
  x.v[0] += fv * (r1x + 2.0f * (r2x + r3x) + r4x);
  x.v[1] += fv * (r1y + 2.0f * (r2y + r3y) + r4y);
  x.v[2] += fv * (r1z + 2.0f * (r2z + r3z) + r4z) - gv;
  const float cq = 1.0f - 0.5f * hh + hh * hh * (1.0f / 24.0f);
  const float ca = h * (1.0f - hh * (1.0f / 6.0f));
  const float n0 = cq * q[0] + ca * a0, n1 = cq * q[1] + ca * a1;
  const float n2 = cq * q[2] + ca * a2, n3 = cq * q[3] + ca * a3;
  const float inv = fast_rsqrt(n0 * n0 + n1 * n1 + n2 * n2 + n3 * n3);
  x.q[0] = n0 * inv;
  x.q[1] = n1 * inv;
  x.q[2] = n2 * inv;
  x.q[3] = n3 * inv;
}

// The same step split by dependence (Stage II's noise-free rollouts): the
// attitude update does not depend on p or v, so a trajectory's quaternions can
// be chained alone.  With b = ca / 2, the unnormalised q+ = cq q + ca A q is
// the map M q, M = [[cq, -b wx, -b wy, -b wz], [b wx, cq, b wz, -b wy],
// [b wy, -b wz, cq, b wx], [b wz, b wy, -b wx, cq]]; rk4_attitude_coefs gives
// (cq, b wx, b wy, b wz) of a step and attitude_map applies M and renormalises.
__device__ __forceinline__ float4 rk4_attitude_coefs(float4 u, const DynParams& dp) {
  const float h = dp.dt;
  const float s = 0.25f * (u.y * u.y + u.z * u.z + u.w * u.w);
  const float hh = h * h * s;
  const float cq = 1.0f - 0.5f * hh + hh * hh * (1.0f / 24.0f);
  const float b = 0.5f * h * (1.0f - hh * (1.0f / 6.0f));
  return make_float4(cq, b * u.y, b * u.z, b * u.w);
}

__device__ __forceinline__ void attitude_map(float4 m, float* q) {
  const float n0 = m.x * q[0] - m.y * q[1] - m.z * q[2] - m.w * q[3];
  const float n1 = m.y * q[0] + m.x * q[1] + m.w * q[2] - m.z * q[3];
  const float n2 = m.z * q[0] - m.w * q[1] + m.x * q[2] + m.y * q[3];
  const float n3 = m.w * q[0] + m.z * q[1] - m.y * q[2] + m.x * q[3];
  const float inv = rsqrtf(n0 * n0 + n1 * n1 + n2 * n2 + n3 * n3);
  q[0] = n0 * inv;
  q[1] = n1 * inv;
  q[2] = n2 * inv;
  q[3] = n3 * inv;
}

// Quaternion product a (x) b, components (w, x, y, z) in (.x, .y, .z, .w).
// attitude_map(m, q) is q (x) m renormalised, so a trajectory's attitudes
// are the normalised prefix products q0 (x) m_0 (x) ... (x) m_j.
__device__ __forceinline__ float4 quat_mul4(float4 a, float4 b) {
  return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w,
                     a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                     a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y,
                     a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}

__device__ __forceinline__ float4 shfl_up4(float4 v, int o) {
  return make_float4(__shfl_up_sync(0xffffffffu, v.x, o), __shfl_up_sync(0xffffffffu, v.y, o),
                     __shfl_up_sync(0xffffffffu, v.z, o), __shfl_up_sync(0xffffffffu, v.w, o));
}

// Inclusive prefix products x_0 (x) ... (x) x_t over the threads t of a CTA
// of kWarps warps (order kept: earlier factors on the left); warp_tot: kWarps
// float4 of shared memory.  Every thread of the CTA calls it.
template <int kWarps>
__device__ __forceinline__ float4 block_quat_scan(float4 x, float4* warp_tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float4 y = shfl_up4(x, o);
    if (lane >= o) x = quat_mul4(y, x);
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  float4 pre = make_float4(1.f, 0.f, 0.f, 0.f);
  for (int w = 0; w < wid; ++w) pre = quat_mul4(pre, warp_tot[w]);
  __syncthreads();
  return quat_mul4(pre, x);
}

// Inclusive prefix sums of three components over the threads of a CTA of
// kWarps warps; warp_tot: kWarps float4 of shared memory.
template <int kWarps>
__device__ __forceinline__ float3 block_sum_scan3(float3 x, float4* warp_tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float a = __shfl_up_sync(0xffffffffu, x.x, o), b = __shfl_up_sync(0xffffffffu, x.y, o),
                c = __shfl_up_sync(0xffffffffu, x.z, o);
    if (lane >= o) x = make_float3(a + x.x, b + x.y, c + x.z);
  }
  if (lane == 31) warp_tot[wid] = make_float4(x.x, x.y, x.z, 0.f);
  __syncthreads();
  float3 pre = make_float3(0.f, 0.f, 0.f);
  for (int w = 0; w < wid; ++w) {
    const float4 t = warp_tot[w];
    pre = make_float3(pre.x + t.x, pre.y + t.y, pre.z + t.z);
  }
  __syncthreads();
  return make_float3(pre.x + x.x, pre.y + x.y, pre.z + x.z);
}

// The position and velocity increments of one step from the step's start
// attitude q and control u (the RK4 stage sums of rk4_step):
// p+ = p + h v + inc[0..2], v+ = v + inc[3..5].
__device__ __forceinline__ void rk4_translation_increments(const float* q, float4 u, const DynParams& dp,
                                                           float* inc) {
  const float h = dp.dt;
  const float wx = u.y, wy = u.z, wz = u.w;
  const float a0 = 0.5f * (-q[1] * wx - q[2] * wy - q[3] * wz);
  const float a1 = 0.5f * (q[0] * wx + q[2] * wz - q[3] * wy);
  const float a2 = 0.5f * (q[0] * wy - q[1] * wz + q[3] * wx);
  const float a3 = 0.5f * (q[0] * wz + q[1] * wy - q[2] * wx);
  const float s = 0.25f * (wx * wx + wy * wy + wz * wz);
  const float hh = h * h * s;
  const float c3 = 1.0f - 0.25f * hh, c4 = 1.0f - 0.5f * hh;
  const float hb = 0.5f * h, h4 = h * c3;
  float r1x, r1y, r1z, r2x, r2y, r2z, r3x, r3y, r3z, r4x, r4y, r4z;
  r_e3(q[0], q[1], q[2], q[3], r1x, r1y, r1z);
  r_e3(q[0] + hb * a0, q[1] + hb * a1, q[2] + hb * a2, q[3] + hb * a3, r2x, r2y, r2z);
  r_e3(c3 * q[0] + hb * a0, c3 * q[1] + hb * a1, c3 * q[2] + hb * a2, c3 * q[3] + hb * a3, r3x,
       r3y, r3z);
  r_e3(c4 * q[0] + h4 * a0, c4 * q[1] + h4 * a1, c4 * q[2] + h4 * a2, c4 * q[3] + h4 * a3, r4x,
       r4y, r4z);
  const float f = u.x * dp.inv_mass;
  const float fp = h * h * (1.0f / 6.0f) * f, fv = h * (1.0f / 6.0f) * f;
  const float gp = 0.5f * h * h * dp.g, gv = h * dp.g;
  inc[0] = fp * (r1x + r2x + r3x);
  inc[1] = fp * (r1y + r2y + r3y);
  inc[2] = fp * (r1z + r2z + r3z) - gp;
  inc[3] = fv * (r1x + 2.0f * (r2x + r3x) + r4x);
  inc[4] = fv * (r1y + 2.0f * (r2y + r3y) + r4y);
  inc[5] = fv * (r1z + 2.0f * (r2z + r3z) + r4z) - gv;
}

// The states x_0 .. x_T of the noise-free rollout of u (T <= kWarps * 32
// steps, thread j takes step j) into xs [T + 1][10] (shared memory), the RK4
// step split by dependence and every part a scan over the steps: the
// attitude update is q_{j+1} = N(q_j (x) m_j) with m_j from u_j alone, so
// q_{j+1} = N(q_0 (x) m_0 (x) ... (x) m_j), a prefix product; then each
// step's position and velocity increments from q_j and u_j; then
// v_{j+1} = v_0 + the velocity increments up to j and p_{j+1} = p_0 + the
// sums of h v_i and the position increments up to j.  tot: kWarps float4 of
// shared memory.  Every thread of the CTA calls it; xs is complete when it
// returns.
template <int kWarps>
__device__ __forceinline__ void rollout_by_scans(const float4* u, int T, const float* x0,
                                                 const DynParams& dp, float* xs, float4* tot) {
  const int tid = threadIdx.x;
  const bool on = tid < T;
  const float h = dp.dt;
  const float4 uj = on ? u[tid] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 m = on ? rk4_attitude_coefs(uj, dp) : make_float4(1.f, 0.f, 0.f, 0.f);
  const float4 pm = block_quat_scan<kWarps>(m, tot);
  if (on) {
    const float4 q = quat_mul4(make_float4(x0[3], x0[4], x0[5], x0[6]), pm);
    const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    float* X = xs + (tid + 1) * 10 + 3;
    X[0] = q.x * inv;
    X[1] = q.y * inv;
    X[2] = q.z * inv;
    X[3] = q.w * inv;
  }
  if (tid < 10) xs[tid] = x0[tid];
  __syncthreads();
  float inc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (on) rk4_translation_increments(xs + tid * 10 + 3, uj, dp, inc);
  const float3 dv = block_sum_scan3<kWarps>(make_float3(inc[3], inc[4], inc[5]), tot);
  // v_{j+1} = v0 + dv (inclusive); v_j = v_{j+1} - the step's own increment
  const float3 v1 = make_float3(x0[7] + dv.x, x0[8] + dv.y, x0[9] + dv.z);
  const float3 vj = make_float3(v1.x - inc[3], v1.y - inc[4], v1.z - inc[5]);
  const float3 dpos =
      block_sum_scan3<kWarps>(make_float3(h * vj.x + inc[0], h * vj.y + inc[1], h * vj.z + inc[2]), tot);
  if (on) {
    float* X = xs + (tid + 1) * 10;
    X[0] = x0[0] + dpos.x;
    X[1] = x0[1] + dpos.y;
    X[2] = x0[2] + dpos.z;
    X[7] = v1.x;
    X[8] = v1.y;
    X[9] = v1.z;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Collision queries on the candidate lists.  The list of the query's cell holds
// every collision point closer than d_max to that cell's box, so the nearest
// point, when closer than d_max, is in it.  Queries outside the grid are
// farther than d_max from every point.  Results are the squared distance to
// the nearest point if that is below d_max^2, else d_max^2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int2 cell_range(float px, float py, float pz, const GridView& g) {
  // (p - origin) / h as one multiply-add; a query rounded into a neighbouring
  // cell is within rounding of that cell's box, inside the lists' reach margin
  const float o = -g.origin * g.inv_h;
  const int ix = __float2int_rd(fmaf(px, g.inv_h, o));
  const int iy = __float2int_rd(fmaf(py, g.inv_h, o));
  const int iz = __float2int_rd(fmaf(pz, g.inv_h, o));
  if ((unsigned)ix < (unsigned)g.G && (unsigned)iy < (unsigned)g.G && (unsigned)iz < (unsigned)g.G)
    return __ldg(g.range + (iz * g.G + iy) * g.G + ix);
  return make_int2(0, 0);
}

__device__ __forceinline__ float dist2_to(const float4 q, float px, float py, float pz) {
  const float ax = px - q.x, ay = py - q.y, az = pz - q.z;
  return ax * ax + ay * ay + az * az;
}

// The collision point of candidate entry e of the grid (either form); its w
// holds the bits of the point's item index (the position of the point in the
// collision set: the fine cone of a P_f point, the index of a kept point).
__device__ __forceinline__ float4 grid_point(const GridView& g, int e) {
  return g.cand ? __ldg(g.pts + __ldg(g.cand + e)) : __ldg(g.pts + e);
}

__device__ __forceinline__ int point_item(float4 p) { return __float_as_int(p.w); }

// The same for a grid whose entry form is known at compile time (kIdx: item
// indices), for the per-entry loop of the one-thread pass.
template <bool kIdx>
__device__ __forceinline__ float4 grid_point_of(const GridView& g, int e) {
  if constexpr (kIdx)
    return __ldg(g.pts + __ldg(g.cand + e));
  else
    return __ldg(g.pts + e);
}

// min(dmax2, squared distances to the points of this lane's candidate list),
// for the 32 lanes of a warp together (all call it): lists of at most thr
// entries are scanned by their own lanes; each longer list is then scanned by
// the whole warp, 32 entries per round, the lanes' minima combined with one
// warp reduction over their bits (non-negative floats order as their bits;
// a NaN distance, like fminf's operand, is never the minimum).  The result is
// the exact minimum over the list, whatever the split; a warp whose lists
// differ widely in length (every kept point as the collision set) no longer
// runs its longest list on one lane while the others idle.
template <bool kIdx>
__device__ __forceinline__ float warp_split_min(const GridView& g, int2 range, float px, float py,
                                                float pz, float dmax2, int thr) {
  const int lane = threadIdx.x & 31;
  const bool lng = range.y > thr;
  float d2 = dmax2;
  if (!lng)
    for (int i = 0; i < range.y; ++i)
      d2 = fminf(d2, dist2_to(grid_point_of<kIdx>(g, range.x + i), px, py, pz));
  unsigned pend = __ballot_sync(0xffffffffu, lng);
  while (pend) {
    const int L = __ffs(pend) - 1;
    pend &= pend - 1;
    const int first = __shfl_sync(0xffffffffu, range.x, L);
    const int n = __shfl_sync(0xffffffffu, range.y, L);
    const float qx = __shfl_sync(0xffffffffu, px, L);
    const float qy = __shfl_sync(0xffffffffu, py, L);
    const float qz = __shfl_sync(0xffffffffu, pz, L);
    unsigned best = __float_as_uint(dmax2);
    for (int i = lane; i < n; i += 32) {
      const float d = dist2_to(grid_point_of<kIdx>(g, first + i), qx, qy, qz);
      if (d < dmax2) best = min(best, __float_as_uint(d));
    }
    best = __reduce_min_sync(0xffffffffu, best);
    if (lane == L) d2 = __uint_as_float(best);
  }
  return d2;
}

// min(best, squared distances to the points of the n candidate entries from
// `first`), kW entries per round so that kW loads are in flight; the last
// round repeats its first entry in place of the missing ones (the minimum is
// exact in any order).
template <int kW = 4>
__device__ __forceinline__ float scan_min(const GridView& g, int first, int n, float px, float py,
                                          float pz, float best) {
  const uint32_t* E = g.cand ? g.cand + first : nullptr;
  const float4* P = g.cand ? g.pts : g.pts + first;
  for (int t = 0; t < n; t += kW) {
    float4 c[kW];
    if (E) {
      uint32_t id[kW];
      id[0] = __ldg(E + t);
#pragma unroll
      for (int i = 1; i < kW; ++i) id[i] = t + i < n ? __ldg(E + t + i) : id[0];
#pragma unroll
      for (int i = 0; i < kW; ++i) c[i] = __ldg(P + id[i]);
    } else {
      c[0] = __ldg(P + t);
#pragma unroll
      for (int i = 1; i < kW; ++i) c[i] = t + i < n ? __ldg(P + t + i) : c[0];
    }
    float m = dist2_to(c[0], px, py, pz);
#pragma unroll
    for (int i = 1; i < kW; ++i) m = fminf(m, dist2_to(c[i], px, py, pz));
    best = fminf(best, m);
  }
  return best;
}



// Piecewise collision penalty from a squared distance (d >= d_max -> 0).
__device__ __forceinline__ float jcol_from_d2(float d2, const CostParams& c, float dmax2) {
  if (!(d2 < dmax2)) return 0.0f;
  const float d = fast_sqrt(d2);
  return d < c.d_min ? c.C_col : c.C_col * expf(-c.a_col * (d - c.d_min));
}

// The same value computed without branches (both outcomes evaluated), for
// code that interleaves several independent evaluations.
__device__ __forceinline__ float jcol_select(float d2, const CostParams& c, float dmax2) {
  const float d = fast_sqrt(d2);
  const float ex = c.C_col * expf(-c.a_col * (d - c.d_min));
  return d2 < dmax2 ? (d < c.d_min ? c.C_col : ex) : 0.0f;
}

// ||R(q) R(q_g)^T - I||_F = 2 sqrt(2) |vec(q (x) conj(q_g))| for unit quaternions.
__device__ __forceinline__ float attitude_err(const float* q, const float* g) {
  const float r1 = -q[0] * g[1] + q[1] * g[0] - q[2] * g[3] + q[3] * g[2];
  const float r2 = -q[0] * g[2] + q[1] * g[3] + q[2] * g[0] - q[3] * g[1];
  const float r3 = -q[0] * g[3] - q[1] * g[2] + q[2] * g[1] + q[3] * g[0];
  return 2.8284271247461903f * fast_sqrt(r1 * r1 + r2 * r2 + r3 * r3);
}

__device__ __forceinline__ float norm3f(float a, float b, float c) {
  return fast_sqrt(a * a + b * b + c * c);
}

// A goal at rest: v_goal = 0 and q_goal = (1, 0, 0, 0), the defaults.  Then
// the velocity error is |v| and the attitude error 2 sqrt(2) |vec(q)| (the
// quaternion product's factors 0 and 1 are exact), which goal_term evaluates
// without the product.  Decided once per kernel, before the step loop.
__device__ __forceinline__ bool goal_at_rest(const CostParams& c) {
  return c.v_goal[0] == 0.0f && c.v_goal[1] == 0.0f && c.v_goal[2] == 0.0f && c.q_goal[0] == 1.0f &&
         c.q_goal[1] == 0.0f && c.q_goal[2] == 0.0f && c.q_goal[3] == 0.0f;
}

// Goal term of one step: Q_p |p - p_goal| + Q_v |v - v_goal| + Q_q ||R R_g^T - I||_F.
__device__ __forceinline__ float goal_term(const State& x, const CostParams& c, bool at_rest) {
  const float tp = c.Q_p * norm3f(x.p[0] - c.goal_rel[0], x.p[1] - c.goal_rel[1], x.p[2] - c.goal_rel[2]);
  if (at_rest)
    return tp + c.Q_v * norm3f(x.v[0], x.v[1], x.v[2]) +
           c.Q_q * (2.8284271247461903f * fast_sqrt(x.q[1] * x.q[1] + x.q[2] * x.q[2] + x.q[3] * x.q[3]));
  return tp + c.Q_v * norm3f(x.v[0] - c.v_goal[0], x.v[1] - c.v_goal[1], x.v[2] - c.v_goal[2]) +
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

// Barrier among the kWarps warps that execute it: barrier 0 (the CTA's,
// kWarps = all of them) or named barrier kBar among a subset of warps.
template <int kWarps, int kBar>
__device__ __forceinline__ void warps_sync() {
  if constexpr (kBar == 0) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"n"(kBar), "n"(kWarps * 32) : "memory");
  }
}

// Exclusive prefix sums of (x, y) over kWarps warps (the CTA, or the warps
// that meet at named barrier kBar, numbered wid = 0..kWarps-1 among
// themselves); `total` receives the sums.  warp_tot: kWarps entries of
// shared memory.
template <int kWarps, int kBar = 0>
__device__ __forceinline__ int2 block_scan2(int2 v, int2* warp_tot, int2& total,
                                            int wid = threadIdx.x >> 5) {
  const int lane = threadIdx.x & 31;
  int2 inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int x = __shfl_up_sync(0xffffffffu, inc.x, o), y = __shfl_up_sync(0xffffffffu, inc.y, o);
    if (lane >= o) {
      inc.x += x;
      inc.y += y;
    }
  }
  if (lane == 31) warp_tot[wid] = inc;
  warps_sync<kWarps, kBar>();
  int2 before = make_int2(0, 0);
  total = make_int2(0, 0);
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const int2 t = warp_tot[w];
    if (w < wid) {
      before.x += t.x;
      before.y += t.y;
    }
    total.x += t.x;
    total.y += t.y;
  }
  return make_int2(before.x + inc.x - v.x, before.y + inc.y - v.y);
}

// The listed query holding work item `it`: the largest q < nq with
// first_item[q] <= it (first_item ascending from first_item[0] = 0).
__device__ __forceinline__ int item_owner(const int* first_item, int nq, int it) {
  int lo = 0, hi = nq - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first_item[mid] <= it) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Batched launches: unit -> planner lookup and block-wide copies of arguments.
// ---------------------------------------------------------------------------
// Largest i in [0, n) with pre[i] <= u (pre ascending from pre[0] = 0, u < pre[n]).
__device__ __forceinline__ int find_unit(const long long* pre, int n, long long u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The block copies n + 1 prefix entries (or n order entries) to shared memory.
__device__ __forceinline__ void load_prefix(long long* dst, const long long* src, int n) {
  for (int i = threadIdx.x; i <= n; i += blockDim.x) dst[i] = __ldg(src + i);
}

template <typename T>
__device__ __forceinline__ void block_copy(T* dst, const T* src) {
  static_assert(sizeof(T) % 4 == 0, "word copy");
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = __ldg(s + i);
}

// Copy of a kernel parameter (no __ldg: parameters are not in global memory).
template <typename T>
__device__ __forceinline__ void block_copy_param(T* dst, const T* src) {
  static_assert(sizeof(T) % 4 == 0, "word copy");
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
}

}  // namespace aero
