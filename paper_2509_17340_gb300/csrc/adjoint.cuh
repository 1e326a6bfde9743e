// Gradient of the Stage I cost S(1) of a noise-free rollout with respect to
// its T x 4 controls, by reverse mode (adjoint) through the rollout: the
// dynamics' vector-Jacobian products at the stages of the classical RK4
// step, the quaternion renormalisation, and the cost terms (tracking, velocity
// norm, control, goal, collision).  Not a step of the paper: it serves the
// gradient refinement of the updated nominals before Stage II.
//
// One warp per control sequence.  Every lane runs the same serial RK4 chain on
// the same operands (so all lanes hold the same values); the nearest-point
// queries and the state terms of each 8-step segment run side by side on the
// lanes.  The forward pass keeps a checkpoint every 8 steps; the backward pass
// recomputes each 8-step segment from its checkpoint.
#pragma once

#include "device.cuh"
#include "internal.h"

namespace aero {

constexpr int kCkpt = 8;  // steps per checkpoint segment

// Scratch of one warp in shared memory.
struct AdjScratch {
  float ck[(kMaxT / kCkpt + 1) * 10];  // checkpoints x_0, x_8, x_16, ...
  float seg[(kCkpt + 1) * 10];         // the states of one segment
  float gs[kCkpt][10];                 // state-term gradients of the segment's states
  float d2[kCkpt];                     // their nearest-point squared distances
  float4 nearest[kCkpt];               // and nearest points
};

__device__ __forceinline__ void state_store(float* d, const State& x) {
#pragma unroll
  for (int i = 0; i < 3; ++i) d[i] = x.p[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) d[3 + i] = x.q[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) d[7 + i] = x.v[i];
}

__device__ __forceinline__ State state_load(const float* d) {
  State x;
#pragma unroll
  for (int i = 0; i < 3; ++i) x.p[i] = d[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) x.q[i] = d[3 + i];
#pragma unroll
  for (int i = 0; i < 3; ++i) x.v[i] = d[7 + i];
  return x;
}

// Nearest collision points of the n <= 8 states seg[1..n] by the warp, four
// lanes per state: squared distances (d_max^2 when none is closer) and the
// nearest points into sc.d2 / sc.nearest.  Among equidistant points the one of
// lowest item index wins (the collision set's order, as the oracle breaks
// ties), whatever the order of the entries in the cell's list.
__device__ __forceinline__ void warp_nn_segment(AdjScratch& sc, int n, const GridView& g,
                                                float dmax2, int lane) {
  const int k = lane >> 2, q = lane & 3;
  float best = dmax2;
  int bitem = 0x7fffffff;
  float4 bp = make_float4(0.f, 0.f, 0.f, 0.f);
  if (k < n) {
    const float* x = sc.seg + (k + 1) * 10;
    const int2 r = cell_range(x[0], x[1], x[2], g);
    for (int i = q; i < r.y; i += 4) {
      const float4 p = grid_point(g, r.x + i);
      const float d2 = dist2_to(p, x[0], x[1], x[2]);
      const int item = point_item(p);
      if (d2 < best || (d2 == best && d2 < dmax2 && item < bitem)) {
        best = d2;
        bitem = item;
        bp = p;
      }
    }
  }
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bitem, o);
    const float ox = __shfl_xor_sync(0xffffffffu, bp.x, o);
    const float oy = __shfl_xor_sync(0xffffffffu, bp.y, o);
    const float oz = __shfl_xor_sync(0xffffffffu, bp.z, o);
    if (ob < best || (ob == best && oi < bitem)) {
      best = ob;
      bitem = oi;
      bp = make_float4(ox, oy, oz, bp.w);
    }
  }
  if (k < n && q == 0) {
    sc.d2[k] = best;
    sc.nearest[k] = bitem != 0x7fffffff ? bp : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Stage I state terms at the post-step state x against guide sample (gx, gy,
// gz), given its nearest-point squared distance d2 and nearest point; the
// form the rollout kernels use.  kGrad: the gradient into gs[10] (overwritten).
template <bool kGrad>
__device__ __forceinline__ float state_terms(const State& x, float gx, float gy, float gz,
                                             float d2, float4 nearest, const CostParams& cp,
                                             float dmax2, float* gs) {
  const float ex = x.p[0] - gx, ey = x.p[1] - gy, ez = x.p[2] - gz;
  const float et = norm3f(ex, ey, ez);
  const float px = x.p[0] - cp.goal_rel[0], py = x.p[1] - cp.goal_rel[1], pz = x.p[2] - cp.goal_rel[2];
  const float np = norm3f(px, py, pz);
  const float vx = x.v[0] - cp.v_goal[0], vy = x.v[1] - cp.v_goal[1], vz = x.v[2] - cp.v_goal[2];
  const float nv = norm3f(vx, vy, vz);
  const float* q = x.q;
  const float* qg = cp.q_goal;
  const float r1 = -q[0] * qg[1] + q[1] * qg[0] - q[2] * qg[3] + q[3] * qg[2];
  const float r2 = -q[0] * qg[2] + q[1] * qg[3] + q[2] * qg[0] - q[3] * qg[1];
  const float r3 = -q[0] * qg[3] - q[1] * qg[2] + q[2] * qg[1] + q[3] * qg[0];
  const float nr = fast_sqrt(r1 * r1 + r2 * r2 + r3 * r3);
  const float jc = jcol_from_d2(d2, cp, dmax2);
  const float c = cp.Q_track * et + cp.Q_vnorm * (x.v[0] * x.v[0] + x.v[1] * x.v[1] + x.v[2] * x.v[2]) +
                  cp.Q_p * np + cp.Q_v * nv + cp.Q_q * 2.8284271247461903f * nr + jc;
  if (kGrad) {
#pragma unroll
    for (int i = 0; i < 10; ++i) gs[i] = 0.0f;
    if (et > 0.0f) {
      const float s = cp.Q_track / et;
      gs[0] += s * ex; gs[1] += s * ey; gs[2] += s * ez;
    }
    if (np > 0.0f) {
      const float s = cp.Q_p / np;
      gs[0] += s * px; gs[1] += s * py; gs[2] += s * pz;
    }
    gs[7] += 2.0f * cp.Q_vnorm * x.v[0];
    gs[8] += 2.0f * cp.Q_vnorm * x.v[1];
    gs[9] += 2.0f * cp.Q_vnorm * x.v[2];
    if (nv > 0.0f) {
      const float s = cp.Q_v / nv;
      gs[7] += s * vx; gs[8] += s * vy; gs[9] += s * vz;
    }
    if (nr > 0.0f) {
      // d r / d q: r1 (-g1, g0, -g3, g2), r2 (-g2, g3, g0, -g1), r3 (-g3, -g2, g1, g0)
      const float s = cp.Q_q * 2.8284271247461903f / nr;
      const float a = s * r1, b = s * r2, e = s * r3;
      gs[3] += -a * qg[1] - b * qg[2] - e * qg[3];
      gs[4] += a * qg[0] + b * qg[3] - e * qg[2];
      gs[5] += -a * qg[3] + b * qg[0] + e * qg[1];
      gs[6] += a * qg[2] - b * qg[1] + e * qg[0];
    }
    if (d2 < dmax2) {
      const float d = fast_sqrt(d2);  // as jcol_from_d2 takes it: the same branch of J_col
      if (d >= cp.d_min && d > 0.0f) {
        const float s = -cp.a_col * jc / d;
        gs[0] += s * (x.p[0] - nearest.x);
        gs[1] += s * (x.p[1] - nearest.y);
        gs[2] += s * (x.p[2] - nearest.z);
      }
    }
  }
  return c;
}

// xd = f(x, u) of the quadrotor model (Eq. dynamics) at a stage state.
__device__ __forceinline__ void dyn_f(const float* x, float4 u, const DynParams& dp, float* xd) {
  const float qw = x[3], qx = x[4], qy = x[5], qz = x[6];
  xd[0] = x[7]; xd[1] = x[8]; xd[2] = x[9];
  xd[3] = 0.5f * (-qx * u.y - qy * u.z - qz * u.w);
  xd[4] = 0.5f * (qw * u.y + qy * u.w - qz * u.z);
  xd[5] = 0.5f * (qw * u.z - qx * u.w + qz * u.y);
  xd[6] = 0.5f * (qw * u.w + qx * u.z - qy * u.y);
  float rx, ry, rz;
  r_e3(qw, qx, qy, qz, rx, ry, rz);
  const float f = u.x * dp.inv_mass;
  xd[7] = f * rx; xd[8] = f * ry; xd[9] = f * rz - dp.g;
}

// w^T df/dx added to gx, w^T df/du added to gu, at stage state x.
__device__ __forceinline__ void dyn_vjp(const float* x, float4 u, const DynParams& dp,
                                        const float* w, float* gx, float* gu) {
  const float qw = x[3], qx = x[4], qy = x[5], qz = x[6];
  const float ox = u.y, oy = u.z, oz = u.w;
  gx[7] += w[0]; gx[8] += w[1]; gx[9] += w[2];
  const float W0 = 0.5f * w[3], W1 = 0.5f * w[4], W2 = 0.5f * w[5], W3 = 0.5f * w[6];
  gx[3] += W1 * ox + W2 * oy + W3 * oz;
  gx[4] += -W0 * ox - W2 * oz + W3 * oy;
  gx[5] += -W0 * oy + W1 * oz - W3 * ox;
  gx[6] += -W0 * oz - W1 * oy + W2 * ox;
  gu[1] += -W0 * qx + W1 * qw + W2 * qz - W3 * qy;
  gu[2] += -W0 * qy - W1 * qz + W2 * qw + W3 * qx;
  gu[3] += -W0 * qz + W1 * qy - W2 * qx + W3 * qw;
  const float V0 = w[7], V1 = w[8], V2 = w[9];
  float rx, ry, rz;
  r_e3(qw, qx, qy, qz, rx, ry, rz);
  gu[0] += (V0 * rx + V1 * ry + V2 * rz) * dp.inv_mass;
  const float s = u.x * dp.inv_mass;
  gx[3] += s * (2.0f * qy * V0 - 2.0f * qx * V1);
  gx[4] += s * (2.0f * qz * V0 - 2.0f * qw * V1 - 4.0f * qx * V2);
  gx[5] += s * (2.0f * qw * V0 + 2.0f * qz * V1 - 4.0f * qy * V2);
  gx[6] += s * (2.0f * qx * V0 + 2.0f * qy * V1);
}

// The stage states of one RK4 step from x with control u (Eq. dynamics):
// t2 = x + h/2 k1, t3 = x + h/2 k2, t4 = x + h k3, and the quaternion before
// renormalisation y = q + h/6 (k1 + 2 k2 + 2 k3 + k4) (quaternion part).
__device__ __forceinline__ void rk4_stages(const float* x, float4 u, const DynParams& dp, float* t2,
                                           float* t3, float* t4, float* y) {
  const float h = dp.dt;
  float k1[10], k2[10], k3[10], k4[10];
  dyn_f(x, u, dp, k1);
#pragma unroll
  for (int i = 0; i < 10; ++i) t2[i] = x[i] + 0.5f * h * k1[i];
  dyn_f(t2, u, dp, k2);
#pragma unroll
  for (int i = 0; i < 10; ++i) t3[i] = x[i] + 0.5f * h * k2[i];
  dyn_f(t3, u, dp, k3);
#pragma unroll
  for (int i = 0; i < 10; ++i) t4[i] = x[i] + h * k3[i];
  dyn_f(t4, u, dp, k4);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    y[i] = x[3 + i] + h * (1.0f / 6.0f) * (k1[3 + i] + 2.0f * k2[3 + i] + 2.0f * k3[3 + i] + k4[3 + i]);
}

// Reverse of one RK4 step given its stage states: lam holds dS/dx_{j+1} on
// entry and dS/dx_j on return; gu gets dS/du_j from the dynamics.  Through the
// renormalisation q+ = y/|y| (projection (I - q+ q+^T)/|y|), then the four
// stages in reverse.
__device__ __forceinline__ void rk4_vjp_stages(const float* x, const float* t2, const float* t3,
                                               const float* t4, const float* y, float4 u,
                                               const DynParams& dp, float* lam, float* gu) {
  const float h = dp.dt;
  const float inv = rsqrtf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + y[3] * y[3]);
  const float dot = (y[0] * lam[3] + y[1] * lam[4] + y[2] * lam[5] + y[3] * lam[6]) * inv;
  float ly[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) ly[i] = lam[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) ly[3 + i] = (lam[3 + i] - y[i] * inv * dot) * inv;
  float l1[10], l2[10], l3[10], l4[10], lt[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    lam[i] = ly[i];
    l1[i] = h * (1.0f / 6.0f) * ly[i];
    l2[i] = h * (1.0f / 3.0f) * ly[i];
    l3[i] = l2[i];
    l4[i] = l1[i];
  }
#pragma unroll
  for (int i = 0; i < 10; ++i) lt[i] = 0.0f;
  dyn_vjp(t4, u, dp, l4, lt, gu);
#pragma unroll
  for (int i = 0; i < 10; ++i) { lam[i] += lt[i]; l3[i] += h * lt[i]; lt[i] = 0.0f; }
  dyn_vjp(t3, u, dp, l3, lt, gu);
#pragma unroll
  for (int i = 0; i < 10; ++i) { lam[i] += lt[i]; l2[i] += 0.5f * h * lt[i]; lt[i] = 0.0f; }
  dyn_vjp(t2, u, dp, l2, lt, gu);
#pragma unroll
  for (int i = 0; i < 10; ++i) { lam[i] += lt[i]; l1[i] += 0.5f * h * lt[i]; }
  dyn_vjp(x, u, dp, l1, lam, gu);
}

// Reverse of one RK4 step from x with control u (stage states recomputed).
__device__ __forceinline__ void rk4_vjp(const float* x, float4 u, const DynParams& dp, float* lam,
                                        float* gu) {
  float t2[10], t3[10], t4[10], y[4];
  rk4_stages(x, u, dp, t2, t3, t4, y);
  rk4_vjp_stages(x, t2, t3, t4, y, u, dp, lam, gu);
}

// S(1) of the noise-free rollout of u (shared, T entries) from x0 and, with
// kGrad, dS/du into g (shared, T entries).  guide: T x 3 (shared or global).
// Called by all 32 lanes of one warp; returns S on every lane.
//
// Per 8-step segment: the serial RK4 steps (every lane, identical), the
// segment's nearest-point queries side by side (four lanes per state), its
// state terms side by side (one lane per state).  The backward pass
// recomputes the segment from its checkpoint and runs only the serial
// vector-Jacobian products in order.
template <bool kGrad>
__device__ float warp_cost_grad(const float4* u, float4* g, const float* guide, int T,
                                const float* x0, const DynParams& dp, const CostParams& cp,
                                const GridView& grid, AdjScratch& sc, int lane) {
  const float dmax2 = cp.d_max * cp.d_max;
  const int nseg = (T + kCkpt - 1) / kCkpt;
  State x = state_load(x0);
  float S = 0.0f;
  for (int s = 0; s < nseg; ++s) {
    const int j0 = s * kCkpt, n = min(T, j0 + kCkpt) - j0;
    if (lane == 0) {
      state_store(sc.ck + s * 10, x);
      state_store(sc.seg, x);
    }
    for (int k = 0; k < n; ++k) {
      rk4_step(x, u[j0 + k], dp);
      if (lane == 0) state_store(sc.seg + (k + 1) * 10, x);
    }
    __syncwarp();
    warp_nn_segment(sc, n, grid, dmax2, lane);
    __syncwarp();
    float c = 0.0f;
    if (lane < n) {
      const int j = j0 + lane;
      c = state_terms<false>(state_load(sc.seg + (lane + 1) * 10), guide[3 * j], guide[3 * j + 1],
                             guide[3 * j + 2], sc.d2[lane], sc.nearest[lane], cp, dmax2, nullptr);
    }
    S += warp_sum(c);
    __syncwarp();
  }
  // J_ctrl: Q_c |u_t|^2 (t <= T-2) and Q_cd |u_t - u_{t-1}|^2 (1 <= t <= T-2)
  float jc = 0.0f;
  for (int t = lane; t <= T - 2; t += 32) {
    const float4 a = u[t];
    jc += cp.Q_c * (a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w);
    if (t >= 1) {
      const float4 b = u[t - 1];
      const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
      jc += cp.Q_cd * (dx * dx + dy * dy + dz * dz + dw * dw);
    }
  }
  S += warp_sum(jc);
  if constexpr (kGrad) {
    float lam[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) lam[i] = 0.0f;
    for (int s = nseg - 1; s >= 0; --s) {
      const int j0 = s * kCkpt, n = min(T, j0 + kCkpt) - j0;
      // recompute the segment's states from its checkpoint
      State y = state_load(sc.ck + s * 10);
      if (lane == 0) state_store(sc.seg, y);
      for (int k = 0; k < n; ++k) {
        rk4_step(y, u[j0 + k], dp);
        if (lane == 0) state_store(sc.seg + (k + 1) * 10, y);
      }
      __syncwarp();
      warp_nn_segment(sc, n, grid, dmax2, lane);
      __syncwarp();
      if (lane < n) {
        const int j = j0 + lane;
        float gs[10];
        state_terms<true>(state_load(sc.seg + (lane + 1) * 10), guide[3 * j], guide[3 * j + 1],
                          guide[3 * j + 2], sc.d2[lane], sc.nearest[lane], cp, dmax2, gs);
#pragma unroll
        for (int i = 0; i < 10; ++i) sc.gs[lane][i] = gs[i];
      }
      __syncwarp();
      for (int k = n - 1; k >= 0; --k) {
#pragma unroll
        for (int i = 0; i < 10; ++i) lam[i] += sc.gs[k][i];
        float gu[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        rk4_vjp(sc.seg + k * 10, u[j0 + k], dp, lam, gu);
        if (lane == 0) g[j0 + k] = make_float4(gu[0], gu[1], gu[2], gu[3]);
      }
      __syncwarp();
    }
    // control terms
    for (int t = lane; t < T; t += 32) {
      float4 a = g[t];
      const float4 ut = u[t];
      if (t <= T - 2) {
        a.x += 2.0f * cp.Q_c * ut.x; a.y += 2.0f * cp.Q_c * ut.y;
        a.z += 2.0f * cp.Q_c * ut.z; a.w += 2.0f * cp.Q_c * ut.w;
      }
      if (t >= 1 && t <= T - 2) {
        const float4 b = u[t - 1];
        a.x += 2.0f * cp.Q_cd * (ut.x - b.x); a.y += 2.0f * cp.Q_cd * (ut.y - b.y);
        a.z += 2.0f * cp.Q_cd * (ut.z - b.z); a.w += 2.0f * cp.Q_cd * (ut.w - b.w);
      }
      if (t + 1 >= 1 && t + 1 <= T - 2) {
        const float4 c = u[t + 1];
        a.x -= 2.0f * cp.Q_cd * (c.x - ut.x); a.y -= 2.0f * cp.Q_cd * (c.y - ut.y);
        a.z -= 2.0f * cp.Q_cd * (c.z - ut.z); a.w -= 2.0f * cp.Q_cd * (c.w - ut.w);
      }
      g[t] = a;
    }
    __syncwarp();
  }
  return S;
}

// ---------------------------------------------------------------------------
// Gradient refinement by a whole CTA (the update kernels): the forward
// states by scans over the steps (rollout_by_scans); the backward pass split
// by dependence (suffix sums for the position and velocity adjoints, the 4x4
// attitude recurrence on one thread, the vector-Jacobian products of every
// step in parallel); everything else over the CTA: the stage states of every
// step, the nearest point of every
// state (candidate lists cut into items of kRefItem entries; a 64-bit atomic
// minimum of (squared distance bits, item index) keeps the lowest item among
// equidistant points, the collision set's order), the state terms and their
// gradients, the control terms and the clamped step.  The same arithmetic as
// warp_cost_grad<true> followed by the clamped step.
// ---------------------------------------------------------------------------
constexpr int kRefItem = 8;

struct RefineScratch {
  float4* tot;               // warps: scan totals of the forward rollout
  float4* g;                 // T: dS/du
  unsigned long long* key;   // T: (bits(d2) << 32) | item of the nearest point of x_{j+1}
  float4* near;              // T: that point (entries holding points: found by a second pass)
  int2* qrange;              // T: candidate range of each listed query
  int2* scan;                // warps: block-scan totals
  float* xs;                 // (T + 1) x 10: states x_0 .. x_T
  float* st;                 // T x 34: stage states t2, t3, t4 and y of step j
  float* gs;                 // T x 10: state-term gradients at x_{j+1}
  int* qitem;                // T + 1: first item of each listed query
  int* qslot;                // T: step of each listed query
  float* afm;                // 4 x 20: the attitude adjoint scan's warp compositions
};

__host__ __device__ constexpr size_t refine_smem_bytes(int T, int warps) {
  return 16 * (size_t)warps + 16 * (size_t)T + 8 * (size_t)T + 16 * (size_t)T + 8 * (size_t)T + 8 * (size_t)warps +
         4 * (size_t)(T + 1) * 10 + 4 * (size_t)T * 34 + 4 * (size_t)T * 10 + 4 * (size_t)(T + 1) +
         4 * (size_t)T + 4 * 80;
}

__device__ __forceinline__ RefineScratch refine_layout(unsigned char* base, int T, int warps) {
  RefineScratch r;
  r.tot = reinterpret_cast<float4*>(base);
  r.g = r.tot + warps;
  r.key = reinterpret_cast<unsigned long long*>(r.g + T);
  r.near = reinterpret_cast<float4*>(r.key + T);
  r.qrange = reinterpret_cast<int2*>(r.near + T);
  r.scan = r.qrange + T;
  r.xs = reinterpret_cast<float*>(r.scan + warps);
  r.st = r.xs + (size_t)(T + 1) * 10;
  r.gs = r.st + (size_t)T * 34;
  r.qitem = reinterpret_cast<int*>(r.gs + (size_t)T * 10);
  r.qslot = r.qitem + T + 1;
  r.afm = reinterpret_cast<float*>(r.qslot + T);
  return r;
}


// `steps` clamped gradient steps u <- clamp(u - alpha dS/du) on the nominal u
// (shared, T <= kThreads entries), by all kThreads threads of the CTA.
template <int kThreads>
__device__ void block_refine(float4* u, const float* guide, int T, const float* x0,
                             const DynParams& dp, const CostParams& cp, const GridView& grid,
                             const float* umin, const float* umax, int steps, float alpha,
                             const RefineScratch& rs) {
  const int tid = threadIdx.x;
  const float dmax2 = cp.d_max * cp.d_max;
  const unsigned long long none =
      ((unsigned long long)__float_as_uint(dmax2) << 32) | 0xffffffffull;
  for (int r = 0; r < steps; ++r) {
    // forward: the states x_0 .. x_T, by scans over the steps
    rollout_by_scans<kThreads / 32>(u, T, x0, dp, rs.xs, rs.tot);
    // step tid: its stage states and the candidate range of x_{tid+1}
    int2 rg = make_int2(0, 0);
    if (tid < T) {
      float* stj = rs.st + (size_t)tid * 34;
      rk4_stages(rs.xs + tid * 10, u[tid], dp, stj, stj + 10, stj + 20, stj + 30);
      rs.key[tid] = none;
      const float* x1 = rs.xs + (tid + 1) * 10;
      rg = cell_range(x1[0], x1[1], x1[2], grid);
    }
    int2 total;
    const int2 off = block_scan2<kThreads / 32>(
        rg.y > 0 ? make_int2(1, (rg.y + kRefItem - 1) / kRefItem) : make_int2(0, 0), rs.scan, total);
    if (rg.y > 0) {
      rs.qitem[off.x] = off.y;
      rs.qrange[off.x] = rg;
      rs.qslot[off.x] = tid;
    }
    __syncthreads();
    // the nearest point of a listed query's item of entries: (squared
    // distance, item index) of the point of lowest (distance, item), and the point
    auto item_min = [&](int it, int& j, float& best, int& bitem, float4& bp) {
      const int lo = item_owner(rs.qitem, total.x, it);
      const int2 q = rs.qrange[lo];
      j = rs.qslot[lo];
      const int first = (it - rs.qitem[lo]) * kRefItem;
      const int n = q.y - first < kRefItem ? q.y - first : kRefItem;
      best = dmax2;
      bitem = -1;
      if (!AERO_CHECK(j < T && first >= 0 && n > 0 && q.x >= 0, kChkQuery)) return;
      const float* x1 = rs.xs + (j + 1) * 10;
      for (int c = 0; c < n; ++c) {
        const float4 p = grid_point(grid, q.x + first + c);
        const float d2 = dist2_to(p, x1[0], x1[1], x1[2]);
        const int item = point_item(p);
        if (d2 < best || (d2 == best && bitem >= 0 && item < bitem)) {
          best = d2;
          bitem = item;
          bp = p;
        }
      }
    };
    for (int it = tid; it < total.y; it += kThreads) {
      int j, bitem;
      float best;
      float4 bp;
      item_min(it, j, best, bitem, bp);
      if (bitem >= 0)
        atomicMin(rs.key + j, ((unsigned long long)__float_as_uint(best) << 32) | (unsigned)bitem);
    }
    __syncthreads();
    if (!grid.cand) {
      // entries holding the points: the winner's point from the item that
      // holds the winning (distance, item) pair
      for (int it = tid; it < total.y; it += kThreads) {
        int j, bitem;
        float best;
        float4 bp;
        item_min(it, j, best, bitem, bp);
        if (bitem >= 0 &&
            rs.key[j] == (((unsigned long long)__float_as_uint(best) << 32) | (unsigned)bitem))
          rs.near[j] = bp;
      }
      __syncthreads();
    }
    // state-term gradients at x_{tid+1}
    if (tid < T) {
      const unsigned long long kk = rs.key[tid];
      const float d2 = __uint_as_float((unsigned)(kk >> 32));
      const unsigned bi = (unsigned)kk;
      // entries holding item indices: the item's point directly
      const float4 nearest = bi == 0xffffffffu ? make_float4(0.f, 0.f, 0.f, 0.f)
                             : grid.cand       ? __ldg(grid.pts + bi)
                                               : rs.near[tid];
      state_terms<true>(state_load(rs.xs + (tid + 1) * 10), guide[3 * tid], guide[3 * tid + 1],
                        guide[3 * tid + 2], d2, nearest, cp, dmax2, rs.gs + tid * 10);
    }
    __syncthreads();
    // backward.  With L_{k+1} = dS/dx_{k+1} (the state terms at x_{k+1} plus
    // what flows back from later steps), L_{k+1} = gs[k] + J_{k+1}^T L_{k+2},
    // J the step Jacobian.  Positions feed only positions and velocities only
    // positions and velocities, so the position and velocity parts are
    // suffix sums: Lp_{k+1} = sum_{i >= k} gs_p[i], Lv_{k+1} = sum_{i >= k}
    // (gs_v[i] + h Lp_{i+2}).  The attitude part is the linear recurrence
    // Lq_{k+1} = gs_q[k] + b_{k+1} + A_{k+1}^T Lq_{k+2}: b the attitude part of
    // J^T (Lp, 0, Lv) (the step's vector-Jacobian product, in parallel), A the
    // 4x4 attitude Jacobian, whose transpose is applied in closed form: the
    // unnormalised y = q (x) m, so A^T l = ((l - yh (yh . l)) / |y|) (x) conj(m),
    // yh = y / |y|; one thread chains it.  Then every step's dS/du_k is the
    // control part of J_k^T L_{k+1}, in parallel.
    {
      const float h = dp.dt;
      // (a) the suffix sums, thread t taking step k = T - 1 - t
      const int k = T - 1 - tid;
      const bool on = tid < T;
      const float* g = rs.gs + (on ? k : 0) * 10;
      const float3 gp = on ? make_float3(g[0], g[1], g[2]) : make_float3(0.f, 0.f, 0.f);
      const float3 gv = on ? make_float3(g[7], g[8], g[9]) : make_float3(0.f, 0.f, 0.f);
      const float3 lp = block_sum_scan3<kThreads / 32>(gp, rs.tot);
      const float3 lp2 = make_float3(lp.x - gp.x, lp.y - gp.y, lp.z - gp.z);  // Lp_{k+2}
      const float3 lv = block_sum_scan3<kThreads / 32>(
          make_float3(gv.x + h * lp2.x, gv.y + h * lp2.y, gv.z + h * lp2.z), rs.tot);
      if (on) {
        float* L = rs.gs + k * 10;
        L[0] = lp.x; L[1] = lp.y; L[2] = lp.z;
        L[7] = lv.x; L[8] = lv.y; L[9] = lv.z;
      }
      __syncthreads();
      // (b) b_k for every step k = tid, into rs.g
      if (tid < T) {
        const float* L = rs.gs + tid * 10;
        float lam[10] = {L[0], L[1], L[2], 0.f, 0.f, 0.f, 0.f, L[7], L[8], L[9]};
        float gu[4] = {0.f, 0.f, 0.f, 0.f};
        const float* stk = rs.st + (size_t)tid * 34;
        rk4_vjp_stages(rs.xs + tid * 10, stk, stk + 10, stk + 20, stk + 30, u[tid], dp, lam, gu);
        rs.g[tid] = make_float4(lam[3], lam[4], lam[5], lam[6]);
      }
      __syncthreads();
      // (c) the attitude recurrence Lq_k = C_k + A_{k+1}^T Lq_{k+1} (k = T-2
      // .. 0; C_k = gs_q[k] + b_{k+1}; Lq_{T-1} = gs_q[T-1]) is affine in Lq:
      // thread t = T-2-k holds the map x -> C_k + M x (M = A_{k+1}^T as a 4x4
      // matrix, its columns the images of the unit vectors), and an inclusive
      // scan composes the maps, later ones outside, so that thread t ends with
      // the composition that takes Lq_{T-1} to Lq_k.  T - 1 <= 127 maps: up to
      // four warps, each carrying the earlier warps' compositions.
      static_assert(kMaxT - 1 <= 128 && kThreads >= 128, "the attitude adjoint scan spans four warps");
      {
        const int kk = T - 2 - tid, wid = tid >> 5;
        const bool on = kk >= 0;
        float M[16], c[4];
#pragma unroll
        for (int i = 0; i < 16; ++i) M[i] = (i % 5 == 0) ? 1.0f : 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) c[i] = 0.0f;
        if (on) {
          const int j = kk + 1;  // A_j: the attitude Jacobian of step j
          const float* y = rs.st + (size_t)j * 34 + 30;
          const float inv = rsqrtf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + y[3] * y[3]);
          const float4 m = rk4_attitude_coefs(u[j], dp);
          const float4 mc = make_float4(m.x, -m.y, -m.z, -m.w);
#pragma unroll
          for (int col = 0; col < 4; ++col) {
            // A_j^T e_col = ((e_col - yh (yh . e_col)) / |y|) (x) conj(m)
            const float d = y[col] * inv * inv;
            const float4 pl = make_float4(((col == 0 ? 1.f : 0.f) - y[0] * d) * inv,
                                          ((col == 1 ? 1.f : 0.f) - y[1] * d) * inv,
                                          ((col == 2 ? 1.f : 0.f) - y[2] * d) * inv,
                                          ((col == 3 ? 1.f : 0.f) - y[3] * d) * inv);
            const float4 at = quat_mul4(pl, mc);
            M[col] = at.x;
            M[4 + col] = at.y;
            M[8 + col] = at.z;
            M[12 + col] = at.w;
          }
          const float* Lk = rs.gs + kk * 10 + 3;
          const float4 b = rs.g[j];
          c[0] = Lk[0] + b.x;
          c[1] = Lk[1] + b.y;
          c[2] = Lk[2] + b.z;
          c[3] = Lk[3] + b.w;
        }
        // (M, c) o (M', c') = (M M', M c' + c)
        auto compose = [&](const float* M2, const float* c2) {
          float R[16], r[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              R[4 * i + q] = M[4 * i] * M2[q] + M[4 * i + 1] * M2[4 + q] + M[4 * i + 2] * M2[8 + q] +
                             M[4 * i + 3] * M2[12 + q];
            r[i] = M[4 * i] * c2[0] + M[4 * i + 1] * c2[1] + M[4 * i + 2] * c2[2] +
                   M[4 * i + 3] * c2[3] + c[i];
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) M[i] = R[i];
#pragma unroll
          for (int i = 0; i < 4; ++i) c[i] = r[i];
        };
        if (wid < 4) {
          const int lane = tid & 31;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            float M2[16], c2[4];
#pragma unroll
            for (int i = 0; i < 16; ++i) M2[i] = __shfl_up_sync(0xffffffffu, M[i], o);
#pragma unroll
            for (int i = 0; i < 4; ++i) c2[i] = __shfl_up_sync(0xffffffffu, c[i], o);
            if (lane >= o) compose(M2, c2);
          }
          if (lane == 31) {
#pragma unroll
            for (int i = 0; i < 16; ++i) rs.afm[20 * wid + i] = M[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) rs.afm[20 * wid + 16 + i] = c[i];
          }
        }
        __syncthreads();
        if (on) {
          // the earlier warps' compositions, the latest one first (inside)
          for (int v = wid - 1; v >= 0; --v) {
            float M2[16], c2[4];
#pragma unroll
            for (int i = 0; i < 16; ++i) M2[i] = rs.afm[20 * v + i];
#pragma unroll
            for (int i = 0; i < 4; ++i) c2[i] = rs.afm[20 * v + 16 + i];
            compose(M2, c2);
          }
        }
        if (on) {
          const float* L = rs.gs + (T - 1) * 10 + 3;  // Lq_{T-1}
          const float l0 = L[0], l1 = L[1], l2 = L[2], l3 = L[3];
          float* Lk = rs.gs + kk * 10 + 3;
          float lo[4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
            lo[i] = M[4 * i] * l0 + M[4 * i + 1] * l1 + M[4 * i + 2] * l2 + M[4 * i + 3] * l3 + c[i];
#pragma unroll
          for (int i = 0; i < 4; ++i) Lk[i] = lo[i];
        }
      }
      __syncthreads();
      // (d) dS/du_k = the control part of J_k^T L_{k+1}
      if (tid < T) {
        float lam[10];
#pragma unroll
        for (int i = 0; i < 10; ++i) lam[i] = rs.gs[tid * 10 + i];
        float gu[4] = {0.f, 0.f, 0.f, 0.f};
        const float* stk = rs.st + (size_t)tid * 34;
        rk4_vjp_stages(rs.xs + tid * 10, stk, stk + 10, stk + 20, stk + 30, u[tid], dp, lam, gu);
        rs.g[tid] = make_float4(gu[0], gu[1], gu[2], gu[3]);
      }
    }
    __syncthreads();
    // control terms, then the clamped step
    if (tid < T) {
      const int t = tid;
      float4 a = rs.g[t];
      const float4 ut = u[t];
      if (t <= T - 2) {
        a.x += 2.0f * cp.Q_c * ut.x; a.y += 2.0f * cp.Q_c * ut.y;
        a.z += 2.0f * cp.Q_c * ut.z; a.w += 2.0f * cp.Q_c * ut.w;
      }
      if (t >= 1 && t <= T - 2) {
        const float4 b = u[t - 1];
        a.x += 2.0f * cp.Q_cd * (ut.x - b.x); a.y += 2.0f * cp.Q_cd * (ut.y - b.y);
        a.z += 2.0f * cp.Q_cd * (ut.z - b.z); a.w += 2.0f * cp.Q_cd * (ut.w - b.w);
      }
      if (t + 1 >= 1 && t + 1 <= T - 2) {
        const float4 c = u[t + 1];
        a.x -= 2.0f * cp.Q_cd * (c.x - ut.x); a.y -= 2.0f * cp.Q_cd * (c.y - ut.y);
        a.z -= 2.0f * cp.Q_cd * (c.z - ut.z); a.w -= 2.0f * cp.Q_cd * (c.w - ut.w);
      }
      rs.g[t] = a;
    }
    __syncthreads();
    if (tid < T) {
      const float4 a = u[tid], d = rs.g[tid];
      u[tid] = make_float4(fminf(fmaxf(a.x - alpha * d.x, umin[0]), umax[0]),
                           fminf(fmaxf(a.y - alpha * d.y, umin[1]), umax[1]),
                           fminf(fmaxf(a.z - alpha * d.z, umin[2]), umax[2]),
                           fminf(fmaxf(a.w - alpha * d.w, umin[3]), umax[3]));
    }
    __syncthreads();
  }
}

}  // namespace aero

