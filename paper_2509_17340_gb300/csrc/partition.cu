// Multi-resolution partition (Sec. IV-A), anchors (Sec. IV-B.1-2), quintic
// guides (Sec. IV-B.3) and the uniform collision grid over the collision set.
//
// Integer decisions (cone of a point, its range key, the coarse winner, the
// goal's cone) are taken in binary32 with explicitly rounded operations
// (__fmul_rn / __fadd_rn / __fsub_rn never fuse into FMA), in a fixed order,
// so they are a defined function of the binary32 inputs.
#include <cfloat>
#include <cstdint>

#include "device.cuh"
#include "internal.h"

namespace aero {
namespace {

constexpr unsigned long long kEmpty = 0xFFFFFFFFFFFFFFFFull;

__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }

// b = R^T (p - p0), each dot product summed left to right.
__device__ __forceinline__ void to_body(const float* R, float dx, float dy, float dz, float* b) {
  b[0] = add(add(mul(R[0], dx), mul(R[3], dy)), mul(R[6], dz));
  b[1] = add(add(mul(R[1], dx), mul(R[4], dy)), mul(R[7], dz));
  b[2] = add(add(mul(R[2], dx), mul(R[5], dy)), mul(R[8], dz));
}

// Largest azimuth edge index reached, by bisection within the half plane.
__device__ __forceinline__ int az_bin(const float* ca, const float* sa, int A, float bx, float by) {
  const int half = A >> 1;
  const bool upper = (by > 0.0f) || (by == 0.0f && bx > 0.0f);
  int lo = upper ? half : 0, hi = upper ? A - 1 : half - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const float s = sub(mul(by, ca[mid]), mul(bx, sa[mid]));
    if (s >= 0.0f) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int el_bin(const float* ce, const float* se, int El, float bz, float rho) {
  int lo = 0, hi = El - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const float s = sub(mul(bz, ce[mid]), mul(rho, se[mid]));
    if (s >= 0.0f) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int grid_cell(float dx, float dy, float dz, const GridGeom& g) {
  int cx = __float2int_rd((dx - g.origin) * g.inv_h);
  int cy = __float2int_rd((dy - g.origin) * g.inv_h);
  int cz = __float2int_rd((dz - g.origin) * g.inv_h);
  cx = min(max(cx, 0), g.G - 1);
  cy = min(max(cy, 0), g.G - 1);
  cz = min(max(cz, 0), g.G - 1);
  return (cz * g.G + cy) * g.G + cx;
}

// ---------------------------------------------------------------------------
// K1: cone of every point and atomic minimum of its key per cone.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_partition(PartitionArgs a, PartTables t) {
  __shared__ float s_ca[kMaxAz], s_sa[kMaxAz], s_ce[kMaxEl + 1], s_se[kMaxEl + 1];
  for (int i = threadIdx.x; i < a.A; i += blockDim.x) {
    s_ca[i] = t.ca[i];
    s_sa[i] = t.sa[i];
  }
  for (int i = threadIdx.x; i <= a.El; i += blockDim.x) {
    s_ce[i] = t.ce[i];
    s_se[i] = t.se[i];
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const float px = __ldg(a.cloud + 3 * i), py = __ldg(a.cloud + 3 * i + 1),
                pz = __ldg(a.cloud + 3 * i + 2);
    int cell = -1;
    if (isfinite(px) && isfinite(py) && isfinite(pz)) {
      const float dx = sub(px, a.p0[0]), dy = sub(py, a.p0[1]), dz = sub(pz, a.p0[2]);
      float b[3];
      to_body(a.R, dx, dy, dz, b);
      const float rxy2 = add(mul(b[0], b[0]), mul(b[1], b[1]));
      const float r2 = add(rxy2, mul(b[2], b[2]));
      if (r2 > 0.0f && r2 <= a.rmax2) {
        const float rho = __fsqrt_rn(rxy2);
        bool ok = true;
        if (a.check_lo && !(sub(mul(b[2], s_ce[0]), mul(rho, s_se[0])) >= 0.0f)) ok = false;
        if (a.check_hi && (sub(mul(b[2], s_ce[a.El]), mul(rho, s_se[a.El])) > 0.0f)) ok = false;
        if (ok) {
          const int ia = az_bin(s_ca, s_sa, a.A, b[0], b[1]);
          const int je = el_bin(s_ce, s_se, a.El, b[2], rho);
          const int c = je * a.A + ia;
          const unsigned long long key =
              ((unsigned long long)__float_as_uint(r2) << 32) | (unsigned long long)(uint32_t)i;
          atomicMin(a.keys + c, key);
          cell = c;
          if (a.raw) {
            const int gc = grid_cell(dx, dy, dz, a.grid);
            a.item_cell[i] = gc;
            a.item_slot[i] = atomicAdd(a.grid_count + gc, 1);
          }
        }
      }
    }
    if (a.raw && cell < 0) a.item_cell[i] = -1;
  }
}

// ---------------------------------------------------------------------------
// K2a (collision set = P_f): grid cell of the winner of every non-empty cone.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_pf_count(const unsigned long long* __restrict__ keys,
                                                  int ncell, const float* __restrict__ cloud,
                                                  float p0x, float p0y, float p0z, GridGeom g,
                                                  int* grid_count, int* item_cell,
                                                  int* item_slot) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const unsigned long long key = keys[c];
  if (key == kEmpty) {
    item_cell[c] = -1;
    return;
  }
  const int64_t i = (int64_t)(key & 0xFFFFFFFFull);
  const float dx = sub(__ldg(cloud + 3 * i), p0x), dy = sub(__ldg(cloud + 3 * i + 1), p0y),
              dz = sub(__ldg(cloud + 3 * i + 2), p0z);
  const int gc = grid_cell(dx, dy, dz, g);
  item_cell[c] = gc;
  item_slot[c] = atomicAdd(grid_count + gc, 1);
}

// ---------------------------------------------------------------------------
// K2b + K3: block 0 turns the grid counts into cell starts (exclusive scan);
// block 1 runs the coarse argmax, the goal cone, the anchor cells, the anchors
// and the quintic guides.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;

__device__ void scan_block(int* data, int n) {
  __shared__ int s_warp[32];
  __shared__ int s_carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 4 * kScanThreads) {
    const int i0 = base + 4 * tid;
    int v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = (i0 + u < n) ? data[i0 + u] : 0;
    const int tsum = v[0] + v[1] + v[2] + v[3];
    int incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int w = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      s_warp[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    int run = s_carry + (wid > 0 ? s_warp[wid - 1] : 0) + incl - tsum;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (i0 + u < n) data[i0 + u] = run;
      run += v[u];
    }
    __syncthreads();
    if (tid == kScanThreads - 1) s_carry = run;
    __syncthreads();
  }
  if (tid == 0) data[n] = s_carry;
}

__device__ void coarse_guides_block(const GuideArgs& a, const PartTables& t) {
  __shared__ float s_ca[kMaxAz], s_sa[kMaxAz], s_ce[kMaxEl + 1], s_se[kMaxEl + 1];
  __shared__ float s_coef[kMaxE][3][6];
  for (int i = threadIdx.x; i < a.A; i += blockDim.x) {
    s_ca[i] = t.ca[i];
    s_sa[i] = t.sa[i];
  }
  for (int i = threadIdx.x; i <= a.El; i += blockDim.x) {
    s_ce[i] = t.ce[i];
    s_se[i] = t.se[i];
  }
  __syncthreads();
  // coarse argmax (Eq. safe-vector): larger r, then nearer the coarse centre,
  // then lower fine index; empty cones count as r_max.
  const uint32_t empty_bits = __float_as_uint(a.rmax2);
  const int ncoarse = a.Ac * a.Ec;
  for (int cc = threadIdx.x; cc < ncoarse; cc += blockDim.x) {
    const int I = cc % a.Ac, J = cc / a.Ac;
    int best = -1, bdist = 0;
    uint32_t bkey = 0;
    for (int b = 0; b < a.Pe; ++b)
      for (int q = 0; q < a.Pa; ++q) {
        const int c = (J * a.Pe + b) * a.A + I * a.Pa + q;
        const unsigned long long k = a.keys[c];
        const uint32_t rk = k == kEmpty ? empty_bits : (uint32_t)(k >> 32);
        const int dist = abs(2 * q + 1 - a.Pa) + abs(2 * b + 1 - a.Pe);
        if (best < 0 || rk > bkey || (rk == bkey && (dist < bdist || (dist == bdist && c < best)))) {
          best = c;
          bkey = rk;
          bdist = dist;
        }
      }
    a.coarse_win[cc] = best;
  }
  __syncthreads();
  // goal cone and the M_h x M_v anchor cells around it (Sec. IV-B.1)
  __shared__ int s_goal;
  if (threadIdx.x == 0) {
    float b[3];
    to_body(a.R, a.goal_rel[0], a.goal_rel[1], a.goal_rel[2], b);
    const float rho = __fsqrt_rn(add(mul(b[0], b[0]), mul(b[1], b[1])));
    s_goal = el_bin(s_ce, s_se, a.El, b[2], rho) * a.A + az_bin(s_ca, s_sa, a.A, b[0], b[1]);
    a.cells[0] = s_goal;
  }
  __syncthreads();
  if (threadIdx.x < a.E) {
    const int e = threadIdx.x, m = e % a.M_h, n = e / a.M_h;
    const int Ig = (s_goal % a.A) / a.Pa, Jg = (s_goal / a.A) / a.Pe;
    const int I = ((Ig + m - a.M_h / 2) % a.Ac + a.Ac) % a.Ac;
    const int J = min(max(Jg + n - a.M_v / 2, 0), a.Ec - 1);
    const int cc = J * a.Ac + I;
    a.cells[1 + e] = cc;
    // direction of the winning cone's centre (Eq. unit direction), binary64
    const int w = a.coarse_win[cc];
    const int i = w % a.A, j = w / a.A;
    const double lo = (double)a.el_lo, hi = (double)a.el_hi;
    const double al = -3.141592653589793 + (i + 0.5) * (2.0 * 3.141592653589793 / a.A);
    const double be = lo + (j + 0.5) * ((hi - lo) / a.El);
    double sa, ca, sb, cb;
    sincos(al, &sa, &ca);
    sincos(be, &sb, &cb);
    const float db[3] = {(float)(cb * ca), (float)(cb * sa), (float)sb};
    // anchor p_ref - p0 = ell R(q0) d (Eq. anchor-point)
    float pr[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      pr[r] = a.ell * (a.R[3 * r] * db[0] + a.R[3 * r + 1] * db[1] + a.R[3 * r + 2] * db[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      a.anchors[3 * e + r] = pr[r];
    }
    // quintic in normalised time s = t / Tg: f(s) = sum b_i s^i with
    // f(0)=0, f'(0)=v0 Tg, f''(0)=0, f(1)=p_ref, f'(1)=v_end u Tg, f''(1)=0
    const float Tg = a.T * a.dt;
    const float v_end = a.v_end > 0.0f ? a.v_end : a.ell / Tg;
    const float L = sqrtf(pr[0] * pr[0] + pr[1] * pr[1] + pr[2] * pr[2]);
    const float sc = L > 0.0f ? v_end / L : 0.0f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float h = pr[r];
      const float V0 = a.v0[r] * Tg, V1 = sc * pr[r] * Tg;
      s_coef[e][r][0] = 0.0f;
      s_coef[e][r][1] = V0;
      s_coef[e][r][2] = 0.0f;
      s_coef[e][r][3] = 10.0f * h - 6.0f * V0 - 4.0f * V1;
      s_coef[e][r][4] = -15.0f * h + 8.0f * V0 + 7.0f * V1;
      s_coef[e][r][5] = 6.0f * h - 3.0f * V0 - 3.0f * V1;
    }
  }
  __syncthreads();
  // guide samples at t = (j+1) dt
  const float inv_T = 1.0f / a.T;
  for (int idx = threadIdx.x; idx < a.E * a.T; idx += blockDim.x) {
    const int e = idx / a.T, j = idx % a.T;
    const float s = (j + 1) * inv_T;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float* c = s_coef[e][r];
      const float f = ((((c[5] * s + c[4]) * s + c[3]) * s + c[2]) * s + c[1]) * s + c[0];
      a.guides[(e * a.T + j) * 3 + r] = f;
    }
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_guides(GuideArgs a, PartTables t) {
  if (blockIdx.x == 0)
    scan_block(a.grid_start, a.ncells);
  else
    coarse_guides_block(a, t);
}

// ---------------------------------------------------------------------------
// K2c: place every collision point at start[cell] + slot.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scatter(ScatterArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.n_items; c += stride) {
    const int gc = a.item_cell[c];
    if (gc < 0) continue;
    const int64_t i = a.raw ? c : (int64_t)(a.keys[c] & 0xFFFFFFFFull);
    const float dx = sub(__ldg(a.cloud + 3 * i), a.p0[0]);
    const float dy = sub(__ldg(a.cloud + 3 * i + 1), a.p0[1]);
    const float dz = sub(__ldg(a.cloud + 3 * i + 2), a.p0[2]);
    a.grid_pts[a.grid_start[gc] + a.item_slot[c]] = make_float4(dx, dy, dz, 0.0f);
  }
}

__global__ void k_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3,
                         int64_t n, uint4* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = philox4x32_10(make_uint4((uint32_t)i, c1, c2, c3), k0, k1);
}

int blocks_for(int64_t n, int threads, int cap) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

}  // namespace

cudaError_t launch_partition(const PartitionArgs& a, const PartTables& t, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  k_partition<<<blocks_for(a.n, 256, 152 * 16), 256, 0, s>>>(a, t);
  return cudaGetLastError();
}

cudaError_t launch_pf_count(const unsigned long long* keys, int ncell, const float* cloud,
                            const float p0[3], GridGeom g, int* grid_count, int* item_cell,
                            int* item_slot, cudaStream_t s) {
  k_pf_count<<<blocks_for(ncell, 256, 1 << 20), 256, 0, s>>>(keys, ncell, cloud, p0[0], p0[1],
                                                             p0[2], g, grid_count, item_cell,
                                                             item_slot);
  return cudaGetLastError();
}

cudaError_t launch_scan_guides(const GuideArgs& a, const PartTables& t, cudaStream_t s) {
  k_scan_guides<<<2, kScanThreads, 0, s>>>(a, t);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const ScatterArgs& a, cudaStream_t s) {
  if (a.n_items == 0) return cudaSuccess;
  k_scatter<<<blocks_for(a.n_items, 256, 152 * 16), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3,
                          int64_t n, uint32_t* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_philox<<<blocks_for(n, 256, 152 * 16), 256, 0, s>>>(k0, k1, c1, c2, c3, n,
                                                          reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

}  // namespace aero
