// Multi-resolution partition (Sec. IV-A), anchors (Sec. IV-B.1-2), quintic
// guides (Sec. IV-B.3) and the collision grid: per-cell candidate lists over
// the collision set (P_f of Sec. IV-C, or every kept point).
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

// A guess of atan2(y, x), within 1e-4 rad: the octant folded to t = min/max
// in [0, 1] and atan t by an odd polynomial of degree 7 fitted to it on [0, 1]
// (coefficients from a least-squares fit made for this kernel; maximum error
// 8.3e-5 rad).  It only picks where the exact predicates start: the bins below
// are decided by those predicates.
__device__ __forceinline__ float atan2_guess(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  const float t = mx > 0.0f ? __fdividef(mn, mx) : 0.0f;
  const float t2 = t * t;
  float r = t * (0.99921519f + t2 * (-0.32118943f + t2 * (0.14629962f + t2 * -0.039010014f)));
  if (ay > ax) r = 1.570796327f - r;
  if (x < 0.0f) r = 3.141592654f - r;
  return y < 0.0f ? -r : r;
}

// The bisection's result -- the largest k in (lo, hi] whose predicate holds,
// else lo -- found from a guess g: g is that index iff (g == lo or pred(g))
// and (g == hi or not pred(g + 1)), which singles it out because the
// predicate holds up to the point's direction and not after it (only the edge
// nearest the point can be within rounding of it, and the same arithmetic
// decides it either way).  A guess one edge off is corrected with one more
// predicate; anything else falls back to the bisection.
template <typename Pred>
__device__ __forceinline__ int bin_from_guess(int g, int lo, int hi, Pred pred) {
  g = min(max(g, lo), hi);
  const bool at_or_above = g == lo || pred(g);      // the result is >= g
  const bool at_or_below = g == hi || !pred(g + 1);  // the result is <= g
  if (at_or_above && at_or_below) return g;
  if (!at_or_above && at_or_below && (g - 1 == lo || pred(g - 1))) return g - 1;
  if (at_or_above && !at_or_below && (g + 1 == hi || !pred(g + 2))) return g + 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pred(mid)) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// az_bin and el_bin from an angle guess (the same results).
__device__ __forceinline__ int az_bin_guess(const float* ca, const float* sa, int A, float bx, float by) {
  const int half = A >> 1;
  const bool upper = (by > 0.0f) || (by == 0.0f && bx > 0.0f);
  const int g = __float2int_rd((atan2_guess(by, bx) + 3.141592654f) * ((float)A * 0.159154943f));
  return bin_from_guess(g, upper ? half : 0, upper ? A - 1 : half - 1, [&](int k) {
    return sub(mul(by, ca[k]), mul(bx, sa[k])) >= 0.0f;
  });
}

__device__ __forceinline__ int el_bin_guess(const float* ce, const float* se, int El, float bz, float rho,
                                            float el_lo, float el_inv) {
  const int g = __float2int_rd((atan2_guess(bz, rho) - el_lo) * el_inv);
  return bin_from_guess(g, 0, El - 1, [&](int k) { return sub(mul(bz, ce[k]), mul(rho, se[k])) >= 0.0f; });
}

// ---------------------------------------------------------------------------
// K1: cone of every point and atomic minimum of its key per cone.
// ---------------------------------------------------------------------------
// Edge tables in shared memory.
struct SmemTables {
  float ca[kMaxAz], sa[kMaxAz], ce[kMaxEl + 1], se[kMaxEl + 1];
};

__device__ __forceinline__ void load_tables(const PartTables& t, int A, int El, SmemTables& s) {
  for (int i = threadIdx.x; i < A; i += blockDim.x) {
    s.ca[i] = t.ca[i];
    s.sa[i] = t.sa[i];
  }
  for (int i = threadIdx.x; i <= El; i += blockDim.x) {
    s.ce[i] = t.ce[i];
    s.se[i] = t.se[i];
  }
}

__device__ __forceinline__ float3 cloud_point(const PartitionArgs& a, int64_t i) {
  return make_float3(__ldg(a.cloud + 3 * i), __ldg(a.cloud + 3 * i + 1), __ldg(a.cloud + 3 * i + 2));
}

constexpr int kNonFinite = -2;  // cone_of: a non-finite point
constexpr int kOutside = -1;    // cone_of: outside the range or the elevation span

// The fine cone of the point at pt, or kOutside / kNonFinite; *r2 its squared
// range in binary32 (set for a cone only).
__device__ __forceinline__ int cone_of(const PartitionArgs& a, const SmemTables& st, float3 pt,
                                       float* r2_out) {
  const float px = pt.x, py = pt.y, pz = pt.z;
  if (!(isfinite(px) && isfinite(py) && isfinite(pz))) return kNonFinite;
  const float dx = sub(px, a.p0[0]), dy = sub(py, a.p0[1]), dz = sub(pz, a.p0[2]);
  float b[3];
  to_body(a.R, dx, dy, dz, b);
  const float rxy2 = add(mul(b[0], b[0]), mul(b[1], b[1]));
  const float r2 = add(rxy2, mul(b[2], b[2]));
  if (!(r2 > 0.0f && r2 <= a.rmax2)) return kOutside;
  const float rho = __fsqrt_rn(rxy2);
  if (a.check_lo && !(sub(mul(b[2], st.ce[0]), mul(rho, st.se[0])) >= 0.0f)) return kOutside;
  if (a.check_hi && (sub(mul(b[2], st.ce[a.El]), mul(rho, st.se[a.El])) > 0.0f)) return kOutside;
  const int ia = az_bin_guess(st.ca, st.sa, a.A, b[0], b[1]);
  const int je = el_bin_guess(st.ce, st.se, a.El, b[2], rho, a.el_lo, a.el_inv);
  const int c = je * a.A + ia;
  if (!AERO_CHECK(c >= 0 && c < a.A * a.El, kChkFineCell)) return kOutside;
  *r2_out = r2;
  return c;
}

// The key of point i at squared range r2: the range bits above the index, so
// that the minimum is the nearest point, the lowest index among equals.
__device__ __forceinline__ unsigned long long cone_key(float r2, uint32_t i) {
  return ((unsigned long long)__float_as_uint(r2) << 32) | (unsigned long long)i;
}

// Point i at (px, py, pz).  Returns 0 for a non-finite point, 1 for a point
// outside the partition's range or elevation span, 2 for a kept point.
__device__ __forceinline__ int partition_point(const PartitionArgs& a, const SmemTables& st,
                                               int64_t i, float3 pt) {
  float r2 = 0.0f;
  const int c = cone_of(a, st, pt, &r2);
  if (c >= 0) {
    const unsigned long long key = cone_key(r2, (uint32_t)i);
    // dense clouds: a key at or above the cone's current minimum cannot
    // lower it, so the atomic is skipped.  Keys only decrease during the
    // pass, so a value read earlier is never below the current one and
    // the test skips no atomic that would lower the key.
    if (!a.filter || key < __ldcg(a.keys + c)) atomicMin(a.keys + c, key);
  }
  if (a.item_flag) a.item_flag[i] = c >= 0 ? 1 : 0;
  return c == kNonFinite ? 0 : c >= 0 ? 2 : 1;
}

// Points 4 g .. 4 g + 3 (a 16-byte aligned cloud: three float4 loads).  The
// four cones are found first and their keys read together, so that the four
// reads of the current minima are in flight at once.
__device__ __forceinline__ void partition_group(const PartitionArgs& a, const SmemTables& st,
                                                int64_t g, float4 v0, float4 v1, float4 v2,
                                                int& nf, int& kept) {
  const float3 pt[4] = {make_float3(v0.x, v0.y, v0.z), make_float3(v0.w, v1.x, v1.y),
                        make_float3(v1.z, v1.w, v2.x), make_float3(v2.y, v2.z, v2.w)};
  const uint32_t i0 = (uint32_t)(4 * g);
  int c[4];
  unsigned long long key[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float r2 = 0.0f;
    c[j] = cone_of(a, st, pt[j], &r2);
    key[j] = cone_key(r2, i0 + j);
  }
  unsigned long long cur[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) cur[j] = (a.filter && c[j] >= 0) ? __ldcg(a.keys + c[j]) : kEmpty;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (c[j] >= 0 && key[j] < cur[j]) atomicMin(a.keys + c[j], key[j]);
    nf += c[j] == kNonFinite;
    kept += c[j] >= 0;
  }
  if (a.item_flag)
    reinterpret_cast<int4*>(a.item_flag)[g] =
        make_int4(c[0] >= 0 ? 1 : 0, c[1] >= 0 ? 1 : 0, c[2] >= 0 ? 1 : 0, c[3] >= 0 ? 1 : 0);
}

// The block's totals of (non-finite, kept) points, stored by thread 0 at *out.
__device__ __forceinline__ void block_count2(int nf, int kept, int2* out) {
  __shared__ int s_nf, s_kept;
  if (threadIdx.x == 0) {
    s_nf = 0;
    s_kept = 0;
  }
  __syncthreads();
  nf = __reduce_add_sync(0xffffffffu, nf);
  kept = __reduce_add_sync(0xffffffffu, kept);
  if ((threadIdx.x & 31) == 0 && (nf | kept)) {
    atomicAdd(&s_nf, nf);
    atomicAdd(&s_kept, kept);
  }
  __syncthreads();
  if (threadIdx.x == 0) *out = make_int2(s_nf, s_kept);
}

// Clouds of at least this many points (16-byte aligned) take four points per
// thread (three float4 loads, the four cones' minima read together); smaller
// ones, where the launch is latency bound and the occupancy of the one-point
// instance (fewer registers) pays more, one.
constexpr int64_t kPartVecMin = 4000000;
constexpr int kPartBlocksPerSm = 16;


// kGroups: four points per thread (launched for clouds of at least
// kPartVecMin points whose buffers are 16-byte aligned), else one.
template <bool kGroups>
__global__ void __launch_bounds__(256) k_partition(PartitionArgs a, const PartTables* __restrict__ t) {
  pdl_start();
  __shared__ SmemTables st;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int nf = 0, kept = 0;
  if constexpr (kGroups) {
    const int64_t ng = a.n >> 2;
    const float4* c4 = reinterpret_cast<const float4*>(a.cloud);
    float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0, v2 = v0;
    int64_t g = tid;
    // the first group is fetched while the edge tables load, each next one
    // before the current one is partitioned
    if (g < ng) {
      v0 = __ldg(c4 + 3 * g);
      v1 = __ldg(c4 + 3 * g + 1);
      v2 = __ldg(c4 + 3 * g + 2);
    }
    load_tables(*t, a.A, a.El, st);
    __syncthreads();
    for (; g < ng; g += stride) {
      const float4 w0 = v0, w1 = v1, w2 = v2;
      if (g + stride < ng) {
        v0 = __ldg(c4 + 3 * (g + stride));
        v1 = __ldg(c4 + 3 * (g + stride) + 1);
        v2 = __ldg(c4 + 3 * (g + stride) + 2);
      }
      if (a.copy_to) {
        float4* d = reinterpret_cast<float4*>(a.copy_to) + 3 * g;
        d[0] = w0;
        d[1] = w1;
        d[2] = w2;
      }
      partition_group(a, st, g, w0, w1, w2, nf, kept);
    }
    // the last n mod 4 points
    const int64_t i = 4 * ng + tid;
    if (i < a.n) {
      const float3 pt = cloud_point(a, i);
      if (a.copy_to) {
        a.copy_to[3 * i] = pt.x;
        a.copy_to[3 * i + 1] = pt.y;
        a.copy_to[3 * i + 2] = pt.z;
      }
      const int r = partition_point(a, st, i, pt);
      nf += r == 0;
      kept += r == 2;
    }
  } else {
    int64_t i = tid;
    // the first point is fetched while the edge tables load
    float3 pt = i < a.n ? cloud_point(a, i) : make_float3(0.f, 0.f, 0.f);
    load_tables(*t, a.A, a.El, st);
    __syncthreads();
    for (; i < a.n; i += stride) {
      if (a.copy_to) {
        a.copy_to[3 * i] = pt.x;
        a.copy_to[3 * i + 1] = pt.y;
        a.copy_to[3 * i + 2] = pt.z;
      }
      const int r = partition_point(a, st, i, pt);
      nf += r == 0;
      kept += r == 2;
      if (i + stride < a.n) pt = cloud_point(a, i + stride);
    }
  }
  if (a.counts) block_count2(nf, kept, a.counts + blockIdx.x);
}

// ---------------------------------------------------------------------------
// K2a / K2d: candidate lists.  For every collision point p (item i), every
// cell whose box is closer to p than `reach` gets p: the count pass adds to
// the cell's counter, the scatter pass writes the entry at start(cell) + its
// fill ticket.  An entry is either i (4 bytes; the count pass stores p at
// pts[i], and the points, far fewer than the entries, stay in L1) or p itself
// (16 bytes, one load fewer per entry read).  Either way a point carries its
// item index in w (bits of an int), so that ties between equidistant points
// are broken by item, the collision set's order, whatever the order of the
// entries within a cell, which depends on the atomics.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool cand_item(const CandArgs& a, int64_t it, float& px, float& py,
                                          float& pz) {
  int64_t i;
  if (a.raw) {
    if (!a.item_flag[it]) return false;
    i = it;
  } else {
    const unsigned long long key = a.keys[it];
    if (key == kEmpty) return false;
    i = (int64_t)(key & 0xFFFFFFFFull);
  }
  px = sub(__ldg(a.cloud + 3 * i), a.p0[0]);
  py = sub(__ldg(a.cloud + 3 * i + 1), a.p0[1]);
  pz = sub(__ldg(a.cloud + 3 * i + 2), a.p0[2]);
  return true;
}

// Squared distance from v to the interval [lo, lo + h].
__device__ __forceinline__ float gap2(float v, float lo, float h) {
  const float d = fmaxf(fmaxf(lo - v, v - (lo + h)), 0.0f);
  return d * d;
}

// One warp per collision item; its lanes share the item's block of cells.
// kIdx: the entries are item indices (a single planner's step), else points
// (batched steps); the form is fixed per launch, so it is a template argument.
template <bool kScatter, bool kIdx>
__device__ __forceinline__ void cand_task(const CandArgs& a, int64_t it, int lane) {
  const GridGeom& g = a.grid;
  const float r2 = g.reach * g.reach;
  float px, py, pz;
  if (!cand_item(a, it, px, py, pz)) return;  // uniform across the warp
  if (kScatter && a.reset_keys && !a.raw) {
    // the scatter pass is the key's last reader in a step
    __syncwarp();
    if (lane == 0) a.reset_keys[it] = kEmpty;
  }
  if constexpr (!kScatter && kIdx) {
    if (lane == 0) a.pts[it] = make_float4(px, py, pz, __int_as_float((int)it));
  }
  const int x0 = max(__float2int_rd((px - g.reach - g.origin) * g.inv_h), 0);
  const int x1 = min(__float2int_rd((px + g.reach - g.origin) * g.inv_h), g.G - 1);
  const int y0 = max(__float2int_rd((py - g.reach - g.origin) * g.inv_h), 0);
  const int y1 = min(__float2int_rd((py + g.reach - g.origin) * g.inv_h), g.G - 1);
  const int z0 = max(__float2int_rd((pz - g.reach - g.origin) * g.inv_h), 0);
  const int z1 = min(__float2int_rd((pz + g.reach - g.origin) * g.inv_h), g.G - 1);
  const int nx = x1 - x0 + 1, ny = y1 - y0 + 1, nz = z1 - z0 + 1;
  if (nx <= 0 || ny <= 0 || nz <= 0) return;
  const int ncand = nx * ny * nz;
  // the cell of block offset o if the point is within reach of its box, else -1
  auto cell_of = [&](int o) {
    if (o >= ncand) return -1;
    const int x = x0 + o % nx, y = y0 + (o / nx) % ny, z = z0 + o / (nx * ny);
    const float d2 = gap2(px, g.origin + x * g.h, g.h) + gap2(py, g.origin + y * g.h, g.h) +
                     gap2(pz, g.origin + z * g.h, g.h);
    if (d2 >= r2) return -1;
    const int c = (z * g.G + y) * g.G + x;
    return AERO_CHECK(c >= 0 && c < g.G * g.G * g.G, kChkGridCell) ? c : -1;
  };
  if constexpr (!kScatter) {
    for (int o = lane; o < ncand; o += 32) {
      const int c = cell_of(o);
      if (c >= 0) atomicAdd(a.count + c, 1);
    }
  } else {
    // kB cells per lane at a time: their list offsets and fill tickets are all
    // requested before the first is used, so the round trips overlap
    constexpr int kB = 4;
    for (int o0 = lane; o0 < ncand; o0 += 32 * kB) {
      int c[kB], base[kB], ticket[kB];
#pragma unroll
      for (int b = 0; b < kB; ++b) c[b] = cell_of(o0 + 32 * b);
#pragma unroll
      for (int b = 0; b < kB; ++b)
        if (c[b] >= 0) {
          base[b] = a.local[c[b]] + a.tile_off[c[b] >> kScanTileShift];
          ticket[b] = atomicAdd(a.fill + c[b], 1);
        }
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        if (c[b] < 0) continue;
        const int pos = base[b] + ticket[b];
        if (pos < g.cap) {
          if constexpr (kIdx)
            a.cand[pos] = (uint32_t)it;
          else
            a.cand4[pos] = make_float4(px, py, pz, __int_as_float((int)it));
        } else {
          atomicOr(a.status, 2);
        }
      }
    }
  }
}

// `block` / `nblocks`: this block's index within the blocks given to the pass.
template <bool kScatter>
__device__ void cand_pass(const CandArgs& a, int block, int nblocks) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)nblocks * (blockDim.x >> 5);
  for (int64_t it = ((int64_t)block * blockDim.x + threadIdx.x) >> 5; it < a.n_items; it += warps)
    cand_task<kScatter, true>(a, it, lane);
}

// ---------------------------------------------------------------------------
// K2b: tile-local exclusive scan of the counts (4096 cells per block); the
// counts are cleared for reuse as fill cursors by the scatter pass.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;

__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  total = s_warp[(blockDim.x >> 5) - 1];
  const int r = (wid > 0 ? s_warp[wid - 1] : 0) + incl - v;
  __syncthreads();
  return r;
}

__device__ void scan_tile_offsets(const int* tile_sum, int* tile_off, int ntiles) {
  __shared__ int s_warp[32];
  __shared__ int s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < ntiles; base += kScanThreads) {
    const int i = base + threadIdx.x;
    const int v = i < ntiles ? __ldcg(tile_sum + i) : 0;
    int total;
    const int r = block_exclusive_scan(v, s_warp, total);
    if (i < ntiles) tile_off[i] = s_carry + r;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_off[ntiles] = s_carry;
}

// K2b: tile-local exclusive scan of the counts (4096 cells per block, the
// counts cleared for reuse as fill cursors by the scatter); the last block to
// finish scans the tile totals into tile offsets.
// One tile: writes the tile-local prefix and the tile total; returns whether
// this block finished the last tile of the grid (then it has scanned the tile
// totals into tile offsets).
__device__ bool scan_tile(int* count, int* fill, int* local, int* tile_sum, int* tile_off,
                          int ncells, int ntiles, int tile, unsigned int* counter) {
  __shared__ int s_warp[32];
  __shared__ bool s_last;
  const int i0 = tile * kScanTile + 4 * threadIdx.x;  // a multiple of 4: int4-aligned
  const bool full = i0 + 3 < ncells;
  int v[4];
  if (full) {
    const int4 c4 = *reinterpret_cast<const int4*>(count + i0);
    v[0] = c4.x; v[1] = c4.y; v[2] = c4.z; v[3] = c4.w;
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = (i0 + u < ncells) ? count[i0 + u] : 0;
  }
  int total;
  const int run = block_exclusive_scan(v[0] + v[1] + v[2] + v[3], s_warp, total);
  // counts and fill cursors are left at zero: the next step counts from zero
  const int r1 = run + v[0], r2 = r1 + v[1], r3 = r2 + v[2];
  if (full) {
    *reinterpret_cast<int4*>(local + i0) = make_int4(run, r1, r2, r3);
    *reinterpret_cast<int4*>(count + i0) = make_int4(0, 0, 0, 0);
    *reinterpret_cast<int4*>(fill + i0) = make_int4(0, 0, 0, 0);
  } else {
    const int r[4] = {run, r1, r2, r3};
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u < ncells) {
        local[i0 + u] = r[u];
        count[i0 + u] = 0;
        fill[i0 + u] = 0;
      }
  }
  // the last block reads only the tile totals: only their writer fences.
  // Without a ticket the tile offsets are left to the next launch.
  if (threadIdx.x == 0) {
    tile_sum[tile] = total;
    if (counter) {
      __threadfence();
      s_last = atomicAdd(counter, 1u) == (unsigned)(ntiles - 1);
    } else {
      s_last = false;
    }
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  if (threadIdx.x == 0) *counter = 0u;
  scan_tile_offsets(tile_sum, tile_off, ntiles);
  return true;
}



// Coarse argmax of one coarse cell (Eq. safe-vector) by one warp: larger r,
// then nearer the coarse centre, then lower fine index; empty cones count as
// r_max.  Each lane takes a strided share of the pooled cones, then the warp
// reduces (r key, centre distance, fine index).
__device__ __forceinline__ void coarse_cell(const GuideArgs& a, int cc, int lane) {
  const uint32_t empty_bits = __float_as_uint(a.rmax2);
  const int npool = a.Pa * a.Pe;
  const int I = cc % a.Ac, J = cc / a.Ac;
  uint32_t bkey = 0;
  int bdist = 0x7fffffff, best = 0x7fffffff;
  for (int m = lane; m < npool; m += 32) {
    const int q = m % a.Pa, b = m / a.Pa;
    const int c = (J * a.Pe + b) * a.A + I * a.Pa + q;
    const unsigned long long k = a.keys[c];
    const uint32_t rk = k == kEmpty ? empty_bits : (uint32_t)(k >> 32);
    const int dist = abs(2 * q + 1 - a.Pa) + abs(2 * b + 1 - a.Pe);
    if (rk > bkey || (rk == bkey && (dist < bdist || (dist == bdist && c < best)))) {
      best = c;
      bkey = rk;
      bdist = dist;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t ok = __shfl_xor_sync(0xffffffffu, bkey, o);
    const int od = __shfl_xor_sync(0xffffffffu, bdist, o);
    const int oc = __shfl_xor_sync(0xffffffffu, best, o);
    if (ok > bkey || (ok == bkey && (od < bdist || (od == bdist && oc < best)))) {
      best = oc;
      bkey = ok;
      bdist = od;
    }
  }
  if (lane == 0) a.coarse_win[cc] = best;
}

// Goal cone, anchors and guides of one planner by one block, after every
// coarse winner is written; `st` holds the edge tables.
__device__ void guides_block(const GuideArgs& a, const SmemTables& st) {
  __shared__ float s_coef[kMaxE][3][6];
  __shared__ int s_goal;
  // goal cone and the M_h x M_v anchor cells around it (Sec. IV-B.1)
  if (threadIdx.x == 0) {
    float b[3];
    to_body(a.R, a.goal_rel[0], a.goal_rel[1], a.goal_rel[2], b);
    const float rho = __fsqrt_rn(add(mul(b[0], b[0]), mul(b[1], b[1])));
    s_goal = el_bin(st.ce, st.se, a.El, b[2], rho) * a.A + az_bin(st.ca, st.sa, a.A, b[0], b[1]);
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
    // direction of the winning cone's centre (Eq. unit direction); the azimuth
    // in units of pi is -1 + (2i + 1) / A
    const int w = __ldcg(a.coarse_win + cc);
    const int i = w % a.A, j = w / a.A;
    const float be = a.el_lo + (j + 0.5f) * ((a.el_hi - a.el_lo) / a.El);
    float sa, ca, sb, cb;
    sincospif(-1.0f + (float)(2 * i + 1) / (float)a.A, &sa, &ca);
    sincosf(be, &sb, &cb);
    const float db[3] = {cb * ca, cb * sa, sb};
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

// K2a + K3a: the coarse argmax (one warp per coarse cell; it needs only the
// keys) in the first blocks, dispatched first; the count pass of the candidate
// lists in the remaining blocks.  The goal cone, anchors and guides follow in
// the scan launch, once every coarse winner is written.
__global__ void __launch_bounds__(256) k_grid_count(CandArgs ca, GuideArgs ga, int count_blocks) {
  pdl_start();
  const int ncb = (int)gridDim.x - count_blocks;
  if ((int)blockIdx.x < ncb) {
    const int ncoarse = ga.Ac * ga.Ec;
    const int lane = threadIdx.x & 31, nwarp = ncb * (blockDim.x >> 5);
    for (int cc = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); cc < ncoarse; cc += nwarp)
      coarse_cell(ga, cc, lane);
  } else {
    cand_pass<false>(ca, blockIdx.x - ncb, count_blocks);
  }
}

// K2b + K3b: the tile scans in blocks [0, ntiles); block ntiles computes the
// goal cone, anchors and guides (Sec. IV-B) from the coarse winners of the
// count launch.
__global__ void __launch_bounds__(kScanThreads) k_grid_scan(int* count, int* fill, int* local,
                                                            int* tile_sum, int* tile_off, int ncells,
                                                            int ntiles, unsigned int* counter,
                                                            GuideArgs ga,
                                                            const PartTables* __restrict__ t) {
  pdl_start();
  if ((int)blockIdx.x < ntiles) {
    scan_tile(count, fill, local, tile_sum, tile_off, ncells, ntiles, blockIdx.x, counter);
    return;
  }
  __shared__ SmemTables st;
  load_tables(*t, ga.A, ga.El, st);
  __syncthreads();
  guides_block(ga, st);
}

// {first entry, count} of cell c from the scanned counts.
__device__ __forceinline__ void range_cell(const int* local, const int* tile_off, int cap,
                                           int2* range, int c) {
  const int s = min(local[c] + tile_off[c >> kScanTileShift], cap);
  const int e = min(local[c + 1] + tile_off[(c + 1) >> kScanTileShift], cap);
  range[c] = AERO_CHECK(s >= 0 && e >= s, kChkRange) ? make_int2(s, e - s) : make_int2(0, 0);
}

// K2c: the scatter pass and, in the remaining blocks, the {start, count} of
// every cell (which needs only the scan).  Every block first turns the scan's
// tile totals into tile offsets in shared memory (at most kMaxTiles of them);
// block 0 also stores them.
__global__ void __launch_bounds__(256) k_grid_scatter(CandArgs ca, int scatter_blocks,
                                                      int2* __restrict__ range, int ncells,
                                                      const int* tile_sum, int* tile_off,
                                                      int ntiles) {
  pdl_start();
  __shared__ int s_off[kMaxTiles + 1];
  __shared__ int s_warp[32];
  __shared__ int s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < ntiles; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < ntiles ? __ldg(tile_sum + i) : 0;
    int total;
    const int r = block_exclusive_scan(v, s_warp, total);
    if (i < ntiles) s_off[i] = s_carry + r;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) s_off[ntiles] = s_carry;
  __syncthreads();
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i <= ntiles; i += blockDim.x) tile_off[i] = s_off[i];
  if ((int)blockIdx.x < scatter_blocks) {
    CandArgs a = ca;
    a.tile_off = s_off;
    cand_pass<true>(a, blockIdx.x, scatter_blocks);
    return;
  }
  const int nrb = (int)gridDim.x - scatter_blocks;
  for (int c = (blockIdx.x - scatter_blocks) * blockDim.x + threadIdx.x; c < ncells;
       c += nrb * blockDim.x)
    range_cell(ca.local, s_off, ca.grid.cap, range, c);
}

__global__ void k_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3,
                         int64_t n, uint4* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = philox4x32_10(make_uint4((uint32_t)i, c1, c2, c3), k0, k1);
}

// ---------------------------------------------------------------------------
// Batched launches: the same stages over the units of many planners.  Work
// that depends on the planner (tables, arguments) is reloaded into shared
// memory only when a block moves on to another planner.
// ---------------------------------------------------------------------------
// Contiguous share [t, t1) of `total` tasks for worker w of nw.
__device__ __forceinline__ void share_of(long long total, long long w, long long nw, long long& t,
                                         long long& t1) {
  const long long per = (total + nw - 1) / nw;
  t = w * per;
  t1 = min(total, t + per);
}

__global__ void __launch_bounds__(256) k_b_partition(BatchView v) {
  pdl_start();
  __shared__ long long s_pre[kBatchMax + 1];
  __shared__ SmemTables st;
  __shared__ PartitionArgs s_pa;
  const int n = v.n;
  load_prefix(s_pre, v.pre + kPrePoints * (n + 1), n);
  __syncthreads();
  long long u, u1;
  share_of(s_pre[n], blockIdx.x, gridDim.x, u, u1);
  int cur = -1;
  for (; u < u1; ++u) {
    const int it = find_unit(s_pre, n, u);
    if (it != cur) {
      __syncthreads();  // the previous planner's tables are no longer read
      const BatchItem* bi = v.items + it;
      block_copy(&s_pa, &bi->pa);
      load_tables(*bi->tab, bi->pa.A, bi->pa.El, st);
      __syncthreads();
      cur = it;
    }
    const int64_t chunk = u - s_pre[it], base = chunk * kPartChunk;
    int nf = 0, kept = 0;
    for (int r = threadIdx.x; r < kPartChunk; r += blockDim.x)
      if (base + r < s_pa.n) {
        const int c = partition_point(s_pa, st, base + r, cloud_point(s_pa, base + r));
        nf += c == 0;
        kept += c == 2;
      }
    if (s_pa.counts) block_count2(nf, kept, s_pa.counts + chunk);
  }
}

// Collision-item tasks (one warp each) in chunks of kTaskChunk consecutive
// tasks, chunks dealt to the warps round robin (balances dense and empty
// stretches of the fine partition).  kScatter: the scatter pass, else the count.
constexpr int kTaskChunk = 4;

template <bool kScatter>
__device__ __forceinline__ void cand_tasks(const BatchView& v, const long long* s_pi, int n,
                                           long long w, long long nw, int lane) {
  const long long ni = s_pi[n];
  const long long nch = (ni + kTaskChunk - 1) / kTaskChunk;
  for (long long q = w; q < nch; q += nw) {
    long long t = q * kTaskChunk;
    const long long t1 = min(ni, t + kTaskChunk);
    int it = find_unit(s_pi, n, t);
    CandArgs a = v.items[it].ca;
    for (; t < t1; ++t) {
      if (t >= s_pi[it + 1]) {
        while (t >= s_pi[it + 1]) ++it;
        a = v.items[it].ca;
      }
      cand_task<kScatter, false>(a, t - s_pi[it], lane);
    }
  }
}

// Count tasks, then the coarse cells (one warp each).
__global__ void __launch_bounds__(256) k_b_count(BatchView v) {
  pdl_start();
  __shared__ long long s_pi[kBatchMax + 1], s_pc[kBatchMax + 1];
  const int n = v.n;
  load_prefix(s_pi, v.pre + kPreItems * (n + 1), n);
  load_prefix(s_pc, v.pre + kPreCoarse * (n + 1), n);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  cand_tasks<false>(v, s_pi, n, w, nw, lane);
  for (long long c = w; c < s_pc[n]; c += nw) {
    const int it = find_unit(s_pc, n, c);
    coarse_cell(v.items[it].ga, (int)(c - s_pc[it]), lane);
  }
}

// Units [0, n): goal cone, anchors and guides of planner u; then the scan tiles.
__global__ void __launch_bounds__(kScanThreads) k_b_scan(BatchView v) {
  pdl_start();
  __shared__ long long s_pre[kBatchMax + 1];
  __shared__ SmemTables st;
  __shared__ GuideArgs s_ga;
  const int n = v.n;
  load_prefix(s_pre, v.pre + kPreTiles * (n + 1), n);
  __syncthreads();
  const long long total = n + s_pre[n];
  for (long long u = blockIdx.x; u < total; u += gridDim.x) {
    __syncthreads();
    if (u < n) {
      const BatchItem* bi = v.items + u;
      block_copy(&s_ga, &bi->ga);
      load_tables(*bi->tab, bi->ga.A, bi->ga.El, st);
      __syncthreads();
      guides_block(s_ga, st);
    } else {
      const long long t = u - n;
      const int it = find_unit(s_pre, n, t);
      const BatchItem* bi = v.items + it;
      scan_tile(bi->count, bi->fill, bi->local, bi->tile_sum, bi->tile_off, bi->gcells + 1,
                bi->ntiles, (int)(t - s_pre[it]), bi->scan_counter);
    }
  }
}

// Scatter tasks (emptying the keys they read); then the cell ranges and the
// keys of planners whose collision set is every kept point (read only by the
// coarse pass, so emptied here).
__global__ void __launch_bounds__(256) k_b_scatter(BatchView v) {
  pdl_start();
  __shared__ long long s_pi[kBatchMax + 1], s_pc[kBatchMax + 1];
  const int n = v.n;
  load_prefix(s_pi, v.pre + kPreItems * (n + 1), n);
  load_prefix(s_pc, v.pre + kPreCells * (n + 1), n);
  __syncthreads();
  cand_tasks<true>(v, s_pi, n, ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                   (long long)gridDim.x * (blockDim.x >> 5), threadIdx.x & 31);
  const long long total = s_pc[n];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c0 = (long long)blockIdx.x * blockDim.x; c0 < total; c0 += stride) {
    const long long c = c0 + threadIdx.x;
    if (c >= total) break;
    int it = find_unit(s_pc, n, c0);
    while (c >= s_pc[it + 1]) ++it;
    const BatchItem* bi = v.items + it;
    const long long l = c - s_pc[it];
    if (l < bi->gcells)
      range_cell(bi->local, bi->tile_off, bi->ca.grid.cap, bi->range, (int)l);
    else
      bi->keys[l - bi->gcells] = kEmpty;
  }
}

int blocks_for(int64_t n, int threads, int cap) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

}  // namespace

int partition_blocks(int64_t n) {
  const int cap = kPartBlocksPerSm * device_sms();
  const int64_t threads = n >= kPartVecMin ? (n + 3) / 4 : n;  // four points per thread
  return n > 0 ? blocks_for(threads, 256, cap < kPartBlocksMax ? cap : kPartBlocksMax) : 0;
}

cudaError_t launch_partition(const PartitionArgs& a, const PartTables* t, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  const uintptr_t bits = reinterpret_cast<uintptr_t>(a.cloud) |
                         reinterpret_cast<uintptr_t>(a.copy_to) |
                         reinterpret_cast<uintptr_t>(a.item_flag);
  if (a.n >= kPartVecMin && (bits & 15u) == 0)
    return launch_k(k_partition<true>, dim3(partition_blocks(a.n)), dim3(256), s, true, a, t);
  return launch_k(k_partition<false>, dim3(partition_blocks(a.n)), dim3(256), s, true, a, t);
}

cudaError_t launch_grid_count(const CandArgs& ca, const GuideArgs& ga, cudaStream_t s) {
  // one warp per collision item up to four blocks per SM, then items per warp
  const int count_blocks = ca.n_items > 0 ? blocks_for(ca.n_items * 32, 256, 4 * device_sms()) : 0;
  const int coarse_blocks = (ga.Ac * ga.Ec + 7) / 8;  // 8 warps per block
  return launch_k(k_grid_count, dim3(count_blocks + coarse_blocks), dim3(256), s, true, ca, ga,
                  count_blocks);
}

cudaError_t launch_grid_scan(int* count, int* fill, int* local, int* tile_sum, int* tile_off,
                             int ncells, int ntiles, unsigned int* counter, const GuideArgs& ga,
                             const PartTables* t, cudaStream_t s) {
  return launch_k(k_grid_scan, dim3(ntiles + 1), dim3(kScanThreads), s, true, count, fill, local,
                  tile_sum, tile_off, ncells, ntiles, counter, ga, t);
}

cudaError_t launch_grid_scatter(const CandArgs& ca, int2* range, int ncells, const int* tile_sum,
                                int* tile_off, int ntiles, cudaStream_t s) {
  const int sms = device_sms();
  const int scatter_blocks = ca.n_items > 0 ? blocks_for(ca.n_items * 32, 256, 4 * sms) : 0;
  const int range_blocks = blocks_for(ncells, 256, 2 * sms);
  return launch_k(k_grid_scatter, dim3(scatter_blocks + range_blocks), dim3(256), s, true, ca,
                  scatter_blocks, range, ncells, tile_sum, tile_off, ntiles);
}

cudaError_t batch_grid_occupancy(int out[4]) {
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out + 0, k_b_partition, 256, 0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out + 1, k_b_count, 256, 0);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out + 2, k_b_scan, kScanThreads, 0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out + 3, k_b_scatter, 256, 0);
  for (int i = 0; i < 4; ++i)
    if (out[i] < 1) out[i] = 1;
  return e;
}

cudaError_t launch_batch_partition(const BatchView& v, int blocks, cudaStream_t s) {
  k_b_partition<<<blocks, 256, 0, s>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_batch_count(const BatchView& v, int blocks, cudaStream_t s) {
  return launch_k(k_b_count, dim3(blocks), dim3(256), s, true, v);
}

cudaError_t launch_batch_scan(const BatchView& v, int blocks, cudaStream_t s) {
  return launch_k(k_b_scan, dim3(blocks), dim3(kScanThreads), s, true, v);
}

cudaError_t launch_batch_scatter(const BatchView& v, int blocks, cudaStream_t s) {
  return launch_k(k_b_scatter, dim3(blocks), dim3(256), s, true, v);
}

cudaError_t launch_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3,
                          int64_t n, uint32_t* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_philox<<<blocks_for(n, 256, 16 * device_sms()), 256, 0, s>>>(k0, k1, c1, c2, c3, n,
                                                          reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

cudaError_t raise_check_partition(int bits) {
#ifdef AERO_CHECKED
  int w = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&w, g_check_word, sizeof(int));
  w |= bits;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_check_word, &w, sizeof(int));
  return e;
#else
  (void)bits;
  return cudaErrorNotSupported;
#endif
}

cudaError_t check_word_partition(int* out, bool clear) {
#ifdef AERO_CHECKED
  cudaError_t e = cudaMemcpyFromSymbol(out, g_check_word, sizeof(int));
  const int zero = 0;
  if (e == cudaSuccess && clear) e = cudaMemcpyToSymbol(g_check_word, &zero, sizeof(int));
  return e;
#else
  (void)clear;
  *out = 0;
  return cudaSuccess;
#endif
}

}  // namespace aero

