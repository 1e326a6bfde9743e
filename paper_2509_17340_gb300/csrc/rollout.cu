// Stage I of the MPPI ensemble (Sec. III-B, Sec. IV-C): one CTA of 128 threads
// (one warp-group) rolls out 128 samples of one instance.  Per sample and
// step: Philox noise in registers, clamp, RK4, the S(1) cost terms with the
// nearest-point distance from the collision grid.  Then per CTA: the minimum
// cost rho_b, eta_b = sum exp(-(S - rho_b)/lambda) and W_b[j][c] = sum
// exp(-(S - rho_b)/lambda) du[j][c], the perturbations regenerated from the
// counter-based generator for the samples whose weight is not zero (nothing
// is stored per sample and step).  The update kernel merges the per-CTA
// partials (log-sum-exp rescaling by the global minimum), updates the nominal
// (Eq. mppi_update_simplified), and on the last iteration runs Stage II and
// the selection.
#include <atomic>
#include <cfloat>
#include <cstdint>

#include "adjoint.cuh"
#include "device.cuh"
#include "internal.h"

namespace aero {
namespace {

constexpr int NT = kRolloutThreads;

__device__ __forceinline__ float4 clamp4(float4 u, float4 lo, float4 hi) {
  return make_float4(fminf(fmaxf(u.x, lo.x), hi.x), fminf(fmaxf(u.y, lo.y), hi.y),
                     fminf(fmaxf(u.z, lo.z), hi.z), fminf(fmaxf(u.w, lo.w), hi.w));
}

// Plain binary32 accumulation of the per-step costs: T <= 128 positive
// terms, relative error below T * 2^-24 (under 1e-5, a tenth of the cost
// tolerance), with one dependent addition per step instead of four.
struct CostSum {
  float s = 0.0f;
  __device__ __forceinline__ void add(float v) { s += v; }
};

// Samples [b * kNT, (b + 1) * kNT) of instance e, one per thread (kNT: the
// CTA's threads, a multiple of 32); ctr3: the noise counter's last word,
// (step_id << 8) | iteration.  kIdx: the grid's candidate entries are item
// indices (a single planner's step), else points (batched steps).
// kWarpLists: long candidate lists scanned by the whole warp (warp_split_min,
// lists longer than a.list_thr), for the every-point collision set; the
// short lists of P_f keep the per-lane scan, compiled without that path.
template <bool kIdx, int kNT = NT, bool kWarpLists = false, bool kRestForm = kIdx && !kWarpLists>
__device__ __forceinline__ void rollout_unit(const RolloutArgs& a, int e, int b, uint32_t ctr3) {
  constexpr int kNW = kNT / 32;
  constexpr int kSW = kNT > kMaxT ? kNT : kMaxT;
  __shared__ float4 s_un[kMaxT];
  __shared__ float s_gd[kMaxT * 3];
  __shared__ float s_red[kNW];
  __shared__ int s_nz[kNW];      // weighted samples per warp
  __shared__ int s_lk[kNT];      // the CTA's samples of non-zero weight, in sample order
  __shared__ float s_lw[kNT];    // and their weights
  __shared__ float4 s_w[kSW];    // W_b partial sums [replica][step]

  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int T = a.T;
  for (int i = tid; i < T; i += kNT) s_un[i] = reinterpret_cast<const float4*>(a.u_nom)[e * T + i];
  for (int i = tid; i < 3 * T; i += kNT) s_gd[i] = a.guides[e * T * 3 + i];
  __syncthreads();

  const int k = b * kNT + tid;
  const bool active = k < a.K;
  const CostParams& cp = a.cost;
  const float dmax2 = cp.d_max * cp.d_max;
  // kRestForm: the at-rest goal term compiled in.  Left out of the batched
  // passes built for 80 registers (the test's registers made them spill) and
  // of the every-point instance (17% slower with it)
  const bool at_rest = kRestForm && goal_at_rest(cp);
  const int dbg = (active && k < a.dbg_D) ? (e * a.dbg_D + k) : -1;
  const float4 sigma = make_float4(a.sigma[0], a.sigma[1], a.sigma[2], a.sigma[3]);
  const float4 umin = make_float4(a.umin[0], a.umin[1], a.umin[2], a.umin[3]);
  const float4 umax = make_float4(a.umax[0], a.umax[1], a.umax[2], a.umax[3]);

  State x;
#pragma unroll
  for (int i = 0; i < 3; ++i) x.p[i] = a.x0[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) x.q[i] = a.x0[3 + i];
#pragma unroll
  for (int i = 0; i < 3; ++i) x.v[i] = a.x0[7 + i];
  if (dbg >= 0) {
    float* X = a.dbg_x + (size_t)dbg * (T + 1) * 10;
    for (int i = 0; i < 10; ++i) X[i] = a.x0[i];
  }

  CostSum S;
  // step j's control: prefetched noise, clamp, J_ctrl's
  // terms Q_c |u_j|^2 (j <= T-2) and Q_cd |u_j - u_{j-1}|^2 (1 <= j <= T-2)
  // a single planner's arguments are kernel parameters: the Philox round keys
  // are read as constant operands; the batched kernels' are in shared memory,
  // where recomputing the schedule is cheaper than reading it
  auto noise = [&](uint32_t kk, uint32_t j) {
    if constexpr (kIdx)
      return noise_delta_rk(kk, j, e, ctr3, a.rk, sigma);
    else
      return noise_delta(kk, j, e, ctr3, a.key0, a.key1, sigma);
  };
  float4 d_next = noise(k, 0);
  float4 un_next = s_un[0];
  float4 u_prev = make_float4(0.f, 0.f, 0.f, 0.f);
  auto control = [&](int j, float& c_ctrl) -> float4 {
    const float4 un = un_next, d = d_next;
    if (j + 1 < T) {
      d_next = noise(k, j + 1);
      un_next = s_un[j + 1];
    }
    const float4 u = clamp4(make_float4(un.x + d.x, un.y + d.y, un.z + d.z, un.w + d.w), umin, umax);
    c_ctrl = 0.0f;
    if (j <= T - 2) {
      c_ctrl = cp.Q_c * (u.x * u.x + u.y * u.y + u.z * u.z + u.w * u.w);
      if (j >= 1) {
        const float ax = u.x - u_prev.x, ay = u.y - u_prev.y, az = u.z - u_prev.z, aw = u.w - u_prev.w;
        c_ctrl += cp.Q_cd * (ax * ax + ay * ay + az * az + aw * aw);
      }
    }
    u_prev = u;
    return u;
  };

  // x holds x_j; its candidate range was loaded one iteration earlier, so the
  // load overlaps the next RK4 step (with one lane per sample the GPU holds
  // enough warps to hide the candidate loads themselves)
  float c_ctrl;
  float4 u_j = control(0, c_ctrl);
  rk4_step(x, u_j, a.dyn);
  int2 range = cell_range(x.p[0], x.p[1], x.p[2], a.grid);
  // a single planner: two steps per iteration, so that the state carried
  // from one step to the next alternates between two register sets instead
  // of being copied (the batched kernels, with their arguments in shared
  // memory, would spill)
  constexpr int kUnroll = kIdx ? 2 : 1;
#pragma unroll kUnroll
  for (int j = 1; j <= T; ++j) {
    const int2 range_j = range;
    State xn = x;
    float c_next = 0.0f;
    float4 u_next = u_j;
    if (j < T) {
      u_next = control(j, c_next);
      rk4_step(xn, u_next, a.dyn);
      range = cell_range(xn.p[0], xn.p[1], xn.p[2], a.grid);
    }
    // (a runtime test in the warp-list instance too: compiled with both scans
    // that instance ran 2.85 instead of 3.33 ms at 200,000 kept points)
    float d2 = dmax2;
    if (kWarpLists && a.list_thr > 0) {
      d2 = warp_split_min<kIdx>(a.grid, active ? range_j : make_int2(0, 0), x.p[0], x.p[1], x.p[2],
                                dmax2, a.list_thr);
    } else {
      for (int i = 0; i < range_j.y; ++i)
        d2 = fminf(d2, dist2_to(grid_point_of<kIdx>(a.grid, range_j.x + i), x.p[0], x.p[1], x.p[2]));
    }
    // state terms at x_j against the guide at t = j dt
    const float gx = s_gd[3 * (j - 1)], gy = s_gd[3 * (j - 1) + 1], gz = s_gd[3 * (j - 1) + 2];
    float c = c_ctrl;
    c += cp.Q_track * norm3f(x.p[0] - gx, x.p[1] - gy, x.p[2] - gz);
    c += cp.Q_vnorm * (x.v[0] * x.v[0] + x.v[1] * x.v[1] + x.v[2] * x.v[2]);
    c += goal_term(x, cp, at_rest);
    c += jcol_from_d2(d2, cp, dmax2);
    S.add(c);
    if (dbg >= 0) {
      reinterpret_cast<float4*>(a.dbg_u)[(size_t)dbg * T + j - 1] = u_j;
      float* X = a.dbg_x + ((size_t)dbg * (T + 1) + j) * 10;
      for (int i = 0; i < 3; ++i) X[i] = x.p[i];
      for (int i = 0; i < 4; ++i) X[3 + i] = x.q[i];
      for (int i = 0; i < 3; ++i) X[7 + i] = x.v[i];
      a.dbg_d[(size_t)dbg * T + j - 1] = d2 < dmax2 ? sqrtf(d2) : INFINITY;
    }
    x = xn;
    u_j = u_next;
    c_ctrl = c_next;
  }
  const float Sk = S.s;
  if (active) a.sample_costs[(size_t)e * a.K + k] = Sk;

  // rho_b = min S over the CTA
  float m = warp_min(active ? Sk : INFINITY);
  if (lane == 0) s_red[wid] = m;
  __syncthreads();
  float rho = s_red[0];
#pragma unroll
  for (int w = 1; w < kNW; ++w) rho = fminf(rho, s_red[w]);
  __syncthreads();
  const float wk = active ? expf((rho - Sk) * a.inv_lambda) : 0.0f;
  const float ws = warp_sum(wk);
  // the samples of non-zero weight, listed in sample order: a sample whose
  // weight underflows to zero adds exactly nothing to W_b, so only the listed
  // ones regenerate their perturbations (with lambda = 1, a sample whose cost
  // exceeds the CTA's best by more than about 104 is not listed)
  const unsigned nzb = __ballot_sync(0xffffffffu, wk > 0.0f);
  if (lane == 0) {
    s_red[wid] = ws;
    s_nz[wid] = __popc(nzb);
  }
  __syncthreads();
  int nz = 0, before = 0;
#pragma unroll
  for (int w = 0; w < kNW; ++w) {
    before += w < wid ? s_nz[w] : 0;
    nz += s_nz[w];
  }
  if (wk > 0.0f) {
    const int pos = before + __popc(nzb & ((1u << lane) - 1u));
    s_lk[pos] = k;
    s_lw[pos] = wk;
  }
  __syncthreads();
  // W_b[j] = sum over the listed samples of w_k du_k[j]: slot t takes step
  // j = t mod T and the listed samples i = r, r + R, ... of replica r = t / T
  // (R = max(1, kNT / T) replicas; the CTA's threads take the R T slots in
  // turn; a fixed order, so the sums are reproducible)
  const int R = T <= kNT ? kNT / T : 1;
  for (int slot = tid; slot < R * T; slot += kNT) {
    const int j = slot % T, r = slot / T;
    const float4 un = s_un[j];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = r; i < nz; i += R) {
      const float w = s_lw[i];
      const float4 d = noise(s_lk[i], j);
      const float4 u = clamp4(make_float4(un.x + d.x, un.y + d.y, un.z + d.z, un.w + d.w), umin, umax);
      acc.x += w * (u.x - un.x);
      acc.y += w * (u.y - un.y);
      acc.z += w * (u.z - un.z);
      acc.w += w * (u.w - un.w);
    }
    s_w[slot] = acc;
  }
  __syncthreads();
  float* out = a.partials + ((size_t)e * a.nb + b) * (4 + 4 * T);
  if (!AERO_CHECK(b < a.nb && e < a.E, kChkPartial)) return;
  if (tid == 0) {
    float eta = 0.0f;
#pragma unroll
    for (int w = 0; w < kNW; ++w) eta += s_red[w];
    out[0] = rho;
    out[1] = eta;
  }
  for (int i = tid; i < 4 * T; i += kNT) {
    const int j = i >> 2, cc = i & 3;
    float s = 0.0f;
    for (int r = 0; r < R; ++r) s += reinterpret_cast<const float*>(&s_w[r * T + j])[cc];
    out[4 + i] = s;
  }
}

// ---------------------------------------------------------------------------
// The Stage I pass for problems too small to fill the GPU with one lane per
// sample, split into phases so that only the dynamics stays sequential: 32
// samples per CTA (eight threads per sample, one in each of its eight warps);
// the horizon in chunks of at most kChunk steps.
//   noise    the perturbations of every step, drawn by all warps before
//            the first chunk; the clamped controls stay in shared memory for
//            the whole horizon;
//   dynamics one warp (the integrator), one lane per sample, applies a
//            chunk's controls with RK4 and stores the states in one of two
//            chunk buffers;
//   queries  the seven other warps (the workers) look up the cell of every
//            (sample, step) of the chunk integrated before; the non-empty
//            candidate lists are cut into items of kItem entries and the
//            workers take the items in turn, each folding its squared
//            distances into the query's minimum with a shared-memory atomic
//            minimum (exact in any order).  A warp therefore scans items, not
//            its longest lane's list: the lists of one step's samples are
//            mostly empty, with a few of up to a hundred entries;
//   costs    the workers evaluate every (sample, step) pair's control, state
//            and collision terms.
// The integrator runs chunk c + 1 while the workers query and score chunk c
// (they meet at a named barrier; the CTA's barrier closes each round), so the
// serial chain overlaps the rest.  Then the per-CTA minimum, weights and
// weighted perturbation sums as in the one-lane pass: every warp holds the 32
// samples' costs and reduces them itself.
// ---------------------------------------------------------------------------
constexpr int ST = 256;          // threads per CTA (eight per sample)
constexpr int SW = ST / 32;      // warps per CTA
constexpr int SWK = SW - 1;      // worker warps (all but the integrator)
constexpr int kWorkBar = 1;      // the workers' named barrier
constexpr int QS = 32;           // samples per CTA
constexpr int kChunk = 20;       // steps per chunk
constexpr int kQ = (kChunk + SWK - 1) / SWK;  // queries per worker thread and chunk, at most
constexpr int kItem = 8;         // candidate entries per scan item
constexpr int kChunkQ = kChunk * QS;

// Dynamic shared memory of the split pass (bytes), for horizons up to T.
__host__ __device__ constexpr size_t split_smem_bytes(int T) {
  return 16 * (size_t)T * QS       // u: clamped controls [T][QS]
         + 16 * (size_t)T          // un: nominal [T]
         + 8 * (size_t)kChunkQ     // qrange: candidate range of each listed query
         + 80 * (size_t)kChunkQ    // xa, xb, xc: states x_{j+1} [2][kChunk][QS]
         + 4 * (size_t)kChunkQ     // d2: squared distance bits [kChunk][QS]
         + 4 * (size_t)SW * QS     // cost: partial sums [SW][QS]
         + 4 * (size_t)(kChunkQ + 2)  // qitem: first item of each listed query (+ pad)
         + 4 * (size_t)SW * 2      // scan: warp totals
         + 12 * (size_t)T          // gd: guides [T][3]
         + 2 * (size_t)kChunkQ;    // qslot: (step, sample) slot of each listed query
}

struct SplitSmem {
  float4* u;
  float4* un;
  int2* qrange;
  float4* xa;  // p, q0        [2][kChunkQ]
  float4* xb;  // q1, q2, q3, v0
  float2* xc;  // v1, v2
  int* d2;
  float* cost;
  int* qitem;
  int2* scan;
  float* gd;
  unsigned short* qslot;
};

__device__ __forceinline__ SplitSmem split_layout(unsigned char* base, int T) {
  SplitSmem m;
  m.u = reinterpret_cast<float4*>(base);
  m.un = m.u + (size_t)T * QS;
  m.qrange = reinterpret_cast<int2*>(m.un + T);
  m.xa = reinterpret_cast<float4*>(m.qrange + kChunkQ);
  m.xb = m.xa + 2 * kChunkQ;
  m.xc = reinterpret_cast<float2*>(m.xb + 2 * kChunkQ);
  m.d2 = reinterpret_cast<int*>(m.xc + 2 * kChunkQ);
  m.cost = reinterpret_cast<float*>(m.d2 + kChunkQ);
  m.qitem = reinterpret_cast<int*>(m.cost + SW * QS);
  m.scan = reinterpret_cast<int2*>(m.qitem + kChunkQ + 1 + 1);  // +1 word keeps int2 aligned
  m.gd = reinterpret_cast<float*>(m.scan + SW);
  m.qslot = reinterpret_cast<unsigned short*>(m.gd + 3 * T);
  return m;
}

__device__ __forceinline__ void rollout_split_unit(const RolloutArgs& a, int e, int b,
                                                   uint32_t ctr3) {
  extern __shared__ __align__(16) unsigned char split_smem[];
  const int T = a.T;
  const SplitSmem m = split_layout(split_smem, T);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int k = b * QS + lane;  // this thread's sample in every phase
  const bool active = k < a.K;
  const CostParams& cp = a.cost;
  const float dmax2 = cp.d_max * cp.d_max;
  const bool at_rest = goal_at_rest(cp);
  const int dbg = (active && k < a.dbg_D) ? (e * a.dbg_D + k) : -1;
  const float4 sigma = make_float4(a.sigma[0], a.sigma[1], a.sigma[2], a.sigma[3]);
  const float4 umin = make_float4(a.umin[0], a.umin[1], a.umin[2], a.umin[3]);
  const float4 umax = make_float4(a.umax[0], a.umax[1], a.umax[2], a.umax[3]);
  const int nch = (T + kChunk - 1) / kChunk;
  const int tcb = (T + nch - 1) / nch;  // steps per chunk (the last may be shorter)

  State x;
#pragma unroll
  for (int i = 0; i < 3; ++i) x.p[i] = a.x0[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) x.q[i] = a.x0[3 + i];
#pragma unroll
  for (int i = 0; i < 3; ++i) x.v[i] = a.x0[7 + i];
  // the integrator rotates with the block index, so that the integrators of
  // the CTAs sharing an SM sit on different schedulers; the workers are
  // numbered widx = 0..SWK-1 from the warp after it
  const int wint = b & (SW - 1);
  const bool integrator = wid == wint;
  const int widx = (wid + SW - 1 - wint) & (SW - 1);
  float S = 0.0f;  // every worker thread: the cost terms of its (sample, step) pairs

  // the perturbations first: they read only the kernel's parameters, so they
  // are drawn before the wait for the preceding launches (which may still
  // write the nominal, the grid and the guides); then the nominal and the
  // guides, and the clamped controls: each thread rereads only what it wrote
  for (int j = wid; j < T; j += SW)
    m.u[j * QS + lane] = noise_delta(k, j, e, ctr3, a.key0, a.key1, sigma);
  pdl_wait();
  if (dbg >= 0 && integrator) {
    float* X = a.dbg_x + (size_t)dbg * (T + 1) * 10;
    for (int i = 0; i < 10; ++i) X[i] = a.x0[i];
  }
  for (int i = tid; i < T; i += ST) m.un[i] = reinterpret_cast<const float4*>(a.u_nom)[e * T + i];
  for (int i = tid; i < 3 * T; i += ST) m.gd[i] = a.guides[e * T * 3 + i];
  __syncthreads();  // un, gd
  for (int j = wid; j < T; j += SW) {
    const float4 un = m.un[j], d = m.u[j * QS + lane];
    m.u[j * QS + lane] = clamp4(make_float4(un.x + d.x, un.y + d.y, un.z + d.z, un.w + d.w), umin, umax);
  }
  __syncthreads();

  // the integrator: the states of chunk c into buffer c & 1
  auto integrate = [&](int c) {
    const int j0 = c * tcb, tc = tcb < T - j0 ? tcb : T - j0;
    float4* xa = m.xa + (c & 1) * kChunkQ;
    float4* xb = m.xb + (c & 1) * kChunkQ;
    float2* xc = m.xc + (c & 1) * kChunkQ;
    float4 u_nx = m.u[j0 * QS + lane];
    for (int jj = 0; jj < tc; ++jj) {
      const int j = j0 + jj;
      const float4 u = u_nx;
      if (jj + 1 < tc) u_nx = m.u[(j + 1) * QS + lane];  // one step ahead
      rk4_step(x, u, a.dyn);
      xa[jj * QS + lane] = make_float4(x.p[0], x.p[1], x.p[2], x.q[0]);
      xb[jj * QS + lane] = make_float4(x.q[1], x.q[2], x.q[3], x.v[0]);
      xc[jj * QS + lane] = make_float2(x.v[1], x.v[2]);
      if (dbg >= 0) {
        reinterpret_cast<float4*>(a.dbg_u)[(size_t)dbg * T + j] = u;
        float* X = a.dbg_x + ((size_t)dbg * (T + 1) + j + 1) * 10;
        for (int i = 0; i < 3; ++i) X[i] = x.p[i];
        for (int i = 0; i < 4; ++i) X[3 + i] = x.q[i];
        for (int i = 0; i < 3; ++i) X[7 + i] = x.v[i];
      }
    }
  };

  // the workers: queries and costs of chunk c
  auto score_chunk = [&](int c) {
    const int j0 = c * tcb, tc = tcb < T - j0 ? tcb : T - j0;
    const float4* xa = m.xa + (c & 1) * kChunkQ;
    const float4* xb = m.xb + (c & 1) * kChunkQ;
    const float2* xc = m.xc + (c & 1) * kChunkQ;
    // this thread's queries: steps jj = widx + SWK i of the chunk, sample `lane`
    int2 rg[kQ];
    int2 cnt = make_int2(0, 0);  // (listed queries, items)
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const int jj = widx + SWK * i;
      rg[i] = make_int2(0, 0);
      if (jj < tc) {
        m.d2[jj * QS + lane] = __float_as_int(dmax2);
        if (active) {
          const float4 p = xa[jj * QS + lane];
          rg[i] = cell_range(p.x, p.y, p.z, a.grid);
        }
      }
      if (rg[i].y > 0) {
        cnt.x += 1;
        cnt.y += (rg[i].y + kItem - 1) / kItem;
      }
    }
    int2 total;
    int2 off = block_scan2<SWK, kWorkBar>(cnt, m.scan, total, widx);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      if (rg[i].y > 0) {
        m.qitem[off.x] = off.y;
        m.qrange[off.x] = rg[i];
        m.qslot[off.x] = (unsigned short)((widx + SWK * i) * QS + lane);
        off.x += 1;
        off.y += (rg[i].y + kItem - 1) / kItem;
      }
    }
    if (widx == 0 && lane == 0) m.qitem[total.x] = total.y;
    warps_sync<SWK, kWorkBar>();  // query list complete
    for (int it = widx * 32 + lane; it < total.y; it += SWK * 32) {
      const int lo = item_owner(m.qitem, total.x, it);
      const int2 r = m.qrange[lo];
      const int slot = m.qslot[lo];
      const int first = (it - m.qitem[lo]) * kItem;
      const int n = r.y - first < kItem ? r.y - first : kItem;
      if (!AERO_CHECK(slot < kChunkQ && first >= 0 && n > 0 && r.x >= 0, kChkQuery)) continue;
      const float4 p = xa[slot];
      const float d2 = scan_min<kItem>(a.grid, r.x + first, n, p.x, p.y, p.z, dmax2);
      if (d2 < dmax2) atomicMin(m.d2 + slot, __float_as_int(d2));  // non-negative: int order
    }
    warps_sync<SWK, kWorkBar>();  // minima complete
    // the cost of every (sample, step) pair of this thread: J_ctrl's terms
    // Q_c |u_j|^2 (j <= T-2) and Q_cd |u_j - u_{j-1}|^2 (1 <= j <= T-2), the
    // state terms at x_{j+1} against the guide at t = (j + 1) dt, J_col.  The
    // pairs are evaluated without branches (a missing pair repeats the last
    // step and is masked) so that their latencies overlap.
    float cs[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const int jq = widx + SWK * i;
      const int jj = jq < tc ? jq : tc - 1, j = j0 + jj;
      const float4 u = m.u[j * QS + lane];
      const float4 up = m.u[(j >= 1 ? j - 1 : 0) * QS + lane];
      const float ax = u.x - up.x, ay = u.y - up.y, az = u.z - up.z, aw = u.w - up.w;
      const float c_u = cp.Q_c * (u.x * u.x + u.y * u.y + u.z * u.z + u.w * u.w);
      const float c_du = cp.Q_cd * (ax * ax + ay * ay + az * az + aw * aw);
      float cj = j <= T - 2 ? (j >= 1 ? c_u + c_du : c_u) : 0.0f;
      const float4 pa = xa[jj * QS + lane], pb = xb[jj * QS + lane];
      const float2 pc = xc[jj * QS + lane];
      State y;
      y.p[0] = pa.x; y.p[1] = pa.y; y.p[2] = pa.z;
      y.q[0] = pa.w; y.q[1] = pb.x; y.q[2] = pb.y; y.q[3] = pb.z;
      y.v[0] = pb.w; y.v[1] = pc.x; y.v[2] = pc.y;
      const float gx = m.gd[3 * j], gy = m.gd[3 * j + 1], gz = m.gd[3 * j + 2];
      cj += cp.Q_track * norm3f(y.p[0] - gx, y.p[1] - gy, y.p[2] - gz);
      cj += cp.Q_vnorm * (y.v[0] * y.v[0] + y.v[1] * y.v[1] + y.v[2] * y.v[2]);
      cj += goal_term(y, cp, at_rest);
      const float d2 = __int_as_float(m.d2[jj * QS + lane]);
      cj += jcol_select(d2, cp, dmax2);
      cs[i] = jq < tc && active ? cj : 0.0f;
      if (jq < tc && dbg >= 0) a.dbg_d[(size_t)dbg * T + j] = d2 < dmax2 ? sqrtf(d2) : INFINITY;
    }
#pragma unroll
    for (int i = 0; i < kQ; ++i) S += cs[i];
  };

  if (integrator) integrate(0);
  __syncthreads();  // chunk 0's states filled
  for (int c = 0; c < nch; ++c) {
    if (integrator) {
      if (c + 1 < nch) integrate(c + 1);
    } else {
      score_chunk(c);
    }
    __syncthreads();  // chunk c + 1 filled; chunk c's buffer free
  }
  m.cost[wid * QS + lane] = S;
  __syncthreads();
  float Sk = 0.0f;  // the warps' partial sums in a fixed order
#pragma unroll
  for (int w = 0; w < SW; ++w) Sk += m.cost[w * QS + lane];
  if (active && wid == 0) a.sample_costs[(size_t)e * a.K + k] = Sk;
  // every warp: rho_b = min S, w_k = exp(-(S_k - rho_b)/lambda), eta_b = sum w_k
  const float rho = warp_min(active ? Sk : INFINITY);
  const float wk = active ? expf((rho - Sk) * a.inv_lambda) : 0.0f;
  const float eta = warp_sum(wk);
  float* out = a.partials + ((size_t)e * a.nb + b) * (4 + 4 * T);
  const bool row_ok = AERO_CHECK(b < a.nb && e < a.E, kChkPartial);
  if (tid == 0 && row_ok) {
    out[0] = rho;
    out[1] = eta;
  }
  // W_b[j] = sum_k w_k du_k[j], warp w the steps j = w (mod 8)
  for (int j = wid; j < T; j += SW) {
    const float4 u = m.u[j * QS + lane], un = m.un[j];
    const float4 du = active ? make_float4(u.x - un.x, u.y - un.y, u.z - un.z, u.w - un.w)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    const float r = warp_sum4(wk * du.x, wk * du.y, wk * du.z, wk * du.w, lane);
    if ((lane & 7) == 0 && row_ok) out[4 + 4 * j + (lane >> 3)] = r;
  }
  __syncthreads();  // shared memory free for the next unit
}

// ---------------------------------------------------------------------------
// Merge the per-CTA partials of one instance and update its nominal; on the
// final iteration roll out the updated nominal (Stage II), score S(2), and let
// the last CTA to finish pick the argmin.
// ---------------------------------------------------------------------------
constexpr int UT = 128;  // threads of the update kernels

__host__ __device__ constexpr size_t round16(size_t n) { return (n + 15) & ~(size_t)15; }

// Shared memory of update_unit (bytes) for horizon T and `warps` warps: its
// own arrays, then the refinement's scratch when `refine`.
__host__ __device__ constexpr size_t update_smem_bytes(int T, int warps, bool refine) {
  return 16 * (size_t)warps * T          // acc: weighted sums [warps][T]
         + round16(40 * (size_t)(T + 1))  // x: Stage II states [T + 1][10]
         + 16 * (size_t)T                 // u: the updated nominal [T]
         + round16(8 * (size_t)T)         // qrange: candidate range of each listed query
         + 4 * 1024                       // scale: exp(-(rho_b - rho)/lambda), b < 1024
         + 4 * round16(4 * (size_t)(T + 1))  // c, qitem, qslot, d2
         + round16(4 * (size_t)warps)     // red: warp reductions
         + round16(8 * (size_t)warps)     // scan: warp totals
         + (refine ? refine_smem_bytes(T, warps) : 0);
}

struct UpdSmem {
  float4* acc;
  float* x;
  float4* u4;
  int2* qrange;
  float* scale;
  float* c;
  int* qitem;
  int* qslot;
  int* d2;
  float* red;
  int2* scan;
  unsigned char* refine;
};

__device__ __forceinline__ UpdSmem update_layout(unsigned char* base, int T, int warps) {
  UpdSmem m;
  size_t o = 0;
  auto take = [&](size_t n) {
    unsigned char* p = base + o;
    o += round16(n);
    return p;
  };
  m.acc = reinterpret_cast<float4*>(take(16 * (size_t)warps * T));
  m.x = reinterpret_cast<float*>(take(40 * (size_t)(T + 1)));
  m.u4 = reinterpret_cast<float4*>(take(16 * (size_t)T));
  m.qrange = reinterpret_cast<int2*>(take(8 * (size_t)T));
  m.scale = reinterpret_cast<float*>(take(4 * 1024));
  m.c = reinterpret_cast<float*>(take(4 * (size_t)(T + 1)));
  m.qitem = reinterpret_cast<int*>(take(4 * (size_t)(T + 1)));
  m.qslot = reinterpret_cast<int*>(take(4 * (size_t)(T + 1)));
  m.d2 = reinterpret_cast<int*>(take(4 * (size_t)(T + 1)));
  m.red = reinterpret_cast<float*>(take(4 * (size_t)warps));
  m.scan = reinterpret_cast<int2*>(take(8 * (size_t)warps));
  m.refine = base + o;
  return m;
}

// kThreads: the CTA's threads (128 in the update kernels, 256 in the split
// Stage I pass).  smem: update_smem_bytes(T, kThreads / 32, refine) bytes of
// dynamic shared memory (16-byte aligned).  The partials are read through L2
// (ld.cg): in the split pass other CTAs of the same launch wrote them.
template <int kThreads>
__device__ __forceinline__ void update_unit(const UpdateArgs& a, int e, bool final_stage,
                                            unsigned char* smem) {
  constexpr int UT = kThreads;
  const int T = a.T, stride = 4 + 4 * T;
  const UpdSmem sm = update_layout(smem, T, UT / 32);
  float* const s_scale = sm.scale;
  float* const s_red = sm.red;
  float* const s_x = sm.x;  // Stage II states
  float4* const s_u4 = sm.u4;
  float* const s_u = reinterpret_cast<float*>(s_u4);
  float* const s_c = sm.c;
  __shared__ bool s_last;
  // Stage II's nearest-point queries (one per step, cut into items)
  int* const s_qitem = sm.qitem;
  int2* const s_qrange = sm.qrange;
  int* const s_qslot = sm.qslot;
  int* const s_d2 = sm.d2;
  int2* const s_scan = sm.scan;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const float* P = a.partials + (size_t)e * a.nb * stride;

  // the loads that do not wait for rho go out first, in one round trip with
  // the first rows: the first kPre rows of this warp's weighted sums and this
  // thread's nominal entries
  constexpr int kW = UT / 32;
  constexpr int kCol = kMaxT / 32;
  constexpr int kPre = 4;
  constexpr int kUn = (4 * kMaxT + UT - 1) / UT;
  float4 pre[kPre][kCol];
#pragma unroll
  for (int r = 0; r < kPre; ++r) {
    const int b = wid + r * kW;
    const float4* row = reinterpret_cast<const float4*>(P + (size_t)b * stride + 4);
#pragma unroll
    for (int q = 0; q < kCol; ++q) {
      const int c4 = lane + 32 * q;
      pre[r][q] = b < a.nb && c4 < T ? __ldcg(row + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  float* un = a.u_nom + (size_t)e * T * 4;
  float un_pre[kUn];
#pragma unroll
  for (int r = 0; r < kUn; ++r) {
    const int i = tid + r * UT;
    un_pre[r] = i < 4 * T ? un[i] : 0.0f;
  }
  // rho = min rho_b (a thread's first row keeps its rho_b and eta_b for the sum)
  float m = INFINITY;
  const float2 first_row = tid < a.nb ? __ldcg(reinterpret_cast<const float2*>(P + (size_t)tid * stride))
                                      : make_float2(INFINITY, 0.0f);
  for (int b = tid; b < a.nb; b += UT) m = fminf(m, b == tid ? first_row.x : __ldcg(P + (size_t)b * stride));
  m = warp_min(m);
  if (lane == 0) s_red[wid] = m;
  __syncthreads();
  float rho = s_red[0];
  for (int w = 1; w < UT / 32; ++w) rho = fminf(rho, s_red[w]);
  __syncthreads();
  // eta = sum eta_b exp(-(rho_b - rho)/lambda)
  float eta = 0.0f;
  for (int b = tid; b < a.nb; b += UT) {
    const float sc = expf((rho - (b == tid ? first_row.x : __ldcg(P + (size_t)b * stride))) * a.inv_lambda);
    if (b < 1024) s_scale[b] = sc;
    eta += sc * (b == tid ? first_row.y : __ldcg(P + (size_t)b * stride + 1));
  }
  eta = warp_sum(eta);
  if (lane == 0) s_red[wid] = eta;
  __syncthreads();
  eta = 0.0f;
  for (int w = 0; w < UT / 32; ++w) eta += s_red[w];
  if (!(eta > 0.0f) || !isfinite(eta) || !isfinite(rho)) {
    if (tid == 0) atomicOr(a.status, 1);
  }
  const float inv_eta = 1.0f / eta;
  auto scale = [&](int b) {
    return b < 1024 ? s_scale[b] : expf((rho - __ldcg(P + (size_t)b * stride)) * a.inv_lambda);
  };
  __syncthreads();  // s_scale complete
  // sum_b scale_b W_b: warp w takes the rows b = w (mod kW) in order (the
  // first kPre of them loaded above), lane the float4 columns lane, lane + 32,
  // ...; all of a thread's loads are independent
  float4 acc[kCol];
#pragma unroll
  for (int q = 0; q < kCol; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int r = 0; r < kPre; ++r) {
    const int b = wid + r * kW;
    if (b < a.nb) {
      const float sc = scale(b);
#pragma unroll
      for (int q = 0; q < kCol; ++q) {
        if (lane + 32 * q < T) {
          acc[q].x += sc * pre[r][q].x;
          acc[q].y += sc * pre[r][q].y;
          acc[q].z += sc * pre[r][q].z;
          acc[q].w += sc * pre[r][q].w;
        }
      }
    }
  }
#pragma unroll 4
  for (int b = wid + kPre * kW; b < a.nb; b += kW) {
    const float sc = scale(b);
    const float4* row = reinterpret_cast<const float4*>(P + (size_t)b * stride + 4);
#pragma unroll
    for (int q = 0; q < kCol; ++q) {
      const int c4 = lane + 32 * q;
      if (c4 < T) {
        const float4 w4 = __ldcg(row + c4);
        acc[q].x += sc * w4.x;
        acc[q].y += sc * w4.y;
        acc[q].z += sc * w4.z;
        acc[q].w += sc * w4.w;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kCol; ++q)
    if (lane + 32 * q < T) sm.acc[wid * T + lane + 32 * q] = acc[q];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kUn; ++r) {
    const int i = tid + r * UT;
    if (i < 4 * T) {
      const int j = i >> 2, c = i & 3;
      float sum = 0.0f;
#pragma unroll
      for (int w = 0; w < kW; ++w) sum += reinterpret_cast<const float*>(&sm.acc[w * T + j])[c];
      const float v = un_pre[r] + sum * inv_eta;
      un[i] = v;
      s_u[i] = v;
    }
  }
  if (!final_stage) return;
  __syncthreads();

  // gradient refinement of the updated nominal by the whole CTA (the scratch
  // after the update's own arrays)
  if (a.refine_steps > 0) {
    if (a.dbg_pre)
      for (int i = tid; i < 4 * T; i += UT) a.dbg_pre[(size_t)e * T * 4 + i] = s_u[i];
    block_refine<UT>(s_u4, a.guides + (size_t)e * T * 3, T, a.x0, a.dyn, a.cost, a.grid, a.umin,
                     a.umax, a.refine_steps, a.refine_step, refine_layout(sm.refine, T, UT / 32));
    for (int i = tid; i < 4 * T; i += UT) un[i] = s_u[i];
    __syncthreads();
  }

  // Stage II: noise-free rollout of the (updated, refined) nominal, by scans
  // over the steps (rollout_by_scans); the merge's scratch (acc) is free again
  // and holds the warps' scan totals
  static_assert(kMaxT <= UT, "one Stage II step per thread");
  rollout_by_scans<UT / 32>(s_u4, T, a.x0, a.dyn, s_x, sm.acc);
  // the nearest point of every state x_{j+1} (thread j): the non-empty
  // candidate lists cut into items of kItem entries, taken by all threads
  static_assert(kMaxT <= UT, "one Stage II query per thread");
  const float dmax2 = a.cost.d_max * a.cost.d_max;
  int2 rg = make_int2(0, 0);
  if (tid < T) {
    const float* X = s_x + (tid + 1) * 10;
    rg = cell_range(X[0], X[1], X[2], a.grid);
    s_d2[tid] = __float_as_int(dmax2);
  }
  int2 total;
  const int2 off = block_scan2<UT / 32>(
      rg.y > 0 ? make_int2(1, (rg.y + kItem - 1) / kItem) : make_int2(0, 0), s_scan, total);
  if (rg.y > 0) {
    s_qitem[off.x] = off.y;
    s_qrange[off.x] = rg;
    s_qslot[off.x] = tid;
  }
  __syncthreads();
  for (int it = tid; it < total.y; it += UT) {
    const int lo = item_owner(s_qitem, total.x, it);
    const int2 r = s_qrange[lo];
    const int j = s_qslot[lo];
    const int first = (it - s_qitem[lo]) * kItem;
    const int n = r.y - first < kItem ? r.y - first : kItem;
    if (!AERO_CHECK(j < T && first >= 0 && n > 0 && r.x >= 0, kChkQuery)) continue;
    const float* X = s_x + (j + 1) * 10;
    const float d2 = scan_min<kItem>(a.grid, r.x + first, n, X[0], X[1], X[2], dmax2);
    if (d2 < dmax2) atomicMin(s_d2 + j, __float_as_int(d2));  // non-negative: int order
  }
  __syncthreads();
  if (tid < T) {
    const float* X = s_x + (tid + 1) * 10;
    State x;
    for (int i = 0; i < 3; ++i) x.p[i] = X[i];
    for (int i = 0; i < 4; ++i) x.q[i] = X[3 + i];
    for (int i = 0; i < 3; ++i) x.v[i] = X[7 + i];
    s_c[tid] = goal_term(x, a.cost, goal_at_rest(a.cost)) + jcol_from_d2(__int_as_float(s_d2[tid]), a.cost, dmax2);
  }
  for (int i = tid; i < (T + 1) * 10; i += UT) a.stage2_x[(size_t)e * (T + 1) * 10 + i] = s_x[i];
  __syncthreads();
  if (wid == 0) {
    // S(2): fixed-order sum (strided per lane, then a shuffle tree)
    float s2 = 0.0f;
    for (int j = lane; j < T; j += 32) s2 += s_c[j];
    s2 = warp_sum(s2);
    if (lane == 0) a.cand[e] = s2;
  }
  // last CTA to arrive selects the best instance
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(a.counter, 1u) == (unsigned)(a.E - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ int s_best;
  if (wid == 0) {
    // argmin over the instances, ties to the lower index (E <= 64: two per lane)
    float bc = INFINITY;
    int best = 0x7fffffff;
    for (int i = lane; i < a.E; i += 32) {
      const float c = __ldcg(a.cand + i);
      if (c < bc) { bc = c; best = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oc = __shfl_xor_sync(0xffffffffu, bc, o);
      const int ob = __shfl_xor_sync(0xffffffffu, best, o);
      if (oc < bc || (oc == bc && ob < best)) { bc = oc; best = ob; }
    }
    if (lane == 0) {
      // no candidate with a finite S(2) below +inf (every one NaN or +inf): the
      // first instance, and bit 2 of the status word
      if (best >= a.E) {
        best = 0;
        atomicOr(a.status, 4);
      }
      s_best = best;
      *a.best_idx = best;
      *a.counter = 0u;
    }
  }
  __syncthreads();
  const float* ub = a.u_nom + (size_t)s_best * T * 4;
  for (int i = tid; i < 4 * T; i += UT) a.u_best[i] = __ldcg(ub + i);
}

template <bool kWarpLists>
__global__ void __launch_bounds__(NT, 6) k_rollout(RolloutArgs a) {
  pdl_start();
  rollout_unit<true, NT, kWarpLists>(a, blockIdx.y, blockIdx.x, a.ctr3);
  if (a.done != nullptr) {
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(a.done, 1u);
  }
}

// A warm-up run of the update's code on instance e's inputs: s_ua (a copy of
// ua in shared memory) gets every output of the update (nominal, Stage II
// states, costs, selection, tickets, status) in region e of ua.warm; instance
// e's nominal is copied there first and the ticket set so that the selection
// runs too.  The update runs once per launch, so without it its instructions
// would be fetched cold (from DRAM once the L2 has been overwritten) on the
// critical path; the warm-up run's results are discarded.  It may read
// partials that other CTAs are writing: every access of the update stays in
// bounds whatever the values read.  Every thread of the CTA calls it.
__device__ __forceinline__ void warm_setup(UpdateArgs* s_ua, const UpdateArgs& ua, int e) {
  const int E = ua.E, T = ua.T;
  float* const sc = ua.warm + (size_t)e * warm_words(E, T);
  if (threadIdx.x == 0) {
    s_ua->u_nom = sc;
    s_ua->stage2_x = sc + (size_t)E * T * 4;
    s_ua->cand = s_ua->stage2_x + (size_t)(T + 1) * 10;
    s_ua->u_best = s_ua->cand + E;
    s_ua->best_idx = reinterpret_cast<int*>(s_ua->u_best + (size_t)T * 4);
    s_ua->counter = reinterpret_cast<unsigned int*>(s_ua->best_idx + 1);
    s_ua->status = reinterpret_cast<int*>(s_ua->counter + 1);
    s_ua->dbg_pre = nullptr;
    *s_ua->counter = (unsigned)(E - 1);
  }
  for (int i = threadIdx.x; i < 4 * T; i += blockDim.x) sc[(size_t)e * T * 4 + i] = ua.u_nom[(size_t)e * T * 4 + i];
  __syncthreads();
}

// The split pass with the update of every instance run by the last of its
// CTAs to finish (a ticket per instance, reset by that CTA): no update launch.
// Block b >= w runs CTA (b - w) mod nb of instance (b - w) / nb.  With a
// warm-up block (w = 1: ua.warm set), block 0 runs the same update code (one
// call site) at the start of the launch as a warm-up run on instance 0's
// inputs (warm_setup), so that the code is in L2 when the CTAs that finish
// last reach it.
__global__ void __launch_bounds__(ST, 2) k_rollout_split(RolloutArgs a, UpdateArgs ua) {
  // the wait for the preceding launches comes after the noise (in
  // rollout_split_unit), so that drawing it overlaps them
  pdl_trigger();
  __shared__ bool s_last_b;
  __shared__ UpdateArgs s_ua;
  const int w = ua.warm != nullptr ? 1 : 0;
  const bool warm = w == 1 && blockIdx.x == 0;
  const int lin = (int)blockIdx.x - w;
  const int e = warm ? 0 : lin / a.nb;
  if (!warm) {
    rollout_split_unit(a, e, lin - e * a.nb, a.ctr3);
    __threadfence();  // this CTA's partials are visible before its ticket
    __syncthreads();
    if (threadIdx.x == 0) s_last_b = atomicAdd(ua.inst_counter + e, 1u) == (unsigned)(a.nb - 1);
    __syncthreads();
    if (!s_last_b) return;
    __threadfence();
    if (threadIdx.x == 0) ua.inst_counter[e] = 0u;
  }
  if (warm) pdl_wait();  // the warm-up run reads the grid
  block_copy_param(&s_ua, &ua);
  __syncthreads();
  if (warm) warm_setup(&s_ua, ua, 0);
  extern __shared__ __align__(16) unsigned char fused_smem[];  // the split pass's, free again
  update_unit<ST>(s_ua, e, s_ua.final_stage != 0, fused_smem);
}

// The single-planner update: one CTA of ST threads per instance (the split
// pass's update runs on as many; twice the batched update's, so the merge of
// the partial rows and the Stage II scans take fewer rounds: 22.0 -> 19.8 us
// at E = 32, K = 8192, T = 64).  It reads its arguments from shared memory, as
// the batched one does (from kernel parameters the compiler contracts some
// products differently).
//
// With a.warm set, a CTA that starts while Stage I still runs first runs its
// instance's update as a warm-up run (warm_setup) before it waits for Stage I:
// the launch is programmatic, so its CTAs start as soon as the last CTAs of
// Stage I have started, and the warm-up runs overlap Stage I's last wave; the
// real update then finds its code in L2 and this SM's instruction caches.  A
// CTA that starts after Stage I has finished (every one of its CTAs counted
// in a.done[0]: the launch was not overlapped) skips the warm-up run.  One
// call site for both runs (the same code).
__global__ void __launch_bounds__(ST) k_update(UpdateArgs a) {
  __shared__ UpdateArgs s_a;
  __shared__ bool s_warm;
  extern __shared__ __align__(16) unsigned char upd_smem[];  // update_smem_bytes(T, ST / 32, refine)
  if (threadIdx.x == 0)
    s_warm = a.warm != nullptr &&
             (a.done == nullptr || *reinterpret_cast<volatile unsigned int*>(a.done) < (unsigned)(a.nb * a.E));
  __syncthreads();
#pragma unroll 1
  for (int run = s_warm ? 0 : 1; run < 2; ++run) {
    if (run == 1) pdl_start();
    else pdl_trigger();
    block_copy_param(&s_a, &a);
    __syncthreads();
    if (run == 0) warm_setup(&s_a, a, blockIdx.x);
    update_unit<ST>(s_a, blockIdx.x, s_a.final_stage != 0, upd_smem);
    __syncthreads();  // s_a and the scratch free for the next run
  }
  // the last CTA to leave resets the count and the exit ticket (every CTA has
  // read the count by then, and Stage I has finished)
  if (a.done != nullptr && threadIdx.x == 0 && atomicAdd(a.done + 1, 1u) == gridDim.x - 1) {
    a.done[0] = 0u;
    a.done[1] = 0u;
  }
}

// ---------------------------------------------------------------------------
// Batched Stage I: units (planner, instance, block of samples) in the order of
// the planners' positions (longest horizon first).  dynamic: every CTA takes its
// next unit from the work queue (an atomic counter; the last CTA to leave
// resets it), else units are strided by the grid.  Planners whose iteration
// count is at most `it` skip their units.
// ---------------------------------------------------------------------------
// kNT: samples per CTA of the one-lane pass (the autotuner's choice).
template <int kLanes, int kMinCtas, int kNT = NT>
__global__ void __launch_bounds__(kLanes == 4 ? ST : kNT, kMinCtas)
    k_b_rollout(BatchView v, int it, int dynamic) {
  pdl_start();
  __shared__ long long s_pre[kBatchMax + 1];
  __shared__ int s_order[kBatchMax];
  __shared__ RolloutArgs s_a;
  __shared__ int s_iters;
  __shared__ unsigned int s_u;
  const int n = v.n;
  load_prefix(s_pre, v.pre + (kLanes == 1 ? kPreRoll1 : kPreRoll4) * (n + 1), n);
  const int* order = kLanes == 1 ? v.order1 : v.order4;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s_order[i] = __ldg(order + i);
  unsigned int* queue = v.queue + (kLanes == 1 ? 0 : 2);
  __syncthreads();
  const long long total = s_pre[n];
  int cur = -1;
  long long u = blockIdx.x;
  for (;;) {
    if (dynamic) {
      if (threadIdx.x == 0) s_u = atomicAdd(queue, 1u);
      __syncthreads();
      u = s_u;
    }
    if (u >= total) break;
    const int pos = find_unit(s_pre, n, u);
    const int item = s_order[pos];
    if (item != cur) {
      block_copy(&s_a, &v.items[item].ra);
      if (threadIdx.x == 0) s_iters = v.items[item].iters;
      __syncthreads();
      cur = item;
    }
    if (it < s_iters) {
      const long long l = u - s_pre[pos];
      const int e = (int)(l / s_a.nb), b = (int)(l % s_a.nb);
      if constexpr (kLanes == 1)
        rollout_unit<false, kNT, false, (kMinCtas == 5 && kNT == NT)>(s_a, e, b, s_a.ctr3 | (uint32_t)it);
      else
        rollout_split_unit(s_a, e, b, s_a.ctr3 | (uint32_t)it);
    }
    if (!dynamic) u += gridDim.x;
    __syncthreads();  // the unit's shared memory is free again
  }
  if (dynamic && threadIdx.x == 0) {
    // every CTA has drawn past the end before it counts itself out
    if (atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
      queue[0] = 0u;
      queue[1] = 0u;
    }
  }
}

// Batched merge and update: units (planner, instance); the last iteration of a
// planner runs its Stage II and selection.
__global__ void __launch_bounds__(UT) k_b_update(BatchView v, int it) {
  pdl_start();
  extern __shared__ __align__(16) unsigned char upd_smem[];  // update_smem_bytes(T_max, UT / 32, true)
  __shared__ long long s_pre[kBatchMax + 1];
  __shared__ UpdateArgs s_a;
  __shared__ int s_iters;
  const int n = v.n;
  load_prefix(s_pre, v.pre + kPreUpdate * (n + 1), n);
  __syncthreads();
  const long long total = s_pre[n];
  int cur = -1;
  for (long long u = blockIdx.x; u < total; u += gridDim.x) {
    const int item = find_unit(s_pre, n, u);
    if (item != cur) {
      block_copy(&s_a, &v.items[item].ua);
      if (threadIdx.x == 0) s_iters = v.items[item].iters;
      __syncthreads();
      cur = item;
    }
    if (it < s_iters) update_unit<UT>(s_a, (int)(u - s_pre[item]), it == s_iters - 1, upd_smem);
    __syncthreads();
  }
}

constexpr bool fused_update_fits() {
  for (int T = 1; T <= kMaxT; ++T)
    if (update_smem_bytes(T, ST / 32, true) > split_smem_bytes(T)) return false;
  return true;
}
static_assert(fused_update_fits(),
              "the split pass's shared memory holds the fused update and its refinement scratch");

// One warp per control sequence: S(1) of its noise-free rollout and dS/dU.
constexpr int kCgWarps = 4;

__global__ void __launch_bounds__(32 * kCgWarps) k_cost_grad(CostGradArgs a) {
  __shared__ float4 s_u[kCgWarps][kMaxT];
  __shared__ float4 s_g[kCgWarps][kMaxT];
  __shared__ AdjScratch s_sc[kCgWarps];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kCgWarps + wid;
  if (i >= a.n) return;  // uniform over the warp
  const int T = a.ctx.T;
  for (int t = lane; t < T; t += 32) s_u[wid][t] = a.U[(size_t)i * T + t];
  __syncwarp();
  const float* guide = a.ctx.guides + (size_t)a.instance * T * 3;
  float S;
  if (a.G)
    S = warp_cost_grad<true>(s_u[wid], s_g[wid], guide, T, a.ctx.x0, a.ctx.dyn, a.ctx.cost,
                             a.ctx.grid, s_sc[wid], lane);
  else
    S = warp_cost_grad<false>(s_u[wid], s_g[wid], guide, T, a.ctx.x0, a.ctx.dyn, a.ctx.cost,
                              a.ctx.grid, s_sc[wid], lane);
  if (lane == 0) a.S[i] = S;
  if (a.G)
    for (int t = lane; t < T; t += 32) a.G[(size_t)i * T + t] = s_g[wid][t];
}

}  // namespace

cudaError_t launch_cost_grad(const CostGradArgs& a, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  k_cost_grad<<<(a.n + kCgWarps - 1) / kCgWarps, 32 * kCgWarps, 0, s>>>(a);
  return cudaGetLastError();
}

// The split pass reads its shared memory as one dynamic block sized for the
// horizon; allow the largest.  The attribute belongs to the device, so it is
// set once per device (the create functions call this first, so that no
// launch captured into a graph is the first on its device).
cudaError_t split_attributes() {
  static std::atomic<int> done[64];  // 0: not yet, 1: set, else the error + 2
  int dev = 0;
  cudaError_t r = cudaGetDevice(&dev);
  if (r != cudaSuccess) return r;
  const bool cached = dev >= 0 && dev < 64;
  if (cached) {
    const int d = done[dev].load();
    if (d == 1) return cudaSuccess;
    if (d > 1) return (cudaError_t)(d - 2);
  }
  const int most = (int)split_smem_bytes(kMaxT);
  r = cudaFuncSetAttribute(k_rollout_split, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(k_b_rollout<4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  const int refine = (int)update_smem_bytes(kMaxT, UT / 32, true);
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)update_smem_bytes(kMaxT, ST / 32, true));
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(k_b_update, cudaFuncAttributeMaxDynamicSharedMemorySize, refine);
  if (cached) done[dev].store(r == cudaSuccess ? 1 : (int)r + 2);
  return r;
}

// Few CTAs per SM run the single-planner split pass and its candidate scans
// live on L1 hits: the carveout asked for is the smallest that still holds
// two of its CTAs (as a percentage of the 228 KB an SM can give).  Like the
// size limit, the carveout is an attribute per device.
cudaError_t split_carveout(int T) {
  static std::atomic<int> current[64];  // the percentage set on each device, plus one
  static const size_t static_bytes = [] {
    cudaFuncAttributes fa{};
    return cudaFuncGetAttributes(&fa, k_rollout_split) == cudaSuccess ? fa.sharedSizeBytes : 0;
  }();
  const size_t need = 2 * (split_smem_bytes(T) + static_bytes + 1024);
  int pct = (int)((need * 100 + 228 * 1024 - 1) / (228 * 1024));
  if (pct > 100) pct = 100;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cached = dev >= 0 && dev < 64;
  if (cached && current[dev].load() == pct + 1) return cudaSuccess;
  e = cudaFuncSetAttribute(k_rollout_split, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  if (e == cudaSuccess && cached) current[dev].store(pct + 1);
  return e;
}

cudaError_t batch_rollout_occupancy(int out[6], int T_max) {
  cudaError_t e = split_attributes();
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out + 0, k_b_rollout<1, 5>, NT, 0);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out + 1, k_b_rollout<4, 2>, ST,
                                                      split_smem_bytes(T_max));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out + 2, k_b_update, UT,
                                                      update_smem_bytes(T_max, UT / 32, true));
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out + 3, k_b_rollout<1, 6>, NT, 0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out + 4, k_b_rollout<1, 12, 64>, 64, 0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out + 5, k_b_rollout<1, 3, 256>, 256, 0);
  for (int i = 0; i < 6; ++i)
    if (out[i] < 1) out[i] = 1;
  return e;
}

cudaError_t launch_batch_rollout(const BatchView& v, int lanes, int it, int blocks, int dynamic,
                                 int six, int samples_per_cta, cudaStream_t s) {
  if (lanes == 4)
    return launch_ks(k_b_rollout<4, 2>, dim3(blocks), dim3(ST), split_smem_bytes(v.T_max), s, true, v,
                     it, dynamic);
  if (samples_per_cta == 64)
    return launch_k(k_b_rollout<1, 12, 64>, dim3(blocks), dim3(64), s, true, v, it, dynamic);
  if (samples_per_cta == 256)
    return launch_k(k_b_rollout<1, 3, 256>, dim3(blocks), dim3(256), s, true, v, it, dynamic);
  if (six) return launch_k(k_b_rollout<1, 6>, dim3(blocks), dim3(NT), s, true, v, it, dynamic);
  return launch_k(k_b_rollout<1, 5>, dim3(blocks), dim3(NT), s, true, v, it, dynamic);
}

cudaError_t launch_batch_update(const BatchView& v, int it, int blocks, cudaStream_t s) {
  return launch_ks(k_b_update, dim3(blocks), dim3(UT), update_smem_bytes(v.T_max, UT / 32, true), s,
                   true, v, it);
}

bool rollout_runs_update(const RolloutArgs& a) { return a.lanes_per_sample == 4; }

cudaError_t launch_rollout(const RolloutArgs& a, const UpdateArgs& ua, cudaStream_t s) {
  if (a.lanes_per_sample == 4) {
    cudaError_t e = split_attributes();
    // the carveout is a hint: a launch being captured into a graph keeps the
    // one set by earlier launches
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (e == cudaSuccess) e = cudaStreamIsCapturing(s, &cs);
    if (e == cudaSuccess && cs == cudaStreamCaptureStatusNone) e = split_carveout(a.T);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)a.nb * a.E + (ua.warm != nullptr ? 1u : 0u));
    return launch_ks(k_rollout_split, grid, dim3(ST), split_smem_bytes(a.T), s, true, a, ua);
  }
  if (a.list_thr > 0) return launch_k(k_rollout<true>, dim3(a.nb, a.E), dim3(NT), s, true, a);
  return launch_k(k_rollout<false>, dim3(a.nb, a.E), dim3(NT), s, true, a);
}

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s) {
  const cudaError_t e = split_attributes();  // also the update kernels' scratch limit
  if (e != cudaSuccess) return e;
  const size_t smem = update_smem_bytes(a.T, ST / 32, a.refine_steps > 0);
  return launch_ks(k_update, dim3(a.E), dim3(ST), smem, s, true, a);
}

cudaError_t check_word_rollout(int* out, bool clear) {
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

