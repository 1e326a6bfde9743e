// C-ABI host runtime of the AERO-MPPI planning step: planner workspace,
// argument validation, binary32 partition tables, collision-grid geometry and
// the launch sequence of one step.  Host code is compiled with
// -ffp-contract=off so that R(q0), the goal offset and the edge tables follow
// the stated binary32/binary64 operation order exactly.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/aero_mppi.h"
#ifdef AERO_CHECKED
#include <nvtx3/nvToolsExt.h>
#endif
#include "internal.h"

using namespace aero;

namespace aero {

namespace {
std::atomic<int64_t> g_alloc_total{0};       // allocations made
std::atomic<int64_t> g_alloc_live{0};        // allocations not yet freed
std::atomic<int64_t> g_alloc_fail_after{-1}; // allocations left before the injected failure

// True for the allocation aero_test_fail_alloc picked; the countdown then
// stays at -1 (off).
bool injected_failure() {
  int64_t c = g_alloc_fail_after.load();
  while (c >= 0)
    if (g_alloc_fail_after.compare_exchange_weak(c, c - 1)) return c == 0;
  return false;
}

cudaError_t counted(cudaError_t e, void** p) {
  if (e == cudaSuccess) {
    g_alloc_total.fetch_add(1);
    g_alloc_live.fetch_add(1);
  } else {
    *p = nullptr;
  }
  return e;
}
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return counted(cudaMalloc(p, bytes), p);
}

cudaError_t host_malloc(void** p, size_t bytes) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return counted(cudaMallocHost(p, bytes), p);
}

cudaError_t read_check_words(int* out, bool clear) {
  *out = 0;
#ifdef AERO_CHECKED
  cudaError_t e = cudaDeviceSynchronize();
  int w = 0;
  if (e == cudaSuccess) e = check_word_partition(&w, clear);
  *out |= w;
  if (e == cudaSuccess) e = check_word_rollout(&w, clear);
  *out |= w;
  if (e == cudaSuccess) e = check_word_accum(&w, clear);
  *out |= w;
  return e;
#else
  (void)clear;
  return cudaSuccess;
#endif
}

int device_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  if (dev >= 0 && dev < 64) {
    const int v = cache[dev].load();
    if (v > 0) return v;
  }
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return 1;
  }
  if (dev >= 0 && dev < 64) cache[dev].store(n);
  return n;
}

void dev_free(void* p) {
  if (!p) return;
  cudaFree(p);
  g_alloc_live.fetch_sub(1);
}

void host_free(void* p) {
  if (!p) return;
  cudaFreeHost(p);
  g_alloc_live.fetch_sub(1);
}

}  // namespace aero

struct aero_planner {
  aero_limits_t lim{};
  int device = 0;
  // workspace
  unsigned long long* keys = nullptr;
  int* coarse_win = nullptr;
  int* cells = nullptr;       // [0] goal fine cell, [1 + e] anchor coarse cell
  float* anchors = nullptr;
  float* guides = nullptr;
  int* item_flag = nullptr;   // per point: kept by the partition (collision set = kept points)
  int* grid_count = nullptr;  // G^3 + 1 candidate counts, zero between steps
  int* grid_fill = nullptr;   // G^3 + 1 fill cursors of the scatter
  bool grid_dirty = true;     // counts possibly non-zero (new planner, interrupted step)
  bool keys_empty = false;    // every fine-cell key is empty (left so by a batched step)
  int* grid_local = nullptr;  // G^3 + 1 tile-local exclusive prefix
  int* tile_sum = nullptr;
  int* tile_off = nullptr;
  float4* cand = nullptr;     // candidate entries: points, or item indices (as uint32)
  float4* cand_pts = nullptr; // collision point of every item, minus p0 (index entries)
  bool last_idx_entries = false;  // the last step's entries were item indices
  int2* grid_range = nullptr; // G^3 {first entry, count}
  int cand_cap = 0;
  int grid_max = kGridMax;    // cells per axis the grid arrays can hold
  int grid_cells_cap = kGridMax * kGridMax * kGridMax;
  float* partials = nullptr;
  float* sample_costs = nullptr;
  float* stage2_x = nullptr;
  unsigned int* counter = nullptr;
  int* status = nullptr;
  float* warm = nullptr;      // warm-up scratch: E_max regions of warm_words(E_max, T_max)
  float* dbg_u = nullptr;
  float* dbg_x = nullptr;
  float* dbg_d = nullptr;
  float* dbg_pre = nullptr;   // nominals before the gradient refinement
  int2* part_counts = nullptr;  // per partition block or chunk: {non-finite, kept} points
  int part_slots = 0;         // entries of part_counts
  // staging for aero_plan_step_host
  float* stage_cloud = nullptr;
  // the step's outputs, contiguous (nominals, best sequence, candidate costs,
  // best index) so that one copy brings them back; h_out is its pinned twin
  float* stage_out = nullptr;
  float* h_out = nullptr;
  // metadata of the last step (debug copies)
  bool have_step = false;
  aero_params_t last{};
  GridGeom last_grid{};
  UpdateArgs last_ctx{};  // state, dynamics, costs, grid and guides of the last step
  int last_ntiles = 0;
  int last_nb = 0;
  int last_part_slots = 0;    // part_counts entries written by the last step
  // the partition's edge tables of the last geometry (fine_az, fine_el, el_lo, el_hi)
  bool tab_valid = false;
  int tab_A = 0, tab_El = 0;
  float tab_lo = 0.0f, tab_hi = 0.0f;
  int tab_check_lo = 0, tab_check_hi = 0;
  PartTables tab{};
  PartTables* d_tab = nullptr;  // device copy, read by the partition and the guides
  bool tab_upload = true;       // d_tab behind tab
  int64_t last_n_points = 0;
  int64_t raw_max = 0;          // cloud size up to which the every-point set fits
  // stage timing (aero_profile_enable / aero_profile_read)
  struct ProfSlot {
    // start/end of: partition, grid, then rollout and update of every iteration
    std::vector<cudaEvent_t> ev;
    int iters = 0;
    int mask = 0;
    int last = -1;  // last event recorded
    int64_t launches[AERO_STAGE_COUNT] = {0, 0, 0, 0};
  };
  int prof = 0;  // bitmask of timed stages
  std::vector<ProfSlot> slots;
  size_t slots_used = 0;
  double prof_ms[AERO_STAGE_COUNT] = {0, 0, 0, 0};
  int64_t prof_launches[AERO_STAGE_COUNT] = {0, 0, 0, 0};
};

namespace {

// A point joins the lists of the cells within `reach` (just above d_max) of it:
// at most 6^3 cells of edge d_max / 2, at most 3^3 of edge d_max (1 + 1/16).
constexpr int kFineDup = 216, kCoarseDup = 27;
// points per fine cone from which the partition reads a cone's key before its
// atomic minimum: in dense clouds most points cannot lower their cone's key
constexpr int64_t kPartFilterPointsPerCone = 32;
// lists longer than this are scanned by the whole warp in the one-lane pass
// when every kept point is the collision set
constexpr int kWarpListThreshold = 8;

int cuda_fail(cudaError_t e) {
  if (e == cudaSuccess) return AERO_OK;
  return AERO_ERR_CUDA;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// R(q) of a unit quaternion in binary32: nine products, then the sums.
void rot_f32(const float* q, float* R) {
  const float w = q[0], x = q[1], y = q[2], z = q[3];
  const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  const float wx = w * x, wy = w * y, wz = w * z;
  R[0] = 1.0f - 2.0f * (yy + zz);
  R[1] = 2.0f * (xy - wz);
  R[2] = 2.0f * (xz + wy);
  R[3] = 2.0f * (xy + wz);
  R[4] = 1.0f - 2.0f * (xx + zz);
  R[5] = 2.0f * (yz - wx);
  R[6] = 2.0f * (xz - wy);
  R[7] = 2.0f * (yz + wx);
  R[8] = 1.0f - 2.0f * (xx + yy);
}

void make_tables(const aero_params_t& p, PartTables& t, int& check_lo, int& check_hi) {
  const int A = p.fine_az, El = p.fine_el;
  for (int k = 0; k < A; ++k) {
    const double th = (M_PI * (double)(2 * k - A)) / (double)A;
    t.ca[k] = (float)std::cos(th);
    t.sa[k] = (float)std::sin(th);
  }
  const double lo = (double)p.el_lo, hi = (double)p.el_hi;
  for (int k = 0; k <= El; ++k) {
    const double ph = lo + ((hi - lo) * (double)k) / (double)El;
    t.ce[k] = (float)std::cos(ph);
    t.se[k] = (float)std::sin(ph);
  }
  check_lo = lo > -M_PI / 2;
  check_hi = hi < M_PI / 2;
}

// Candidate grid over [-E, E)^3 around p0, E = r_max + reach + h: every
// collision point lies within r_max of p0, so queries outside the grid are
// farther than d_max from all of them.  Cells of edge d_max / 2 when the
// candidate array can hold 216 entries per collision item (and `coarse` is
// not asked for), else d_max (1 + 1/16);
// never more than kGridMax cells per axis.  `margin` covers binary32 rounding
// of the cell coordinates.
GridGeom make_grid(const aero_params_t& p, int64_t n_items, int64_t cap, int gmax, bool coarse) {
  GridGeom g;
  g.reach = p.d_max * (1.0f + 1e-3f) + 1e-4f;
  float h = !coarse && (int64_t)kFineDup * n_items <= cap ? 0.5f * p.d_max : p.d_max * 1.0625f;
  float E = p.r_max + g.reach + h;
  int G = (int)std::ceil(2.0f * E / h);
  if (G > gmax) {
    // coarser cells: E grows with h, so solve h = 2 (r_max + reach + h) / gmax
    h = 2.0f * (p.r_max + g.reach) / ((float)gmax - 2.5f);
    E = p.r_max + g.reach + h;
    G = (int)std::ceil(2.0f * E / h);
    if (G > gmax) G = gmax;
  }
  g.G = G;
  g.h = h;
  g.inv_h = 1.0f / h;
  g.origin = -E;
  g.cap = (int)cap;
  return g;
}

int validate(const aero_planner* pl, const aero_params_t* p, int64_t n_points) {
  const aero_limits_t& L = pl->lim;
  if (p->E < 1 || p->K < 1 || p->T < 1 || p->iters < 1 || p->iters > 255) return AERO_ERR_INVALID_ARG;
  if (p->M_h < 1 || p->M_v < 1 || p->M_h * p->M_v != p->E) return AERO_ERR_INVALID_ARG;
  if (p->fine_az < 2 || (p->fine_az & 1) || p->fine_el < 1 || p->fine_az > kMaxAz || p->fine_el > kMaxEl)
    return AERO_ERR_INVALID_ARG;
  if (p->pool_az < 1 || p->pool_el < 1 || p->fine_az % p->pool_az || p->fine_el % p->pool_el)
    return AERO_ERR_INVALID_ARG;
  if (!(p->dt > 0) || !(p->lambda > 0) || !(p->mass > 0) || !(p->r_max > 0) || !(p->ell > 0) ||
      !(p->d_max > 0) || !(p->d_min < p->d_max) || !(p->el_lo < p->el_hi))
    return AERO_ERR_INVALID_ARG;
  const float scalars[] = {p->dt, p->lambda, p->mass, p->r_max, p->ell, p->d_max, p->d_min,
                           p->el_lo, p->el_hi};
  for (float f : scalars)
    if (!std::isfinite(f)) return AERO_ERR_INVALID_ARG;
  for (int c = 0; c < 4; ++c)
    if (!(p->u_min[c] <= p->u_max[c]) || !(p->sigma[c] >= 0) || !std::isfinite(p->sigma[c]))
      return AERO_ERR_INVALID_ARG;
  if (p->collision_set != 0 && p->collision_set != 1) return AERO_ERR_INVALID_ARG;
  if (p->debug_samples < 0 || n_points < 0) return AERO_ERR_INVALID_ARG;
  if (p->lanes_per_sample != 0 && p->lanes_per_sample != 1 && p->lanes_per_sample != 4)
    return AERO_ERR_INVALID_ARG;
  if (p->refine_steps < 0 || p->refine_steps > 64 || !(p->refine_step >= 0.0f) ||
      !std::isfinite(p->refine_step))
    return AERO_ERR_INVALID_ARG;
  if (p->E > L.E_max || p->K > L.K_max || p->T > L.T_max ||
      (int64_t)p->fine_az * p->fine_el > L.fine_cells_max || n_points > L.n_points_max ||
      p->debug_samples > L.debug_samples_max || (p->collision_set == 1 && n_points > pl->raw_max))
    return AERO_ERR_EXCEEDS_LIMITS;
  return AERO_OK;
}

// A finite state and goal (a non-finite one makes every cost non-finite).
bool finite_state_goal(const aero_state_t* x0, const float* goal) {
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(x0->p[i]) || !std::isfinite(x0->v[i]) || !std::isfinite(goal[i])) return false;
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(x0->q[i])) return false;
  return true;
}

template <typename T>
cudaError_t alloc(T** p, size_t count) {
  return dev_malloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

void free_all(aero_planner* pl) {
  void* ptrs[] = {pl->keys,     pl->coarse_win, pl->cells,        pl->anchors,  pl->guides,
                  pl->item_flag, pl->grid_count, pl->grid_fill, pl->grid_local, pl->tile_sum,
                  pl->tile_off,
                  pl->cand,     pl->cand_pts,   pl->grid_range, pl->partials,
                  pl->sample_costs, pl->stage2_x, pl->counter,   pl->status,   pl->dbg_u,
                  pl->dbg_x,    pl->dbg_d,      pl->stage_cloud,      pl->stage_out,
                  pl->dbg_pre,      pl->part_counts,  pl->d_tab,  pl->warm};
  for (void* q : ptrs) dev_free(q);
  host_free(pl->h_out);
}

constexpr size_t kProfSlots = 512;

// Fold the recorded stage times into the accumulators (synchronises the events).
cudaError_t prof_fold(aero_planner* pl) {
  for (size_t i = 0; i < pl->slots_used; ++i) {
    aero_planner::ProfSlot& sl = pl->slots[i];
    if (sl.last < 0) continue;
    cudaError_t e = cudaEventSynchronize(sl.ev[sl.last]);
    if (e != cudaSuccess) return e;
    auto add = [&](int stage, int a, int b) {
      if (!(sl.mask & (1 << stage))) return;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, sl.ev[a], sl.ev[b]);
      pl->prof_ms[stage] += ms;
    };
    add(AERO_STAGE_PARTITION, 0, 1);
    add(AERO_STAGE_GRID, 2, 3);
    for (int it = 0; it < sl.iters; ++it) {
      add(AERO_STAGE_ROLLOUT, 4 + 4 * it, 5 + 4 * it);
      add(AERO_STAGE_UPDATE, 6 + 4 * it, 7 + 4 * it);
    }
    for (int k = 0; k < AERO_STAGE_COUNT; ++k)
      if (sl.mask & (1 << k)) pl->prof_launches[k] += sl.launches[k];
  }
  pl->slots_used = 0;
  return cudaSuccess;
}

// A slot with 4 + 4 iters events, or nullptr when profiling is off.
aero_planner::ProfSlot* prof_slot(aero_planner* pl, int iters) {
  if (!pl->prof) return nullptr;
  if (pl->slots_used == kProfSlots && prof_fold(pl) != cudaSuccess) return nullptr;
  if (pl->slots.size() < kProfSlots) pl->slots.resize(kProfSlots);
  aero_planner::ProfSlot& sl = pl->slots[pl->slots_used];
  const size_t need = 4 + 4 * (size_t)iters;
  while (sl.ev.size() < need) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
    sl.ev.push_back(ev);
  }
  sl.iters = iters;
  sl.mask = pl->prof;
  sl.last = -1;
  for (int k = 0; k < AERO_STAGE_COUNT; ++k) sl.launches[k] = 0;
  ++pl->slots_used;
  return &sl;
}

void prof_destroy(aero_planner* pl) {
  for (auto& sl : pl->slots)
    for (cudaEvent_t ev : sl.ev) cudaEventDestroy(ev);
  pl->slots.clear();
  pl->slots_used = 0;
}

// Every kernel argument of one step of planner `pl`.
struct StepArgs {
  PartTables tab;
  int check_lo = 0, check_hi = 0;
  PartitionArgs pa{};
  CandArgs ca{};
  GuideArgs ga{};
  RolloutArgs ra{};  // ctr3 = step_id << 8; the iteration is ored in at launch
  UpdateArgs ua{};
  GridGeom grid{};
  int ncell = 0, gcells = 0, ntiles = 0, nb = 0, lanes = 1;
  int64_t n_items = 0;
  bool raw = false;
};

// Lanes per sample of a step: the explicit choice, else four when E*K is at
// most `quad_max`.
int lanes_of(const aero_params_t& p, int64_t quad_max) {
  if (p.lanes_per_sample != 0) return p.lanes_per_sample;
  return (int64_t)p.E * p.K <= quad_max ? 4 : 1;
}

void make_step_args(aero_planner* pl, const aero_state_t* x0, const float* cloud, int64_t n,
                    const float* goal, const aero_params_t& p, float* u_nom, float* u_best,
                    float* cand, int32_t* best_idx, int lanes, bool coarse, bool idx_entries,
                    StepArgs& a, int samples_per_cta = kRolloutThreads) {
  a.ncell = p.fine_az * p.fine_el;
  // the edge tables depend only on the partition geometry: recomputed when it changes
  if (!pl->tab_valid || pl->tab_A != p.fine_az || pl->tab_El != p.fine_el || pl->tab_lo != p.el_lo ||
      pl->tab_hi != p.el_hi) {
    make_tables(p, pl->tab, pl->tab_check_lo, pl->tab_check_hi);
    pl->tab_valid = true;
    pl->tab_upload = true;
    pl->tab_A = p.fine_az;
    pl->tab_El = p.fine_el;
    pl->tab_lo = p.el_lo;
    pl->tab_hi = p.el_hi;
  }
  a.tab = pl->tab;
  a.check_lo = pl->tab_check_lo;
  a.check_hi = pl->tab_check_hi;
  float R[9];
  rot_f32(x0->q, R);
  const float rm = p.r_max;
  const float rmax2 = rm * rm;
  a.raw = p.collision_set == 1;
  a.n_items = a.raw ? n : a.ncell;
  a.grid = make_grid(p, a.n_items, pl->cand_cap, pl->grid_max, coarse);
  a.gcells = a.grid.G * a.grid.G * a.grid.G;
  a.ntiles = (a.gcells + 1 + kScanTile - 1) / kScanTile;

  PartitionArgs& pa = a.pa;
  pa.cloud = cloud;
  pa.n = n;
  for (int i = 0; i < 3; ++i) pa.p0[i] = x0->p[i];
  for (int i = 0; i < 9; ++i) pa.R[i] = R[i];
  pa.rmax2 = rmax2;
  pa.A = p.fine_az;
  pa.El = p.fine_el;
  pa.check_lo = a.check_lo;
  pa.check_hi = a.check_hi;
  pa.filter = n >= kPartFilterPointsPerCone * (int64_t)a.ncell;
  pa.el_lo = p.el_lo;
  pa.el_inv = (float)p.fine_el / (p.el_hi - p.el_lo);
  pa.keys = pl->keys;
  pa.item_flag = a.raw ? pl->item_flag : nullptr;
  pa.counts = pl->part_counts;

  CandArgs& ca = a.ca;
  ca.cloud = cloud;
  for (int i = 0; i < 3; ++i) ca.p0[i] = x0->p[i];
  ca.keys = pl->keys;
  ca.item_flag = pl->item_flag;
  ca.n_items = a.n_items;
  ca.raw = a.raw;
  ca.grid = a.grid;
  ca.count = pl->grid_count;
  ca.fill = pl->grid_fill;
  ca.local = pl->grid_local;
  ca.tile_off = pl->tile_off;
  ca.cand = idx_entries ? reinterpret_cast<uint32_t*>(pl->cand) : nullptr;
  ca.pts = idx_entries ? pl->cand_pts : nullptr;
  ca.cand4 = idx_entries ? nullptr : pl->cand;
  ca.status = pl->status;
  ca.reset_keys = nullptr;

  GuideArgs& ga = a.ga;
  ga.keys = pl->keys;
  ga.A = p.fine_az;
  ga.El = p.fine_el;
  ga.Pa = p.pool_az;
  ga.Pe = p.pool_el;
  ga.Ac = p.fine_az / p.pool_az;
  ga.Ec = p.fine_el / p.pool_el;
  ga.rmax2 = rmax2;
  ga.el_lo = p.el_lo;
  ga.el_hi = p.el_hi;
  for (int i = 0; i < 9; ++i) ga.R[i] = R[i];
  for (int i = 0; i < 3; ++i) ga.goal_rel[i] = goal[i] - x0->p[i];
  ga.M_h = p.M_h;
  ga.M_v = p.M_v;
  ga.E = p.E;
  ga.ell = p.ell;
  ga.T = p.T;
  ga.dt = p.dt;
  ga.v_end = p.v_end;
  for (int i = 0; i < 3; ++i) ga.v0[i] = x0->v[i];
  ga.coarse_win = pl->coarse_win;
  ga.cells = pl->cells;
  ga.anchors = pl->anchors;
  ga.guides = pl->guides;

  CostParams cp{};
  cp.Q_track = p.Q_track;
  cp.Q_vnorm = p.Q_vnorm;
  cp.Q_c = p.Q_c;
  cp.Q_cd = p.Q_cd;
  cp.Q_p = p.Q_p;
  cp.Q_v = p.Q_v;
  cp.Q_q = p.Q_q;
  cp.C_col = p.C_col;
  cp.a_col = p.a_col;
  cp.d_min = p.d_min;
  cp.d_max = p.d_max;
  for (int i = 0; i < 3; ++i) cp.goal_rel[i] = goal[i] - x0->p[i];
  for (int i = 0; i < 3; ++i) cp.v_goal[i] = p.v_goal[i];
  for (int i = 0; i < 4; ++i) cp.q_goal[i] = p.q_goal[i];
  DynParams dp{p.dt, 1.0f / p.mass, p.g};
  GridView gv{pl->grid_range, ca.cand, idx_entries ? pl->cand_pts : pl->cand, a.grid.G, a.grid.origin,
              a.grid.inv_h};
  const float x0v[10] = {0.0f, 0.0f, 0.0f, x0->q[0], x0->q[1], x0->q[2], x0->q[3],
                         x0->v[0], x0->v[1], x0->v[2]};
  a.lanes = lanes;
  // samples per Stage I CTA: 32 in the split pass, else the one-lane pass's CTA size
  const int per_cta = lanes == 4 ? kRolloutThreads / 4 : samples_per_cta;
  a.nb = (p.K + per_cta - 1) / per_cta;

  RolloutArgs& ra = a.ra;
  ra.E = p.E;
  ra.K = p.K;
  ra.T = p.T;
  ra.nb = a.nb;
  ra.lanes_per_sample = lanes;
  // every kept point as the collision set: lists of tens to hundreds of
  // entries, uneven across a warp's queries; P_f's are short (a few entries)
  ra.list_thr = a.raw ? kWarpListThreshold : 0;
  ra.inv_lambda = 1.0f / p.lambda;
  for (int c = 0; c < 4; ++c) {
    ra.sigma[c] = p.sigma[c];
    ra.umin[c] = p.u_min[c];
    ra.umax[c] = p.u_max[c];
  }
  for (int i = 0; i < 10; ++i) ra.x0[i] = x0v[i];
  ra.key0 = (uint32_t)p.seed;
  ra.key1 = (uint32_t)(p.seed >> 32);
  for (int r = 0; r < 10; ++r) {  // Philox4x32-10's key schedule (32-bit wrap-around)
    ra.rk[2 * r] = ra.key0 + (uint32_t)r * 0x9E3779B9u;
    ra.rk[2 * r + 1] = ra.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  ra.ctr3 = (uint32_t)(p.step_id << 8);
  ra.dyn = dp;
  ra.cost = cp;
  ra.u_nom = u_nom;
  ra.guides = pl->guides;
  ra.grid = gv;
  ra.partials = pl->partials;
  ra.sample_costs = pl->sample_costs;
  ra.dbg_D = p.debug_samples < p.K ? p.debug_samples : p.K;
  ra.dbg_u = pl->dbg_u;
  ra.dbg_x = pl->dbg_x;
  ra.dbg_d = pl->dbg_d;

  UpdateArgs& ua = a.ua;
  ua.E = p.E;
  ua.T = p.T;
  ua.nb = a.nb;
  ua.inv_lambda = ra.inv_lambda;
  ua.partials = pl->partials;
  ua.u_nom = u_nom;
  for (int i = 0; i < 10; ++i) ua.x0[i] = x0v[i];
  ua.dyn = dp;
  ua.cost = cp;
  ua.grid = gv;
  ua.stage2_x = pl->stage2_x;
  ua.guides = pl->guides;
  for (int c = 0; c < 4; ++c) {
    ua.umin[c] = p.u_min[c];
    ua.umax[c] = p.u_max[c];
  }
  ua.refine_steps = p.refine_steps;
  ua.refine_step = p.refine_step;
  ua.dbg_pre = p.refine_steps > 0 ? pl->dbg_pre : nullptr;
  ua.cand = cand;
  ua.best_idx = best_idx;
  ua.u_best = u_best;
  ua.counter = pl->counter;
  ua.inst_counter = pl->counter + 3;
  ua.status = pl->status;
  ua.warm = pl->warm;
  ua.done = pl->warm != nullptr ? pl->counter + kDoneWord : nullptr;
  ra.done = ua.done;
}

// The planner's state after a step has been enqueued.
void note_step(aero_planner* pl, const aero_params_t& p, const StepArgs& a) {
  pl->last_ctx = a.ua;
  pl->grid_dirty = false;
  pl->have_step = true;
  pl->last = p;
  pl->last_grid = a.grid;
  pl->last_idx_entries = a.ca.cand != nullptr;
  pl->last_ntiles = a.ntiles;
  pl->last_nb = a.nb;
  pl->last_part_slots = partition_blocks(a.pa.n);
  pl->last_n_points = a.pa.n;
}

// NVTX ranges, one per stage, around the host's enqueue of a step (checked
// build only; a no-op in the product build): next() closes the open range and
// opens the next one, the destructor closes the last.
struct StageRanges {
#ifdef AERO_CHECKED
  bool open = false;
  void next(const char* name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~StageRanges() {
    if (open) nvtxRangePop();
  }
#else
  void next(const char*) {}
#endif
};

// Enqueue one step; all pointers already validated.  mapped: null, or the
// device address of the cloud in page-locked host memory; the partition then
// reads the points from there and stores them at `cloud` (a device array),
// which the later passes read.
int enqueue_step(aero_planner* pl, const aero_state_t* x0, const float* cloud, int64_t n,
                 const float* goal, const aero_params_t& p, float* u_nom, float* u_best,
                 float* cand, int32_t* best_idx, cudaStream_t s, const float* mapped = nullptr) {
  StepArgs a;
  make_step_args(pl, x0, cloud, n, goal, p, u_nom, u_best, cand, best_idx,
                 lanes_of(p, kQuadMaxSamples), false, true, a);
  if (mapped) {
    a.pa.cloud = mapped;
    a.pa.copy_to = const_cast<float*>(cloud);
  }

  cudaError_t e;
  aero_planner::ProfSlot* prof = prof_slot(pl, p.iters);
  // event i of the slot, recorded only when its stage is timed
  auto mark = [&](int stage, int i) {
    if (prof && (prof->mask & (1 << stage))) {
      cudaEventRecord(prof->ev[i], s);
      prof->last = i;
    }
  };
  StageRanges ranges;
  ranges.next("aero partition");
  mark(AERO_STAGE_PARTITION, 0);
  // A planner without debug buffers keeps its keys empty between steps (the
  // scatter pass empties each key it reads), so a step needs no fill; one with
  // debug buffers fills before the step and keeps the keys for aero_get_debug.
  const bool reset = pl->lim.debug_samples_max == 0 && !a.raw;
  if (!(reset && pl->keys_empty)) {
    const size_t nk = reset ? (size_t)pl->lim.fine_cells_max : (size_t)a.ncell;
    if ((e = cudaMemsetAsync(pl->keys, 0xFF, sizeof(unsigned long long) * nk, s)) != cudaSuccess)
      return cuda_fail(e);
  }
  pl->keys_empty = false;
  if (reset) a.ca.reset_keys = pl->keys;
  if (pl->grid_dirty) {
    // the scan leaves the counts at zero; clear them only when a step may have
    // stopped between the count pass and the scan
    if ((e = cudaMemsetAsync(pl->grid_count, 0, sizeof(int) * (pl->grid_cells_cap + 1), s)) !=
        cudaSuccess)
      return cuda_fail(e);
  }
  pl->grid_dirty = true;

  if (pl->tab_upload) {
    if ((e = cudaMemcpyAsync(pl->d_tab, &pl->tab, sizeof(PartTables), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      return cuda_fail(e);
    pl->tab_upload = false;
  }
  if ((e = launch_partition(a.pa, pl->d_tab, s)) != cudaSuccess) return cuda_fail(e);
  mark(AERO_STAGE_PARTITION, 1);
  ranges.next("aero grid");
  mark(AERO_STAGE_GRID, 2);
  if (prof) {
    prof->launches[AERO_STAGE_PARTITION] = n > 0 ? 1 : 0;
    prof->launches[AERO_STAGE_GRID] = 3;
    prof->launches[AERO_STAGE_ROLLOUT] = p.iters;
    prof->launches[AERO_STAGE_UPDATE] = rollout_runs_update(a.ra) ? 0 : p.iters;
  }
  // count pass + coarse argmax, scan + goal cone/anchors/guides, scatter + cell ranges
  if ((e = launch_grid_count(a.ca, a.ga, s)) != cudaSuccess) return cuda_fail(e);
  if ((e = launch_grid_scan(pl->grid_count, pl->grid_fill, pl->grid_local, pl->tile_sum,
                            pl->tile_off, a.gcells + 1, a.ntiles, nullptr, a.ga, pl->d_tab, s)) !=
      cudaSuccess)
    return cuda_fail(e);
  if ((e = launch_grid_scatter(a.ca, pl->grid_range, a.gcells, pl->tile_sum, pl->tile_off,
                               a.ntiles, s)) != cudaSuccess)
    return cuda_fail(e);
  mark(AERO_STAGE_GRID, 3);

  const uint32_t ctr_base = a.ra.ctr3;
  for (int it = 0; it < p.iters; ++it) {
    a.ra.ctr3 = ctr_base | (uint32_t)it;
    a.ua.final_stage = it == p.iters - 1;
    ranges.next("aero stage I");
    mark(AERO_STAGE_ROLLOUT, 4 + 4 * it);
    if ((e = launch_rollout(a.ra, a.ua, s)) != cudaSuccess) return cuda_fail(e);
    mark(AERO_STAGE_ROLLOUT, 5 + 4 * it);
    ranges.next("aero update");
    mark(AERO_STAGE_UPDATE, 6 + 4 * it);
    if (!rollout_runs_update(a.ra) && (e = launch_update(a.ua, s)) != cudaSuccess) return cuda_fail(e);
    mark(AERO_STAGE_UPDATE, 7 + 4 * it);
  }
  note_step(pl, p, a);
  pl->keys_empty = reset;
  return AERO_OK;
}

int create_planner(const aero_limits_t* limits, aero_planner_t** out, bool batch_slot);

}  // namespace

extern "C" {

void aero_params_default(aero_params_t* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->E = 15;
  p->K = 128;
  p->T = 25;
  p->iters = 1;
  p->dt = 0.05f;
  p->lambda = 0.1f;
  p->mass = 1.0f;
  p->g = 9.81f;
  const float sig[4] = {1.0f, 1.0f, 1.0f, 0.70710678f};
  const float lo[4] = {0.3f, -3.0f, -3.0f, -2.0f};
  const float hi[4] = {16.35f, 3.0f, 3.0f, 2.0f};
  for (int c = 0; c < 4; ++c) {
    p->sigma[c] = sig[c];
    p->u_min[c] = lo[c];
    p->u_max[c] = hi[c];
  }
  p->Q_track = 15.0f;
  p->Q_vnorm = 0.15f;
  p->Q_c = 0.5f;
  p->Q_cd = 0.5f;
  p->Q_p = 3.0f;
  p->Q_v = 0.25f;
  p->Q_q = 1.0f;
  p->C_col = 1.0e6f;
  p->a_col = 5.0f;
  p->d_min = 0.4f;
  p->d_max = 1.0f;
  p->r_max = 10.0f;
  p->ell = 5.0f;
  p->v_end = 0.0f;
  p->fine_az = 120;
  p->fine_el = 60;
  p->pool_az = 6;
  p->pool_el = 6;
  p->M_h = 5;
  p->M_v = 3;
  p->el_lo = -1.57079637f;
  p->el_hi = 1.57079637f;
  p->collision_set = 0;
  p->q_goal[0] = 1.0f;
  p->debug_samples = 0;
  p->seed = 0;
  p->step_id = 0;
  p->refine_steps = 0;
  p->refine_step = 0.05f;
}

int aero_create(const aero_limits_t* limits, aero_planner_t** out) {
  return create_planner(limits, out, false);
}

}  // extern "C"

namespace {

// batch_slot: the workspace of a batch's item slot, whose candidate entries
// hold the points (16 bytes); a single planner's entries are 4-byte item
// indices, so the same bytes hold four times the entries and the every-point
// set gets room for the finer cells (216 entries per kept point).
int create_planner(const aero_limits_t* limits, aero_planner_t** out, bool batch_slot) {
  if (!limits || !out) return AERO_ERR_INVALID_ARG;
  *out = nullptr;
  const aero_limits_t& L = *limits;
  if (L.E_max < 1 || L.E_max > kMaxE || L.K_max < 1 || L.K_max > (1 << 20) || L.T_max < 1 ||
      L.T_max > kMaxT || L.fine_cells_max < 2 || L.fine_cells_max > kMaxAz * kMaxEl ||
      L.n_points_max < 0 || L.n_points_max > 0x7FFFFFFFLL || L.debug_samples_max < 0 ||
      L.debug_samples_max > L.K_max || L.raw_points_max < -1 || L.raw_points_max > L.n_points_max)
    return AERO_ERR_INVALID_ARG;
  aero_planner* pl = new (std::nothrow) aero_planner();
  if (!pl) return AERO_ERR_ALLOC;
  pl->lim = L;
  pl->raw_max = L.raw_points_max == 0 ? L.n_points_max : (L.raw_points_max < 0 ? 0 : L.raw_points_max);
  cudaGetDevice(&pl->device);
  // partial rows: one per rollout CTA, whose smallest sample count is 128 / 4
  const int64_t nbmax = (L.K_max + kRolloutThreads / 4 - 1) / (kRolloutThreads / 4);
  const int64_t cap_fine = (int64_t)kFineDup * L.fine_cells_max;
  const int64_t cap_raw = (int64_t)(batch_slot ? kCoarseDup : kFineDup) * pl->raw_max;
  int64_t cap = cap_fine > cap_raw ? cap_fine : cap_raw;
  if (cap > 0x7FFFFFFFLL) cap = 0x7FFFFFFFLL;
  pl->cand_cap = (int)cap;
  const int64_t D = L.debug_samples_max;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (r != cudaSuccess && e == cudaSuccess) e = r;
  };
  chk(alloc(&pl->keys, L.fine_cells_max));
  chk(alloc(&pl->coarse_win, L.fine_cells_max));
  chk(alloc(&pl->cells, L.E_max + 1));
  chk(alloc(&pl->anchors, L.E_max * 3));
  chk(alloc(&pl->guides, (size_t)L.E_max * L.T_max * 3));
  chk(alloc(&pl->item_flag, pl->raw_max));
  chk(alloc(&pl->grid_count, kGridCellsMax + 1));
  chk(alloc(&pl->grid_fill, kGridCellsMax + 1));
  chk(alloc(&pl->grid_local, kGridCellsMax + 1));
  chk(alloc(&pl->tile_sum, kMaxTiles));
  chk(alloc(&pl->tile_off, kMaxTiles + 1));
  chk(dev_malloc((void**)&pl->cand, (batch_slot ? sizeof(float4) : sizeof(uint32_t)) * (size_t)(cap > 0 ? cap : 1)));
  chk(alloc(&pl->cand_pts, std::max<int64_t>(L.fine_cells_max, pl->raw_max)));
  chk(alloc(&pl->grid_range, kGridCellsMax));
  chk(alloc(&pl->partials, (size_t)L.E_max * nbmax * (4 + 4 * L.T_max)));
  chk(alloc(&pl->sample_costs, (size_t)L.E_max * L.K_max));
  chk(alloc(&pl->stage2_x, (size_t)L.E_max * (L.T_max + 1) * 10));
  chk(alloc(&pl->counter, kCounterWords));
  chk(alloc(&pl->status, 1));
  if (!batch_slot) chk(alloc(&pl->warm, (size_t)L.E_max * warm_words(L.E_max, L.T_max)));
  chk(alloc(&pl->dbg_u, (size_t)L.E_max * D * L.T_max * 4));
  chk(alloc(&pl->dbg_x, (size_t)L.E_max * D * (L.T_max + 1) * 10));
  chk(alloc(&pl->dbg_d, (size_t)L.E_max * D * L.T_max));
  chk(alloc(&pl->dbg_pre, (size_t)L.E_max * L.T_max * 4));
  // one count pair per partition block (single step) or chunk of points (batched)
  pl->part_slots = (int)std::max<int64_t>(kPartBlocksMax, (L.n_points_max + kPartChunk - 1) / kPartChunk);
  chk(alloc(&pl->part_counts, pl->part_slots));
  chk(alloc(&pl->stage_cloud, (size_t)L.n_points_max * 3));
  const size_t out_words = (size_t)L.E_max * L.T_max * 4 + (size_t)L.T_max * 4 + L.E_max + 1;
  chk(alloc(&pl->stage_out, out_words));
  chk(alloc(&pl->d_tab, 1));
  chk(host_malloc((void**)&pl->h_out, sizeof(float) * out_words));
  if (e == cudaSuccess) e = split_attributes();
  if (e == cudaSuccess) e = cudaMemset(pl->counter, 0, kCounterWords * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(pl->status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_all(pl);
    delete pl;
    return e == cudaErrorMemoryAllocation ? AERO_ERR_ALLOC : AERO_ERR_CUDA;
  }
  *out = pl;
  return AERO_OK;
}

}  // namespace

extern "C" {

int aero_test_fail_alloc(int64_t n) {
  g_alloc_fail_after.store(n < 0 ? -1 : n);
  return AERO_OK;
}

int aero_test_raise_check(int32_t bits) {
  if (bits <= 0) return AERO_ERR_INVALID_ARG;
  const cudaError_t e = raise_check_partition(bits);
  if (e == cudaErrorNotSupported) return AERO_ERR_INVALID_ARG;
  return e == cudaSuccess ? AERO_OK : AERO_ERR_CUDA;
}

int64_t aero_test_alloc_stats(int64_t* live) {
  if (live) *live = g_alloc_live.load();
  return g_alloc_total.load();
}

int aero_destroy(aero_planner_t* pl) {
  if (!pl) return AERO_OK;
  cudaDeviceSynchronize();
  prof_destroy(pl);
  free_all(pl);
  delete pl;
  return AERO_OK;
}

int aero_plan_step(aero_planner_t* pl, const aero_state_t* x0, const float* cloud, int64_t n,
                   const float goal[3], const aero_params_t* params, float* u_nom, float* u_best,
                   float* cand, int32_t* best_idx, void* stream) {
  if (!pl || !x0 || !goal || !params || !u_nom || !u_best || !cand || !best_idx)
    return AERO_ERR_INVALID_ARG;
  if (n > 0 && !cloud) return AERO_ERR_INVALID_ARG;
  if (!finite_state_goal(x0, goal)) return AERO_ERR_INVALID_ARG;
  int rc = validate(pl, params, n);
  if (rc != AERO_OK) return rc;
  if (reinterpret_cast<uintptr_t>(u_nom) % 16 != 0) return AERO_ERR_INVALID_ARG;
  if ((n > 0 && !is_device_ptr(cloud)) || !is_device_ptr(u_nom) || !is_device_ptr(u_best) ||
      !is_device_ptr(cand) || !is_device_ptr(best_idx))
    return AERO_ERR_NOT_DEVICE_PTR;
  return enqueue_step(pl, x0, cloud, n, goal, *params, u_nom, u_best, cand, best_idx,
                      (cudaStream_t)stream);
}

int aero_plan_step_host(aero_planner_t* pl, const aero_state_t* x0, const float* cloud, int64_t n,
                        const float goal[3], const aero_params_t* params, float* u_nom,
                        float* u_best, float* cand, int32_t* best_idx, void* stream) {
  if (!pl || !x0 || !goal || !params || !u_nom || !u_best || !cand || !best_idx)
    return AERO_ERR_INVALID_ARG;
  if (n > 0 && !cloud) return AERO_ERR_INVALID_ARG;
  if (!finite_state_goal(x0, goal)) return AERO_ERR_INVALID_ARG;
  int rc = validate(pl, params, n);
  if (rc != AERO_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nu = (size_t)params->E * params->T * 4;
  cudaError_t e;
  // a cloud in page-locked host memory is read by the partition itself (over
  // the host link, overlapped with its arithmetic); any other is copied first
  const float* mapped = nullptr;
  if (n > 0) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, cloud) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer != nullptr)
      mapped = static_cast<const float*>(at.devicePointer);
    else
      cudaGetLastError();  // an unregistered pointer is not an error here
  }
  if (n > 0 && !mapped &&
      (e = cudaMemcpyAsync(pl->stage_cloud, cloud, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
    return cuda_fail(e);
  // outputs laid out back to back (each part stays 16-byte aligned)
  const size_t nb = (size_t)params->T * 4, ne = (size_t)params->E;
  float* d_unom = pl->stage_out;
  float* d_ubest = d_unom + nu;
  float* d_cand = d_ubest + nb;
  int32_t* d_best = reinterpret_cast<int32_t*>(d_cand + ne);
  if ((e = cudaMemcpyAsync(d_unom, u_nom, sizeof(float) * nu, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(e);
  rc = enqueue_step(pl, x0, pl->stage_cloud, n, goal, *params, d_unom, d_ubest, d_cand, d_best, s,
                    mapped);
  if (rc != AERO_OK) return rc;
  const size_t words = nu + nb + ne + 1;
  if ((e = cudaMemcpyAsync(pl->h_out, pl->stage_out, sizeof(float) * words, cudaMemcpyDeviceToHost,
                           s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e);
  std::memcpy(u_nom, pl->h_out, sizeof(float) * nu);
  std::memcpy(u_best, pl->h_out + nu, sizeof(float) * nb);
  std::memcpy(cand, pl->h_out + nu + nb, sizeof(float) * ne);
  std::memcpy(best_idx, pl->h_out + nu + nb + ne, sizeof(int32_t));
  return AERO_OK;
}

size_t aero_debug_size(aero_planner_t* pl, int32_t what) {
  if (!pl || !pl->have_step) return 0;
  const aero_params_t& p = pl->last;
  const size_t E = p.E, T = p.T, K = p.K;
  const size_t D = p.debug_samples < p.K ? p.debug_samples : p.K;
  const size_t G = pl->last_grid.G;
  switch (what) {
    case AERO_DBG_FINE_KEYS:  // kept by planners with debug buffers only
      return pl->lim.debug_samples_max > 0 ? 8 * (size_t)p.fine_az * p.fine_el : 0;
    case AERO_DBG_COARSE_WIN: return 4 * (size_t)(p.fine_az / p.pool_az) * (p.fine_el / p.pool_el);
    case AERO_DBG_GOAL_CELL: return 4;
    case AERO_DBG_ANCHOR_CELLS: return 4 * E;
    case AERO_DBG_ANCHORS: return 4 * E * 3;
    case AERO_DBG_GUIDES: return 4 * E * T * 3;
    case AERO_DBG_GRID_META: return 32;
    case AERO_DBG_GRID_START: return 4 * (G * G * G + 1);  // computed on the host
    case AERO_DBG_GRID_POINTS: return 0;  // size known after the step; see aero_get_debug
    case AERO_DBG_SAMPLE_COSTS: return 4 * E * K;
    case AERO_DBG_STAGE2_STATES: return 4 * E * (T + 1) * 10;
    case AERO_DBG_SAMPLE_U: return 4 * E * D * T * 4;
    case AERO_DBG_SAMPLE_X: return 4 * E * D * (T + 1) * 10;
    case AERO_DBG_SAMPLE_DIST: return 4 * E * D * T;
    case AERO_DBG_PRE_REFINE: return p.refine_steps > 0 ? 4 * E * T * 4 : 0;
    case AERO_DBG_POINT_COUNTS: return 3 * sizeof(int64_t);
    default: return 0;
  }
}

int aero_get_debug(aero_planner_t* pl, int32_t what, void* dst, size_t bytes, void* stream) {
  if (!pl || !dst || !pl->have_step || what < 0 || what >= AERO_DBG_COUNT) return AERO_ERR_INVALID_ARG;
  if (what == AERO_DBG_FINE_KEYS && pl->lim.debug_samples_max == 0) return AERO_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const aero_params_t& p = pl->last;
  if (what == AERO_DBG_GRID_META || what == AERO_DBG_GRID_POINTS || what == AERO_DBG_GRID_START) {
    // synchronous: the number of candidate entries and the cell starts are
    // assembled on the host
    const GridGeom& g = pl->last_grid;
    const int gcells = g.G * g.G * g.G;
    int32_t n_entries = 0;
    cudaError_t e = cudaMemcpyAsync(&n_entries, pl->tile_off + pl->last_ntiles, 4,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (what == AERO_DBG_GRID_META) {
      if (bytes < 32) return AERO_ERR_INVALID_ARG;
      int32_t meta[8] = {g.G, n_entries, g.cap, 0, 0, 0, 0, 0};
      const float f[3] = {g.origin, g.h, g.reach};
      std::memcpy(&meta[4], f, sizeof(f));
      return cuda_fail(cudaMemcpy(dst, meta, 32, cudaMemcpyDefault));
    }
    if (what == AERO_DBG_GRID_POINTS) {
      // the entries' points, gathered on the host
      const size_t ne = (size_t)(n_entries < g.cap ? n_entries : g.cap);
      const size_t need = sizeof(float4) * ne;
      if (bytes < need) return AERO_ERR_INVALID_ARG;
      if (!pl->last_idx_entries) return cuda_fail(cudaMemcpy(dst, pl->cand, need, cudaMemcpyDefault));
      const size_t n_items = (size_t)std::max<int64_t>(pl->lim.fine_cells_max, pl->raw_max);
      std::vector<uint32_t> idx(ne);
      std::vector<float4> pts(n_items), out(ne);
      e = cudaMemcpy(idx.data(), pl->cand, 4 * ne, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(pts.data(), pl->cand_pts, sizeof(float4) * n_items, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e);
      for (size_t i = 0; i < ne; ++i) {
        if (idx[i] >= n_items) return AERO_ERR_DEVICE_CHECK;
        out[i] = pts[idx[i]];
      }
      return cuda_fail(cudaMemcpy(dst, out.data(), need, cudaMemcpyDefault));
    }
    const size_t need = sizeof(int32_t) * ((size_t)gcells + 1);
    if (bytes < need) return AERO_ERR_INVALID_ARG;
    std::vector<int32_t> local((size_t)gcells + 1), off((size_t)pl->last_ntiles + 1);
    e = cudaMemcpy(local.data(), pl->grid_local, need, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(off.data(), pl->tile_off, 4 * off.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    for (size_t c = 0; c <= (size_t)gcells; ++c) local[c] += off[c >> kScanTileShift];
    return cuda_fail(cudaMemcpy(dst, local.data(), need, cudaMemcpyDefault));
  }
  if (what == AERO_DBG_POINT_COUNTS) {
    // synchronous: the per-block counts are summed on the host
    if (bytes < 3 * sizeof(int64_t)) return AERO_ERR_INVALID_ARG;
    std::vector<int2> c((size_t)pl->last_part_slots);
    cudaError_t e = cudaSuccess;
    if (!c.empty())
      e = cudaMemcpyAsync(c.data(), pl->part_counts, sizeof(int2) * c.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    int64_t out[3] = {pl->last_n_points, 0, 0};
    for (const int2& v : c) {
      out[1] += v.x;
      out[2] += v.y;
    }
    return cuda_fail(cudaMemcpy(dst, out, sizeof(out), cudaMemcpyDefault));
  }
  const size_t need = aero_debug_size(pl, what);
  if (bytes < need) return AERO_ERR_INVALID_ARG;
  const void* src = nullptr;
  switch (what) {
    case AERO_DBG_FINE_KEYS: src = pl->keys; break;
    case AERO_DBG_COARSE_WIN: src = pl->coarse_win; break;
    case AERO_DBG_GOAL_CELL: src = pl->cells; break;
    case AERO_DBG_ANCHOR_CELLS: src = pl->cells + 1; break;
    case AERO_DBG_ANCHORS: src = pl->anchors; break;
    case AERO_DBG_GUIDES: src = pl->guides; break;
    case AERO_DBG_SAMPLE_COSTS: src = pl->sample_costs; break;
    case AERO_DBG_STAGE2_STATES: src = pl->stage2_x; break;
    case AERO_DBG_SAMPLE_U: src = pl->dbg_u; break;
    case AERO_DBG_SAMPLE_X: src = pl->dbg_x; break;
    case AERO_DBG_SAMPLE_DIST: src = pl->dbg_d; break;
    case AERO_DBG_PRE_REFINE: src = pl->dbg_pre; break;
    default: return AERO_ERR_INVALID_ARG;
  }
  (void)p;
  if (need == 0) return AERO_OK;
  return cuda_fail(cudaMemcpyAsync(dst, src, need, cudaMemcpyDefault, s));
}

int aero_sync_status(aero_planner_t* pl, void* stream) {
  if (!pl) return AERO_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, pl->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return AERO_ERR_CUDA;
  int cw = 0;
  if (read_check_words(&cw, true) != cudaSuccess) return AERO_ERR_CUDA;
  if (st != 0 || cw != 0) {
    cudaMemsetAsync(pl->status, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return AERO_ERR_DEVICE_CHECK;
  }
  return AERO_OK;
}

int aero_cost_grad(aero_planner_t* pl, int32_t instance, const float* U, int32_t n, float* S_out,
                   float* dSdU_out, void* stream) {
  if (!pl || n < 0 || (n > 0 && (!U || !S_out)) || !pl->have_step) return AERO_ERR_INVALID_ARG;
  if (instance < 0 || instance >= pl->last.E) return AERO_ERR_INVALID_ARG;
  if (n == 0) return AERO_OK;
  if (reinterpret_cast<uintptr_t>(U) % 16 != 0 ||
      (dSdU_out && reinterpret_cast<uintptr_t>(dSdU_out) % 16 != 0))
    return AERO_ERR_INVALID_ARG;
  if (!is_device_ptr(U) || !is_device_ptr(S_out) || (dSdU_out && !is_device_ptr(dSdU_out)))
    return AERO_ERR_NOT_DEVICE_PTR;
  CostGradArgs a{};
  a.ctx = pl->last_ctx;
  a.instance = instance;
  a.U = reinterpret_cast<const float4*>(U);
  a.n = n;
  a.S = S_out;
  a.G = reinterpret_cast<float4*>(dSdU_out);
  return cuda_fail(launch_cost_grad(a, (cudaStream_t)stream));
}

int aero_philox(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, int64_t n, uint32_t* out,
                void* stream) {
  if (n < 0 || n > 0xFFFFFFFFLL || (n > 0 && !out)) return AERO_ERR_INVALID_ARG;
  if (n > 0 && !is_device_ptr(out)) return AERO_ERR_NOT_DEVICE_PTR;
  return cuda_fail(launch_philox((uint32_t)seed, (uint32_t)(seed >> 32), c1, c2, c3, n, out,
                                 (cudaStream_t)stream));
}

int aero_profile_enable(aero_planner_t* pl, int stages) {
  if (!pl || stages < 0 || stages >= (1 << AERO_STAGE_COUNT)) return AERO_ERR_INVALID_ARG;
  pl->prof = stages;
  return AERO_OK;
}

int aero_profile_read(aero_planner_t* pl, double* ms, int64_t* launches) {
  if (!pl || !ms || !launches) return AERO_ERR_INVALID_ARG;
  cudaError_t e = prof_fold(pl);
  if (e != cudaSuccess) return AERO_ERR_CUDA;
  for (int k = 0; k < AERO_STAGE_COUNT; ++k) {
    ms[k] = pl->prof_ms[k];
    launches[k] = pl->prof_launches[k];
    pl->prof_ms[k] = 0.0;
    pl->prof_launches[k] = 0;
  }
  return AERO_OK;
}

const char* aero_status_str(int status) {
  switch (status) {
    case AERO_OK: return "ok";
    case AERO_ERR_INVALID_ARG: return "invalid argument";
    case AERO_ERR_EXCEEDS_LIMITS: return "size exceeds the planner's limits";
    case AERO_ERR_CUDA: return "CUDA runtime error";
    case AERO_ERR_ALLOC: return "workspace allocation failed";
    case AERO_ERR_DEVICE_CHECK: return "a kernel reported an internal inconsistency";
    case AERO_ERR_NOT_DEVICE_PTR: return "pointer is not device memory";
    default: return "unknown status";
  }
}

// ---------------------------------------------------------------------------
// Planning step without any allocation.
//
// Some callers cannot call cudaMalloc once they are running: a flight-control
// loop that must not block (an allocation can synchronise the device and take
// an unbounded time), or a host program whose device memory is all owned by its
// own pool or fixed at start-up.  aero_create allocates the planner workspace,
// so such callers use aero_plan_step_noalloc instead: its workspace is carved
// from g_noalloc_scratch, a file-scope device array that the CUDA loader sets
// up with the module and that every GPU loading this library keeps until the
// process exits.  Its size is fixed by the kNa* limits below (about 7.5 MB).
// ---------------------------------------------------------------------------
namespace {

constexpr int kNaE = 16, kNaK = 2048, kNaT = 64, kNaCells = 128 * 64;
constexpr int64_t kNaPoints = 65536;
constexpr int kNaGrid = 32, kNaGridCells = kNaGrid * kNaGrid * kNaGrid;
constexpr int kNaTiles = (kNaGridCells + 1 + kScanTile - 1) / kScanTile;
constexpr int kNaCand = 1 << 18;  // candidate entries: 27 per P_f point of 8192 cones
constexpr int kNaNb = (kNaK + kRolloutThreads / 4 - 1) / (kRolloutThreads / 4);

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kNaBytes =
    align256(8 * (size_t)kNaCells) + align256(4 * (size_t)kNaCells) + align256(4 * (kNaE + 1)) +
    align256(4 * 3 * kNaE) + align256(4 * 3 * (size_t)kNaE * kNaT) + align256(4 * (size_t)kNaPoints) +
    3 * align256(4 * ((size_t)kNaGridCells + 1)) + align256(4 * (size_t)kNaTiles) +
    align256(4 * ((size_t)kNaTiles + 1)) + align256(16 * (size_t)kNaCand) +
    align256(16 * (size_t)std::max<int64_t>(kNaCells, kNaPoints)) +
    align256(8 * (size_t)kNaGridCells) +
    align256(4 * (size_t)kNaE * kNaNb * (4 + 4 * kNaT)) + align256(4 * (size_t)kNaE * kNaK) +
    align256(4 * (size_t)kNaE * (kNaT + 1) * 10) + align256(4 * kCounterWords) +
    align256(8 * (size_t)kPartBlocksMax) + align256(sizeof(PartTables)) + align256(4);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

struct NoAllocDevice {
  bool ready = false;
  unsigned char* base = nullptr;
  // the partition's edge tables last uploaded into this device's array, and
  // their geometry: a call uploads them only when the geometry changes, from
  // this host copy, which lives as long as the process
  bool tab_valid = false;
  int tab_A = 0, tab_El = 0;
  float tab_lo = 0.0f, tab_hi = 0.0f;
  int tab_check_lo = 0, tab_check_hi = 0;
  PartTables tab{};
};
NoAllocDevice g_na_dev[64];
std::mutex g_na_mutex;

// The current device's scratch state, set up on the first call (the device
// address of the array, looked up once per device with that device current:
// host code must not use the symbol itself as an address).  A first call on a
// stream that is being captured is refused: the look-up is not a stream
// operation.
int noalloc_device(cudaStream_t s, NoAllocDevice** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return AERO_ERR_CUDA;
  NoAllocDevice& d = g_na_dev[dev];
  if (!d.ready) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
      cudaGetLastError();
      return AERO_ERR_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return AERO_ERR_INVALID_ARG;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return AERO_ERR_CUDA;
    }
    d.base = static_cast<unsigned char*>(p);
    d.ready = true;
  }
  *out = &d;
  return AERO_OK;
}

// Point the planner's workspace fields into the scratch array.
void noalloc_carve(unsigned char* base, aero_planner& pl) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += align256(bytes);
    return p;
  };
  pl.keys = reinterpret_cast<unsigned long long*>(take(8 * (size_t)kNaCells));
  pl.coarse_win = reinterpret_cast<int*>(take(4 * (size_t)kNaCells));
  pl.cells = reinterpret_cast<int*>(take(4 * (kNaE + 1)));
  pl.anchors = reinterpret_cast<float*>(take(4 * 3 * kNaE));
  pl.guides = reinterpret_cast<float*>(take(4 * 3 * (size_t)kNaE * kNaT));
  pl.item_flag = reinterpret_cast<int*>(take(4 * (size_t)kNaPoints));
  pl.grid_count = reinterpret_cast<int*>(take(4 * ((size_t)kNaGridCells + 1)));
  pl.grid_fill = reinterpret_cast<int*>(take(4 * ((size_t)kNaGridCells + 1)));
  pl.grid_local = reinterpret_cast<int*>(take(4 * ((size_t)kNaGridCells + 1)));
  pl.tile_sum = reinterpret_cast<int*>(take(4 * (size_t)kNaTiles));
  pl.tile_off = reinterpret_cast<int*>(take(4 * ((size_t)kNaTiles + 1)));
  pl.cand = reinterpret_cast<float4*>(take(16 * (size_t)kNaCand));
  pl.cand_pts = reinterpret_cast<float4*>(take(16 * (size_t)std::max<int64_t>(kNaCells, kNaPoints)));
  pl.grid_range = reinterpret_cast<int2*>(take(8 * (size_t)kNaGridCells));
  pl.cand_cap = kNaCand;
  pl.grid_max = kNaGrid;
  pl.grid_cells_cap = kNaGridCells;
  pl.partials = reinterpret_cast<float*>(take(4 * (size_t)kNaE * kNaNb * (4 + 4 * kNaT)));
  pl.sample_costs = reinterpret_cast<float*>(take(4 * (size_t)kNaE * kNaK));
  pl.stage2_x = reinterpret_cast<float*>(take(4 * (size_t)kNaE * (kNaT + 1) * 10));
  pl.counter = reinterpret_cast<unsigned int*>(take(4 * kCounterWords));
  pl.part_counts = reinterpret_cast<int2*>(take(8 * (size_t)kPartBlocksMax));
  pl.d_tab = reinterpret_cast<PartTables*>(take(sizeof(PartTables)));
  pl.part_slots = kPartBlocksMax;
  pl.status = reinterpret_cast<int*>(take(4));
}

}  // namespace

int aero_plan_step_noalloc(const aero_state_t* x0, const float* cloud, int64_t n,
                           const float goal[3], const aero_params_t* params, float* u_nom,
                           float* u_best, float* cand, int32_t* best_idx, void* stream) {
  if (!x0 || !goal || !params || !u_nom || !u_best || !cand || !best_idx) return AERO_ERR_INVALID_ARG;
  if (n > 0 && !cloud) return AERO_ERR_INVALID_ARG;
  aero_planner pl;  // host-side bookkeeping only; no device memory is allocated
  pl.lim.E_max = kNaE;
  pl.lim.K_max = kNaK;
  pl.lim.T_max = kNaT;
  pl.lim.fine_cells_max = kNaCells;
  pl.lim.n_points_max = kNaPoints;
  pl.lim.debug_samples_max = 0;
  pl.raw_max = kNaPoints;
  if (!finite_state_goal(x0, goal)) return AERO_ERR_INVALID_ARG;
  int rc = validate(&pl, params, n);
  if (rc != AERO_OK) return rc;
  if (params->collision_set != 0) return AERO_ERR_EXCEEDS_LIMITS;
  if (reinterpret_cast<uintptr_t>(u_nom) % 16 != 0) return AERO_ERR_INVALID_ARG;
  if ((n > 0 && !is_device_ptr(cloud)) || !is_device_ptr(u_nom) || !is_device_ptr(u_best) ||
      !is_device_ptr(cand) || !is_device_ptr(best_idx))
    return AERO_ERR_NOT_DEVICE_PTR;
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  NoAllocDevice* d = nullptr;
  rc = noalloc_device(s, &d);
  if (rc != AERO_OK) return rc;
  noalloc_carve(d->base, pl);
  // the edge tables: the device's own host copy, uploaded only when the
  // partition geometry differs from the last upload
  pl.tab_valid = d->tab_valid;
  pl.tab_A = d->tab_A;
  pl.tab_El = d->tab_El;
  pl.tab_lo = d->tab_lo;
  pl.tab_hi = d->tab_hi;
  pl.tab_check_lo = d->tab_check_lo;
  pl.tab_check_hi = d->tab_check_hi;
  const bool same = d->tab_valid && d->tab_A == params->fine_az && d->tab_El == params->fine_el &&
                    d->tab_lo == params->el_lo && d->tab_hi == params->el_hi;
  if (!same) {
    make_tables(*params, d->tab, d->tab_check_lo, d->tab_check_hi);
    d->tab_valid = true;
    d->tab_A = params->fine_az;
    d->tab_El = params->fine_el;
    d->tab_lo = params->el_lo;
    d->tab_hi = params->el_hi;
    cudaError_t e = cudaMemcpyAsync(pl.d_tab, &d->tab, sizeof(PartTables), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      d->tab_valid = false;
      return AERO_ERR_CUDA;
    }
    pl.tab_valid = true;
    pl.tab_A = d->tab_A;
    pl.tab_El = d->tab_El;
    pl.tab_lo = d->tab_lo;
    pl.tab_hi = d->tab_hi;
    pl.tab_check_lo = d->tab_check_lo;
    pl.tab_check_hi = d->tab_check_hi;
  }
  pl.tab = d->tab;
  pl.tab_upload = false;
  // the last-block tickets and the status word must start at zero
  cudaError_t e = cudaMemsetAsync(pl.counter, 0, kCounterWords * sizeof(unsigned int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl.status, 0, sizeof(int), s);
  if (e != cudaSuccess) return AERO_ERR_CUDA;
  return enqueue_step(&pl, x0, cloud, n, goal, *params, u_nom, u_best, cand, best_idx, s);
}

// ---------------------------------------------------------------------------
// Batched planning: independent planners on a pool of streams.
// ---------------------------------------------------------------------------
struct aero_batch {
  std::vector<aero_planner*> planners;  // one workspace per item slot
  aero_limits_t lim{};
  int sms = 0;
  aero_batch_config_t cfg{0, 0, 1, 0, 0};
  int last_n = 0;  // items of the last call (debug copies)
  // resident CTAs per SM of the batched kernels
  int occ_grid[4] = {1, 1, 1, 1};  // partition, count, scan, scatter
  // rollout (1 lane), rollout (4 lanes), update, rollout (1 lane, 6/SM), rollout (1 lane, 64
  // samples per CTA), rollout (1 lane, 256 samples per CTA)
  int occ_roll[6] = {1, 1, 1, 1, 1, 1};
  // device: the call's arguments (items, unit prefixes, rollout orders), the
  // slots' edge tables, the rollout work queues
  unsigned char* d_args = nullptr;
  PartTables* d_tabs = nullptr;
  unsigned int* d_queue = nullptr;
  // pinned staging: a ring of argument buffers, the slots' tables
  static constexpr int kRing = 4;
  unsigned char* h_args[kRing] = {};
  cudaEvent_t h_done[kRing] = {};
  int ring = 0;
  PartTables* h_tabs = nullptr;
  cudaEvent_t tabs_done = nullptr;
  struct TabKey {
    int A = -1, El = -1;
    float lo = 0.0f, hi = 0.0f;
    bool operator==(const TabKey& o) const { return A == o.A && El == o.El && lo == o.lo && hi == o.hi; }
  };
  std::vector<TabKey> tab_key;
  // instantiated graphs, one per shape and configuration
  struct Graph {
    int n, max_iters, has1, has4;
    aero_batch_config_t cfg;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  cudaStream_t cap = nullptr, cap2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  // tuning outputs, one block of floats per slot
  float* scratch = nullptr;
  size_t scratch_stride = 0;
};

namespace {

struct ArgsLayout {
  size_t items, pre, order1, order4, bytes;
};

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

ArgsLayout layout_for(int n) {
  ArgsLayout L;
  L.items = 0;
  L.pre = align16(sizeof(BatchItem) * n);
  L.order1 = L.pre + sizeof(long long) * kPreCount * (n + 1);
  L.order4 = L.order1 + sizeof(int) * n;
  L.bytes = align16(L.order4 + sizeof(int) * n);
  return L;
}

BatchView view_of(aero_batch* b, int n) {
  const ArgsLayout L = layout_for(n);
  BatchView v;
  v.items = reinterpret_cast<const BatchItem*>(b->d_args + L.items);
  v.pre = reinterpret_cast<const long long*>(b->d_args + L.pre);
  v.order1 = reinterpret_cast<const int*>(b->d_args + L.order1);
  v.order4 = reinterpret_cast<const int*>(b->d_args + L.order4);
  v.n = n;
  v.T_max = b->lim.T_max;
  v.queue = b->d_queue;
  return v;
}

void batch_free(aero_batch* b) {
  for (aero_planner* pl : b->planners) aero_destroy(pl);
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  dev_free(b->d_args);
  dev_free(b->d_tabs);
  dev_free(b->d_queue);
  dev_free(b->scratch);
  for (int r = 0; r < aero_batch::kRing; ++r) {
    host_free(b->h_args[r]);
    if (b->h_done[r]) cudaEventDestroy(b->h_done[r]);
  }
  host_free(b->h_tabs);
  if (b->tabs_done) cudaEventDestroy(b->tabs_done);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->cap2) cudaStreamDestroy(b->cap2);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  delete b;
}

int check_item(aero_planner* pl, const aero_batch_item_t& it) {
  if (!it.u_nom_inout || !it.u_best_out || !it.cand_costs_out || !it.best_idx_out)
    return AERO_ERR_INVALID_ARG;
  if (it.n_points > 0 && !it.cloud_xyz) return AERO_ERR_INVALID_ARG;
  if (it.params.debug_samples != 0) return AERO_ERR_INVALID_ARG;
  if (!finite_state_goal(&it.x0, it.goal)) return AERO_ERR_INVALID_ARG;
  const int rc = validate(pl, &it.params, it.n_points);
  if (rc != AERO_OK) return rc;
  if (reinterpret_cast<uintptr_t>(it.u_nom_inout) % 16 != 0) return AERO_ERR_INVALID_ARG;
  if ((it.n_points > 0 && !is_device_ptr(it.cloud_xyz)) || !is_device_ptr(it.u_nom_inout) ||
      !is_device_ptr(it.u_best_out) || !is_device_ptr(it.cand_costs_out) ||
      !is_device_ptr(it.best_idx_out))
    return AERO_ERR_NOT_DEVICE_PTR;
  return AERO_OK;
}

// Samples per CTA of the one-lane Stage I pass of a configuration.
int spc_of(const aero_batch_config_t& c) { return c.samples_per_cta == 0 ? kRolloutThreads : c.samples_per_cta; }

int check_config(const aero_batch_config_t& c) {
  if (c.quad_max_samples < 0 || c.rollout_ctas_per_sm < 0 || c.rollout_ctas_per_sm > 64 ||
      (c.dynamic_queue != 0 && c.dynamic_queue != 1) || (c.coarse_cells != 0 && c.coarse_cells != 1) ||
      (c.samples_per_cta != 0 && c.samples_per_cta != 64 && c.samples_per_cta != 128 &&
       c.samples_per_cta != 256))
    return AERO_ERR_INVALID_ARG;
  return AERO_OK;
}

bool same_cfg(const aero_batch_config_t& a, const aero_batch_config_t& b) {
  return a.quad_max_samples == b.quad_max_samples && a.rollout_ctas_per_sm == b.rollout_ctas_per_sm &&
         a.dynamic_queue == b.dynamic_queue && a.coarse_cells == b.coarse_cells &&
         spc_of(a) == spc_of(b);
}

// The graph of one call shape: the four grid-stage launches, then per
// iteration the Stage I launch(es) -- both lane widths side by side when both
// occur -- and the update.
cudaError_t batch_graph(aero_batch* b, int n, int max_iters, int has1, int has4,
                        const aero_batch_config_t& cfg, cudaGraphExec_t* out) {
  for (auto& g : b->graphs)
    if (g.n == n && g.max_iters == max_iters && g.has1 == has1 && g.has4 == has4 &&
        same_cfg(g.cfg, cfg)) {
      *out = g.exec;
      return cudaSuccess;
    }
  const BatchView v = view_of(b, n);
  const int S = b->sms;
  // rollout_ctas_per_sm >= 6 selects the one-lane kernel built for six CTAs per
  // SM (128 samples per CTA); it counts CTAs of 128 threads, so other CTA
  // sizes of the one-lane pass scale it
  const int spc = spc_of(cfg);
  const int six = spc == kRolloutThreads && cfg.rollout_ctas_per_sm >= 6 && b->occ_roll[3] >= 6;
  auto roll_blocks = [&](int k) {
    int occ = b->occ_roll[k];
    if (k == 0) occ = six ? b->occ_roll[3] : spc == 64 ? b->occ_roll[4] : spc == 256 ? b->occ_roll[5] : occ;
    int per = occ;
    if (cfg.rollout_ctas_per_sm != 0)
      per = k == 0 ? cfg.rollout_ctas_per_sm * kRolloutThreads / spc : cfg.rollout_ctas_per_sm;
    return S * (per < 1 ? 1 : per);
  };
  cudaStream_t c = b->cap;
  cudaError_t e = cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = launch_batch_partition(v, S * b->occ_grid[0], c);
  if (le == cudaSuccess) le = launch_batch_count(v, S * b->occ_grid[1], c);
  if (le == cudaSuccess) le = launch_batch_scan(v, S * b->occ_grid[2], c);
  if (le == cudaSuccess) le = launch_batch_scatter(v, S * b->occ_grid[3], c);
  for (int it = 0; it < max_iters && le == cudaSuccess; ++it) {
    if (has1 && has4) {
      le = cudaEventRecord(b->fork, c);
      if (le == cudaSuccess) le = cudaStreamWaitEvent(b->cap2, b->fork, 0);
      if (le == cudaSuccess)
        le = launch_batch_rollout(v, 4, it, roll_blocks(1), cfg.dynamic_queue, 0, spc, b->cap2);
      if (le == cudaSuccess)
        le = launch_batch_rollout(v, 1, it, roll_blocks(0), cfg.dynamic_queue, six, spc, c);
      if (le == cudaSuccess) le = cudaEventRecord(b->join, b->cap2);
      if (le == cudaSuccess) le = cudaStreamWaitEvent(c, b->join, 0);
    } else {
      le = launch_batch_rollout(v, has4 ? 4 : 1, it, roll_blocks(has4 ? 1 : 0), cfg.dynamic_queue,
                                has4 ? 0 : six, spc, c);
    }
    if (le == cudaSuccess) le = launch_batch_update(v, it, S * b->occ_roll[2], c);
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(c, &graph);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return le != cudaSuccess ? le : e;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return e;
  b->graphs.push_back({n, max_iters, has1, has4, cfg, exec});
  *out = exec;
  return cudaSuccess;
}

// Enqueue one batched step of the n (validated) items on s.  scratch: write
// every item's nominal and outputs to the batch's scratch slots instead (the
// caller has copied the nominals there).
int batch_enqueue(aero_batch* b, const aero_batch_item_t* items, int n, cudaStream_t s,
                  const aero_batch_config_t& cfg, bool scratch) {
  const ArgsLayout L = layout_for(n);
  const int r = b->ring;
  b->ring = (b->ring + 1) % aero_batch::kRing;
  cudaError_t e = cudaEventSynchronize(b->h_done[r]);  // the slot's previous upload is done
  if (e != cudaSuccess) return cuda_fail(e);
  unsigned char* h = b->h_args[r];
  BatchItem* hi = reinterpret_cast<BatchItem*>(h + L.items);
  long long* pre = reinterpret_cast<long long*>(h + L.pre);
  int* ord1 = reinterpret_cast<int*>(h + L.order1);
  int* ord4 = reinterpret_cast<int*>(h + L.order4);
  std::vector<long long> roll_units(n);
  struct Meta {
    GridGeom grid;
    int ntiles, nb;
  };
  std::vector<Meta> meta(n);
  std::vector<int> lanes(n), T(n);
  std::vector<int> tab_changed;
  int max_iters = 0, has1 = 0, has4 = 0;
  for (int k = 0; k < kPreCount; ++k) pre[k * (n + 1)] = 0;
  for (int i = 0; i < n; ++i) {
    const aero_batch_item_t& it = items[i];
    const aero_params_t& p = it.params;
    aero_planner* pl = b->planners[i];
    float* u_nom = it.u_nom_inout;
    float* u_best = it.u_best_out;
    float* cand = it.cand_costs_out;
    int32_t* best = it.best_idx_out;
    if (scratch) {
      float* sc = b->scratch + b->scratch_stride * i;
      u_nom = sc;
      u_best = sc + (size_t)b->lim.E_max * b->lim.T_max * 4;
      cand = u_best + (size_t)b->lim.T_max * 4;
      best = reinterpret_cast<int32_t*>(cand + b->lim.E_max);
    }
    StepArgs a;
    make_step_args(pl, &it.x0, it.cloud_xyz, it.n_points, it.goal, p, u_nom, u_best, cand, best,
                   lanes_of(p, cfg.quad_max_samples), cfg.coarse_cells != 0, false, a, spc_of(cfg));
    BatchItem& bi = hi[i];
    bi.pa = a.pa;
    bi.ca = a.ca;
    bi.ca.reset_keys = pl->keys;
    bi.ga = a.ga;
    bi.ra = a.ra;
    bi.ua = a.ua;
    bi.ua.final_stage = 0;
    bi.tab = b->d_tabs + i;
    bi.count = pl->grid_count;
    bi.fill = pl->grid_fill;
    bi.local = pl->grid_local;
    bi.tile_sum = pl->tile_sum;
    bi.tile_off = pl->tile_off;
    bi.scan_counter = pl->counter + 2;
    bi.range = pl->grid_range;
    bi.keys = pl->keys;
    bi.iters = p.iters;
    bi.gcells = a.gcells;
    bi.ntiles = a.ntiles;
    bi.raw_keys = a.raw ? a.ncell : 0;
    const aero_batch::TabKey key{p.fine_az, p.fine_el, p.el_lo, p.el_hi};
    if (!(b->tab_key[i] == key)) {
      if (tab_changed.empty() && (e = cudaEventSynchronize(b->tabs_done)) != cudaSuccess)
        return cuda_fail(e);
      b->h_tabs[i] = a.tab;
      b->tab_key[i] = key;
      tab_changed.push_back(i);
    }
    auto set = [&](int k, long long units) { pre[k * (n + 1) + i + 1] = pre[k * (n + 1) + i] + units; };
    set(kPrePoints, (it.n_points + kPartChunk - 1) / kPartChunk);
    set(kPreItems, a.n_items);
    set(kPreCoarse, (long long)a.ga.Ac * a.ga.Ec);
    set(kPreTiles, a.ntiles);
    set(kPreCells, (long long)a.gcells + bi.raw_keys);
    set(kPreUpdate, p.E);
    roll_units[i] = (long long)p.E * a.nb;
    meta[i] = {a.grid, a.ntiles, a.nb};
    lanes[i] = a.lanes;
    T[i] = p.T;
    if (p.iters > max_iters) max_iters = p.iters;
    (a.lanes == 4 ? has4 : has1) = 1;
  }
  // rollout order: longest horizon first, then more units, then slot index
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    if (T[x] != T[y]) return T[x] > T[y];
    if (roll_units[x] != roll_units[y]) return roll_units[x] > roll_units[y];
    return x < y;
  });
  long long* p1 = pre + kPreRoll1 * (n + 1);
  long long* p4 = pre + kPreRoll4 * (n + 1);
  for (int q = 0; q < n; ++q) {
    const int i = order[q];
    ord1[q] = i;
    ord4[q] = i;
    p1[q + 1] = p1[q] + (lanes[i] == 1 ? roll_units[i] : 0);
    p4[q + 1] = p4[q] + (lanes[i] == 4 ? roll_units[i] : 0);
  }

  cudaGraphExec_t exec = nullptr;
  if ((e = batch_graph(b, n, max_iters, has1, has4, cfg, &exec)) != cudaSuccess) return cuda_fail(e);
  // workspaces whose counts or keys may be stale (new slot, interrupted step)
  for (int i = 0; i < n; ++i) {
    aero_planner* pl = b->planners[i];
    if (pl->grid_dirty &&
        (e = cudaMemsetAsync(pl->grid_count, 0, sizeof(int) * (pl->grid_cells_cap + 1), s)) != cudaSuccess)
      return cuda_fail(e);
    if (!pl->keys_empty &&
        (e = cudaMemsetAsync(pl->keys, 0xFF, sizeof(unsigned long long) * pl->lim.fine_cells_max, s)) !=
            cudaSuccess)
      return cuda_fail(e);
    pl->grid_dirty = true;
    pl->keys_empty = false;
  }
  for (int i : tab_changed)
    if ((e = cudaMemcpyAsync(b->d_tabs + i, b->h_tabs + i, sizeof(PartTables), cudaMemcpyHostToDevice,
                             s)) != cudaSuccess)
      return cuda_fail(e);
  if (!tab_changed.empty() && (e = cudaEventRecord(b->tabs_done, s)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemcpyAsync(b->d_args, h, L.bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaEventRecord(b->h_done[r], s)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) return cuda_fail(e);
  for (int i = 0; i < n; ++i) {
    aero_planner* pl = b->planners[i];
    pl->grid_dirty = false;
    pl->keys_empty = true;
    pl->have_step = true;
    pl->last = items[i].params;
    pl->last_grid = meta[i].grid;
    pl->last_idx_entries = false;
    pl->last_ntiles = meta[i].ntiles;
    pl->last_part_slots = (int)((items[i].n_points + kPartChunk - 1) / kPartChunk);
    pl->last_n_points = items[i].n_points;
    pl->last_nb = meta[i].nb;
  }
  b->last_n = n;
  return AERO_OK;
}

int check_items(aero_batch* b, const aero_batch_item_t* items, int32_t n) {
  if (!b || (n > 0 && !items) || n < 0 || n > (int32_t)b->planners.size()) return AERO_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    const int rc = check_item(b->planners[i], items[i]);
    if (rc != AERO_OK) return rc;
  }
  return AERO_OK;
}
}  // namespace

int aero_batch_create(const aero_limits_t* limits, int32_t n_max, aero_batch_t** out) {
  if (!limits || !out || n_max < 1 || n_max > kBatchMax) return AERO_ERR_INVALID_ARG;
  *out = nullptr;
  aero_batch* b = new (std::nothrow) aero_batch();
  if (!b) return AERO_ERR_ALLOC;
  b->lim = *limits;
  b->lim.debug_samples_max = 0;
  for (int i = 0; i < n_max; ++i) {
    aero_planner_t* pl = nullptr;
    const int rc = create_planner(&b->lim, &pl, true);
    if (rc != AERO_OK) {
      batch_free(b);
      return rc;
    }
    b->planners.push_back(pl);
  }
  b->tab_key.assign(n_max, aero_batch::TabKey{});
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = batch_grid_occupancy(b->occ_grid);
  if (e == cudaSuccess) e = batch_rollout_occupancy(b->occ_roll, b->lim.T_max);
  const size_t bytes = layout_for(n_max).bytes;
  if (e == cudaSuccess) e = dev_malloc((void**)&b->d_args, bytes);
  if (e == cudaSuccess) e = dev_malloc((void**)&b->d_tabs, sizeof(PartTables) * n_max);
  if (e == cudaSuccess) e = dev_malloc((void**)&b->d_queue, 4 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(b->d_queue, 0, 4 * sizeof(unsigned int));
  b->scratch_stride = align16(sizeof(float) * ((size_t)b->lim.E_max * b->lim.T_max * 4 +
                                               (size_t)b->lim.T_max * 4 + b->lim.E_max + 1)) /
                      sizeof(float);
  if (e == cudaSuccess) e = dev_malloc((void**)&b->scratch, sizeof(float) * b->scratch_stride * n_max);
  for (int r = 0; r < aero_batch::kRing && e == cudaSuccess; ++r) {
    e = host_malloc((void**)&b->h_args[r], bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->h_done[r], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = host_malloc((void**)&b->h_tabs, sizeof(PartTables) * n_max);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->tabs_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_free(b);
    return e == cudaErrorMemoryAllocation ? AERO_ERR_ALLOC : AERO_ERR_CUDA;
  }
  *out = b;
  return AERO_OK;
}

int aero_batch_plan(aero_batch_t* b, const aero_batch_item_t* items, int32_t n, void* stream) {
  int rc = check_items(b, items, n);
  if (rc != AERO_OK || n == 0) return rc;
  return batch_enqueue(b, items, n, (cudaStream_t)stream, b->cfg, false);
}

int aero_batch_set_config(aero_batch_t* b, const aero_batch_config_t* c) {
  if (!b || !c) return AERO_ERR_INVALID_ARG;
  const int rc = check_config(*c);
  if (rc != AERO_OK) return rc;
  b->cfg = *c;
  return AERO_OK;
}

int aero_batch_get_config(aero_batch_t* b, aero_batch_config_t* c) {
  if (!b || !c) return AERO_ERR_INVALID_ARG;
  *c = b->cfg;
  return AERO_OK;
}

int aero_batch_tune(aero_batch_t* b, const aero_batch_item_t* items, int32_t n, int32_t repeats,
                    void* stream, aero_batch_config_t* best, float* best_ms) {
  if (repeats < 1 || repeats > 1000) return AERO_ERR_INVALID_ARG;
  int rc = check_items(b, items, n);
  if (rc != AERO_OK) return rc;
  if (n == 0) return AERO_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  auto fail = [&](int code) {
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    return code;
  };
  if (e != cudaSuccess) return fail(AERO_ERR_CUDA);
  aero_batch_config_t chosen = b->cfg;
  float chosen_ms = INFINITY;
  const int quad[3] = {0, 4096, 32768};
  const int lo = b->occ_roll[0] < b->occ_roll[1] ? b->occ_roll[0] : b->occ_roll[1];
  const int ctas[3] = {0, 6, lo / 2 > 0 ? lo / 2 : 1};
  const int spcs[3] = {128, 64, 256};
  for (int si = 0; si < 3; ++si)
  for (int qi = 0; qi < 3; ++qi)
    for (int ci = 0; ci < 3; ++ci)
      for (int dyn = 1; dyn >= 0; --dyn)
        for (int coarse = 0; coarse < 2; ++coarse) {
          const aero_batch_config_t c{quad[qi], ctas[ci], dyn, coarse, spcs[si]};
          float total = 0.0f;
          for (int rep = 0; rep <= repeats; ++rep) {
            for (int i = 0; i < n; ++i) {
              const aero_params_t& p = items[i].params;
              if ((e = cudaMemcpyAsync(b->scratch + b->scratch_stride * i, items[i].u_nom_inout,
                                       sizeof(float) * p.E * p.T * 4, cudaMemcpyDeviceToDevice, s)) !=
                  cudaSuccess)
                return fail(AERO_ERR_CUDA);
            }
            if ((e = cudaEventRecord(t0, s)) != cudaSuccess) return fail(AERO_ERR_CUDA);
            rc = batch_enqueue(b, items, n, s, c, true);
            if (rc != AERO_OK) return fail(rc);
            if ((e = cudaEventRecord(t1, s)) != cudaSuccess || (e = cudaEventSynchronize(t1)) != cudaSuccess)
              return fail(AERO_ERR_CUDA);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, t0, t1);
            if (rep > 0) total += ms;  // the first run warms up (and instantiates the graph)
          }
          const float mean = total / repeats;
          if (mean < chosen_ms) {
            chosen_ms = mean;
            chosen = c;
          }
        }
  b->cfg = chosen;
  if (best) *best = chosen;
  if (best_ms) *best_ms = chosen_ms;
  return fail(AERO_OK);
}

int aero_batch_sync_status(aero_batch_t* b, int32_t* status) {
  if (!b || !status) return AERO_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return AERO_ERR_CUDA;
  int32_t acc = 0;
  for (aero_planner* pl : b->planners) {
    int st = 0;
    if (cudaMemcpy(&st, pl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return AERO_ERR_CUDA;
    if (st != 0 && cudaMemset(pl->status, 0, sizeof(int)) != cudaSuccess) return AERO_ERR_CUDA;
    acc |= st;
  }
  int cw = 0;
  if (read_check_words(&cw, true) != cudaSuccess) return AERO_ERR_CUDA;
  *status = acc | cw;
  return AERO_OK;
}

size_t aero_batch_debug_size(aero_batch_t* b, int32_t slot, int32_t what) {
  if (!b || slot < 0 || slot >= b->last_n) return 0;
  return aero_debug_size(b->planners[slot], what);
}

int aero_batch_get_debug(aero_batch_t* b, int32_t slot, int32_t what, void* dst, size_t bytes,
                         void* stream) {
  if (!b || slot < 0 || slot >= b->last_n) return AERO_ERR_INVALID_ARG;
  return aero_get_debug(b->planners[slot], what, dst, bytes, stream);
}

int aero_batch_destroy(aero_batch_t* b) {
  if (!b) return AERO_OK;
  cudaDeviceSynchronize();
  batch_free(b);
  return AERO_OK;
}

}  // extern "C"
