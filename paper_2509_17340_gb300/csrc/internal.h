// Internal interface between the C-ABI host runtime (aero_mppi.cu) and the
// kernel translation units (partition.cu, rollout.cu).  Not installed.
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

namespace aero {

constexpr int kMaxAz = 512;
constexpr int kMaxEl = 256;
constexpr int kMaxE = 64;
// Tickets of last-CTA patterns, zero between launches: [0] the update's
// selection, [1] unused, [2] the batched grid scan, [3 + e] the Stage I CTAs of
// instance e in the split pass that also runs the update.
// [0] selection ticket, [1], [2] grid counters, [3, 3 + kMaxE) the split pass's
// instance tickets, then the one-lane pass's finished-CTA count and the update
// launch's exit ticket
constexpr int kCounterWords = 5 + kMaxE;
constexpr int kDoneWord = 3 + kMaxE;
constexpr int kMaxT = 128;
constexpr int kGridMax = 96;         // collision-grid cells per axis, at most
constexpr int kGridCellsMax = kGridMax * kGridMax * kGridMax;
constexpr int kScanTile = 4096;      // cells per scan tile (1024 threads x 4)
constexpr int kScanTileShift = 12;
constexpr int kMaxTiles = (kGridCellsMax + 1 + kScanTile - 1) / kScanTile;
constexpr int kRolloutThreads = 128; // samples per rollout CTA (one warp-group)
constexpr int kQuadMaxSamples = 32768;  // E*K up to which the split Stage I pass runs

// Binary32 edge tables of the partition, passed by value to the kernels.
// Azimuth edge k: theta_k = pi (2k - A) / A; elevation edge k: phi_k = lo +
// ((hi - lo) k) / El; each entry is the binary64 cos / sin rounded to binary32.
struct PartTables {
  float ca[kMaxAz];
  float sa[kMaxAz];
  float ce[kMaxEl + 1];
  float se[kMaxEl + 1];
};

// Collision grid in world axes, coordinates relative to p0.  Cell (x, y, z)
// is the box [origin + x h, origin + (x+1) h) x ... and its candidate list holds
// every collision point whose distance to that box is below `reach` = d_max
// plus a rounding margin, so the nearest point of any query closer than d_max
// is in the list of the query's cell.
struct GridGeom {
  int G;          // cells per axis
  float origin;   // lower corner, same on all three axes
  float h, inv_h; // cell edge and its reciprocal
  float reach;    // d_max + margin
  int cap;        // capacity of the candidate array (entries)
};

struct PartitionArgs {
  const float* cloud;
  int64_t n;
  float p0[3];
  float R[9];      // R(q0) in binary32, row-major
  float rmax2;     // r_max * r_max in binary32
  int A, El;
  int check_lo, check_hi;
  int filter;      // read a cone's key before its atomic minimum (dense clouds)
  float el_lo, el_inv;  // elevation span start and cones per radian (bin guesses only)
  unsigned long long* keys;
  int* item_flag;  // collision set = every kept point: 1 where the point is kept, else 0
  int2* counts;    // per block (batched: per chunk of points): {non-finite points, kept points}
  float* copy_to;  // or null; else every point read is stored here too (n x 3): a cloud read
                   // from page-locked host memory leaves its device copy for the later passes
};

// Count and scatter passes of the candidate lists.
struct CandArgs {
  const float* cloud;
  float p0[3];
  const unsigned long long* keys;  // collision set = P_f: item c is the winner of fine cell c
  const int* item_flag;            // collision set = kept points: item i is point i
  int64_t n_items;
  int raw;
  GridGeom grid;
  int* count;          // G^3 + 1: entries per cell (count pass); zero between steps
  int* fill;           // G^3 + 1: fill cursors of the scatter pass; zeroed by the scan
  const int* local;    // tile-local exclusive prefix of the counts (scatter pass)
  const int* tile_off; // exclusive prefix of the tile totals (scatter pass)
  // candidate entries (scatter pass), in one of two forms: item indices into
  // pts, whose points the count pass stores (cand non-null), or the points
  // themselves (cand4)
  uint32_t* cand;
  float4* pts;         // n_items: collision point of each item, minus p0 (w: the item index's bits)
  float4* cand4;       // entries holding the points (w: the item index's bits)
  int* status;
  unsigned long long* reset_keys;  // non-null: the scatter pass empties each key it reads
};

struct GuideArgs {
  // partition
  const unsigned long long* keys;
  int A, El, Pa, Pe, Ac, Ec;
  float rmax2;
  float el_lo, el_hi;  // binary32 span, promoted to binary64 for cell centres
  float R[9];          // R(q0) binary32
  float goal_rel[3];   // goal - p0, binary32
  int M_h, M_v, E;
  float ell;
  // guides
  int T;
  float dt, v_end;     // v_end <= 0: ell / (T dt)
  float v0[3];
  // outputs
  int* coarse_win;     // Ac * Ec
  int* cells;          // [0] goal fine cell, [1 + e] anchor coarse cell
  float* anchors;      // E x 3 (relative to p0)
  float* guides;       // E x T x 3 (relative to p0)
};

struct GridView {
  const int2* range;     // G^3 cell ranges into the candidate entries
  const uint32_t* cand;  // entries as item indices into pts, grouped by cell; or null:
  const float4* pts;     // the items' collision points (minus p0), or (cand null) the entries' own
  int G;
  float origin, inv_h;
};

struct CostParams {
  float Q_track, Q_vnorm, Q_c, Q_cd, Q_p, Q_v, Q_q;
  float C_col, a_col, d_min, d_max;
  float goal_rel[3], v_goal[3], q_goal[4];
};

struct DynParams {
  float dt, inv_mass, g;
};

struct RolloutArgs {
  int E, K, T, nb;         // nb = CTAs per instance
  int lanes_per_sample;    // 1, or 4 (k_rollout_split) for small E*K
  float inv_lambda;
  float sigma[4], umin[4], umax[4];
  float x0[10];            // p = 0 (relative), q0, v0
  uint32_t key0, key1, ctr3;
  uint32_t rk[20];         // Philox round keys: (key0, key1) + r (Weyl constants), r = 0..9
  DynParams dyn;
  CostParams cost;
  const float* u_nom;      // E x T x 4
  const float* guides;     // E x T x 3 (relative)
  GridView grid;
  float* partials;         // E x nb x (4 + 4T): rho, eta, 2 pad, W (16-byte aligned)
  float* sample_costs;     // E x K
  int dbg_D;
  float* dbg_u;            // E x D x T x 4
  float* dbg_x;            // E x D x (T+1) x 10
  float* dbg_d;            // E x D x T
  unsigned int* done;      // the one-lane pass: its CTAs count themselves here when they finish
                           // (read by the update launch), or null
  int list_thr;            // single planner's one-lane pass: lists longer than this are
                           // scanned by the whole warp (warp_split_min, its own kernel
                           // instance); 0: every lane scans its own list
};

struct UpdateArgs {
  int E, T, nb;
  float inv_lambda;
  const float* partials;
  float* u_nom;            // E x T x 4 (in/out)
  int final_stage;         // run Stage II and the selection
  float x0[10];
  DynParams dyn;
  CostParams cost;
  GridView grid;
  float* stage2_x;         // E x (T+1) x 10
  const float* guides;     // E x T x 3 (relative): the tracking term of the refinement
  float umin[4], umax[4];
  int refine_steps;        // gradient steps on each updated nominal before Stage II
  float refine_step;
  float* dbg_pre;          // E x T x 4: the nominals before the refinement (refine_steps > 0)
  float* cand;             // E
  int* best_idx;
  float* u_best;           // T x 4
  unsigned int* counter;   // last-CTA ticket, 0 between launches
  unsigned int* inst_counter;  // E tickets of the split Stage I pass, 0 between launches
  int* status;             // bit 0: a normaliser eta was not a positive finite number
  float* warm;             // scratch of the warm-up runs of the update's code: E regions of
                           // warm_words(E, T) floats; null: no warm-up runs
  unsigned int* done;      // the update launch: {finished CTAs of the one-lane pass, exit
                           // ticket}, both reset by its last CTA; or null
};

// One region of the warm-up scratch for E instances of horizon T (floats):
// nominals E x T x 4, Stage II states (T + 1) x 10, candidate costs E, best
// sequence T x 4, then three words (best index, ticket, status).
__host__ __device__ constexpr size_t warm_words(int E, int T) {
  return (size_t)E * T * 4 + (size_t)(T + 1) * 10 + E + (size_t)T * 4 + 3;
}

// ---------------------------------------------------------------------------
// Batched step: the planning steps of many independent planners, each stage one
// launch over the work units of all of them.  A unit maps to its planner through
// an exclusive prefix of the per-planner unit counts (binary search in shared
// memory); the rollout takes its units from a device work queue in the order of
// `order1` / `order4` (longest horizon first).
// ---------------------------------------------------------------------------
constexpr int kBatchMax = 256;       // planners per batched call
constexpr int kPartChunk = 1024;     // points per partition unit

enum BatchPrefix {
  kPrePoints = 0,  // partition units (kPartChunk points)
  kPreItems,       // collision items (count and scatter tasks, one warp each)
  kPreCoarse,      // coarse cells (one warp each)
  kPreTiles,       // scan tiles
  kPreCells,       // grid cells (range of each) and, after them, raw-set keys to reset
  kPreRoll1,       // rollout units, one lane per sample, in order1
  kPreRoll4,       // rollout units, four lanes per sample, in order4
  kPreUpdate,      // (planner, instance) units of the update
  kPreCount
};

struct BatchItem {
  PartitionArgs pa;
  CandArgs ca;
  GuideArgs ga;
  RolloutArgs ra;            // ctr3 = step_id << 8: the launch ors in the iteration
  UpdateArgs ua;             // final_stage unused: iteration it is final when it == iters - 1
  const PartTables* tab;     // device copy of the planner's tables
  int* count;
  int* fill;
  int* local;
  int* tile_sum;
  int* tile_off;
  unsigned int* scan_counter;
  int2* range;
  unsigned long long* keys;  // fine-cell keys, left empty (all ones) by the step
  int iters;
  int gcells;                // G^3
  int ntiles;
  int raw_keys;              // fine cells whose keys the scatter launch resets (raw set), else 0
};

struct BatchView {
  const BatchItem* items;
  const long long* pre;      // kPreCount x (n + 1) exclusive prefixes of unit counts
  const int* order1;         // rollout position -> planner (one lane per sample)
  const int* order4;         // (four lanes per sample)
  int n;
  int T_max;                 // longest horizon a planner of the batch may use
  unsigned int* queue;       // per rollout kernel: {next unit, exit ticket}, zero between launches
};

cudaError_t launch_batch_partition(const BatchView& v, int blocks, cudaStream_t s);
cudaError_t launch_batch_count(const BatchView& v, int blocks, cudaStream_t s);
cudaError_t launch_batch_scan(const BatchView& v, int blocks, cudaStream_t s);
cudaError_t launch_batch_scatter(const BatchView& v, int blocks, cudaStream_t s);
// lanes 1 or 4; dynamic: take units from the work queue, else stride by the grid;
// six: the one-lane kernel compiled for six resident CTAs per SM (fewer
// registers) instead of five; samples_per_cta: the one-lane pass's CTA size
// (64, 128 or 256; the items' partial rows were laid out for it)
cudaError_t launch_batch_rollout(const BatchView& v, int lanes, int it, int blocks, int dynamic,
                                 int six, int samples_per_cta, cudaStream_t s);
cudaError_t launch_batch_update(const BatchView& v, int it, int blocks, cudaStream_t s);

// Resident CTAs per SM: {partition, count, scan, scatter} and {rollout with one
// lane per sample, with four, update, rollout with one lane compiled for six,
// one lane with 64 samples per CTA, one lane with 256}.
cudaError_t batch_grid_occupancy(int out[4]);
cudaError_t batch_rollout_occupancy(int out[6], int T_max);

// t: the edge tables in device memory
cudaError_t launch_partition(const PartitionArgs& a, const PartTables* t, cudaStream_t s);
int partition_blocks(int64_t n);  // CTAs of launch_partition for n points (0 when n == 0)
constexpr int kPartBlocksMax = 4096;  // CTAs of launch_partition, at most (16 per SM, capped)
// Streaming multiprocessors of the current device, queried once per device
// (1 if the query fails: the launches stay correct, only slower).
int device_sms();
// count pass + coarse argmax; then the tile scans + goal cone, anchors, guides
cudaError_t launch_grid_count(const CandArgs& ca, const GuideArgs& ga, cudaStream_t s);
cudaError_t launch_grid_scan(int* count, int* fill, int* local, int* tile_sum, int* tile_off,
                             int ncells, int ntiles, unsigned int* counter, const GuideArgs& ga,
                             const PartTables* t, cudaStream_t s);
// scatter + cell ranges; the tile offsets are computed here from the tile
// totals of the scan launch (and written to tile_off)
cudaError_t launch_grid_scatter(const CandArgs& ca, int2* range, int ncells, const int* tile_sum,
                                int* tile_off, int ntiles, cudaStream_t s);
// S(1) of n noise-free rollouts of instance `instance` and their gradients.
struct CostGradArgs {
  UpdateArgs ctx;          // x0, dynamics, costs, grid, guides, T of the last step
  int instance;
  const float4* U;         // n x T
  int n;
  float* S;                // n
  float4* G;               // n x T, or null
};

// Stage I; the split pass (lanes_per_sample 4) also runs the update `ua` in
// the last CTA of every instance, the others leave it to launch_update.
cudaError_t launch_rollout(const RolloutArgs& a, const UpdateArgs& ua, cudaStream_t s);
bool rollout_runs_update(const RolloutArgs& a);
// Sets the kernels' shared-memory limits (once per device).
cudaError_t split_attributes();
cudaError_t launch_cost_grad(const CostGradArgs& a, cudaStream_t s);
cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s);
cudaError_t launch_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3,
                          int64_t n, uint32_t* out, cudaStream_t s);

// Launch with programmatic stream serialization when `pdl` is set: the
// kernel may be scheduled while its predecessor in the stream still runs and
// waits for it in griddepcontrol.wait (see pdl_wait), which hides the launch
// latency of a chain of dependent kernels.
template <typename... KArgs, typename... Args>
cudaError_t launch_ks(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                      bool pdl, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, bool pdl,
                     Args&&... args) {
  return launch_ks(kernel, grid, block, 0, s, pdl, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------
// Checked builds (-DAERO_CHECKED, libaero_mppi_checked.so).  AERO_CHECK(cond,
// bit) guards an index the kernels rely on: in a checked build a failed
// condition records `bit` in the translation unit's check word and the guarded
// access is skipped (no trap, no assert); aero_sync_status then reports
// AERO_ERR_DEVICE_CHECK.  In the product build it is the constant true.
// ---------------------------------------------------------------------------
enum CheckBit : int {
  kChkFineCell = 1 << 8,     // partition: fine cell outside the partition
  kChkGridCell = 1 << 9,     // candidate grid: cell outside the grid
  kChkRange = 1 << 10,       // candidate range beyond the entries written
  kChkQuery = 1 << 11,       // split pass / Stage II: query slot or item outside its list
  kChkPartial = 1 << 12,     // partial row or sample outside the instance's block
  kChkAccum = 1 << 13,       // accumulation ring slot
};
#ifdef AERO_CHECKED
static __device__ int g_check_word;
__device__ __forceinline__ bool check_fail(int bit) {
  atomicOr(&g_check_word, bit);
  return false;
}
#define AERO_CHECK(cond, bit) ((cond) ? true : ::aero::check_fail(bit))
#else
#define AERO_CHECK(cond, bit) true
#endif
// The check words of the library's translation units, or'ed (0 in the product
// build); `clear` resets them.  Synchronises the device.
cudaError_t read_check_words(int* out, bool clear);
cudaError_t check_word_partition(int* out, bool clear);
cudaError_t check_word_rollout(int* out, bool clear);
cudaError_t check_word_accum(int* out, bool clear);
cudaError_t raise_check_partition(int bits);  // checked build: record `bits` (tests)

// Every device and pinned host allocation of the library goes through these
// four calls.  They count live allocations and let a test make the n-th next
// allocation fail (aero_test_fail_alloc), so that each error path of the
// create functions can be driven without exhausting the device.
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t host_malloc(void** p, size_t bytes);
void dev_free(void* p);
void host_free(void* p);

}  // namespace aero
