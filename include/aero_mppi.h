/*
 * aero_mppi.h -- C ABI of the GB300 (sm_103a) AERO-MPPI planning step.
 *
 * One call of aero_plan_step() runs one planning step of AERO-MPPI
 * (arXiv 2509.17340) on the GPU, entirely in this library's CUDA kernels:
 *
 *   1. fine spherical partition of the cloud around the drone
 *      (Sec. IV-A.1: r_ij = min |p_c| over the points in cone C_ij);
 *   2. coarse pooling argmax (Sec. IV-A.2, Eq. safe-vector), the M_h x M_v
 *      coarse cells around the goal direction (Sec. IV-B.1) and the anchors
 *      p_ref = p0 + ell d_IJ (Eq. anchor-point);
 *   3. quintic guides from the current state to each anchor (Eq. polynomial);
 *   4. for each of the E = M_h M_v MPPI instances: K Gaussian perturbations of
 *      the nominal controls (Sec. III-B), RK4 rollouts of the quadrotor model
 *      (Eq. dynamics, Eq. mppi_rollout_simplified), the Stage I cost S(1)
 *      (Eq. total cost and the cost terms of Sec. IV-C, collision distances
 *      against the filtered cloud P_f), softmax weights (Eq. mppi_weights) and
 *      the update of the nominal (Eq. mppi_update_simplified);
 *   5. Stage II: noise-free rollout of the E updated nominals, S(2) = J_goal +
 *      J_col, and the argmin (Sec. IV-C).
 *
 * Conventions
 *   - Every function returns an aero status code (AERO_OK = 0, negative on
 *     error) except aero_params_default and aero_status_str.  No exception,
 *     exit, abort or device trap crosses this boundary.
 *   - "device" pointers are CUDA global-memory pointers on the planner's device
 *     (cudaMalloc, torch CUDA tensors); "host" pointers are CPU memory.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     aero_plan_step only enqueues work and returns; its outputs are valid once
 *     the stream has reached that point.  It allocates nothing, so a sequence of
 *     calls with fixed pointers can be captured into a CUDA graph.
 *   - The caller owns every input and output buffer; the planner owns its
 *     workspace, allocated once by aero_create and freed by aero_destroy.
 *   - One planner must not be used by two streams at the same time: calls share
 *     its workspace.
 *   - Angles are radians, lengths metres, times seconds; quaternions are
 *     (w, x, y, z), unit length, body to world (Hamilton product).
 */
#ifndef AERO_MPPI_H
#define AERO_MPPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define AERO_OK 0
#define AERO_ERR_INVALID_ARG (-1)    /* null pointer, bad size, inconsistent params */
#define AERO_ERR_EXCEEDS_LIMITS (-2) /* a size above the planner's aero_limits_t */
#define AERO_ERR_CUDA (-3)           /* a CUDA runtime call failed */
#define AERO_ERR_ALLOC (-4)          /* workspace allocation failed */
#define AERO_ERR_DEVICE_CHECK (-5)   /* a kernel reported an internal inconsistency */
#define AERO_ERR_NOT_DEVICE_PTR (-6) /* a pointer that must be device memory is not */

/* ---- debug buffers (aero_get_debug) ------------------------------------
 * Positions in debug buffers are relative to the start position p0 of the
 * last step (world axes), as the kernels keep them. */
#define AERO_DBG_FINE_KEYS 0     /* uint64 [fine_el][fine_az]: (bits(r^2 f32) << 32) | point index
                                    (kept by planners created with debug_samples_max > 0: the
                                    others empty their keys during the step, saving a fill);
                                    0xFFFFFFFFFFFFFFFF = empty cone */
#define AERO_DBG_COARSE_WIN 1    /* int32 [E_c][A_c]: winning fine cell j*fine_az+i of each coarse cell */
#define AERO_DBG_GOAL_CELL 2     /* int32 [1]: fine cell of the goal direction */
#define AERO_DBG_ANCHOR_CELLS 3  /* int32 [E]: coarse cell J*A_c+I of instance e = n*M_h+m */
#define AERO_DBG_ANCHORS 4       /* float [E][3]: anchor - p0 */
#define AERO_DBG_GUIDES 5        /* float [E][T][3]: guide at t=(j+1)dt, minus p0 */
#define AERO_DBG_GRID_META 6     /* int32 [4] = {G, n_entries, capacity, 0} then float [4] =
                                    {origin, h, reach, 0}: G^3 cells of edge h from origin
                                    (all axes); cell c lists every collision point closer
                                    than reach (>= d_max) to its box */
#define AERO_DBG_GRID_START 7    /* int32 [G*G*G + 1]: first entry of cell (z*G+y)*G+x */
#define AERO_DBG_GRID_POINTS 8   /* float4 [n_entries]: candidate points - p0, grouped by cell */
#define AERO_DBG_SAMPLE_COSTS 9  /* float [E][K]: S(1) of every sample, last iteration */
#define AERO_DBG_STAGE2_STATES 10 /* float [E][T+1][10]: Stage II states (p - p0, q, v) */
#define AERO_DBG_SAMPLE_U 11     /* float [E][D][T][4]: clamped controls of samples k < D */
#define AERO_DBG_SAMPLE_X 12     /* float [E][D][T+1][10]: their states (p - p0, q, v) */
#define AERO_DBG_SAMPLE_DIST 13  /* float [E][D][T]: their nearest-point distances, or
                                    +inf where none is closer than d_max */
#define AERO_DBG_PRE_REFINE 14   /* float [E][T][4]: nominals after the last update, before the
                                    gradient refinement (written when refine_steps > 0) */
#define AERO_DBG_POINT_COUNTS 15 /* int64 [3]: points given, points skipped as non-finite,
                                    points kept by the partition (within r_max and the
                                    elevation span) */
#define AERO_DBG_COUNT 16

/* ---- inputs ----------------------------------------------------------- */

/* Drone state x = [p, q, v] of Eq. dynamics (world frame). */
typedef struct {
  float p[3];
  float q[4]; /* w, x, y, z */
  float v[3];
} aero_state_t;

/* Maxima fixed when the planner is created; they size its workspace. */
typedef struct {
  int32_t E_max;            /* ensemble size, <= 64 */
  int32_t K_max;            /* samples per instance, <= 1<<20 */
  int32_t T_max;            /* horizon steps, <= 128 */
  int32_t fine_cells_max;   /* fine_az * fine_el, <= 512 * 256 */
  int64_t n_points_max;     /* cloud size, <= 2^31 - 1 */
  int32_t debug_samples_max; /* D: samples per instance whose rollouts can be recorded */
  int32_t raw_points_max;   /* cloud size up to which the every-point collision set
                               (collision_set = 1) can be used: 0 = n_points_max, -1 = never
                               (its per-point arrays are then not allocated); otherwise
                               1 .. n_points_max.  A step with collision_set = 1 and more
                               points returns AERO_ERR_EXCEEDS_LIMITS.  The planner's
                               candidate lists then take up to 864 bytes per point */
} aero_limits_t;

/* Parameters of one planning step; aero_params_default() fills Table I. */
typedef struct {
  int32_t E, K, T;        /* ensemble size (= M_h*M_v), samples, horizon N */
  int32_t iters;          /* MPPI iterations (Stage I) per step, 1..255 */
  float dt;               /* RK4 step (s) */
  float lambda;           /* temperature of Eq. mppi_weights, > 0 */
  float mass, g;          /* m (kg); gravity magnitude, acting along -z */
  float sigma[4];         /* standard deviations of (F, wx, wy, wz) perturbations */
  float u_min[4], u_max[4]; /* control bounds; sampled controls are clamped */
  float Q_track, Q_vnorm, Q_c, Q_cd, Q_p, Q_v, Q_q; /* cost weights (Sec. IV-C) */
  float C_col, a_col, d_min, d_max;  /* collision penalty C, a, d_obs_min < d_obs_max */
  float r_max;            /* perception range of the partition (m) */
  float ell;              /* look-ahead distance of the anchors (m) */
  float v_end;            /* guide speed at the anchor; <= 0 means ell / (T dt) */
  int32_t fine_az, fine_el;  /* fine grid (even fine_az <= 512, fine_el <= 256) */
  int32_t pool_az, pool_el;  /* pooling; must divide the fine grid */
  int32_t M_h, M_v;          /* anchor grid; M_h*M_v == E */
  float el_lo, el_hi;     /* elevation span of the partition */
  int32_t collision_set;  /* 0: P_f (nearest point of every cone, Sec. IV-C);
                             1: every point kept by the partition */
  float v_goal[3];        /* goal velocity */
  float q_goal[4];        /* goal attitude (w, x, y, z) */
  int32_t debug_samples;  /* D: record rollouts of samples k < D (0 = off) */
  int32_t lanes_per_sample; /* Stage I kernel: 1 = one thread per sample; 4 = the split
                             pass for small problems (eight threads per sample: noise
                             for the whole horizon, then one warp integrates the next
                             chunk of steps while the others run the nearest-point
                             queries and costs of the last; the update run by each
                             instance's last CTA);
                             0 = automatic (4 when E*K <= 32768, else 1) */
  uint64_t seed;          /* Philox key */
  uint64_t step_id;       /* enters the Philox counter: (k, j, e, (step_id << 8) | iter) */
  int32_t refine_steps;   /* gradient refinement of every updated nominal before Stage II:
                             this many steps u <- clamp(u - refine_step dS(1)/du, u_min, u_max),
                             dS(1)/du of the noise-free rollout (0 = off, at most 64) */
  float refine_step;      /* their step size (default 0.05) */
} aero_params_t;

typedef struct aero_planner aero_planner_t;

/* Fill p with the paper's defaults: Table I (m = 1 kg, F in [0.3, 16.35] N,
 * |w_xy| <= 3, |w_z| <= 2 rad/s, Sigma = (1, 1, 1, 0.5) as std sqrt(Sigma),
 * dt = 50 ms, K = 128, N = 25, lambda = 0.1, Q_p = 3, Q_v = 0.25, Q_q = 1,
 * Q_vnorm = 0.15, Q_track = 15, Q_c = Q_cd = 0.5, ell = 5 m, C = 1e6, a = 5,
 * d_min = 0.4 m, d_max = 1 m), r_max = 10 m and the 120 x 60 fine grid pooled
 * 6 x 6 (Sec. IV-A), M_h x M_v = 5 x 3 (Sec. V-A), g = 9.81, seed 0. */
void aero_params_default(aero_params_t* p);

/* Create a planner on the current CUDA device and allocate its workspace for
 * the given maxima.  *out receives the handle.  Errors: INVALID_ARG (null or
 * out-of-range limit), ALLOC, CUDA. */
int aero_create(const aero_limits_t* limits, aero_planner_t** out);

/* Free the planner and its workspace (synchronises the device first).
 * A NULL planner is accepted. */
int aero_destroy(aero_planner_t* planner);

/* One planning step (see the top of this file).
 *   x0          host, the current state.
 *   cloud_xyz   device, n_points x 3 float, row-major (x, y, z), world frame;
 *               may be NULL when n_points == 0.  Non-finite points, points at
 *               p0 and points beyond r_max are ignored.
 *   goal        host, 3 floats, goal position (world).
 *   params      host.
 *   u_nom_inout device, E x T x 4 float (F, wx, wy, wz) per instance and step,
 *               16-byte aligned: the warm start on entry, the updated nominals
 *               on return.
 *   u_best_out  device, T x 4 float: the nominal of the selected instance.
 *   cand_costs_out device, E float: Stage II cost S(2) of each instance.
 *   best_idx_out device, 1 int32: index of the selected instance (lowest
 *               S(2), ties to the lower index).
 * The call only enqueues work on `stream` (it neither allocates nor
 * synchronises), so it can be captured into a CUDA graph and replayed; the
 * graph replays the captured arguments (state, goal, step_id, buffers).
 * Errors (nothing is enqueued): INVALID_ARG (also for a non-finite state,
 * goal, sigma or scalar parameter), EXCEEDS_LIMITS, NOT_DEVICE_PTR; CUDA if a
 * launch fails. */
int aero_plan_step(aero_planner_t* planner, const aero_state_t* x0, const float* cloud_xyz,
                   int64_t n_points, const float goal[3], const aero_params_t* params,
                   float* u_nom_inout, float* u_best_out, float* cand_costs_out,
                   int32_t* best_idx_out, void* stream);

/* The same step for callers whose data lives in host memory: every array
 * argument is a host pointer.  A cloud in page-locked (pinned or registered)
 * host memory is read in place by the partition pass over the host link,
 * which also stores the points in the planner's device buffer for the later
 * passes; a pageable cloud is copied into that buffer first.  The warm start
 * is copied into the planner's device buffer (pinned is fastest), the step
 * runs on `stream`, its outputs come back in one copy into the planner's
 * pinned staging buffer, and the call returns after synchronising the stream
 * and copying them into the caller's buffers.  The cloud must not change
 * during the call. */
int aero_plan_step_host(aero_planner_t* planner, const aero_state_t* x0, const float* cloud_xyz,
                        int64_t n_points, const float goal[3], const aero_params_t* params,
                        float* u_nom_inout, float* u_best_out, float* cand_costs_out,
                        int32_t* best_idx_out, void* stream);

/* The planning step of aero_plan_step for callers that cannot allocate device
 * memory while running (no counterpart in the paper: an engineering addition).
 * A flight-control loop must not block on cudaMalloc, which can synchronise
 * the device and take an unbounded time, and some host programs own all device
 * memory through their own pool; aero_create allocates, so they call this
 * instead.  No planner is needed and nothing is allocated: the workspace is a
 * fixed file-scope device array of about 7.5 MB that every GPU loading this
 * library keeps until the process exits.
 *   Limits: E <= 16, K <= 2048, T <= 64, fine_az * fine_el <= 8192,
 *   n_points <= 65536, collision_set == 0 (P_f), debug_samples == 0; the
 *   collision grid has at most 32^3 cells (coarser cells for a large r_max, which
 *   keeps the distances exact).  Larger requests return AERO_ERR_EXCEEDS_LIMITS.
 *   Arguments are those of aero_plan_step (same layout, ownership and errors);
 *   there are no debug buffers.
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any stream
 *   capture: a first call on a stream that is being captured returns
 *   AERO_ERR_INVALID_ARG.  The partition's edge tables are copied into the
 *   array from a host copy that the library keeps per device, only when the
 *   partition geometry (fine_az, fine_el, el_lo, el_hi) differs from the last
 *   call's.  All calls share the array, which keeps the last call's contents:
 *   calls whose work overlaps on the GPU (other streams, other host threads)
 *   race on it, so order them on one stream. */
int aero_plan_step_noalloc(const aero_state_t* x0, const float* cloud_xyz, int64_t n_points,
                           const float goal[3], const aero_params_t* params, float* u_nom_inout,
                           float* u_best_out, float* cand_costs_out, int32_t* best_idx_out,
                           void* stream);

/* ---- batched planning ----------------------------------------------------
 * Many independent planning steps (different drones or scenes, uneven E, K, T
 * and cloud sizes) in one call.  Each stage of the step (Sec. IV-A partition,
 * Sec. IV-B anchors and guides, the collision lists, the Stage I rollouts of
 * Sec. III-B with the update of Eq. mppi_update_simplified, Stage II and the
 * selection) runs as ONE launch over the work units of all items; the Stage I
 * launch is persistent (a fixed number of CTAs per SM) and takes its units --
 * (item, instance, block of samples), longest horizon first -- from a device
 * work queue.  The launches of a call form a CUDA graph, instantiated once per
 * batch shape (item count, largest iteration count, configuration) and then
 * replayed; a call uploads the items' arguments in one host-to-device copy and
 * launches the graph on `stream`.
 * Every item computes what aero_plan_step computes with the same
 * lanes_per_sample: the partition and grid decisions are identical and the
 * floating-point results agree to rounding (the unit code is compiled in other
 * contexts, and the batched update merges the partials with other thread
 * counts). */
typedef struct {
  aero_state_t x0;            /* current state */
  const float* cloud_xyz;     /* device, n_points x 3 float (may be NULL if n_points == 0) */
  int64_t n_points;
  float goal[3];
  aero_params_t params;       /* debug_samples must be 0 */
  float* u_nom_inout;         /* device, E x T x 4 float, 16-byte aligned */
  float* u_best_out;          /* device, T x 4 */
  float* cand_costs_out;      /* device, E */
  int32_t* best_idx_out;      /* device, 1 */
} aero_batch_item_t;

typedef struct aero_batch aero_batch_t;

/* Launch configuration of a batch (the autotuner's search space). */
typedef struct {
  int32_t quad_max_samples;    /* items with lanes_per_sample == 0 use the split pass (4)
                                  when E*K <= this, else one thread per sample */
  int32_t rollout_ctas_per_sm; /* persistent Stage I CTAs per SM; 0 = as many as fit; 6 or more
                                  also selects the one-lane kernel built for six per SM
                                  (fewer registers) */
  int32_t dynamic_queue;       /* 1: CTAs take units from the work queue; 0: strided by the grid */
  int32_t coarse_cells;        /* 1: collision-grid cells of edge d_max (1 + 1/16) (fewer list
                                  entries to build, longer lists to scan); 0: edge d_max / 2 when
                                  the candidate array can hold it.  Results do not depend on it:
                                  every list holds the nearest point of every query within d_max */
  int32_t samples_per_cta;     /* samples (threads) per CTA of the one-lane Stage I pass: 64, 128
                                  or 256 (0 = 128); rollout_ctas_per_sm counts CTAs of 128
                                  threads and is scaled for the other sizes.  The floating-point
                                  results agree to rounding (the per-CTA partial sums group the
                                  samples differently) */
} aero_batch_config_t;

/* Create a batch of up to n_max <= 256 item slots, each with a planner
 * workspace sized by `limits` (every item of a call must fit them; the limits'
 * debug_samples_max is ignored).  The default configuration is
 * {0, 0, 1, 0, 0}.  Errors: INVALID_ARG, ALLOC, CUDA. */
int aero_batch_create(const aero_limits_t* limits, int32_t n_max, aero_batch_t** out);

/* Enqueue the n <= n_max steps of `items` (host array; item i uses slot i) on
 * `stream`; returns after enqueuing.  Every item is validated first: on an
 * error nothing is enqueued (INVALID_ARG, EXCEEDS_LIMITS, NOT_DEVICE_PTR).
 * Calls on one batch must be ordered on the device (one stream, or
 * synchronised): they share the slots' workspaces and the argument buffer.
 * The host may reuse `items` as soon as the call returns. */
int aero_batch_plan(aero_batch_t* batch, const aero_batch_item_t* items, int32_t n, void* stream);

int aero_batch_set_config(aero_batch_t* batch, const aero_batch_config_t* config);
int aero_batch_get_config(aero_batch_t* batch, aero_batch_config_t* config);

/* Autotune: time every configuration of a small search space (quad_max_samples
 * in {0, 4096, 32768}; rollout_ctas_per_sm in {as many as fit, 6, half of the
 * fewest that fit}; dynamic_queue in {1, 0}; coarse_cells in {0, 1};
 * samples_per_cta in {128, 64, 256}: 108 configurations) on `items`, `repeats` timed calls each after one
 * warm-up, keep the fastest as the batch's configuration and return it with
 * its mean time in *best_ms.  The items' clouds and states are read; the
 * outputs go to scratch buffers of the batch, so the items' u_nom_inout and
 * outputs are left untouched.  Synchronous (returns when done). */
int aero_batch_tune(aero_batch_t* batch, const aero_batch_item_t* items, int32_t n, int32_t repeats,
                    void* stream, aero_batch_config_t* best, float* best_ms);

/* OR of the status words of the batch's slots (bit 0: an update's normaliser
 * was not a positive finite number; bit 1: a candidate list overflowed; bit 2:
 * no candidate had a finite S(2), the first instance was taken) and, in
 * the checked build, of the index-check bits (1 << 8 and up, see
 * aero_sync_status), which are then cleared.  Synchronous. */
int aero_batch_sync_status(aero_batch_t* batch, int32_t* status);

/* Debug copies of slot `slot`'s last step, as aero_debug_size / aero_get_debug
 * for a planner (no per-sample buffers; FINE_KEYS reads back emptied: the
 * batched step leaves its keys empty for the next call).  INVALID_ARG for a
 * slot the last call did not use. */
size_t aero_batch_debug_size(aero_batch_t* batch, int32_t slot, int32_t what);
int aero_batch_get_debug(aero_batch_t* batch, int32_t slot, int32_t what, void* dst, size_t bytes,
                         void* stream);

/* Free the batch (synchronises the device first). */
int aero_batch_destroy(aero_batch_t* batch);

/* Bytes of debug buffer `what` (AERO_DBG_*) for the last step; 0 if unknown. */
size_t aero_debug_size(aero_planner_t* planner, int32_t what);

/* S(1) and its gradient for n control sequences of instance `instance`, in the
 * context of the planner's last step (state, guide of that instance, collision
 * grid, parameters): S = the Stage I cost of the noise-free rollout of each
 * sequence (the terms of Sec. IV-C: tracking, velocity norm, control, goal,
 * collision) and dS/dU by the adjoint of the rollout (reverse mode through
 * the RK4 steps, checkpoints every 8 steps) -- the gradient the refinement
 * (refine_steps) follows.  U: device, n x T x 4 float, 16-byte aligned;
 * S_out: device, n; dSdU_out: device, n x T x 4 (16-byte aligned), or NULL for
 * the costs only.  Enqueued on `stream`; the context is valid until the
 * planner's next step.  Where a term is not differentiable (a norm at zero,
 * J_col at d_min and d_max, a tie of nearest points) the gradient of the piece
 * in use is taken.  Errors: INVALID_ARG (no step yet, instance >= E, n < 0,
 * misaligned), NOT_DEVICE_PTR. */
int aero_cost_grad(aero_planner_t* planner, int32_t instance, const float* U, int32_t n,
                   float* S_out, float* dSdU_out, void* stream);

/* ---- multi-sweep accumulation (Sec. IV-A.1) ------------------------------
 * The partition of a step sees the most recent LiDAR frames, each taken from
 * its own pose and brought into common coordinates with the transforms of state
 * estimation (the paper accumulates 10 frames, about 200,000 points).  An
 * accumulator keeps a ring of `frames` slots of `points_per_frame` points on
 * the device, in world coordinates (float x, y, z per point):
 *  - aero_accum_push transforms a frame's sensor-frame points p_s (device, n x 3,
 *    n <= points_per_frame) by the capture pose (p, q): p_w = p + R(q) p_s with
 *    q normalised and R(q) in binary32, into the oldest slot, and fills the
 *    slot's remaining points with NaN;
 *  - aero_accum_view returns the ring itself (frames x points_per_frame points):
 *    a valid cloud for aero_plan_step, whose partition drops the NaN padding;
 *  - aero_accum_gather writes the live frames' points, oldest frame first and
 *    in push order within a frame, compacted into dst (device, capacity points
 *    x 3): in world coordinates when p0 and q0 are NULL, else projected into the
 *    body frame R(q0)^T (p_w - p0) (host p0[3], q0[4]); *n_out gets the count.
 * All work is enqueued on `stream`; the caller orders pushes and readers.
 * Errors: INVALID_ARG (sizes, a zero quaternion, capacity), NOT_DEVICE_PTR,
 * ALLOC, CUDA. */
typedef struct aero_accum aero_accum_t;
int aero_accum_create(int32_t frames, int64_t points_per_frame, aero_accum_t** out);
int aero_accum_push(aero_accum_t* acc, const float* pts_sensor, int64_t n, const float pose_p[3],
                    const float pose_q[4], void* stream);
int aero_accum_view(aero_accum_t* acc, const float** cloud, int64_t* n_points, int64_t* n_valid);
int aero_accum_gather(aero_accum_t* acc, const float* p0, const float* q0, float* dst,
                      int64_t dst_capacity, int64_t* n_out, void* stream);
int aero_accum_reset(aero_accum_t* acc, void* stream);  /* forget every frame */
int aero_accum_destroy(aero_accum_t* acc);

/* Receding-horizon warm start: after `shift` executed steps, every instance's
 * nominal moves forward, u[e][j] = u[e][min(j + shift, T - 1)] (the last control
 * repeated).  u_nom: device E x T x 4, in place; scratch: device, E x T x 4
 * floats the call may overwrite.  Enqueued on `stream`.  Errors: INVALID_ARG,
 * NOT_DEVICE_PTR, CUDA. */
int aero_shift_nominal(float* u_nom, int32_t E, int32_t T, int32_t shift, float* scratch,
                       void* stream);

/* ---- test hooks ----------------------------------------------------------
 * Every device and pinned host allocation of the library (aero_create,
 * aero_batch_create, aero_accum_create) is counted.  aero_test_fail_alloc(n)
 * makes the n-th next allocation (0 = the next one) return
 * cudaErrorMemoryAllocation once, so that a test can drive each error path of
 * the create functions (they return AERO_ERR_ALLOC and free what they had
 * allocated); n < 0 cancels a pending failure.  aero_test_alloc_stats returns
 * the number of allocations made since the library was loaded and stores the
 * number not yet freed in *live (when live is not null).  Process-wide; not
 * meant for production callers. */
int aero_test_fail_alloc(int64_t n);
int64_t aero_test_alloc_stats(int64_t* live);
/* Checked build only: record `bits` (> 0) as if an index check had failed, so
 * that a test can see aero_sync_status report it; the product build returns
 * AERO_ERR_INVALID_ARG. */
int aero_test_raise_check(int32_t bits);

/* Copy debug buffer `what` of the last step into dst (host or device), at most
 * `bytes` bytes, ordered on `stream` (asynchronous for device dst and pinned
 * host dst).  Errors: INVALID_ARG (unknown id, no step yet, bytes too small). */
int aero_get_debug(aero_planner_t* planner, int32_t what, void* dst, size_t bytes, void* stream);

/* Synchronise `stream`, then report the kernels' status word: AERO_OK, or
 * DEVICE_CHECK when a kernel recorded an internal inconsistency or a
 * non-finite result (an update's normaliser not a positive finite number, a
 * candidate list overflow, no candidate with a finite S(2): the first instance
 * is then the one selected), or CUDA when the stream holds an error.  Clears
 * the status word.
 * The checked build of the library (libaero_mppi_checked.so, compiled with
 * AERO_CHECKED) also guards the indices the kernels rely on (fine cell, grid
 * cell, candidate range, query slot and item, partial row, accumulation slot):
 * a failed check skips the access and is reported here as DEVICE_CHECK (it then
 * synchronises the device).  The product build has no such checks. */
int aero_sync_status(aero_planner_t* planner, void* stream);

/* ---- stage timing --------------------------------------------------------
 * aero_profile_enable(planner, stages): `stages` is a bitmask of
 * (1 << AERO_STAGE_*); aero_plan_step then records a pair of CUDA events on its
 * stream around each selected stage (every event costs a little device time,
 * so select only the stages you need; 0 turns timing off).  aero_profile_read
 * synchronises them, adds the elapsed device times since the last read into
 * ms[AERO_STAGE_COUNT] and the number of kernel launches per timed stage into
 * launches[AERO_STAGE_COUNT], and starts over.
 *   AERO_STAGE_PARTITION: workspace clears + fine partition (Sec. IV-A.1)
 *   AERO_STAGE_GRID: P_f / grid counts, coarse argmax + anchors + guides with the
 *                    grid scan, grid scatter (Sec. IV-A.2, IV-B)
 *   AERO_STAGE_ROLLOUT: sampling, rollouts and S(1) (Sec. III-B, IV-C)
 *   AERO_STAGE_UPDATE: weights, update, Stage II and selection */
#define AERO_STAGE_PARTITION 0
#define AERO_STAGE_GRID 1
#define AERO_STAGE_ROLLOUT 2
#define AERO_STAGE_UPDATE 3
#define AERO_STAGE_COUNT 4
int aero_profile_enable(aero_planner_t* planner, int stages);
int aero_profile_read(aero_planner_t* planner, double* ms, int64_t* launches);

/* Test hook for the noise generator (Sec. III-B): out[4i .. 4i+3] =
 * Philox4x32-10(counter = (i, c1, c2, c3), key = (lo32(seed), hi32(seed))) for
 * i < n.  out is device memory of 4n uint32. */
int aero_philox(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, int64_t n, uint32_t* out,
                void* stream);

/* Static description of a status code. */
const char* aero_status_str(int status);

#ifdef __cplusplus
}
#endif

#endif /* AERO_MPPI_H */
