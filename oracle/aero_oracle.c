/*
 * AERO-MPPI planning step -- CPU ORACLE (test infrastructure only).
 *
 * A plain, slow, double-precision restatement of one planning step of
 * "AERO-MPPI: Anchor-Guided Ensemble Trajectory Optimization for Agile Mapless
 * Drone Navigation" (arXiv 2509.17340).  It exists so that the CUDA planner can
 * be checked against something written straight from the paper.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * planner library never calls it and shares no code, header or table with it.
 *
 * Order of the steps (as in Sec. IV of the paper):
 *   fine spherical partition (Sec. IV-A.1) -> cell directions (Eq. "unit
 *   direction") -> coarse pooling argmax (Eq. safe-vector) -> initial endpoints
 *   around the goal direction (Sec. IV-B.1) -> anchors (Eq. anchor-point) ->
 *   quintic guides (Eq. polynomial) -> Gaussian perturbations (Sec. III-B) ->
 *   dynamics (Eq. dynamics) with RK4 (Eq. mppi_rollout_simplified) -> costs
 *   (Eq. total cost and the five cost terms of Sec. IV-C) -> weights
 *   (Eq. mppi_weights) -> update (Eq. mppi_update_simplified) -> Stage II
 *   re-rollout and argmin (Sec. IV-C).
 *
 * Precision.  Everything is binary64 except the integer decisions of the
 * partition (which cone a point falls in, its range key, which cone wins),
 * which are taken in binary32 with a fixed sequence of correctly rounded
 * operations, because the planner takes them in binary32.  This file must be
 * compiled with -ffp-contract=off so that no multiply-add is fused.
 *
 * Nearest-obstacle distances are brute force over the whole collision set.
 * Noise is drawn from an own Philox4x32-10 (Salmon et al., SC'11) and mapped to
 * normals with the Box-Muller transform in binary64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
  int32_t E, K, T, iters;
  double dt, lam, mass, g;
  double sigma[4], u_min[4], u_max[4];
  double Q_track, Q_vnorm, Q_c, Q_cd, Q_p, Q_v, Q_q;
  double C_col, a_col, d_min, d_max;
  double r_max, ell, v_end;
  int32_t A_f, E_f, P_a, P_e, M_h, M_v;
  double el_lo, el_hi;
  int32_t collision_set; /* 0: filtered cloud P_f, 1: every in-range point */
  int32_t pad_;
  double v_goal[3], q_goal[4];
  uint64_t seed, step_id;
  int32_t refine_steps;  /* gradient steps on each updated nominal before Stage II */
  int32_t pad2_;
  double refine_step;    /* their step size */
} orc_params;

#define ORC_EMPTY 0xFFFFFFFFFFFFFFFFull

/* ======================================================================
 * Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two
 * 32x32->64 multiplies, with the key bumped by the Weyl constants between
 * rounds.
 * ====================================================================== */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)pb;
    uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)pa;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1): the top 23 bits of a word, centred, (2m+1) 2^-24. */
static double u01(uint32_t w) { return (double)(2u * (w >> 9) + 1u) * 0x1p-24; }

/* Sec. III-B: delta ~ N(0, Sigma) with Sigma = diag(sigma^2).  Counter
 * (k, j, e, (step_id << 8) | iter), key = seed; Box-Muller on (u0,u1), (u2,u3). */
void orc_noise(const orc_params* P, int e, int k, int j, int iter, double delta[4]) {
  uint32_t ctr[4] = {(uint32_t)k, (uint32_t)j, (uint32_t)e,
                     (uint32_t)((P->step_id << 8) | (uint64_t)(uint32_t)iter)};
  uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  double ra = sqrt(-2.0 * log(u01(w[0])));
  double rb = sqrt(-2.0 * log(u01(w[2])));
  double n[4] = {ra * cos(2.0 * M_PI * u01(w[1])), ra * sin(2.0 * M_PI * u01(w[1])),
                 rb * cos(2.0 * M_PI * u01(w[3])), rb * sin(2.0 * M_PI * u01(w[3]))};
  for (int c = 0; c < 4; ++c) delta[c] = P->sigma[c] * n[c];
}

/* delta for samples k0 .. k0+nk-1 of instance e, all T steps: nk x T x 4. */
void orc_noise_fill(const orc_params* P, int e, int k0, int nk, int iter, double* out) {
  for (int a = 0; a < nk; ++a)
    for (int j = 0; j < P->T; ++j) orc_noise(P, e, k0 + a, j, iter, out + ((int64_t)a * P->T + j) * 4);
}

/* ======================================================================
 * Quadrotor model (Eq. dynamics): p' = v, q' = 1/2 q (x) [0, w],
 * v' = (1/m) R(q) [0,0,F]^T + g, with g = (0,0,-g) and u = (F, w).
 * ====================================================================== */

/* Hamilton product a (x) b, quaternions as (w, x, y, z). */
void orc_quat_mul(const double a[4], const double b[4], double r[4]) {
  r[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  r[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  r[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  r[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

/* R(q): rotation matrix of the unit quaternion q (body to world), row-major. */
void orc_rotation(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* State x = [p(3), q(4), v(3)], control u = [F, wx, wy, wz]. */
void orc_dynamics(const double x[10], const double u[4], double m, double g, double xd[10]) {
  const double* q = x + 3;
  const double* v = x + 7;
  double om[4] = {0.0, u[1], u[2], u[3]};
  double qo[4], R[9];
  orc_quat_mul(q, om, qo);
  orc_rotation(q, R);
  for (int i = 0; i < 3; ++i) xd[i] = v[i];
  for (int i = 0; i < 4; ++i) xd[3 + i] = 0.5 * qo[i];
  double f[3] = {0.0, 0.0, u[0]};
  for (int i = 0; i < 3; ++i)
    xd[7 + i] = (R[3 * i + 0] * f[0] + R[3 * i + 1] * f[1] + R[3 * i + 2] * f[2]) / m;
  xd[9] -= g;
}

/* Eq. mppi_rollout_simplified: classical RK4 with the control held over the
 * step, followed by renormalising the quaternion to unit length. */
void orc_rk4_step(const double x[10], const double u[4], double dt, double m, double g,
                  double xn[10]) {
  double k1[10], k2[10], k3[10], k4[10], t[10];
  orc_dynamics(x, u, m, g, k1);
  for (int i = 0; i < 10; ++i) t[i] = x[i] + 0.5 * dt * k1[i];
  orc_dynamics(t, u, m, g, k2);
  for (int i = 0; i < 10; ++i) t[i] = x[i] + 0.5 * dt * k2[i];
  orc_dynamics(t, u, m, g, k3);
  for (int i = 0; i < 10; ++i) t[i] = x[i] + dt * k3[i];
  orc_dynamics(t, u, m, g, k4);
  for (int i = 0; i < 10; ++i) xn[i] = x[i] + dt / 6.0 * (k1[i] + 2 * k2[i] + 2 * k3[i] + k4[i]);
  double nq = sqrt(xn[3] * xn[3] + xn[4] * xn[4] + xn[5] * xn[5] + xn[6] * xn[6]);
  for (int i = 3; i < 7; ++i) xn[i] /= nq;
}

/* X[(T+1) x 10]: X[0] = x0, X[j+1] = RK4(X[j], U[j]). */
void orc_rollout(const double x0[10], const double* U, int T, double dt, double m, double g,
                 double* X) {
  memcpy(X, x0, 10 * sizeof(double));
  for (int j = 0; j < T; ++j) orc_rk4_step(X + 10 * j, U + 4 * j, dt, m, g, X + 10 * (j + 1));
}

/* ======================================================================
 * Multi-resolution partition (Sec. IV-A).  Integer decisions in binary32.
 * ====================================================================== */

static uint32_t fbits(float f) {
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
}

/* R(q0) in binary32: nine products, then the sums of the unit-quaternion formula. */
static void rot_f32(const float q[4], float R[9]) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  float wx = w * x, wy = w * y, wz = w * z;
  R[0] = 1.0f - 2.0f * (yy + zz); R[1] = 2.0f * (xy - wz);        R[2] = 2.0f * (xz + wy);
  R[3] = 2.0f * (xy + wz);        R[4] = 1.0f - 2.0f * (xx + zz); R[5] = 2.0f * (yz - wx);
  R[6] = 2.0f * (xz - wy);        R[7] = 2.0f * (yz + wx);        R[8] = 1.0f - 2.0f * (xx + yy);
}

/* Body-frame coordinates b = R(q0)^T (p - p0) in binary32, left to right. */
static void to_body_f32(const float R[9], const float p0[3], const float p[3], float b[3]) {
  float dx = p[0] - p0[0], dy = p[1] - p0[1], dz = p[2] - p0[2];
  b[0] = R[0] * dx + R[3] * dy + R[6] * dz;
  b[1] = R[1] * dx + R[4] * dy + R[7] * dz;
  b[2] = R[2] * dx + R[5] * dy + R[8] * dz;
}

typedef struct {
  int A, El;
  float* ca; float* sa;   /* A entries: azimuth edges theta_k = pi (2k - A) / A */
  float* ce; float* se;   /* El+1 entries: elevation edges phi_k = lo + ((hi-lo) k) / El */
  int check_lo, check_hi;
} orc_edges;

static void edges_make(const orc_params* P, orc_edges* ed) {
  ed->A = P->A_f;
  ed->El = P->E_f;
  ed->ca = malloc(sizeof(float) * ed->A);
  ed->sa = malloc(sizeof(float) * ed->A);
  ed->ce = malloc(sizeof(float) * (ed->El + 1));
  ed->se = malloc(sizeof(float) * (ed->El + 1));
  for (int k = 0; k < ed->A; ++k) {
    double th = (M_PI * (double)(2 * k - ed->A)) / (double)ed->A;
    ed->ca[k] = (float)cos(th);
    ed->sa[k] = (float)sin(th);
  }
  double lo = (double)(float)P->el_lo, hi = (double)(float)P->el_hi;
  for (int k = 0; k <= ed->El; ++k) {
    double ph = lo + ((hi - lo) * (double)k) / (double)ed->El;
    ed->ce[k] = (float)cos(ph);
    ed->se[k] = (float)sin(ph);
  }
  ed->check_lo = lo > -M_PI / 2;
  ed->check_hi = hi < M_PI / 2;
}

static void edges_free(orc_edges* ed) {
  free(ed->ca); free(ed->sa); free(ed->ce); free(ed->se);
}

/* Largest index in [lo, hi] whose edge the direction has reached, by bisection
 * on the sign of a cross product; lo itself is taken as reached. */
static int az_bin(const orc_edges* ed, float bx, float by) {
  int half = ed->A / 2;
  int upper = (by > 0.0f) || (by == 0.0f && bx > 0.0f);
  int lo = upper ? half : 0, hi = upper ? ed->A - 1 : half - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    float s = by * ed->ca[mid] - bx * ed->sa[mid];
    if (s >= 0.0f) lo = mid; else hi = mid - 1;
  }
  return lo;
}

static int el_bin(const orc_edges* ed, float bz, float rho) {
  int lo = 0, hi = ed->El - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    float s = bz * ed->ce[mid] - rho * ed->se[mid];
    if (s >= 0.0f) lo = mid; else hi = mid - 1;
  }
  return lo;
}

/* Fine cell of one point, or -1 when the point is not in P_t (non-finite,
 * at the origin, beyond r_max or outside the elevation span).  Writes r^2. */
static int fine_cell(const orc_edges* ed, const float R[9], const float p0[3], float rmax2,
                     const float p[3], float* r2out) {
  if (!isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2])) return -1;
  float b[3];
  to_body_f32(R, p0, p, b);
  float r2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  if (!(r2 > 0.0f) || r2 > rmax2) return -1;
  float rho = sqrtf(b[0] * b[0] + b[1] * b[1]);
  if (ed->check_lo && !(b[2] * ed->ce[0] - rho * ed->se[0] >= 0.0f)) return -1;
  if (ed->check_hi && (b[2] * ed->ce[ed->El] - rho * ed->se[ed->El] > 0.0f)) return -1;
  int i = az_bin(ed, b[0], b[1]);
  int j = el_bin(ed, b[2], rho);
  *r2out = r2;
  return j * ed->A + i;
}

/* Sec. IV-A.1: r_ij = min |p_c| over P_t in cone C_ij.  Key of a point is
 * (bits(r^2) << 32) | index, so the minimum key is the nearest point, lowest
 * index first; an empty cone keeps ORC_EMPTY.  Returns the number of points kept. */
int64_t orc_partition(const float* cloud, int64_t n, const float p0[3], const float q0[4],
                      const orc_params* P, uint64_t* keys) {
  orc_edges ed;
  edges_make(P, &ed);
  float R[9];
  rot_f32(q0, R);
  float rm = (float)P->r_max;
  float rmax2 = rm * rm;
  int ncell = P->A_f * P->E_f;
  for (int c = 0; c < ncell; ++c) keys[c] = ORC_EMPTY;
  int64_t kept = 0;
  for (int64_t i = 0; i < n; ++i) {
    float r2;
    int c = fine_cell(&ed, R, p0, rmax2, cloud + 3 * i, &r2);
    if (c < 0) continue;
    ++kept;
    uint64_t key = ((uint64_t)fbits(r2) << 32) | (uint64_t)(uint32_t)i;
    if (key < keys[c]) keys[c] = key;
  }
  edges_free(&ed);
  return kept;
}

/* Fine cell of the goal direction (no range or span test). */
int orc_goal_fine_cell(const float goal[3], const float p0[3], const float q0[4],
                       const orc_params* P) {
  orc_edges ed;
  edges_make(P, &ed);
  float R[9], b[3];
  rot_f32(q0, R);
  to_body_f32(R, p0, goal, b);
  float rho = sqrtf(b[0] * b[0] + b[1] * b[1]);
  int c = el_bin(&ed, b[2], rho) * ed.A + az_bin(&ed, b[0], b[1]);
  edges_free(&ed);
  return c;
}

/* Eq. "unit direction": d_ij at the cone centre (alpha_i, beta_j). */
void orc_cell_direction(const orc_params* P, int c, double d[3]) {
  int i = c % P->A_f, j = c / P->A_f;
  double lo = (double)(float)P->el_lo, hi = (double)(float)P->el_hi;
  double al = -M_PI + (i + 0.5) * (2.0 * M_PI / P->A_f);
  double be = lo + (j + 0.5) * ((hi - lo) / P->E_f);
  d[0] = cos(be) * cos(al);
  d[1] = cos(be) * sin(al);
  d[2] = sin(be);
}

/* Eq. safe-vector: (i*, j*) = argmax over Omega_IJ of r_ij.  Empty cones count
 * as r_max.  Ties: nearer to the coarse-cell centre (doubled L1 index
 * distance), then the lower fine index.  Writes the winning fine cell per coarse
 * cell (A_c * E_c, coarse index J*A_c + I) and r of the winner. */
void orc_coarse(const uint64_t* keys, const orc_params* P, int32_t* win, double* rwin) {
  int A_c = P->A_f / P->P_a, E_c = P->E_f / P->P_e;
  float rm = (float)P->r_max;
  uint32_t empty_bits = fbits(rm * rm);
  for (int J = 0; J < E_c; ++J)
    for (int I = 0; I < A_c; ++I) {
      int best = -1, bdist = 0;
      uint32_t bkey = 0;
      for (int b = 0; b < P->P_e; ++b)
        for (int a = 0; a < P->P_a; ++a) {
          int i = I * P->P_a + a, j = J * P->P_e + b;
          int c = j * P->A_f + i;
          uint32_t rk = keys[c] == ORC_EMPTY ? empty_bits : (uint32_t)(keys[c] >> 32);
          int dist = abs(2 * a + 1 - P->P_a) + abs(2 * b + 1 - P->P_e);
          int better = best < 0 || rk > bkey || (rk == bkey && dist < bdist) ||
                       (rk == bkey && dist == bdist && c < best);
          if (better) { best = c; bkey = rk; bdist = dist; }
        }
      win[J * A_c + I] = best;
      float r2;
      memcpy(&r2, &bkey, 4);
      rwin[J * A_c + I] = sqrt((double)r2);
    }
}

/* Sec. IV-B.1: the M_h x M_v coarse cells centred on the goal's coarse cell
 * (azimuth wraps, elevation clamps); instance e = n*M_h + m. */
void orc_anchor_cells(int goal_fine, const orc_params* P, int32_t* cells) {
  int A_c = P->A_f / P->P_a, E_c = P->E_f / P->P_e;
  int Ig = (goal_fine % P->A_f) / P->P_a, Jg = (goal_fine / P->A_f) / P->P_e;
  for (int n = 0; n < P->M_v; ++n)
    for (int m = 0; m < P->M_h; ++m) {
      int I = ((Ig + m - P->M_h / 2) % A_c + A_c) % A_c;
      int J = Jg + n - P->M_v / 2;
      if (J < 0) J = 0;
      if (J > E_c - 1) J = E_c - 1;
      cells[n * P->M_h + m] = J * A_c + I;
    }
}

/* Eq. anchor-point: p_ref = p0 + ell * d_IJ, the direction taken from the body
 * frame into the world frame with R(q0). */
void orc_anchor(const double p0[3], const double q0[4], const double d_body[3], double ell,
                double pref[3]) {
  double R[9];
  orc_rotation(q0, R);
  for (int i = 0; i < 3; ++i)
    pref[i] = p0[i] + ell * (R[3 * i] * d_body[0] + R[3 * i + 1] * d_body[1] + R[3 * i + 2] * d_body[2]);
}

/* Solve A x = b (n x n, row-major, destroyed) by Gaussian elimination with
 * partial pivoting. */
static void solve_dense(double* A, double* b, int n) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
    if (p != c) {
      for (int k = 0; k < n; ++k) { double t = A[c * n + k]; A[c * n + k] = A[p * n + k]; A[p * n + k] = t; }
      double t = b[c]; b[c] = b[p]; b[p] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
    b[r] = s / A[r * n + r];
  }
}

/* Eq. polynomial: f(t) = sum_i a_i t^i on [0, Tg] fixed by position, velocity
 * and acceleration at both ends; one 6x6 system per axis. */
void orc_quintic(const double p_s[3], const double v_s[3], const double a_s[3],
                 const double p_e[3], const double v_e[3], const double a_e[3], double Tg,
                 double coef[18]) {
  for (int mu = 0; mu < 3; ++mu) {
    double A[36] = {0}, b[6];
    /* rows: f(0), f'(0), f''(0), f(T), f'(T), f''(T) */
    for (int i = 0; i < 6; ++i) {
      A[0 * 6 + i] = i == 0 ? 1.0 : 0.0;
      A[1 * 6 + i] = i == 1 ? 1.0 : 0.0;
      A[2 * 6 + i] = i == 2 ? 2.0 : 0.0;
      A[3 * 6 + i] = pow(Tg, i);
      A[4 * 6 + i] = i >= 1 ? i * pow(Tg, i - 1) : 0.0;
      A[5 * 6 + i] = i >= 2 ? i * (i - 1) * pow(Tg, i - 2) : 0.0;
    }
    b[0] = p_s[mu]; b[1] = v_s[mu]; b[2] = a_s[mu];
    b[3] = p_e[mu]; b[4] = v_e[mu]; b[5] = a_e[mu];
    solve_dense(A, b, 6);
    for (int i = 0; i < 6; ++i) coef[mu * 6 + i] = b[i];
  }
}

double orc_poly_eval(const double coef6[6], double t) {
  double s = 0.0;
  for (int i = 0; i < 6; ++i) s += coef6[i] * pow(t, i);
  return s;
}

/* Guide of instance e: p(0)=p0, v(0)=v0, a(0)=0; p(Tg)=p_ref,
 * v(Tg)=v_end * unit(p_ref - p0), a(Tg)=0, Tg = T dt; sampled at t = (j+1) dt. */
void orc_guide(const double p0[3], const double v0[3], const double pref[3], const orc_params* P,
               double coef[18], double* guide /* T x 3 */) {
  double Tg = P->T * P->dt;
  double v_end = P->v_end > 0 ? P->v_end : P->ell / Tg;
  double dp[3] = {pref[0] - p0[0], pref[1] - p0[1], pref[2] - p0[2]};
  double L = sqrt(dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2]);
  double ve[3], zero[3] = {0, 0, 0};
  for (int i = 0; i < 3; ++i) ve[i] = L > 0 ? v_end * dp[i] / L : 0.0;
  orc_quintic(p0, v0, zero, pref, ve, zero, Tg, coef);
  for (int j = 0; j < P->T; ++j)
    for (int mu = 0; mu < 3; ++mu) guide[3 * j + mu] = orc_poly_eval(coef + 6 * mu, (j + 1) * P->dt);
}

/* ======================================================================
 * Costs (Sec. IV-C)
 * ====================================================================== */

/* d_t = min over the collision set of |p - p_obs| (brute force); +inf if empty. */
double orc_nn_dist(const double p[3], const double* pts, int64_t n) {
  double best = INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    double dx = p[0] - pts[3 * i], dy = p[1] - pts[3 * i + 1], dz = p[2] - pts[3 * i + 2];
    double d = sqrt(dx * dx + dy * dy + dz * dz);
    if (d < best) best = d;
  }
  return best;
}

/* Piecewise collision penalty J_col,t. */
double orc_jcol(double d, const orc_params* P) {
  if (d < P->d_min) return P->C_col;
  if (d < P->d_max) return P->C_col * exp(-P->a_col * (d - P->d_min));
  return 0.0;
}

static double norm3(const double a[3]) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* || R(q) R(q_goal)^T - I ||_F from the two matrices. */
double orc_attitude_err(const double q[4], const double qg[4]) {
  double R[9], Rg[9], s = 0.0;
  orc_rotation(q, R);
  orc_rotation(qg, Rg);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double m = 0.0;
      for (int k = 0; k < 3; ++k) m += R[3 * r + k] * Rg[3 * c + k];
      m -= (r == c) ? 1.0 : 0.0;
      s += m * m;
    }
  return sqrt(s);
}

/* Per-step goal term: Q_p|p-p_goal| + Q_v|v-v_goal| + Q_q||R R_g^T - I||_F. */
static double goal_term(const double* x, const double goal[3], const orc_params* P) {
  double dp[3] = {x[0] - goal[0], x[1] - goal[1], x[2] - goal[2]};
  double dv[3] = {x[7] - P->v_goal[0], x[8] - P->v_goal[1], x[9] - P->v_goal[2]};
  return P->Q_p * norm3(dp) + P->Q_v * norm3(dv) + P->Q_q * orc_attitude_err(x + 3, P->q_goal);
}

/* Cost terms of one rollout.  X holds the T+1 states, the terms use the
 * post-step states X[j+1] against guide sample j (time (j+1) dt).  terms[6] =
 * {J_track, J_vnorm, J_ctrl, J_goal, J_col, S}: S = S^(1) when stage == 1 and
 * S^(2) = J_goal + J_col when stage == 2.  dist (optional, T) gets d_t. */
void orc_cost_terms(const double* X, const double* U, const double* guide, const double goal[3],
                    const double* pts, int64_t npts, const orc_params* P, int stage,
                    double terms[6], double* dist) {
  double jt = 0, jv = 0, jc = 0, jg = 0, jl = 0;
  int T = P->T;
  for (int j = 0; j < T; ++j) {
    const double* x = X + 10 * (j + 1);
    if (guide) {
      double e[3] = {x[0] - guide[3 * j], x[1] - guide[3 * j + 1], x[2] - guide[3 * j + 2]};
      jt += P->Q_track * norm3(e);
    }
    jv += P->Q_vnorm * (x[7] * x[7] + x[8] * x[8] + x[9] * x[9]);
    jg += goal_term(x, goal, P);
    double d = orc_nn_dist(x, pts, npts);
    if (dist) dist[j] = d;
    jl += orc_jcol(d, P);
  }
  /* J_ctrl: sum_{t=0}^{N-2} Q_c|u_t|^2 + sum_{t=1}^{N-2} Q_cd|u_t - u_{t-1}|^2 */
  for (int t = 0; t <= T - 2; ++t) {
    const double* u = U + 4 * t;
    jc += P->Q_c * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
  }
  for (int t = 1; t <= T - 2; ++t) {
    double s = 0.0;
    for (int c = 0; c < 4; ++c) {
      double du = U[4 * t + c] - U[4 * (t - 1) + c];
      s += du * du;
    }
    jc += P->Q_cd * s;
  }
  terms[0] = jt; terms[1] = jv; terms[2] = jc; terms[3] = jg; terms[4] = jl;
  terms[5] = stage == 1 ? jt + jv + jc + jg + jl : jg + jl;
}

/* ======================================================================
 * Gradient of S^(1) with respect to the controls, by reverse mode through
 * the rollout (not a step of the paper: it serves the gradient refinement of
 * the updated nominals before Stage II).  Written out from the definitions
 * above: the dynamics, the literal RK4 stages, the renormalisation, and the
 * cost terms of orc_cost_terms with stage 1.  Where a term is not
 * differentiable (a norm at zero, J_col at d_min and d_max, a tie between
 * nearest points) its gradient is taken from the piece in use: zero for a
 * zero norm, the collision term's own branch.
 * ====================================================================== */

/* w^T d(xd)/dx added to gx and w^T d(xd)/du added to gu, for xd = f(x, u) of
 * orc_dynamics. */
static void dyn_vjp(const double x[10], const double u[4], double m, const double w[10],
                    double gx[10], double gu[4]) {
  const double qw = x[3], qx = x[4], qy = x[5], qz = x[6];
  const double ox = u[1], oy = u[2], oz = u[3];
  /* p' = v */
  for (int i = 0; i < 3; ++i) gx[7 + i] += w[i];
  /* q' = 1/2 q (x) [0, w]: components
   *   r0 = -qx ox - qy oy - qz oz,  r1 = qw ox + qy oz - qz oy,
   *   r2 = qw oy - qx oz + qz ox,   r3 = qw oz + qx oy - qy ox */
  const double W0 = 0.5 * w[3], W1 = 0.5 * w[4], W2 = 0.5 * w[5], W3 = 0.5 * w[6];
  gx[3] += W1 * ox + W2 * oy + W3 * oz;
  gx[4] += -W0 * ox - W2 * oz + W3 * oy;
  gx[5] += -W0 * oy + W1 * oz - W3 * ox;
  gx[6] += -W0 * oz - W1 * oy + W2 * ox;
  gu[1] += -W0 * qx + W1 * qw + W2 * qz - W3 * qy;
  gu[2] += -W0 * qy - W1 * qz + W2 * qw + W3 * qx;
  gu[3] += -W0 * qz + W1 * qy - W2 * qx + W3 * qw;
  /* v' = (F/m) (R[2], R[5], R[8]) + (0, 0, -g) with
   *   R[2] = 2(xz + wy), R[5] = 2(yz - wx), R[8] = 1 - 2(x^2 + y^2) */
  const double V0 = w[7], V1 = w[8], V2 = w[9];
  const double r2 = 2 * (qx * qz + qw * qy), r5 = 2 * (qy * qz - qw * qx), r8 = 1 - 2 * (qx * qx + qy * qy);
  gu[0] += (V0 * r2 + V1 * r5 + V2 * r8) / m;
  const double s = u[0] / m;
  gx[3] += s * (2 * qy * V0 - 2 * qx * V1);
  gx[4] += s * (2 * qz * V0 - 2 * qw * V1 - 4 * qx * V2);
  gx[5] += s * (2 * qw * V0 + 2 * qz * V1 - 4 * qy * V2);
  gx[6] += s * (2 * qx * V0 + 2 * qy * V1);
}

/* Reverse of one orc_rk4_step: given lam = dS/d(xn), set gx = dS/dx through
 * this step and add dS/du to gu. */
static void rk4_vjp(const double x[10], const double u[4], double dt, double m, double g,
                    const double lam[10], double gx[10], double gu[4]) {
  double k1[10], k2[10], k3[10], k4[10], t2[10], t3[10], t4[10], y[10];
  orc_dynamics(x, u, m, g, k1);
  for (int i = 0; i < 10; ++i) t2[i] = x[i] + 0.5 * dt * k1[i];
  orc_dynamics(t2, u, m, g, k2);
  for (int i = 0; i < 10; ++i) t3[i] = x[i] + 0.5 * dt * k2[i];
  orc_dynamics(t3, u, m, g, k3);
  for (int i = 0; i < 10; ++i) t4[i] = x[i] + dt * k3[i];
  orc_dynamics(t4, u, m, g, k4);
  for (int i = 0; i < 10; ++i) y[i] = x[i] + dt / 6.0 * (k1[i] + 2 * k2[i] + 2 * k3[i] + k4[i]);
  /* renormalisation qn = y_q / |y_q|: dqn/dy_q = (I - qn qn^T) / |y_q| */
  double ly[10];
  memcpy(ly, lam, sizeof(ly));
  const double nq = sqrt(y[3] * y[3] + y[4] * y[4] + y[5] * y[5] + y[6] * y[6]);
  double dot = 0.0;
  for (int i = 3; i < 7; ++i) dot += (y[i] / nq) * lam[i];
  for (int i = 3; i < 7; ++i) ly[i] = (lam[i] - (y[i] / nq) * dot) / nq;
  /* y = x + dt/6 (k1 + 2 k2 + 2 k3 + k4) */
  double l1[10], l2[10], l3[10], l4[10], lt[10];
  for (int i = 0; i < 10; ++i) {
    gx[i] = ly[i];
    l1[i] = dt / 6.0 * ly[i];
    l2[i] = dt / 3.0 * ly[i];
    l3[i] = dt / 3.0 * ly[i];
    l4[i] = dt / 6.0 * ly[i];
  }
  /* k4 = f(t4), t4 = x + dt k3 */
  memset(lt, 0, sizeof(lt));
  dyn_vjp(t4, u, m, l4, lt, gu);
  for (int i = 0; i < 10; ++i) { gx[i] += lt[i]; l3[i] += dt * lt[i]; }
  /* k3 = f(t3), t3 = x + dt/2 k2 */
  memset(lt, 0, sizeof(lt));
  dyn_vjp(t3, u, m, l3, lt, gu);
  for (int i = 0; i < 10; ++i) { gx[i] += lt[i]; l2[i] += 0.5 * dt * lt[i]; }
  /* k2 = f(t2), t2 = x + dt/2 k1 */
  memset(lt, 0, sizeof(lt));
  dyn_vjp(t2, u, m, l2, lt, gu);
  for (int i = 0; i < 10; ++i) { gx[i] += lt[i]; l1[i] += 0.5 * dt * lt[i]; }
  /* k1 = f(x) */
  dyn_vjp(x, u, m, l1, gx, gu);
}

/* dR[k][i] = d R[k] / d q_i of orc_rotation (q = (w, x, y, z)). */
static void rotation_grad(const double q[4], double dR[9][4]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  const double t[9][4] = {
      {0, 0, -4 * y, -4 * z},          {-2 * z, 2 * y, 2 * x, -2 * w}, {2 * y, 2 * z, 2 * w, 2 * x},
      {2 * z, 2 * y, 2 * x, 2 * w},    {0, -4 * x, 0, -4 * z},         {-2 * x, -2 * w, 2 * z, 2 * y},
      {-2 * y, 2 * z, -2 * w, 2 * x},  {2 * x, 2 * w, 2 * z, 2 * y},   {0, -4 * x, -4 * y, 0}};
  memcpy(dR, t, sizeof(t));
}

static void add_unit(double* g, const double* e, double n, double wgt) {
  if (n > 0)
    for (int i = 0; i < 3; ++i) g[i] += wgt * e[i] / n;
}

/* Stage I state terms at the post-step state x (guide sample gj or NULL) and
 * their gradient gx (overwritten); returns the terms' value. */
static double state_cost_grad(const double* x, const double* gj, const double goal[3],
                              const double* pts, int64_t npts, const orc_params* P, double gx[10]) {
  double c = 0.0;
  memset(gx, 0, 10 * sizeof(double));
  if (gj) {
    double e[3] = {x[0] - gj[0], x[1] - gj[1], x[2] - gj[2]};
    double n = norm3(e);
    c += P->Q_track * n;
    add_unit(gx, e, n, P->Q_track);
  }
  c += P->Q_vnorm * (x[7] * x[7] + x[8] * x[8] + x[9] * x[9]);
  for (int i = 0; i < 3; ++i) gx[7 + i] += 2 * P->Q_vnorm * x[7 + i];
  double dp[3] = {x[0] - goal[0], x[1] - goal[1], x[2] - goal[2]};
  double dv[3] = {x[7] - P->v_goal[0], x[8] - P->v_goal[1], x[9] - P->v_goal[2]};
  double np = norm3(dp), nv = norm3(dv);
  c += P->Q_p * np + P->Q_v * nv;
  add_unit(gx, dp, np, P->Q_p);
  add_unit(gx + 7, dv, nv, P->Q_v);
  /* ||R(q) R_g^T - I||_F */
  double R[9], Rg[9], M[9], dR[9][4], a2 = 0.0;
  orc_rotation(x + 3, R);
  orc_rotation(P->q_goal, Rg);
  for (int r = 0; r < 3; ++r)
    for (int cc = 0; cc < 3; ++cc) {
      double m = -((r == cc) ? 1.0 : 0.0);
      for (int k = 0; k < 3; ++k) m += R[3 * r + k] * Rg[3 * cc + k];
      M[3 * r + cc] = m;
      a2 += m * m;
    }
  double att = sqrt(a2);
  c += P->Q_q * att;
  if (att > 0) {
    rotation_grad(x + 3, dR);
    for (int i = 0; i < 4; ++i) {
      double s = 0.0;
      for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc)
          for (int k = 0; k < 3; ++k) s += M[3 * r + cc] * dR[3 * r + k][i] * Rg[3 * cc + k];
      gx[3 + i] += P->Q_q * s / att;
    }
  }
  /* J_col at the nearest point (brute force; the lowest index among ties) */
  double best = INFINITY;
  int64_t arg = -1;
  for (int64_t i = 0; i < npts; ++i) {
    double ex = x[0] - pts[3 * i], ey = x[1] - pts[3 * i + 1], ez = x[2] - pts[3 * i + 2];
    double d = sqrt(ex * ex + ey * ey + ez * ez);
    if (d < best) { best = d; arg = i; }
  }
  c += orc_jcol(best, P);
  if (arg >= 0 && best >= P->d_min && best < P->d_max && best > 0) {
    double e[3] = {x[0] - pts[3 * arg], x[1] - pts[3 * arg + 1], x[2] - pts[3 * arg + 2]};
    add_unit(gx, e, best, -P->a_col * orc_jcol(best, P));
  }
  return c;
}

/* S^(1) of the noise-free rollout of U (T x 4) from x0, with guide (T x 3 or
 * NULL); G (T x 4) gets dS/dU.  Returns S. */
double orc_cost_grad(const double x0[10], const double* U, const double* guide, const double goal[3],
                     const double* pts, int64_t npts, const orc_params* P, double* G) {
  const int T = P->T;
  double* X = malloc(sizeof(double) * (T + 1) * 10);
  orc_rollout(x0, U, T, P->dt, P->mass, P->g, X);
  double S = 0.0, lam[10] = {0}, gs[10], gx[10];
  for (int j = T - 1; j >= 0; --j) {
    S += state_cost_grad(X + 10 * (j + 1), guide ? guide + 3 * j : NULL, goal, pts, npts, P, gs);
    for (int i = 0; i < 10; ++i) lam[i] += gs[i];
    double gu[4] = {0, 0, 0, 0};
    rk4_vjp(X + 10 * j, U + 4 * j, P->dt, P->mass, P->g, lam, gx, gu);
    for (int c = 0; c < 4; ++c) G[4 * j + c] = gu[c];
    memcpy(lam, gx, sizeof(lam));
  }
  /* J_ctrl: Q_c |u_t|^2 (t <= T-2) and Q_cd |u_t - u_{t-1}|^2 (1 <= t <= T-2) */
  for (int t = 0; t <= T - 2; ++t)
    for (int c = 0; c < 4; ++c) {
      S += P->Q_c * U[4 * t + c] * U[4 * t + c];
      G[4 * t + c] += 2 * P->Q_c * U[4 * t + c];
    }
  for (int t = 1; t <= T - 2; ++t)
    for (int c = 0; c < 4; ++c) {
      double d = U[4 * t + c] - U[4 * (t - 1) + c];
      S += P->Q_cd * d * d;
      G[4 * t + c] += 2 * P->Q_cd * d;
      G[4 * (t - 1) + c] -= 2 * P->Q_cd * d;
    }
  free(X);
  return S;
}

/* refine_steps gradient steps u <- clamp(u - refine_step dS/du, u_min, u_max)
 * on one nominal (T x 4). */
void orc_refine(const double x0[10], double* u, const double* guide, const double goal[3],
                const double* pts, int64_t npts, const orc_params* P) {
  const int T = P->T;
  double* G = malloc(sizeof(double) * T * 4);
  for (int r = 0; r < P->refine_steps; ++r) {
    orc_cost_grad(x0, u, guide, goal, pts, npts, P, G);
    for (int j = 0; j < T; ++j)
      for (int c = 0; c < 4; ++c) {
        double v = u[4 * j + c] - P->refine_step * G[4 * j + c];
        if (v < P->u_min[c]) v = P->u_min[c];
        if (v > P->u_max[c]) v = P->u_max[c];
        u[4 * j + c] = v;
      }
  }
  free(G);
}

/* ======================================================================
 * Multi-sweep accumulation (Sec. IV-A.1): a frame's sensor-frame points
 * brought into world coordinates by the capture pose, p_w = p + R(q/|q|) p_s;
 * and the projection of world points into a body frame, R(q0)^T (p_w - p0).
 * ====================================================================== */
void orc_accumulate(const double* ps, int64_t n, const double p[3], const double q[4], double* pw) {
  double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double qu[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq}, R[9];
  orc_rotation(qu, R);
  for (int64_t i = 0; i < n; ++i)
    for (int r = 0; r < 3; ++r)
      pw[3 * i + r] = p[r] + R[3 * r] * ps[3 * i] + R[3 * r + 1] * ps[3 * i + 1] + R[3 * r + 2] * ps[3 * i + 2];
}

void orc_project(const double* pw, int64_t n, const double p0[3], const double q0[4], double* pb) {
  double nq = sqrt(q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] + q0[3] * q0[3]);
  double qu[4] = {q0[0] / nq, q0[1] / nq, q0[2] / nq, q0[3] / nq}, R[9];
  orc_rotation(qu, R);
  for (int64_t i = 0; i < n; ++i) {
    double d[3] = {pw[3 * i] - p0[0], pw[3 * i + 1] - p0[1], pw[3 * i + 2] - p0[2]};
    for (int c = 0; c < 3; ++c) pb[3 * i + c] = R[c] * d[0] + R[3 + c] * d[1] + R[6 + c] * d[2];
  }
}

/* Eq. mppi_weights and Eq. mppi_update_simplified for one instance:
 * rho = min S, eta = sum exp(-(S-rho)/lam), eps_k = exp(-(S_k-rho)/lam)/eta,
 * u_nom += sum_k eps_k du^k.  dU is K x (T*4). */
void orc_mppi_update(const double* S, const double* dU, int K, int T, double lam, double* u_nom,
                     double* eps_out) {
  double rho = S[0];
  for (int k = 1; k < K; ++k) if (S[k] < rho) rho = S[k];
  double eta = 0.0;
  for (int k = 0; k < K; ++k) eta += exp(-(S[k] - rho) / lam);
  for (int k = 0; k < K; ++k) {
    double eps = exp(-(S[k] - rho) / lam) / eta;
    if (eps_out) eps_out[k] = eps;
    for (int i = 0; i < 4 * T; ++i) u_nom[i] += eps * dU[(int64_t)k * 4 * T + i];
  }
}

/* ======================================================================
 * One planning step
 * ====================================================================== */

/* Threads of the per-sample loop of orc_plan_step (OpenMP builds; 1 = serial).
 * Returns the count in use, which stays 1 when the library was built without
 * OpenMP. */
static int g_threads = 1;

int orc_set_threads(int n) {
#ifdef _OPENMP
  g_threads = n > 0 ? n : 1;
#else
  (void)n;
  g_threads = 1;
#endif
  return g_threads;
}

/* Collision set: P_f (the winning point of every non-empty cone, Sec. IV-C) or
 * every point kept by the partition.  Returns its size; pts gets 3 per point. */
int64_t orc_collision_set(const float* cloud, int64_t n, const float p0[3], const float q0[4],
                          const uint64_t* keys, const orc_params* P, double* pts) {
  int64_t m = 0;
  if (P->collision_set == 0) {
    for (int c = 0; c < P->A_f * P->E_f; ++c)
      if (keys[c] != ORC_EMPTY) {
        int64_t i = (int64_t)(keys[c] & 0xFFFFFFFFull);
        for (int a = 0; a < 3; ++a) pts[3 * m + a] = cloud[3 * i + a];
        ++m;
      }
  } else {
    orc_edges ed;
    edges_make(P, &ed);
    float R[9];
    rot_f32(q0, R);
    float rm = (float)P->r_max;
    for (int64_t i = 0; i < n; ++i) {
      float r2;
      if (fine_cell(&ed, R, p0, rm * rm, cloud + 3 * i, &r2) < 0) continue;
      for (int a = 0; a < 3; ++a) pts[3 * m + a] = cloud[3 * i + a];
      ++m;
    }
    edges_free(&ed);
  }
  return m;
}

/* Inputs: state (p0, q0 w-first, v0) and goal in binary32 as the planner
 * receives them; u_nom E x T x 4 updated in place.  Outputs: u_best (T x 4),
 * cand (E, S^(2)), best index.  Optional debug outputs (NULL to skip):
 * keys (A_f*E_f), anchors (E x 3), guides (E x T x 3), S1 (E x K, last iteration),
 * X2 (E x (T+1) x 10 Stage II states). */
int orc_plan_step(const float* cloud, int64_t n, const float p0f[3], const float q0f[4],
                  const float v0f[3], const float goalf[3], const orc_params* P,
                  double* u_nom, double* u_best, double* cand, int32_t* best_idx,
                  uint64_t* keys_out, double* anchors_out, double* guides_out, double* S1_out,
                  double* X2_out) {
  int E = P->E, K = P->K, T = P->T;
  int ncell = P->A_f * P->E_f;
  uint64_t* keys = malloc(sizeof(uint64_t) * ncell);
  orc_partition(cloud, n, p0f, q0f, P, keys);

  double p0[3], q0[4], v0[3], goal[3];
  for (int i = 0; i < 3; ++i) { p0[i] = p0f[i]; v0[i] = v0f[i]; goal[i] = goalf[i]; }
  for (int i = 0; i < 4; ++i) q0[i] = q0f[i];
  double x0[10] = {p0[0], p0[1], p0[2], q0[0], q0[1], q0[2], q0[3], v0[0], v0[1], v0[2]};

  int A_c = P->A_f / P->P_a, E_c = P->E_f / P->P_e;
  int32_t* win = malloc(sizeof(int32_t) * A_c * E_c);
  double* rwin = malloc(sizeof(double) * A_c * E_c);
  orc_coarse(keys, P, win, rwin);
  int gcell = orc_goal_fine_cell(goalf, p0f, q0f, P);
  int32_t* acell = malloc(sizeof(int32_t) * E);
  orc_anchor_cells(gcell, P, acell);

  double* guides = malloc(sizeof(double) * E * T * 3);
  double coef[18];
  for (int e = 0; e < E; ++e) {
    double d[3], pref[3];
    orc_cell_direction(P, win[acell[e]], d);
    orc_anchor(p0, q0, d, P->ell, pref);
    if (anchors_out) for (int i = 0; i < 3; ++i) anchors_out[3 * e + i] = pref[i];
    orc_guide(p0, v0, pref, P, coef, guides + (int64_t)e * T * 3);
  }
  if (guides_out) memcpy(guides_out, guides, sizeof(double) * E * T * 3);

  int64_t cap = P->collision_set == 0 ? ncell : (n > 0 ? n : 1);
  double* pts = malloc(sizeof(double) * 3 * (cap > 0 ? cap : 1));
  int64_t npts = orc_collision_set(cloud, n, p0f, q0f, keys, P, pts);

  double* dU = malloc(sizeof(double) * (int64_t)K * T * 4);
  double* S = malloc(sizeof(double) * K);
  double* X = malloc(sizeof(double) * (T + 1) * 10);
  for (int it = 0; it < P->iters; ++it)
    for (int e = 0; e < E; ++e) {
      double* un = u_nom + (int64_t)e * T * 4;
      /* the samples are independent: with OpenMP (orc_set_threads) they are
       * shared among threads; each writes only its own S[k] and dU row, and
       * the update below runs serially in sample order, so the result does
       * not depend on the thread count */
#ifdef _OPENMP
#pragma omp parallel num_threads(g_threads)
#endif
      {
        double* Uk = malloc(sizeof(double) * T * 4);
        double* Xk = malloc(sizeof(double) * (T + 1) * 10);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int k = 0; k < K; ++k) {
          for (int j = 0; j < T; ++j) {
            double delta[4];
            orc_noise(P, e, k, j, it, delta);
            for (int c = 0; c < 4; ++c) {
              double u = un[4 * j + c] + delta[c];
              if (u < P->u_min[c]) u = P->u_min[c];
              if (u > P->u_max[c]) u = P->u_max[c];
              Uk[4 * j + c] = u;
              dU[(int64_t)k * T * 4 + 4 * j + c] = u - un[4 * j + c];
            }
          }
          orc_rollout(x0, Uk, T, P->dt, P->mass, P->g, Xk);
          double terms[6];
          orc_cost_terms(Xk, Uk, guides + (int64_t)e * T * 3, goal, pts, npts, P, 1, terms, NULL);
          S[k] = terms[5];
          if (S1_out) S1_out[(int64_t)e * K + k] = S[k];
        }
        free(Uk);
        free(Xk);
      }
      orc_mppi_update(S, dU, K, T, P->lam, un, NULL);
    }

  /* optional gradient refinement of each updated nominal */
  if (P->refine_steps > 0)
    for (int e = 0; e < E; ++e)
      orc_refine(x0, u_nom + (int64_t)e * T * 4, guides + (int64_t)e * T * 3, goal, pts, npts, P);

  /* Stage II: roll out each updated nominal, score S^(2), keep the argmin. */
  int best = 0;
  for (int e = 0; e < E; ++e) {
    orc_rollout(x0, u_nom + (int64_t)e * T * 4, T, P->dt, P->mass, P->g, X);
    if (X2_out) memcpy(X2_out + (int64_t)e * (T + 1) * 10, X, sizeof(double) * (T + 1) * 10);
    double terms[6];
    orc_cost_terms(X, u_nom + (int64_t)e * T * 4, NULL, goal, pts, npts, P, 2, terms, NULL);
    cand[e] = terms[5];
    if (cand[e] < cand[best]) best = e;
  }
  *best_idx = best;
  memcpy(u_best, u_nom + (int64_t)best * T * 4, sizeof(double) * T * 4);
  if (keys_out) memcpy(keys_out, keys, sizeof(uint64_t) * ncell);

  free(keys); free(win); free(rwin); free(acell); free(guides); free(pts);
  free(dU); free(S); free(X);
  return 0;
}
