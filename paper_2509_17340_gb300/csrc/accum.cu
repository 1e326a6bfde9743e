// Multi-sweep accumulation (Sec. IV-A.1): the most recent LiDAR frames, each
// taken from its own pose, brought into common coordinates with the
// transforms of state estimation.  A ring of F frame slots of N points each,
// in world coordinates: a push transforms a frame's sensor-frame points by the
// capture pose, p_w = p + R(q) p_s, into the oldest slot and pads the slot's
// tail with NaN.  The ring is a cloud for aero_plan_step as it stands (the
// partition drops non-finite points); the gather compacts the live frames,
// oldest first, in world coordinates or projected into a body frame
// R(q0)^T (p_w - p0).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/aero_mppi.h"
#include "internal.h"

using aero::dev_free;
using aero::dev_malloc;

struct aero_accum {
  int F = 0;                  // frame slots
  int64_t N = 0;              // points per slot
  float* ring = nullptr;      // F x N x 3, world coordinates, NaN padding
  std::vector<int64_t> count; // points of each slot
  int head = 0;               // next slot to write
  int live = 0;               // frames held (<= F)
};

namespace {

constexpr int kAccumMaxFrames = 64;
constexpr int kThreads = 256;

struct Pose32 {
  float R[9];  // row-major
  float t[3];
};

// R(q) of the normalised quaternion in binary32 (nine products, then the sums).
Pose32 pose_of(const float p[3], const float q[4]) {
  const double n = std::sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] +
                             (double)q[3] * q[3]);
  const float w = (float)(q[0] / n), x = (float)(q[1] / n), y = (float)(q[2] / n), z = (float)(q[3] / n);
  const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  const float wx = w * x, wy = w * y, wz = w * z;
  Pose32 P;
  P.R[0] = 1.0f - 2.0f * (yy + zz);
  P.R[1] = 2.0f * (xy - wz);
  P.R[2] = 2.0f * (xz + wy);
  P.R[3] = 2.0f * (xy + wz);
  P.R[4] = 1.0f - 2.0f * (xx + zz);
  P.R[5] = 2.0f * (yz - wx);
  P.R[6] = 2.0f * (xz - wy);
  P.R[7] = 2.0f * (yz + wx);
  P.R[8] = 1.0f - 2.0f * (xx + yy);
  for (int i = 0; i < 3; ++i) P.t[i] = p[i];
  return P;
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

// p_w = t + R p_s for the n points of src; NaN for the slot's remaining N - n.
__global__ void __launch_bounds__(kThreads) k_accum_push(const float* __restrict__ src, int64_t n,
                                                         int64_t N, float* __restrict__ dst,
                                                         Pose32 P) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    float wx = NAN, wy = NAN, wz = NAN;
    if (i < n) {
      const float x = __ldg(src + 3 * i), y = __ldg(src + 3 * i + 1), z = __ldg(src + 3 * i + 2);
      wx = __fadd_rn(P.t[0], __fadd_rn(__fadd_rn(__fmul_rn(P.R[0], x), __fmul_rn(P.R[1], y)), __fmul_rn(P.R[2], z)));
      wy = __fadd_rn(P.t[1], __fadd_rn(__fadd_rn(__fmul_rn(P.R[3], x), __fmul_rn(P.R[4], y)), __fmul_rn(P.R[5], z)));
      wz = __fadd_rn(P.t[2], __fadd_rn(__fadd_rn(__fmul_rn(P.R[6], x), __fmul_rn(P.R[7], y)), __fmul_rn(P.R[8], z)));
    }
    dst[3 * i] = wx;
    dst[3 * i + 1] = wy;
    dst[3 * i + 2] = wz;
  }
}

struct GatherArgs {
  int64_t pre[kAccumMaxFrames + 1];  // exclusive prefix of the live frames' counts, oldest first
  int slot[kAccumMaxFrames];         // their ring slots
  int nframes;
  int body;                          // 1: project into the body frame (R0, p0)
  Pose32 P0;
};

// The live frames' points, oldest frame first, into dst (world or body frame).
__global__ void __launch_bounds__(kThreads) k_accum_gather(const float* __restrict__ ring, int64_t N,
                                                           float* __restrict__ dst, GatherArgs a) {
  const int64_t total = a.pre[a.nframes];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    int lo = 0, hi = a.nframes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.pre[mid] <= i) lo = mid; else hi = mid - 1;
    }
    if (!AERO_CHECK(a.slot[lo] >= 0 && i - a.pre[lo] < N, ::aero::kChkAccum)) continue;
    const int64_t src = (int64_t)a.slot[lo] * N + (i - a.pre[lo]);
    float x = __ldg(ring + 3 * src), y = __ldg(ring + 3 * src + 1), z = __ldg(ring + 3 * src + 2);
    if (a.body) {
      const float* R = a.P0.R;
      const float dx = __fsub_rn(x, a.P0.t[0]), dy = __fsub_rn(y, a.P0.t[1]), dz = __fsub_rn(z, a.P0.t[2]);
      // R^T (p - p0), each dot product left to right
      x = __fadd_rn(__fadd_rn(__fmul_rn(R[0], dx), __fmul_rn(R[3], dy)), __fmul_rn(R[6], dz));
      y = __fadd_rn(__fadd_rn(__fmul_rn(R[1], dx), __fmul_rn(R[4], dy)), __fmul_rn(R[7], dz));
      z = __fadd_rn(__fadd_rn(__fmul_rn(R[2], dx), __fmul_rn(R[5], dy)), __fmul_rn(R[8], dz));
    }
    dst[3 * i] = x;
    dst[3 * i + 1] = y;
    dst[3 * i + 2] = z;
  }
}

// Warm-start shift of the receding horizon: u[e][j] = u[e][j + shift] for
// j < T - shift, then the last control repeated.  One thread per (e, j, c),
// reading from a copy so that the shift is in place.
__global__ void __launch_bounds__(kThreads) k_shift(float* __restrict__ u, const float* __restrict__ src,
                                                    int E, int T, int shift) {
  const int64_t n = (int64_t)E * T * 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int c = (int)(i & 3);
    const int64_t ej = i >> 2;
    const int e = (int)(ej / T), j = (int)(ej % T);
    const int s = min(j + shift, T - 1);
    u[i] = __ldg(src + ((int64_t)e * T + s) * 4 + c);
  }
}

int blocks_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  const int cap = 16 * aero::device_sms();
  return (int)(b < cap ? b : cap);
}

int fail(cudaError_t e) { return e == cudaSuccess ? AERO_OK : AERO_ERR_CUDA; }

}  // namespace

namespace aero {
cudaError_t check_word_accum(int* out, bool clear) {
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

extern "C" {

int aero_accum_create(int32_t frames, int64_t points_per_frame, aero_accum_t** out) {
  if (!out || frames < 1 || frames > kAccumMaxFrames || points_per_frame < 1 ||
      points_per_frame > ((int64_t)1 << 28))
    return AERO_ERR_INVALID_ARG;
  *out = nullptr;
  aero_accum* a = new (std::nothrow) aero_accum();
  if (!a) return AERO_ERR_ALLOC;
  a->F = frames;
  a->N = points_per_frame;
  a->count.assign(frames, 0);
  const size_t bytes = sizeof(float) * 3 * (size_t)frames * (size_t)points_per_frame;
  cudaError_t e = dev_malloc((void**)&a->ring, bytes);
  if (e == cudaSuccess) e = cudaMemset(a->ring, 0xFF, bytes);  // all-ones words are NaN
  if (e != cudaSuccess) {
    cudaGetLastError();
    dev_free(a->ring);
    delete a;
    return e == cudaErrorMemoryAllocation ? AERO_ERR_ALLOC : AERO_ERR_CUDA;
  }
  *out = a;
  return AERO_OK;
}

int aero_accum_push(aero_accum_t* a, const float* pts, int64_t n, const float pose_p[3],
                    const float pose_q[4], void* stream) {
  if (!a || !pose_p || !pose_q || n < 0 || n > a->N || (n > 0 && !pts)) return AERO_ERR_INVALID_ARG;
  const double qn = (double)pose_q[0] * pose_q[0] + (double)pose_q[1] * pose_q[1] +
                    (double)pose_q[2] * pose_q[2] + (double)pose_q[3] * pose_q[3];
  if (!(qn > 0.0) || !std::isfinite(qn)) return AERO_ERR_INVALID_ARG;
  if (n > 0 && !is_device_ptr(pts)) return AERO_ERR_NOT_DEVICE_PTR;
  const int slot = a->head;
  k_accum_push<<<blocks_for(a->N), kThreads, 0, (cudaStream_t)stream>>>(
      pts, n, a->N, a->ring + (size_t)3 * slot * a->N, pose_of(pose_p, pose_q));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return AERO_ERR_CUDA;
  a->count[slot] = n;
  a->head = (a->head + 1) % a->F;
  if (a->live < a->F) ++a->live;
  return AERO_OK;
}

int aero_accum_view(aero_accum_t* a, const float** cloud, int64_t* n_points, int64_t* n_valid) {
  if (!a || !cloud || !n_points) return AERO_ERR_INVALID_ARG;
  *cloud = a->ring;
  *n_points = (int64_t)a->F * a->N;
  if (n_valid) {
    int64_t v = 0;
    for (int k = 0; k < a->F; ++k) v += a->count[k];
    *n_valid = v;
  }
  return AERO_OK;
}

int aero_accum_gather(aero_accum_t* a, const float* p0, const float* q0, float* dst,
                      int64_t dst_capacity, int64_t* n_out, void* stream) {
  if (!a || !n_out || (p0 == nullptr) != (q0 == nullptr)) return AERO_ERR_INVALID_ARG;
  GatherArgs g{};
  g.nframes = a->live;
  g.pre[0] = 0;
  for (int k = 0; k < a->live; ++k) {
    const int slot = (a->head - a->live + k + a->F) % a->F;  // oldest first
    g.slot[k] = slot;
    g.pre[k + 1] = g.pre[k] + a->count[slot];
  }
  const int64_t total = g.pre[a->live];
  *n_out = total;
  if (total == 0) return AERO_OK;
  if (!dst || dst_capacity < total) return AERO_ERR_INVALID_ARG;
  if (!is_device_ptr(dst)) return AERO_ERR_NOT_DEVICE_PTR;
  g.body = p0 != nullptr;
  if (g.body) {
    const double qn = (double)q0[0] * q0[0] + (double)q0[1] * q0[1] + (double)q0[2] * q0[2] +
                      (double)q0[3] * q0[3];
    if (!(qn > 0.0) || !std::isfinite(qn)) return AERO_ERR_INVALID_ARG;
    g.P0 = pose_of(p0, q0);
  }
  k_accum_gather<<<blocks_for(total), kThreads, 0, (cudaStream_t)stream>>>(a->ring, a->N, dst, g);
  return fail(cudaGetLastError());
}

int aero_accum_reset(aero_accum_t* a, void* stream) {
  if (!a) return AERO_ERR_INVALID_ARG;
  const size_t bytes = sizeof(float) * 3 * (size_t)a->F * (size_t)a->N;
  const cudaError_t e = cudaMemsetAsync(a->ring, 0xFF, bytes, (cudaStream_t)stream);
  if (e != cudaSuccess) return AERO_ERR_CUDA;
  for (auto& c : a->count) c = 0;
  a->head = 0;
  a->live = 0;
  return AERO_OK;
}

int aero_shift_nominal(float* u_nom, int32_t E, int32_t T, int32_t shift, float* scratch,
                       void* stream) {
  if (!u_nom || !scratch || E < 1 || T < 1 || shift < 0) return AERO_ERR_INVALID_ARG;
  if (!is_device_ptr(u_nom) || !is_device_ptr(scratch)) return AERO_ERR_NOT_DEVICE_PTR;
  if (shift == 0) return AERO_OK;
  const size_t bytes = sizeof(float) * 4 * (size_t)E * T;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(scratch, u_nom, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return AERO_ERR_CUDA;
  k_shift<<<blocks_for((int64_t)E * T * 4), kThreads, 0, s>>>(u_nom, scratch, E, T, shift);
  return fail(cudaGetLastError());
}

int aero_accum_destroy(aero_accum_t* a) {
  if (!a) return AERO_OK;
  cudaDeviceSynchronize();
  dev_free(a->ring);
  delete a;
  return AERO_OK;
}

}  // extern "C"
