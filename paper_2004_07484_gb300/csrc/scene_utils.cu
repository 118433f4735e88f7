// Scene and camera utilities (include/pulsar_scene.h): the camera of
// Listing 1 (axis-angle rotation) to the renderer's 6D form, and back for
// gradients.  One thread per camera.
#include "pulsar_internal.cuh"
#include "pulsar_scene.h"

namespace pulsar {
namespace {

// Rodrigues' formula written as B = (1 - b t) I + a [w]_x + b w w^T with
// t = |w|^2, a = sin(s)/s, b = (1 - cos s)/s^2 (s = |w|), and the
// derivatives a' = da/dt, b' = db/dt.  Near t = 0 the Taylor series stand in
// for the quotients (relative error below 1e-15 there).
struct RodriguesCoef {
  double a, b, da, db;
};

__device__ RodriguesCoef rodrigues_coef(double t) {
  RodriguesCoef c;
  if (t < 1e-6) {
    c.a = 1.0 - t / 6.0 + t * t / 120.0;
    c.b = 0.5 - t / 24.0 + t * t / 720.0;
    c.da = -1.0 / 6.0 + t / 60.0 - t * t / 2520.0;
    c.db = -1.0 / 24.0 + t / 360.0 - t * t / 13440.0;
  } else {
    const double s = sqrt(t);
    c.a = sin(s) / s;
    c.b = (1.0 - cos(s)) / t;
    c.da = (cos(s) - c.a) / (2.0 * t);
    c.db = (c.a - 2.0 * c.b) / (2.0 * t);
  }
  return c;
}

// Entry (i, j) of [w]_x.
__device__ __forceinline__ double skew(const double w[3], int i, int j) {
  if (i == j) return 0.0;
  const int k = 3 - i - j;   // the remaining axis
  const double sgn = ((j - i + 3) % 3 == 1) ? -1.0 : 1.0;   // (0,1) -> -w2, (1,0) -> +w2, ...
  return sgn * w[k];
}

__device__ double rot_entry(const double w[3], double t, const RodriguesCoef& c, int i, int j) {
  return (i == j ? 1.0 - c.b * t : 0.0) + c.a * skew(w, i, j) + c.b * w[i] * w[j];
}

__global__ void axis_angle_fwd_kernel(const float* __restrict__ cam8, float* __restrict__ cam11, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float* in = cam8 + 8 * (size_t)k;
  float* out = cam11 + 11 * (size_t)k;
  const double w[3] = {in[3], in[4], in[5]};
  const double t = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const RodriguesCoef c = rodrigues_coef(t);
  out[0] = in[0];
  out[1] = in[1];
  out[2] = in[2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) out[3 + 3 * i + j] = (float)rot_entry(w, t, c, i, j);
  out[9] = in[6];
  out[10] = in[7];
}

__global__ void axis_angle_bwd_kernel(const float* __restrict__ cam8, const float* __restrict__ g11,
                                      float* __restrict__ g8, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float* in = cam8 + 8 * (size_t)k;
  const float* g = g11 + 11 * (size_t)k;
  float* out = g8 + 8 * (size_t)k;
  const double w[3] = {in[3], in[4], in[5]};
  const double t = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const RodriguesCoef c = rodrigues_coef(t);
  double gw[3] = {0.0, 0.0, 0.0};
  // dB_ij/dw_m = 2 w_m (-(b' t + b) d_ij + a' [w]_x,ij + b' w_i w_j)
  //              + a d[w]_x,ij/dw_m + b (d_im w_j + w_i d_jm)
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      const double gij = g[3 + 3 * i + j];
      const double common = (i == j ? -(c.db * t + c.b) : 0.0) + c.da * skew(w, i, j) + c.db * w[i] * w[j];
      for (int m = 0; m < 3; ++m) {
        double e_m[3] = {0.0, 0.0, 0.0};
        e_m[m] = 1.0;
        const double d = 2.0 * w[m] * common + c.a * skew(e_m, i, j) +
                         c.b * ((i == m ? w[j] : 0.0) + (j == m ? w[i] : 0.0));
        gw[m] += gij * d;
      }
    }
  out[0] = g[0];
  out[1] = g[1];
  out[2] = g[2];
  out[3] = (float)gw[0];
  out[4] = (float)gw[1];
  out[5] = (float)gw[2];
  out[6] = g[9];
  out[7] = g[10];
}

}  // namespace
}  // namespace pulsar

using namespace pulsar;

extern "C" pulsar_status pulsar_camera_from_axis_angle(const float* cam8, float* cam11, int n, void* stream) {
  if (n < 0 || (n > 0 && (!cam8 || !cam11))) return PULSAR_ERR_INVALID_ARG;
  if (n == 0) return PULSAR_OK;
  axis_angle_fwd_kernel<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(cam8, cam11, n);
  return cudaGetLastError() == cudaSuccess ? PULSAR_OK : PULSAR_ERR_CUDA;
}

extern "C" pulsar_status pulsar_camera_axis_angle_backward(const float* cam8, const float* g_cam11, float* g_cam8,
                                                           int n, void* stream) {
  if (n < 0 || (n > 0 && (!cam8 || !g_cam11 || !g_cam8))) return PULSAR_ERR_INVALID_ARG;
  if (n == 0) return PULSAR_OK;
  axis_angle_bwd_kernel<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(cam8, g_cam11, g_cam8, n);
  return cudaGetLastError() == cudaSuccess ? PULSAR_OK : PULSAR_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Pruning: a stable stream compaction in three launches (per-CTA counts, a
// scan of the counts, scatter), 2048 spheres per CTA.
namespace pulsar {
namespace {

constexpr int kPruneThreads = 256;
constexpr int kPrunePer = 8;
constexpr int kPruneTile = kPruneThreads * kPrunePer;

struct PruneArgs {
  int64_t n;
  int C;
  const float *pos, *rad, *opa, *feat, *bg, *activity;
  float color_tol;
  float *out_pos, *out_rad, *out_opa, *out_feat;
  int64_t* n_out;
  uint32_t* cta_cnt;
  uint32_t* cta_off;
};

__device__ __forceinline__ bool keep_sphere(const PruneArgs& a, int64_t i) {
  if (a.activity && !(a.activity[i] > 0.0f)) return false;
  if (a.color_tol < 0.0f) return true;
  // a decision: explicitly rounded float32 operations in a fixed order
  float s = 0.0f;
  for (int c = 0; c < a.C; ++c) {
    const float d = __fsub_rn(a.feat[i * a.C + c], a.bg[c]);
    s = __fadd_rn(s, __fmul_rn(d, d));
  }
  return __fsqrt_rn(s) > a.color_tol;
}

__global__ void __launch_bounds__(kPruneThreads) prune_count_kernel(const PruneArgs a) {
  __shared__ uint32_t warp_tot[33];
  uint32_t cnt = 0;
  const int64_t i0 = (int64_t)blockIdx.x * kPruneTile + (int64_t)threadIdx.x * kPrunePer;
  for (int k = 0; k < kPrunePer; ++k)
    if (i0 + k < a.n && keep_sphere(a, i0 + k)) ++cnt;
  uint32_t tot;
  block_exclusive_scan<kPruneThreads>(cnt, warp_tot, tot);
  if (threadIdx.x == 0) a.cta_cnt[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) prune_scan_kernel(const PruneArgs a, int n_ctas) {
  __shared__ uint32_t warp_tot[33];
  uint64_t carry = 0;
  for (int j0 = 0; j0 < n_ctas; j0 += 1024) {
    const int j = j0 + (int)threadIdx.x;
    const uint32_t x = j < n_ctas ? a.cta_cnt[j] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan<1024>(x, warp_tot, tot);
    if (j < n_ctas) a.cta_off[j] = (uint32_t)(carry + ex);
    carry += tot;
  }
  if (threadIdx.x == 0) *a.n_out = (int64_t)carry;
}

__global__ void __launch_bounds__(kPruneThreads) prune_scatter_kernel(const PruneArgs a) {
  __shared__ uint32_t warp_tot[33];
  const int64_t i0 = (int64_t)blockIdx.x * kPruneTile + (int64_t)threadIdx.x * kPrunePer;
  uint32_t keep = 0u, cnt = 0u;
  for (int k = 0; k < kPrunePer; ++k)
    if (i0 + k < a.n && keep_sphere(a, i0 + k)) {
      keep |= 1u << k;
      ++cnt;
    }
  uint32_t tot;
  int64_t pos = (int64_t)a.cta_off[blockIdx.x] + block_exclusive_scan<kPruneThreads>(cnt, warp_tot, tot);
  for (int k = 0; k < kPrunePer; ++k) {
    if (!((keep >> k) & 1u)) continue;
    const int64_t i = i0 + k;
    for (int d = 0; d < 3; ++d) a.out_pos[3 * pos + d] = a.pos[3 * i + d];
    a.out_rad[pos] = a.rad[i];
    a.out_opa[pos] = a.opa[i];
    for (int c = 0; c < a.C; ++c) a.out_feat[pos * a.C + c] = a.feat[i * a.C + c];
    ++pos;
  }
}

// Subdivision: one thread per child.
__global__ void subdivide_kernel(int64_t n, int C, const float* __restrict__ pos, const float* __restrict__ rad,
                                 const float* __restrict__ opa, const float* __restrict__ feat, float offset_scale,
                                 float radius_scale, float* __restrict__ out_pos, float* __restrict__ out_rad,
                                 float* __restrict__ out_opa, float* __restrict__ out_feat) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 12 * n) return;
  const int64_t i = j / 12;
  const int k = (int)(j - i * 12);
  // nearest-neighbour directions of the face-centred cubic lattice: the zero
  // in axis k / 4, signs from the low two bits of k
  const int zero_axis = k >> 2;
  const float s0 = (k & 1) ? -1.0f : 1.0f, s1 = (k & 2) ? -1.0f : 1.0f;
  float u[3];
  const int a0 = zero_axis == 0 ? 1 : 0, a1 = zero_axis == 2 ? 1 : 2;
  u[zero_axis] = 0.0f;
  u[a0] = s0 * 0.70710678118654752f;
  u[a1] = s1 * 0.70710678118654752f;
  const float r = rad[i];
  const float off = offset_scale * r;
  for (int d = 0; d < 3; ++d) out_pos[3 * j + d] = fmaf(off, u[d], pos[3 * i + d]);
  out_rad[j] = radius_scale * r;
  out_opa[j] = opa[i];
  for (int c = 0; c < C; ++c) out_feat[j * C + c] = feat[i * C + c];
}

}  // namespace
}  // namespace pulsar

extern "C" size_t pulsar_prune_scratch_bytes(int64_t n) {
  if (n < 0) return 0;
  const int64_t ctas = (n + pulsar::kPruneTile - 1) / pulsar::kPruneTile;
  return (size_t)(2 * ctas + 4) * sizeof(uint32_t);
}

extern "C" pulsar_status pulsar_prune(int64_t n, int C, const float* pos, const float* rad, const float* opa,
                                      const float* feat, const float* bg, const float* activity, float color_tol,
                                      float* out_pos, float* out_rad, float* out_opa, float* out_feat,
                                      int64_t* n_out, void* scratch, size_t scratch_bytes, void* stream) {
  if (n < 0 || C < 1 || !n_out) return PULSAR_ERR_INVALID_ARG;
  if (n > 0 && (!pos || !rad || !opa || !feat || !bg || !out_pos || !out_rad || !out_opa || !out_feat || !scratch))
    return PULSAR_ERR_INVALID_ARG;
  if (scratch_bytes < pulsar_prune_scratch_bytes(n)) return PULSAR_ERR_INVALID_ARG;
  if (n > ((int64_t)1 << 31) * pulsar::kPruneTile / 2) return PULSAR_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n == 0) return cudaMemsetAsync(n_out, 0, sizeof(int64_t), st) == cudaSuccess ? PULSAR_OK : PULSAR_ERR_CUDA;
  const int ctas = (int)((n + pulsar::kPruneTile - 1) / pulsar::kPruneTile);
  pulsar::PruneArgs a{n, C, pos, rad, opa, feat, bg, activity, color_tol, out_pos, out_rad, out_opa, out_feat,
                      n_out, static_cast<uint32_t*>(scratch), static_cast<uint32_t*>(scratch) + ctas};
  pulsar::prune_count_kernel<<<ctas, pulsar::kPruneThreads, 0, st>>>(a);
  pulsar::prune_scan_kernel<<<1, 1024, 0, st>>>(a, ctas);
  pulsar::prune_scatter_kernel<<<ctas, pulsar::kPruneThreads, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? PULSAR_OK : PULSAR_ERR_CUDA;
}

extern "C" pulsar_status pulsar_subdivide(int64_t n, int C, const float* pos, const float* rad, const float* opa,
                                          const float* feat, float offset_scale, float radius_scale, float* out_pos,
                                          float* out_rad, float* out_opa, float* out_feat, void* stream) {
  if (n < 0 || C < 1) return PULSAR_ERR_INVALID_ARG;
  if (n > 0 && (!pos || !rad || !opa || !feat || !out_pos || !out_rad || !out_opa || !out_feat))
    return PULSAR_ERR_INVALID_ARG;
  if (n == 0) return PULSAR_OK;
  const int64_t m = 12 * n;
  const int64_t blocks = (m + 255) / 256;
  if (blocks > 0x7fffffff) return PULSAR_ERR_UNSUPPORTED;
  pulsar::subdivide_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, C, pos, rad, opa, feat, offset_scale, radius_scale, out_pos, out_rad, out_opa, out_feat);
  return cudaGetLastError() == cudaSuccess ? PULSAR_OK : PULSAR_ERR_CUDA;
}
