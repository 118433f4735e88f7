// Scene setup, Step 0 projection (App. B, "Step 0: Enclosing Rectangle
// Calculation"), and the per-sphere gradient finalisation with the
// camera-gradient reduction (App. B, "The Backward Pass").
#include "pulsar_internal.cuh"

namespace pulsar {

namespace {

template <int N>
struct SetupPack {
  int n;
  int full;   // 1: derive camera data and reset counters; 0: refresh pointers only
  int64_t n_spheres;
  SceneDev s[N];
};

// Gram-Schmidt of the 6D rotation in double, for the value path.
__device__ __forceinline__ void rows_from_rot6_f64(const float* a, double* B) {
  const double a0 = a[0], a1 = a[1], a2 = a[2], a3 = a[3], a4 = a[4], a5 = a[5];
  const double n1 = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
  const double b1x = a0 / n1, b1y = a1 / n1, b1z = a2 / n1;
  const double dt = b1x * a3 + b1y * a4 + b1z * a5;
  const double ux = a3 - dt * b1x, uy = a4 - dt * b1y, uz = a5 - dt * b1z;
  const double n2 = sqrt(ux * ux + uy * uy + uz * uz);
  const double b2x = ux / n2, b2y = uy / n2, b2z = uz / n2;
  B[0] = b1x; B[1] = b1y; B[2] = b1z;
  B[3] = b2x; B[4] = b2y; B[5] = b2z;
  B[6] = b1y * b2z - b1z * b2y;
  B[7] = b1z * b2x - b1x * b2z;
  B[8] = b1x * b2y - b1y * b2x;
}

template <int N>
__global__ void setup_kernel(WsView v, const SetupPack<N> pk) {
  pdl_wait();
  pdl_trigger();
  const int i = threadIdx.x;
  if (i < pk.n) {
    SceneDev d = pk.s[i];
    if (pk.full) {
      rows_from_rot6(d.cam + 3, d.rows);
      const bool ortho = (d.flags & PULSAR_FLAG_ORTHOGRAPHIC) != 0;
      d.kappa = pixel_pitch(d.cam, d.width, ortho);
      rows_from_rot6_f64(d.cam + 3, d.rows64);
      for (int k = 0; k < 9; ++k) {
        d.rows_hi[k] = (float)d.rows64[k];
        d.rows_lo[k] = (float)(d.rows64[k] - (double)d.rows_hi[k]);
      }
      d.kappa64 = ortho ? (double)d.cam[10] / (double)d.width
                        : (double)d.cam[10] / ((double)d.width * (double)d.cam[9]);
      d.kappa_hi = (float)d.kappa64;
      d.kappa_lo = (float)(d.kappa64 - (double)d.kappa_hi);
      d.omax_bits = 0u;
    } else {
      const SceneDev& o = v.scenes[i];
      for (int k = 0; k < 9; ++k) {
        d.rows[k] = o.rows[k];
        d.rows64[k] = o.rows64[k];
        d.rows_hi[k] = o.rows_hi[k];
        d.rows_lo[k] = o.rows_lo[k];
      }
      d.kappa = o.kappa;
      d.kappa64 = o.kappa64;
      d.kappa_hi = o.kappa_hi;
      d.kappa_lo = o.kappa_lo;
      d.omax_bits = o.omax_bits;
    }
    v.scenes[i] = d;
  }
  if (i < pk.n && pk.full) v.cam_done[i] = 0;
  if (i == 0 && pk.full) {
    v.hdr->n_scenes = pk.n;
    v.hdr->n_sort = (int32_t)pk.n_spheres;
    v.hdr->overflow = 0;
    v.hdr->timeout = 0;
    v.hdr->count_done = 0;
    v.hdr->work_next = 0;
  }
}

// One thread per sphere: draw record, sort key and value, and the scene-wide
// maximum of |o| (used by the exact early-termination bound).
__global__ void __launch_bounds__(kThreads) project_kernel(WsView v) {
  pdl_wait();
  pdl_trigger();
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool live = i < v.n_spheres;
  const int s = live ? scene_of_sphere(v.scenes, v.n_scenes, i) : 0;
  uint32_t om = 0u;
  if (live) {
    const SceneDev& S = v.scenes[s];
    const int64_t li = i - S.sphere_begin;
    const float* p = S.pos + 3 * li;
    const float r = S.rad[li];
    const float o = S.opa[li];
    Projected pr = project_sphere(S.rows, S.cam, S.kappa, p[0], p[1], p[2], r, S.width, S.height,
                                  S.znear, S.zfar, !(S.flags & PULSAR_FLAG_NO_MIN_SIZE),
                                  (S.flags & PULSAR_FLAG_ORTHOGRAPHIC) != 0);
    v.rec0[i] = make_float4(pr.cx, pr.cy, pr.cz, pr.R2);
    v.rec1[i] = make_float4(pr.key, o, __uint_as_float(pack_range(pr.x0, pr.x1)),
                            __uint_as_float(pack_range(pr.y0, pr.y1)));
    v.key[0][i] = pr.visible ? __float_as_uint(pr.key) - v.key_base : v.key_culled;
    v.val[0][i] = (uint32_t)i;
    // value path: the centre to about 2^-46 relative (float-float), kept as
    // the float32 decision centre plus a float correction; the radius as
    // used by the value path
    FF c[3];
    {
      const FF d0 = two_sum(p[0], -S.cam[0]), d1 = two_sum(p[1], -S.cam[1]), d2 = two_sum(p[2], -S.cam[2]);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const FF b0 = {S.rows_hi[3 * k], S.rows_lo[3 * k]};
        const FF b1 = {S.rows_hi[3 * k + 1], S.rows_lo[3 * k + 1]};
        const FF b2 = {S.rows_hi[3 * k + 2], S.rows_lo[3 * k + 2]};
        c[k] = ff_add(ff_add(ff_mul(b0, d0), ff_mul(b1, d1)), ff_mul(b2, d2));
      }
    }
    float Rv = r;
    if (pr.R != r && (S.flags & PULSAR_FLAG_ORTHOGRAPHIC)) {   // R = 0.75 kappa
      const FF q = two_prod(S.kappa_hi, 0.75f);
      Rv = __fadd_rn(q.hi, __fmaf_rn(0.75f, S.kappa_lo, q.lo));
    } else if (pr.R != r) {   // R = 0.75 |c| kappa
      FF n2 = two_prod(c[0].hi, c[0].hi);
      n2.lo = __fmaf_rn(2.0f * c[0].hi, c[0].lo, n2.lo);
#pragma unroll
      for (int k = 1; k < 3; ++k) {
        FF t = two_prod(c[k].hi, c[k].hi);
        t.lo = __fmaf_rn(2.0f * c[k].hi, c[k].lo, t.lo);
        n2 = ff_add(n2, t);
      }
      const float sh = __fsqrt_rn(n2.hi);
      const float sl = __fdiv_rn(__fadd_rn(__fmaf_rn(-sh, sh, n2.hi), n2.lo), __fmul_rn(2.0f, sh));
      const FF rk = ff_mul(FF{sh, sl}, FF{S.kappa_hi, S.kappa_lo});
      const FF q = two_prod(rk.hi, 0.75f);
      Rv = __fadd_rn(q.hi, __fmaf_rn(0.75f, rk.lo, q.lo));
    }
    v.rec2[i] = make_float4(__fadd_rn(__fsub_rn(c[0].hi, pr.cx), c[0].lo),
                            __fadd_rn(__fsub_rn(c[1].hi, pr.cy), c[1].lo),
                            __fadd_rn(__fsub_rn(c[2].hi, pr.cz), c[2].lo), Rv);
    if (pr.visible) om = __float_as_uint(fabsf(o));
  }
  // warp-aggregated maxima per scene (non-negative floats order as integers)
  const unsigned peers = __match_any_sync(0xffffffffu, live ? s : -1);
  const uint32_t om_w = __reduce_max_sync(peers, om);
  // (a read first: once the scene's maximum is known, most warps need no atomic)
  if (live && (threadIdx.x & 31) == __ffs(peers) - 1 && om_w &&
      om_w > *reinterpret_cast<volatile uint32_t*>(&v.scenes[s].omax_bits))
    atomicMax(&v.scenes[s].omax_bits, om_w);
}

// One thread per sphere of the batch: clears the per-sphere accumulators the
// backward pass adds into (dL/dc, dL/dR in the workspace; dL/do and dL/df in
// the caller's buffers).
__global__ void __launch_bounds__(kThreads) zero_grads_kernel(WsView v, uint32_t mask) {
  pdl_wait();
  pdl_trigger();
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= v.n_spheres) return;
  v.gacc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int s = scene_of_sphere(v.scenes, v.n_scenes, i);
  const SceneDev& S = v.scenes[s];
  if (S.flags & PULSAR_FLAG_PAPER_GRADIENTS) {   // sums in the workspace; finalize writes the outputs
    v.pg_cnt[i] = 0;
    if (mask & PULSAR_GRAD_OPA) v.pg_opa[i] = 0.0f;
    if (mask & PULSAR_GRAD_FEAT)
      for (int c = 0; c < S.n_channels; ++c) v.pg_feat[i * S.n_channels + c] = 0.0f;
    return;
  }
  if (S.flags & PULSAR_FLAG_ACCUMULATE) return;   // the caller's buffers are added into
  const int64_t li = i - S.sphere_begin;
  if (mask & PULSAR_GRAD_OPA) S.g_opa[li] = 0.0f;
  if (mask & PULSAR_GRAD_FEAT) {
    const int C = S.n_channels;
    float* f = S.g_feat + li * C;
    if ((C & 3) == 0 && (reinterpret_cast<uintptr_t>(f) & 15) == 0) {
      for (int c = 0; c < C; c += 4) *reinterpret_cast<float4*>(f + c) = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      for (int c = 0; c < C; ++c) f[c] = 0.0f;
    }
  }
}

// One thread per sphere: dL/dc and dL/dR from the pixel pass become dL/dp,
// dL/dr and the sphere's camera contribution (App. B: camera gradients are
// gathered per sphere and reduced device-wide afterwards).
__global__ void __launch_bounds__(kFinalizeThreads) finalize_kernel(WsView v, uint32_t mask) {
  pdl_wait();
  pdl_trigger();
  const int blk = blockIdx.x;
  int s = 0;
  for (int k = 1; k < v.n_scenes; ++k)
    if (v.scenes[k].fin_block_begin <= blk) s = k;
  const SceneDev& S = v.scenes[s];
  const int64_t li = (int64_t)(blk - S.fin_block_begin) * kFinalizeThreads + threadIdx.x;
  float cam_part[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) cam_part[k] = 0.0f;
  if (li < S.n_spheres) {
    const int64_t i = S.sphere_begin + li;
    const float4 g = v.gacc[i];
    const float* p = S.pos + 3 * li;
    const float r = S.rad[li];
    // the centre and radius exactly as the projection formed them (no rectangle needed)
    Projected pr;
    sphere_centre_radius(S.rows, S.cam, S.kappa, p[0], p[1], p[2], r, !(S.flags & PULSAR_FLAG_NO_MIN_SIZE),
                         (S.flags & PULSAR_FLAG_ORTHOGRAPHIC) != 0, pr);
    float gc0 = g.x, gc1 = g.y, gc2 = g.z;
    float gk = 0.0f, grad_r = 0.0f;
    const bool clamped = pr.R != r;
    if (clamped && (S.flags & PULSAR_FLAG_ORTHOGRAPHIC)) {
      gk = g.w * 0.75f;   // R = 0.75 kappa
    } else if (clamped) {
      // R = 0.75 |c| kappa
      float cn = sqrtf(pr.cx * pr.cx + pr.cy * pr.cy + pr.cz * pr.cz);
      float f = g.w * 0.75f * S.kappa / cn;
      gc0 += f * pr.cx;
      gc1 += f * pr.cy;
      gc2 += f * pr.cz;
      gk = g.w * 0.75f * cn;
    } else {
      grad_r = g.w;
    }
    const float* B = S.rows;
    float gp0 = B[0] * gc0 + B[3] * gc1 + B[6] * gc2;
    float gp1 = B[1] * gc0 + B[4] * gc1 + B[7] * gc2;
    float gp2 = B[2] * gc0 + B[5] * gc1 + B[8] * gc2;
    const bool acc = (S.flags & PULSAR_FLAG_ACCUMULATE) != 0;
    // paper gradients: averages over the pixels that track the sphere, and
    // positions and radii only above 3 pixels projected radius (the camera
    // terms below keep the plain per-sphere sums)
    float geo_scale = 1.0f;
    if (S.flags & PULSAR_FLAG_PAPER_GRADIENTS) {
      const int np = v.pg_cnt[i];
      const float inv = 1.0f / (float)(np > 1 ? np : 1);
      const float px_size = (S.flags & PULSAR_FLAG_ORTHOGRAPHIC) ? S.kappa : __fmul_rn(pr.cz, S.kappa);
      geo_scale = __fdiv_rn(pr.R, px_size) > 3.0f ? inv : 0.0f;
      if (mask & PULSAR_GRAD_OPA) {
        const float go = v.pg_opa[i] * inv;
        if (acc)
          atomicAdd(S.g_opa + li, go);
        else
          S.g_opa[li] = go;
      }
      if (mask & PULSAR_GRAD_FEAT) {
        const int C = S.n_channels;
        for (int c = 0; c < C; ++c) {
          const float gf = v.pg_feat[i * C + c] * inv;
          if (acc)
            atomicAdd(S.g_feat + li * C + c, gf);
          else
            S.g_feat[li * C + c] = gf;
        }
      }
    }
    if (mask & PULSAR_GRAD_POS) {
      float* gp = S.g_pos + 3 * li;
      if (acc) {
        atomicAdd(gp, geo_scale * gp0);
        atomicAdd(gp + 1, geo_scale * gp1);
        atomicAdd(gp + 2, geo_scale * gp2);
      } else {
        gp[0] = geo_scale * gp0;
        gp[1] = geo_scale * gp1;
        gp[2] = geo_scale * gp2;
      }
    }
    if (mask & PULSAR_GRAD_RAD) {
      if (acc)
        atomicAdd(S.g_rad + li, geo_scale * grad_r);
      else
        S.g_rad[li] = geo_scale * grad_r;
    }
    if (mask & PULSAR_GRAD_CAM) {
      float d0 = p[0] - S.cam[0], d1 = p[1] - S.cam[1], d2 = p[2] - S.cam[2];
      cam_part[0] = gc0 * d0; cam_part[1] = gc0 * d1; cam_part[2] = gc0 * d2;
      cam_part[3] = gc1 * d0; cam_part[4] = gc1 * d1; cam_part[5] = gc1 * d2;
      cam_part[6] = gc2 * d0; cam_part[7] = gc2 * d1; cam_part[8] = gc2 * d2;
      cam_part[9] = -gp0; cam_part[10] = -gp1; cam_part[11] = -gp2;
      cam_part[12] = gk;
    }
  }
  if (mask & PULSAR_GRAD_CAM) {
    // the 13 sums at once: warp sums into shared memory, one barrier, then
    // thread k adds up the warps' k-th sums
    __shared__ float part[kFinalizeThreads / 32][13];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 13; ++k) {
      const float t = warp_sum(cam_part[k]);
      if (lane == 0) part[warp][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < 13) {
      float t = 0.0f;
      for (int w = 0; w < kFinalizeThreads / 32; ++w) t += part[w][threadIdx.x];
      v.fin_part[(size_t)blk * kCamPartials + threadIdx.x] = t;
    }
  }
}

__device__ __forceinline__ void cross3(const float* a, const float* b, float* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ float dot3(const float* a, const float* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

constexpr int kRedParts = 64;   // CTAs per scene in the first reduction stage
constexpr int kRedValues = 13 + 32;

// Second stage, run by the scene's last first-stage CTA to finish: sums the
// first stage's partials in a fixed order, then chains the camera sums through
// the pixel pitch kappa = s / (W f) and the Gram-Schmidt map of the 6D rotation.
__device__ __forceinline__ void camera_finish(const WsView& v, uint32_t mask, int scene) {
  __shared__ float tot[kRedValues];
  __shared__ float gcam[11];
  const SceneDev& S = v.scenes[scene];
  const int C = S.n_channels;
  if (threadIdx.x < kRedValues) {
    float x = 0.0f;
    for (int p = 0; p < kRedParts; ++p)
      x += __ldcg(v.red_part + ((size_t)scene * kRedParts + p) * kRedValues + threadIdx.x);
    tot[threadIdx.x] = x;
    if ((mask & PULSAR_GRAD_BG) && threadIdx.x >= 13 && threadIdx.x < 13 + C) {
      if (S.flags & PULSAR_FLAG_ACCUMULATE)
        atomicAdd(S.g_bg + threadIdx.x - 13, x);
      else
        S.g_bg[threadIdx.x - 13] = x;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && (mask & PULSAR_GRAD_CAM)) {
    const float* a = S.cam + 3;
    float a1[3] = {a[0], a[1], a[2]}, a2[3] = {a[3], a[4], a[5]};
    float n1 = sqrtf(dot3(a1, a1));
    float b1[3] = {a1[0] / n1, a1[1] / n1, a1[2] / n1};
    float dt = dot3(b1, a2);
    float u[3] = {a2[0] - dt * b1[0], a2[1] - dt * b1[1], a2[2] - dt * b1[2]};
    float n2 = sqrtf(dot3(u, u));
    float b2[3] = {u[0] / n2, u[1] / n2, u[2] / n2};
    float gB1[3] = {tot[0], tot[1], tot[2]};
    float gB2[3] = {tot[3], tot[4], tot[5]};
    float gB3[3] = {tot[6], tot[7], tot[8]};
    // b3 = b1 x b2
    float gb1[3], gb2[3], t3[3];
    cross3(b2, gB3, t3);
    for (int k = 0; k < 3; ++k) gb1[k] = gB1[k] + t3[k];
    cross3(gB3, b1, t3);
    for (int k = 0; k < 3; ++k) gb2[k] = gB2[k] + t3[k];
    // b2 = u / |u|
    float pb = dot3(b2, gb2);
    float gu[3];
    for (int k = 0; k < 3; ++k) gu[k] = (gb2[k] - b2[k] * pb) / n2;
    // u = a2 - (b1.a2) b1
    float ub = dot3(b1, gu);
    float ga2[3];
    for (int k = 0; k < 3; ++k) {
      ga2[k] = gu[k] - b1[k] * ub;
      gb1[k] += -a2[k] * ub - dt * gu[k];
    }
    // b1 = a1 / |a1|
    float pa = dot3(b1, gb1);
    float ga1[3];
    for (int k = 0; k < 3; ++k) ga1[k] = (gb1[k] - b1[k] * pa) / n1;
    const float f = S.cam[9];
    gcam[0] = tot[9]; gcam[1] = tot[10]; gcam[2] = tot[11];
    gcam[3] = ga1[0]; gcam[4] = ga1[1]; gcam[5] = ga1[2];
    gcam[6] = ga2[0]; gcam[7] = ga2[1]; gcam[8] = ga2[2];
    if (S.flags & PULSAR_FLAG_ORTHOGRAPHIC) {   // kappa = s / W
      gcam[9] = 0.0f;
      gcam[10] = tot[12] / (float)S.width;
    } else {                                    // kappa = s / (W f)
      gcam[9] = -tot[12] * S.kappa / f;
      gcam[10] = tot[12] / ((float)S.width * f);
    }
  }
  __syncthreads();
  if ((mask & PULSAR_GRAD_CAM) && threadIdx.x < 11) {
    // paper gradients: the area-weighted average of the per-sphere terms times
    // 1e-3, with the area taken as the tracked pixels: 1e-3 of the plain sum
    const float g = (S.flags & PULSAR_FLAG_PAPER_GRADIENTS) ? 1e-3f * gcam[threadIdx.x] : gcam[threadIdx.x];
    if (S.flags & PULSAR_FLAG_ACCUMULATE)
      atomicAdd(S.g_cam + threadIdx.x, g);
    else
      S.g_cam[threadIdx.x] = g;
  }
}

// First stage of the camera and background reduction: CTA (scene, part)
// sums its share of the per-block camera partials, the per-(item, pixel
// block) pitch partials and the per-(tile, pixel block) background partials.
__global__ void __launch_bounds__(256) camera_partials_kernel(WsView v, uint32_t mask) {
  pdl_wait();
  pdl_trigger();
  __shared__ float red[8][kRedValues];
  const SceneDev& S = v.scenes[blockIdx.x];
  const int part = blockIdx.y;
  const int C = S.n_channels;
  const int64_t nt = (int64_t)S.tiles_x * S.tiles_y;
  const int stride = kRedParts * blockDim.x;
  const int start = part * blockDim.x + threadIdx.x;
  float acc[kRedValues];
#pragma unroll
  for (int k = 0; k < kRedValues; ++k) acc[k] = 0.0f;
  if (mask & PULSAR_GRAD_CAM) {
    for (int b = start; b < S.fin_blocks; b += stride) {
      const float* fp = v.fin_part + (size_t)(S.fin_block_begin + b) * kCamPartials;
#pragma unroll
      for (int k = 0; k < 13; ++k) acc[k] += fp[k];
    }
    const int i0 = 8 * v.item_begin[S.tile_begin], i1 = 8 * v.item_begin[S.tile_begin + nt];
    for (int i = i0 + start; i < i1; i += stride) acc[12] += v.item_kappa[i];
  }
  if (mask & PULSAR_GRAD_BG) {
    const float* rows = v.tile_bg + (size_t)S.tile_begin * 8 * C;
    for (int64_t t = start; t < 8 * nt; t += stride) {
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < C) acc[13 + c] += rows[t * C + c];
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < kRedValues; ++k) {
    const float x = warp_sum(acc[k]);
    if (lane == 0) red[warp][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < kRedValues) {
    float x = 0.0f;
    for (int w = 0; w < 8; ++w) x += red[w][threadIdx.x];
    v.red_part[((size_t)blockIdx.x * kRedParts + part) * kRedValues + threadIdx.x] = x;
  }
  // the scene's last CTA to finish sums every CTA's partials (its own stores
  // are made visible before it counts itself)
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(v.cam_done + blockIdx.x, 1) == kRedParts - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  camera_finish(v, mask, blockIdx.x);
  if (threadIdx.x == 0) v.cam_done[blockIdx.x] = 0;   // ready for the next backward pass
}

static_assert(sizeof(SetupPack<kMaxScenes>) + sizeof(WsView) <= 32000,
              "scene descriptors must fit the kernel parameter space");

template <int N>
cudaError_t setup_n(const WsView& v, const SceneDev* hs, int n, int full, cudaStream_t st) {
  SetupPack<N> pk;
  pk.n = n;
  pk.full = full;
  pk.n_spheres = v.n_spheres;
  for (int i = 0; i < n; ++i) pk.s[i] = hs[i];
  return launch_pdl(setup_kernel<N>, dim3(1), dim3(N < 32 ? 32 : N), 0, st, v, pk);
}

}  // namespace

cudaError_t launch_setup(const WsView& v, const SceneDev* hs, int n, cudaStream_t st) {
  // the sign of n selects the mode: n > 0 full set-up, n < 0 pointer refresh
  int full = n > 0 ? 1 : 0;
  int m = n > 0 ? n : -n;
  if (m <= 1) return setup_n<1>(v, hs, m, full, st);
  if (m <= 8) return setup_n<8>(v, hs, m, full, st);
  return setup_n<kMaxScenes>(v, hs, m, full, st);
}

cudaError_t launch_project(const WsView& v, cudaStream_t st) {
  if (v.n_spheres == 0) return cudaSuccess;
  const int64_t blocks = (v.n_spheres + kThreads - 1) / kThreads;
  return launch_pdl(project_kernel, dim3((unsigned)blocks), dim3(kThreads), 0, st, v);
}

cudaError_t launch_zero_grads(const WsView& v, uint32_t mask, cudaStream_t st) {
  if (v.n_spheres == 0) return cudaSuccess;
  const int64_t blocks = (v.n_spheres + kThreads - 1) / kThreads;
  return launch_pdl(zero_grads_kernel, dim3((unsigned)blocks), dim3(kThreads), 0, st, v, mask);
}

cudaError_t launch_finalize(const WsView& v, uint32_t mask, cudaStream_t st) {
  const uint32_t fin_mask = PULSAR_GRAD_POS | PULSAR_GRAD_RAD | PULSAR_GRAD_CAM |
                            (v.paper ? (PULSAR_GRAD_OPA | PULSAR_GRAD_FEAT) : 0u);
  if (v.fin_blocks > 0 && (mask & fin_mask))
    return launch_pdl(finalize_kernel, dim3(v.fin_blocks), dim3(kFinalizeThreads), 0, st, v, mask);
  return cudaSuccess;
}

cudaError_t launch_camera_reduce(const WsView& v, uint32_t mask, cudaStream_t st) {
  if (mask & (PULSAR_GRAD_CAM | PULSAR_GRAD_BG))
    return launch_pdl(camera_partials_kernel, dim3(v.n_scenes, kRedParts), dim3(256), 0, st, v, mask);
  return cudaSuccess;
}

}  // namespace pulsar
