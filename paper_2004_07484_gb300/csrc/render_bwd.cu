// Backward pass (App. B, "The Backward Pass"), parallel over pixels.
//
// A hit is tracked when its (depth, index) is at most the pixel's n_track-th
// tracked hit.  That threshold is kept per pixel by the forward pass (store
// mode, App. B "Preparing for the Backward Pass") or recomputed before this
// pass by the forward traversal without blending (recompute mode).  Work is
// split into the same one-warp (segment, pixel block) CTAs as the forward
// pass; gradients are sums, so segments need no merge.  As in the forward
// pass, each batch of staged spheres is first hit-tested by every lane, then
// each lane walks its own tracked hits and adds their gradients with (vector)
// atomics, so lanes never wait on one another's hits.  A pixel stops at the
// first key beyond its threshold.
//
// Derivatives (Eq. 1 with a = o d e^{o z / gamma}, D its denominator, G = dL/dF):
//   dL/df_i = w_i G,   dL/da_i = G.(f_i - F) / D,
//   da/do = d e^s (1 + s),  da/dd = o e^s,  da/dz = a o / gamma,  s = o z / gamma,
//   z = (zfar - t) / (zfar - znear),
//   t = t_c - sqrt(disc)/|r|^2 (front root), dist = |e|, e = c - t_c r,
//   dt/dc = r/|r|^2 + e/sqrt(disc),  dt/dR = -R/sqrt(disc),
//   dt/dr = (e (1 - b/sqrt(disc)) - t r)/|r|^2,  b = r.c,
//   ddist/dc = e/dist,  ddist/dr = -t_c e/dist.
// Ray slopes depend on the pixel pitch kappa: dr/dkappa = (u + 1/2 - W/2, v + 1/2 - H/2, 0).
// G.(f_i - F) is formed as G.(f_i - f_ref) - G.(F - f_ref) from the forward's
// reference feature, exactly -G.(F - f_ref) for the reference hit itself,
// which keeps it accurate where one hit carries nearly all the weight.
#include "render_common.cuh"

namespace pulsar {

namespace {

// Adds one tracked hit's gradients to its sphere (vector atomics where the
// layout allows).
template <int CMAX>
__device__ __forceinline__ void add_hit_grads(int id_global, int64_t id_local, float gc0, float gc1,
                                              float gc2, float gR, float go, const float (&gf)[CMAX],
                                              int C, const WsView& v, const SceneDev& S, bool geo,
                                              bool opa, bool feat) {
  if (geo) atomicAdd(&v.gacc[id_global], make_float4(gc0, gc1, gc2, gR));
  if (opa) atomicAdd(S.g_opa + id_local, go);
  if (feat) {
    float* dst = S.g_feat + id_local * C;
    if ((C & 3) == 0) {
#pragma unroll
      for (int c = 0; c < CMAX; c += 4)
        if (c < C)
          atomicAdd(reinterpret_cast<float4*>(dst + c), make_float4(gf[c], gf[c + 1], gf[c + 2], gf[c + 3]));
    } else {
#pragma unroll
      for (int c = 0; c < CMAX; ++c)
        if (c < C) atomicAdd(dst + c, gf[c]);
    }
  }
}

// Per-pixel data of the warp's block, in shared memory behind the staging
// buffers: any lane may process any pixel's hits.
template <int CMAX>
struct BwdPixels {
  float G[32][CMAX + 4];   // upstream gradient (rows padded against bank conflicts)
  float gfres[32];         // G . (F - f_ref)
  float gref[32];          // G . f_ref
  float logd[32];          // log D
  float thr_t[32];         // depth and index of the n_track-th tracked hit
  int thr_i[32];
  int dom[32];             // reference sphere (-1: background)
  uint32_t hmask[32];      // this batch's tracked-hit candidates of each pixel
  int hoff[33];            // their exclusive prefix over the pixels
};

// Position of the r-th (0-based) set bit of m (r < popc(m)).
__device__ __forceinline__ int nth_set_bit(uint32_t m, int r) {
  int pos = 0;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const int c = __popc(m & ((1u << s) - 1u));
    if (r >= c) {
      r -= c;
      m >>= s;
      pos += s;
    }
  }
  return pos;
}

// Back-propagates through work unit w (a pixel block of one work item) with
// one warp.  Per batch, every pixel's candidate hits (its mask bits up to its
// stop point) are enumerated across the warp, and lane k takes the k-th hit
// of the batch, 32 at a time, whatever pixel it belongs to: the gradient of
// a hit depends only on the hit and its pixel's forward data, and gradients
// are sums, so all lanes stay busy however the hits are spread over pixels.
template <int CMAX>
__device__ __forceinline__ void bwd_unit(const WsView& v, uint32_t mask, int w, StageBuf<CMAX>& sb,
                                         BwdPixels<CMAX>& px) {
  ItemCtx it;
  if (!item_ctx(v, w, it)) return;
  const int si = scene_of_tile(v.scenes, v.n_scenes, it.tile);
  const SceneDev& S = v.scenes[si];
  const PixelCtx pc = pixel_ctx(S, it.tile, it.block);
  const int C = S.n_channels;
  const float gamma = S.gamma, zfar = S.zfar, znear = S.znear;
  const float inv_gamma = 1.0f / gamma;
  const float inv_range = 1.0f / (zfar - znear);
  const bool literal = (S.flags & PULSAR_FLAG_DIST_LITERAL) != 0;
  const bool geo = (mask & (PULSAR_GRAD_POS | PULSAR_GRAD_RAD | PULSAR_GRAD_CAM)) != 0;
  const bool opa = (mask & PULSAR_GRAD_OPA) != 0;
  const bool feat = (mask & PULSAR_GRAD_FEAT) != 0;
  const bool cam = (mask & PULSAR_GRAD_CAM) != 0;
  const bool bgw = (mask & PULSAR_GRAD_BG) != 0;
  const int lane = threadIdx.x & 31;

  // this lane's pixel: upstream data into shared memory
  float thr_t = __int_as_float(0x7f800000);
  float logD = 0.0f;
  {
    const int64_t pix = pc.inside ? (int64_t)pc.py * S.width + pc.px : 0;
    const int64_t gpix = S.pixel_begin + pix;
    float gfres = 0.0f, gref = 0.0f;
    int thr_i = 0x7fffffff, dom = -1;
    float* G = px.G[lane];
#pragma unroll
    for (int c = 0; c < CMAX; ++c) G[c] = 0.0f;
    if (pc.inside) {
      const float* g = S.grad_image + pix * C;
      const float* fr = v.fres + gpix * C;
      const float4 aux = v.pix_aux[gpix];
      thr_t = aux.x;
      thr_i = __float_as_int(aux.y);
      dom = __float_as_int(aux.z);
      const float* fref = dom < 0 ? S.bg : S.feat + (int64_t)(dom - S.sphere_begin) * C;
#pragma unroll
      for (int c = 0; c < CMAX; ++c)
        if (c < C) {
          const float gc = g[c];
          G[c] = gc;
          gfres = fmaf(gc, fr[c], gfres);
          gref = fmaf(gc, fref[c], gref);
        }
      logD = S.log_norm_in[pix];
    }
    px.gfres[lane] = gfres;
    px.gref[lane] = gref;
    px.logd[lane] = logD;
    px.thr_t[lane] = thr_t;
    px.thr_i[lane] = thr_i;
    px.dom[lane] = dom;
  }
  __syncwarp();

  // background gradient: sum over the block of w_B G (first segment only)
  if (bgw && it.seg == 0) {
    const float wB = pc.inside ? __expf(S.eps * inv_gamma - logD) : 0.0f;
    float* dst = v.tile_bg + ((size_t)it.tile * kBlocksPerTile + it.block) * C;
#pragma unroll
    for (int c = 0; c < CMAX; ++c) {
      const float x = warp_sum(wB * px.G[lane][c]);
      if (lane == 0 && c < C) dst[c] = x;
    }
  }
  if (!(geo || opa || feat)) {
    if (cam && lane == 0) v.item_kappa[it.slot] = 0.0f;
    return;
  }

  const float kstop = next_up(thr_t);
  bool done = !pc.inside;
  float gk_sum = 0.0f;
  UnitStream<CMAX> ws;
  ws.start(sb, v, S, it, true);
  for (; ws.base < ws.n; ws.advance()) {
    if (__all_sync(0xffffffffu, done)) break;
    uint32_t h = ws.begin(sb, v, S, true);
    const int cur = ws.buf;
    const int cnt = ws.count();
    if (done) h = 0u;
    if (h) {
      // keys rise along the list: this pixel stops at its first entry keyed
      // at or beyond its bound
      int lo = 0, hi = cnt;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sb.rec1[cur][mid].x >= kstop) hi = mid; else lo = mid + 1;
      }
      if (lo < 32) h &= (1u << lo) - 1u;
    }
    if (!done && sb.rec1[cur][cnt - 1].x >= kstop) done = true;
    // enumerate the batch's candidate hits over the warp
    const int nh = __popc(h);
    int off = nh;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, off, d);
      if (lane >= d) off += y;
    }
    const int total = __shfl_sync(0xffffffffu, off, 31);
    px.hmask[lane] = h;
    px.hoff[lane] = off - nh;
    __syncwarp();
    for (int k = lane; k - lane < total; k += 32) {
      if (k >= total) break;
      // owner pixel q: the last pixel whose hits start at or before k
      int q = 0;
      {
        int l = 0, r = 31;
        while (l < r) {
          const int mid = (l + r + 1) >> 1;
          if (px.hoff[mid] <= k) l = mid; else r = mid - 1;
        }
        q = l;
      }
      const int j = nth_set_bit(px.hmask[q], k - px.hoff[q]);
      const float4 a = sb.rec0[cur][j];
      const float4 b = sb.rec1[cur][j];
      const int qx = pc.tile_x0 + (it.block & 1) * 8 + (q & 7);
      const int qy = pc.tile_y0 + (it.block >> 1) * 4 + (q >> 3);
      const float rx_d = ray_coord(qx, S.width, S.kappa), ry_d = ray_coord(qy, S.height, S.kappa);
      RayHit hh;
      if (!ray_hit(a.x, a.y, a.z, a.w, b.x, rx_d, ry_d, zfar, hh)) continue;
      const int id = sb.id[cur][j];
      if (hit_less(px.thr_t[q], px.thr_i[q], hh.t, id)) continue;   // beyond the tracked set
      const ValueRay vr = value_ray(qx, qy, S.width, S.height, S.kappa_hi, S.kappa_lo);
      const float4 c2 = sb.rec2[cur][j];
      const ValueGeom g = value_geom(a, c2, vr);
      const float R = c2.w;
      const float inv_rr = vdiv(1.0f, g.rr);
      const float dist = g.dist;
      const float qd = dist / R;
      const float qdc = fminf(qd, 1.0f);
      const float d = literal ? qdc : 1.0f - qdc;
      const float z = (((zfar - a.z) - c2.z) + g.off) * inv_range;
      const float t_val = (a.z - g.off) + c2.z;
      const float o = b.y;
      const float s = o * z * inv_gamma;
      // e^{s} / D; the clamp only matters for zero-weight hits, whose
      // exponent may exceed log D by any amount
      const float E = __expf(fminf(s - px.logd[q], 80.0f));
      const float wgt = o * d * E;
      const float* f = &sb.feat[cur][j * CMAX];
      const float* G = px.G[q];
      float gdot;   // G.(f_i - F)
      if (id == px.dom[q]) {
        gdot = -px.gfres[q];
      } else {
        gdot = -px.gref[q] - px.gfres[q];
#pragma unroll
        for (int c = 0; c < CMAX; ++c) gdot = fmaf(G[c], f[c], gdot);
      }
      float gf[CMAX];
#pragma unroll
      for (int c = 0; c < CMAX; ++c) gf[c] = wgt * G[c];
      const float go = gdot * d * E * (1.0f + s);
      const float gd = gdot * o * E;
      const float gz = gdot * wgt * o * inv_gamma;
      const float gt = -gz * inv_range;
      float gdist = 0.0f, gR = 0.0f;
      if (qd < 1.0f) {
        const float sgn = literal ? 1.0f : -1.0f;
        gdist = sgn * vdiv(gd, R);
        gR = -sgn * gd * vdiv(qd, R);
      }
      // e = (r x (c x r)) / |r|^2 with c x r = (-ey, ex, ez)
      const float rx = vr.rx, ry = vr.ry;
      const float e0 = (ry * g.ez - g.ex) * inv_rr;
      const float e1 = (-g.ey - rx * g.ez) * inv_rr;
      const float e2 = (rx * g.ex + ry * g.ey) * inv_rr;
      // gt / sqrt(disc): the depth derivatives carry 1/sqrt(disc), which
      // diverges at the rim, while gt carries d.  With d = 1 - dist/R,
      // d / sqrt(disc) = sqrt(disc) / (|r|^2 R (R + dist)) exactly, so
      // the product is formed without dividing by a vanishing sqrt(disc)
      // (d itself has a float32 floor of ~1e-7 there).  With the
      // literal d the product diverges in exact arithmetic too.
      float gt_sq;
      if (literal) {
        gt_sq = g.sq > 0.0f ? vdiv(gt, g.sq) : 0.0f;
      } else {
        const float d_over_sq = vdiv(g.sq * inv_rr, R * (R + dist));
        gt_sq = -gdot * o * E * o * inv_gamma * inv_range * d_over_sq;
      }
      const float tc = t_val + g.sq * inv_rr;   // closest-approach parameter
      const float b_ = tc * g.rr;               // r . c
      float gc0 = gt * rx * inv_rr + gt_sq * e0;
      float gc1 = gt * ry * inv_rr + gt_sq * e1;
      float gc2 = gt * inv_rr + gt_sq * e2;
      gR += -R * gt_sq;
      float grx = (gt * e0 - gt_sq * b_ * e0 - gt * t_val * rx) * inv_rr;
      float gry = (gt * e1 - gt_sq * b_ * e1 - gt * t_val * ry) * inv_rr;
      if (dist > 0.0f) {
        const float gi = vdiv(gdist, dist);
        gc0 += gi * e0;
        gc1 += gi * e1;
        gc2 += gi * e2;
        grx += -gi * tc * e0;
        gry += -gi * tc * e1;
      }
      const float pxo = (float)(2 * qx + 1 - S.width) * 0.5f;
      const float pyo = (float)(2 * qy + 1 - S.height) * 0.5f;
      gk_sum += grx * pxo + gry * pyo;
      add_hit_grads<CMAX>(id, (int64_t)id - S.sphere_begin, gc0, gc1, gc2, gR, go, gf, C, v, S, geo,
                          opa, feat);
    }
    __syncwarp();   // hmask / hoff are rewritten by the next batch
  }
  ws.drain();
  if (cam) {
    const float x = warp_sum(gk_sum);
    if (lane == 0) v.item_kappa[it.slot] = x;
  }
}

// One CTA per work unit, or (persistent) one resident CTA per slot taking
// units from the workspace counter.
template <int CMAX>
__global__ void __launch_bounds__(32, 16) render_bwd_kernel(const WsView v, uint32_t mask) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StageBuf<CMAX>& sb = *reinterpret_cast<StageBuf<CMAX>*>(smem_raw);
  BwdPixels<CMAX>& px = *reinterpret_cast<BwdPixels<CMAX>*>(smem_raw + sizeof(StageBuf<CMAX>));
  if (!v.persistent) {
    bwd_unit<CMAX>(v, mask, blockIdx.x, sb, px);
    return;
  }
  const int n_units = v.hdr->n_items * kBlocksPerTile;
  for (;;) {
    const int w = next_unit(v);
    if (w >= n_units) break;
    bwd_unit<CMAX>(v, mask, w, sb, px);
    __syncwarp();
  }
}

template <int CMAX>
cudaError_t launch_bwd_t(const WsView& v, uint32_t mask, cudaStream_t st) {
  const size_t smem = sizeof(StageBuf<CMAX>) + sizeof(BwdPixels<CMAX>);
  auto kern = render_bwd_kernel<CMAX>;
  unsigned grid = (unsigned)v.max_items * kBlocksPerTile;
  if (v.persistent) {
    const unsigned slots = resident_slots(kern, 32, smem);
    if (slots == 0) return cudaErrorLaunchOutOfResources;
    if (slots < grid) grid = slots;
    cudaError_t e = cudaMemsetAsync(&v.hdr->work_next, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, 32, smem, st>>>(v, mask);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_render_bwd(const WsView& v, uint32_t mask, cudaStream_t st) {
  if (v.max_items == 0) return cudaSuccess;
  const int C = v.n_channels;
  if (C <= 4) return launch_bwd_t<4>(v, mask, st);
  if (C <= 8) return launch_bwd_t<8>(v, mask, st);
  if (C <= 16) return launch_bwd_t<16>(v, mask, st);
  return launch_bwd_t<32>(v, mask, st);
}

}  // namespace pulsar
