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
// first key beyond its threshold, or (PULSAR_FLAG_PAPER_STOP) at the list
// position where the forward pass's early termination stopped it.
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

// Staging depth of the backward pass (batches staged ahead + 1); staging two
// batches ahead measured slower than one.
constexpr int kBwdBuffers = 2;

// Adds one tracked hit's gradients to its sphere (vector atomics where the
// layout allows).
template <int CMAX>
__device__ __forceinline__ void add_hit_grads(int id_global, int64_t id_local, float gc0, float gc1,
                                              float gc2, float gR, float go, const float (&gf)[CMAX],
                                              int C, const WsView& v, const SceneDev& S, bool geo,
                                              bool opa, bool feat) {
  if (geo) atomicAdd(&v.gacc[id_global], make_float4(gc0, gc1, gc2, gR));
  // paper gradients: opacity and feature sums stay in the workspace, with the
  // count of pixels that track the sphere, until finalize averages them
  const bool paper = v.paper != 0;
  if (paper) atomicAdd(v.pg_cnt + id_global, 1);
  if (opa) atomicAdd(paper ? v.pg_opa + id_global : S.g_opa + id_local, go);
  if (feat) {
    float* dst = paper ? v.pg_feat + (int64_t)id_global * C : S.g_feat + id_local * C;
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

// Back-propagates through work unit w (a pixel block of one work item) with
// one warp.
template <int CMAX, bool CHAIN>
__device__ __forceinline__ void bwd_unit(const WsView& v, uint32_t mask, int w, StageBuf<CMAX, kBwdBuffers>& sb) {
  ItemCtx it;
  if (!item_ctx(v, w, it)) return;
  const bool cam = (mask & PULSAR_GRAD_CAM) != 0;
  // a chained walk handles the tile's later segments from its first
  if (CHAIN && it.seg != 0) {
    if (cam && threadIdx.x == 0) v.item_kappa[it.slot] = 0.0f;
    return;
  }
  const SceneDev& S = v.scenes[it.scene];
  const PixelCtx pc = pixel_ctx(S, it.tile, it.block);
  const int C = S.n_channels;
  const float gamma = S.gamma, zfar = S.zfar, znear = S.znear;
  const float inv_gamma = 1.0f / gamma;
  const float inv_range = 1.0f / (zfar - znear);
  const bool literal = (S.flags & PULSAR_FLAG_DIST_LITERAL) != 0;
  const bool ortho = (S.flags & PULSAR_FLAG_ORTHOGRAPHIC) != 0;
  const bool geo = (mask & (PULSAR_GRAD_POS | PULSAR_GRAD_RAD | PULSAR_GRAD_CAM)) != 0;
  const bool opa = (mask & PULSAR_GRAD_OPA) != 0;
  const bool feat = (mask & PULSAR_GRAD_FEAT) != 0;
  const bool bgw = (mask & PULSAR_GRAD_BG) != 0;
  const bool per_hit = geo || opa || feat;
  const int lane = threadIdx.x & 31;

  // the first batches of the block list stage while the pixel data loads
  UnitStream<CMAX, kBwdBuffers, CHAIN> ws;
  if (per_hit) ws.start(sb, v, S, it, true);

  // per-pixel upstream data
  const int64_t pix = pc.inside ? (int64_t)pc.py * S.width + pc.px : 0;
  const int64_t gpix = S.pixel_begin + pix;
  float G[CMAX];
  float logD = 0.0f, GFres = 0.0f, Gref = 0.0f;
  float thr_t = __int_as_float(0x7f800000);
  int thr_i = 0x7fffffff, dom = -1;
  int stop_pos = 0x7fffffff;   // list position where the paper's early termination stopped
#pragma unroll
  for (int c = 0; c < CMAX; ++c) G[c] = 0.0f;
  if (pc.inside) {
    const float4 aux = v.pix_aux[gpix];
    logD = S.log_norm_in[pix];
    const float* g = S.grad_image + pix * C;
    const float* fr = v.fres + gpix * C;
    // 16-byte loads where the layout allows
    const bool vec = (C & 3) == 0 && ((reinterpret_cast<uintptr_t>(g) | reinterpret_cast<uintptr_t>(fr)) & 15) == 0;
    if (vec) {
#pragma unroll
      for (int c = 0; c < CMAX; c += 4)
        if (c < C) {
          const float4 x = __ldg(reinterpret_cast<const float4*>(g + c));
          const float4 y = __ldg(reinterpret_cast<const float4*>(fr + c));
          G[c] = x.x; G[c + 1] = x.y; G[c + 2] = x.z; G[c + 3] = x.w;
          GFres = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, GFres))));
        }
    } else {
#pragma unroll
      for (int c = 0; c < CMAX; ++c)
        if (c < C) {
          G[c] = __ldg(g + c);
          GFres = fmaf(G[c], __ldg(fr + c), GFres);
        }
    }
    thr_t = aux.x;
    thr_i = __float_as_int(aux.y);
    dom = __float_as_int(aux.z);
    if (CHAIN && (S.flags & PULSAR_FLAG_PAPER_STOP)) stop_pos = __float_as_int(aux.w);
    const float* fref = dom < 0 ? S.bg : S.feat + (int64_t)(dom - S.sphere_begin) * C;
#pragma unroll
    for (int c = 0; c < CMAX; ++c)
      if (c < C) Gref = fmaf(G[c], __ldg(fref + c), Gref);
  }

  // background gradient: sum over the block of w_B G (first segment only)
  if (bgw && it.seg == 0) {
    const float wB = pc.inside ? __expf(S.eps * inv_gamma - logD) : 0.0f;
    float* dst = v.tile_bg + ((size_t)it.tile * kBlocksPerTile + it.block) * C;
#pragma unroll
    for (int c = 0; c < CMAX; ++c) {
      const float x = warp_sum(wB * G[c]);
      if (lane == 0 && c < C) dst[c] = x;
    }
  }
  if (!per_hit) {
    if (cam && lane == 0) v.item_kappa[it.slot] = 0.0f;
    return;
  }

  const float kstop = next_up(thr_t);
  bool done = !pc.inside;
  float gk_sum = 0.0f;
  for (; ws.base < ws.n; ws.advance()) {
    if (__all_sync(0xffffffffu, done)) break;
    uint32_t hits = ws.begin(sb, v, S, true);
    const int cur = ws.buf;
    if (done) hits = 0u;
    // phase 2: this lane's tracked hits, in list order
    while (hits) {
      const int j = __ffs(hits) - 1;
      hits &= hits - 1u;
      const float4 a = sb.rec0[cur][j];
      const float4 b = sb.rec1[cur][j];
      if (b.x >= kstop || ws.base + j >= stop_pos) {
        done = true;
        break;
      }
      const int id = sb.id[cur][j];
      const float4 c2 = sb.rec2[cur][j];
      // Tracked: a hit (depth below zfar) with (t, id) at most the pixel's
      // threshold.  A sphere whose far side lies in front of both the
      // threshold depth and zfar is a tracked hit whatever its exact hit
      // depth (every hit depth is at most c_z + R, up to rounding), so the
      // hit depth is evaluated only for spheres near the threshold.
      if (!(fmaf(1.0001f, a.z, 1.001f * c2.w) < fminf(thr_t, zfar))) {
        RayHit h;
        if (!pixel_ray_hit(a, b.x, pc.rx, pc.ry, zfar, ortho, h)) continue;
        if (hit_less(thr_t, thr_i, h.t, id)) continue;   // beyond the tracked set
      }
      float gc0 = 0.f, gc1 = 0.f, gc2 = 0.f, gR = 0.f, go = 0.f;
      float gf[CMAX];
      const ValueGeom g = pixel_value_geom(a, c2, pc.vr, ortho);
      const float R = c2.w;
      const float inv_rr = vdiv(1.0f, g.rr);
      const float qd = g.qd;            // as the forward pass blended it
      const float dist = qd * R;
      const float qdc = fminf(qd, 1.0f);
      const float d = literal ? qdc : 1.0f - qdc;
      const float z = (((zfar - a.z) - c2.z) + g.off) * inv_range;
      const float t_val = (a.z - g.off) + c2.z;
      const float o = b.y;
      const float s = o * z * inv_gamma;
      // e^{s} / D; the clamp only matters for zero-weight hits, whose
      // exponent may exceed log D by any amount
      const float E = __expf(fminf(s - logD, 80.0f));
      const float w = o * d * E;
      const float* f = &sb.feat[cur][j * StageBuf<CMAX, kBwdBuffers>::FS];
      float gdot;   // G.(f_i - F)
      if (id == dom) {
        gdot = -GFres;
      } else {
        gdot = -Gref - GFres;
#pragma unroll
        for (int c = 0; c < CMAX; ++c) gdot = fmaf(G[c], f[c], gdot);
      }
#pragma unroll
      for (int c = 0; c < CMAX; ++c) gf[c] = w * G[c];
      go = gdot * d * E * (1.0f + s);
      const float gd = gdot * o * E;
      const float gz = gdot * w * o * inv_gamma;
      const float gt = -gz * inv_range;
      float gdist = 0.0f;
      if (qd < 1.0f) {
        const float sgn = literal ? 1.0f : -1.0f;
        gdist = sgn * vdiv(gd, R);
        gR = -sgn * gd * vdiv(qd, R);
      }
      // e = (r x (c x r)) / |r|^2 with c x r = (-ey, ex, ez); orthographic:
      // c the shifted centre and r = (0, 0, 1)
      const float rx = ortho ? 0.0f : pc.vr.rx, ry = ortho ? 0.0f : pc.vr.ry;
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
      gc0 = gt * rx * inv_rr + gt_sq * e0;
      gc1 = gt * ry * inv_rr + gt_sq * e1;
      gc2 = gt * inv_rr + gt_sq * e2;
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
      const float pxo = (float)(2 * pc.px + 1 - S.width) * 0.5f;
      const float pyo = (float)(2 * pc.py + 1 - S.height) * 0.5f;
      // the pitch enters through the ray slopes (pinhole) or through the
      // shift c - k (pxo, pyo, 0) of the centre (orthographic)
      gk_sum += ortho ? -(gc0 * pxo + gc1 * pyo) : grx * pxo + gry * pyo;
      add_hit_grads<CMAX>(id, (int64_t)id - S.sphere_begin, gc0, gc1, gc2, gR, go, gf, C, v, S, geo,
                          opa, feat);
    }
    if (!done && sb.rec1[cur][ws.count() - 1].x >= kstop) done = true;
  }
  ws.drain();
  if (cam) {
    const float x = warp_sum(gk_sum);
    if (lane == 0) v.item_kappa[it.slot] = x;
  }
}

// One CTA per work unit, or (persistent) one resident CTA per slot taking
// units from the workspace counter.
template <int CMAX, bool CHAIN>
__global__ void __launch_bounds__(32, 16) render_bwd_kernel(const WsView v, uint32_t mask) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StageBuf<CMAX, kBwdBuffers>& sb = *reinterpret_cast<StageBuf<CMAX, kBwdBuffers>*>(smem_raw);
  if (!v.persistent) {
    bwd_unit<CMAX, CHAIN>(v, mask, blockIdx.x, sb);
    return;
  }
  const int n_units = v.hdr->n_items * kBlocksPerTile;
  for (;;) {
    const int w = next_unit(v);
    if (w >= n_units) {
      done_units(v, w, n_units);
      break;
    }
    bwd_unit<CMAX, CHAIN>(v, mask, w, sb);
    __syncwarp();
  }
}

template <int CMAX>
cudaError_t launch_bwd_t(const WsView& v, uint32_t mask, cudaStream_t st) {
  const size_t smem = sizeof(StageBuf<CMAX, kBwdBuffers>);
  // the paper's early termination walks a tile's segments in order
  auto kern = v.chain ? render_bwd_kernel<CMAX, true> : render_bwd_kernel<CMAX, false>;
  unsigned grid = (unsigned)v.max_items * kBlocksPerTile;
  if (v.persistent) {
    const unsigned slots = resident_slots(kern, 32, smem);
    if (slots == 0) return cudaErrorLaunchOutOfResources;
    if (slots < grid) grid = slots;
  }
  return launch_pdl(kern, dim3(grid), dim3(32), smem, st, v, mask);
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
