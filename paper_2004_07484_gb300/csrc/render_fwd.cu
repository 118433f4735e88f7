// Forward pass: App. B, Step 1 (intersection search) and Step 2 (draw).
//
// Work decomposition.  A tile's depth-ordered list is cut into segments of
// at most `segment` entries, and every (segment, 8 x 4 pixel block) pair is
// one warp-sized CTA, so a few very long lists no longer serialise the launch
// and an idle block never waits for a busy one.  Eq. 1 is a commutative sum
// (App. A) and the n_track closest hits of a union are the closest of the
// per-part closest, so segments are combined afterwards: the warp that
// finishes a block's segments last (a per-block atomic counter) merges the
// partial states the others left in the workspace and writes the pixels.
//
// Each batch of up to 32 staged spheres is handled in two phases: every lane
// first runs the cheap float32 hit test of its pixel against all of them and
// records its hits in a bit mask, then lanes walk their own hits in list
// order.  The expensive per-hit work (hit depth, Eq. 1 update, queue) thus
// runs once per hit of the busiest lane instead of once per sphere any lane
// hits.  Handling a lane's hits in list order (and skipping its non-hits)
// leaves every decision unchanged: keys rise along the list and the stop
// bound only falls, so the first hit at or beyond the bound is where a pixel
// would have stopped anyway.
//
// Per pixel, hits are blended with the largest exponent o z / gamma divided
// out of numerator and denominator, and the numerator is kept relative to a
// reference feature: the feature of the hit with the largest weight so far
// (initially the background), i.e. the state is
//   den = e^{eps/g - m} + sum_k a_k e^{-m},
//   res = sum_k a_k e^{-m} (f_k - f_ref) + e^{eps/g - m} (bg - f_ref),
//   F   = f_ref + res / den.
// F - f_ref is thereby kept to float precision even where one hit carries
// nearly all the weight; the backward pass needs exactly that difference.
//
// The n_track closest hits (by float32 depth, then index) are kept in a
// register queue (App. B, Step 2).  Early termination (Sec. 3.2, App. B
// Step 2), exact: a pixel stops at the first listed sphere whose key
// (earliest depth) is
//   (i)  beyond the depth of its n_track-th tracked hit, so no later sphere
//        can enter the tracked set (every hit depth is >= its sphere's key), and
//   (ii) so far that the largest total weight all remaining spheres of the
//        segment could still add, N_rem |o|max exp(|o|max z(key) / gamma), is
//        at most 1e-7 of the segment's own denominator (a lower bound of the
//        pixel's).
// Both tests only use the segment's own state, so they stay exact when the
// segments are merged.
//
// With PULSAR_FLAG_PAPER_STOP a pixel also stops, as the paper's renderer
// does (App. B, Step 2), before the first hit whose largest possible weight
// A = e^{o_max z_b / g} is below tau (1 % by default) of D + A; that is, with
// D = e^{m} den, beyond the key
//   k3 = zfar - (zfar - znear) (g / o_max) (m + ln den + ln(tau / (1 - tau))),
// which only falls as hits are blended.  The pixel's list position where it
// stopped goes to the backward pass with the tracked set.  Tiles then have a
// chained walk: one render unit takes every segment of its tile's list in
// order (the block lists are still built per segment), as the rule needs the
// pixel's whole denominator.
#include "render_common.cuh"

namespace pulsar {

namespace {

// Fields of a partial forward state, each a plane of 32 floats (one per lane).
enum : int { kPM = 0, kPDen = 1, kPAdom = 2, kPDom = 3, kPHits = 4, kPTests = 5, kPRes = 6 };

template <int CMAX>
struct BlendState {
  float m, den, adom;
  int dom;            // global index of the reference sphere, -1 = background
  float* fref;   // this lane's reference feature: a padded row in shared memory
  float res[CMAX];
};

template <int CMAX>
__device__ __forceinline__ void blend_hit(BlendState<CMAX>& b, float s, float od, const float* f, int id) {
  if (s > b.m) {
    const float sc = __expf(b.m - s);
    b.den *= sc;
    b.adom *= sc;
#pragma unroll
    for (int c = 0; c < CMAX; ++c) b.res[c] *= sc;
    b.m = s;
  }
  const float ap = od * __expf(s - b.m);
  if (ap > b.adom) {
    // the new hit becomes the reference: re-express the numerator
#pragma unroll
    for (int c = 0; c < CMAX; ++c) {
      b.res[c] = fmaf(b.den, b.fref[c] - f[c], b.res[c]);
      b.fref[c] = f[c];
    }
    b.adom = ap;
    b.dom = id;
  } else {
#pragma unroll
    for (int c = 0; c < CMAX; ++c) b.res[c] = fmaf(ap, f[c] - b.fref[c], b.res[c]);
  }
  b.den += ap;
}

// Reference feature of a sphere index (-1 = background).
__device__ __forceinline__ const float* ref_feature(const SceneDev& S, int dom) {
  return dom < 0 ? S.bg : S.feat + (int64_t)(dom - S.sphere_begin) * S.n_channels;
}

// Renders work unit w (a pixel block of one work item) with one warp.
template <int KMAX, int CMAX, bool BLEND, bool CHAIN>
__device__ __forceinline__ void traverse_unit(const WsView& v, int w, StageBuf<CMAX>& sb) {
  ItemCtx it;
  if (!item_ctx(v, w, it)) return;
  // a chained walk renders the tile's later segments from its first
  if (CHAIN && it.seg != 0) return;
  const SceneDev& S = v.scenes[it.scene];
  PixelCtx pc = pixel_ctx(S, it.tile, it.block);
  const int C = S.n_channels;
  const int K = S.n_track;
  const float gamma = S.gamma, zfar = S.zfar, znear = S.znear;
  const float inv_gamma = 1.0f / gamma;
  const float range = zfar - znear, inv_range = 1.0f / range;
  const float omax = __uint_as_float(S.omax_bits);
  const bool literal = (S.flags & PULSAR_FLAG_DIST_LITERAL) != 0;
  const bool ortho = (S.flags & PULSAR_FLAG_ORTHOGRAPHIC) != 0;
  const int lane = threadIdx.x;

  // the first batches of the block list stage while the state is set up
  UnitStream<CMAX, 2, CHAIN> ws;
  ws.start(sb, v, S, it, BLEND);

  // the background term e^{eps/g - m} belongs to the first segment only
  BlendState<CMAX> bs;
  bs.fref = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(&sb) + sizeof(StageBuf<CMAX>)) +
            lane * StageBuf<CMAX>::FS;
  bs.m = S.eps * inv_gamma;
  bs.den = it.seg == 0 ? 1.0f : 0.0f;
  bs.adom = bs.den;
  bs.dom = -1;
#pragma unroll
  for (int c = 0; c < CMAX; ++c) {
    if (BLEND) bs.fref[c] = c < C ? S.bg[c] : 0.0f;
    bs.res[c] = 0.0f;
  }
  uint64_t q[KMAX];
  queue_init<KMAX>(q, K);
  int nhit = 0, ntest = 0;
  bool done = !pc.inside;
  float kstop1 = __int_as_float(0x7f800000);   // tracked-set bound (i)
  // the paper's early termination: its key bound and where the pixel stopped
  // (the paper's rule comes with the chained walk: other instantiations never take it)
  const bool pstop = CHAIN && BLEND && (S.flags & PULSAR_FLAG_PAPER_STOP) != 0 && omax > 0.0f;
  const float pscale = range * gamma / omax;
  const float log_ratio = S.stop_log_ratio;
  auto paper_bound = [&]() { return zfar - pscale * ((bs.m + __logf(bs.den)) + log_ratio); };
  float kstop3 = pstop ? paper_bound() : __int_as_float(0x7f800000);
  int stop_pos = 0x7fffffff;
  // the n_tests diagnostic of a chained walk: every segment's tests
  if (CHAIN && S.n_tests)
    for (int k = it.first; k < it.first + it.nseg; ++k)
      ntest += v.unit_tests[((size_t)k * kBlocksPerTile + it.block) * 32 + lane];

  for (; ws.base < ws.n; ws.advance()) {
    if (__all_sync(0xffffffffu, done)) break;
    // remaining-mass bound (ii), from the state at the start of this batch;
    // the unit's remaining entries are every sphere that can still reach
    // this block's pixels
    float kstop2 = -__int_as_float(0x7f800000);
    if (BLEND && !done && omax > 0.0f) {
      const float lr = bs.m + __logf(1e-7f * bs.den / ((float)(ws.n - ws.base) * omax));
      const float zthr = lr * gamma / omax;
      kstop2 = zthr >= 1.0f ? -__int_as_float(0x7f800000) : zfar - range * zthr;
    }
    uint32_t hits = ws.begin(sb, v, S, BLEND);
    const int cur = ws.buf;
    if (done) hits = 0u;
    // phase 2: this lane's hits, in list order
    while (hits) {
      const int j = __ffs(hits) - 1;
      hits &= hits - 1u;
      const float4 a = sb.rec0[cur][j];
      const float4 b = sb.rec1[cur][j];
      if (b.x >= fmaxf(kstop1, kstop2)) {
        done = true;
        break;
      }
      if (b.x > kstop3) {
        done = true;
        stop_pos = ws.base + j;
        break;
      }
      // The float32 hit depth orders the queue and makes the far-plane cut.
      // Every hit depth is at least the sphere's key, so a sphere keyed
      // beyond the n_track-th tracked depth cannot enter the queue; if its
      // far side also lies well in front of zfar (the depth can exceed
      // c_z + R only by rounding), the hit mask alone decides the hit.
      const bool may_queue = b.x <= key_depth(q[KMAX - 1]);
      float4 c2 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (BLEND) c2 = sb.rec2[cur][j];
      if (!BLEND && !may_queue) continue;   // cannot change the tracked set
      float t = 0.0f;
      if (may_queue || !(fmaf(1.0001f, a.z, 1.001f * c2.w) < zfar)) {
        RayHit h;
        if (!pixel_ray_hit(a, b.x, pc.rx, pc.ry, zfar, ortho, h)) continue;
        t = h.t;
      }
      ++nhit;
      const int id = sb.id[cur][j];
      if (BLEND) {
        const ValueGeom vg = pixel_value_geom(a, c2, pc.vr, ortho);
        const float qd = fminf(vg.qd, 1.0f);
        const float d = literal ? qd : 1.0f - qd;
        const float od = b.y * d;
        if (od != 0.0f) {   // a zero weight adds nothing and must not move the shift
          const float z = (((zfar - a.z) - c2.z) + vg.off) * inv_range;
          blend_hit<CMAX>(bs, b.y * z * inv_gamma, od, &sb.feat[cur][j * StageBuf<CMAX>::FS], id);
          if (pstop) kstop3 = paper_bound();
        }
      }
      if (may_queue) {
        const uint64_t key = hit_key(t, id);
        if (key < q[KMAX - 1]) {
          queue_insert<KMAX>(q, key);
          kstop1 = next_up(key_depth(q[KMAX - 1]));
        }
      }
    }
    // a pixel that stopped at no hit still stops once the batch's last key
    // passes its bound (keys rise along the list)
    if (!done) {
      const float last = sb.rec1[cur][ws.count() - 1].x;
      if (last >= fmaxf(kstop1, kstop2)) {
        done = true;
      } else if (last > kstop3) {
        done = true;
        stop_pos = ws.base + ws.count();
      }
    }
  }
  ws.drain();

  // the unit's descriptors and pixel are reloaded here rather than kept in
  // registers through the walk (the chained walk's register allocation
  // measured better without)
  if (!CHAIN) {
    item_ctx(v, w, it);
    pc = pixel_ctx(S, it.tile, it.block);
    if (S.n_tests) ntest = v.unit_tests[(size_t)it.slot * 32 + lane];
  }

  if (it.nseg > 1 && !CHAIN) {
    // leave this block's segment state, then let the block's last segment merge
    const int F = v.part_fields;
    const int q0 = kPRes + C;
    float* P = v.partial + (size_t)it.slot * F * 32 + lane;
    if (BLEND) {
      P[kPM * 32] = bs.m;
      P[kPDen * 32] = bs.den;
      P[kPAdom * 32] = bs.adom;
      P[kPDom * 32] = __int_as_float(bs.dom);
      P[kPTests * 32] = __int_as_float(ntest);
#pragma unroll
      for (int c = 0; c < CMAX; ++c)
        if (c < C) P[(kPRes + c) * 32] = bs.res[c];
    }
    P[kPHits * 32] = __int_as_float(nhit);
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
      if (k >= KMAX - K) {
        const int j = k - (KMAX - K);
        P[(q0 + j) * 32] = key_depth(q[k]);
        P[(q0 + K + j) * 32] = __int_as_float(key_index(q[k]));
      }
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0)
      last = atomicAdd(&v.tile_done[it.tile * kBlocksPerTile + it.block], 1) == it.nseg - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    for (int o = it.first; o < it.first + it.nseg; ++o) {
      if (o == it.item) continue;
      const float* Q = v.partial + ((size_t)o * kBlocksPerTile + it.block) * F * 32 + lane;
      if (BLEND) {
        const float mB = __ldcg(Q + kPM * 32);
        float denB = __ldcg(Q + kPDen * 32);
        float adomB = __ldcg(Q + kPAdom * 32);
        const int domB = __float_as_int(__ldcg(Q + kPDom * 32));
        ntest += __float_as_int(__ldcg(Q + kPTests * 32));
        const float m = fmaxf(bs.m, mB);
        const float sa = __expf(bs.m - m), sb = __expf(mB - m);
        bs.den *= sa;
        bs.adom *= sa;
        denB *= sb;
        adomB *= sb;
        const float* fB = ref_feature(S, domB);
        if (adomB > bs.adom) {
          // the other segment's reference carries more weight: re-express ours
#pragma unroll
          for (int c = 0; c < CMAX; ++c)
            if (c < C) {
              const float fb = fB[c];
              bs.res[c] = fmaf(sb, __ldcg(Q + (kPRes + c) * 32),
                               fmaf(bs.den, bs.fref[c] - fb, bs.res[c] * sa));
              bs.fref[c] = fb;
            }
          bs.adom = adomB;
          bs.dom = domB;
        } else {
#pragma unroll
          for (int c = 0; c < CMAX; ++c)
            if (c < C)
              bs.res[c] = fmaf(sb, __ldcg(Q + (kPRes + c) * 32),
                               fmaf(denB, fB[c] - bs.fref[c], bs.res[c] * sa));
        }
        bs.den += denB;
        bs.m = m;
      }
      nhit += __float_as_int(__ldcg(Q + kPHits * 32));
      for (int j = 0; j < K; ++j) {
        const uint64_t key = hit_key(__ldcg(Q + (q0 + j) * 32), __float_as_int(__ldcg(Q + (q0 + K + j) * 32)));
        if (key < q[KMAX - 1]) queue_insert<KMAX>(q, key);
        else break;   // the other segment's entries ascend
      }
    }
    if (lane == 0) v.tile_done[it.tile * kBlocksPerTile + it.block] = 0;   // ready for the next launch
  }

  const int64_t pix = (int64_t)pc.py * S.width + pc.px;
  const int64_t gpix = S.pixel_begin + pix;
  if (BLEND) {
    // F and F - f_ref of the block's pixels, staged in shared memory (the
    // staging buffers are free now), then written row by row: each pixel row
    // of the block is one contiguous run of the row-major outputs
    float* st_img = &sb.feat[0][0];
    float* st_res = &sb.feat[1][0];
    constexpr int SS = CMAX >= 8 ? CMAX + 1 : CMAX;   // staging row stride (bank-conflict free)
    const float inv = 1.0f / bs.den;
#pragma unroll
    for (int c = 0; c < CMAX; ++c)
      if (c < C) {
        const float r = bs.res[c] * inv;
        st_img[lane * SS + c] = bs.fref[c] + r;
        st_res[lane * SS + c] = r;
      }
    __syncwarp();
    const int bx0 = pc.tile_x0 + (it.block & 1) * 8, by0 = pc.tile_y0 + (it.block >> 1) * 4;
    const int nx = min(8, S.width - bx0);
    for (int r = 0; r < 4 && by0 + r < S.height; ++r) {
      const int64_t p0 = (int64_t)(by0 + r) * S.width + bx0;
      float* img = S.image + p0 * C;
      float* fr = v.fres + (S.pixel_begin + p0) * C;
      for (int f = lane; f < nx * C; f += 32) {
        const int pxl = f / C;
        const int src = (r * 8 + pxl) * SS + (f - pxl * C);
        img[f] = st_img[src];
        fr[f] = st_res[src];
      }
    }
    if (!pc.inside) return;
    S.log_norm[pix] = bs.m + __logf(bs.den);
    if (S.n_hits) S.n_hits[pix] = nhit;
    if (S.n_tests) S.n_tests[pix] = ntest;
    if (S.tracked) {
      int32_t* tr = S.tracked + pix * K;
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        if (k >= KMAX - K) {
          const int id = key_index(q[k]);
          tr[k - (KMAX - K)] = id == 0x7fffffff ? -1 : (int32_t)(id - S.sphere_begin);
        }
    }
    v.pix_aux[gpix] = make_float4(key_depth(q[KMAX - 1]), __int_as_float(key_index(q[KMAX - 1])),
                                  __int_as_float(bs.dom), __int_as_float(stop_pos));
  } else {
    if (!pc.inside) return;
    reinterpret_cast<float2*>(v.pix_aux)[2 * gpix] =
        make_float2(key_depth(q[KMAX - 1]), __int_as_float(key_index(q[KMAX - 1])));
  }
}

// One CTA per work unit, or (persistent) one resident CTA per slot taking
// units from the workspace counter.
template <int KMAX, int CMAX, bool BLEND, bool CHAIN>
__global__ void __launch_bounds__(32, 16) traverse_kernel(const WsView v, int persistent) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StageBuf<CMAX>& sb = *reinterpret_cast<StageBuf<CMAX>*>(smem_raw);
  if (!persistent) {
    traverse_unit<KMAX, CMAX, BLEND, CHAIN>(v, blockIdx.x, sb);
    return;
  }
  const int n_units = v.hdr->n_items * kBlocksPerTile;
  for (;;) {
    const int w = next_unit(v);
    if (w >= n_units) {
      done_units(v, w, n_units);
      break;
    }
    traverse_unit<KMAX, CMAX, BLEND, CHAIN>(v, w, sb);
    __syncwarp();
  }
}

template <int KMAX, int CMAX, bool BLEND, bool CHAIN = false>
cudaError_t launch_t(const WsView& v, cudaStream_t st) {
  // staging buffers, then (blending) every lane's reference feature
  const size_t smem = sizeof(StageBuf<CMAX>) + (BLEND ? sizeof(float) * 32 * StageBuf<CMAX>::FS : 0);
  auto kern = traverse_kernel<KMAX, CMAX, BLEND, CHAIN>;
  unsigned grid = (unsigned)v.max_items * kBlocksPerTile;
  if (v.persistent) {
    const unsigned slots = resident_slots(kern, 32, smem);
    if (slots == 0) return cudaErrorLaunchOutOfResources;
    if (slots < grid) grid = slots;
  }
  return launch_pdl(kern, dim3(grid), dim3(32), smem, st, v, v.persistent);
}

template <int KMAX, bool BLEND>
cudaError_t launch_k(const WsView& v, cudaStream_t st) {
  const int C = v.n_channels;
  if constexpr (!BLEND) {
    return launch_t<KMAX, 4, false>(v, st);
  } else {
    // the paper's early termination walks a tile's segments in order
    if (v.chain) {
      if (C <= 4) return launch_t<KMAX, 4, true, true>(v, st);
      if (C <= 8) return launch_t<KMAX, 8, true, true>(v, st);
      if (C <= 16) return launch_t<KMAX, 16, true, true>(v, st);
      return launch_t<KMAX, 32, true, true>(v, st);
    }
    if (C <= 4) return launch_t<KMAX, 4, true>(v, st);
    if (C <= 8) return launch_t<KMAX, 8, true>(v, st);
    if (C <= 16) return launch_t<KMAX, 16, true>(v, st);
    return launch_t<KMAX, 32, true>(v, st);
  }
}

template <bool BLEND>
cudaError_t launch_any(const WsView& v, cudaStream_t st) {
  if (v.max_items == 0) return cudaSuccess;
  const int K = v.n_track;
  if (K <= 8) return launch_k<8, BLEND>(v, st);
  if (K <= 16) return launch_k<16, BLEND>(v, st);
  return launch_k<32, BLEND>(v, st);
}

}  // namespace

cudaError_t launch_render_fwd(const WsView& v, cudaStream_t st) { return launch_any<true>(v, st); }

// Recomputes each pixel's n_track-th tracked hit (the backward pass's
// threshold) by the forward traversal without blending.
cudaError_t launch_track_pass(const WsView& v, cudaStream_t st) { return launch_any<false>(v, st); }

}  // namespace pulsar
