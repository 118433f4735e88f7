// Forward pass: App. B, Step 1 (intersection search) and Step 2 (draw).
//
// Per pixel, hits are blended by Eq. 1 in the order of the tile's list, with a
// running maximum of the exponents o z / gamma divided out of numerator and
// denominator (the online form of the weighted softmax), and the n_track
// closest hits are kept in a register queue (App. B, Step 2).
//
// Early termination (Sec. 3.2, App. B Step 2) in an exact form: a pixel stops
// at the first listed sphere whose key (earliest depth) is
//   (i)  beyond the depth of its n_track-th tracked hit, so no later sphere
//        can enter the tracked set (every hit depth is >= its sphere's key), and
//   (ii) so far that the largest total weight all remaining spheres could
//        still add, N_rem |o|max exp(|o|max z(key) / gamma), is at most 1e-7 of
//        the current denominator.
// A CTA stops once every pixel has stopped (a barrier vote over all threads).
#include "render_common.cuh"

namespace pulsar {

namespace {

template <int KMAX, int CMAX>
__global__ void __launch_bounds__(kThreads, 2) render_fwd_kernel(const WsView v,
                                                                 const uint32_t* __restrict__ list,
                                                                 int store) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ChunkSmem<CMAX>& sm = *reinterpret_cast<ChunkSmem<CMAX>*>(smem_raw);
  const int64_t tile = blockIdx.x;
  const int si = scene_of_tile(v.scenes, v.n_scenes, tile);
  const SceneDev& S = v.scenes[si];
  const PixelCtx pc = pixel_ctx(S, tile);
  const int2 rg = v.ranges[tile];
  const int C = S.n_channels;
  const int K = S.n_track;
  const float gamma = S.gamma, zfar = S.zfar, znear = S.znear;
  const float inv_gamma = 1.0f / gamma;
  const float range = zfar - znear, inv_range = 1.0f / range;
  const float omax = __uint_as_float(S.omax_bits);
  const bool literal = (S.flags & PULSAR_FLAG_DIST_LITERAL) != 0;

  for (int e = threadIdx.x; e < kChunk * CMAX; e += kThreads) sm.feat[e] = 0.0f;

  // Eq. 1 state, scaled by e^{-m}: m = running maximum exponent (starting with
  // the background's eps / gamma), den = e^{eps/g - m} + sum a_k e^{-m}.
  float m = S.eps * inv_gamma;
  float den = 1.0f;
  float acc[CMAX];
#pragma unroll
  for (int c = 0; c < CMAX; ++c) acc[c] = c < C ? S.bg[c] : 0.0f;
  float qt[KMAX];
  int qi[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    qt[k] = __int_as_float(0x7f800000);
    qi[k] = 0x7fffffff;
  }
  float thr_t = __int_as_float(0x7f800000);
  int thr_i = 0x7fffffff;
  int nhit = 0, ntest = 0;
  bool done = !pc.inside;
  float kstop1 = __int_as_float(0x7f800000);   // tracked-set bound (i)
  float kstop = kstop1;
  const int warp = threadIdx.x >> 5;

  for (int base = rg.x; base < rg.y; base += kChunk) {
    const int n = min(kChunk, rg.y - base);
    // remaining-mass bound (ii), from the state at the start of this chunk
    float kstop2 = -__int_as_float(0x7f800000);
    if (!done && omax > 0.0f) {
      const float lr = m + __logf(1e-7f * den / ((float)(rg.y - base) * omax));
      const float zthr = lr * gamma / omax;
      kstop2 = zthr >= 1.0f ? -__int_as_float(0x7f800000) : zfar - range * zthr;
    }
    kstop = fmaxf(kstop1, kstop2);
    const int cnt = stage_chunk<CMAX>(sm, v, S, list, base, n, pc, true);
    for (int k = 0; k < cnt; ++k) {
      if (__all_sync(0xffffffffu, done)) break;
      const int j = sm.list[warp][k];
      const float4 a = sm.rec0[j];
      const float4 b = sm.rec1[j];
      if (done) continue;
      if (b.x >= kstop) {
        done = true;
        continue;
      }
      if (!in_rect(b, pc.px, pc.py)) continue;
      ++ntest;
      RayHit h;
      if (!ray_hit(a.x, a.y, a.z, a.w, b.x, pc.rx, pc.ry, zfar, h)) continue;
      ++nhit;
      // value path
      const float4 c2 = sm.rec2[j];
      const ValueGeom vg = value_geom(a, c2, pc.vr);
      const float qd = fminf(vg.dist / c2.w, 1.0f);
      const float d = literal ? qd : 1.0f - qd;
      const float z = (((zfar - a.z) - c2.z) + vg.off) * inv_range;
      const float o = b.y;
      if (o * d != 0.0f) {   // a zero weight adds nothing and must not move the shift
        const float s = o * z * inv_gamma;
        if (s > m) {
          const float sc = __expf(m - s);
          den *= sc;
#pragma unroll
          for (int c = 0; c < CMAX; ++c) acc[c] *= sc;
          m = s;
        }
        const float w = o * d * __expf(s - m);
        den += w;
        const float* f = &sm.feat[j * CMAX];
#pragma unroll
        for (int c = 0; c < CMAX; ++c) acc[c] = fmaf(w, f[c], acc[c]);
      }
      const int id = sm.id[j];
      if (hit_less(h.t, id, thr_t, thr_i)) {
        queue_insert<KMAX>(qt, qi, h.t, id);
        queue_select<KMAX>(qt, qi, K, thr_t, thr_i);
        kstop1 = next_up(thr_t);
        kstop = fmaxf(kstop1, kstop2);
      }
    }
    if (__syncthreads_and(done)) break;
  }

  if (!pc.inside) return;
  const int64_t pix = (int64_t)pc.py * S.width + pc.px;
  const float inv = 1.0f / den;
  float* out = S.image + pix * C;
#pragma unroll
  for (int c = 0; c < CMAX; ++c)
    if (c < C) out[c] = acc[c] * inv;
  S.log_norm[pix] = m + __logf(den);
  if (S.n_hits) S.n_hits[pix] = nhit;
  if (S.n_tests) S.n_tests[pix] = ntest;
  if (S.tracked) {
    int32_t* tr = S.tracked + pix * K;
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
      if (k < K) tr[k] = qi[k] == 0x7fffffff ? -1 : (int32_t)(qi[k] - S.sphere_begin);
  }
  if (store) v.thr[S.pixel_begin + pix] = make_float2(thr_t, __int_as_float(thr_i));
}

template <int KMAX, int CMAX>
cudaError_t launch_fwd_t(const WsView& v, const uint32_t* list, bool store, cudaStream_t st) {
  const size_t smem = sizeof(ChunkSmem<CMAX>);
  auto kern = render_fwd_kernel<KMAX, CMAX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)v.n_tiles, kThreads, smem, st>>>(v, list, store ? 1 : 0);
  return cudaGetLastError();
}

template <int KMAX>
cudaError_t launch_fwd_k(const WsView& v, const uint32_t* list, bool store, cudaStream_t st) {
  const int C = v.n_channels;
  if (C <= 4) return launch_fwd_t<KMAX, 4>(v, list, store, st);
  if (C <= 8) return launch_fwd_t<KMAX, 8>(v, list, store, st);
  if (C <= 16) return launch_fwd_t<KMAX, 16>(v, list, store, st);
  return launch_fwd_t<KMAX, 32>(v, list, store, st);
}

}  // namespace

cudaError_t launch_render_fwd(const WsView& v, bool store, cudaStream_t st) {
  if (v.n_tiles == 0) return cudaSuccess;
  const uint32_t* list = v.pval[v.pair_buf];
  const int K = v.n_track;
  if (K <= 8) return launch_fwd_k<8>(v, list, store, st);
  if (K <= 16) return launch_fwd_k<16>(v, list, store, st);
  return launch_fwd_k<32>(v, list, store, st);
}

}  // namespace pulsar
