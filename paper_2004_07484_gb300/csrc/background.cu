// Pixels of tiles that no sphere's rectangle overlaps.  Their Eq. 1 has the
// background term alone: F = bg, D = e^{eps/gamma} (log D = eps / gamma), no
// tracked hits, and every pixel's background weight is w_B = 1.  The binning
// pass gives such tiles no work items, so the render passes never visit them;
// this pass writes their forward outputs (coalesced, row by row) and, in the
// backward pass, their share of dL/dbg, with one warp per 8 x 4 pixel block
// as the render passes use, so the background-gradient partials of all tiles
// sum alike.
#include "render_common.cuh"

namespace pulsar {

namespace {

// Forward outputs of an empty tile, one CTA per tile: every pixel row of the
// tile is a contiguous run of the row-major outputs, written with consecutive
// threads on consecutive elements.
__global__ void __launch_bounds__(256) background_fwd_kernel(const WsView v) {
  const int64_t tile = blockIdx.x;
  const int2 rg = v.ranges[tile];
  if (rg.y > rg.x) return;   // the render passes own this tile
  const SceneDev& S = v.scenes[scene_of_tile(v.scenes, v.n_scenes, tile)];
  const int64_t lt = tile - S.tile_begin;
  const int ty = (int)(lt / S.tiles_x), tx = (int)(lt - (int64_t)ty * S.tiles_x);
  const int x0 = tx * kTile, x1 = min(x0 + kTile, S.width);
  const int y0 = ty * kTile, y1 = min(y0 + kTile, S.height);
  const int C = S.n_channels, K = S.n_track, nx = x1 - x0;
  const float log_d = S.eps * (1.0f / S.gamma) + __logf(1.0f);
  const float4 aux = make_float4(__int_as_float(0x7f800000), __int_as_float(0x7fffffff), __int_as_float(-1), 0.0f);
  for (int y = y0; y < y1; ++y) {
    const int64_t p0 = (int64_t)y * S.width + x0;   // first pixel of the row run
    float* img = S.image + p0 * C;
    float* fr = v.fres + (S.pixel_begin + p0) * C;
    for (int f = threadIdx.x; f < nx * C; f += blockDim.x) {
      img[f] = S.bg[f % C];
      fr[f] = 0.0f;
    }
    if (S.tracked) {
      int32_t* tr = S.tracked + p0 * K;
      for (int f = threadIdx.x; f < nx * K; f += blockDim.x) tr[f] = -1;
    }
    if ((int)threadIdx.x < nx) {
      const int64_t p = p0 + threadIdx.x;
      S.log_norm[p] = log_d;
      if (S.n_hits) S.n_hits[p] = 0;
      if (S.n_tests) S.n_tests[p] = 0;
      v.pix_aux[S.pixel_begin + p] = aux;
    }
  }
}

// Background-gradient partials of an empty tile's 8 x 4 pixel blocks, one
// warp per block as the backward render pass does.
__global__ void __launch_bounds__(256) background_bwd_kernel(const WsView v) {
  const int64_t tile = blockIdx.x;
  const int2 rg = v.ranges[tile];
  if (rg.y > rg.x) return;   // the render passes own this tile
  const int block = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const SceneDev& S = v.scenes[scene_of_tile(v.scenes, v.n_scenes, tile)];
  const PixelCtx pc = pixel_ctx(S, tile, block);
  const int C = S.n_channels;
  const int64_t pix = (int64_t)pc.py * S.width + pc.px;
  float wB = 0.0f;
  const float* g = S.grad_image;
  if (pc.inside) {
    wB = __expf(S.eps * (1.0f / S.gamma) - S.log_norm_in[pix]);
    g += pix * C;
  }
  float* dst = v.tile_bg + ((size_t)tile * kBlocksPerTile + block) * C;
  for (int c = 0; c < C; ++c) {
    float y = 0.0f;
    if (pc.inside) y = wB * g[c];
    const float x = warp_sum(y);
    if (lane == 0) dst[c] = x;
  }
}

}  // namespace

cudaError_t launch_background(const WsView& v, bool backward, uint32_t grad_mask, cudaStream_t st) {
  if (v.n_tiles == 0) return cudaSuccess;
  if (backward) {
    if (grad_mask & PULSAR_GRAD_BG) background_bwd_kernel<<<(unsigned)v.n_tiles, 256, 0, st>>>(v);
  } else {
    background_fwd_kernel<<<(unsigned)v.n_tiles, 256, 0, st>>>(v);
  }
  return cudaGetLastError();
}

}  // namespace pulsar
