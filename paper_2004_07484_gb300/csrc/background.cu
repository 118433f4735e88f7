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
  const int ny = y1 - y0;
  float* const img0 = S.image + ((int64_t)y0 * S.width + x0) * C;
  const int64_t row = (int64_t)S.width * C;   // floats between pixel rows
  const bool vec = (C & 3) == 0 &&
                   ((reinterpret_cast<uintptr_t>(img0) | reinterpret_cast<uintptr_t>(S.bg)) & 15) == 0 &&
                   (row & 3) == 0;
  // (the per-pixel backward data of the render passes, residuals and the
  // tracked threshold, is never read for an empty tile: the backward pass
  // visits it only through the background-gradient kernel below)
  if (vec) {   // 16-byte stores, consecutive threads on consecutive vectors of a row
    const int c4 = C >> 2, per_row = nx * c4;
    const float4* bg4 = reinterpret_cast<const float4*>(S.bg);
    for (int e = threadIdx.x; e < ny * per_row; e += blockDim.x) {
      const int r = e / per_row, q = e - r * per_row;
      reinterpret_cast<float4*>(img0 + r * row)[q] = bg4[q % c4];
    }
  } else {
    for (int e = threadIdx.x; e < ny * nx * C; e += blockDim.x) {
      const int r = e / (nx * C), f = e - r * (nx * C);
      img0[r * row + f] = S.bg[f % C];
    }
  }
  for (int e = threadIdx.x; e < ny * nx; e += blockDim.x) {
    const int r = e / nx, x = e - r * nx;
    const int64_t p = (int64_t)(y0 + r) * S.width + x0 + x;
    S.log_norm[p] = log_d;
    if (S.n_hits) S.n_hits[p] = 0;
    if (S.n_tests) S.n_tests[p] = 0;
    if (S.tracked)
      for (int k = 0; k < K; ++k) S.tracked[p * K + k] = -1;
  }
}

// Background-gradient partials of an empty tile's 8 x 4 pixel blocks, one
// warp per block as the backward render pass does.  Lanes own channels (or
// channel quads): each step reads the channels of consecutive pixels
// (contiguous in the row-major gradient image), weighted by the pixel's
// background weight, and a warp's per-lane sums are added up per channel
// through shared memory.
__global__ void __launch_bounds__(256) background_bwd_kernel(const WsView v) {
  __shared__ float4 red4[kBlocksPerTile][32];
  const int64_t tile = blockIdx.x;
  const int2 rg = v.ranges[tile];
  if (rg.y > rg.x) return;   // the render passes own this tile
  const int block = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const SceneDev& S = v.scenes[scene_of_tile(v.scenes, v.n_scenes, tile)];
  const PixelCtx pc = pixel_ctx(S, tile, block);
  const WarpRect wr = warp_rect(pc, block);
  const int C = S.n_channels;
  // this lane's pixel weight w_B = e^{eps/gamma} / D
  float wB = 0.0f;
  if (pc.inside) wB = __expf(S.eps * (1.0f / S.gamma) - S.log_norm_in[(int64_t)pc.py * S.width + pc.px]);
  float* dst = v.tile_bg + ((size_t)tile * kBlocksPerTile + block) * C;
  if ((C & 3) == 0 && (reinterpret_cast<uintptr_t>(S.grad_image) & 15) == 0) {
    // lanes own channel quads: 16-byte loads, all of a lane's loads in flight at once
    const int c4 = C >> 2, ppi = 32 / c4;
    const int q = lane % c4, sub = lane / c4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
    for (int p0 = 0; p0 < 32; p0 += ppi) {
      const int p = p0 + sub;
      const float w = __shfl_sync(0xffffffffu, wB, p & 31);
      const int x = wr.x0 + (p & 7), y = wr.y0 + (p >> 3);
      if (sub < ppi && p < 32 && x < S.width && y < S.height) {
        const float4 g = __ldg(reinterpret_cast<const float4*>(S.grad_image + ((int64_t)y * S.width + x) * C) + q);
        acc.x = fmaf(w, g.x, acc.x);
        acc.y = fmaf(w, g.y, acc.y);
        acc.z = fmaf(w, g.z, acc.z);
        acc.w = fmaf(w, g.w, acc.w);
      }
    }
    red4[block][lane] = acc;
    __syncwarp();
    if (lane < c4) {
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int j = 0; j < ppi; ++j) {
        const float4 a = red4[block][j * c4 + lane];
        t.x += a.x;
        t.y += a.y;
        t.z += a.z;
        t.w += a.w;
      }
      reinterpret_cast<float4*>(dst)[lane] = t;
    }
    return;
  }
  // any channel count: lanes own channels
  const int ppi = 32 / C;
  const int ch = lane % C, sub = lane / C;
  float acc = 0.0f;
#pragma unroll 4
  for (int p0 = 0; p0 < 32; p0 += ppi) {
    const int p = p0 + sub;
    const float w = __shfl_sync(0xffffffffu, wB, p & 31);
    const int x = wr.x0 + (p & 7), y = wr.y0 + (p >> 3);
    if (sub < ppi && p < 32 && x < S.width && y < S.height)
      acc = fmaf(w, __ldg(S.grad_image + ((int64_t)y * S.width + x) * C + ch), acc);
  }
  float* red = reinterpret_cast<float*>(red4[block]);
  red[lane] = acc;
  __syncwarp();
  if (lane < C) {
    float x = 0.0f;
    for (int j = 0; j < ppi; ++j) x += red[j * C + lane];
    dst[lane] = x;
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
