// Pixels of tiles that no sphere's rectangle overlaps.  Their Eq. 1 has the
// background term alone: F = bg, D = e^{eps/gamma} (log D = eps / gamma), no
// tracked hits, and every pixel's background weight is w_B = 1.  The binning
// pass gives such tiles no work items, so the render passes never visit them;
// this pass writes their forward outputs and, in the backward pass, their
// per-block dL/dbg partials (the layout the render passes use), reading and
// writing each pixel row of a tile as one contiguous run.
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

// Background-gradient partials of an empty tile's eight 8 x 4 pixel blocks,
// one CTA per tile: the upstream gradient is read row by row as contiguous
// runs, each thread sums w_B G of one (pixel column, channel) over the four
// rows of a block row, and shared-memory atomics gather the block sums.
__global__ void __launch_bounds__(256) background_bwd_kernel(const WsView v) {
  __shared__ float acc[kBlocksPerTile * 32];
  __shared__ float wb[kTile];
  const int64_t tile = blockIdx.x;
  const int2 rg = v.ranges[tile];
  if (rg.y > rg.x) return;   // the render passes own this tile
  const SceneDev& S = v.scenes[scene_of_tile(v.scenes, v.n_scenes, tile)];
  const int64_t lt = tile - S.tile_begin;
  const int ty = (int)(lt / S.tiles_x), tx = (int)(lt - (int64_t)ty * S.tiles_x);
  const int x0 = tx * kTile, nx = min(kTile, S.width - x0);
  const int y0 = ty * kTile, ny = min(kTile, S.height - y0);
  const int C = S.n_channels;
  const float inv_gamma = 1.0f / S.gamma;
  for (int e = threadIdx.x; e < kBlocksPerTile * C; e += blockDim.x) acc[e] = 0.0f;
  for (int br = 0; br < 4; ++br) {   // block rows of the tile
    float sum[2] = {0.0f, 0.0f};     // this thread's elements f and f + 256 of each row
    for (int r = 4 * br; r < min(4 * br + 4, ny); ++r) {
      const int64_t p0 = (int64_t)(y0 + r) * S.width + x0;
      __syncthreads();
      if ((int)threadIdx.x < nx) wb[threadIdx.x] = __expf(S.eps * inv_gamma - S.log_norm_in[p0 + threadIdx.x]);
      __syncthreads();
      const float* g = S.grad_image + p0 * C;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int f = threadIdx.x + 256 * h;
        if (f < nx * C) sum[h] = fmaf(wb[f / C], g[f], sum[h]);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int f = threadIdx.x + 256 * h;
      if (f < nx * C) {
        const int x = f / C, c = f - x * C;
        atomicAdd(&acc[(br * 2 + (x >> 3)) * C + c], sum[h]);
      }
    }
  }
  __syncthreads();
  float* dst = v.tile_bg + (size_t)tile * kBlocksPerTile * C;
  for (int e = threadIdx.x; e < kBlocksPerTile * C; e += blockDim.x) dst[e] = acc[e];
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
