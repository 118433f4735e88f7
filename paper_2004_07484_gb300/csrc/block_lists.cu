// Block lists: the last binning stage (App. B, Step 1, "intersection search",
// moved out of the render passes).
//
// For every work unit (one list segment of a tile x one of the tile's eight
// 8 x 4 pixel blocks) a warp walks the segment once and keeps, in list
// order, the spheres the float32 hit predicate reports for at least one
// pixel of the block, each with its 32-bit hit mask (bit 8 y + x for block
// pixel (x, y)).  Each lane takes one list entry: it intersects the sphere's
// pixel rectangle with the block and tests only the pixels of that overlap.
// The forward pass, the track pass and the backward pass then stream only
// these entries and read each pixel's hits from the masks, so none of them
// repeats the rectangle or ray-disc tests.  Per unit and pixel the warp also
// counts the rectangle tests made (the n_tests diagnostic of the forward).
#include "render_common.cuh"

namespace pulsar {

namespace {

__global__ void __launch_bounds__(256) block_lists_kernel(const WsView v, const uint32_t* __restrict__ list) {
  const int item = blockIdx.x;
  const int block = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  ItemCtx it;
  if (!item_ctx_direct(v, item, block, it)) return;
  const SceneDev& S = v.scenes[scene_of_tile(v.scenes, v.n_scenes, it.tile)];
  const PixelCtx pc = pixel_ctx(S, it.tile, it.block);
  const WarpRect wr = warp_rect(pc, it.block);
  uint2* out = v.unit_list + (size_t)it.block * v.capacity + it.b0;
  int n = 0;
  int tests = 0;   // rectangle tests of this lane's pixel
  for (int base = it.b0; base < it.b1; base += 32) {
    const int i = base + lane;
    uint32_t id = 0u, hm = 0u, rm = 0u;
    if (i < it.b1) {
      id = __ldg(list + i);
      const float4 b = __ldg(v.rec1 + id);
      if (rect_overlaps(b, wr)) {
        const float4 a = __ldg(v.rec0 + id);
        const uint32_t bx = __float_as_uint(b.z), by = __float_as_uint(b.w);
        const int x0 = max((int)(bx & 0xffffu), wr.x0), x1 = min((int)(bx >> 16), wr.x1);
        const int y0 = max((int)(by & 0xffffu), wr.y0), y1 = min((int)(by >> 16), wr.y1);
        for (int y = y0; y <= y1; ++y) {
          const float ry = ray_coord(y, S.height, S.kappa);
          for (int x = x0; x <= x1; ++x) {
            const uint32_t bit = 1u << ((y - wr.y0) * 8 + (x - wr.x0));
            rm |= bit;
            if (ray_disc_positive(a.x, a.y, a.z, a.w, ray_coord(x, S.width, S.kappa), ry)) hm |= bit;
          }
        }
      }
    }
    tests += __popc(transpose32(rm));
    const uint32_t bal = __ballot_sync(0xffffffffu, hm != 0u);
    if (hm) out[n + __popc(bal & lane_lt_mask())] = make_uint2(id, hm);
    n += __popc(bal);
  }
  const int unit = item * kBlocksPerTile + it.block;
  if (lane == 0) v.unit_count[unit] = n;
  v.unit_tests[(size_t)unit * 32 + lane] = tests;
}

}  // namespace

cudaError_t launch_block_lists(const WsView& v, cudaStream_t st) {
  if (v.max_items == 0) return cudaSuccess;
  block_lists_kernel<<<(unsigned)v.max_items, 256, 0, st>>>(v, v.pval[v.pair_buf]);
  return cudaGetLastError();
}

}  // namespace pulsar
