// Tile traversal shared by the forward and backward render kernels.
//
// One CTA renders one 16 x 16 screen tile; each warp owns an 8 x 4 pixel
// block and each thread one pixel, so parallelism is over pixels as the paper
// prescribes (Sec. 3.2, App. B).  The tile's depth-ordered sphere list is
// streamed in chunks of 256 spheres: each thread stages one draw record, the
// CTA stages the feature vectors, and every warp compacts the staged spheres
// whose rectangles overlap its pixel block with a ballot + popcount scan
// (App. B, Step 1: block-wise intersection search with cooperative filtering).
#pragma once

#include "pulsar_internal.cuh"

namespace pulsar {

__device__ __forceinline__ unsigned lane_lt_mask() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Shared-memory layout of one chunk.
template <int CMAX>
struct ChunkSmem {
  float4 rec0[kChunk];
  float4 rec1[kChunk];
  float4 rec2[kChunk];
  float feat[kChunk * CMAX];
  int32_t id[kChunk];
  uint8_t mask[kChunk];
  uint8_t list[kThreads / 32][kChunk];
};

// One work item: a segment of at most `segment` entries of one tile's list.
struct ItemCtx {
  int item;          // work-item index (also the partial-state slot)
  int64_t tile;      // global tile index
  int seg, nseg;     // segment index and segment count of the tile
  int first;         // first work item of the tile
  int b0, b1;        // list range [b0, b1) of this segment
};

// Returns false for grid slots beyond the number of work items.
__device__ __forceinline__ bool item_ctx(const WsView& v, ItemCtx& c) {
  c.item = blockIdx.x;
  if (c.item >= v.hdr->n_items) return false;
  c.tile = v.item_tile[c.item];
  c.first = v.item_begin[c.tile];
  c.nseg = v.item_begin[c.tile + 1] - c.first;
  c.seg = c.item - c.first;
  const int2 rg = v.ranges[c.tile];
  c.b0 = rg.x + c.seg * v.segment;
  c.b1 = min(rg.x + (c.seg + 1) * v.segment, rg.y);
  if (c.b1 < c.b0) c.b1 = c.b0;
  return true;
}

// Geometry of the pixel a thread renders.
struct PixelCtx {
  int tile_x0, tile_y0;   // first pixel of the tile
  int px, py;             // pixel coordinates
  bool inside;            // pixel lies inside the image
  float rx, ry;           // ray slopes (float32 decision values)
  ValueRay vr;            // ray slopes for the value path
};

__device__ __forceinline__ PixelCtx pixel_ctx(const SceneDev& S, int64_t tile) {
  PixelCtx c;
  const int64_t lt = tile - S.tile_begin;
  const int ty = (int)(lt / S.tiles_x), tx = (int)(lt - (int64_t)ty * S.tiles_x);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  c.tile_x0 = tx * kTile;
  c.tile_y0 = ty * kTile;
  c.px = c.tile_x0 + (warp & 1) * 8 + (lane & 7);
  c.py = c.tile_y0 + (warp >> 1) * 4 + (lane >> 3);
  c.inside = c.px < S.width && c.py < S.height;
  c.rx = ray_coord(c.px, S.width, S.kappa);
  c.ry = ray_coord(c.py, S.height, S.kappa);
  c.vr = value_ray(c.px, c.py, S.width, S.height, S.kappa_hi, S.kappa_lo);
  return c;
}

// Stages list[base, base + n) into shared memory and builds every warp's
// compacted list.  Returns this warp's list length.  Ends with a CTA barrier.
template <int CMAX>
__device__ __forceinline__ int stage_chunk(ChunkSmem<CMAX>& sm, const WsView& v, const SceneDev& S,
                                           const uint32_t* __restrict__ list, int base, int n,
                                           const PixelCtx& pc, bool need_feat) {
  const int tid = threadIdx.x;
  __syncthreads();   // the previous chunk is no longer read
  if (tid < n) {
    const uint32_t id = list[base + tid];
    const float4 a = v.rec0[id];
    const float4 b = v.rec1[id];
    sm.id[tid] = (int32_t)id;
    sm.rec0[tid] = a;
    sm.rec1[tid] = b;
    sm.rec2[tid] = v.rec2[id];
    const uint32_t bx = __float_as_uint(b.z), by = __float_as_uint(b.w);
    const int x0 = (int)(bx & 0xffffu), x1 = (int)(bx >> 16);
    const int y0 = (int)(by & 0xffffu), y1 = (int)(by >> 16);
    uint32_t cm = 0u;
    if (x0 <= pc.tile_x0 + 7 && x1 >= pc.tile_x0) cm |= 1u;
    if (x0 <= pc.tile_x0 + 15 && x1 >= pc.tile_x0 + 8) cm |= 2u;
    uint32_t m = 0u;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int ya = pc.tile_y0 + 4 * r;
      if (y0 <= ya + 3 && y1 >= ya) m |= cm << (2 * r);
    }
    sm.mask[tid] = (uint8_t)m;
  }
  __syncthreads();
  if (need_feat) {
    const int C = S.n_channels;
    const float* __restrict__ feat = S.feat;
    const int64_t sb = S.sphere_begin;
    for (int e = tid; e < n * C; e += kThreads) {
      const int s = e / C, c = e - s * C;
      sm.feat[s * CMAX + c] = __ldg(feat + (int64_t)(sm.id[s] - sb) * C + c);
    }
  }
  const int warp = tid >> 5, lane = tid & 31;
  int cnt = 0;
  for (int g = 0; g < n; g += 32) {
    const int j = g + lane;
    const bool f = j < n && ((sm.mask[j] >> warp) & 1u);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (f) sm.list[warp][cnt + __popc(bal & lane_lt_mask())] = (uint8_t)j;
    cnt += __popc(bal);
  }
  __syncthreads();
  return cnt;
}

__device__ __forceinline__ bool in_rect(const float4& b, int px, int py) {
  const uint32_t bx = __float_as_uint(b.z), by = __float_as_uint(b.w);
  return px >= (int)(bx & 0xffffu) && px <= (int)(bx >> 16) && py >= (int)(by & 0xffffu) &&
         py <= (int)(by >> 16);
}

// (t, id) ordering of tracked hits: by depth, then by sphere index.
__device__ __forceinline__ bool hit_less(float t, int id, float qt, int qi) {
  return t < qt || (t == qt && id < qi);
}

// Sorted insertion into the register queue of the KMAX closest hits.  Every
// index is a compile-time constant so the queue stays in registers.
template <int KMAX>
__device__ __forceinline__ void queue_insert(float (&qt)[KMAX], int (&qi)[KMAX], float t, int id) {
  bool lt[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) lt[k] = hit_less(t, id, qt[k], qi[k]);
#pragma unroll
  for (int k = KMAX - 1; k >= 1; --k) {
    const float pt = qt[k - 1];
    const int pi = qi[k - 1];
    qt[k] = lt[k - 1] ? pt : (lt[k] ? t : qt[k]);
    qi[k] = lt[k - 1] ? pi : (lt[k] ? id : qi[k]);
  }
  qt[0] = lt[0] ? t : qt[0];
  qi[0] = lt[0] ? id : qi[0];
}

// The K-th entry (runtime K <= KMAX) as a bitwise one-hot select: a chain of
// conditional moves on k == K - 1 is turned into an indexed local-memory load
// by the compiler, which would move the whole queue out of registers.
template <int KMAX>
__device__ __forceinline__ void queue_select(const float (&qt)[KMAX], const int (&qi)[KMAX], int K,
                                             float& t, int& id) {
  uint32_t tb = 0u, ib = 0u;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const uint32_t m = 0u - (uint32_t)(k == K - 1);
    tb |= m & __float_as_uint(qt[k]);
    ib |= m & (uint32_t)qi[k];
  }
  t = __uint_as_float(tb);
  id = (int)ib;
}

// Next float after a positive depth (+inf stays +inf): spheres whose key is
// at or beyond this value can no longer enter a full tracked set, because
// every hit depth is at least the sphere's key.
__device__ __forceinline__ float next_up(float t) {
  return t < __int_as_float(0x7f800000) ? __uint_as_float(__float_as_uint(t) + 1u) : t;
}

}  // namespace pulsar
