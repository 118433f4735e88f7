// Block lists: the last binning stage (App. B, Step 1, "intersection search",
// moved out of the render passes).
//
// For every work unit (one list segment of a tile x one of the tile's eight
// 8 x 4 pixel blocks) a warp walks the segment once and keeps, in list
// order, the spheres the float32 hit predicate reports for at least one
// pixel of the block, each with its 32-bit hit mask (bit 8 y + x for block
// pixel (x, y)).  The warp reads the segment's pair keys, whose high bits
// say which of the tile's blocks each sphere's rectangle meets, and gathers
// the entries meeting its block into batches of 32; per batch each lane
// intersects one sphere's rectangle with the block, and the pixel tests of
// all overlaps (a few per sphere, very unevenly) are numbered across the warp
// and spread evenly over the lanes, which OR their results into the entries'
// masks in shared memory.  The forward pass, the track pass and the backward pass then
// stream only these entries and read each pixel's hits from the masks, so
// none of them repeats the rectangle or ray-disc tests.
#include "render_common.cuh"

namespace pulsar {

namespace {

// Per warp: sphere indices of the entries whose rectangle meets the warp's block,
// gathered into full batches, and the current batch's test bookkeeping.
struct BlockListWarp {
  uint32_t pos[64];    // gathered sphere indices, in list order
  float4 rec0[32];     // draw record (decision centre, R^2)
  int first[32];       // first test number of each entry
  uint32_t geom[32];   // overlap with the block: x0 | y0 << 8 | width << 16
  uint32_t wdiv[32];   // ceil(2^16 / width): test index / width = (index * wdiv) >> 16
  uint32_t hm[32];     // hit masks being built
  uint8_t owner[1024]; // entry of each test number of the batch
};

// Tests the pixels of the first cnt gathered entries against the block and
// appends the entries with hits, in order, to out (n entries so far).
__device__ __forceinline__ void block_batch(BlockListWarp& W, int cnt, const WsView& v, const SceneDev& S,
                                            const WarpRect& wr, uint2* out, int& n, uint32_t& hits) {
  const int lane = threadIdx.x & 31;
  uint32_t id = 0u;
  int ntest = 0;
  if (lane < cnt) {
    id = W.pos[lane];
    const float4 b = __ldg(v.rec1 + id);
    const uint32_t bx = __float_as_uint(b.z), by = __float_as_uint(b.w);
    const int x0 = max((int)(bx & 0xffffu), wr.x0), x1 = min((int)(bx >> 16), wr.x1);
    const int y0 = max((int)(by & 0xffffu), wr.y0), y1 = min((int)(by >> 16), wr.y1);
    const int w = max(x1 - x0 + 1, 1);
    ntest = (x1 >= x0 && y1 >= y0) ? w * (y1 - y0 + 1) : 0;   // the pair key says they meet
    W.rec0[lane] = __ldg(v.rec0 + id);
    W.geom[lane] = (uint32_t)(x0 - wr.x0) | ((uint32_t)(y0 - wr.y0) << 8) | ((uint32_t)w << 16);
    W.wdiv[lane] = (65536u + (uint32_t)w - 1u) / (uint32_t)w;
  }
  int total;
  const int first = warp_exclusive_scan(ntest, total);
  W.first[lane] = first;
  W.hm[lane] = 0u;
  for (int k = 0; k < ntest; ++k) W.owner[first + k] = (uint8_t)lane;
  __syncwarp();
  // the batch's pixel tests, spread evenly over the lanes
  for (int k = lane; k < total; k += 32) {
    const int e = W.owner[k];
    const uint32_t r = (uint32_t)(k - W.first[e]);
    const uint32_t g = W.geom[e];
    const uint32_t dy = (r * W.wdiv[e]) >> 16;
    const uint32_t dx = r - dy * (g >> 16);
    const int px = (int)(g & 0xffu) + (int)dx, py = (int)((g >> 8) & 0xffu) + (int)dy;
    const float4 a = W.rec0[e];
    if (pixel_disc_positive(a, ray_coord(wr.x0 + px, S.width, S.kappa), ray_coord(wr.y0 + py, S.height, S.kappa),
                            (S.flags & PULSAR_FLAG_ORTHOGRAPHIC) != 0))
      atomicOr(&W.hm[e], 1u << (py * 8 + px));
  }
  __syncwarp();
  const uint32_t hm = W.hm[lane];
  const uint32_t bal = __ballot_sync(0xffffffffu, hm != 0u);
  if (hm) out[n + __popc(bal & lane_lt_mask())] = make_uint2(id, hm);
  n += __popc(bal);
  hits += __popc(hm);
  __syncwarp();   // the batch's shared data is rewritten next
}

// Two warps (two pixel blocks of one item) per CTA: a CTA's warps finish at
// different times, and smaller CTAs hand their slot back sooner.
constexpr int kListWarps = 2;

__global__ void __launch_bounds__(32 * kListWarps) block_lists_kernel(const WsView v,
                                                                       const uint32_t* __restrict__ keys,
                                                                       const uint32_t* __restrict__ list) {
  pdl_wait();
  pdl_trigger();
  __shared__ BlockListWarp warps[kListWarps];
  constexpr int kCtasPerItem = kBlocksPerTile / kListWarps;
  const int rank = blockIdx.x / kCtasPerItem;   // longest items first
  if (rank >= v.hdr->n_items) return;
  const int item = v.item_order[rank];
  const int block = (blockIdx.x % kCtasPerItem) * kListWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  BlockListWarp& W = warps[threadIdx.x >> 5];
  ItemCtx it;
  if (!item_ctx_direct(v, item, block, it)) return;
  const SceneDev& S = v.scenes[it.scene];
  const PixelCtx pc = pixel_ctx(S, it.tile, it.block);
  const WarpRect wr = warp_rect(pc, it.block);
  uint2* out = v.unit_list + (size_t)it.block * v.capacity + it.b0;
  const uint32_t mine = 1u << (kTileKeyBits + block);
  int n = 0, pending = 0;
  uint32_t hits = 0u;   // this lane's share of the unit's pixel hits
  // the pair keys and sphere indices of the next 32 entries load while the current ones are used
  uint32_t key_next = it.b0 + lane < it.b1 ? __ldg(keys + it.b0 + lane) : 0u;
  uint32_t id_next = it.b0 + lane < it.b1 ? __ldg(list + it.b0 + lane) : 0u;
  for (int base = it.b0; base < it.b1; base += 32) {
    const uint32_t key = key_next, id = id_next;
    key_next = base + 32 + lane < it.b1 ? __ldg(keys + base + 32 + lane) : 0u;
    id_next = base + 32 + lane < it.b1 ? __ldg(list + base + 32 + lane) : 0u;
    // gather the entries whose rectangle meets this block (from the pair key)
    const bool ok = base + lane < it.b1 && (key & mine) != 0u;
    const uint32_t bal = __ballot_sync(0xffffffffu, ok);
    if (ok) W.pos[pending + __popc(bal & lane_lt_mask())] = id;
    pending += __popc(bal);
    if (pending >= 32) {
      __syncwarp();
      block_batch(W, 32, v, S, wr, out, n, hits);
      const int rest = pending - 32;
      if (lane < rest) W.pos[lane] = W.pos[32 + lane];
      pending = rest;
      __syncwarp();
    }
  }
  if (pending > 0) {
    __syncwarp();
    block_batch(W, pending, v, S, wr, out, n, hits);
  }
  hits = __reduce_add_sync(0xffffffffu, hits);
  if (lane == 0) {
    v.unit_count[item * kBlocksPerTile + it.block] = n;
    v.unit_cost[item * kBlocksPerTile + it.block] = (uint32_t)n + hits;
  }
}

// Launch order of the render passes' work units: decreasing cost (block-list
// length plus pixel hits), by a counting sort over kCostClasses logarithmic
// cost classes (four per octave; the order within a class is arbitrary).
constexpr int kCostClasses = 64;

__device__ __forceinline__ int cost_class(uint32_t c) {
  if (c < 4u) return kCostClasses - 1 - (int)c;
  const int lg = 31 - __clz(c);                            // >= 2
  const int cls = 4 * lg - 4 + (int)((c >> (lg - 2)) & 3u);  // 4 .. 4 * 31 - 1
  return max(kCostClasses - 1 - cls, 0);
}

// Cost of unit u as the render passes see it: with a chained walk the first
// segment's unit renders all segments of its tile and the others none.
__device__ __forceinline__ uint32_t walk_cost(const WsView& v, uint32_t u) {
  if (!v.chain) return v.unit_cost[u];
  const ItemDesc d = v.item_desc[u / kBlocksPerTile];
  if (d.seg != 0) return 0u;
  uint32_t c = 0;
  for (int k = d.first; k < d.first + d.nseg; ++k) c += v.unit_cost[k * kBlocksPerTile + u % kBlocksPerTile];
  return c;
}

__global__ void __launch_bounds__(1024) order_units_kernel(const WsView v) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t bucket[kCostClasses];
  const uint32_t n = (uint32_t)v.hdr->n_items * kBlocksPerTile;
  if (threadIdx.x < kCostClasses) bucket[threadIdx.x] = 0u;
  __syncthreads();
  for (uint32_t u = threadIdx.x; u < n; u += 1024) atomicAdd(&bucket[cost_class(walk_cost(v, u))], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int b = 0; b < kCostClasses; ++b) {
      const uint32_t c = bucket[b];
      bucket[b] = run;
      run += c;
    }
  }
  __syncthreads();
  for (uint32_t u = threadIdx.x; u < n; u += 1024)
    v.unit_order[atomicAdd(&bucket[cost_class(walk_cost(v, u))], 1u)] = (int32_t)u;
}

// The n_tests diagnostic: per work unit and pixel, the spheres of the
// segment whose rectangle contains the pixel (the tests the block lists
// made), counted through a warp bit-matrix transpose.  Run only when a
// forward pass asks for n_tests.
__global__ void __launch_bounds__(256) count_tests_kernel(const WsView v, const uint32_t* __restrict__ list) {
  pdl_wait();
  pdl_trigger();
  const int item = blockIdx.x;
  const int lane = threadIdx.x & 31;
  ItemCtx it;
  if (!item_ctx_direct(v, item, threadIdx.x >> 5, it)) return;
  const SceneDev& S = v.scenes[it.scene];
  const WarpRect wr = warp_rect(pixel_ctx(S, it.tile, it.block), it.block);
  int tests = 0;
  for (int base = it.b0; base < it.b1; base += 32) {
    const int i = base + lane;
    uint32_t rm = 0u;
    if (i < it.b1) {
      const float4 b = __ldg(v.rec1 + __ldg(list + i));
      if (rect_overlaps(b, wr)) {
        const uint32_t bx = __float_as_uint(b.z), by = __float_as_uint(b.w);
        const int x0 = max((int)(bx & 0xffffu), wr.x0), x1 = min((int)(bx >> 16), wr.x1);
        const int y0 = max((int)(by & 0xffffu), wr.y0), y1 = min((int)(by >> 16), wr.y1);
        const uint32_t row = ((2u << (x1 - wr.x0)) - (1u << (x0 - wr.x0)));
        for (int y = y0; y <= y1; ++y) rm |= row << ((y - wr.y0) * 8);
      }
    }
    tests += __popc(transpose32(rm));
  }
  v.unit_tests[((size_t)item * kBlocksPerTile + it.block) * 32 + lane] = tests;
}

}  // namespace

cudaError_t launch_block_lists(const WsView& v, cudaStream_t st) {
  if (v.max_items == 0) return cudaSuccess;
  cudaError_t e = launch_pdl(block_lists_kernel, dim3((unsigned)v.max_items * (kBlocksPerTile / kListWarps)),
                             dim3(32 * kListWarps), 0, st, v, v.pkey[v.pair_buf], v.pval[v.pair_buf]);
  if (e != cudaSuccess) return e;
  return launch_pdl(order_units_kernel, dim3(1), dim3(1024), 0, st, v);
}

cudaError_t launch_count_tests(const WsView& v, cudaStream_t st) {
  if (v.max_items == 0) return cudaSuccess;
  return launch_pdl(count_tests_kernel, dim3((unsigned)v.max_items), dim3(256), 0, st, v, v.pval[v.pair_buf]);
}

}  // namespace pulsar
