// Tile traversal shared by the forward and backward render kernels.
//
// A 16 x 16 screen tile is rendered as eight 8 x 4 pixel blocks, one warp
// each, and each thread renders one pixel, so parallelism is over pixels as
// the paper prescribes (Sec. 3.2, App. B).  Every warp is its own CTA and
// walks the block list of one segment of its tile's depth-ordered sphere
// list (built by the binning pass: the spheres that hit at least one of the
// block's pixels, each with its 32-bit hit mask; App. B, Step 1's
// intersection search done once for all passes): it stages 32 entries at a
// time in shared memory with their draw records, value records and features,
// and each lane walks the entries that hit its pixel.  A warp with few
// entries never waits for a busy neighbour and frees its slot as soon as it
// is done.
#pragma once

#include "pulsar_internal.cuh"

namespace pulsar {

__device__ __forceinline__ unsigned lane_lt_mask() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

constexpr int kBlocksPerTile = 8;   // 8 x 4 pixel blocks (warps) per 16 x 16 tile

// One work item: a segment of at most `segment` entries of one tile's list;
// each of its eight pixel blocks is a separate one-warp CTA.  CTAs take the
// items longest first (the binning pass orders them), so the hardware's
// in-order CTA dispatch schedules the longest segments earliest and the
// launch does not end on a long segment started last.
struct ItemCtx {
  int item;          // work-item index
  int block;         // pixel block of the tile (0..7)
  int slot;          // item * 8 + block: partial-state and partial-sum slot
  int64_t tile;      // global tile index
  int seg, nseg;     // segment index and segment count of the tile
  int first;         // first work item of the tile
  int b0, b1;        // list range [b0, b1) of this segment
  int scene;         // scene owning the tile
};

// Work item `item` itself and its pixel block `block` (0..7).  Returns false
// for items beyond the number of work items.
__device__ __forceinline__ bool item_ctx_direct(const WsView& v, int item, int block, ItemCtx& c) {
  if (item >= v.hdr->n_items) return false;
  const ItemDesc d = v.item_desc[item];
  c.item = item;
  c.block = block;
  c.slot = item * kBlocksPerTile + block;
  c.tile = d.tile;
  c.first = d.first;
  c.nseg = d.nseg;
  c.seg = d.seg;
  c.b0 = d.b0;
  c.b1 = d.b1;
  c.scene = d.scene;
  return true;
}

// Work unit w of a render pass: the w-th most costly (item, pixel block)
// unit by its block list (length plus pixel hits), so that the longest units
// start first and the passes end with short ones.
__device__ __forceinline__ bool item_ctx(const WsView& v, int w, ItemCtx& c) {
  if (w >= v.hdr->n_items * kBlocksPerTile) return false;
  const int u = v.unit_order[w];
  return item_ctx_direct(v, u / kBlocksPerTile, u % kBlocksPerTile, c);
}

// Next work unit of a persistent render kernel (one atomic per warp).
__device__ __forceinline__ int next_unit(const WsView& v) {
  int w = 0;
  if ((threadIdx.x & 31) == 0) w = atomicAdd(&v.hdr->work_next, 1);
  return __shfl_sync(0xffffffffu, w, 0);
}

// A persistent CTA's fetch past the last unit.  Every CTA of the launch makes
// exactly one such fetch, drawing n_units .. n_units + gridDim.x - 1; the CTA
// that draws the largest knows every other CTA has fetched for the last time
// and resets the counter for the next persistent launch.
__device__ __forceinline__ void done_units(const WsView& v, int w, int n_units) {
  if ((threadIdx.x & 31) == 0 && w == n_units + (int)gridDim.x - 1) v.hdr->work_next = 0;
}

// Resident one-warp CTAs of a kernel on the current device: the grid of a
// persistent launch.
template <typename Kernel>
unsigned resident_slots(Kernel kern, int threads, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess) return 0;
  return (unsigned)sms * (unsigned)per_sm;
}

// Geometry of the pixel a thread renders.
struct PixelCtx {
  int tile_x0, tile_y0;   // first pixel of the tile
  int px, py;             // pixel coordinates
  bool inside;            // pixel lies inside the image
  float rx, ry;           // ray slopes (float32 decision values)
  ValueRay vr;            // ray slopes for the value path
};

__device__ __forceinline__ PixelCtx pixel_ctx(const SceneDev& S, int64_t tile, int block) {
  PixelCtx c;
  const int64_t lt = tile - S.tile_begin;
  const int ty = (int)(lt / S.tiles_x), tx = (int)(lt - (int64_t)ty * S.tiles_x);
  const int warp = block, lane = threadIdx.x & 31;
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

// Pixel rectangle of a warp's 8 x 4 block.
struct WarpRect {
  int x0, x1, y0, y1;
};

__device__ __forceinline__ WarpRect warp_rect(const PixelCtx& pc, int block) {
  const int warp = block;
  WarpRect r;
  r.x0 = pc.tile_x0 + (warp & 1) * 8;
  r.x1 = r.x0 + 7;
  r.y0 = pc.tile_y0 + (warp >> 1) * 4;
  r.y1 = r.y0 + 3;
  return r;
}

__device__ __forceinline__ bool rect_overlaps(const float4& b, const WarpRect& r) {
  const uint32_t bx = __float_as_uint(b.z), by = __float_as_uint(b.w);
  return (int)(bx & 0xffffu) <= r.x1 && (int)(bx >> 16) >= r.x0 && (int)(by & 0xffffu) <= r.y1 &&
         (int)(by >> 16) >= r.y0;
}

// ----------------------------------------------------------------------------
// 32 x 32 bit-matrix transpose across a warp: lane i passes row i (bit j =
// element (i, j)) and receives column i (bit j = element (j, i)).  Five
// butterfly stages, each swapping the off-diagonal blocks of the next finer
// block size.
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t transpose32(uint32_t x) {
  const int lane = threadIdx.x & 31;
  const uint32_t masks[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int s = 16 >> k;
    const uint32_t m = masks[k];
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
    x = (lane & s) ? ((x & ~m) | ((y >> s) & m)) : ((x & m) | ((y << s) & ~m));
  }
  return x;
}

// Exclusive prefix sum over the warp's lanes; total receives the sum.
__device__ __forceinline__ int warp_exclusive_scan(int x, int& total) {
  const int lane = threadIdx.x & 31;
  int inc = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += y;
  }
  total = __shfl_sync(0xffffffffu, inc, 31);
  return inc - x;
}

// ----------------------------------------------------------------------------
// Asynchronous staging of a work unit's block list.  A warp streams the list
// (entries: sphere index, hit mask over the block's 32 pixels), 32 entries
// per batch, through two shared-memory buffers with cp.async: while batch i
// is processed, the draw records, value records and features of batch i + 1
// are in flight and the list entries of batch i + 2 are being loaded.  The
// batch's hit masks, transposed across the warp, give every lane the bit set
// of the batch entries that hit its pixel.
// ----------------------------------------------------------------------------

template <int CMAX, int NB = 2>
struct StageBuf {
  // feature rows are padded so that lanes reading the rows of different
  // spheres with 16-byte loads spread over all shared-memory banks
  static constexpr int FS = CMAX >= 8 ? CMAX + 4 : CMAX;
  float4 rec0[NB][32];
  float4 rec1[NB][32];
  float4 rec2[NB][32];
  float feat[NB][32 * FS];
  int32_t id[NB][32];
  uint32_t hm[NB][32];
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int CMAX, int NB = 2, bool CHAIN = false>
struct UnitStream {
  static_assert(NB >= 2, "at least double buffering");
  const uint2* __restrict__ src;   // the unit's block list (of its pixel block, all segments)
  int n;                           // its length
  int base;                        // first entry of the current batch
  int buf;                         // buffer holding the current batch
  uint2 e_next;                    // this lane's entry of the next batch to stage
  // Chained walk (the paper's early termination, which needs a pixel's whole
  // list): the unit's list is the concatenation of the block lists of every
  // segment of its tile, in segment order.  c_item is the segment holding
  // entry c_cum onwards; loads come at rising positions.
  const ItemDesc* __restrict__ items;
  const int32_t* __restrict__ counts;
  int block, c_item, c_cum, c_cnt, c_b0;   // c_cnt entries of segment c_item start at c_b0

  __device__ __forceinline__ uint2 load(int at) {
    const int i = at + (int)(threadIdx.x & 31);
    if (i >= n) return make_uint2(0u, 0u);
    if constexpr (!CHAIN) {
      return src[i];
    } else {
      // the segment holding `at` (warp-uniform; it moves only at segment ends)
      while (at >= c_cum + c_cnt) {
        c_cum += c_cnt;
        ++c_item;
        c_cnt = counts[c_item * kBlocksPerTile + block];
        c_b0 = items[c_item].b0;
      }
      if (i < c_cum + c_cnt) return src[c_b0 + (i - c_cum)];
      // this lane's entry lies in a later segment
      int k = c_item + 1, cum = c_cum + c_cnt;
      int cnt = counts[k * kBlocksPerTile + block];
      while (i >= cum + cnt) {
        cum += cnt;
        ++k;
        cnt = counts[k * kBlocksPerTile + block];
      }
      return src[items[k].b0 + (i - cum)];
    }
  }

  // One commit group: records (and, with need_values, value records and
  // features) of the batch at `at`, whose lane entries are e, into buffer `to`.
  __device__ __forceinline__ void issue(StageBuf<CMAX, NB>& sb, const WsView& v, const SceneDev& S, uint2 e,
                                        int at, int to, bool need_values) const {
    const int lane = threadIdx.x & 31;
    if (at + lane < n) {
      const uint32_t id = e.x;
      cp_async16(&sb.rec0[to][lane], v.rec0 + id);
      cp_async16(&sb.rec1[to][lane], v.rec1 + id);
      sb.id[to][lane] = (int32_t)id;
      sb.hm[to][lane] = e.y;
      if (need_values) {
        cp_async16(&sb.rec2[to][lane], v.rec2 + id);
        const int C = S.n_channels;
        const float* __restrict__ f = S.feat + (int64_t)(id - S.sphere_begin) * C;
        float* dst = &sb.feat[to][lane * StageBuf<CMAX, NB>::FS];
        if ((C & 3) == 0 && (reinterpret_cast<uintptr_t>(f) & 15) == 0) {
#pragma unroll
          for (int c = 0; c < CMAX; c += 4)
            if (c < C) cp_async16(dst + c, f + c);
        } else {
#pragma unroll
          for (int c = 0; c < CMAX; ++c)
            if (c < C) cp_async4(dst + c, f + c);
        }
      }
    }
    cp_async_commit();
  }

  // Starts the block list of the unit: the first NB - 1 batches are staged
  // ahead.  Feature channels beyond C stay zero.
  __device__ __forceinline__ void start(StageBuf<CMAX, NB>& sb, const WsView& v, const SceneDev& S,
                                        const ItemCtx& it, bool need_values) {
    const int lane = threadIdx.x & 31;
    if (need_values && S.n_channels < CMAX)
      for (int e = lane; e < NB * 32 * StageBuf<CMAX, NB>::FS; e += 32) (&sb.feat[0][0])[e] = 0.0f;
    __syncwarp();
    if constexpr (CHAIN) {
      // every segment of the tile, from its first
      src = v.unit_list + (size_t)it.block * v.capacity;
      items = v.item_desc;
      counts = v.unit_count;
      block = it.block;
      c_item = it.first;
      c_cum = 0;
      c_cnt = counts[it.first * kBlocksPerTile + block];
      c_b0 = items[it.first].b0;
      n = 0;
      for (int k = it.first; k < it.first + it.nseg; ++k) n += counts[k * kBlocksPerTile + block];
    } else {
      src = v.unit_list + (size_t)it.block * v.capacity + it.b0;
      n = v.unit_count[it.slot];
    }
    base = 0;
    buf = 0;
#pragma unroll
    for (int k = 0; k < NB - 1; ++k) issue(sb, v, S, load(32 * k), 32 * k, k, need_values);
    e_next = load(32 * (NB - 1));
  }

  __device__ __forceinline__ int count() const { return min(32, n - base); }

  // Waits for the current batch's staging, starts staging the batch NB - 1
  // ahead, and returns the entries of the current batch that hit this lane's
  // pixel.
  __device__ __forceinline__ uint32_t begin(StageBuf<CMAX, NB>& sb, const WsView& v, const SceneDev& S,
                                            bool need_values) {
    cp_async_wait<NB - 2>();
    __syncwarp();
    const int lane = threadIdx.x & 31;
    const uint32_t hits = transpose32(base + lane < n ? sb.hm[buf][lane] : 0u);
    const int to = buf + NB - 1 < NB ? buf + NB - 1 : buf - 1;
    issue(sb, v, S, e_next, base + 32 * (NB - 1), to, need_values);
    e_next = load(base + 32 * NB);
    return hits;
  }

  // Moves to the next batch once every lane is done with the current one.
  __device__ __forceinline__ void advance() {
    __syncwarp();
    base += 32;
    buf = buf + 1 < NB ? buf + 1 : 0;
  }

  // Waits for every copy still in flight (before the warp leaves).
  __device__ __forceinline__ void drain() const {
    cp_async_wait<0>();
    __syncwarp();
  }
};

// Hit predicate without the depth: the sign test of ray_hit's discriminant,
// with the same operations, so it decides exactly as ray_hit does.
__device__ __forceinline__ bool ray_disc_positive(float cx, float cy, float cz, float R2, float rx,
                                                  float ry) {
  const float ex = __fmaf_rn(cz, rx, -cx);
  const float ey = __fmaf_rn(cz, ry, -cy);
  const float ez = __fmaf_rn(cx, ry, -__fmul_rn(cy, rx));
  const float cr2 = __fmaf_rn(ex, ex, __fmaf_rn(ey, ey, __fmul_rn(ez, ez)));
  const float rr = __fmaf_rn(rx, rx, __fmaf_rn(ry, ry, 1.0f));
  return __fmaf_rn(rr, R2, -cr2) > 0.0f;
}

// The pixel ray of either camera.  An orthographic ray starts at
// (rx, ry, 0) and runs along +z: the pinhole routines then apply to the
// shifted centre c - (rx, ry, 0) and the ray (0, 0, 1), in the same float32
// operations (the shift is one rounded subtraction).
__device__ __forceinline__ bool pixel_disc_positive(const float4& a, float rx, float ry, bool ortho) {
  return ortho ? ray_disc_positive(__fsub_rn(a.x, rx), __fsub_rn(a.y, ry), a.z, a.w, 0.0f, 0.0f)
               : ray_disc_positive(a.x, a.y, a.z, a.w, rx, ry);
}

__device__ __forceinline__ bool pixel_ray_hit(const float4& a, float tmin, float rx, float ry, float zfar,
                                              bool ortho, RayHit& h) {
  return ortho ? ray_hit(__fsub_rn(a.x, rx), __fsub_rn(a.y, ry), a.z, a.w, tmin, 0.0f, 0.0f, zfar, h)
               : ray_hit(a.x, a.y, a.z, a.w, tmin, rx, ry, zfar, h);
}

// Value-path geometry for either camera: the orthographic shift of the
// float-float centre is exact in its leading part (TwoSum).
__device__ __forceinline__ ValueGeom pixel_value_geom(const float4& a, const float4& c2, const ValueRay& r,
                                                      bool ortho) {
  if (!ortho) return value_geom(a, c2, r);
  const FF sx = two_sum(a.x, -r.rx), sy = two_sum(a.y, -r.ry);
  const float4 a2 = make_float4(sx.hi, sy.hi, a.z, a.w);
  const float4 c22 = make_float4(__fadd_rn(__fsub_rn(c2.x, r.rx_lo), sx.lo),
                                 __fadd_rn(__fsub_rn(c2.y, r.ry_lo), sy.lo), c2.z, c2.w);
  const ValueRay axis = {0.0f, 0.0f, 0.0f, 0.0f};
  return value_geom(a2, c22, axis);
}

// (t, id) ordering of tracked hits: by depth, then by sphere index.
__device__ __forceinline__ bool hit_less(float t, int id, float qt, int qi) {
  return t < qt || (t == qt && id < qi);
}

// Tracked-hit queue.  A hit is ordered by the key (depth bits << 32 | index):
// hit depths are positive, so their float bits order as unsigned integers and
// the key order is (depth, then index).  The queue holds the KMAX smallest
// keys in ascending order, right-aligned: the first KMAX - K slots hold the
// sentinel 0, which no hit displaces, so the K-th closest hit (runtime
// K <= KMAX) always sits in the last slot.  Free slots hold kEmptyKey.
constexpr uint64_t kEmptyKey = 0x7f8000007fffffffull;   // (+inf, INT_MAX)

__device__ __forceinline__ uint64_t hit_key(float t, int id) {
  return ((uint64_t)__float_as_uint(t) << 32) | (uint32_t)id;
}
__device__ __forceinline__ float key_depth(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ int key_index(uint64_t k) { return (int)(uint32_t)k; }

template <int KMAX>
__device__ __forceinline__ void queue_init(uint64_t (&q)[KMAX], int K) {
#pragma unroll
  for (int k = 0; k < KMAX; ++k) q[k] = k < KMAX - K ? 0ull : kEmptyKey;
}

// Sorted insertion into q[B, B + N); the largest key falls off the end.
template <int B, int N, int KMAX>
__device__ __forceinline__ void queue_insert_range(uint64_t (&q)[KMAX], uint64_t key) {
  bool lt[N];
#pragma unroll
  for (int k = 0; k < N; ++k) lt[k] = key < q[B + k];
#pragma unroll
  for (int k = N - 1; k >= 1; --k) q[B + k] = lt[k - 1] ? q[B + k - 1] : (lt[k] ? key : q[B + k]);
  q[B] = lt[0] ? key : q[B];
}

// Sorted insertion; the largest key falls off the end.  Every index is a
// compile-time constant so the queue stays in registers.  Queues of 16 and
// more are two halves: a key enters the lower half only if it is below the
// lower half's largest entry, which then moves on to the upper half, and the
// upper half is touched only by a key (or displaced entry) below its largest.
// While a pixel holds at most half the queue's capacity, the upper half is
// all empty keys and its network is skipped.
template <int KMAX>
__device__ __forceinline__ void queue_insert(uint64_t (&q)[KMAX], uint64_t key) {
  if constexpr (KMAX >= 16) {
    constexpr int H = KMAX / 2;
    if (key < q[H - 1]) {
      const uint64_t up = q[H - 1];
      queue_insert_range<0, H>(q, key);
      key = up;
    }
    if (key < q[KMAX - 1]) queue_insert_range<H, KMAX - H>(q, key);
  } else {
    queue_insert_range<0, KMAX>(q, key);
  }
}

// Next float after a positive depth (+inf stays +inf): spheres whose key is
// at or beyond this value can no longer enter a full tracked set, because
// every hit depth is at least the sphere's key.
__device__ __forceinline__ float next_up(float t) {
  return t < __int_as_float(0x7f800000) ? __uint_as_float(__float_as_uint(t) + 1u) : t;
}

}  // namespace pulsar
