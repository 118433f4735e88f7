// Binning (App. B, Step 0 sort and Step 1 region culling, re-designed):
//   1. stable LSD radix sort of (earliest depth, sphere index): the depth
//      key's float bits as an offset from the smallest near plane of the
//      batch (visible keys lie between the planes), 9 bits per pass,
//   2. exclusive scan of each sorted sphere's tile count,
//   3. emission of one (tile, sphere) pair per overlapped tile, in depth order,
//   4. stable LSD radix sort of the pairs by tile (6- or 8-bit digits),
//   5. per-tile [begin, end) ranges,
//   6. work items (list segments) in decreasing length,
//   7. block lists: per segment and 8 x 4 pixel block, the hitting spheres
//      with their per-pixel hit masks (block_lists.cu).
// A stable sort of pairs that arrive in depth order keeps every tile's list in
// (earliest depth, index) order, the order the paper's intersection search
// relies on for early termination (Sec. 3.2, App. B Step 0).
#include "pulsar_internal.cuh"

namespace pulsar {

namespace {

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ int read_count(const int32_t* n_dev, int n_host) {
  return n_dev ? *n_dev : n_host;
}

// Per-CTA digit histogram of one radix pass of RB-bit digits (warp-aggregated
// shared atomics).
template <int RB>
__global__ void __launch_bounds__(kThreads) radix_upsweep(const uint32_t* __restrict__ keys,
                                                          const int32_t* n_dev, int n_host, int shift,
                                                          uint32_t mask, uint32_t* __restrict__ hist,
                                                          int stride) {
  pdl_wait();
  pdl_trigger();
  constexpr int R = 1 << RB;
  __shared__ uint32_t h[R];
  const int n = read_count(n_dev, n_host);
  const int base = blockIdx.x * kSortTile;
  if (base >= n) return;
  for (int i = threadIdx.x; i < R; i += kThreads) h[i] = 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // all of this thread's keys in flight at once, then the ranking
  uint32_t kr[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int idx = base + warp * (kSortItems * 32) + k * 32 + lane;
    kr[k] = idx < n ? __ldg(keys + idx) : 0u;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    int idx = base + warp * (kSortItems * 32) + k * 32 + lane;
    bool valid = idx < n;
    uint32_t d = valid ? (kr[k] >> shift) & mask : 0xffffffffu;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    if (valid && (peers & lanemask_lt()) == 0) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < R; i += kThreads) hist[i * stride + blockIdx.x] = h[i];
}

// Exclusive scan, in place, of one digit's row of per-CTA counts
// (row r = blockIdx.x, cols = ceil(n / kSortTile) entries at data[r * stride]),
// and the row's total into row_tot[r].  One CTA per digit; each thread takes
// kScanPer consecutive columns per sweep, all loaded before the scan, so a
// row of up to kThreads * kScanPer columns is one load round trip and one
// block scan.
constexpr int kScanPer = 8;

__global__ void __launch_bounds__(kThreads) scan_rows(uint32_t* __restrict__ data,
                                                      uint32_t* __restrict__ row_tot,
                                                      const int32_t* n_dev, int n_host, int stride) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t warp_tot[33];
  const int n = read_count(n_dev, n_host);
  const int cols = (n + kSortTile - 1) / kSortTile;
  uint32_t* row = data + (size_t)blockIdx.x * stride;
  uint32_t carry = 0;
  for (int c0 = 0; c0 < cols; c0 += kThreads * kScanPer) {
    const int cb = c0 + threadIdx.x * kScanPer;
    uint32_t x[kScanPer];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) x[k] = cb + k < cols ? row[cb + k] : 0u;
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      const uint32_t t = x[k];
      x[k] = sum;
      sum += t;
    }
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan<kThreads>(sum, warp_tot, tot);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k)
      if (cb + k < cols) row[cb + k] = carry + ex + x[k];
    carry += tot;
  }
  if (threadIdx.x == 0) row_tot[blockIdx.x] = carry;
}

// Stable scatter of one radix pass.  Keys are ranked within each warp with
// match.any in index order; warps are combined in warp order; items are first
// placed in shared memory in their CTA-local sorted order and then written out
// in coalesced runs per digit.
template <int RB>
__global__ void __launch_bounds__(kThreads) radix_downsweep(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, const int32_t* n_dev,
    int n_host, int shift, uint32_t mask, const uint32_t* __restrict__ hist,
    const uint32_t* __restrict__ row_tot, int stride) {
  pdl_wait();
  pdl_trigger();
  constexpr int R = 1 << RB;
  // digits per thread in the per-digit steps (with fewer digits than
  // threads, thread t takes digit t and the others none)
  constexpr int DPT = R >= kThreads ? R / kThreads : 1;
  static_assert(R < kThreads || DPT * kThreads == R, "digits a multiple of the threads");
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[kSortTile];
  __shared__ uint32_t warp_cnt[kThreads / 32][R];
  __shared__ uint32_t digit_local[R];
  __shared__ uint32_t digit_global[R];
  __shared__ uint32_t warp_tot[33];
  const int n = read_count(n_dev, n_host);
  const int base = blockIdx.x * kSortTile;
  if (base >= n) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // all of this thread's keys and values in flight at once, with its digits'
  // global counts (row totals and this CTA's prefix), then the ranking
  uint32_t k_reg[kSortItems], v_reg[kSortItems], rank[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int idx = base + warp * (kSortItems * 32) + k * 32 + lane;
    k_reg[k] = idx < n ? __ldg(keys_in + idx) : 0u;
    v_reg[k] = idx < n ? __ldg(vals_in + idx) : 0u;
  }
  uint32_t rt[DPT], hcta[DPT];
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    const int d = threadIdx.x * DPT + q;
    rt[q] = d < R ? row_tot[d] : 0u;
    hcta[q] = d < R ? hist[d * stride + blockIdx.x] : 0u;
  }
  for (int w = 0; w < kThreads / 32; ++w)
    for (int i = threadIdx.x; i < R; i += kThreads) warp_cnt[w][i] = 0;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    int idx = base + warp * (kSortItems * 32) + k * 32 + lane;
    bool valid = idx < n;
    uint32_t d = valid ? (k_reg[k] >> shift) & mask : 0xffffffffu;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = 0;
    if (valid) before = warp_cnt[warp][d];
    rank[k] = before + __popc(peers & lanemask_lt());
    __syncwarp();
    if (valid && (peers & lanemask_lt()) == 0) warp_cnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, then over digits (thread t takes
  // the DPT consecutive digits from t * DPT)
  {
    uint32_t tot[DPT];
    uint32_t sum = 0, rsum = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = threadIdx.x * DPT + q;
      uint32_t t = 0;
      if (d < R)
        for (int w = 0; w < kThreads / 32; ++w) {
          uint32_t c = warp_cnt[w][d];
          warp_cnt[w][d] = t;
          t += c;
        }
      tot[q] = t;
      sum += t;
      rsum += rt[q];
    }
    uint32_t all;
    uint32_t ex = block_exclusive_scan<kThreads>(sum, warp_tot, all);
    // global start of digit d: all smaller digits, then earlier CTAs of d
    uint32_t base_d = block_exclusive_scan<kThreads>(rsum, warp_tot, all);
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = threadIdx.x * DPT + q;
      if (d < R) {
        digit_local[d] = ex;
        digit_global[d] = base_d + hcta[q];
      }
      ex += tot[q];
      base_d += rt[q];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    int idx = base + warp * (kSortItems * 32) + k * 32 + lane;
    if (idx < n) {
      uint32_t d = (k_reg[k] >> shift) & mask;
      uint32_t pos = digit_local[d] + warp_cnt[warp][d] + rank[k];
      s_keys[pos] = k_reg[k];
      s_vals[pos] = v_reg[k];
    }
  }
  __syncthreads();
  const int count = min(kSortTile, n - base);
  for (int lp = threadIdx.x; lp < count; lp += kThreads) {
    uint32_t key = s_keys[lp];
    uint32_t d = (key >> shift) & mask;
    uint32_t out = digit_global[d] + (lp - digit_local[d]);
    keys_out[out] = key;
    vals_out[out] = s_vals[lp];
  }
}

__device__ __forceinline__ uint32_t tile_count(const float4& r1, bool visible) {
  if (!visible) return 0u;
  uint32_t bx = __float_as_uint(r1.z), by = __float_as_uint(r1.w);
  int tx0 = (int)(bx & 0xffffu) / kTile, tx1 = (int)(bx >> 16) / kTile;
  int ty0 = (int)(by & 0xffffu) / kTile, ty1 = (int)(by >> 16) / kTile;
  return (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
}

// Exclusive scan of the n_blocks tile-count sums (CTA of NT threads); records
// the pair total and the overflow flag.
template <int NT>
__device__ __forceinline__ void scan_block_sums(const WsView& v, int n_blocks, uint32_t* warp_tot) {
  unsigned long long carry = 0;
  for (int b0 = 0; b0 < n_blocks; b0 += NT) {
    int b = b0 + threadIdx.x;
    uint32_t x = b < n_blocks ? __ldcg(v.block_sums + b) : 0u;
    uint32_t tot;
    uint32_t ex = block_exclusive_scan<NT>(x, warp_tot, tot);
    if (b < n_blocks) v.block_sums[b] = (uint32_t)(carry + ex);
    carry += tot;
  }
  if (threadIdx.x == 0) {
    long long total = (long long)carry;
    v.hdr->pairs_needed = total;
    bool over = total > v.capacity;
    v.hdr->overflow = over ? 1 : 0;
    v.hdr->n_pairs = over ? 0 : (int32_t)total;
  }
}

// Clears every tile's list range and merge counters (the kernel's threads in
// a grid-stride loop); the tile-key sort's range pass then fills the ranges of
// the tiles that have pairs.
__device__ __forceinline__ void clear_tile_state(const WsView& v) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < v.n_tiles; t += stride) {
    v.ranges[t] = make_int2(0, 0);
    reinterpret_cast<int4*>(v.tile_done)[2 * t] = make_int4(0, 0, 0, 0);
    reinterpret_cast<int4*>(v.tile_done)[2 * t + 1] = make_int4(0, 0, 0, 0);
  }
}

// Sum of the tile counts of each kSortTile-key tile of the depth-sorted
// spheres; also clears the per-tile state.
__global__ void __launch_bounds__(kThreads) count_reduce(WsView v) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t warp_tot[33];
  clear_tile_state(v);
  const int n = (int)v.n_spheres;
  const int base = blockIdx.x * kSortTile;
  // every load of the thread's spheres in flight at once
  uint32_t key[kSortItems], idx[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int j = base + threadIdx.x * kSortItems + k;
    key[k] = j < n ? __ldg(v.key[v.sort_buf] + j) : v.key_culled;
    idx[k] = j < n ? __ldg(v.val[v.sort_buf] + j) : 0u;
  }
  float4 r1[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) r1[k] = key[k] != v.key_culled ? __ldg(v.rec1 + idx[k]) : make_float4(0.f, 0.f, 0.f, 0.f);
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kSortItems; ++k)
    if (key[k] != v.key_culled) s += tile_count(r1[k], true);
  uint32_t tot;
  block_exclusive_scan<kThreads>(s, warp_tot, tot);
  if (threadIdx.x == 0) v.block_sums[blockIdx.x] = tot;
  // the last CTA to finish scans every CTA's sum (its own store is made
  // visible before it counts itself)
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&v.hdr->count_done, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  scan_block_sums<kThreads>(v, (int)gridDim.x, warp_tot);
  if (threadIdx.x == 0) v.hdr->count_done = 0;   // ready for the next binning
}

// The same scan as its own kernel, for a binning with no sphere (and so no
// tile-count CTA): records a pair total of zero.
__global__ void __launch_bounds__(1024) count_scan(WsView v, int n_blocks) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t warp_tot[33];
  clear_tile_state(v);
  scan_block_sums<1024>(v, n_blocks, warp_tot);
}

// Emits the (tile, sphere) pairs of each depth-sorted sphere at its scanned
// offset.  A pair's key is the global tile index in its low kTileKeyBits bits
// and, above them, the 8-bit set of the tile's 8 x 4 pixel blocks the
// sphere's rectangle meets (bit 2 r + c for block column c, row r).  The sort
// by tile reads only the low bits, so the block set rides along.
__global__ void __launch_bounds__(kThreads) emit_pairs(WsView v) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t warp_tot[33];
  const int n = (int)v.n_spheres;
  if (v.hdr->overflow) return;
  const int base = blockIdx.x * kSortTile;
  // every load of the thread's spheres in flight at once
  uint32_t key[kSortItems], idx[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int j = base + threadIdx.x * kSortItems + k;
    key[k] = j < n ? __ldg(v.key[v.sort_buf] + j) : v.key_culled;
    idx[k] = j < n ? __ldg(v.val[v.sort_buf] + j) : 0u;
  }
  float4 r1s[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k)
    r1s[k] = key[k] != v.key_culled ? __ldg(v.rec1 + idx[k]) : make_float4(0.f, 0.f, 0.f, 0.f);
  uint32_t cnt[kSortItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    cnt[k] = key[k] != v.key_culled ? tile_count(r1s[k], true) : 0u;
    s += cnt[k];
  }
  uint32_t tot;
  uint32_t off = block_exclusive_scan<kThreads>(s, warp_tot, tot) + v.block_sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    if (cnt[k] == 0) continue;
    const uint32_t i = idx[k];
    const float4 r1 = r1s[k];
    int sc = scene_of_sphere(v.scenes, v.n_scenes, i);
    const SceneDev& S = v.scenes[sc];
    uint32_t bx = __float_as_uint(r1.z), by = __float_as_uint(r1.w);
    int tx0 = (int)(bx & 0xffffu) / kTile, tx1 = (int)(bx >> 16) / kTile;
    int ty0 = (int)(by & 0xffffu) / kTile, ty1 = (int)(by >> 16) / kTile;
    uint32_t tb = (uint32_t)S.tile_begin;
    const int x0 = (int)(bx & 0xffffu), x1 = (int)(bx >> 16);
    const int y0 = (int)(by & 0xffffu), y1 = (int)(by >> 16);
    for (int ty = ty0; ty <= ty1; ++ty) {
      // rows of 8 x 4 pixel blocks the rectangle meets in this tile row
      const int r0 = (max(y0 - ty * kTile, 0)) >> 2, r1 = (min(y1 - ty * kTile, kTile - 1)) >> 2;
      const uint32_t rows = ((1u << (2 * r1 + 2)) - (1u << (2 * r0))) / 3u;   // sum of 4^r, r0..r1
      for (int tx = tx0; tx <= tx1; ++tx) {
        const int c0 = (max(x0 - tx * kTile, 0)) >> 3, c1 = (min(x1 - tx * kTile, kTile - 1)) >> 3;
        const uint32_t blocks = ((2u << c1) - (1u << c0)) * rows;   // bit 2 r + c: block (c, r)
        v.pkey[0][off] = (tb + (uint32_t)(ty * S.tiles_x + tx)) | (blocks << kTileKeyBits);
        v.pval[0][off] = i;
        ++off;
      }
    }
  }
}

// Tile ranges from the tile-sorted pairs (ranges are zeroed beforehand).
__global__ void __launch_bounds__(kThreads) tile_ranges(WsView v, int buf) {
  pdl_wait();
  pdl_trigger();
  const int n = v.hdr->n_pairs;
  const uint32_t* keys = v.pkey[buf];
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
    const uint32_t t = keys[i] & kTileKeyMask;
    if (i == 0 || (keys[i - 1] & kTileKeyMask) != t) v.ranges[t].x = i;
    if (i == n - 1 || (keys[i + 1] & kTileKeyMask) != t) v.ranges[t].y = i + 1;
  }
}

// Work items of the render passes: every non-empty tile's list is cut into
// segments of at most v.segment entries (the pixels of empty tiles are
// written by the background pass).  Writes item_begin (n_tiles + 1), one
// descriptor per item, the item count and item_order, the items by
// decreasing length (a counting sort over kOrderBuckets length classes; the
// order within a class is arbitrary).
constexpr int kOrderBuckets = 64;

__global__ void __launch_bounds__(1024) make_items(WsView v) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t warp_tot[33];
  __shared__ uint32_t bucket[kOrderBuckets];
  const int64_t nt = v.n_tiles;
  const int64_t per = (nt + 1023) / 1024;
  const int64_t t0 = (int64_t)threadIdx.x * per;
  const int64_t t1 = t0 + per < nt ? t0 + per : nt;
  const int64_t seg_len = v.segment;
  uint32_t s = 0;
  for (int64_t t = t0; t < t1; ++t) {
    const int2 rg = v.ranges[t];
    s += (uint32_t)(((int64_t)rg.y - rg.x + seg_len - 1) / seg_len);
  }
  uint32_t tot;
  uint32_t base = block_exclusive_scan<1024>(s, warp_tot, tot);
  for (int64_t t = t0; t < t1; ++t) {
    const int2 rg = v.ranges[t];
    const int ns = (int)(((int64_t)rg.y - rg.x + seg_len - 1) / seg_len);
    v.item_begin[t] = (int32_t)base;
    const int scene = ns > 0 ? scene_of_tile(v.scenes, v.n_scenes, t) : 0;
    for (int k = 0; k < ns; ++k) {
      ItemDesc d;
      d.tile = (int32_t)t;
      d.b0 = (int32_t)(rg.x + k * seg_len);
      d.b1 = (int32_t)min(rg.x + (k + 1) * seg_len, (int64_t)rg.y);
      d.seg = k;
      d.nseg = ns;
      d.first = (int32_t)base;
      d.scene = scene;
      d.pad_ = 0;
      v.item_desc[base + k] = d;
    }
    base += (uint32_t)ns;
  }
  if (threadIdx.x == 0) {
    v.item_begin[nt] = (int32_t)tot;
    v.hdr->n_items = (int32_t)tot;
  }
  if (threadIdx.x < kOrderBuckets) bucket[threadIdx.x] = 0u;
  __syncthreads();
  // length class of an item: 0 for a full segment ... kOrderBuckets - 1 for one entry
  auto cls = [&](uint32_t i) {
    const ItemDesc& d = v.item_desc[i];
    const int len = d.b1 - d.b0;
    return (int)(((seg_len - len) * (kOrderBuckets - 1)) / seg_len);
  };
  for (uint32_t i = threadIdx.x; i < tot; i += 1024) atomicAdd(&bucket[cls(i)], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int b = 0; b < kOrderBuckets; ++b) {
      const uint32_t c = bucket[b];
      bucket[b] = run;
      run += c;
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < tot; i += 1024) v.item_order[atomicAdd(&bucket[cls(i)], 1u)] = (int32_t)i;
}

// Stable LSD radix sort of (key, value) by the low `bits` key bits, RB bits
// per pass; buf is the buffer holding the input and, on return, the output.
template <int RB>
cudaError_t radix_sort(const WsView& v, uint32_t* keys[2], uint32_t* vals[2], const int32_t* n_dev,
                       int n_host, int max_items, int bits, int& buf, cudaStream_t st) {
  const int blocks = (max_items + kSortTile - 1) / kSortTile;
  if (blocks == 0) return cudaSuccess;
  for (int shift = 0; shift < bits; shift += RB) {
    uint32_t mask = (uint32_t)((1u << min(RB, bits - shift)) - 1u);
    cudaError_t e = launch_pdl(radix_upsweep<RB>, dim3(blocks), dim3(kThreads), 0, st, keys[buf], n_dev,
                               n_host, shift, mask, v.hist, v.sort_blocks);
    if (e == cudaSuccess)
      e = launch_pdl(scan_rows, dim3(1 << RB), dim3(kThreads), 0, st, v.hist, v.radix_tot, n_dev, n_host,
                     v.sort_blocks);
    if (e == cudaSuccess)
      e = launch_pdl(radix_downsweep<RB>, dim3(blocks), dim3(kThreads), 0, st, keys[buf], vals[buf],
                     keys[buf ^ 1], vals[buf ^ 1], n_dev, n_host, shift, mask, v.hist, v.radix_tot,
                     v.sort_blocks);
    if (e != cudaSuccess) return e;
    buf ^= 1;
  }
  return cudaSuccess;
}

}  // namespace

// Returns, through `tile_bits`, nothing; the pair buffer holding the final
// order is recorded by the caller from the pass count.
cudaError_t launch_bin(const WsView& v, int tile_bits, cudaStream_t st) {
  cudaError_t e;
  const int M = (int)v.n_spheres;
  // 1. spheres by earliest depth (float bits of positive keys sort as integers)
  int buf = 0;
  if (M > 0) {
    uint32_t* k[2] = {v.key[0], v.key[1]};
    uint32_t* val[2] = {v.val[0], v.val[1]};
    e = radix_sort<kDepthRadixBits>(v, k, val, nullptr, M, M, v.key_bits, buf, st);
    if (e != cudaSuccess) return e;
  }
  // the sorted spheres are in buffer v.sort_buf (the parity of the pass count)
  const int nb = (M + kSortTile - 1) / kSortTile;
  if (nb > 0)
    e = launch_pdl(count_reduce, dim3(nb), dim3(kThreads), 0, st, v);   // its last CTA scans the sums
  else
    e = launch_pdl(count_scan, dim3(1), dim3(1024), 0, st, v, 0);
  if (e == cudaSuccess && nb > 0) e = launch_pdl(emit_pairs, dim3(nb), dim3(kThreads), 0, st, v);
  if (e != cudaSuccess) return e;
  // 4. pairs by tile
  int pbuf = 0;
  if (v.capacity > 0) {
    uint32_t* k[2] = {v.pkey[0], v.pkey[1]};
    uint32_t* val[2] = {v.pval[0], v.pval[1]};
    e = tile_radix_bits(tile_bits) == 6
            ? radix_sort<6>(v, k, val, &v.hdr->n_pairs, 0, (int)v.capacity, tile_bits, pbuf, st)
            : radix_sort<kRadixBits>(v, k, val, &v.hdr->n_pairs, 0, (int)v.capacity, tile_bits, pbuf, st);
    if (e != cudaSuccess) return e;
  }
  // 5. ranges (cleared with the tile counts)
  if (v.capacity > 0) {
    const int64_t want = (v.capacity + kThreads - 1) / kThreads;
    const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
    e = launch_pdl(tile_ranges, dim3(blocks), dim3(kThreads), 0, st, v, pbuf);
    if (e != cudaSuccess) return e;
  }
  // 6. work items of the render passes (the merge counters were cleared with the tile counts)
  if (v.n_tiles > 0) {
    e = launch_pdl(make_items, dim3(1), dim3(1024), 0, st, v);
    if (e != cudaSuccess) return e;
  }
  // 7. per pixel block: the spheres hitting it, with their hit masks
  return launch_block_lists(v, st);
}

}  // namespace pulsar
