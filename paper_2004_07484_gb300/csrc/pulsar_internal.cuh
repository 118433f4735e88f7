// Internal declarations of the GB300 sphere renderer: device structures,
// workspace layout, and the float32 decision routines shared by the kernels.
//
// Decision routines (camera rows, projection, culling, rectangle, sort key,
// hit predicate and hit depth) decide discrete outcomes: which tiles list a
// sphere, in which order, and which hits a pixel tracks.  They are written as
// fixed sequences of correctly rounded IEEE operations (__fadd_rn, __fmul_rn,
// __fmaf_rn, __fdiv_rn, __fsqrt_rn), so the compiler cannot fuse or reorder
// them and every launch decides identically.  The numeric value path (weights,
// image, gradients) uses ordinary fast float32 arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pulsar.h"

namespace pulsar {

// Programmatic dependent launch (sm_90 and later).  The kernels of a step are
// launched with programmatic stream serialisation: a kernel may be scheduled
// while the one before it in the stream is still finishing, so its launch and
// CTA rasterisation overlap that kernel's tail.  Every such kernel calls
// pdl_wait() before it touches global memory; it returns once the previous
// grid has completed and its writes are visible (at once when the kernel was
// launched without the attribute).  pdl_trigger() lets the next kernel be
// scheduled as soon as every CTA of this one has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches `kernel` on `st` with programmatic stream serialisation (a plain
// launch where the runtime does not offer it on that stream); the kernel must
// start with pdl_wait().
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              const A&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
  if (e == cudaErrorNotSupported) {
    (void)cudaGetLastError();
    cfg.numAttrs = 0;
    e = cudaLaunchKernelEx(&cfg, kernel, args...);
  }
  return e;
}

constexpr int kThreads = 256;        // threads per CTA for the per-tile kernels (16 x 16 pixels)
constexpr int kTile = 16;            // tile edge in pixels
constexpr int kChunk = 256;          // spheres staged in shared memory per round
constexpr int kSortItems = 8;        // keys per thread in one radix-sort tile
constexpr int kSortTile = kThreads * kSortItems;   // 2048 keys per radix-sort CTA
constexpr int kRadixBits = 8;              // digit bits of the tile-key sort
constexpr int kRadix = 1 << kRadixBits;
// Digit bits of the tile-key sort for a key of `bits` bits: 6 where that
// takes no more passes than 8 (9 to 12 bits: two passes either way, and
// 6-bit digits leave longer runs of equal digits to scatter), else 8.
inline int tile_radix_bits(int bits) { return bits > 8 && bits <= 12 ? 6 : kRadixBits; }
constexpr int kDepthRadixBits = 9;         // digit bits of the depth-key sort
constexpr int kDepthRadix = 1 << kDepthRadixBits;
constexpr int kMaxScenes = 64;
constexpr int kFinalizeThreads = 256;
constexpr int kCamPartials = 16;     // floats per finalize-block camera partial (13 used)
constexpr int kDefaultSegment = 1024;  // list entries one CTA processes per work item
constexpr int kTileKeyBits = 24;        // pair keys: tile index bits (the block set above them)
constexpr uint32_t kTileKeyMask = (1u << kTileKeyBits) - 1u;

// Per-scene description in the workspace.  The host fills the inputs; the
// setup kernel derives the camera rows and pixel pitch.
struct SceneDev {
  // inputs
  const float* pos;
  const float* rad;
  const float* opa;
  const float* feat;
  const float* cam;
  const float* bg;
  // forward outputs
  float* image;
  float* log_norm;
  int32_t* n_hits;
  int32_t* n_tests;
  int32_t* tracked;
  // backward inputs / outputs
  const float* image_in;
  const float* log_norm_in;
  const float* grad_image;
  float* g_pos;
  float* g_rad;
  float* g_opa;
  float* g_feat;
  float* g_cam;
  float* g_bg;
  // sizes
  int32_t width, height, n_spheres, n_channels, n_track;
  uint32_t flags;
  int32_t tiles_x, tiles_y;
  int64_t sphere_begin;      // first global sphere index of this scene
  int64_t tile_begin;        // first global tile index
  int64_t pixel_begin;       // first global pixel index
  int32_t fin_block_begin;   // first finalize block
  int32_t fin_blocks;
  float gamma, eps, znear, zfar;
  // derived on the device by the setup kernel
  double rows64[9];          // camera axes in double (value path)
  float rows_hi[9];          // rows64 as float pairs hi + lo (per-sphere value path)
  float rows_lo[9];
  double kappa64;            // pixel pitch in double (value path)
  float rows[9];             // camera axes b1, b2, b3 (world -> camera rows), float32 decisions
  float kappa;               // pixel pitch on the unit image plane, s / (W f), float32 decisions
  float kappa_hi, kappa_lo;  // kappa64 split into two floats (value path)
  uint32_t omax_bits;        // max |o| over visible spheres, float bits
  float stop_log_ratio;      // ln(tau / (1 - tau)), tau the early-termination threshold
  uint32_t pad_;             // unused
};

// Device-side counters and flags at the start of the workspace.
struct WsHeader {
  int32_t n_scenes;
  int32_t overflow;          // 1 when the pair count exceeded list_capacity
  int64_t pairs_needed;      // pair count the last binning required
  int32_t n_pairs;           // pairs in the lists (0 after an overflow)
  int32_t n_sort;            // keys in the sphere sort (= total spheres)
  int32_t timeout;           // a bounded device loop gave up
  int32_t n_items;           // (tile, segment) work items of the render passes
  int32_t work_next;         // next work unit of a persistent render launch
  int32_t count_done;        // tile-count CTAs finished (the last one scans their sums)
  int32_t pad_[6];
};

// One work item of the render passes: a segment [b0, b1) of a tile's list.
struct __align__(16) ItemDesc {
  int32_t tile;    // global tile index
  int32_t b0, b1;  // list range
  int32_t seg;     // segment index within the tile
  int32_t nseg;    // segments of the tile
  int32_t first;   // first work item of the tile
  int32_t scene;   // scene owning the tile
  int32_t pad_;
};

// Raw pointers into one workspace, passed to kernels by value.
struct WsView {
  WsHeader* hdr;
  SceneDev* scenes;
  int32_t n_scenes;
  int64_t n_spheres;         // total over scenes
  int64_t n_tiles;           // total over scenes
  int64_t n_pixels;          // total over scenes
  int64_t capacity;          // pair capacity
  int32_t sort_blocks;       // radix-sort CTAs covering max(n_spheres, capacity)
  int32_t fin_blocks;        // finalize CTAs over all scenes
  int32_t n_channels;        // common feature length of the batch
  int32_t n_track;           // common n_track of the batch
  int32_t pair_buf;          // ping-pong buffer holding the tile-sorted pairs
  int32_t segment;           // list entries per work item (a multiple of kChunk)
  int32_t max_items;         // bound on work items: n_tiles + capacity / segment
  int32_t part_fields;       // floats per pixel of a partial forward state
  int32_t persistent;        // render passes run as persistent kernels
  int32_t paper;             // the paper's gradient normalisations
  int32_t chain;             // render units walk a tile's segments in order (early termination)
  uint32_t key_base;         // depth sort keys: float bits of the key minus key_base
  uint32_t key_culled;       // the depth sort key of a culled sphere (above every visible one)
  int32_t key_bits;          // significant bits of the depth sort keys
  int32_t sort_buf;          // buffer holding the depth-sorted spheres
  float4* rec0;              // per sphere: c.x, c.y, c.z, R^2
  float4* rec1;              // per sphere: key, o, x-range (x0 | x1 << 16), y-range
  float4* rec2;              // per sphere: c - c.xyz (low-order part of the double centre), R
  uint32_t* key[2];          // radix sort keys (ping-pong)
  uint32_t* val[2];          // radix sort values (ping-pong)
  uint32_t* hist;            // radix histograms [digits][sort_blocks]
  uint32_t* block_sums;      // scan partials [sort_blocks]
  uint32_t* radix_tot;       // per digit: total count of one radix pass
  uint32_t* pkey[2];         // pair tile ids (ping-pong)
  uint32_t* pval[2];         // pair sphere ids (ping-pong)
  int2* ranges;              // per tile [begin, end)
  int32_t* item_begin;       // per tile (+1): first work item
  ItemDesc* item_desc;       // per work item
  int32_t* item_order;       // work items by decreasing segment length (block-list launch order)
  uint2* unit_list;          // block lists: [pixel block][capacity] (sphere, hit mask)
  int32_t* unit_count;       // per work unit (item x 8 + block): block-list length
  uint32_t* unit_cost;       // per work unit: block-list length + pixel hits in its masks
  int32_t* unit_order;       // work units by decreasing cost (render-pass launch order)
  int32_t* unit_tests;       // per work unit x 32 pixels: rectangle tests made
  int32_t* tile_done;        // per tile: finished segments (last-finisher merge)
  float* partial;            // per work item: partial forward state, [field][pixel]
  float* item_kappa;         // per work item: d L / d kappa partial
  float* tile_bg;            // per (tile, pixel block) x C background-gradient partials
  float4* pix_aux;           // per pixel: (t_K, id_K bits, reference sphere bits, 0)
  float* fres;               // per pixel x C: F - f_ref, the image relative to its reference feature
  float4* gacc;              // per sphere: dL/dc (3), dL/dR
  int32_t* pg_cnt;           // paper gradients: per sphere, pixels that track it
  float* pg_opa;             // paper gradients: per sphere, dL/do before averaging
  float* pg_feat;            // paper gradients: per sphere x C, dL/df before averaging
  float* fin_part;           // per finalize block: camera partials
  float* red_part;           // per scene x 64: first-stage camera / background sums (45)
  int32_t* cam_done;         // per scene: first-stage reduction CTAs finished (the last one finishes the sum)
};

// ----------------------------------------------------------------------------
// float32 decision routines
// ----------------------------------------------------------------------------

__device__ __forceinline__ void rows_from_rot6(const float* a, float* B) {
  float n1 = __fsqrt_rn(__fmaf_rn(a[0], a[0], __fmaf_rn(a[1], a[1], __fmul_rn(a[2], a[2]))));
  float b1x = __fdiv_rn(a[0], n1), b1y = __fdiv_rn(a[1], n1), b1z = __fdiv_rn(a[2], n1);
  float dt = __fmaf_rn(b1x, a[3], __fmaf_rn(b1y, a[4], __fmul_rn(b1z, a[5])));
  float ux = __fmaf_rn(-dt, b1x, a[3]);
  float uy = __fmaf_rn(-dt, b1y, a[4]);
  float uz = __fmaf_rn(-dt, b1z, a[5]);
  float n2 = __fsqrt_rn(__fmaf_rn(ux, ux, __fmaf_rn(uy, uy, __fmul_rn(uz, uz))));
  float b2x = __fdiv_rn(ux, n2), b2y = __fdiv_rn(uy, n2), b2z = __fdiv_rn(uz, n2);
  B[0] = b1x; B[1] = b1y; B[2] = b1z;
  B[3] = b2x; B[4] = b2y; B[5] = b2z;
  B[6] = __fmaf_rn(b1y, b2z, -__fmul_rn(b1z, b2y));
  B[7] = __fmaf_rn(b1z, b2x, -__fmul_rn(b1x, b2z));
  B[8] = __fmaf_rn(b1x, b2y, -__fmul_rn(b1y, b2x));
}

__device__ __forceinline__ float pixel_pitch(const float* cam, int width, bool ortho) {
  return ortho ? __fdiv_rn(cam[10], (float)width) : __fdiv_rn(cam[10], __fmul_rn((float)width, cam[9]));
}

struct Projected {
  float cx, cy, cz, R, R2, key;
  bool visible;
  int x0, x1, y0, y1;
};

// One axis of the enclosing rectangle: the tangent slopes of the (axis, z)
// disk seen from the eye, converted to pixel units; the pixels whose centres
// lie within the bounds widened by 1/8 pixel (the float32 hit predicate's
// boundary lies within ~1e-4 pixel of the exact one).  The block lists test
// exactly these pixels.
__device__ __forceinline__ void axis_range(float cx, float cz, float R, float R2, float kappa,
                                           int n, int& lo, int& hi) {
  float den = __fmaf_rn(cz, cz, -R2);
  float disc = __fmaf_rn(cx, cx, den);
  float root = __fsqrt_rn(disc);
  float base = __fmul_rn(cx, cz);
  float rs = __fmul_rn(R, root);
  float mlo = __fdiv_rn(__fsub_rn(base, rs), den);
  float mhi = __fdiv_rn(__fadd_rn(base, rs), den);
  float half = __fmul_rn((float)(n - 1), 0.5f);
  float flo = __fadd_rn(__fdiv_rn(mlo, kappa), half);
  float fhi = __fadd_rn(__fdiv_rn(mhi, kappa), half);
  flo = fmaxf(fminf(flo, (float)n + 2.0f), -4.0f);
  fhi = fmaxf(fminf(fhi, (float)n + 2.0f), -4.0f);
  lo = (int)ceilf(__fsub_rn(flo, 0.125f));
  hi = (int)floorf(__fadd_rn(fhi, 0.125f));
}

// One axis of the rectangle of the orthographic camera: the centre -+ R in
// pixels, widened by 1/8 pixel.
__device__ __forceinline__ void axis_range_ortho(float cx, float R, float kappa, int n, int& lo, int& hi) {
  float half = __fmul_rn((float)(n - 1), 0.5f);
  float flo = __fadd_rn(__fdiv_rn(__fsub_rn(cx, R), kappa), half);
  float fhi = __fadd_rn(__fdiv_rn(__fadd_rn(cx, R), kappa), half);
  flo = fmaxf(fminf(flo, (float)n + 2.0f), -4.0f);
  fhi = fmaxf(fminf(fhi, (float)n + 2.0f), -4.0f);
  lo = (int)ceilf(__fsub_rn(flo, 0.125f));
  hi = (int)floorf(__fadd_rn(fhi, 0.125f));
}

// Step 0 for one sphere: camera-space centre, effective radius (one-pixel
// minimum size), culling, rectangle and sort key.
// The camera-space centre and the radius after the minimum-size rule: the
// first part of project_sphere, for passes that need no rectangle.
__device__ __forceinline__ void sphere_centre_radius(const float* B, const float* cam, float kappa,
                                                     float px, float py, float pz, float r,
                                                     bool min_size, bool ortho, Projected& o) {
  float dx = __fsub_rn(px, cam[0]), dy = __fsub_rn(py, cam[1]), dz = __fsub_rn(pz, cam[2]);
  o.cx = __fmaf_rn(B[0], dx, __fmaf_rn(B[1], dy, __fmul_rn(B[2], dz)));
  o.cy = __fmaf_rn(B[3], dx, __fmaf_rn(B[4], dy, __fmul_rn(B[5], dz)));
  o.cz = __fmaf_rn(B[6], dx, __fmaf_rn(B[7], dy, __fmul_rn(B[8], dz)));
  float R = r;
  if (min_size) {
    float rmin;
    if (ortho) {
      rmin = __fmul_rn(0.75f, kappa);
    } else {
      float cn = __fsqrt_rn(__fmaf_rn(o.cx, o.cx, __fmaf_rn(o.cy, o.cy, __fmul_rn(o.cz, o.cz))));
      rmin = __fmul_rn(0.75f, __fmul_rn(cn, kappa));
    }
    if (rmin > r) R = rmin;
  }
  o.R = R;
}

__device__ __forceinline__ Projected project_sphere(const float* B, const float* cam, float kappa,
                                                    float px, float py, float pz, float r,
                                                    int width, int height, float znear, float zfar,
                                                    bool min_size, bool ortho) {
  Projected o;
  sphere_centre_radius(B, cam, kappa, px, py, pz, r, min_size, ortho, o);
  const float R = o.R;
  o.R2 = __fmul_rn(R, R);
  o.key = __int_as_float(0x7f800000);
  o.visible = false;
  o.x0 = o.x1 = o.y0 = o.y1 = -1;
  float key = __fsub_rn(o.cz, R);
  if (!(R > 0.0f) || !(key > znear) || !(key < zfar)) return o;
  int x0, x1, y0, y1;
  if (ortho) {
    axis_range_ortho(o.cx, R, kappa, width, x0, x1);
    axis_range_ortho(o.cy, R, kappa, height, y0, y1);
  } else {
    axis_range(o.cx, o.cz, R, o.R2, kappa, width, x0, x1);
    axis_range(o.cy, o.cz, R, o.R2, kappa, height, y0, y1);
  }
  if (x1 < 0 || x0 > width - 1 || y1 < 0 || y0 > height - 1) return o;
  o.x0 = max(x0, 0);
  o.x1 = min(x1, width - 1);
  o.y0 = max(y0, 0);
  o.y1 = min(y1, height - 1);
  o.key = key;
  o.visible = true;
  return o;
}

__device__ __forceinline__ float ray_coord(int u, int n, float kappa) {
  return __fmul_rn(__fmul_rn((float)(2 * u + 1 - n), 0.5f), kappa);
}

// Intermediate values of the hit test that the value path reuses.
struct RayHit {
  float ex, ey, ez;   // components of (c x r) up to order and sign
  float cr2;          // |c x r|^2
  float rr;           // |r|^2
  float sq;           // sqrt(rr R^2 - |c x r|^2)
  float off;          // c_z - t_h
  float t;            // front-hit depth (camera z)
};

// Hit predicate of the ray (rx, ry, 1) and the sphere record (c, R^2); the
// hit depth is never taken nearer than tmin = c_z - R (the sort key).
__device__ __forceinline__ bool ray_hit(float cx, float cy, float cz, float R2, float tmin,
                                        float rx, float ry, float zfar, RayHit& h) {
  h.ex = __fmaf_rn(cz, rx, -cx);
  h.ey = __fmaf_rn(cz, ry, -cy);
  h.ez = __fmaf_rn(cx, ry, -__fmul_rn(cy, rx));
  h.cr2 = __fmaf_rn(h.ex, h.ex, __fmaf_rn(h.ey, h.ey, __fmul_rn(h.ez, h.ez)));
  h.rr = __fmaf_rn(rx, rx, __fmaf_rn(ry, ry, 1.0f));
  float disc = __fmaf_rn(h.rr, R2, -h.cr2);
  if (!(disc > 0.0f)) return false;
  h.sq = __fsqrt_rn(disc);
  h.off = __fdiv_rn(__fmaf_rn(rx, h.ex, __fmaf_rn(ry, h.ey, h.sq)), h.rr);
  h.t = fmaxf(__fsub_rn(cz, h.off), tmin);
  return h.t < zfar;
}

// Value-path ray: the slopes (u + 1/2 - W/2) kappa as hi + lo float pairs.
struct ValueRay {
  float rx, rx_lo, ry, ry_lo;
};

__device__ __forceinline__ ValueRay value_ray(int u, int v, int width, int height, float k_hi,
                                              float k_lo) {
  ValueRay r;
  const float px = (float)(2 * u + 1 - width) * 0.5f;
  const float py = (float)(2 * v + 1 - height) * 0.5f;
  r.rx = px * k_hi;
  r.rx_lo = fmaf(px, k_hi, -r.rx) + px * k_lo;
  r.ry = py * k_hi;
  r.ry_lo = fmaf(py, k_hi, -r.ry) + py * k_lo;
  return r;
}

// Value-path geometry of a hit.  c = c_hi + c_lo (rec0.xyz + rec2.xyz) and
// the ray slopes are carried as float pairs, and the ray-to-centre offsets
// e = c_z r - c are formed with one rounding of the (cancelling) leading
// terms, so dist, the hit depth and z keep about float precision relative to
// the sphere radius even where |c| is large.
struct ValueGeom {
  float ex, ey, ez;   // c x r = (-ey, ex, ez)
  float cr2, rr;      // |c x r|^2, |r|^2
  float qd;           // dist / R
  float sq;           // sqrt(|r|^2 R^2 - |c x r|^2) = sqrt(disc)
  float off;          // c_z - t_h
};

// Value-path square root and quotient: hardware approximations (about 2 ulp),
// well inside the value path's tolerance.
__device__ __forceinline__ float vsqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ float vdiv(float a, float b) { return __fdividef(a, b); }

// The forward pass blends with these values and the backward pass
// differentiates the same ones: every operation that sets dist / R and the
// depth offset is an explicitly rounded intrinsic, so the compiler fuses none
// of them differently in the two kernels and both passes see bit-identical
// d and z.  (At the rim, d = 1 - dist/R is a difference of nearly equal
// numbers; two differently rounded evaluations would differ in d by a large
// relative amount there, and the backward pass's weight a'/D' would no longer
// match the forward pass's denominator.)  dist / R = sqrt(|c x r|^2 /
// (|r|^2 R^2)) takes one correctly rounded division and square root.
__device__ __forceinline__ ValueGeom value_geom(const float4& a, const float4& c2, const ValueRay& r) {
  ValueGeom g;
  g.ex = __fadd_rn(__fmaf_rn(a.z, r.rx, -a.x), __fmaf_rn(a.z, r.rx_lo, __fmaf_rn(c2.z, r.rx, -c2.x)));
  g.ey = __fadd_rn(__fmaf_rn(a.z, r.ry, -a.y), __fmaf_rn(a.z, r.ry_lo, __fmaf_rn(c2.z, r.ry, -c2.y)));
  g.ez = __fdiv_rn(__fmaf_rn(a.x, g.ey, -__fmul_rn(a.y, g.ex)), a.z);
  g.cr2 = __fmaf_rn(g.ex, g.ex, __fmaf_rn(g.ey, g.ey, __fmul_rn(g.ez, g.ez)));
  g.rr = __fmaf_rn(r.rx, r.rx, __fmaf_rn(r.ry, r.ry, 1.0f));
  const float R = c2.w;
  const float R2 = __fmul_rn(R, R);
  g.qd = __fsqrt_rn(__fdiv_rn(g.cr2, __fmul_rn(g.rr, R2)));
  g.sq = vsqrt(__fmaf_rn(g.rr, R2, -g.cr2));
  g.off = vdiv(__fmaf_rn(r.rx, g.ex, __fmaf_rn(r.ry, g.ey, g.sq)), g.rr);
  return g;
}

// Float-float arithmetic (a value is hi + lo, |lo| <= ulp(hi) / 2) from the
// error-free transformations TwoSum (Knuth) and TwoProd (one FMA).  The
// per-sphere value path uses it instead of double: FP64 throughput is a small
// fraction of FP32 on this GPU.
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ FF two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// (ah + al) * (bh + bl), dropping al * bl.
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  FF p = two_prod(a.hi, b.hi);
  p.lo = __fadd_rn(p.lo, __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi)));
  return p;
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return s;
}

__device__ __forceinline__ uint32_t pack_range(int lo, int hi) {
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

// Scene owning a global index: the last scene whose first index is at most
// the given one (begin offsets ascend; an empty scene shares its begin with
// the next scene and is never returned for an index it does not own).
__device__ __forceinline__ int scene_of_tile(const SceneDev* scenes, int n_scenes, int64_t tile) {
  int lo = 0, hi = n_scenes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (scenes[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int scene_of_sphere(const SceneDev* scenes, int n_scenes, int64_t i) {
  int lo = 0, hi = n_scenes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (scenes[mid].sphere_begin <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Block-wide exclusive scan of one value per thread (kThreads or 1024 threads).
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot,
                                                         uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < NT / 32 ? warp_tot[lane] : 0;
    uint32_t s = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NT / 32) warp_tot[lane] = s - w;
    if (lane == NT / 32 - 1) warp_tot[32] = s;
  }
  __syncthreads();
  uint32_t r = warp_tot[warp] + x - v;
  total = warp_tot[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ----------------------------------------------------------------------------
// host-side launch helpers (defined in the .cu files)
// ----------------------------------------------------------------------------

// Host-side validation of one scene's parameters (the checks every
// single-scene entry point makes first).
pulsar_status validate_params(const pulsar_params* p);

cudaError_t launch_setup(const WsView& v, const SceneDev* host_scenes, int n, cudaStream_t st);
cudaError_t launch_project(const WsView& v, cudaStream_t st);
cudaError_t launch_bin(const WsView& v, int tile_bits, cudaStream_t st);
cudaError_t launch_block_lists(const WsView& v, cudaStream_t st);
cudaError_t launch_count_tests(const WsView& v, cudaStream_t st);
cudaError_t launch_background(const WsView& v, bool backward, uint32_t grad_mask, cudaStream_t st);
cudaError_t launch_render_fwd(const WsView& v, cudaStream_t st);
cudaError_t launch_track_pass(const WsView& v, cudaStream_t st);
cudaError_t launch_render_bwd(const WsView& v, uint32_t grad_mask, cudaStream_t st);
cudaError_t launch_finalize(const WsView& v, uint32_t grad_mask, cudaStream_t st);
cudaError_t launch_camera_reduce(const WsView& v, uint32_t grad_mask, cudaStream_t st);
cudaError_t launch_zero_grads(const WsView& v, uint32_t grad_mask, cudaStream_t st);

}  // namespace pulsar
