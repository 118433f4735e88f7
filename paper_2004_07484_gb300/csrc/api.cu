// Host side of the C ABI declared in include/pulsar.h: argument validation,
// the workspace layout, and the launch sequence of each entry point.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "pulsar_internal.cuh"

namespace pulsar {
namespace {

constexpr size_t kAlign = 256;

// A second stream per device for launches that may overlap the main
// sequence, with its fork and join events; created on first use.  The mutex
// makes each fork - launch - join sequence atomic among host threads (a
// stream wait binds to the event's latest record when it is issued).
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
std::mutex g_side_mutex;
SideStream g_side[64];

cudaError_t side_stream(SideStream*& out) {   // call with g_side_mutex held
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  SideStream& sd = g_side[dev];
  if (!sd.s) {
    SideStream made;
    e = cudaStreamCreateWithFlags(&made.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&made.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&made.join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      if (made.join) cudaEventDestroy(made.join);
      if (made.fork) cudaEventDestroy(made.fork);
      if (made.s) cudaStreamDestroy(made.s);
      return e;
    }
    sd = made;
  }
  out = &sd;
  return cudaSuccess;
}

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t hdr, scenes, rec0, rec1, rec2, key0, key1, val0, val1, hist, block_sums, pkey0, pkey1, pval0,
      pval1, radix_tot, ranges, item_begin, item_desc, item_order, unit_list, unit_count, unit_cost, unit_order, unit_tests, tile_done, partial, item_kappa, tile_bg, pix_aux, fres,
      gacc, pg_cnt, pg_opa, pg_feat, fin_part, red_part, cam_done, total;
  int64_t n_spheres, n_tiles, n_pixels, capacity, max_items;
  int32_t sort_blocks, fin_blocks, tile_bits, segment, part_fields;
};

bool tiles_of(const pulsar_params& p, int& tx, int& ty) {
  tx = (p.width + kTile - 1) / kTile;
  ty = (p.height + kTile - 1) / kTile;
  return true;
}

pulsar_status validate(const pulsar_params* p) {
  if (!p) return PULSAR_ERR_INVALID_ARG;
  if (p->width < 1 || p->width > 65535 || p->height < 1 || p->height > 65535)
    return PULSAR_ERR_INVALID_ARG;
  if (p->n_spheres < 0 || p->n_channels < 1 || p->n_track < 1 || p->list_capacity < 0)
    return PULSAR_ERR_INVALID_ARG;
  if (p->n_channels > 32 || p->n_track > 32) return PULSAR_ERR_UNSUPPORTED;
  if (p->tile != kTile) return PULSAR_ERR_UNSUPPORTED;
  if (p->list_capacity > (int64_t)INT32_MAX - kSortTile) return PULSAR_ERR_UNSUPPORTED;
  if (!(p->gamma >= 1e-5f && p->gamma <= 1.0f)) return PULSAR_ERR_INVALID_ARG;
  if (!(p->eps >= 0.0f) || !(p->znear > 0.0f) || !(p->zfar > p->znear)) return PULSAR_ERR_INVALID_ARG;
  if (p->flags & ~(uint32_t)(PULSAR_FLAG_STORE_HITS | PULSAR_FLAG_DIST_LITERAL | PULSAR_FLAG_NO_MIN_SIZE |
                             PULSAR_FLAG_PERSISTENT | PULSAR_FLAG_ACCUMULATE | PULSAR_FLAG_PAPER_GRADIENTS |
                             PULSAR_FLAG_ORTHOGRAPHIC | PULSAR_FLAG_PAPER_STOP))
    return PULSAR_ERR_INVALID_ARG;
  if (p->segment != 0 && (p->segment < 32 || p->segment > 65536 || p->segment % 32 != 0))
    return PULSAR_ERR_INVALID_ARG;
  if (!(p->min_contrib >= 0.0f && p->min_contrib < 1.0f)) return PULSAR_ERR_INVALID_ARG;
  return PULSAR_OK;
}

Layout make_layout(const pulsar_params* ps, int n) {
  Layout L;
  memset(&L, 0, sizeof(L));
  int64_t M = 0, NT = 0, P = 0, cap = 0;
  int fin = 0;
  const int C = ps[0].n_channels;
  const int K = ps[0].n_track;
  for (int s = 0; s < n; ++s) {
    int tx, ty;
    tiles_of(ps[s], tx, ty);
    M += ps[s].n_spheres;
    NT += (int64_t)tx * ty;
    P += (int64_t)ps[s].width * ps[s].height;
    cap += ps[s].list_capacity;
    fin += (ps[s].n_spheres + kFinalizeThreads - 1) / kFinalizeThreads;
  }
  L.n_spheres = M;
  L.n_tiles = NT;
  L.n_pixels = P;
  L.capacity = cap;
  L.fin_blocks = fin;
  L.sort_blocks = (int32_t)((std::max<int64_t>(std::max<int64_t>(M, cap), 1) + kSortTile - 1) / kSortTile);
  int bits = 1;
  while (bits < 32 && ((int64_t)1 << bits) < NT) ++bits;
  L.tile_bits = bits;
  L.segment = ps[0].segment > 0 ? ps[0].segment : kDefaultSegment;
  L.max_items = NT + (cap + L.segment - 1) / L.segment;
  L.part_fields = 6 + C + 2 * K;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  L.hdr = take(sizeof(WsHeader));
  L.scenes = take(sizeof(SceneDev) * kMaxScenes);
  L.rec0 = take(16 * (size_t)M);
  L.rec1 = take(16 * (size_t)M);
  L.rec2 = take(16 * (size_t)M);
  L.key0 = take(4 * (size_t)M);
  L.key1 = take(4 * (size_t)M);
  L.val0 = take(4 * (size_t)M);
  L.val1 = take(4 * (size_t)M);
  L.hist = take(4 * (size_t)std::max(kRadix, kDepthRadix) * L.sort_blocks);
  L.block_sums = take(4 * (size_t)L.sort_blocks);
  L.radix_tot = take(4 * (size_t)std::max(kRadix, kDepthRadix));
  L.pkey0 = take(4 * (size_t)cap);
  L.pkey1 = take(4 * (size_t)cap);
  L.pval0 = take(4 * (size_t)cap);
  L.pval1 = take(4 * (size_t)cap);
  L.ranges = take(8 * (size_t)NT);
  L.item_begin = take(4 * (size_t)(NT + 1));
  L.item_desc = take(sizeof(ItemDesc) * (size_t)L.max_items);
  L.item_order = take(4 * (size_t)L.max_items);
  // block lists: per pixel block, one slot per pair of capacity; per work unit a count
  L.unit_list = take(8 * 8 * (size_t)cap);
  L.unit_count = take(4 * 8 * (size_t)L.max_items);
  L.unit_cost = take(4 * 8 * (size_t)L.max_items);
  L.unit_order = take(4 * 8 * (size_t)L.max_items);
  L.unit_tests = take(4 * 8 * 32 * (size_t)L.max_items);
  // per (tile or work item) x 8 pixel blocks of 32 pixels
  L.tile_done = take(4 * 8 * (size_t)NT);
  L.partial = take(4 * 8 * (size_t)L.max_items * 32 * L.part_fields);
  L.item_kappa = take(4 * 8 * (size_t)L.max_items);
  L.tile_bg = take(4 * 8 * (size_t)NT * C);
  L.pix_aux = take(16 * (size_t)P);
  L.fres = take(4 * (size_t)P * C);
  L.gacc = take(16 * (size_t)M);
  // paper gradients: per sphere its tracked pixels and the opacity and feature sums
  const bool paper = (ps[0].flags & PULSAR_FLAG_PAPER_GRADIENTS) != 0;
  L.pg_cnt = take(paper ? 4 * (size_t)M : 0);
  L.pg_opa = take(paper ? 4 * (size_t)M : 0);
  L.pg_feat = take(paper ? 4 * (size_t)M * C : 0);
  L.fin_part = take(4 * (size_t)kCamPartials * std::max(fin, 1));
  L.red_part = take(4 * (size_t)n * 64 * 45);
  L.cam_done = take(4 * (size_t)kMaxScenes);
  L.total = off;
  return L;
}

WsView make_view(void* ws, const Layout& L, const pulsar_params* ps, int n) {
  char* b = static_cast<char*>(ws);
  WsView v;
  memset(&v, 0, sizeof(v));
  v.hdr = reinterpret_cast<WsHeader*>(b + L.hdr);
  v.scenes = reinterpret_cast<SceneDev*>(b + L.scenes);
  v.n_scenes = n;
  v.n_spheres = L.n_spheres;
  v.n_tiles = L.n_tiles;
  v.n_pixels = L.n_pixels;
  v.capacity = L.capacity;
  v.sort_blocks = L.sort_blocks;
  v.fin_blocks = L.fin_blocks;
  v.n_channels = ps[0].n_channels;
  v.n_track = ps[0].n_track;
  const int tile_rb = tile_radix_bits(L.tile_bits);
  v.pair_buf = ((L.tile_bits + tile_rb - 1) / tile_rb) & 1;
  v.segment = L.segment;
  v.max_items = (int32_t)L.max_items;
  v.part_fields = L.part_fields;
  v.persistent = (ps[0].flags & PULSAR_FLAG_PERSISTENT) ? 1 : 0;
  v.paper = (ps[0].flags & PULSAR_FLAG_PAPER_GRADIENTS) ? 1 : 0;
  // the paper's early termination follows a pixel's denominator along its
  // whole list: one render unit walks every segment of its tile in order
  v.chain = (ps[0].flags & PULSAR_FLAG_PAPER_STOP) ? 1 : 0;
  // depth sort keys: visible keys lie strictly between a scene's planes, so
  // their float bits minus those of the batch's smallest znear lie in
  // (0, top - base), top the bits of the largest zfar; culled spheres take
  // top - base, the passes cover the bits of that range
  {
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (int s = 0; s < n; ++s) {
      uint32_t a, z;
      memcpy(&a, &ps[s].znear, 4);
      memcpy(&z, &ps[s].zfar, 4);
      lo = std::min(lo, a);
      hi = std::max(hi, z);
    }
    v.key_base = lo;
    v.key_culled = hi - lo;
    int bits = 1;
    while (bits < 32 && (v.key_culled >> bits) != 0u) ++bits;
    v.key_bits = bits;
    v.sort_buf = ((bits + kDepthRadixBits - 1) / kDepthRadixBits) & 1;
  }
  v.rec0 = reinterpret_cast<float4*>(b + L.rec0);
  v.rec1 = reinterpret_cast<float4*>(b + L.rec1);
  v.rec2 = reinterpret_cast<float4*>(b + L.rec2);
  v.key[0] = reinterpret_cast<uint32_t*>(b + L.key0);
  v.key[1] = reinterpret_cast<uint32_t*>(b + L.key1);
  v.val[0] = reinterpret_cast<uint32_t*>(b + L.val0);
  v.val[1] = reinterpret_cast<uint32_t*>(b + L.val1);
  v.hist = reinterpret_cast<uint32_t*>(b + L.hist);
  v.block_sums = reinterpret_cast<uint32_t*>(b + L.block_sums);
  v.radix_tot = reinterpret_cast<uint32_t*>(b + L.radix_tot);
  v.pkey[0] = reinterpret_cast<uint32_t*>(b + L.pkey0);
  v.pkey[1] = reinterpret_cast<uint32_t*>(b + L.pkey1);
  v.pval[0] = reinterpret_cast<uint32_t*>(b + L.pval0);
  v.pval[1] = reinterpret_cast<uint32_t*>(b + L.pval1);
  v.ranges = reinterpret_cast<int2*>(b + L.ranges);
  v.item_begin = reinterpret_cast<int32_t*>(b + L.item_begin);
  v.item_desc = reinterpret_cast<ItemDesc*>(b + L.item_desc);
  v.item_order = reinterpret_cast<int32_t*>(b + L.item_order);
  v.unit_list = reinterpret_cast<uint2*>(b + L.unit_list);
  v.unit_count = reinterpret_cast<int32_t*>(b + L.unit_count);
  v.unit_cost = reinterpret_cast<uint32_t*>(b + L.unit_cost);
  v.unit_order = reinterpret_cast<int32_t*>(b + L.unit_order);
  v.unit_tests = reinterpret_cast<int32_t*>(b + L.unit_tests);
  v.tile_done = reinterpret_cast<int32_t*>(b + L.tile_done);
  v.partial = reinterpret_cast<float*>(b + L.partial);
  v.item_kappa = reinterpret_cast<float*>(b + L.item_kappa);
  v.tile_bg = reinterpret_cast<float*>(b + L.tile_bg);
  v.pix_aux = reinterpret_cast<float4*>(b + L.pix_aux);
  v.fres = reinterpret_cast<float*>(b + L.fres);
  v.gacc = reinterpret_cast<float4*>(b + L.gacc);
  v.pg_cnt = reinterpret_cast<int32_t*>(b + L.pg_cnt);
  v.pg_opa = reinterpret_cast<float*>(b + L.pg_opa);
  v.pg_feat = reinterpret_cast<float*>(b + L.pg_feat);
  v.fin_part = reinterpret_cast<float*>(b + L.fin_part);
  v.red_part = reinterpret_cast<float*>(b + L.red_part);
  v.cam_done = reinterpret_cast<int32_t*>(b + L.cam_done);
  return v;
}

// Host copies of the per-scene descriptors (sizes and offsets; pointers are
// filled per entry point).
void fill_scenes(const pulsar_params* ps, const pulsar_scene* sc, int n, SceneDev* out) {
  int64_t sb = 0, tb = 0, pb = 0;
  int fb = 0;
  for (int s = 0; s < n; ++s) {
    SceneDev& d = out[s];
    memset(&d, 0, sizeof(d));
    const pulsar_params& p = ps[s];
    if (sc) {
      d.pos = sc[s].pos;
      d.rad = sc[s].rad;
      d.opa = sc[s].opa;
      d.feat = sc[s].feat;
      d.cam = sc[s].cam;
      d.bg = sc[s].bg;
    }
    d.width = p.width;
    d.height = p.height;
    d.n_spheres = p.n_spheres;
    d.n_channels = p.n_channels;
    d.n_track = p.n_track;
    d.flags = p.flags;
    {
      // ln(tau / (1 - tau)) of the paper's early termination
      const double tau = p.min_contrib > 0.0f ? (double)p.min_contrib : 0.01;
      d.stop_log_ratio = (float)std::log(tau / (1.0 - tau));
    }
    tiles_of(p, d.tiles_x, d.tiles_y);
    d.sphere_begin = sb;
    d.tile_begin = tb;
    d.pixel_begin = pb;
    d.fin_block_begin = fb;
    d.fin_blocks = (p.n_spheres + kFinalizeThreads - 1) / kFinalizeThreads;
    d.gamma = p.gamma;
    d.eps = p.eps;
    d.znear = p.znear;
    d.zfar = p.zfar;
    sb += p.n_spheres;
    tb += (int64_t)d.tiles_x * d.tiles_y;
    pb += (int64_t)p.width * p.height;
    fb += d.fin_blocks;
  }
}

// A batch is valid when every scene is, and the scenes share the settings
// the kernels are specialised on.
pulsar_status validate_batch(int n, const pulsar_params* ps) {
  if (n < 1 || n > kMaxScenes || !ps) return n > kMaxScenes ? PULSAR_ERR_UNSUPPORTED : PULSAR_ERR_INVALID_ARG;
  int64_t M = 0, cap = 0;
  for (int s = 0; s < n; ++s) {
    pulsar_status st = validate(&ps[s]);
    if (st != PULSAR_OK) return st;
    if (ps[s].n_channels != ps[0].n_channels || ps[s].n_track != ps[0].n_track ||
        ps[s].tile != ps[0].tile || ps[s].flags != ps[0].flags || ps[s].segment != ps[0].segment)
      return PULSAR_ERR_INVALID_ARG;
    M += ps[s].n_spheres;
    cap += ps[s].list_capacity;
  }
  if (M > (int64_t)INT32_MAX - kSortTile || cap > (int64_t)INT32_MAX - kSortTile) return PULSAR_ERR_UNSUPPORTED;
  int64_t nt = 0;
  for (int s = 0; s < n; ++s) {
    int tx, ty;
    tiles_of(ps[s], tx, ty);
    nt += (int64_t)tx * ty;
  }
  if (nt > ((int64_t)1 << kTileKeyBits)) return PULSAR_ERR_UNSUPPORTED;   // tile index bits of a pair key
  return PULSAR_OK;
}

pulsar_status check_ws(int n, const pulsar_params* p, void* ws, size_t bytes, Layout& L) {
  pulsar_status st = validate_batch(n, p);
  if (st != PULSAR_OK) return st;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return PULSAR_ERR_INVALID_ARG;
  L = make_layout(p, n);
  if (bytes < L.total) return PULSAR_ERR_CAPACITY;
  return PULSAR_OK;
}

bool scene_ok(const pulsar_params* p, const pulsar_scene* s) {
  if (!s || !s->cam || !s->bg) return false;
  if (p->n_spheres > 0 && (!s->pos || !s->rad || !s->opa || !s->feat)) return false;
  return true;
}

bool scenes_ok(int n, const pulsar_params* p, const pulsar_scene* s) {
  if (!s) return false;
  for (int k = 0; k < n; ++k)
    if (!scene_ok(&p[k], &s[k])) return false;
  return true;
}

pulsar_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PULSAR_OK : PULSAR_ERR_CUDA; }

pulsar_status project_n(int n, const pulsar_params* params, const pulsar_scene* scenes, void* ws,
                        size_t bytes, cudaStream_t s) {
  Layout L;
  pulsar_status st = check_ws(n, params, ws, bytes, L);
  if (st != PULSAR_OK) return st;
  if (!scenes_ok(n, params, scenes)) return PULSAR_ERR_INVALID_ARG;
  WsView v = make_view(ws, L, params, n);
  SceneDev d[kMaxScenes];
  fill_scenes(params, scenes, n, d);
  cudaError_t e = launch_setup(v, d, n, s);
  if (e == cudaSuccess) e = launch_project(v, s);
  return cuda_status(e);
}

pulsar_status bin_n(int n, const pulsar_params* params, void* ws, size_t bytes, cudaStream_t s) {
  Layout L;
  pulsar_status st = check_ws(n, params, ws, bytes, L);
  if (st != PULSAR_OK) return st;
  WsView v = make_view(ws, L, params, n);
  return cuda_status(launch_bin(v, L.tile_bits, s));
}

pulsar_status fwd_n(int n, const pulsar_params* params, const pulsar_scene* scenes, void* ws,
                    size_t bytes, const pulsar_fwd_out* out, cudaStream_t s) {
  Layout L;
  pulsar_status st = check_ws(n, params, ws, bytes, L);
  if (st != PULSAR_OK) return st;
  if (!scenes_ok(n, params, scenes) || !out) return PULSAR_ERR_INVALID_ARG;
  for (int k = 0; k < n; ++k)
    if (!out[k].image || !out[k].log_norm) return PULSAR_ERR_INVALID_ARG;
  WsView v = make_view(ws, L, params, n);
  SceneDev d[kMaxScenes];
  fill_scenes(params, scenes, n, d);
  for (int k = 0; k < n; ++k) {
    d[k].image = out[k].image;
    d[k].log_norm = out[k].log_norm;
    d[k].n_hits = out[k].n_hits;
    d[k].n_tests = out[k].n_tests;
    d[k].tracked = out[k].tracked;
  }
  bool tests = false;
  for (int k = 0; k < n; ++k) tests = tests || out[k].n_tests != nullptr;
  cudaError_t e = launch_setup(v, d, -n, s);
  if (e == cudaSuccess && tests) e = launch_count_tests(v, s);
  if (e != cudaSuccess) return cuda_status(e);
  // the pixels of empty tiles (background pass) are written on the side
  // stream while the render pass draws the others
  std::lock_guard<std::mutex> lock(g_side_mutex);
  SideStream* side = nullptr;
  e = side_stream(side);
  if (e == cudaSuccess) e = cudaEventRecord(side->fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(side->s, side->fork, 0);
  if (e == cudaSuccess) e = launch_background(v, false, 0u, side->s);
  if (e == cudaSuccess) e = cudaEventRecord(side->join, side->s);
  if (e == cudaSuccess) e = launch_render_fwd(v, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, side->join, 0);
  return cuda_status(e);
}

pulsar_status bwd_n(int n, const pulsar_params* params, const pulsar_scene* scenes, void* ws,
                    size_t bytes, const pulsar_bwd_io* io, uint32_t grad_mask, cudaStream_t s) {
  Layout L;
  pulsar_status st = check_ws(n, params, ws, bytes, L);
  if (st != PULSAR_OK) return st;
  if (!scenes_ok(n, params, scenes) || !io) return PULSAR_ERR_INVALID_ARG;
  if (grad_mask & ~(uint32_t)PULSAR_GRAD_ALL) return PULSAR_ERR_INVALID_ARG;
  // where the paper's early termination stopped a pixel is known from the
  // forward pass only
  if ((params[0].flags & PULSAR_FLAG_PAPER_STOP) && !(params[0].flags & PULSAR_FLAG_STORE_HITS))
    return PULSAR_ERR_UNSUPPORTED;
  for (int k = 0; k < n; ++k) {
    const pulsar_bwd_io& q = io[k];
    if (!q.image || !q.log_norm || !q.grad_image) return PULSAR_ERR_INVALID_ARG;
    if (params[k].n_spheres > 0) {
      if ((grad_mask & PULSAR_GRAD_POS) && !q.g_pos) return PULSAR_ERR_INVALID_ARG;
      if ((grad_mask & PULSAR_GRAD_RAD) && !q.g_rad) return PULSAR_ERR_INVALID_ARG;
      if ((grad_mask & PULSAR_GRAD_OPA) && !q.g_opa) return PULSAR_ERR_INVALID_ARG;
      if ((grad_mask & PULSAR_GRAD_FEAT) && !q.g_feat) return PULSAR_ERR_INVALID_ARG;
    }
    if ((grad_mask & PULSAR_GRAD_CAM) && !q.g_cam) return PULSAR_ERR_INVALID_ARG;
    if ((grad_mask & PULSAR_GRAD_BG) && !q.g_bg) return PULSAR_ERR_INVALID_ARG;
  }
  WsView v = make_view(ws, L, params, n);
  SceneDev d[kMaxScenes];
  fill_scenes(params, scenes, n, d);
  for (int k = 0; k < n; ++k) {
    const pulsar_bwd_io& q = io[k];
    d[k].image_in = q.image;
    d[k].log_norm_in = q.log_norm;
    d[k].grad_image = q.grad_image;
    d[k].g_pos = q.g_pos;
    d[k].g_rad = q.g_rad;
    d[k].g_opa = q.g_opa;
    d[k].g_feat = q.g_feat;
    d[k].g_cam = q.g_cam;
    d[k].g_bg = q.g_bg;
  }
  cudaError_t e = launch_setup(v, d, -n, s);
  if (e != cudaSuccess) return cuda_status(e);
  // the background-gradient partials of empty tiles are summed on the side
  // stream while the render pass runs; the camera reduction joins them
  std::lock_guard<std::mutex> lock(g_side_mutex);
  SideStream* side = nullptr;
  const bool bg = (grad_mask & PULSAR_GRAD_BG) != 0;
  if (bg) {
    e = side_stream(side);
    if (e == cudaSuccess) e = cudaEventRecord(side->fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side->s, side->fork, 0);
    if (e == cudaSuccess) e = launch_background(v, true, grad_mask, side->s);
    if (e == cudaSuccess) e = cudaEventRecord(side->join, side->s);
  }
  if (e == cudaSuccess) e = launch_zero_grads(v, grad_mask, s);
  const bool geo_or_values = (grad_mask & ~(uint32_t)PULSAR_GRAD_BG) != 0;
  if (e == cudaSuccess && geo_or_values && !(params[0].flags & PULSAR_FLAG_STORE_HITS))
    e = launch_track_pass(v, s);
  if (e == cudaSuccess) e = launch_render_bwd(v, grad_mask, s);
  if (e == cudaSuccess) e = launch_finalize(v, grad_mask, s);
  if (e == cudaSuccess && bg) e = cudaStreamWaitEvent(s, side->join, 0);
  if (e == cudaSuccess) e = launch_camera_reduce(v, grad_mask, s);
  return cuda_status(e);
}

pulsar_status read_lists_n(int n, const pulsar_params* params, void* ws, size_t bytes,
                           int32_t* ranges, int32_t* ids, cudaStream_t s) {
  Layout L;
  pulsar_status st = check_ws(n, params, ws, bytes, L);
  if (st != PULSAR_OK) return st;
  if (!ranges || (!ids && L.capacity > 0)) return PULSAR_ERR_INVALID_ARG;
  WsView v = make_view(ws, L, params, n);
  cudaError_t e = cudaMemcpyAsync(ranges, v.ranges, sizeof(int2) * (size_t)L.n_tiles,
                                  cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && L.capacity > 0)
    e = cudaMemcpyAsync(ids, v.pval[v.pair_buf], sizeof(int32_t) * (size_t)L.capacity,
                        cudaMemcpyDeviceToDevice, s);
  return cuda_status(e);
}

}  // namespace

pulsar_status validate_params(const pulsar_params* p) { return validate_batch(1, p); }

}  // namespace pulsar

using namespace pulsar;

extern "C" size_t pulsar_workspace_size(const pulsar_params* params) {
  return pulsar_workspace_size_batched(1, params);
}

extern "C" size_t pulsar_workspace_size_batched(int n_scenes, const pulsar_params* params) {
  if (validate_batch(n_scenes, params) != PULSAR_OK) return 0;
  return make_layout(params, n_scenes).total;
}

extern "C" pulsar_status pulsar_project(const pulsar_params* params, const pulsar_scene* scene,
                                        void* workspace, size_t workspace_bytes, void* stream) {
  return project_n(1, params, scene, workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

extern "C" pulsar_status pulsar_project_batched(int n_scenes, const pulsar_params* params,
                                                const pulsar_scene* scenes, void* workspace,
                                                size_t workspace_bytes, void* stream) {
  return project_n(n_scenes, params, scenes, workspace, workspace_bytes,
                   static_cast<cudaStream_t>(stream));
}

extern "C" pulsar_status pulsar_bin(const pulsar_params* params, void* workspace,
                                    size_t workspace_bytes, void* stream) {
  return bin_n(1, params, workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

extern "C" pulsar_status pulsar_bin_batched(int n_scenes, const pulsar_params* params,
                                            void* workspace, size_t workspace_bytes, void* stream) {
  return bin_n(n_scenes, params, workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

extern "C" pulsar_status pulsar_render_fwd(const pulsar_params* params, const pulsar_scene* scene,
                                           void* workspace, size_t workspace_bytes, float* image,
                                           float* log_norm, int32_t* n_hits, int32_t* n_tests,
                                           int32_t* tracked, void* stream) {
  const pulsar_fwd_out out = {image, log_norm, n_hits, n_tests, tracked};
  return fwd_n(1, params, scene, workspace, workspace_bytes, &out, static_cast<cudaStream_t>(stream));
}

extern "C" pulsar_status pulsar_render_fwd_batched(int n_scenes, const pulsar_params* params,
                                                   const pulsar_scene* scenes, void* workspace,
                                                   size_t workspace_bytes, const pulsar_fwd_out* out,
                                                   void* stream) {
  return fwd_n(n_scenes, params, scenes, workspace, workspace_bytes, out,
               static_cast<cudaStream_t>(stream));
}

extern "C" pulsar_status pulsar_render_bwd(const pulsar_params* params, const pulsar_scene* scene,
                                           void* workspace, size_t workspace_bytes,
                                           const float* image, const float* log_norm,
                                           const float* grad_image, uint32_t grad_mask,
                                           float* g_pos, float* g_rad, float* g_opa, float* g_feat,
                                           float* g_cam, float* g_bg, void* stream) {
  const pulsar_bwd_io io = {image, log_norm, grad_image, g_pos, g_rad, g_opa, g_feat, g_cam, g_bg};
  return bwd_n(1, params, scene, workspace, workspace_bytes, &io, grad_mask,
               static_cast<cudaStream_t>(stream));
}

extern "C" pulsar_status pulsar_render_bwd_batched(int n_scenes, const pulsar_params* params,
                                                   const pulsar_scene* scenes, void* workspace,
                                                   size_t workspace_bytes, const pulsar_bwd_io* io,
                                                   uint32_t grad_mask, void* stream) {
  return bwd_n(n_scenes, params, scenes, workspace, workspace_bytes, io, grad_mask,
               static_cast<cudaStream_t>(stream));
}

extern "C" pulsar_status pulsar_read_tile_lists(const pulsar_params* params, void* workspace,
                                                size_t workspace_bytes, int32_t* ranges,
                                                int32_t* ids, void* stream) {
  return read_lists_n(1, params, workspace, workspace_bytes, ranges, ids,
                      static_cast<cudaStream_t>(stream));
}

extern "C" pulsar_status pulsar_read_tile_lists_batched(int n_scenes, const pulsar_params* params,
                                                        void* workspace, size_t workspace_bytes,
                                                        int32_t* ranges, int32_t* ids, void* stream) {
  return read_lists_n(n_scenes, params, workspace, workspace_bytes, ranges, ids,
                      static_cast<cudaStream_t>(stream));
}

extern "C" pulsar_status pulsar_read_status(void* workspace, size_t workspace_bytes,
                                            int64_t* pairs_needed, void* stream) {
  if (!workspace || workspace_bytes < sizeof(WsHeader)) return PULSAR_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return PULSAR_ERR_CUDA;
  WsHeader h;
  if (cudaMemcpy(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PULSAR_ERR_CUDA;
  if (pairs_needed) *pairs_needed = h.pairs_needed;
  if (h.timeout) return PULSAR_ERR_TIMEOUT;
  if (h.overflow) return PULSAR_ERR_CAPACITY;
  return PULSAR_OK;
}

extern "C" pulsar_status pulsar_last_overflow(const pulsar_params* params, void* workspace,
                                              size_t workspace_bytes, size_t* needed_bytes, void* stream) {
  if (validate(params) != PULSAR_OK) return PULSAR_ERR_INVALID_ARG;
  int64_t pairs = 0;
  const pulsar_status st = pulsar_read_status(workspace, workspace_bytes, &pairs, stream);
  if (st != PULSAR_OK && st != PULSAR_ERR_CAPACITY) return st;
  if (needed_bytes) {
    pulsar_params p = *params;
    if (pairs > p.list_capacity) p.list_capacity = pairs;
    *needed_bytes = pulsar_workspace_size(&p);
  }
  return st;
}

extern "C" pulsar_status pulsar_render_batched(int n_scenes, const pulsar_params* params,
                                               const pulsar_scene* scenes, void* workspace,
                                               size_t workspace_bytes, const pulsar_fwd_out* out,
                                               void* stream) {
  pulsar_status st = pulsar_project_batched(n_scenes, params, scenes, workspace, workspace_bytes, stream);
  if (st == PULSAR_OK) st = pulsar_bin_batched(n_scenes, params, workspace, workspace_bytes, stream);
  if (st == PULSAR_OK)
    st = pulsar_render_fwd_batched(n_scenes, params, scenes, workspace, workspace_bytes, out, stream);
  return st;
}

extern "C" const char* pulsar_status_string(pulsar_status status) {
  switch (status) {
    case PULSAR_OK: return "ok";
    case PULSAR_ERR_INVALID_ARG: return "invalid argument";
    case PULSAR_ERR_CAPACITY: return "workspace or pair-list capacity too small";
    case PULSAR_ERR_CUDA: return "CUDA runtime error";
    case PULSAR_ERR_TIMEOUT: return "bounded device loop gave up";
    case PULSAR_ERR_UNSUPPORTED: return "unsupported setting";
  }
  return "unknown status";
}
