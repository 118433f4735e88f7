/*
 * pulsar.h: C ABI of the GB300-native differentiable sphere renderer.
 *
 * The renderer maps a sphere scene S = {(p_i, f_i, r_i, o_i)} and a camera
 * (R, t, K) to a feature image F = R(S, R, t, K) (Sec. 3.2, App. A of
 * Lassner & Zollhoefer, "Pulsar", arXiv 2004.07484) and back-propagates a
 * gradient dL/dF to every scene and camera parameter (App. B, "The Backward
 * Pass").  Pixel weights follow Eq. 1:
 *
 *   w_i = o_i d_i exp(o_i z_i / gamma) / (exp(eps / gamma) + sum_k o_k d_k exp(o_k z_k / gamma))
 *   F   = sum_i w_i f_i + w_B bg,   w_B = exp(eps / gamma) / D
 *
 * with z_i the normalised depth of the ray's entry point (0 = far plane) and
 * d_i the normalised distance of the ray to the sphere centre.
 *
 * Conventions shared by every entry point
 *   - All array pointers are DEVICE pointers to contiguous float32 (or int32)
 *     memory owned by the caller.  The library never allocates device memory:
 *     scratch space is the caller's workspace, sized by pulsar_workspace_size.
 *   - Calls are asynchronous on the given CUDA stream (NULL = legacy default)
 *     and never synchronise, except pulsar_read_status.
 *   - Argument errors are detected on the host and returned before anything
 *     is enqueued.  Data-dependent overflow (more (tile, sphere) pairs than
 *     list_capacity) is recorded in the workspace; the outputs of that call
 *     are then undefined and pulsar_read_status reports it.
 *   - Layouts: positions M x 3, features M x C (row-major), images H x W x C
 *     (row-major, pixel (x, y) at offset (y * W + x) * C), per-pixel planes
 *     H x W.
 *   - Camera vector, in the order printed in Listing 1 with the 6D rotation
 *     of Zhou et al. that the paper accepts natively:
 *       cam[0..2]  t, the camera centre in world coordinates
 *       cam[3..8]  a1, a2: 6D rotation; Gram-Schmidt gives the camera axes
 *                  b1 = a1/|a1|, b2 = unit(a2 - (b1.a2) b1), b3 = b1 x b2,
 *                  and the camera-space centre is c = (b1.(p-t), b2.(p-t), b3.(p-t))
 *       cam[9]     focal length f
 *       cam[10]    sensor width s; the pixel pitch on the unit image plane is
 *                  s / (W f), the principal point is the image centre, the
 *                  camera looks down +z with x to the right and y downwards.
 */
#ifndef PULSAR_H
#define PULSAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PULSAR_OK = 0,
  PULSAR_ERR_INVALID_ARG = 1,  /* a host-side argument check failed */
  PULSAR_ERR_CAPACITY = 2,     /* workspace or pair list too small */
  PULSAR_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  PULSAR_ERR_TIMEOUT = 4,      /* a bounded device loop gave up */
  PULSAR_ERR_UNSUPPORTED = 5   /* valid request the library does not handle */
} pulsar_status;

/* pulsar_params.flags */
enum {
  /* The forward pass stores, per pixel, the depth and index of the n_track-th
   * closest hit, so the backward pass reads it instead of searching again
   * (App. B, "Preparing for the Backward Pass").  Without it the backward
   * pass recomputes each pixel's tracked hits. */
  PULSAR_FLAG_STORE_HITS = 1u << 0,
  /* d_i = min(1, dist/R) as printed in Sec. 3.2; the default is
   * d_i = 1 - min(1, dist/R) (weight 1 at the centre, 0 at the rim). */
  PULSAR_FLAG_DIST_LITERAL = 1u << 1,
  /* Disable the one-pixel minimum size (App. B, Step 0). */
  PULSAR_FLAG_NO_MIN_SIZE = 1u << 2,
  /* Scheduling only (results are unchanged): the render passes run as
   * persistent kernels, one resident CTA per slot, each taking work items
   * from a counter, instead of one CTA per work item. */
  PULSAR_FLAG_PERSISTENT = 1u << 3,
  /* The backward pass adds its gradients into the caller's gradient buffers
   * instead of overwriting them (the caller zeroes them when it wants plain
   * gradients).  Scenes of one batch may then share gradient buffers: views
   * of one sphere set, rendered as a batch, accumulate the gradient of a loss
   * summed over views (Sec. 3.4).  Every output is added with atomics, so
   * shared buffers are safe; the summation order is unspecified. */
  PULSAR_FLAG_ACCUMULATE = 1u << 4,
  /* The paper's gradient normalisations (App. B, end of "The Backward Pass";
   * Sec. 6), in place of the plain gradients: every sphere gradient is
   * divided by the number of pixels at which the sphere is a tracked hit;
   * position and radius gradients are zero unless the sphere's projected
   * radius R / (c_z k) exceeds 3 pixels; the camera gradient is the
   * area-weighted sum of the averaged per-sphere terms times 1e-3, which with
   * the area taken as the sphere's tracked pixels is 1e-3 times the plain
   * camera gradient.  The background gradient is unchanged. */
  PULSAR_FLAG_PAPER_GRADIENTS = 1u << 5,
  /* Orthographic camera (Sec. 1: "pinhole and orthogonal camera model"):
   * pixel (u, v) sees along +z from (rho_x, rho_y, 0) in camera space, rho =
   * ((u + 1/2 - W/2) k, (v + 1/2 - H/2) k) with k = sensor_width / W; the
   * focal length does not enter.  The minimum size is R = max(r, 0.75 k). */
  PULSAR_FLAG_ORTHOGRAPHIC = 1u << 6,
  /* The paper's early termination (App. B, Step 2; an approximation, the
   * paper's default), on top of the exact one: a pixel takes its hits in list
   * order (sort key, then index) and stops before the first hit whose largest
   * possible weight e^{o_max z_k / g} / (D + e^{o_max z_k / g}) is below
   * min_contrib (the paper's "n percent" as a fraction, 1 % by default),
   * z_k the depth term of the sphere's sort key, o_max the largest |o| of
   * the scene's visible spheres and D the denominator of Eq. 1 over the hits
   * taken; blending and tracking see only the hits taken.  The decision is
   * taken in float32.  A render unit then walks every segment of its tile's
   * list in order, and the backward pass needs PULSAR_FLAG_STORE_HITS
   * (without it PULSAR_ERR_UNSUPPORTED): the forward pass records where each
   * pixel stopped.  Forward and backward calls take the same flags. */
  PULSAR_FLAG_PAPER_STOP = 1u << 7
};

/* grad_mask bits of pulsar_render_bwd: gradients are computed only where
 * requested (App. B, end of "The Backward Pass"). */
enum {
  PULSAR_GRAD_POS = 1u << 0,
  PULSAR_GRAD_RAD = 1u << 1,
  PULSAR_GRAD_OPA = 1u << 2,
  PULSAR_GRAD_FEAT = 1u << 3,
  PULSAR_GRAD_CAM = 1u << 4,
  PULSAR_GRAD_BG = 1u << 5,
  PULSAR_GRAD_ALL = 63u
};

/* Per-scene settings.  Host memory, read during the call only. */
typedef struct {
  int32_t width, height;   /* image size; 1..65535 (App. B stores the sphere
                              rectangle in 16-bit fields) */
  int32_t n_spheres;       /* M >= 0 */
  int32_t n_channels;      /* C = feature length, 1..32 */
  int32_t n_track;         /* closest hits kept per pixel for the backward
                              pass (App. B, Step 2), 1..32 */
  int32_t tile;            /* screen tile edge in pixels; 16 */
  int64_t list_capacity;   /* maximum number of (tile, sphere) pairs */
  float gamma;             /* blending sharpness, [1e-5, 1] (Sec. 3.2) */
  float eps;               /* background offset eps of Eq. 1, >= 0 */
  float znear, zfar;       /* depth range mapped to z in [0, 1]; 0 < znear < zfar */
  uint32_t flags;          /* PULSAR_FLAG_* */
  int32_t segment;         /* scheduling only: list entries per work item of the
                              render passes (a tile's list is split into segments
                              rendered in parallel and merged); 0 = 1024, else a
                              multiple of 32 in [32, 65536] */
  float min_contrib;       /* PULSAR_FLAG_PAPER_STOP: the fraction of the blend below
                              which a hit stops a pixel, in [0, 1); 0 = 0.01, the
                              paper's default.  Ignored without the flag. */
} pulsar_params;

/* Scene inputs: device pointers, float32, contiguous. */
typedef struct {
  const float* pos;   /* M x 3 sphere centres p_i */
  const float* rad;   /* M radii r_i */
  const float* opa;   /* M opacities o_i */
  const float* feat;  /* M x C feature vectors f_i */
  const float* cam;   /* 11 camera values (layout above) */
  const float* bg;    /* C background features */
} pulsar_scene;

/* Bytes of device workspace a render with these settings needs (0 when the
 * settings are invalid).  The workspace holds the projected sphere records,
 * sort buffers, the (tile, sphere) pair lists, tile ranges, per-pixel
 * backward data and gradient accumulators.  It must be 256-byte aligned. */
size_t pulsar_workspace_size(const pulsar_params* params);

/* Step 0 of App. B: projects every sphere through the pinhole camera.
 * Writes, into the workspace, a 32-byte draw record per sphere (camera-space
 * centre, squared effective radius, earliest intersection depth, opacity and
 * the inclusive pixel rectangle) and the sort key (the earliest depth, +inf
 * for culled spheres). */
pulsar_status pulsar_project(const pulsar_params* params, const pulsar_scene* scene,
                             void* workspace, size_t workspace_bytes, void* stream);

/* Builds the per-tile sphere lists (App. B, Step 1, replacing the paper's
 * nine-part split and flag compaction): sorts spheres by (earliest depth,
 * index), emits one (tile, sphere) pair per tile each sphere's rectangle
 * overlaps, and sorts pairs stably by tile, so every tile's list is ordered
 * by (earliest depth, index).  Requires pulsar_project on the same workspace. */
pulsar_status pulsar_bin(const pulsar_params* params, void* workspace, size_t workspace_bytes,
                         void* stream);

/* Forward pass (App. B, Steps 1-2): per pixel, intersects the tile's spheres
 * in list order, blends every hit by Eq. 1 and tracks the n_track closest.
 *   image      H x W x C output F
 *   log_norm   H x W output, log of Eq. 1's denominator D (needed by the
 *              backward pass)
 *   n_hits     optional (may be NULL) H x W int32: hits blended
 *   n_tests    optional (may be NULL) H x W int32: ray-sphere tests made
 *              (spheres whose rectangle contains the pixel)
 *   tracked    optional (may be NULL) H x W x n_track int32: indices of the
 *              tracked hits, closest first (by depth, then index), -1 padded
 * Requires pulsar_bin on the same workspace. */
pulsar_status pulsar_render_fwd(const pulsar_params* params, const pulsar_scene* scene,
                                void* workspace, size_t workspace_bytes, float* image,
                                float* log_norm, int32_t* n_hits, int32_t* n_tests,
                                int32_t* tracked, void* stream);

/* Backward pass (App. B, "The Backward Pass"): given G = dL/dF, returns the
 * gradients through each pixel's tracked hits.  Outputs selected by grad_mask
 * are overwritten (zeroed in-stream first), or added into with
 * PULSAR_FLAG_ACCUMULATE; the others may be NULL.
 *   image, log_norm   the forward outputs of the same call sequence
 *   grad_image        H x W x C upstream gradient
 *   g_pos M x 3, g_rad M, g_opa M, g_feat M x C, g_cam 11, g_bg C
 * Requires pulsar_render_fwd on the same workspace (and, without
 * PULSAR_FLAG_STORE_HITS, the unchanged tile lists of pulsar_bin). */
pulsar_status pulsar_render_bwd(const pulsar_params* params, const pulsar_scene* scene,
                                void* workspace, size_t workspace_bytes, const float* image,
                                const float* log_norm, const float* grad_image, uint32_t grad_mask,
                                float* g_pos, float* g_rad, float* g_opa, float* g_feat,
                                float* g_cam, float* g_bg, void* stream);

/* Copies the per-tile sphere lists built by pulsar_bin (App. B, Step 1) out
 * of the workspace, asynchronously on the stream:
 *   ranges  n_tiles x 2 int32 device array: [begin, end) of each tile's list
 *           (tiles row-major, ceil(W/tile) per row; empty tiles get [0, 0))
 *   ids     list_capacity int32 device array: sphere indices, each tile's
 *           list ordered by (earliest depth, index)
 * Valid only when the last pulsar_bin did not overflow. */
pulsar_status pulsar_read_tile_lists(const pulsar_params* params, void* workspace,
                                     size_t workspace_bytes, int32_t* ranges, int32_t* ids,
                                     void* stream);

/* Synchronises the stream, then reads the workspace's device flags.
 * Returns PULSAR_ERR_CAPACITY when the last pulsar_bin overflowed
 * list_capacity; *pairs_needed (may be NULL) receives the pair count the
 * last pulsar_bin required. */
pulsar_status pulsar_read_status(void* workspace, size_t workspace_bytes, int64_t* pairs_needed,
                                 void* stream);

/* The overflow check in workspace terms: synchronises the stream, and when
 * the last pulsar_bin overflowed list_capacity returns PULSAR_ERR_CAPACITY
 * and writes through needed_bytes (may be NULL) the workspace bytes these
 * params need with list_capacity raised to the pairs that binning required.
 * Returns PULSAR_OK (needed_bytes = the current requirement) otherwise. */
pulsar_status pulsar_last_overflow(const pulsar_params* params, void* workspace,
                                   size_t workspace_bytes, size_t* needed_bytes, void* stream);

/* Size of the device array pulsar_render_fwd_static uses as its workspace. */
#define PULSAR_STATIC_WORKSPACE_BYTES (64u << 20)

/* Forward render without a caller-provided workspace and without allocating
 * (the paper has no counterpart; this exists for callers that cannot
 * allocate device memory when they render, e.g. code running where another
 * component owns the device memory, or code that must avoid the device-wide
 * synchronisation cudaFree can cause).
 *   Runs pulsar_project, pulsar_bin and pulsar_render_fwd with a 64 MiB
 *   device array inside the library as the workspace.  Inputs and outputs
 *   are the caller's, as for pulsar_render_fwd.
 *   Validates params exactly as pulsar_render_fwd does (same status codes),
 *   then returns PULSAR_ERR_CAPACITY, before enqueuing anything, when
 *   pulsar_workspace_size(params) exceeds PULSAR_STATIC_WORKSPACE_BYTES.
 *   The array is shared by every call in the process and keeps the last
 *   call's contents; calls that overlap on the GPU (other streams, other
 *   threads) race on it and must be serialised by the caller.
 *   Its device address is looked up in the current context on every call
 *   (valid across device resets); the first call on a device loads the
 *   library's module there, so make it before any stream capture.
 *   A list_capacity overflow (the image is then background only) is read
 *   back with pulsar_static_read_status. */
pulsar_status pulsar_render_fwd_static(const pulsar_params* params, const pulsar_scene* scene,
                                       float* image, float* log_norm, void* stream);

/* Status of the last pulsar_render_fwd_static call on the current device, as
 * pulsar_read_status reports it for a caller workspace: PULSAR_OK, or
 * PULSAR_ERR_CAPACITY after a list_capacity overflow, with the pair count the
 * call needed in *pairs_needed (may be NULL).  Synchronises the stream. */
pulsar_status pulsar_static_read_status(int64_t* pairs_needed, void* stream);

/* ------------------------------------------------------------------------
 * Batched rendering: several independent scenes (each with its own sphere
 * count, image size, camera, gamma, eps and depth range) rendered by one
 * sequence of launches.  The paper renders one scene per call; batching is
 * this library's scheduling of many such calls: the scenes' spheres, tiles
 * and pixels are concatenated, every kernel covers all of them, and the
 * render kernels draw work items of all scenes from one list, longest first.
 *
 * Rules shared by the batched entry points
 *   - 1 <= n_scenes <= PULSAR_MAX_SCENES; params[s] and scenes[s] describe
 *     scene s.  All scenes share n_channels, n_track, tile and flags.
 *   - The batch's pair capacity is the sum of the scenes' list_capacity; an
 *     overflow of that sum is reported by pulsar_read_status, and
 *     pairs_needed is then the batch's total.
 *   - A batched workspace serves only batched calls with the same n_scenes
 *     and params, and each scene's results are those of the single-scene
 *     entry points on that scene (up to float rounding of the Eq. 1 sums,
 *     whose summation order may differ).
 * ------------------------------------------------------------------------ */

#define PULSAR_MAX_SCENES 64

/* Per-scene outputs of pulsar_render_fwd_batched (same meaning and layout as
 * the arguments of pulsar_render_fwd; the optional ones may be NULL). */
typedef struct {
  float* image;       /* H x W x C */
  float* log_norm;    /* H x W */
  int32_t* n_hits;    /* optional H x W */
  int32_t* n_tests;   /* optional H x W */
  int32_t* tracked;   /* optional H x W x n_track */
} pulsar_fwd_out;

/* Per-scene inputs and outputs of pulsar_render_bwd_batched (same meaning as
 * the arguments of pulsar_render_bwd; outputs not selected by grad_mask may
 * be NULL). */
typedef struct {
  const float* image;
  const float* log_norm;
  const float* grad_image;
  float* g_pos;
  float* g_rad;
  float* g_opa;
  float* g_feat;
  float* g_cam;
  float* g_bg;
} pulsar_bwd_io;

/* Workspace bytes for a batch (0 when the settings are invalid). */
size_t pulsar_workspace_size_batched(int n_scenes, const pulsar_params* params);

/* pulsar_project over every scene of the batch, in one launch. */
pulsar_status pulsar_project_batched(int n_scenes, const pulsar_params* params,
                                     const pulsar_scene* scenes, void* workspace,
                                     size_t workspace_bytes, void* stream);

/* pulsar_bin over every scene of the batch: one depth sort of all spheres
 * (a sphere's key orders it only against spheres of its own scene, since
 * tiles are per scene) and one pair sort by global tile. */
pulsar_status pulsar_bin_batched(int n_scenes, const pulsar_params* params, void* workspace,
                                 size_t workspace_bytes, void* stream);

/* pulsar_render_fwd over every scene of the batch; out[s] receives scene s. */
pulsar_status pulsar_render_fwd_batched(int n_scenes, const pulsar_params* params,
                                        const pulsar_scene* scenes, void* workspace,
                                        size_t workspace_bytes, const pulsar_fwd_out* out,
                                        void* stream);

/* The whole batched forward in one call: pulsar_project_batched,
 * pulsar_bin_batched and pulsar_render_fwd_batched on the same workspace. */
pulsar_status pulsar_render_batched(int n_scenes, const pulsar_params* params,
                                    const pulsar_scene* scenes, void* workspace,
                                    size_t workspace_bytes, const pulsar_fwd_out* out, void* stream);

/* pulsar_render_bwd over every scene of the batch; io[s] holds scene s's
 * forward outputs, upstream gradient and gradient outputs. */
pulsar_status pulsar_render_bwd_batched(int n_scenes, const pulsar_params* params,
                                        const pulsar_scene* scenes, void* workspace,
                                        size_t workspace_bytes, const pulsar_bwd_io* io,
                                        uint32_t grad_mask, void* stream);

/* The batch's tile lists, as pulsar_read_tile_lists: ranges holds the tiles
 * of scene 0, then scene 1, ... (n_tiles summed over scenes, x 2 int32), and
 * ids (the summed list_capacity int32) holds indices into the concatenation
 * of the scenes' spheres (scene s's sphere i is sum_{k<s} M_k + i). */
pulsar_status pulsar_read_tile_lists_batched(int n_scenes, const pulsar_params* params,
                                             void* workspace, size_t workspace_bytes,
                                             int32_t* ranges, int32_t* ids, void* stream);

/* Static description of a status code. */
const char* pulsar_status_string(pulsar_status status);

#ifdef __cplusplus
}
#endif

#endif /* PULSAR_H */
