/*
 * pulsar_scene.h: scene and camera utilities around the renderer.
 *
 * Camera in the form of Listing 1 (translation, rotation as an axis-angle
 * vector, focal length, sensor width) converted to the renderer's 11-vector
 * (translation, 6D rotation of Zhou et al., focal length, sensor width), and
 * the gradient back through the conversion; pruning and subdivision of the
 * sphere set between optimisation stages (Sec. 5).
 */
#ifndef PULSAR_SCENE_H
#define PULSAR_SCENE_H

#include "pulsar.h"

#ifdef __cplusplus
extern "C" {
#endif

/* n cameras, device pointers, contiguous:
 *   cam8   n x 8  [t(3), w(3), focal, sensor_width]; w is the axis-angle
 *          vector of the world-to-camera rotation B = exp([w]_x) (Rodrigues:
 *          B = I + sin|w|/|w| [w]_x + (1 - cos|w|)/|w|^2 [w]_x^2; B = I at w = 0)
 *   cam11  n x 11 [t(3), b1(3), b2(3), focal, sensor_width], b1 and b2 the first
 *          two rows of B (so the renderer's Gram-Schmidt returns B itself)
 * Asynchronous on the stream.  PULSAR_ERR_INVALID_ARG for n < 0 or a NULL
 * pointer when n > 0. */
pulsar_status pulsar_camera_from_axis_angle(const float* cam8, float* cam11, int n, void* stream);

/* Gradient through pulsar_camera_from_axis_angle: given dL/dcam11 (n x 11),
 * writes dL/dcam8 (n x 8).  Same arguments and errors. */
pulsar_status pulsar_camera_axis_angle_backward(const float* cam8, const float* g_cam11, float* g_cam8,
                                                int n, void* stream);

/* Sphere pruning (the head reconstruction of Sec. 5: spheres are removed
 * when their colour has converged to the background colour or when they
 * received no gradient from any view).  Sphere i of n is kept when
 *   (activity == NULL or activity[i] > 0)  and
 *   (color_tol < 0 or ||f_i - bg||_2 > color_tol),
 * activity being any non-negative per-sphere measure of the gradients it
 * received (e.g. Adam's second moment of its opacity).  The kept spheres are
 * written in their input order to out_* (each with room for n spheres), and
 * their count to *n_out (device int64).  Device pointers; C = feature length;
 * scratch: pulsar_prune_scratch_bytes(n) bytes of device memory.
 * PULSAR_ERR_INVALID_ARG for n < 0, C < 1, a NULL array when n > 0 (activity
 * may be NULL), or a short scratch. */
size_t pulsar_prune_scratch_bytes(int64_t n);
pulsar_status pulsar_prune(int64_t n, int C, const float* pos, const float* rad, const float* opa,
                           const float* feat, const float* bg, const float* activity, float color_tol,
                           float* out_pos, float* out_rad, float* out_opa, float* out_feat, int64_t* n_out,
                           void* scratch, size_t scratch_bytes, void* stream);

/* Sphere subdivision (Sec. 5: every sphere refined into 12 spheres in a
 * face-centred cubic arrangement).  Child k of sphere i (output 12 i + k) sits
 * at p_i + offset_scale r_i u_k, u_k the 12 unit vectors from a site of the
 * face-centred cubic lattice to its nearest neighbours (the permutations of
 * (+-1, +-1, 0) / sqrt 2), with radius radius_scale r_i and the parent's
 * opacity and features.  out_* hold 12 n spheres.  Device pointers.
 * PULSAR_ERR_INVALID_ARG for n < 0, C < 1 or a NULL array when n > 0. */
pulsar_status pulsar_subdivide(int64_t n, int C, const float* pos, const float* rad, const float* opa,
                               const float* feat, float offset_scale, float radius_scale, float* out_pos,
                               float* out_rad, float* out_opa, float* out_feat, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PULSAR_SCENE_H */
