"""Oracle of the scene and camera utilities: the camera of Listing 1
(translation, axis-angle rotation, focal length, sensor width) as the
renderer's 11-vector (translation, 6D rotation, focal length, sensor width);
pruning and subdivision of a sphere set (Sec. 5).

TEST INFRASTRUCTURE ONLY: tests call this module; the CUDA product path never
does.  Float64 NumPy, from Rodrigues' formula: B = I + sin|w|/|w| [w]_x +
(1 - cos|w|)/|w|^2 [w]_x^2, the world-to-camera rotation; the 6D rotation is
its first two rows.
"""
from __future__ import annotations

import numpy as np


def skew(w) -> np.ndarray:
    w = np.asarray(w, np.float64)
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def rotation(w) -> np.ndarray:
    w = np.asarray(w, np.float64)
    s = float(np.linalg.norm(w))
    K = skew(w)
    if s == 0.0:
        return np.eye(3)
    return np.eye(3) + np.sin(s) / s * K + (1.0 - np.cos(s)) / s ** 2 * (K @ K)


def cam11_from_cam8(cam8) -> np.ndarray:
    c = np.asarray(cam8, np.float64)
    B = rotation(c[3:6])
    return np.concatenate([c[0:3], B[0], B[1], c[6:8]])


def prune_keep(feat, bg, activity=None, color_tol=-1.0) -> np.ndarray:
    """Spheres kept by the pruning rule: received gradients (activity > 0) and,
    unless color_tol < 0, a feature vector farther than color_tol from the
    background.  The distance decides a discrete outcome, so it is evaluated
    in float32 with the library's operation order (one rounding per step)."""
    feat = np.asarray(feat, np.float32)
    bg = np.asarray(bg, np.float32)
    keep = np.ones(feat.shape[0], bool)
    if activity is not None:
        keep &= np.asarray(activity, np.float32) > 0
    if color_tol >= 0:
        s = np.zeros(feat.shape[0], np.float32)
        for c in range(feat.shape[1]):
            d = (feat[:, c] - bg[c]).astype(np.float32)
            s = (s + (d * d).astype(np.float32)).astype(np.float32)
        keep &= np.sqrt(s) > np.float32(color_tol)
    return keep


FCC_DIRECTIONS = np.array([[0, 1, 1], [0, -1, 1], [0, 1, -1], [0, -1, -1],
                           [1, 0, 1], [-1, 0, 1], [1, 0, -1], [-1, 0, -1],
                           [1, 1, 0], [-1, 1, 0], [1, -1, 0], [-1, -1, 0]], np.float64) / np.sqrt(2.0)


def subdivide(pos, rad, opa, feat, offset_scale, radius_scale):
    """Every sphere as 12 children at p + offset_scale r u_k (u_k the nearest-
    neighbour directions of the face-centred cubic lattice), radius
    radius_scale r, the parent's opacity and features; child k of sphere i is
    entry 12 i + k."""
    pos = np.asarray(pos, np.float64)
    rad = np.asarray(rad, np.float64)
    n = pos.shape[0]
    out_pos = (pos[:, None, :] + offset_scale * rad[:, None, None] * FCC_DIRECTIONS[None]).reshape(12 * n, 3)
    return (out_pos, np.repeat(radius_scale * rad, 12), np.repeat(np.asarray(opa, np.float64), 12),
            np.repeat(np.asarray(feat, np.float64), 12, axis=0))
