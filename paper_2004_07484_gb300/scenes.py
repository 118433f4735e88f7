"""Seeded synthetic sphere scenes.

This module only draws random numbers; it contains none of the renderer's
arithmetic, so both the CUDA path and the CPU oracle can consume its output.

The scene tuple follows Sec. 3.1: M spheres with position p_i (3), feature
vector f_i (C), radius r_i and opacity o_i.  The camera vector follows the
order printed in Listing 1 (translation first, then rotation, focal length,
sensor width), with the rotation given as the 6D vector of Zhou et al. that
Listing 1's caption paragraph says Pulsar accepts natively:

    cam = [t_x, t_y, t_z, a1_x, a1_y, a1_z, a2_x, a2_y, a2_z, focal, sensor_width]

All arrays are float32 and C-contiguous.  Every generator is driven by a
``numpy.random.Generator(PCG64(seed))`` sampled in float64 and cast to float32.

The workload shapes stand in for the paper's own captures and datasets
(Tab. 2, Fig. 3, Sec. 5), none of which are available here.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

IDENTITY_ROT6 = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0)


@dataclass
class Scene:
    """One render job: spheres, camera, background and blending settings."""

    pos: np.ndarray          # (M, 3) float32
    rad: np.ndarray          # (M,)   float32
    opa: np.ndarray          # (M,)   float32
    feat: np.ndarray         # (M, C) float32
    cam: np.ndarray          # (11,)  float32
    bg: np.ndarray           # (C,)   float32
    width: int
    height: int
    gamma: float
    n_track: int
    eps: float = 1e-5
    znear: float = 1.0
    zfar: float = 20.0
    name: str = ""
    meta: dict = field(default_factory=dict)
    ortho: bool = False      # orthographic camera (rays along +z from the sensor plane)
    paper_stop: bool = False # the paper's early termination (an approximation)
    min_contrib: float = 0.01  # its threshold (the paper's "n percent" as a fraction)

    @property
    def n_spheres(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_channels(self) -> int:
        return int(self.feat.shape[1])


def make_cam(t=(0.0, 0.0, 0.0), rot6=IDENTITY_ROT6, focal=1.0, sensor_width=2.0) -> np.ndarray:
    return np.asarray(list(t) + list(rot6) + [focal, sensor_width], dtype=np.float32)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _log_uniform(g: np.random.Generator, lo: float, hi: float, n: int) -> np.ndarray:
    return np.exp(g.uniform(np.log(lo), np.log(hi), n))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def random_rotation(g: np.random.Generator) -> np.ndarray:
    """Haar-random 3x3 rotation from the QR factorisation of a Gaussian matrix."""
    a = g.standard_normal((3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 2] = -q[:, 2]
    return q


def uniform_cloud(seed: int, n: int, width: int, height: int, n_channels: int = 3,
                  gamma: float = 0.1, n_track: int = 5, xy=(-1.0, 1.0), z=(5.0, 10.0),
                  rad=(0.01, 0.1), opa=(0.5, 1.0), feat: str = "uniform", name: str = "") -> Scene:
    """Uniform box of spheres in front of an identity camera (the 1000-sphere, 64x64 case)."""
    g = _rng(seed)
    pos = np.stack([g.uniform(*xy, n), g.uniform(*xy, n), g.uniform(*z, n)], axis=1)
    r = _log_uniform(g, rad[0], rad[1], n)
    o = g.uniform(opa[0], opa[1], n)
    f = g.uniform(0.0, 1.0, (n, n_channels)) if feat == "uniform" else g.standard_normal((n, n_channels))
    return Scene(_f32(pos), _f32(r), _f32(o), _f32(f), make_cam(), np.zeros(n_channels, np.float32),
                 width, height, gamma, n_track, name=name or f"uniform{n}_{width}x{height}")


def gaussian_mixture(seed: int, n: int, width: int, height: int, n_channels: int = 3,
                     gamma: float = 1e-2, n_track: int = 10, n_modes: int = 8, std: float = 0.3,
                     mean_xy=(-1.5, 1.5), mean_z=(5.0, 11.0), z_keep=(4.0, 12.0),
                     rad=(0.005, 0.05), opa=(0.5, 1.0), feat: str = "uniform",
                     cam: np.ndarray | None = None, name: str = "") -> Scene:
    """Mixture of isotropic Gaussian blobs (the 100k-sphere, 512x512 case)."""
    g = _rng(seed)
    mu = np.stack([g.uniform(*mean_xy, n_modes), g.uniform(*mean_xy, n_modes),
                   g.uniform(*mean_z, n_modes)], axis=1)
    out = np.empty((0, 3))
    while out.shape[0] < n:
        k = g.integers(0, n_modes, 2 * n)
        p = mu[k] + std * g.standard_normal((2 * n, 3))
        p = p[(p[:, 2] >= z_keep[0]) & (p[:, 2] <= z_keep[1])]
        out = np.concatenate([out, p], axis=0)
    pos = out[:n]
    r = _log_uniform(g, rad[0], rad[1], n)
    o = g.uniform(opa[0], opa[1], n)
    f = g.uniform(0.0, 1.0, (n, n_channels)) if feat == "uniform" else g.standard_normal((n, n_channels))
    return Scene(_f32(pos), _f32(r), _f32(o), _f32(f), make_cam() if cam is None else _f32(cam),
                 np.zeros(n_channels, np.float32), width, height, gamma, n_track,
                 name=name or f"gmm{n}_{width}x{height}")


def ellipsoid_surfaces(seed: int, n: int, width: int, height: int, n_channels: int = 16,
                       gamma: float = 1e-2, n_track: int = 16, n_ellipsoids: int = 20,
                       centre_xy=(-2.0, 2.0), centre_z=(6.0, 10.0), axes=(0.2, 1.5),
                       jitter: float = 0.01, rad=(0.005, 0.05), opa=(0.3, 1.0),
                       feat: str = "normal", name: str = "") -> Scene:
    """Points on the surfaces of random ellipsoids, like a sensor point cloud (the 1M, 1024^2 case)."""
    g = _rng(seed)
    per = np.full(n_ellipsoids, n // n_ellipsoids)
    per[: n - per.sum()] += 1
    chunks = []
    for e in range(n_ellipsoids):
        c = np.array([g.uniform(*centre_xy), g.uniform(*centre_xy), g.uniform(*centre_z)])
        ax = g.uniform(axes[0], axes[1], 3)
        rot = random_rotation(g)
        u = g.standard_normal((per[e], 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        pts = c[None, :] + (u * ax[None, :]) @ rot.T + jitter * g.standard_normal((per[e], 3))
        chunks.append(pts)
    pos = np.concatenate(chunks, axis=0)
    r = _log_uniform(g, rad[0], rad[1], n)
    o = g.uniform(opa[0], opa[1], n)
    f = g.standard_normal((n, n_channels)) if feat == "normal" else g.uniform(0.0, 1.0, (n, n_channels))
    return Scene(_f32(pos), _f32(r), _f32(o), _f32(f), make_cam(), np.zeros(n_channels, np.float32),
                 width, height, gamma, n_track, name=name or f"ellipsoids{n}_{width}x{height}")


def rot6_from_matrix(rows: np.ndarray) -> np.ndarray:
    """6D vector whose Gram-Schmidt rows reproduce ``rows`` (first two rows)."""
    return np.concatenate([rows[0], rows[1]])


def look_at_rows(g: np.random.Generator) -> np.ndarray:
    return random_rotation(g).T


def batch_scenes(seed: int, n_scenes: int = 32, n_channels: int = 8, n_track: int = 10,
                 m_range=(1e3, 5e5), resolutions=(128, 256, 512, 1024),
                 gamma_range=(1e-3, 0.1)) -> list[Scene]:
    """Independent scenes with uneven sphere counts and resolutions (the 32-scene batched case).

    Each scene uses the Gaussian-mixture distribution with N(0,1) features.  Its
    camera gets a random rotation and is placed so that the mixture centroid sits
    at distance 8 on the optical axis.
    """
    g = _rng(seed)
    scenes = []
    for s in range(n_scenes):
        m = int(round(float(np.exp(g.uniform(np.log(m_range[0]), np.log(m_range[1]))))))
        res = int(resolutions[g.integers(0, len(resolutions))])
        gam = float(np.exp(g.uniform(np.log(gamma_range[0]), np.log(gamma_range[1]))))
        sub_seed = int(g.integers(0, 2**31 - 1))
        sc = gaussian_mixture(sub_seed, m, res, res, n_channels=n_channels, gamma=gam,
                              n_track=n_track, feat="normal", name=f"batch{s}_{m}_{res}")
        rows = random_rotation(g).T          # world -> camera rows, det +1
        centroid = sc.pos.astype(np.float64).mean(axis=0)
        t = centroid - 8.0 * rows[2]         # camera centre: 8 units behind the centroid on its z axis
        sc.cam = make_cam(t=t, rot6=rot6_from_matrix(rows))
        scenes.append(sc)
    return scenes


def orbit_cameras(seed: int, centre, n_views: int = 4, distance: float = 8.0, focal: float = 1.0,
                  sensor_width: float = 2.0) -> list[np.ndarray]:
    """Cameras at random rotations about ``centre``, each ``distance`` behind it
    on its own optical axis (the views of the scene fit)."""
    g = _rng(seed)
    c = np.asarray(centre, dtype=np.float64)
    cams = []
    for _ in range(n_views):
        rows = random_rotation(g).T
        cams.append(make_cam(t=c - distance * rows[2], rot6=rot6_from_matrix(rows), focal=focal,
                             sensor_width=sensor_width))
    return cams


def perturbed(scene: Scene, seed: int, pos_sigma: float = 0.05, rad_frac: float = 0.3) -> Scene:
    """Initial guess of the scene fit: positions + N(0, pos_sigma^2), radii
    times U[1 - rad_frac, 1 + rad_frac]; opacities, features and camera kept."""
    g = _rng(seed)
    n = scene.n_spheres
    pos = scene.pos.astype(np.float64) + pos_sigma * g.standard_normal((n, 3))
    rad = scene.rad.astype(np.float64) * g.uniform(1.0 - rad_frac, 1.0 + rad_frac, n)
    return Scene(_f32(pos), _f32(rad), scene.opa.copy(), scene.feat.copy(), scene.cam.copy(), scene.bg.copy(),
                 scene.width, scene.height, scene.gamma, scene.n_track, scene.eps, scene.znear, scene.zfar,
                 name=scene.name + "_perturbed")


def config_scene(index: int, gamma: float | None = None, n: int | None = None,
                 res: int | None = None) -> Scene:
    """The synthetic stand-in for each benchmark workload, seeded with 1000 + index.

    0: 1,000 spheres, 64x64, uniform box, C=3, gamma 0.1, n_track 5.
    1: 100k spheres, 512x512, 8-Gaussian mixture, C=3, n_track 10 (gamma swept).
    2: 1M spheres, 1024x1024, 20 ellipsoid surfaces, C=16 N(0,1), gamma 1e-2, n_track 16.
    4: 5M spheres, 1920x1080, ellipsoid surfaces, C=3, gamma 1e-2, n_track 8.
    ``n``/``res`` shrink a workload with the same distribution for quick checks.
    """
    seed = 1000 + index
    if index == 0:
        return uniform_cloud(seed, n or 1000, res or 64, res or 64, n_channels=3,
                             gamma=gamma or 0.1, n_track=5)
    if index == 1:
        return gaussian_mixture(seed, n or 100_000, res or 512, res or 512, n_channels=3,
                                gamma=gamma or 1e-2, n_track=10)
    if index == 2:
        return ellipsoid_surfaces(seed, n or 1_000_000, res or 1024, res or 1024, n_channels=16,
                                  gamma=gamma or 1e-2, n_track=16)
    if index == 4:
        w, h = (res, res) if res else (1920, 1080)
        return ellipsoid_surfaces(seed, n or 5_000_000, w, h, n_channels=3, gamma=gamma or 1e-2,
                                  n_track=8, feat="uniform")
    raise ValueError(f"no single-scene workload {index}")


def grad_image(seed: int, height: int, width: int, n_channels: int) -> np.ndarray:
    """Seeded N(0,1) upstream gradient dL/dF for a linear loss <G, F>."""
    return _f32(_rng(seed).standard_normal((height, width, n_channels)))
