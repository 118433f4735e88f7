"""ctypes binding of the brute-force reference renderer (the oracle).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the CPU-baseline leg of
the benchmark call this module; the CUDA product path never does.

``build()`` compiles ``pulsar_oracle.c`` with the system C compiler into
``liboracle.so`` next to it.  Every function takes a ``Scene``-like object
(attributes pos, rad, opa, feat, cam, bg, width, height, gamma, n_track, eps,
znear, zfar) so that it shares no code with the product package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pulsar_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("n_spheres", ctypes.c_int32), ("n_channels", ctypes.c_int32),
        ("n_track", ctypes.c_int32), ("tile", ctypes.c_int32),
        ("min_size", ctypes.c_int32), ("dist_literal", ctypes.c_int32), ("paper_grad", ctypes.c_int32),
        ("ortho", ctypes.c_int32), ("paper_stop", ctypes.c_int32),
        ("gamma", ctypes.c_double), ("eps", ctypes.c_double),
        ("znear", ctypes.c_double), ("zfar", ctypes.c_double),
        ("min_contrib", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle; returns the library path."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        d, f, i32, i64 = ctypes.c_double, ctypes.c_float, ctypes.c_int32, ctypes.c_int64
        L.orc_project.argtypes = [P(OrcParams), P(d), P(d), P(d), P(f), P(f), P(f), P(i32)]
        L.orc_project.restype = None
        L.orc_tile_lists.argtypes = [P(OrcParams), P(f), P(i32), P(i64), P(i32), i64]
        L.orc_tile_lists.restype = i64
        L.orc_render_fwd.argtypes = [P(OrcParams), P(d), P(d), P(d), P(d), P(d), P(d),
                                     P(d), P(d), P(d),
                                     P(d), P(d), P(i32), P(i32), P(f), P(d)]
        L.orc_render_fwd.restype = None
        L.orc_render_bwd.argtypes = [P(OrcParams), P(d), P(d), P(d), P(d), P(d), P(d), P(d),
                                     P(d), P(d), P(d), P(d), P(d), P(d)]
        L.orc_render_bwd.restype = None
        L.orc_render_bwd_window.argtypes = [P(OrcParams), P(d), P(d), P(d), P(d), P(d), P(d), P(d),
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            P(d), P(d), P(d), P(d), P(d), P(d)]
        L.orc_render_bwd_window.restype = None
        L.orc_paper_stop_margin.argtypes = [P(OrcParams), P(d), P(d), P(d), P(d), P(d)]
        L.orc_paper_stop_margin.restype = None
        L.orc_rows.argtypes = [P(d), P(d)]
        L.orc_rows.restype = None
        L.orc_hit_f32.argtypes = [P(OrcParams), P(d), d, P(d), ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, P(f)]
        L.orc_hit_f32.restype = ctypes.c_int
        L.orc_hit_map.argtypes = [P(OrcParams), P(d), d, P(d), ctypes.c_int, P(ctypes.c_uint8)]
        L.orc_hit_map.restype = None
        L.orc_render_pixels.argtypes = [P(OrcParams), P(d), P(d), P(d), P(d), P(d), P(d), ctypes.c_int,
                                        P(i32), P(d), P(d), P(i32), P(i32), P(f)]
        L.orc_render_pixels.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def params(scene, tile: int = 16, min_size: bool = True, dist_literal: bool = False,
           n_track: int | None = None, paper_grad: bool = False, ortho: bool | None = None) -> OrcParams:
    """ortho=None takes the scene's own ``ortho`` attribute (False when absent);
    the scene's ``paper_stop`` attribute selects the paper's early termination,
    with the threshold ``min_contrib`` (float32 value; 0.01 when absent)."""
    if ortho is None:
        ortho = bool(getattr(scene, "ortho", False))
    paper_stop = bool(getattr(scene, "paper_stop", False))
    return OrcParams(int(scene.width), int(scene.height), int(scene.pos.shape[0]),
                     int(scene.feat.shape[1]), int(n_track if n_track is not None else scene.n_track),
                     int(tile), int(bool(min_size)), int(bool(dist_literal)), int(bool(paper_grad)),
                     int(bool(ortho)), int(paper_stop),
                     float(np.float32(scene.gamma)), float(np.float32(scene.eps)),
                     float(np.float32(scene.znear)), float(np.float32(scene.zfar)),
                     float(np.float32(getattr(scene, "min_contrib", 0.01))))


@dataclass
class Projection:
    c: np.ndarray      # (M, 3) float32 camera-space centres
    R: np.ndarray      # (M,) float32 effective radii
    key: np.ndarray    # (M,) float32 sort keys, +inf when culled
    rect: np.ndarray   # (M, 4) int32 inclusive x0, x1, y0, y1; -1 when culled


def project(scene, **kw) -> Projection:
    p = params(scene, **kw)
    M = p.n_spheres
    c = np.zeros((M, 3), np.float32)
    R = np.zeros(M, np.float32)
    key = np.zeros(M, np.float32)
    rect = np.zeros((M, 4), np.int32)
    lib().orc_project(ctypes.byref(p), _ptr(_d(scene.pos), ctypes.c_double),
                      _ptr(_d(scene.rad), ctypes.c_double), _ptr(_d(scene.cam), ctypes.c_double),
                      _ptr(c, ctypes.c_float), _ptr(R, ctypes.c_float), _ptr(key, ctypes.c_float),
                      _ptr(rect, ctypes.c_int32))
    return Projection(c, R, key, rect)


def tile_lists(scene, tile: int = 16, **kw):
    """(offsets[n_tiles+1], ids[L]) of the per-tile lists, tiles in row-major order."""
    pr = project(scene, tile=tile, **kw)
    p = params(scene, tile=tile, **kw)
    ntx = (scene.width + tile - 1) // tile
    nty = (scene.height + tile - 1) // tile
    offsets = np.zeros(ntx * nty + 1, np.int64)
    cap = 1 << 16
    while True:
        ids = np.zeros(cap, np.int32)
        total = lib().orc_tile_lists(ctypes.byref(p), _ptr(pr.key, ctypes.c_float),
                                     _ptr(pr.rect, ctypes.c_int32), _ptr(offsets, ctypes.c_int64),
                                     _ptr(ids, ctypes.c_int32), cap)
        if total >= 0:
            return offsets, ids[:total]
        cap = int(offsets[-1]) + 1


@dataclass
class Forward:
    image: np.ndarray      # (H, W, C) float64
    log_d: np.ndarray      # (H, W) float64, log of Eq. 1's denominator
    n_hits: np.ndarray     # (H, W) int32
    tracked: np.ndarray    # (H, W, K) int32, -1 padded
    tracked_t: np.ndarray  # (H, W, K) float32 hit depths, +inf padded
    wsum: np.ndarray       # (H, W) float64, sum of sphere weights


def _scene_arrays(scene, pos=None, rad=None, opa=None, feat=None, cam=None, bg=None):
    return (_d(scene.pos if pos is None else pos), _d(scene.rad if rad is None else rad),
            _d(scene.opa if opa is None else opa), _d(scene.feat if feat is None else feat),
            _d(scene.cam if cam is None else cam), _d(scene.bg if bg is None else bg))


def render(scene, n_track: int | None = None, min_size: bool = True, dist_literal: bool = False,
           freeze_decisions: bool = False, **override) -> Forward:
    """Brute-force forward pass.

    ``override`` replaces inputs by float64 arrays.  With ``freeze_decisions``
    the float32 decisions (hits, order, culling, minimum size) are taken from
    the unmodified scene, so that finite differences see a smooth function.
    """
    p = params(scene, n_track=n_track, min_size=min_size, dist_literal=dist_literal)
    H, W, C, K = p.height, p.width, p.n_channels, p.n_track
    arrs = _scene_arrays(scene, **override)
    if freeze_decisions:
        dec = [_ptr(_d(scene.pos), ctypes.c_double), _ptr(_d(scene.rad), ctypes.c_double),
               _ptr(_d(scene.cam), ctypes.c_double)]
    else:
        dec = [None, None, None]
    img = np.zeros((H, W, C), np.float64)
    ld = np.zeros((H, W), np.float64)
    nh = np.zeros((H, W), np.int32)
    tr = np.zeros((H, W, K), np.int32)
    tt = np.zeros((H, W, K), np.float32)
    ws = np.zeros((H, W), np.float64)
    D = ctypes.c_double
    lib().orc_render_fwd(ctypes.byref(p), *[_ptr(a, D) for a in arrs], *dec, _ptr(img, D), _ptr(ld, D),
                         _ptr(nh, ctypes.c_int32), _ptr(tr, ctypes.c_int32), _ptr(tt, ctypes.c_float),
                         _ptr(ws, D))
    return Forward(img, ld, nh, tr, tt, ws)


def paper_stop_margin(scene, **kw) -> np.ndarray:
    """(H, W) float64: per pixel the smallest |ln(a / min_contrib)| over the early-
    termination tests the pixel takes (scene.paper_stop set), a the largest
    possible weight tested; +inf where no test is taken."""
    p = params(scene, **kw)
    out = np.zeros((p.height, p.width), np.float64)
    D = ctypes.c_double
    lib().orc_paper_stop_margin(ctypes.byref(p), _ptr(_d(scene.pos), D), _ptr(_d(scene.rad), D),
                                _ptr(_d(scene.opa), D), _ptr(_d(scene.cam), D), _ptr(out, D))
    return out


@dataclass
class Gradients:
    pos: np.ndarray
    rad: np.ndarray
    opa: np.ndarray
    feat: np.ndarray
    cam: np.ndarray
    bg: np.ndarray


def render_backward(scene, grad: np.ndarray, n_track: int | None = None, min_size: bool = True,
                    dist_literal: bool = False, paper_grad: bool = False, **override) -> Gradients:
    """Analytic gradients of L = <grad, F> through the tracked hits; with
    paper_grad, the paper's normalisations (per-pixel averaging, the 3-pixel
    position gate, camera scaled by 1e-3)."""
    p = params(scene, n_track=n_track, min_size=min_size, dist_literal=dist_literal, paper_grad=paper_grad)
    M, C = p.n_spheres, p.n_channels
    arrs = _scene_arrays(scene, **override)
    G = _d(grad)
    assert G.shape == (p.height, p.width, C)
    out = Gradients(np.zeros((M, 3)), np.zeros(M), np.zeros(M), np.zeros((M, C)), np.zeros(11),
                    np.zeros(C))
    D = ctypes.c_double
    lib().orc_render_bwd(ctypes.byref(p), *[_ptr(a, D) for a in arrs], _ptr(G, D),
                         _ptr(out.pos, D), _ptr(out.rad, D), _ptr(out.opa, D), _ptr(out.feat, D),
                         _ptr(out.cam, D), _ptr(out.bg, D))
    return out


def render_backward_window(scene, grad: np.ndarray, u0: int, v0: int, n_track: int | None = None,
                           min_size: bool = True, dist_literal: bool = False) -> Gradients:
    """render_backward with dL/dF given on the window of grad's shape at
    (u0, v0) and zero elsewhere (not with the paper's normalisations)."""
    p = params(scene, n_track=n_track, min_size=min_size, dist_literal=dist_literal)
    M, C = p.n_spheres, p.n_channels
    G = _d(grad)
    wh, ww = G.shape[0], G.shape[1]
    assert G.shape[2] == C and 0 <= u0 and u0 + ww <= p.width and 0 <= v0 and v0 + wh <= p.height
    arrs = _scene_arrays(scene)
    out = Gradients(np.zeros((M, 3)), np.zeros(M), np.zeros(M), np.zeros((M, C)), np.zeros(11),
                    np.zeros(C))
    D = ctypes.c_double
    lib().orc_render_bwd_window(ctypes.byref(p), *[_ptr(a, D) for a in arrs], _ptr(G, D), int(u0), int(v0),
                                int(ww), int(wh), _ptr(out.pos, D), _ptr(out.rad, D), _ptr(out.opa, D),
                                _ptr(out.feat, D), _ptr(out.cam, D), _ptr(out.bg, D))
    return out


def rows(rot6) -> np.ndarray:
    a = _d(rot6)
    B = np.zeros(9, np.float64)
    lib().orc_rows(_ptr(a, ctypes.c_double), _ptr(B, ctypes.c_double))
    return B.reshape(3, 3)


def hit_f32(scene, pos3, rad, u: int, v: int, min_size: bool = True, ignore_cull: bool = False):
    p = params(scene, min_size=min_size)
    t = ctypes.c_float(0.0)
    h = lib().orc_hit_f32(ctypes.byref(p), _ptr(_d(pos3), ctypes.c_double), float(rad),
                          _ptr(_d(scene.cam), ctypes.c_double), int(u), int(v),
                          int(bool(ignore_cull)), ctypes.byref(t))
    return bool(h), float(t.value)


def hit_map(scene, pos3, rad, min_size: bool = True, ignore_cull: bool = False) -> np.ndarray:
    """(H, W) bool map of the float32 hit predicate of one sphere."""
    p = params(scene, min_size=min_size)
    m = np.zeros((scene.height, scene.width), np.uint8)
    lib().orc_hit_map(ctypes.byref(p), _ptr(_d(pos3), ctypes.c_double), float(rad),
                      _ptr(_d(scene.cam), ctypes.c_double), int(bool(ignore_cull)),
                      _ptr(m, ctypes.c_uint8))
    return m.astype(bool)


def render_pixels(scene, pixels, n_track: int | None = None, min_size: bool = True,
                  dist_literal: bool = False) -> Forward:
    """Forward pass at the listed (u, v) pixels only; arrays are indexed by list position."""
    p = params(scene, n_track=n_track, min_size=min_size, dist_literal=dist_literal)
    pix = np.ascontiguousarray(np.asarray(pixels, np.int32).reshape(-1, 2))
    n, C, K = pix.shape[0], p.n_channels, p.n_track
    arrs = _scene_arrays(scene)
    img = np.zeros((n, C), np.float64)
    ld = np.zeros(n, np.float64)
    nh = np.zeros(n, np.int32)
    tr = np.zeros((n, K), np.int32)
    tt = np.zeros((n, K), np.float32)
    D = ctypes.c_double
    lib().orc_render_pixels(ctypes.byref(p), *[_ptr(a, D) for a in arrs], int(n),
                            _ptr(pix, ctypes.c_int32), _ptr(img, D), _ptr(ld, D),
                            _ptr(nh, ctypes.c_int32), _ptr(tr, ctypes.c_int32),
                            _ptr(tt, ctypes.c_float))
    return Forward(img, ld, nh, tr, tt, np.zeros(n))
