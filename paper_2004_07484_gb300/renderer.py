"""PyTorch front end: ``Renderer`` (an ``nn.Module``) and its autograd function.

The call mirrors Listing 1 of the paper: a renderer is constructed for an
image size and sphere count, then called with sphere positions, features,
radii and a camera vector; the result is registered with autograd, and the
backward pass returns gradients for positions, radii, opacities, features,
camera and background (App. B, "The Backward Pass").

PyTorch provides device memory, streams and autograd only.  Every step of the
render runs in ``libpulsar_gb300.so`` through ``_lib``; tensors must already
be CUDA float32.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import torch

from . import _lib


@dataclass
class RenderSettings:
    width: int
    height: int
    n_channels: int
    n_track: int = 5                 # closest hits kept per pixel (App. B, Step 2)
    gamma: float = 0.1               # blending sharpness, [1e-5, 1] (Sec. 3.2)
    eps: float = 1e-5                # background offset of Eq. 1
    znear: float = 1.0
    zfar: float = 20.0               # Listing 1's max_depth
    store_hits: bool = True          # keep the n_track-th hit per pixel for the backward pass
    dist_literal: bool = False       # d = min(1, dist/R) instead of 1 - min(1, dist/R)
    min_size: bool = True            # every sphere covers at least one pixel (App. B, Step 0)
    tile: int = 16
    segment: int = 0                 # scheduling: list entries per work item (0 = library default)
    persistent: bool = False         # scheduling: persistent render kernels
    accumulate: bool = False         # backward adds into the gradient buffers (views sharing them)
    paper_gradients: bool = False    # the paper's gradient normalisations (App. B, Sec. 6)
    orthographic: bool = False       # orthographic camera: pitch = sensor width / W (Sec. 1)
    paper_stop: bool = False         # the paper's early termination (App. B, Step 2; approximate)
    min_contrib: float = 0.0         # its threshold as a fraction of the blend; 0 = 0.01 (the paper's)

    def flags(self) -> int:
        f = 0
        if self.store_hits:
            f |= _lib.FLAG_STORE_HITS
        if self.dist_literal:
            f |= _lib.FLAG_DIST_LITERAL
        if not self.min_size:
            f |= _lib.FLAG_NO_MIN_SIZE
        if self.persistent:
            f |= _lib.FLAG_PERSISTENT
        if self.accumulate:
            f |= _lib.FLAG_ACCUMULATE
        if self.paper_gradients:
            f |= _lib.FLAG_PAPER_GRADIENTS
        if self.orthographic:
            f |= _lib.FLAG_ORTHOGRAPHIC
        if self.paper_stop:
            f |= _lib.FLAG_PAPER_STOP
        return f

    def params(self, n_spheres: int, capacity: int) -> _lib.Params:
        return _lib.Params(int(self.width), int(self.height), int(n_spheres), int(self.n_channels),
                           int(self.n_track), int(self.tile), int(capacity), float(self.gamma),
                           float(self.eps), float(self.znear), float(self.zfar), int(self.flags()),
                           int(self.segment), float(self.min_contrib))


def _dev_f32(name: str, t: torch.Tensor, shape) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.contiguous()


def _ptr(t):
    return None if t is None else t.data_ptr()


def scene_args(pos, feat, rad, opa, cam, bg) -> _lib.SceneArgs:
    return _lib.SceneArgs(_ptr(pos), _ptr(rad), _ptr(opa), _ptr(feat), _ptr(cam), _ptr(bg))


class Frame:
    """Device state of one render: the workspace and the forward outputs."""

    def __init__(self, settings: RenderSettings, n_spheres: int, capacity: int, device):
        self.settings = settings
        self.params = settings.params(n_spheres, capacity)
        self.ws_bytes = _lib.workspace_size(self.params)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)


def _default_capacity(s: RenderSettings, n_spheres: int) -> int:
    tiles = ((s.width + s.tile - 1) // s.tile) * ((s.height + s.tile - 1) // s.tile)
    return max(4 * n_spheres, tiles, 1 << 16)


def forward_frame(settings: RenderSettings, pos, feat, rad, opa, cam, bg, capacity: int,
                  check_overflow: bool = True, n_hits=None, tracked=None, n_tests=None):
    """Runs project -> bin -> render_fwd.  Returns (frame, image, log_norm)."""
    M = int(pos.shape[0])
    stream = torch.cuda.current_stream(pos.device).cuda_stream
    sc = scene_args(pos, feat, rad, opa, cam, bg)
    while True:
        fr = Frame(settings, M, capacity, pos.device)
        _lib.project(fr.params, sc, fr.ws.data_ptr(), fr.ws_bytes, stream)
        _lib.bin(fr.params, fr.ws.data_ptr(), fr.ws_bytes, stream)
        if not check_overflow:
            break
        st, need = _lib.read_status(fr.ws.data_ptr(), fr.ws_bytes, stream)
        if st == _lib.OK:
            break
        if st != _lib.ERR_CAPACITY:
            raise _lib.PulsarError(st, "pulsar_bin")
        capacity = int(need * 1.25) + 1024
    H, W, C = settings.height, settings.width, settings.n_channels
    image = torch.empty((H, W, C), dtype=torch.float32, device=pos.device)
    log_norm = torch.empty((H, W), dtype=torch.float32, device=pos.device)
    _lib.render_fwd(fr.params, sc, fr.ws.data_ptr(), fr.ws_bytes, image.data_ptr(), log_norm.data_ptr(),
                    _ptr(n_hits), _ptr(n_tests), _ptr(tracked), stream)
    return fr, image, log_norm


def backward_frame(fr: Frame, pos, feat, rad, opa, cam, bg, image, log_norm, grad_image,
                   grad_mask: int = _lib.GRAD_ALL):
    """Runs render_bwd on a forward frame.  Returns the six gradients (None where not asked)."""
    M = int(pos.shape[0])
    C = fr.settings.n_channels
    dev = pos.device
    g_pos = torch.empty((M, 3), dtype=torch.float32, device=dev) if grad_mask & _lib.GRAD_POS else None
    g_rad = torch.empty((M,), dtype=torch.float32, device=dev) if grad_mask & _lib.GRAD_RAD else None
    g_opa = torch.empty((M,), dtype=torch.float32, device=dev) if grad_mask & _lib.GRAD_OPA else None
    g_feat = torch.empty((M, C), dtype=torch.float32, device=dev) if grad_mask & _lib.GRAD_FEAT else None
    g_cam = torch.empty((11,), dtype=torch.float32, device=dev) if grad_mask & _lib.GRAD_CAM else None
    g_bg = torch.empty((C,), dtype=torch.float32, device=dev) if grad_mask & _lib.GRAD_BG else None
    stream = torch.cuda.current_stream(dev).cuda_stream
    _lib.render_bwd(fr.params, scene_args(pos, feat, rad, opa, cam, bg), fr.ws.data_ptr(), fr.ws_bytes,
                    image.data_ptr(), log_norm.data_ptr(), grad_image.data_ptr(), int(grad_mask),
                    _ptr(g_pos), _ptr(g_rad), _ptr(g_opa), _ptr(g_feat), _ptr(g_cam), _ptr(g_bg),
                    stream)
    return g_pos, g_rad, g_opa, g_feat, g_cam, g_bg


class BatchFrame:
    """Device state of one batched render: the settings of every scene and the workspace."""

    def __init__(self, settings: list[RenderSettings], n_spheres: list[int], capacities: list[int],
                 device):
        if not 1 <= len(settings) <= _lib.MAX_SCENES:
            raise ValueError(f"a batch holds 1..{_lib.MAX_SCENES} scenes, got {len(settings)}")
        self.settings = list(settings)
        self.n = len(settings)
        self.params = (_lib.Params * self.n)(*[s.params(m, c) for s, m, c in
                                              zip(settings, n_spheres, capacities)])
        self.ws_bytes = _lib.workspace_size_batched(self.params)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)

    def capacities(self) -> list[int]:
        return [int(p.list_capacity) for p in self.params]


def _scene_array(inputs):
    return (_lib.SceneArgs * len(inputs))(*[scene_args(*x) for x in inputs])


def forward_batch(settings: list[RenderSettings], inputs, capacities: list[int],
                  check_overflow: bool = True, n_hits=None, tracked=None, n_tests=None):
    """Batched project -> bin -> render_fwd over independent scenes.

    ``inputs[s]`` is scene s's (pos, feat, rad, opa, cam, bg); ``n_hits``,
    ``tracked`` and ``n_tests`` are optional per-scene lists of output
    tensors.  Returns (frame, images, log_norms)."""
    dev = inputs[0][0].device
    stream = torch.cuda.current_stream(dev).cuda_stream
    ms = [int(x[0].shape[0]) for x in inputs]
    ss = _scene_array(inputs)
    caps = list(capacities)
    while True:
        fr = BatchFrame(settings, ms, caps, dev)
        _lib.project_batched(fr.params, ss, fr.ws.data_ptr(), fr.ws_bytes, stream)
        _lib.bin_batched(fr.params, fr.ws.data_ptr(), fr.ws_bytes, stream)
        if not check_overflow:
            break
        st, need = _lib.read_status(fr.ws.data_ptr(), fr.ws_bytes, stream)
        if st == _lib.OK:
            break
        if st != _lib.ERR_CAPACITY:
            raise _lib.PulsarError(st, "pulsar_bin_batched")
        scale = 1.25 * need / max(sum(caps), 1)
        caps = [int(c * scale) + 1024 for c in caps]
    images, log_norms = [], []
    outs = (_lib.FwdOut * len(inputs))()
    for k, s in enumerate(settings):
        image = torch.empty((s.height, s.width, s.n_channels), dtype=torch.float32, device=dev)
        log_norm = torch.empty((s.height, s.width), dtype=torch.float32, device=dev)
        images.append(image)
        log_norms.append(log_norm)
        outs[k] = _lib.FwdOut(image.data_ptr(), log_norm.data_ptr(),
                              _ptr(n_hits[k]) if n_hits else None,
                              _ptr(n_tests[k]) if n_tests else None,
                              _ptr(tracked[k]) if tracked else None)
    _lib.render_fwd_batched(fr.params, ss, fr.ws.data_ptr(), fr.ws_bytes, outs, stream)
    return fr, images, log_norms


def backward_batch(fr: BatchFrame, inputs, images, log_norms, grad_images,
                   grad_mask: int = _lib.GRAD_ALL, out=None):
    """Batched render_bwd.  Returns, per scene, the six gradients (None where not asked).

    ``out[s]``, when given, holds scene s's six gradient tensors (None where
    not asked) and receives the result; with ``accumulate`` settings several
    scenes may share them and the gradients are added into them."""
    dev = inputs[0][0].device
    stream = torch.cuda.current_stream(dev).cuda_stream
    ios = (_lib.BwdIO * len(inputs))()
    grads = []
    for k, (x, s) in enumerate(zip(inputs, fr.settings)):
        M, C = int(x[0].shape[0]), s.n_channels

        def alloc(flag, shape):
            return torch.empty(shape, dtype=torch.float32, device=dev) if grad_mask & flag else None

        if out is not None:
            g = tuple(out[k])
            shapes = ((M, 3), (M,), (M,), (M, C), (11,), (C,))
            for t, shape, flag in zip(g, shapes, (_lib.GRAD_POS, _lib.GRAD_RAD, _lib.GRAD_OPA,
                                                  _lib.GRAD_FEAT, _lib.GRAD_CAM, _lib.GRAD_BG)):
                if grad_mask & flag:
                    _dev_f32("gradient output", t, shape)
                    if not t.is_contiguous():
                        raise ValueError("gradient outputs must be contiguous")
        else:
            g = (alloc(_lib.GRAD_POS, (M, 3)), alloc(_lib.GRAD_RAD, (M,)), alloc(_lib.GRAD_OPA, (M,)),
                 alloc(_lib.GRAD_FEAT, (M, C)), alloc(_lib.GRAD_CAM, (11,)), alloc(_lib.GRAD_BG, (C,)))
        grads.append(g)
        ios[k] = _lib.BwdIO(images[k].data_ptr(), log_norms[k].data_ptr(), grad_images[k].data_ptr(),
                            *[_ptr(t) for t in g])
    _lib.render_bwd_batched(fr.params, _scene_array(inputs), fr.ws.data_ptr(), fr.ws_bytes, ios,
                            int(grad_mask), stream)
    return grads


class _RenderFunction(torch.autograd.Function):
    """The render as an autograd node.  Store: the forward's workspace (sphere
    records, tile and block lists, each pixel's tracked-hit bound and blend
    reference) stays alive until the backward pass.  Recompute (the
    renderer's memory budget is smaller than that workspace): the workspace is
    released after the forward pass, and the backward pass rebuilds it (the
    lists and every pixel's n_track hit list) by rendering again before it
    differentiates."""

    @staticmethod
    def forward(ctx, renderer, pos, feat, rad, opa, cam, bg):
        s = renderer.settings
        fr, image, log_norm = forward_frame(s, pos, feat, rad, opa, cam, bg, renderer.capacity,
                                            check_overflow=renderer.check_overflow)
        renderer.capacity = max(renderer.capacity, int(fr.params.list_capacity))
        renderer.last_workspace_bytes = int(fr.ws_bytes)
        keep = renderer.keeps_workspace(fr.ws_bytes)
        renderer.last_mode = "store" if keep else "recompute"
        ctx.frame = fr if keep else None
        # what the backward pass re-renders with, should it recompute
        ctx.settings = replace(s)
        ctx.capacity = int(fr.params.list_capacity)
        ctx.check_overflow = renderer.check_overflow
        ctx.save_for_backward(pos, feat, rad, opa, cam, bg, image, log_norm)
        ctx.mark_non_differentiable(log_norm)
        return image, log_norm

    @staticmethod
    def backward(ctx, grad_image, _grad_log_norm):
        pos, feat, rad, opa, cam, bg, image, log_norm = ctx.saved_tensors
        need = ctx.needs_input_grad
        mask = 0
        for flag, k in ((_lib.GRAD_POS, 1), (_lib.GRAD_FEAT, 2), (_lib.GRAD_RAD, 3), (_lib.GRAD_OPA, 4),
                        (_lib.GRAD_CAM, 5), (_lib.GRAD_BG, 6)):
            if need[k]:
                mask |= flag
        if mask == 0:
            return (None,) * 7
        fr = ctx.frame
        if fr is None:   # recompute: the lists and hit lists of the same render, rebuilt
            fr, image, log_norm = forward_frame(ctx.settings, pos, feat, rad, opa, cam, bg, ctx.capacity,
                                                check_overflow=ctx.check_overflow)
        g_pos, g_rad, g_opa, g_feat, g_cam, g_bg = backward_frame(
            fr, pos, feat, rad, opa, cam, bg, image, log_norm, grad_image.contiguous(), mask)
        ctx.frame = None
        return None, g_pos, g_feat, g_rad, g_opa, g_cam, g_bg


class _AxisAngleCamera(torch.autograd.Function):
    """Listing 1's 8-vector camera [t, axis-angle rotation, focal, sensor
    width] as the renderer's 11-vector, with the gradient back through the
    conversion (both in the library)."""

    @staticmethod
    def forward(ctx, cam8):
        cam8 = cam8.contiguous()
        cam11 = torch.empty((11,), dtype=torch.float32, device=cam8.device)
        _lib.camera_from_axis_angle(cam8.data_ptr(), cam11.data_ptr(), 1,
                                    torch.cuda.current_stream(cam8.device).cuda_stream)
        ctx.save_for_backward(cam8)
        return cam11

    @staticmethod
    def backward(ctx, g11):
        (cam8,) = ctx.saved_tensors
        g11 = g11.contiguous()
        g8 = torch.empty((8,), dtype=torch.float32, device=cam8.device)
        _lib.camera_axis_angle_backward(cam8.data_ptr(), g11.data_ptr(), g8.data_ptr(), 1,
                                        torch.cuda.current_stream(cam8.device).cuda_stream)
        return g8


def camera_from_axis_angle(cam8: torch.Tensor) -> torch.Tensor:
    """The 11-vector camera of an 8-vector [t(3), axis-angle(3), focal, sensor width]."""
    return _AxisAngleCamera.apply(_dev_f32("cam", cam8, (8,)))


class Renderer(torch.nn.Module):
    """Differentiable sphere renderer for a fixed image size (Listing 1).

    ``forward(pos, feat, rad, cam, opa=None, bg=None)`` returns the H x W x C
    feature image.  ``cam`` is the 11-vector [t, 6D rotation, focal, sensor
    width] or Listing 1's 8-vector [t, axis-angle rotation, focal, sensor
    width]; opacities default to 1 and the background to 0.

    ``memory_budget`` (bytes, None = unlimited) is what a render may keep
    alive between its forward and backward pass.  When the render's
    workspace fits, it is kept (store); otherwise it is released after the
    forward pass and the backward pass recomputes the tile lists and each
    pixel's n_track hit list by rendering again (recompute).  ``last_mode``
    and ``last_workspace_bytes`` report the choice of the latest forward.
    ``segment`` and ``persistent`` are the scheduling options of
    ``RenderSettings`` (the autotuner's choice can be passed here).
    """

    def __init__(self, width: int, height: int, max_n_spheres: int, n_channels: int = 3,
                 n_track: int = 5, gamma: float = 0.1, eps: float = 1e-5, znear: float = 1.0,
                 zfar: float = 20.0, store_hits: bool = True, dist_literal: bool = False,
                 min_size: bool = True, list_capacity: int | None = None,
                 check_overflow: bool = True, memory_budget: int | None = None, segment: int = 0,
                 persistent: bool = False):
        super().__init__()
        self.settings = RenderSettings(width, height, n_channels, n_track, gamma, eps, znear, zfar,
                                       store_hits, dist_literal, min_size, segment=segment,
                                       persistent=persistent)
        self.max_n_spheres = int(max_n_spheres)
        self.capacity = int(list_capacity or _default_capacity(self.settings, self.max_n_spheres))
        self.check_overflow = check_overflow
        self.memory_budget = memory_budget
        self.last_log_norm = None
        self.last_mode = None
        self.last_workspace_bytes = 0

    def keeps_workspace(self, ws_bytes: int) -> bool:
        """Whether a render whose workspace takes ws_bytes keeps it for the backward pass."""
        return self.memory_budget is None or int(ws_bytes) <= int(self.memory_budget)

    def forward(self, pos, feat, rad, cam, opa=None, bg=None, gamma: float | None = None,
                max_depth: float | None = None):
        s = self.settings
        if gamma is not None:
            s.gamma = float(gamma)
        if max_depth is not None:
            s.zfar = float(max_depth)
        M = int(pos.shape[0])
        if M > self.max_n_spheres:
            raise ValueError(f"{M} spheres exceed max_n_spheres={self.max_n_spheres}")
        C = s.n_channels
        dev = pos.device
        if opa is None:
            opa = torch.ones((M,), dtype=torch.float32, device=dev)
        if bg is None:
            bg = torch.zeros((C,), dtype=torch.float32, device=dev)
        pos = _dev_f32("pos", pos, (M, 3))
        feat = _dev_f32("feat", feat, (M, C))
        rad = _dev_f32("rad", rad, (M,))
        opa = _dev_f32("opa", opa, (M,))
        if cam.numel() == 8:
            cam = camera_from_axis_angle(cam.reshape(8))
        cam = _dev_f32("cam", cam, (11,))
        bg = _dev_f32("bg", bg, (C,))
        image, log_norm = _RenderFunction.apply(self, pos, feat, rad, opa, cam, bg)
        self.last_log_norm = log_norm
        return image
