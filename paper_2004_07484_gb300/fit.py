"""Fitting a sphere scene to target views (Sec. 3.4, "End-to-end Optimization";
the scene fit of Sec. 5).

``ViewFit`` holds one sphere set (positions, radii, opacities, features) and
V target views with their cameras.  One ``step`` renders every view as one
batch whose scenes share the sphere arrays, takes the image loss against the
targets with its gradient dL/dF, runs the batched backward pass with every
view adding into one set of gradient buffers, and applies one Adam step
(Kingma & Ba), which also zeroes the gradients for the next step.  All of it
runs in ``libpulsar_gb300.so`` (include/pulsar.h, include/pulsar_fit.h) on
buffers allocated once, so a step can be captured in a CUDA graph and
replayed (``capture`` / ``replay``).

Parameters are kept in a box after each update (box-projected Adam): radii
at or above ``rad_min``, opacities in [0, 1], positions and features free.
The paper states no constraint; the renderer's early-termination bound
assumes opacities of at most 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import torch

from . import _lib
from .renderer import RenderSettings, _dev_f32, scene_args

PARAM_NAMES = ("pos", "rad", "opa", "feat")


@dataclass
class AdamSettings:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    loss: str = "l2"              # "l2": sum (F - T)^2; "l1": sum |F - T|
    loss_scale: float = 1.0       # L is multiplied by this (1 / n for a mean)
    rad_min: float = 1e-4
    opa_range: tuple = (0.0, 1.0)


class ViewFit:
    """Adam fit of one sphere set to V views (all of one image size)."""

    def __init__(self, settings: RenderSettings, cams: list, targets: torch.Tensor, pos, rad, opa, feat,
                 bg, capacity: int | list[int], adam: AdamSettings | None = None):
        V = len(cams)
        if not 1 <= V <= _lib.MAX_SCENES:
            raise ValueError(f"1..{_lib.MAX_SCENES} views, got {V}")
        dev = pos.device
        M, C = int(pos.shape[0]), settings.n_channels
        H, W = settings.height, settings.width
        self.settings = replace(settings, accumulate=True)
        self.adam = adam or AdamSettings()
        self.n_views, self.n_spheres, self.device = V, M, dev
        self.params = {
            "pos": _dev_f32("pos", pos, (M, 3)).clone(),
            "rad": _dev_f32("rad", rad, (M,)).clone(),
            "opa": _dev_f32("opa", opa, (M,)).clone(),
            "feat": _dev_f32("feat", feat, (M, C)).clone(),
        }
        self.bg = _dev_f32("bg", bg, (C,)).clone()
        self.cams = torch.stack([_dev_f32("cam", c, (11,)) for c in cams]).contiguous()
        self.targets = _dev_f32("targets", targets, (V, H, W, C)).contiguous()
        self.grads = {k: torch.zeros_like(t) for k, t in self.params.items()}
        self.m = {k: torch.zeros_like(t) for k, t in self.params.items()}
        self.v = {k: torch.zeros_like(t) for k, t in self.params.items()}
        self.state = torch.zeros(_lib.ADAM_STATE_BYTES // 4, dtype=torch.int32, device=dev)
        self.images = torch.empty((V, H, W, C), dtype=torch.float32, device=dev)
        self.log_norms = torch.empty((V, H, W), dtype=torch.float32, device=dev)
        self.grad_images = torch.empty((V, H, W, C), dtype=torch.float32, device=dev)
        self.loss = torch.zeros((1,), dtype=torch.float32, device=dev)
        self.scratch = torch.empty((_lib.LOSS_SCRATCH_FLOATS,), dtype=torch.float32, device=dev)
        caps = capacity if isinstance(capacity, list) else [int(capacity)] * V
        self._set_capacities(caps)
        p = self.params
        self.ss = (_lib.SceneArgs * V)(*[scene_args(p["pos"], p["feat"], p["rad"], p["opa"], self.cams[k],
                                                    self.bg) for k in range(V)])
        self.outs = (_lib.FwdOut * V)(*[_lib.FwdOut(self.images[k].data_ptr(), self.log_norms[k].data_ptr(),
                                                    None, None, None) for k in range(V)])
        g = self.grads
        self.ios = (_lib.BwdIO * V)(*[_lib.BwdIO(self.images[k].data_ptr(), self.log_norms[k].data_ptr(),
                                                 self.grad_images[k].data_ptr(), g["pos"].data_ptr(),
                                                 g["rad"].data_ptr(), g["opa"].data_ptr(),
                                                 g["feat"].data_ptr(), None, None) for k in range(V)])
        a = self.adam
        inf = math.inf
        bounds = {"pos": (-inf, inf), "rad": (a.rad_min, inf), "opa": tuple(a.opa_range), "feat": (-inf, inf)}
        self.adam_tensors = (_lib.AdamTensor * len(PARAM_NAMES))(*[
            _lib.AdamTensor(p[k].data_ptr(), g[k].data_ptr(), self.m[k].data_ptr(), self.v[k].data_ptr(),
                            p[k].numel(), bounds[k][0], bounds[k][1]) for k in PARAM_NAMES])
        self.hyper = _lib.AdamHyper(a.lr, a.beta1, a.beta2, a.eps, 1)
        self.loss_kind = {"l2": _lib.LOSS_L2, "l1": _lib.LOSS_L1}[a.loss]
        self.grad_mask = _lib.GRAD_POS | _lib.GRAD_RAD | _lib.GRAD_OPA | _lib.GRAD_FEAT
        self.graph = None

    def _set_capacities(self, caps: list[int]) -> None:
        V = self.n_views
        self.ps = (_lib.Params * V)(*[self.settings.params(self.n_spheres, int(c)) for c in caps])
        self.ws_bytes = _lib.workspace_size_batched(self.ps)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.graph = None

    def capacities(self) -> list[int]:
        return [int(p.list_capacity) for p in self.ps]

    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def _render(self, stream: int) -> None:
        _lib.render_batched(self.ps, self.ss, self.ws.data_ptr(), self.ws_bytes, self.outs, stream)

    def _loss(self, with_grad: bool, stream: int) -> None:
        _lib.image_loss(self.loss_kind, self.images.data_ptr(), self.targets.data_ptr(), self.images.numel(),
                        self.adam.loss_scale, self.grad_images.data_ptr() if with_grad else None,
                        self.loss.data_ptr(), self.scratch.data_ptr(), stream)

    def _step(self, stream: int) -> None:
        self._render(stream)
        self._loss(True, stream)
        _lib.render_bwd_batched(self.ps, self.ss, self.ws.data_ptr(), self.ws_bytes, self.ios,
                                self.grad_mask, stream)
        _lib.adam_step(self.adam_tensors, self.hyper, self.state.data_ptr(), stream)

    def step(self) -> torch.Tensor:
        """One fit step; returns the device loss of the parameters before the update."""
        self._step(self._stream())
        return self.loss

    def evaluate(self) -> torch.Tensor:
        """Renders the views and returns the device loss (no update)."""
        s = self._stream()
        self._render(s)
        self._loss(False, s)
        return self.loss

    def capture(self) -> None:
        """Captures one step in a CUDA graph on a side stream (capture runs nothing;
        ``replay`` runs the step)."""
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=side):
            self._step(side.cuda_stream)
        torch.cuda.current_stream(self.device).wait_stream(side)

    def replay(self) -> torch.Tensor:
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.loss

    def steps_taken(self) -> int:
        return int(self.state[0].item())

    def overflowed(self) -> int:
        """0 when every view's (tile, sphere) pairs fitted the capacities at
        the last render; else the pairs the batch needed (synchronises)."""
        st, need = _lib.read_status(self.ws.data_ptr(), self.ws_bytes, self._stream())
        if st == _lib.OK:
            return 0
        if st != _lib.ERR_CAPACITY:
            raise _lib.PulsarError(st, "pulsar_read_status")
        return need

    def grow(self, pairs_needed: int, margin: float = 1.25) -> None:
        """Raises the capacities (proportionally) to hold pairs_needed with a
        margin; drops a captured graph."""
        caps = self.capacities()
        f = margin * pairs_needed / max(sum(caps), 1)
        self._set_capacities([int(c * f) + 1024 for c in caps])

    def run(self, n_steps: int, graph: bool = True) -> None:
        for _ in range(n_steps):
            if graph:
                self.replay()
            else:
                self.step()


# Pruning and subdivision between fit stages (Sec. 5, head reconstruction):
# spheres whose colour converged to the background or that received no
# gradient are removed; every sphere can be refined into 12 in a face-centred
# cubic arrangement.  The printed child radius ("sqrt 2 r") cannot be a
# refinement; the defaults below place the 12 children at distance r / sqrt 2
# with radius r / (2 sqrt 2), so neighbouring children touch and all stay
# within about the parent's radius.
SUBDIVIDE_OFFSET = 2.0 ** -0.5
SUBDIVIDE_RADIUS = 2.0 ** -1.5


def prune_spheres(pos, rad, opa, feat, bg, activity=None, color_tol: float = -1.0):
    """The kept spheres, in order: (pos, rad, opa, feat)."""
    M, C = int(pos.shape[0]), int(feat.shape[1])
    dev = pos.device
    outs = (torch.empty_like(pos), torch.empty_like(rad), torch.empty_like(opa), torch.empty_like(feat))
    n_out = torch.zeros((1,), dtype=torch.int64, device=dev)
    nb = _lib.prune_scratch_bytes(M)
    scratch = torch.empty((max(nb, 16),), dtype=torch.uint8, device=dev)
    args = [t.contiguous() for t in (pos, rad, opa, feat, bg)]
    act = None if activity is None else activity.contiguous()
    _lib.prune(M, C, *[t.data_ptr() for t in args], None if act is None else act.data_ptr(), color_tol,
               *[t.data_ptr() for t in outs], n_out.data_ptr(), scratch.data_ptr(), scratch.numel(),
               torch.cuda.current_stream(dev).cuda_stream)
    n = int(n_out.item())
    return tuple(t[:n].clone() for t in outs)


def subdivide_spheres(pos, rad, opa, feat, offset_scale: float = SUBDIVIDE_OFFSET,
                      radius_scale: float = SUBDIVIDE_RADIUS):
    """Each sphere as 12 children: (pos, rad, opa, feat) with 12 M spheres."""
    M, C = int(pos.shape[0]), int(feat.shape[1])
    dev = pos.device
    outs = (torch.empty((12 * M, 3), device=dev), torch.empty((12 * M,), device=dev),
            torch.empty((12 * M,), device=dev), torch.empty((12 * M, C), device=dev))
    args = [t.contiguous() for t in (pos, rad, opa, feat)]
    _lib.subdivide(M, C, *[t.data_ptr() for t in args], offset_scale, radius_scale, *[t.data_ptr() for t in outs],
                   torch.cuda.current_stream(dev).cuda_stream)
    return outs
