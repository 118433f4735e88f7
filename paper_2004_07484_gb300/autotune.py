"""Scheduling autotuner for batched renders.

The paper renders one scene per call with a fixed launch shape.  For a batch
of uneven scenes, two scheduling choices of this library change only the
speed, never the result: the segment length (list entries per work item; a
tile's list is split into segments rendered in parallel and merged; with the
paper's early termination one unit walks a tile's segments in order) and the
kernel form (one CTA per work unit, or persistent CTAs taking units from a
counter).  ``tune`` sizes every scene's pair-list capacity from one binning
pass of the batch itself, then times the batch's forward + backward for each
candidate and keeps the fastest.  Results are cached per batch signature
(scene count, image sizes, sphere counts rounded to powers of two, channels,
n_track and mode flags).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import torch

from . import _lib
from .renderer import RenderSettings, backward_batch, forward_batch

SEGMENTS = (512, 1024, 2048, 2560, 3072, 4096, 8192)
FORMS = (False, True)          # persistent
CAPACITY_MARGIN = 1.25


@dataclass
class Choice:
    segment: int
    persistent: bool
    capacities: list[int]
    ms: dict                   # (segment, persistent) -> median fwd+bwd milliseconds


_cache: dict[tuple, Choice] = {}


def signature(settings: list[RenderSettings], n_spheres: list[int]) -> tuple:
    s0 = settings[0]
    sizes = tuple(sorted((s.width, s.height, max(0, int(math.log2(max(m, 1))))) for s, m in
                         zip(settings, n_spheres)))
    return (len(settings), sizes, s0.n_channels, s0.n_track, s0.store_hits, s0.dist_literal, s0.min_size,
            s0.paper_stop, s0.orthographic, s0.paper_gradients)


def pairs_per_scene(settings: list[RenderSettings], inputs) -> list[int]:
    """(tile, sphere) pairs each scene needs, from one binning pass of the batch."""
    caps = [max(4 * int(x[0].shape[0]), 1 << 12) for x in inputs]
    fr, _, _ = forward_batch(settings, inputs, caps, check_overflow=True)
    nt = [((s.width + s.tile - 1) // s.tile) * ((s.height + s.tile - 1) // s.tile) for s in settings]
    dev = inputs[0][0].device
    ranges = torch.empty((sum(nt), 2), dtype=torch.int32, device=dev)
    ids = torch.empty((max(sum(fr.capacities()), 1),), dtype=torch.int32, device=dev)
    _lib.read_tile_lists_batched(fr.params, fr.ws.data_ptr(), fr.ws_bytes, ranges.data_ptr(),
                                 ids.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
    lens = (ranges[:, 1] - ranges[:, 0]).to(torch.int64).cpu()
    out, t0 = [], 0
    for n in nt:
        out.append(int(lens[t0:t0 + n].sum()))
        t0 += n
    return out


L2_FLUSH_BYTES = 256 << 20   # more than the GPU's L2
_flush: dict = {}


def _flush_l2(dev):
    """Overwrites a buffer larger than L2, so that each timed step starts with
    the cold cache a training step meets after its optimiser update."""
    buf = _flush.get(dev)
    if buf is None:
        buf = _flush[dev] = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    buf.zero_()


def time_step(settings, inputs, grads, capacities, reps: int = 5) -> float:
    """Median milliseconds of one batched forward + backward (CUDA events),
    each started with a flushed L2."""
    dev = inputs[0][0].device
    stream = torch.cuda.current_stream(dev)
    times = []
    for i in range(reps + 1):
        _flush_l2(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fr, images, log_norms = forward_batch(settings, inputs, capacities, check_overflow=False)
        backward_batch(fr, inputs, images, log_norms, grads)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if i:
            times.append(e0.elapsed_time(e1))
    times.sort()
    return times[len(times) // 2]


def tune(settings: list[RenderSettings], inputs, grads, reps: int = 5, use_cache: bool = True) -> Choice:
    """Picks segment length and kernel form for this batch; returns the choice
    (the settings themselves are not modified: apply it with ``apply``)."""
    key = signature(settings, [int(x[0].shape[0]) for x in inputs])
    if use_cache and key in _cache:
        return _cache[key]
    pairs = pairs_per_scene(settings, inputs)
    caps = [int(p * CAPACITY_MARGIN) + 1024 for p in pairs]
    ms = {}
    for seg in SEGMENTS:
        for pers in FORMS:
            cand = [replace(s, segment=seg, persistent=pers) for s in settings]
            ms[(seg, pers)] = time_step(cand, inputs, grads, caps, reps)
    best = min(ms, key=ms.get)
    choice = Choice(best[0], best[1], caps, ms)
    _cache[key] = choice
    return choice


def apply(settings: list[RenderSettings], choice: Choice) -> list[RenderSettings]:
    return [replace(s, segment=choice.segment, persistent=choice.persistent) for s in settings]
