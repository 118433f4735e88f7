"""GB300-native differentiable sphere renderer (Pulsar, arXiv 2004.07484).

The hot path (projection, depth sort, tile binning, forward blend and
backward pass) runs in hand-written CUDA kernels for sm_103a behind the C ABI
of include/pulsar.h; ``renderer.Renderer`` wraps it as a PyTorch module.
"""
from .renderer import (BatchFrame, Renderer, RenderSettings, backward_batch,  # noqa: F401
                       backward_frame, camera_from_axis_angle, forward_batch, forward_frame)

__all__ = ["Renderer", "RenderSettings", "forward_frame", "backward_frame", "BatchFrame",
           "forward_batch", "backward_batch", "camera_from_axis_angle"]
