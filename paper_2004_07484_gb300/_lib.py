"""ctypes binding of ``libpulsar_gb300.so`` (the C ABI in include/pulsar.h).

Argument marshalling only: every step of the renderer runs in the library's
CUDA kernels.  Importing this module loads the in-tree library and fails
loudly when it is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpulsar_gb300.so")

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = range(6)

FLAG_STORE_HITS = 1 << 0
FLAG_DIST_LITERAL = 1 << 1
FLAG_NO_MIN_SIZE = 1 << 2
FLAG_PERSISTENT = 1 << 3
FLAG_ACCUMULATE = 1 << 4
FLAG_PAPER_GRADIENTS = 1 << 5
FLAG_ORTHOGRAPHIC = 1 << 6
FLAG_PAPER_STOP = 1 << 7

GRAD_POS, GRAD_RAD, GRAD_OPA, GRAD_FEAT, GRAD_CAM, GRAD_BG = (1 << k for k in range(6))
GRAD_ALL = 63

EXPORTED = ("pulsar_workspace_size", "pulsar_project", "pulsar_bin", "pulsar_render_fwd",
            "pulsar_render_bwd", "pulsar_read_tile_lists", "pulsar_read_status",
            "pulsar_status_string", "pulsar_render_fwd_static", "pulsar_static_read_status", "pulsar_workspace_size_batched",
            "pulsar_project_batched", "pulsar_bin_batched", "pulsar_render_fwd_batched",
            "pulsar_render_bwd_batched", "pulsar_read_tile_lists_batched",
            "pulsar_probe_fma_throughput", "pulsar_last_overflow", "pulsar_render_batched",
            "pulsar_image_loss", "pulsar_adam_step", "pulsar_camera_from_axis_angle",
            "pulsar_camera_axis_angle_backward", "pulsar_prune_scratch_bytes", "pulsar_prune", "pulsar_subdivide")

MAX_SCENES = 64
LOSS_L2, LOSS_L1 = 0, 1
LOSS_SCRATCH_FLOATS = 1024
ADAM_MAX_TENSORS = 8


class Params(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("n_spheres", ctypes.c_int32), ("n_channels", ctypes.c_int32),
        ("n_track", ctypes.c_int32), ("tile", ctypes.c_int32),
        ("list_capacity", ctypes.c_int64),
        ("gamma", ctypes.c_float), ("eps", ctypes.c_float),
        ("znear", ctypes.c_float), ("zfar", ctypes.c_float),
        ("flags", ctypes.c_uint32), ("segment", ctypes.c_int32),
        ("min_contrib", ctypes.c_float),
    ]


class SceneArgs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("pos", "rad", "opa", "feat", "cam", "bg")]


class FwdOut(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("image", "log_norm", "n_hits", "n_tests", "tracked")]


class BwdIO(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("image", "log_norm", "grad_image", "g_pos", "g_rad",
                                               "g_opa", "g_feat", "g_cam", "g_bg")]


class AdamTensor(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("n", ctypes.c_int64), ("lo", ctypes.c_float), ("hi", ctypes.c_float)]


class AdamHyper(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("zero_grad", ctypes.c_int32)]


ADAM_STATE_BYTES = 16   # pulsar_adam_state: int32 t, float step_size, float inv_sqrt_bc2, int32


class PulsarError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


_lib = None


def lib():
    """The loaded library.  Raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2004_07484_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz, u32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32
        P, S = ctypes.POINTER(Params), ctypes.POINTER(SceneArgs)
        L.pulsar_workspace_size.argtypes = [P]
        L.pulsar_workspace_size.restype = sz
        L.pulsar_project.argtypes = [P, S, vp, sz, vp]
        L.pulsar_project.restype = ctypes.c_int
        L.pulsar_bin.argtypes = [P, vp, sz, vp]
        L.pulsar_bin.restype = ctypes.c_int
        L.pulsar_render_fwd.argtypes = [P, S, vp, sz, vp, vp, vp, vp, vp, vp]
        L.pulsar_render_fwd.restype = ctypes.c_int
        L.pulsar_render_bwd.argtypes = [P, S, vp, sz, vp, vp, vp, u32, vp, vp, vp, vp, vp, vp, vp]
        L.pulsar_render_bwd.restype = ctypes.c_int
        L.pulsar_read_tile_lists.argtypes = [P, vp, sz, vp, vp, vp]
        L.pulsar_read_tile_lists.restype = ctypes.c_int
        L.pulsar_read_status.argtypes = [vp, sz, ctypes.POINTER(ctypes.c_int64), vp]
        L.pulsar_read_status.restype = ctypes.c_int
        L.pulsar_status_string.argtypes = [ctypes.c_int]
        L.pulsar_status_string.restype = ctypes.c_char_p
        L.pulsar_render_fwd_static.argtypes = [P, S, vp, vp, vp]
        L.pulsar_render_fwd_static.restype = ctypes.c_int
        L.pulsar_static_read_status.argtypes = [ctypes.POINTER(ctypes.c_int64), vp]
        L.pulsar_static_read_status.restype = ctypes.c_int
        i32 = ctypes.c_int
        L.pulsar_workspace_size_batched.argtypes = [i32, P]
        L.pulsar_workspace_size_batched.restype = sz
        L.pulsar_project_batched.argtypes = [i32, P, S, vp, sz, vp]
        L.pulsar_project_batched.restype = ctypes.c_int
        L.pulsar_bin_batched.argtypes = [i32, P, vp, sz, vp]
        L.pulsar_bin_batched.restype = ctypes.c_int
        L.pulsar_render_fwd_batched.argtypes = [i32, P, S, vp, sz, ctypes.POINTER(FwdOut), vp]
        L.pulsar_render_fwd_batched.restype = ctypes.c_int
        L.pulsar_render_bwd_batched.argtypes = [i32, P, S, vp, sz, ctypes.POINTER(BwdIO), u32, vp]
        L.pulsar_render_bwd_batched.restype = ctypes.c_int
        L.pulsar_read_tile_lists_batched.argtypes = [i32, P, vp, sz, vp, vp, vp]
        L.pulsar_read_tile_lists_batched.restype = ctypes.c_int
        L.pulsar_last_overflow.argtypes = [P, vp, sz, ctypes.POINTER(ctypes.c_size_t), vp]
        L.pulsar_last_overflow.restype = ctypes.c_int
        L.pulsar_render_batched.argtypes = [i32, P, S, vp, sz, ctypes.POINTER(FwdOut), vp]
        L.pulsar_render_batched.restype = ctypes.c_int
        L.pulsar_probe_fma_throughput.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_float), vp]
        L.pulsar_probe_fma_throughput.restype = ctypes.c_int
        L.pulsar_image_loss.argtypes = [i32, vp, vp, ctypes.c_int64, ctypes.c_float, vp, vp, vp, vp]
        L.pulsar_image_loss.restype = ctypes.c_int
        L.pulsar_adam_step.argtypes = [i32, ctypes.POINTER(AdamTensor), ctypes.POINTER(AdamHyper), vp, vp]
        L.pulsar_adam_step.restype = ctypes.c_int
        L.pulsar_camera_from_axis_angle.argtypes = [vp, vp, i32, vp]
        L.pulsar_camera_from_axis_angle.restype = ctypes.c_int
        L.pulsar_camera_axis_angle_backward.argtypes = [vp, vp, vp, i32, vp]
        L.pulsar_camera_axis_angle_backward.restype = ctypes.c_int
        i64, f32 = ctypes.c_int64, ctypes.c_float
        L.pulsar_prune_scratch_bytes.argtypes = [i64]
        L.pulsar_prune_scratch_bytes.restype = sz
        L.pulsar_prune.argtypes = [i64, i32, vp, vp, vp, vp, vp, vp, f32, vp, vp, vp, vp, vp, vp, sz, vp]
        L.pulsar_prune.restype = ctypes.c_int
        L.pulsar_subdivide.argtypes = [i64, i32, vp, vp, vp, vp, f32, f32, vp, vp, vp, vp, vp]
        L.pulsar_subdivide.restype = ctypes.c_int
        _lib = L
    return _lib


STATIC_WORKSPACE_BYTES = 64 << 20


def render_fwd_static(p: Params, s: SceneArgs, image: int, log_norm: int, stream: int) -> None:
    """Forward render using the library's fixed device array as workspace (no allocation)."""
    _check(lib().pulsar_render_fwd_static(ctypes.byref(p), ctypes.byref(s), image, log_norm, stream),
           "pulsar_render_fwd_static")


def static_read_status(stream: int) -> tuple[int, int]:
    """(status, pairs_needed) of the last render_fwd_static call; synchronises the stream."""
    need = ctypes.c_int64(0)
    st = lib().pulsar_static_read_status(ctypes.byref(need), stream)
    return int(st), int(need.value)


def status_string(status: int) -> str:
    return lib().pulsar_status_string(int(status)).decode()


def _check(status: int, where: str) -> None:
    if status != OK:
        raise PulsarError(status, where)


def workspace_size(p: Params) -> int:
    n = lib().pulsar_workspace_size(ctypes.byref(p))
    if n == 0:
        raise PulsarError(ERR_INVALID_ARG, "pulsar_workspace_size")
    return int(n)


def project(p: Params, s: SceneArgs, ws: int, ws_bytes: int, stream: int) -> None:
    _check(lib().pulsar_project(ctypes.byref(p), ctypes.byref(s), ws, ws_bytes, stream), "pulsar_project")


def bin(p: Params, ws: int, ws_bytes: int, stream: int) -> None:  # noqa: A001 - C name
    _check(lib().pulsar_bin(ctypes.byref(p), ws, ws_bytes, stream), "pulsar_bin")


def render_fwd(p: Params, s: SceneArgs, ws: int, ws_bytes: int, image: int, log_norm: int,
               n_hits: int | None, n_tests: int | None, tracked: int | None, stream: int) -> None:
    _check(lib().pulsar_render_fwd(ctypes.byref(p), ctypes.byref(s), ws, ws_bytes, image, log_norm,
                                   n_hits, n_tests, tracked, stream), "pulsar_render_fwd")


def render_bwd(p: Params, s: SceneArgs, ws: int, ws_bytes: int, image: int, log_norm: int,
               grad_image: int, grad_mask: int, g_pos, g_rad, g_opa, g_feat, g_cam, g_bg,
               stream: int) -> None:
    _check(lib().pulsar_render_bwd(ctypes.byref(p), ctypes.byref(s), ws, ws_bytes, image, log_norm,
                                   grad_image, grad_mask, g_pos, g_rad, g_opa, g_feat, g_cam, g_bg,
                                   stream), "pulsar_render_bwd")


def read_tile_lists(p: Params, ws: int, ws_bytes: int, ranges: int, ids: int, stream: int) -> None:
    _check(lib().pulsar_read_tile_lists(ctypes.byref(p), ws, ws_bytes, ranges, ids, stream),
           "pulsar_read_tile_lists")


def read_status(ws: int, ws_bytes: int, stream: int) -> tuple[int, int]:
    """(status, pairs_needed); synchronises the stream."""
    need = ctypes.c_int64(0)
    st = lib().pulsar_read_status(ws, ws_bytes, ctypes.byref(need), stream)
    return int(st), int(need.value)


# ---------------------------------------------------------------------------
# batched entry points: `ps` is a ctypes array of Params, `ss` of SceneArgs,
# `outs` of FwdOut, `ios` of BwdIO (one element per scene)
# ---------------------------------------------------------------------------

def workspace_size_batched(ps) -> int:
    n = lib().pulsar_workspace_size_batched(len(ps), ps)
    if n == 0:
        raise PulsarError(ERR_INVALID_ARG, "pulsar_workspace_size_batched")
    return int(n)


def project_batched(ps, ss, ws: int, ws_bytes: int, stream: int) -> None:
    _check(lib().pulsar_project_batched(len(ps), ps, ss, ws, ws_bytes, stream), "pulsar_project_batched")


def bin_batched(ps, ws: int, ws_bytes: int, stream: int) -> None:
    _check(lib().pulsar_bin_batched(len(ps), ps, ws, ws_bytes, stream), "pulsar_bin_batched")


def render_fwd_batched(ps, ss, ws: int, ws_bytes: int, outs, stream: int) -> None:
    _check(lib().pulsar_render_fwd_batched(len(ps), ps, ss, ws, ws_bytes, outs, stream),
           "pulsar_render_fwd_batched")


def render_bwd_batched(ps, ss, ws: int, ws_bytes: int, ios, grad_mask: int, stream: int) -> None:
    _check(lib().pulsar_render_bwd_batched(len(ps), ps, ss, ws, ws_bytes, ios, grad_mask, stream),
           "pulsar_render_bwd_batched")


def read_tile_lists_batched(ps, ws: int, ws_bytes: int, ranges: int, ids: int, stream: int) -> None:
    _check(lib().pulsar_read_tile_lists_batched(len(ps), ps, ws, ws_bytes, ranges, ids, stream),
           "pulsar_read_tile_lists_batched")


def probe_fma_throughput(sink: int, iters: int, stream: int) -> tuple[float, float]:
    """(FP32 FLOP/s, kernel milliseconds) of the FMA probe; synchronises the stream."""
    f, ms = ctypes.c_double(0.0), ctypes.c_float(0.0)
    _check(lib().pulsar_probe_fma_throughput(sink, int(iters), ctypes.byref(f), ctypes.byref(ms), stream),
           "pulsar_probe_fma_throughput")
    return float(f.value), float(ms.value)


def last_overflow(p: Params, ws: int, ws_bytes: int, stream: int) -> tuple[int, int]:
    """(status, workspace bytes needed); synchronises the stream."""
    need = ctypes.c_size_t(0)
    st = lib().pulsar_last_overflow(ctypes.byref(p), ws, ws_bytes, ctypes.byref(need), stream)
    return int(st), int(need.value)


def render_batched(ps, ss, ws: int, ws_bytes: int, outs, stream: int) -> None:
    _check(lib().pulsar_render_batched(len(ps), ps, ss, ws, ws_bytes, outs, stream), "pulsar_render_batched")


def image_loss(kind: int, image: int, target: int, n: int, scale: float, grad: int | None,
               loss: int | None, scratch: int, stream: int) -> None:
    _check(lib().pulsar_image_loss(int(kind), image, target, int(n), float(scale), grad, loss, scratch, stream),
           "pulsar_image_loss")


def adam_step(tensors, hyper: AdamHyper, state: int, stream: int) -> None:
    """`tensors`: ctypes array of AdamTensor."""
    _check(lib().pulsar_adam_step(len(tensors), tensors, ctypes.byref(hyper), state, stream), "pulsar_adam_step")


def camera_from_axis_angle(cam8: int, cam11: int, n: int, stream: int) -> None:
    _check(lib().pulsar_camera_from_axis_angle(cam8, cam11, int(n), stream), "pulsar_camera_from_axis_angle")


def camera_axis_angle_backward(cam8: int, g_cam11: int, g_cam8: int, n: int, stream: int) -> None:
    _check(lib().pulsar_camera_axis_angle_backward(cam8, g_cam11, g_cam8, int(n), stream),
           "pulsar_camera_axis_angle_backward")


def prune_scratch_bytes(n: int) -> int:
    return int(lib().pulsar_prune_scratch_bytes(int(n)))


def prune(n, C, pos, rad, opa, feat, bg, activity, color_tol, out_pos, out_rad, out_opa, out_feat, n_out,
          scratch, scratch_bytes, stream) -> None:
    _check(lib().pulsar_prune(int(n), int(C), pos, rad, opa, feat, bg, activity, float(color_tol), out_pos, out_rad,
                              out_opa, out_feat, n_out, scratch, int(scratch_bytes), stream), "pulsar_prune")


def subdivide(n, C, pos, rad, opa, feat, offset_scale, radius_scale, out_pos, out_rad, out_opa, out_feat,
              stream) -> None:
    _check(lib().pulsar_subdivide(int(n), int(C), pos, rad, opa, feat, float(offset_scale), float(radius_scale),
                                  out_pos, out_rad, out_opa, out_feat, stream), "pulsar_subdivide")
