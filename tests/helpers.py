"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare it with the oracle."""
from __future__ import annotations

import numpy as np

from paper_2004_07484_gb300.scenes import Scene

GRAD_NAMES = ("pos", "rad", "opa", "feat", "cam", "bg")


def to_dev(scene: Scene):
    import torch
    d = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k))).cuda()
         for k in ("pos", "rad", "opa", "feat", "cam", "bg")}
    return d


def settings_of(scene: Scene, store=True, dist_literal=False, min_size=True, n_track=None, segment=0,
                persistent=False, paper=False):
    from paper_2004_07484_gb300 import RenderSettings
    return RenderSettings(scene.width, scene.height, scene.n_channels,
                          n_track or scene.n_track, float(scene.gamma), float(scene.eps),
                          float(scene.znear), float(scene.zfar), store, dist_literal, min_size,
                          segment=segment, persistent=persistent, paper_gradients=paper,
                          orthographic=bool(getattr(scene, "ortho", False)),
                          paper_stop=bool(getattr(scene, "paper_stop", False)),
                          min_contrib=float(getattr(scene, "min_contrib", 0.01)))


def gpu_forward(scene: Scene, store=True, dist_literal=False, min_size=True, capacity=None,
                n_track=None, dev=None, segment=0, persistent=False, paper=False):
    import torch
    from paper_2004_07484_gb300 import forward_frame
    dev = dev or to_dev(scene)
    s = settings_of(scene, store, dist_literal, min_size, n_track, segment, persistent, paper)
    H, W, K = scene.height, scene.width, s.n_track
    n_hits = torch.empty((H, W), dtype=torch.int32, device="cuda")
    tracked = torch.empty((H, W, K), dtype=torch.int32, device="cuda")
    cap = capacity or max(8 * scene.n_spheres, 1 << 16)
    fr, image, log_norm = forward_frame(s, dev["pos"], dev["feat"], dev["rad"], dev["opa"], dev["cam"],
                                        dev["bg"], cap, check_overflow=True, n_hits=n_hits,
                                        tracked=tracked)
    torch.cuda.synchronize()
    return dict(frame=fr, dev=dev, image=image, log_norm=log_norm, n_hits=n_hits, tracked=tracked)


def gpu_tile_lists(fr):
    import torch
    from paper_2004_07484_gb300 import _lib
    s = fr.settings
    nt = ((s.width + 15) // 16) * ((s.height + 15) // 16)
    ranges = torch.empty((nt, 2), dtype=torch.int32, device="cuda")
    cap = max(int(fr.params.list_capacity), 1)
    ids = torch.empty((cap,), dtype=torch.int32, device="cuda")
    _lib.read_tile_lists(fr.params, fr.ws.data_ptr(), fr.ws_bytes, ranges.data_ptr(), ids.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return ranges.cpu().numpy(), ids.cpu().numpy()


def gpu_backward(out, G: np.ndarray, mask=None):
    import torch
    from paper_2004_07484_gb300 import backward_frame, _lib
    d = out["dev"]
    g = torch.from_numpy(np.ascontiguousarray(G.astype(np.float32))).cuda()
    res = backward_frame(out["frame"], d["pos"], d["feat"], d["rad"], d["opa"], d["cam"], d["bg"],
                         out["image"], out["log_norm"], g, _lib.GRAD_ALL if mask is None else mask)
    torch.cuda.synchronize()
    return {k: (None if v is None else v.cpu().numpy().astype(np.float64)) for k, v in zip(GRAD_NAMES, res)}


def assert_tile_lists_equal(ranges, ids, off, oids):
    nt = len(off) - 1
    assert ranges.shape[0] == nt
    for t in range(nt):
        b, e = ranges[t]
        got = ids[b:e] if e > b else ids[:0]
        want = oids[off[t]:off[t + 1]]
        assert np.array_equal(got, want), (t, got[:10], want[:10], len(got), len(want))


# Gradient tolerance.  The bar is 1e-3 relative per tensor (max-norm).  Each
# element is also held to 1e-3 of itself, with an absolute floor of 1e-5 of
# the tensor's largest element: a float32 element is a sum of per-pixel
# contributions up to ~0.2 of that scale, each with up to ~3e-5 relative error
# at sphere rims (d = 1 - dist/R has an absolute float32 error of ~1e-7), so
# an element whose contributions cancel to a small total cannot be held
# tighter than that.
ELEM_FLOOR = 1e-2   # floor = 1e-3 * ELEM_FLOOR * max|ref| = 1e-5 * max|ref|


def _elem_bound(ref: np.ndarray, scale: float) -> np.ndarray:
    return 1e-3 * (np.abs(ref) + ELEM_FLOOR * scale)


def grad_error(g: np.ndarray, ref: np.ndarray):
    """(max-norm relative error, worst elementwise ratio to its bound)."""
    g = np.asarray(g, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    scale = float(np.abs(ref).max()) if ref.size else 0.0
    if scale == 0.0:
        return float(np.abs(g).max()) if g.size else 0.0, 0.0
    rel = float(np.abs(g - ref).max()) / scale
    worst = float((np.abs(g - ref) / _elem_bound(ref, scale)).max())
    return rel, worst


def camera_term_scale(scene, ref) -> float:
    """Sum of magnitudes of the per-sphere terms the camera gradient adds up.

    dL/dt = -sum_i dL/dp_i and dL/dR = sum_i (R dL/dp_i) (p_i - t)^T, so every
    camera element is a sum over spheres whose terms are bounded by
    |dL/dp_i| max(1, |p_i - t|).  Summing terms that each carry the float32
    relative error the per-sphere gradients are held to, an element cannot be
    held tighter than that error times this scale (the standard bound for a
    sum); it takes the place of max|dL/dcam| in the elementwise floor when it
    is the larger."""
    p = np.asarray(scene.pos, np.float64)
    if p.size == 0:
        return 0.0
    d = np.linalg.norm(p - np.asarray(scene.cam[:3], np.float64), axis=1)
    return float((np.linalg.norm(np.asarray(ref.pos, np.float64), axis=1) * np.maximum(1.0, d)).sum())


def grad_error_scaled(g: np.ndarray, ref: np.ndarray, floor_scale: float):
    """grad_error with the elementwise floor taken from max(max|ref|, floor_scale)."""
    g = np.asarray(g, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    scale = float(np.abs(ref).max()) if ref.size else 0.0
    if scale == 0.0:
        return float(np.abs(g).max()) if g.size else 0.0, 0.0
    rel = float(np.abs(g - ref).max()) / scale
    worst = float((np.abs(g - ref) / _elem_bound(ref, max(scale, floor_scale))).max())
    return rel, worst


def assert_grads_close(got: dict, ref, names=GRAD_NAMES, rtol=1e-3, scene=None):
    for n in names:
        g = got[n]
        r = getattr(ref, n)
        if n == "cam" and scene is not None:
            rel, worst = grad_error_scaled(g, r, camera_term_scale(scene, ref))
        else:
            rel, worst = grad_error(g, r)
        if not (rel <= rtol and worst <= 1.0):
            gg, rr = np.asarray(g, np.float64).ravel(), np.asarray(r, np.float64).ravel()
            scale = np.abs(rr).max()
            ratio = np.abs(gg - rr) / _elem_bound(rr, scale)
            idx = np.argsort(ratio)[::-1][:5]
            detail = [(int(i), float(gg[i]), float(rr[i]), float(ratio[i])) for i in idx]
            raise AssertionError(f"{n}: max-norm rel {rel:.3e}, worst elementwise ratio {worst:.2f}; "
                                 f"scale {scale:.3e}; worst (index, got, want, ratio): {detail}")
