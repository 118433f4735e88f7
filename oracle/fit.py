"""Oracle of the scene fit (Sec. 3.4, "End-to-end Optimization"; the fit of
Sec. 5): image loss, Adam, and the loop that combines them with the
brute-force renderer.

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the CPU-baseline leg of
the benchmark call this module; the CUDA product path never does.

Everything is float64 NumPy, written from the definitions:
  - the loss over V views, L = scale * sum_v sum_pixels l(F_v - T_v), with
    l(d) = d^2 (dL/dF = 2 scale d) or l(d) = |d| (dL/dF = scale sign(d), 0 at d = 0);
  - Adam as stated by Kingma & Ba (2015), Algorithm 1, followed by clamping
    every parameter into its box [lo, hi];
  - one fit step: render every view (``oracle.render``), take the loss and
    dL/dF, run each view's backward pass (``oracle.render_backward``), sum the
    views' gradients, take the Adam step.  Parameters are stored as float32
    between steps, as the renderer's inputs are float32.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np

from . import oracle

PARAM_NAMES = ("pos", "rad", "opa", "feat")


def image_loss(kind: str, image, target, scale: float = 1.0):
    """(loss, dL/dF) in float64; kind 'l2' or 'l1'."""
    d = np.asarray(image, np.float64) - np.asarray(target, np.float64)
    if kind == "l2":
        return scale * float(np.sum(d * d)), 2.0 * scale * d
    if kind == "l1":
        return scale * float(np.sum(np.abs(d))), scale * np.sign(d)
    raise ValueError(kind)


def adam_step(theta, g, m, v, t: int, lr: float, beta1: float, beta2: float, eps: float,
              lo: float = -np.inf, hi: float = np.inf):
    """Step t (1-based) of Adam; returns (theta, m, v), all float64."""
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    theta = np.asarray(theta, np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps)
    return np.clip(theta, lo, hi), m, v


def view_scene(base, params: dict, cam):
    """A scene-like object: the base scene's settings with the given sphere
    parameters and camera."""
    return SimpleNamespace(pos=params["pos"], rad=params["rad"], opa=params["opa"], feat=params["feat"],
                           cam=np.asarray(cam, np.float32), bg=base.bg, width=base.width, height=base.height,
                           gamma=base.gamma, n_track=base.n_track, eps=base.eps, znear=base.znear,
                           zfar=base.zfar, ortho=getattr(base, "ortho", False),
                           paper_stop=getattr(base, "paper_stop", False),
                           min_contrib=getattr(base, "min_contrib", 0.01))


def loss_and_grads(base, params: dict, cams, targets, kind: str = "l2", scale: float = 1.0):
    """The fit's loss over all views and its gradient for every sphere parameter."""
    total = 0.0
    grads = {k: np.zeros(np.shape(params[k]), np.float64) for k in PARAM_NAMES}
    for cam, target in zip(cams, targets):
        sc = view_scene(base, params, cam)
        fwd = oracle.render(sc)
        loss, G = image_loss(kind, fwd.image, target, scale)
        total += loss
        g = oracle.render_backward(sc, G)
        for k in PARAM_NAMES:
            grads[k] += getattr(g, k)
    return total, grads


def fit(base, params: dict, cams, targets, steps: int, lr: float = 1e-3, beta1: float = 0.9,
        beta2: float = 0.999, eps: float = 1e-8, kind: str = "l2", scale: float = 1.0,
        bounds: dict | None = None, history: list | None = None):
    """``steps`` Adam steps from ``params`` (float32 arrays).  Returns (losses
    before each step, final params as float32, final loss).  Each step's
    gradients are appended to ``history`` when it is a list."""
    bounds = bounds or {}
    p = {k: np.asarray(params[k], np.float32).copy() for k in PARAM_NAMES}
    m = {k: np.zeros(p[k].shape) for k in PARAM_NAMES}
    v = {k: np.zeros(p[k].shape) for k in PARAM_NAMES}
    losses = []
    for t in range(1, steps + 1):
        loss, grads = loss_and_grads(base, p, cams, targets, kind, scale)
        losses.append(loss)
        if history is not None:
            history.append(grads)
        for k in PARAM_NAMES:
            lo, hi = bounds.get(k, (-np.inf, np.inf))
            theta, m[k], v[k] = adam_step(p[k], grads[k], m[k], v[k], t, lr, beta1, beta2, eps, lo, hi)
            p[k] = theta.astype(np.float32)
    final, _ = loss_and_grads(base, p, cams, targets, kind, scale)
    return losses, p, final
