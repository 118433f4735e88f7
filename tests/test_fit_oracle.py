"""Pins of the scene-fit oracle (oracle/fit.py) against what fixes it from outside:

  - Adam against PyTorch's own ``torch.optim.Adam`` (float64, CPU) over several
    steps, and the first step's closed form theta - lr g / (|g| + eps);
  - the box projection against clipping of the unconstrained step;
  - the losses against hand-computed values and central differences;
  - the multi-view gradient of the fit (loss gradient through every view's
    backward pass, summed) against central differences of the total loss;
  - the camera of Listing 1: Rodrigues' rotation against scipy's rotation
    vectors, and the renderer's Gram-Schmidt giving the rotation back.
"""
import numpy as np
import pytest
import torch

from paper_2004_07484_gb300.scenes import config_scene, orbit_cameras, perturbed


@pytest.fixture(scope="module")
def fit_orc(orc):
    from oracle import fit
    return fit


def test_adam_matches_torch_adam_over_several_steps(fit_orc):
    rng = np.random.default_rng(3)
    theta0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) * 10.0 ** rng.uniform(-3, 1, 50) for _ in range(6)]
    lr, b1, b2, eps = 3e-3, 0.8, 0.95, 1e-6
    p = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=lr, betas=(b1, b2), eps=eps)
    theta, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, start=1):
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        theta, m, v = fit_orc.adam_step(theta, g, m, v, t, lr, b1, b2, eps)
        np.testing.assert_allclose(theta, p.detach().numpy(), rtol=0, atol=1e-14)


def test_adam_first_step_closed_form(fit_orc):
    g = np.array([2.0, -1e-3, 0.0, 5e-9, -7.0])
    theta0 = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    lr, eps = 1e-2, 1e-8
    theta, m, v = fit_orc.adam_step(theta0, g, np.zeros(5), np.zeros(5), 1, lr, 0.9, 0.999, eps)
    np.testing.assert_allclose(theta, theta0 - lr * g / (np.abs(g) + eps), rtol=1e-15, atol=1e-16)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_adam_box_projection_clips_the_free_step(fit_orc):
    rng = np.random.default_rng(5)
    theta0 = rng.uniform(0.0, 1.0, 200)
    g = rng.standard_normal(200)
    m0, v0 = rng.standard_normal(200) * 0.1, rng.uniform(0.0, 0.1, 200)
    free, _, _ = fit_orc.adam_step(theta0, g, m0, v0, 4, 0.2, 0.9, 0.999, 1e-8)
    boxed, m1, v1 = fit_orc.adam_step(theta0, g, m0, v0, 4, 0.2, 0.9, 0.999, 1e-8, 0.0, 1.0)
    assert ((free < 0) | (free > 1)).any()
    np.testing.assert_array_equal(boxed, np.minimum(np.maximum(free, 0.0), 1.0))
    assert boxed.min() >= 0.0 and boxed.max() <= 1.0


def test_losses_by_hand_and_by_differences(fit_orc):
    F = np.array([[0.5, -1.0], [2.0, 3.0]])
    T = np.array([[0.0, -1.0], [1.0, 5.0]])
    l2, g2 = fit_orc.image_loss("l2", F, T)
    assert l2 == pytest.approx(0.25 + 0.0 + 1.0 + 4.0)
    np.testing.assert_array_equal(g2, [[1.0, 0.0], [2.0, -4.0]])
    l1, g1 = fit_orc.image_loss("l1", F, T, scale=0.5)
    assert l1 == pytest.approx(0.5 * (0.5 + 0.0 + 1.0 + 2.0))
    np.testing.assert_array_equal(g1, [[0.5, 0.0], [0.5, -0.5]])
    rng = np.random.default_rng(9)
    F, T = rng.standard_normal((6, 5, 3)), rng.standard_normal((6, 5, 3))
    for kind in ("l2", "l1"):
        _, g = fit_orc.image_loss(kind, F, T, scale=0.3)
        for idx in [(0, 0, 0), (3, 2, 1), (5, 4, 2)]:
            h = 1e-6
            Fp, Fm = F.copy(), F.copy()
            Fp[idx] += h
            Fm[idx] -= h
            fd = (fit_orc.image_loss(kind, Fp, T, 0.3)[0] - fit_orc.image_loss(kind, Fm, T, 0.3)[0]) / (2 * h)
            assert g[idx] == pytest.approx(fd, rel=1e-6)


def _small_fit_problem(n=60, res=24, views=2):
    hidden = config_scene(4, n=n, res=res)
    hidden.n_track = 32                        # every hit tracked: exact gradients
    centre = hidden.pos.astype(np.float64).mean(axis=0)
    cams = orbit_cameras(11, centre, n_views=views, distance=6.0)
    start = perturbed(hidden, 12)
    return hidden, start, cams


def test_fit_gradient_matches_differences_of_the_total_loss(orc, fit_orc):
    hidden, start, cams = _small_fit_problem()
    targets = [orc.render(fit_orc.view_scene(hidden, {k: getattr(hidden, k) for k in fit_orc.PARAM_NAMES},
                                             c)).image for c in cams]
    params = {k: getattr(start, k).astype(np.float64) for k in fit_orc.PARAM_NAMES}
    loss, grads = fit_orc.loss_and_grads(start, params, cams, targets)
    assert loss > 0.0

    def total(override):
        s = 0.0
        for cam, target in zip(cams, targets):
            sc = fit_orc.view_scene(start, {k: getattr(start, k) for k in fit_orc.PARAM_NAMES}, cam)
            out = orc.render(sc, freeze_decisions=True, cam=np.asarray(cam, np.float64), bg=start.bg,
                             **override)
            s += fit_orc.image_loss("l2", out.image, target)[0]
        return s

    base = {k: getattr(start, k).astype(np.float64) for k in fit_orc.PARAM_NAMES}
    scale = {k: float(np.abs(grads[k]).max()) for k in fit_orc.PARAM_NAMES}
    rng = np.random.default_rng(2)
    checked = 0
    for name in fit_orc.PARAM_NAMES:
        g = grads[name].reshape(-1)
        live = np.flatnonzero(np.abs(g) > 1e-2 * scale[name])
        for idx in rng.choice(live, size=min(6, len(live)), replace=False):
            x0 = base[name].reshape(-1)[idx]
            vals = []
            for h in (1e-5 * max(1.0, abs(x0)), 0.5e-5 * max(1.0, abs(x0))):
                d = []
                for s in (+1, -1):
                    arr = {k: v.copy() for k, v in base.items()}
                    arr[name].reshape(-1)[idx] += s * h
                    d.append(total(arr))
                vals.append((d[0] - d[1]) / (2 * h))
            if abs(vals[0] - vals[1]) > 1e-4 * max(abs(vals[1]), 1e-3 * scale[name]):
                continue                       # the stencil crosses a rim: resample elsewhere
            assert g[idx] == pytest.approx(vals[1], rel=1e-4, abs=1e-6 * scale[name]), (name, idx)
            checked += 1
    assert checked >= 16


def test_fit_loop_lowers_the_loss(orc, fit_orc):
    hidden, start, cams = _small_fit_problem(n=40, res=16)
    targets = [orc.render(fit_orc.view_scene(hidden, {k: getattr(hidden, k) for k in fit_orc.PARAM_NAMES},
                                             c)).image for c in cams]
    params = {k: getattr(start, k) for k in fit_orc.PARAM_NAMES}
    losses, p, final = fit_orc.fit(start, params, cams, targets, steps=4, lr=1e-3,
                                   bounds={"rad": (1e-4, np.inf), "opa": (0.0, 1.0)})
    assert len(losses) == 4 and final < losses[0]
    assert p["opa"].min() >= 0.0 and p["opa"].max() <= 1.0 and p["rad"].min() >= 1e-4
    assert all(p[k].dtype == np.float32 for k in p)


# ---------------------------------------------------------------- camera of Listing 1

def test_axis_angle_rotation_matches_scipy_and_gram_schmidt(orc):
    from scipy.spatial.transform import Rotation
    from oracle import scene_utils
    rng = np.random.default_rng(4)
    for w in [np.zeros(3), np.array([1e-9, 0.0, 0.0]), *rng.normal(size=(6, 3)) * 1.5]:
        B = scene_utils.rotation(w)
        np.testing.assert_allclose(B, Rotation.from_rotvec(w).as_matrix(), atol=1e-14)
        cam = scene_utils.cam11_from_cam8(np.concatenate([[0.1, 0.2, 0.3], w, [1.5, 2.0]]))
        # the renderer's Gram-Schmidt of the two rows gives back B
        np.testing.assert_allclose(orc.rows(cam[3:9]).reshape(3, 3), B, atol=1e-14)
        assert cam[9] == 1.5 and cam[10] == 2.0 and np.array_equal(cam[:3], [0.1, 0.2, 0.3])


# ---------------------------------------------------------------- pruning and subdivision

def test_fcc_directions_are_a_cuboctahedron():
    """The 12 nearest neighbours of a face-centred cubic site: unit vectors
    summing to zero, whose nearest pairwise distance equals the radius (the
    cuboctahedron's edge equals its circumradius), each with 4 such neighbours."""
    from oracle import scene_utils
    u = scene_utils.FCC_DIRECTIONS
    assert u.shape == (12, 3) and len({tuple(np.round(x, 12)) for x in u}) == 12
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose(u.sum(axis=0), 0.0, atol=1e-14)
    d = np.linalg.norm(u[:, None] - u[None], axis=2) + np.eye(12) * 9
    np.testing.assert_allclose(d.min(axis=1), 1.0, atol=1e-14)
    assert np.all((np.abs(d - 1.0) < 1e-12).sum(axis=1) == 4)


def test_subdivision_and_pruning_properties():
    from oracle import scene_utils
    rng = np.random.default_rng(7)
    pos, rad = rng.normal(size=(5, 3)), rng.uniform(0.1, 1.0, 5)
    opa, feat = rng.uniform(0, 1, 5), rng.uniform(0, 1, (5, 3))
    cp, cr, co, cf = scene_utils.subdivide(pos, rad, opa, feat, 0.7, 0.3)
    assert cp.shape == (60, 3)
    np.testing.assert_allclose(cp.reshape(5, 12, 3).mean(axis=1), pos, atol=1e-14)   # centred on the parent
    np.testing.assert_allclose(np.linalg.norm(cp.reshape(5, 12, 3) - pos[:, None], axis=2),
                               0.7 * rad[:, None].repeat(12, 1), rtol=1e-14)
    assert np.all(cr == np.repeat(0.3 * rad, 12)) and np.all(co == np.repeat(opa, 12))
    # pruning: no criterion keeps everything; a larger tolerance keeps a subset; the
    # float32 decision agrees with float64 away from the threshold
    f = rng.uniform(0, 1, (500, 4)).astype(np.float32)
    bg = np.float32([0.5, 0.5, 0.5, 0.5])
    assert scene_utils.prune_keep(f, bg).all()
    k1, k2 = scene_utils.prune_keep(f, bg, color_tol=0.4), scene_utils.prune_keep(f, bg, color_tol=0.6)
    assert np.all(k2 <= k1) and k1.sum() > k2.sum() > 0
    dist = np.linalg.norm(f.astype(np.float64) - bg, axis=1)
    far = np.abs(dist - 0.4) > 1e-5
    assert np.array_equal(k1[far], dist[far] > 0.4)
    act = rng.uniform(-1, 1, 500).astype(np.float32)
    assert np.array_equal(scene_utils.prune_keep(f, bg, act), act > 0)
