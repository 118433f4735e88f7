"""Pins of the brute-force oracle against what the paper and geometry fix.

Each test checks the oracle against something other than itself:
  - closed forms of Eq. 1 for spheres on the optical axis and for off-axis rays
    (derived here by trigonometry, not by the oracle's quadratic),
  - the blend weights plus the background weight summing to one (Eq. 1),
  - invariance to the order of the spheres (App. A: commutativity),
  - the hard z-buffer limit as gamma -> 0 (Sec. 3.2),
  - the one-pixel minimum size (App. B, Step 0),
  - a conservative enclosing rectangle (App. B, Step 0), checked by brute force,
  - the n_track closest hits (App. B, Step 2),
  - rigid-motion invariance of the camera model and a hand-placed 90-degree view,
  - central finite differences for every gradient (Sec. 1: differentiable
    without approximation) and the focal/sensor-width relation of the pinhole.
"""
import math

import numpy as np
import pytest

from paper_2004_07484_gb300.scenes import Scene, config_scene, make_cam, grad_image, random_rotation


def scene_of(pos, rad, opa, feat, W, H, gamma, cam=None, bg=None, n_track=8, eps=1e-5,
             znear=1.0, zfar=20.0):
    feat = np.atleast_2d(np.asarray(feat, np.float32))
    C = feat.shape[1]
    return Scene(np.asarray(pos, np.float32).reshape(-1, 3), np.asarray(rad, np.float32).ravel(),
                 np.asarray(opa, np.float32).ravel(), feat,
                 make_cam() if cam is None else np.asarray(cam, np.float32),
                 np.zeros(C, np.float32) if bg is None else np.asarray(bg, np.float32),
                 W, H, gamma, n_track, eps=eps, znear=znear, zfar=zfar)


def f32(x):
    return float(np.float32(x))


# ---------------------------------------------------------------- Eq. 1 closed forms

def _trig_single_sphere(Z, R, o, f, bg, gamma, eps, znear, zfar, rho_x, rho_y, literal):
    """Eq. 1 for one sphere centred on the optical axis at depth Z, seen along
    the ray with slopes (rho_x, rho_y): the ray makes the angle theta with the
    axis, passes the centre at distance Z sin(theta), and enters the sphere at
    the distance Z cos(theta) - sqrt(R^2 - (Z sin theta)^2) along the ray."""
    theta = math.atan(math.hypot(rho_x, rho_y))
    dist = Z * math.sin(theta)
    B = math.exp(eps / gamma)
    if dist >= R:
        return np.asarray(bg, float), False
    ell = Z * math.cos(theta) - math.sqrt(R * R - dist * dist)
    depth = ell * math.cos(theta)
    z = (zfar - depth) / (zfar - znear)
    d = dist / R if literal else 1.0 - dist / R
    a = o * d * math.exp(o * z / gamma)
    return (a * np.asarray(f, float) + B * np.asarray(bg, float)) / (B + a), True


@pytest.mark.parametrize("gamma", [1.0, 0.1, 0.01])
@pytest.mark.parametrize("literal", [False, True])
def test_single_sphere_closed_form(orc, gamma, literal):
    W = H = 33
    Z, r, o = 6.0, 2.0, 0.8
    f = [0.3, 0.7, 0.2]
    bg = [0.1, 0.2, 0.9]
    sc = scene_of([0, 0, Z], [r], [o], [f], W, H, gamma, bg=bg)
    out = orc.render(sc, dist_literal=literal)
    kappa = 2.0 / (W * 1.0)
    checked = 0
    for v in range(H):
        for u in range(W):
            rx = (u + 0.5 - W / 2) * kappa
            ry = (v + 0.5 - H / 2) * kappa
            dist = Z * math.sin(math.atan(math.hypot(rx, ry)))
            if abs(dist - f32(r)) < 1e-4:
                continue  # rounding band of the float32 hit decision
            want, hit = _trig_single_sphere(Z, f32(r), f32(o), [f32(x) for x in f],
                                            [f32(x) for x in bg], f32(gamma), f32(1e-5), 1.0, 20.0,
                                            rx, ry, literal)
            assert out.n_hits[v, u] == int(hit)
            np.testing.assert_allclose(out.image[v, u], want, rtol=1e-11, atol=1e-13)
            checked += hit
    assert checked > 50


def test_two_spheres_on_axis(orc):
    W = H = 65  # small pixels: the minimum-size rule leaves both radii alone
    g, eps = 0.1, 1e-5
    Z = [5.0, 7.0]
    r = [0.3, 0.6]
    o = [0.6, 0.9]
    f = [[1.0, 0.0], [0.0, 1.0]]
    bg = [0.25, 0.5]
    sc = scene_of([[0, 0, Z[1]], [0, 0, Z[0]]], [r[1], r[0]], [o[1], o[0]], [f[1], f[0]], W, H, g,
                  bg=bg, n_track=2)
    out = orc.render(sc)
    c = W // 2
    a = [f32(o[k]) * math.exp(f32(o[k]) * (20.0 - (Z[k] - f32(r[k]))) / 19.0 / f32(g)) for k in range(2)]
    B = math.exp(f32(eps) / f32(g))
    bg64 = np.array(bg, np.float32).astype(np.float64)
    want = (a[0] * np.array(f[0]) + a[1] * np.array(f[1]) + B * bg64) / (B + a[0] + a[1])
    np.testing.assert_allclose(out.image[c, c], want, rtol=1e-12)
    # the closer sphere (index 1) is tracked first
    assert list(out.tracked[c, c]) == [1, 0]
    np.testing.assert_allclose(out.log_d[c, c], math.log(B + a[0] + a[1]), rtol=1e-12)


# ---------------------------------------------------------------- invariants of Eq. 1

@pytest.mark.parametrize("gamma", [1.0, 0.1, 1e-3])
def test_weights_sum_to_one(orc, gamma):
    sc = config_scene(0, gamma=gamma)
    sc.feat = np.ones_like(sc.feat)
    out = orc.render(sc)
    wB = np.exp(f32(sc.eps) / f32(gamma) - out.log_d)
    np.testing.assert_allclose(out.wsum + wB, 1.0, atol=1e-12)
    np.testing.assert_allclose(out.image[..., 0], out.wsum, atol=1e-12)
    sc.bg = np.ones(3, np.float32)
    out = orc.render(sc)
    np.testing.assert_allclose(out.image, 1.0, atol=1e-12)


def test_sphere_order_invariance(orc):
    sc = config_scene(0)
    out = orc.render(sc, n_track=5)
    perm = np.random.default_rng(3).permutation(sc.n_spheres)
    sp = scene_of(sc.pos[perm], sc.rad[perm], sc.opa[perm], sc.feat[perm], sc.width, sc.height,
                  sc.gamma, n_track=5)
    outp = orc.render(sp, n_track=5)
    np.testing.assert_allclose(outp.image, out.image, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(outp.n_hits, out.n_hits)
    mapped = np.where(outp.tracked >= 0, perm[np.maximum(outp.tracked, 0)], -1)
    np.testing.assert_array_equal(mapped, out.tracked)


def test_equal_depth_ties_break_by_index(orc):
    W = H = 9
    sc = scene_of([[0, 0, 6], [0, 0, 6], [0, 0, 6]], [0.5, 0.5, 0.5], [0.5, 0.7, 0.9],
                  [[1.0], [2.0], [3.0]], W, H, 0.1, n_track=3)
    out = orc.render(sc)
    assert list(out.tracked[4, 4]) == [0, 1, 2]
    assert out.tracked_t[4, 4, 0] == out.tracked_t[4, 4, 1] == out.tracked_t[4, 4, 2]


# ---------------------------------------------------------------- gamma -> 0 limits (Sec. 3.2)

def _limit_errors(orc, opa, feat, bg, target):
    W = H = 9
    errs = []
    for g in [1e-1, 1e-2, 1e-3, 1e-4, 1e-5]:
        sc = scene_of([[0, 0, 5.0], [0, 0, 7.0], [0, 0, 9.0]], [0.8, 0.8, 0.8], opa, feat, W, H, g,
                      bg=bg)
        out = orc.render(sc)
        errs.append(float(np.abs(out.image[4, 4] - target).max()))
    return errs


def test_gamma_to_zero_is_hard_zbuffer(orc):
    feat = [[1.0, 0.0], [0.0, 1.0], [0.5, 0.5]]
    errs = _limit_errors(orc, [1.0, 1.0, 1.0], feat, [0.0, 0.0], np.array(feat[0]))
    assert all(b <= a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] <= 1e-6


def test_gamma_to_zero_selects_largest_opacity_times_depth(orc):
    # o*z: front 0.3*0.2158 = 0.0647 < middle 1.0*0.1105 = 0.1105 > back 0.5*0.0053
    feat = [[1.0, 0.0], [0.0, 1.0], [0.5, 0.5]]
    errs = _limit_errors(orc, [0.3, 1.0, 0.5], feat, [0.0, 0.0], np.array(feat[1]))
    assert all(b <= a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] <= 1e-6


def test_gamma_to_zero_background_wins_below_eps(orc):
    feat = [[1.0, 0.0], [0.0, 1.0], [0.5, 0.5]]
    bg = [0.25, 0.75]
    errs = _limit_errors(orc, [1e-6, 1e-6, 1e-6], feat, bg, np.array(bg, np.float32))
    assert all(b <= a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] <= 1e-6


# ---------------------------------------------------------------- Step 0: size, rectangle, culling

def test_every_sphere_covers_a_pixel(orc):
    g = np.random.default_rng(11)
    W, H = 48, 40
    base = scene_of([0, 0, 6], [0.1], [1.0], [[1.0]], W, H, 0.1)
    for k in range(300):
        z = g.uniform(2.0, 19.0)
        kappa = 2.0 / W
        # projected centre anywhere in the image
        x = g.uniform(-W / 2, W / 2) * kappa * z
        y = g.uniform(-H / 2, H / 2) * kappa * z
        m = orc.hit_map(base, [x, y, z], 1e-4)
        assert m.any(), (x, y, z)
    # without the rule such a tiny sphere is almost never seen
    misses = sum(not orc.hit_map(base, [0.0123, -0.0071, 6.0], 1e-4, min_size=False).any() for _ in range(1))
    assert misses == 1


def test_rectangle_is_conservative_and_culling_is_safe(orc):
    g = np.random.default_rng(5)
    W, H = 40, 24
    rows = random_rotation(g).T
    cam = make_cam(t=(0.3, -0.2, 0.1), rot6=np.concatenate([rows[0], rows[1]]), focal=1.3,
                   sensor_width=2.2)
    base = scene_of([0, 0, 6], [0.1], [1.0], [[1.0]], W, H, 0.1, cam=cam)
    n_vis = n_cull = 0
    for k in range(1200):
        # points in a wide frustum around the camera, some outside the image
        zc = g.uniform(0.5, 22.0)
        xc, yc = g.uniform(-1.6, 1.6, 2) * zc
        r = float(np.exp(g.uniform(np.log(0.01), np.log(3.0))))
        p = rows.T @ np.array([xc, yc, zc]) + np.array([0.3, -0.2, 0.1])
        sc1 = scene_of(p, [r], [1.0], [[1.0]], W, H, 0.1, cam=cam)
        pr = orc.project(sc1)
        m = orc.hit_map(base, p, r)
        if pr.rect[0, 0] >= 0:
            n_vis += 1
            x0, x1, y0, y1 = pr.rect[0]
            vv, uu = np.nonzero(m)
            assert np.all((uu >= x0) & (uu <= x1) & (vv >= y0) & (vv <= y1)), (p, r)
        else:
            assert not m.any()
            key_ok = 1.0 < pr.c[0, 2] - pr.R[0] < 20.0
            if key_ok:
                n_cull += 1
                assert not orc.hit_map(base, p, r, ignore_cull=True).any(), (p, r)
    assert n_vis > 200 and n_cull > 50


# ---------------------------------------------------------------- tracking and tile lists

def test_tracked_are_the_closest_hits(orc):
    sc = config_scene(0)
    full = orc.render(sc, n_track=64)
    assert full.n_hits.max() <= 64
    part = orc.render(sc, n_track=5)
    np.testing.assert_array_equal(part.tracked, full.tracked[..., :5])
    t = full.tracked_t
    ids = full.tracked
    valid = ids >= 0
    assert np.array_equal(valid.sum(-1), full.n_hits)
    ordered = (t[..., 1:] > t[..., :-1]) | ((t[..., 1:] == t[..., :-1]) & (ids[..., 1:] > ids[..., :-1]))
    assert np.all(ordered | ~valid[..., 1:])
    # every listed hit is a hit of the float32 predicate at that pixel
    vv, uu = np.nonzero(full.n_hits)
    for v, u in list(zip(vv, uu))[:40]:
        for i in ids[v, u][ids[v, u] >= 0]:
            hit, tt = orc.hit_f32(sc, sc.pos[i], sc.rad[i], u, v)
            assert hit
            assert np.float32(tt) in t[v, u]


def test_tile_lists_cover_every_hit_in_key_order(orc):
    sc = config_scene(0)
    T = 16
    offsets, ids = orc.tile_lists(sc, tile=T)
    pr = orc.project(sc, tile=T)
    full = orc.render(sc, n_track=64)
    ntx = (sc.width + T - 1) // T
    for tile in range(len(offsets) - 1):
        lst = ids[offsets[tile]:offsets[tile + 1]]
        k = pr.key[lst]
        assert np.all((k[1:] > k[:-1]) | ((k[1:] == k[:-1]) & (lst[1:] > lst[:-1])))
        assert np.all(pr.rect[lst, 0] >= 0)
    for v in range(sc.height):
        for u in range(sc.width):
            tile = (v // T) * ntx + u // T
            lst = set(ids[offsets[tile]:offsets[tile + 1]].tolist())
            hits = full.tracked[v, u][full.tracked[v, u] >= 0]
            assert set(hits.tolist()) <= lst


# ---------------------------------------------------------------- camera model

def test_rotation_rows_are_orthonormal(orc):
    g = np.random.default_rng(2)
    for _ in range(20):
        a = g.standard_normal(6)
        B = orc.rows(a)
        np.testing.assert_allclose(B @ B.T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(B) - 1.0) < 1e-12
        np.testing.assert_allclose(B[0], a[:3] / np.linalg.norm(a[:3]), atol=1e-12)


def test_camera_turned_to_world_x(orc):
    # camera x axis = world -z, y axis = world y, so it looks along world +x
    cam = make_cam(rot6=(0.0, 0.0, -1.0, 0.0, 1.0, 0.0))
    W = H = 21
    a = orc.render(scene_of([5.0, 0.3, 0.2], [1.2], [0.9], [[0.2, 0.8]], W, H, 0.1, cam=cam))
    b = orc.render(scene_of([-0.2, 0.3, 5.0], [1.2], [0.9], [[0.2, 0.8]], W, H, 0.1))
    np.testing.assert_allclose(a.image, b.image, atol=1e-12)
    assert a.n_hits.sum() > 10


def test_rigid_motion_invariance(orc):
    sc = config_scene(0)
    g = np.random.default_rng(9)
    Q = random_rotation(g)
    shift = np.array([0.4, -1.1, 2.3])
    pos2 = (sc.pos.astype(np.float64) @ Q.T) + shift
    rows2 = np.eye(3) @ Q.T            # camera axes rotate with the world
    cam2 = np.concatenate([shift, rows2[0], rows2[1], [1.0, 2.0]])
    a = orc.render(sc, freeze_decisions=True, n_track=5)
    b = orc.render(sc, freeze_decisions=True, n_track=5, pos=pos2, cam=cam2)
    np.testing.assert_allclose(a.image, b.image, atol=1e-10)


# ---------------------------------------------------------------- gradients vs central differences

def _fd(orc, sc, G, name, index, h, **kw):
    base = {k: getattr(sc, k).astype(np.float64).copy() for k in ["pos", "rad", "opa", "feat", "cam", "bg"]}
    vals = []
    for s in (+1, -1):
        arr = {k: v.copy() for k, v in base.items()}
        arr[name].reshape(-1)[index] += s * h
        out = orc.render(sc, freeze_decisions=True, n_track=1, **arr, **kw)
        vals.append(float(np.sum(out.image * G)))
    return (vals[0] - vals[1]) / (2 * h)


def _richardson(orc, sc, G, name, idx, h, **kw):
    """Central difference with one Richardson step: error O(h^4)."""
    a = _fd(orc, sc, G, name, idx, h, **kw)
    b = _fd(orc, sc, G, name, idx, h / 2, **kw)
    return (4.0 * b - a) / 3.0, b


def _check_fd(orc, sc, G, grads, name, indices, n_track, rtol=1e-6, hscales=(1.0,), **kw):
    """Analytic gradient entries against Richardson-extrapolated central
    differences.  A stencil that crosses a kink (a sphere rim) shows up as two
    step sizes disagreeing; the next step scale in ``hscales`` is tried, and an
    entry without any consistent pair is skipped (at most 20 % may be)."""
    g = getattr(grads, name).reshape(-1)
    scale = max(float(np.abs(g).max()), 1e-12)
    checked = 0
    for idx in indices:
        x0 = float(getattr(sc, name).reshape(-1)[idx])
        for hs in hscales:
            h = hs * 2e-5 * max(1.0, abs(x0))
            r1, _ = _richardson(orc, sc, G, name, idx, h, **kw)
            r2, _ = _richardson(orc, sc, G, name, idx, h / 2, **kw)
            tol = rtol * max(abs(r2), 1e-3 * scale)
            if abs(r1 - r2) > tol:
                continue  # the stencil crosses a kink (rim of a sphere) or round-off dominates
            assert abs(g[idx] - r2) <= tol + 1e-9, (name, idx, g[idx], r2)
            checked += 1
            break
    assert checked >= max(1, int(0.8 * len(indices))), (name, checked, len(indices))


@pytest.mark.parametrize("min_size,literal", [(True, False), (False, False), (True, True)])
def test_gradients_match_central_differences(orc, min_size, literal):
    sc = config_scene(0)
    W = sc.width
    G = np.zeros((sc.height, W, 3))
    G[24:40, 24:40] = grad_image(77, 16, 16, 3)
    K = 64  # at least the largest hit count: every hit is tracked
    grads = orc.render_backward(sc, G, n_track=K, min_size=min_size, dist_literal=literal)
    full = orc.render(sc, n_track=K, min_size=min_size, dist_literal=literal)
    assert full.n_hits.max() <= K
    seen = np.unique(full.tracked[24:40, 24:40][full.tracked[24:40, 24:40] >= 0])
    rng = np.random.default_rng(1)
    sph = rng.choice(seen, size=min(12, len(seen)), replace=False)
    kw = dict(min_size=min_size, dist_literal=literal)
    _check_fd(orc, sc, G, grads, "pos", [3 * i + k for i in sph for k in range(3)], K, **kw)
    _check_fd(orc, sc, G, grads, "rad", list(sph), K, **kw)
    _check_fd(orc, sc, G, grads, "opa", list(sph), K, **kw)
    _check_fd(orc, sc, G, grads, "feat", [3 * i + k for i in sph[:4] for k in range(3)], K, **kw)
    _check_fd(orc, sc, G, grads, "cam", list(range(11)), K, **kw)
    _check_fd(orc, sc, G, grads, "bg", [0, 1, 2], K, **kw)


def test_gradients_with_rotated_camera(orc):
    sc = config_scene(0)
    g = np.random.default_rng(4)
    rows = random_rotation(g).T
    # keep the cloud in view: look at its centre from 7.5 units away
    centre = np.array([0.0, 0.0, 7.5])
    t = centre - 7.5 * rows[2]
    sc.cam = make_cam(t=t, rot6=np.concatenate([rows[0], rows[1]]), focal=1.1, sensor_width=2.0)
    out = orc.render(sc, n_track=64)
    assert out.n_hits.sum() > 100
    G = grad_image(5, sc.height, sc.width, 3)
    grads = orc.render_backward(sc, G, n_track=64)
    _check_fd(orc, sc, G, grads, "cam", list(range(11)), 64)
    seen = np.unique(out.tracked[out.tracked >= 0])
    sph = np.random.default_rng(0).choice(seen, 6, replace=False)
    _check_fd(orc, sc, G, grads, "pos", [3 * i + k for i in sph for k in range(3)], 64)


def test_focal_and_sensor_width_enter_as_a_ratio(orc):
    sc = config_scene(0)
    G = grad_image(6, sc.height, sc.width, 3)
    gr = orc.render_backward(sc, G, n_track=64)
    f, s = float(sc.cam[9]), float(sc.cam[10])
    assert abs(gr.cam[9] * f + gr.cam[10] * s) <= 1e-12 * max(abs(gr.cam[9] * f), 1e-30)
    assert abs(gr.cam[10]) > 0


def test_untracked_hits_get_no_gradient(orc):
    sc = config_scene(0)
    G = grad_image(8, sc.height, sc.width, 3)
    out = orc.render(sc, n_track=2)
    gr = orc.render_backward(sc, G, n_track=2)
    tracked = np.unique(out.tracked[out.tracked >= 0])
    untracked = np.setdiff1d(np.arange(sc.n_spheres), tracked)
    assert np.all(gr.opa[untracked] == 0) and np.all(gr.feat[untracked] == 0)
    assert np.any(gr.opa[tracked] != 0)


# ---------------------------------------------------------------- paper gradient normalisations

def test_paper_gradients_are_the_exact_ones_averaged_and_gated(orc):
    """The paper mode (App. B, end of "The Backward Pass"; Sec. 6) against the
    exact gradients, which the finite-difference pins fix: sphere gradients
    divided by the number of pixels at which the sphere is tracked (counted
    here from the forward pass's tracked lists), positions and radii only for
    spheres of more than 3 pixels projected radius, camera times 1e-3."""
    from paper_2004_07484_gb300.scenes import uniform_cloud
    sc = uniform_cloud(71, 60, 64, 48, n_channels=3, gamma=0.05, n_track=6, rad=(0.05, 1.2))
    rng = np.random.default_rng(3)
    G = rng.standard_normal((sc.height, sc.width, 3))
    G[::5, ::3] = 0.0                       # pixels without upstream gradient still count
    K = 6
    exact = orc.render_backward(sc, G, n_track=K)
    paper = orc.render_backward(sc, G, n_track=K, paper_grad=True)
    fwd = orc.render(sc, n_track=K)
    tr = fwd.tracked.reshape(-1)
    n_px = np.bincount(tr[tr >= 0], minlength=sc.n_spheres).astype(np.float64)
    n = np.maximum(n_px, 1.0)
    pr = orc.project(sc)
    kf = np.float32(sc.cam[10]) / (np.float32(sc.width) * np.float32(sc.cam[9]))
    rpx = pr.R.astype(np.float32) / (pr.c[:, 2].astype(np.float32) * kf)
    gate = rpx > np.float32(3.0)
    seen = n_px > 0
    assert (gate & seen).sum() >= 3 and (~gate & seen).sum() >= 3 and n_px.max() > 1
    np.testing.assert_allclose(paper.opa * n, exact.opa, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(paper.feat * n[:, None], exact.feat, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(paper.pos * n[:, None], np.where(gate[:, None], exact.pos, 0.0), rtol=1e-12,
                               atol=1e-15)
    clamped = pr.R != sc.rad
    want_rad = np.where(gate & ~clamped, exact.rad, 0.0)
    np.testing.assert_allclose(paper.rad * n, want_rad, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(paper.cam, 1e-3 * exact.cam, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(paper.bg, exact.bg, rtol=1e-12)


# ---------------------------------------------------------------- orthographic camera

def _ortho(sc):
    sc.ortho = True
    return sc


def test_orthographic_single_sphere_closed_form(orc):
    """A sphere seen along parallel rays: at ray offset delta from the centre
    the front hit lies at Z - sqrt(R^2 - delta^2) and d = 1 - delta / R
    (Sec. 3.2); the pixel pitch is the sensor width over the image width and
    the focal length does not enter."""
    W, H, s_w = 40, 30, 3.0
    x0, y0, Z, R, o, f, bg, gamma, eps = 0.31, -0.22, 6.0, 0.9, 0.8, 0.6, 0.1, 0.05, 1e-5
    k = float(np.float32(s_w)) / W   # the value path's pitch (the camera entries are float32)
    out = {}
    for focal in (0.7, 2.3):
        sc = _ortho(scene_of([x0, y0, Z], [R], [o], [[f]], W, H, gamma, bg=[bg], eps=eps,
                             cam=make_cam(sensor_width=s_w, focal=focal)))
        out[focal] = orc.render(sc)
    np.testing.assert_array_equal(out[0.7].image, out[2.3].image)
    img, nh = out[0.7].image[..., 0], out[0.7].n_hits
    checked = 0
    for v in range(H):
        for u in range(W):
            rx, ry = (u + 0.5 - W / 2) * k, (v + 0.5 - H / 2) * k
            delta = math.hypot(rx - f32(x0), ry - f32(y0))
            if abs(delta - f32(R)) < 1e-4:
                continue   # the float32 decision decides the rim
            if delta >= f32(R):
                assert nh[v, u] == 0 and img[v, u] == pytest.approx(f32(bg), abs=1e-15)
                continue
            t = f32(Z) - math.sqrt(f32(R) ** 2 - delta ** 2)
            z = (20.0 - t) / 19.0
            a = f32(o) * (1.0 - delta / f32(R)) * math.exp(f32(o) * z / f32(gamma))
            B = math.exp(f32(eps) / f32(gamma))
            want = (a * f32(f) + B * f32(bg)) / (a + B)
            assert img[v, u] == pytest.approx(want, rel=1e-12, abs=1e-14), (u, v)
            checked += 1
    assert checked > 100


def test_orthographic_every_sphere_covers_a_pixel(orc):
    g = np.random.default_rng(12)
    W, H = 48, 40
    cam = make_cam(sensor_width=2.5)
    base = _ortho(scene_of([0, 0, 6], [0.1], [1.0], [[1.0]], W, H, 0.1, cam=cam))
    k = 2.5 / W
    for _ in range(300):
        x, y = g.uniform(-W / 2, W / 2) * k, g.uniform(-H / 2, H / 2) * k
        assert orc.hit_map(base, [x, y, g.uniform(2.0, 19.0)], 1e-4).any()


def test_orthographic_rectangle_is_conservative(orc):
    g = np.random.default_rng(6)
    W, H = 40, 24
    rows = random_rotation(g).T
    cam = make_cam(t=(0.3, -0.2, 0.1), rot6=np.concatenate([rows[0], rows[1]]), sensor_width=3.0)
    base = _ortho(scene_of([0, 0, 6], [0.1], [1.0], [[1.0]], W, H, 0.1, cam=cam))
    n_vis = 0
    for _ in range(800):
        zc = g.uniform(0.5, 22.0)
        xc, yc = g.uniform(-2.0, 2.0, 2)
        r = float(np.exp(g.uniform(np.log(0.01), np.log(2.0))))
        p = rows.T @ np.array([xc, yc, zc]) + np.array([0.3, -0.2, 0.1])
        sc1 = _ortho(scene_of(p, [r], [1.0], [[1.0]], W, H, 0.1, cam=cam))
        pr = orc.project(sc1)
        m = orc.hit_map(base, p, r)
        if pr.rect[0, 0] >= 0:
            n_vis += 1
            x0, x1, y0, y1 = pr.rect[0]
            vv, uu = np.nonzero(m)
            assert np.all((uu >= x0) & (uu <= x1) & (vv >= y0) & (vv <= y1)), (p, r)
        else:
            assert not m.any()
    assert n_vis > 200


@pytest.mark.parametrize("rotated", [False, True])
def test_orthographic_gradients_match_central_differences(orc, rotated):
    sc = _ortho(config_scene(0))
    rows = np.eye(3)
    t = np.zeros(3)
    if rotated:
        rows = random_rotation(np.random.default_rng(8)).T
        t = np.array([0.0, 0.0, 7.5]) - 7.5 * rows[2]
    # a sensor 6 units wide: 0.75 px minimum size, the regime of the pinhole pins (spheres much
    # larger than a pixel put a rim kink inside nearly every difference stencil)
    sc.cam = make_cam(t=t, rot6=np.concatenate([rows[0], rows[1]]), focal=1.4, sensor_width=6.0)
    G = np.zeros((sc.height, sc.width, 3))
    G[24:40, 24:40] = grad_image(78, 16, 16, 3)
    K = 64
    grads = orc.render_backward(sc, G, n_track=K)
    full = orc.render(sc, n_track=K)
    assert full.n_hits.max() <= K and full.n_hits[24:40, 24:40].sum() > 200
    assert grads.cam[9] == 0.0 and abs(grads.cam[10]) > 0
    seen = np.unique(full.tracked[24:40, 24:40][full.tracked[24:40, 24:40] >= 0])
    sph = np.random.default_rng(2).choice(seen, size=min(10, len(seen)), replace=False)
    _check_fd(orc, sc, G, grads, "pos", [3 * i + k for i in sph for k in range(3)], K)
    _check_fd(orc, sc, G, grads, "rad", list(sph), K)
    _check_fd(orc, sc, G, grads, "opa", list(sph), K)
    _check_fd(orc, sc, G, grads, "feat", [3 * i + k for i in sph[:4] for k in range(3)], K)
    # a camera change moves every sphere across the pixel grid (1/k pixels per unit of
    # translation across the rays, |p - t| per unit of rotation): smaller steps keep rim kinks
    # out of the stencils; a translation along the rays has a small derivative that needs a
    # larger step against round-off
    _check_fd(orc, sc, G, grads, "cam", [0, 1, 2, 3, 4, 5, 6, 7, 8, 10], K, hscales=(0.05, 1.0, 5.0))
    _check_fd(orc, sc, G, grads, "bg", [0, 1, 2], K)


# ---------------------------------------------------------------- the paper's 1 % early termination

def _stop_column(t4):
    """Four unit spheres centred on the optical axis whose front surfaces lie
    at depths 3, 3.5, 4 and t4 (znear 1, zfar 11: depth terms 0.8, 0.75, 0.7
    and (11 - t4) / 10), all opaque, gamma 0.1: at the centre pixel the
    exponents are 8, 7.5, 7 and 10 (11 - t4) with d = 1."""
    sc = scene_of([[0, 0, 4.0], [0, 0, 4.5], [0, 0, 5.0], [0, 0, t4 + 1.0]], [1.0] * 4, [1.0] * 4,
                  [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], 65, 65, 0.1, n_track=8, eps=1e-4,
                  znear=1.0, zfar=11.0, bg=[0.25, 0.5, 0.75])
    sc.paper_stop = True
    return sc


@pytest.mark.parametrize("t4, tau, taken", [(7.0, 0.01, 3), (6.8, 0.01, 4), (6.8, 0.02, 3),
                                             (7.0, 0.005, 4)])
def test_paper_stop_on_a_column_of_spheres(orc, t4, tau, taken):
    """By hand: the fourth sphere's largest possible weight is e^{4} / (e^{8} +
    e^{7.5} + e^{7} + e^{4} + e^{0.001}) = 0.0092 at t4 = 7 and e^{4.2} / (...)
    = 0.0112 at t4 = 6.8, so the pixel stops after three hits where that is
    below the threshold (1 % at t4 = 7, 2 % at t4 = 6.8) and takes all four
    otherwise (1 % at t4 = 6.8, 0.5 % at t4 = 7); the second and third spheres
    pass by far (0.38, 0.19)."""
    sc = _stop_column(t4)
    sc.min_contrib = tau
    out = orc.render(sc)
    c = 32
    assert out.n_hits[c, c] == taken
    assert list(out.tracked[c, c, :taken]) == list(range(taken))
    # the image blends the taken hits only (Eq. 1 over three or four spheres)
    e = [(11.0 - f32(k)) / 10.0 / f32(0.1) for k in (3.0, 3.5, 4.0, f32(t4 + 1.0) - 1.0)]
    B = math.exp(f32(1e-4) / f32(0.1))
    feat = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], np.float64)
    num = B * np.array([0.25, 0.5, 0.75]) + sum(math.exp(e[k]) * feat[k] for k in range(taken))
    den = B + sum(math.exp(e[k]) for k in range(taken))
    np.testing.assert_allclose(out.image[c, c], num / den, rtol=1e-12)
    # the smallest distance to the threshold is the fourth test's
    a4 = math.exp(e[3]) / (B + sum(math.exp(x) for x in e))
    margin = orc.paper_stop_margin(sc)
    assert margin[c, c] == pytest.approx(abs(math.log(a4 / f32(tau))), rel=1e-9)
    # without the option every pixel takes every hit
    sc.paper_stop = False
    assert orc.render(sc).n_hits[c, c] == 4


def test_paper_stop_error_is_bounded_by_the_remaining_hits(orc):
    """Each hit a pixel leaves out has weight numerator o d e^{o z / g} at most
    A = e^{o_max z_b / g} of the first left out (o, d <= 1, z <= z_b, keys in
    increasing order), and A / (D + A) < 1 %; with n hits left out, the
    exact colour differs from the truncated one by at most 2 f_max n A / (D + n A)
    <= 2 f_max n t / (1 + n t), t = 0.01 / 0.99."""
    sc = config_scene(0, n=20000, res=48)
    assert sc.opa.max() <= 1.0 and sc.opa.min() >= 0.0
    exact = orc.render(sc)
    sc.paper_stop = True
    stop = orc.render(sc)
    left = exact.n_hits - stop.n_hits
    assert left.min() >= 0 and (left > 0).mean() > 0.01 and stop.n_hits.sum() > 0
    fmax = max(float(np.abs(sc.feat).max()), float(np.abs(sc.bg).max()))
    t = 0.01 / 0.99
    bound = 2.0 * fmax * left * t / (1.0 + left * t)
    err = np.abs(exact.image - stop.image).max(axis=2)
    assert np.all(err <= bound + 1e-12)
    assert np.all(err[left == 0] <= 1e-12)


def test_windowed_backward_equals_full_image_with_zero_outside(orc):
    """The windowed backward (the CPU baseline's timed unit) is the full-image
    backward whose dL/dF is zero outside the window."""
    sc = config_scene(0)
    g = np.random.default_rng(8)
    u0, v0, ww, wh = 20, 26, 13, 9
    Gw = g.standard_normal((wh, ww, sc.n_channels))
    G = np.zeros((sc.height, sc.width, sc.n_channels))
    G[v0:v0 + wh, u0:u0 + ww] = Gw
    full = orc.render_backward(sc, G)
    win = orc.render_backward_window(sc, Gw, u0, v0)
    for k in ("pos", "rad", "opa", "feat", "cam", "bg"):
        a, b = getattr(full, k), getattr(win, k)
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max()), k
