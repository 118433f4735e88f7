"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: per-tile sphere lists and per-pixel tracked hits bit-exact; images
within 1e-4 max-abs of the FP64 oracle; gradients within 1e-3 relative
(max-norm per tensor, and elementwise |g - ref| <= 1e-3 (|ref| + 1e-3 max|ref|)).
"""
import numpy as np
import pytest

from paper_2004_07484_gb300 import scenes as S
from helpers import (assert_grads_close, assert_tile_lists_equal, gpu_backward, gpu_forward,
                     gpu_tile_lists, grad_error)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_07484_gb300 import build
    build.build()


def ragged_rotated():
    g = np.random.default_rng(21)
    sc = S.gaussian_mixture(1021, 3000, 100, 72, n_channels=3, gamma=0.05, n_track=10)
    rows = S.random_rotation(g).T
    centroid = sc.pos.astype(np.float64).mean(axis=0)
    sc.cam = S.make_cam(t=centroid - 7.0 * rows[2], rot6=np.concatenate([rows[0], rows[1]]),
                        focal=1.2, sensor_width=2.0)
    sc.name = "ragged_rotated"
    return sc


def edge_scene():
    """Spheres behind the camera, straddling the near plane, beyond the far
    plane, far off-screen, huge (covering the image), on tile borders."""
    g = np.random.default_rng(33)
    pts, rad = [], []
    for _ in range(60):                    # ordinary
        pts.append([g.uniform(-2, 2), g.uniform(-2, 2), g.uniform(3, 15)]); rad.append(g.uniform(0.05, 0.6))
    for _ in range(20):                    # behind / straddling the near plane
        pts.append([g.uniform(-1, 1), g.uniform(-1, 1), g.uniform(-3, 1.5)]); rad.append(g.uniform(0.1, 1.0))
    for _ in range(20):                    # beyond / straddling the far plane
        pts.append([g.uniform(-3, 3), g.uniform(-3, 3), g.uniform(18, 25)]); rad.append(g.uniform(0.1, 3.0))
    for _ in range(20):                    # off-screen, wide angles
        z = g.uniform(3, 12)
        pts.append([g.choice([-1, 1]) * g.uniform(1.2, 3) * z, g.uniform(-1.5, 1.5) * z, z]); rad.append(g.uniform(0.1, 2))
    pts.append([0.0, 0.0, 9.0]); rad.append(6.0)      # covers every pixel
    pts.append([0.3, -0.2, 14.0]); rad.append(9.0)
    kappa = 2.0 / 48
    for k in range(8):                     # centred on tile borders
        z = 6.0
        pts.append([(16 * (k % 3) - 24) * kappa * z, (16 * (k // 3) - 20) * kappa * z, z]); rad.append(0.05)
    n = len(pts)
    sc = S.Scene(np.asarray(pts, np.float32), np.asarray(rad, np.float32),
                 g.uniform(0.3, 1.0, n).astype(np.float32), g.uniform(0, 1, (n, 3)).astype(np.float32),
                 S.make_cam(), np.array([0.1, 0.2, 0.3], np.float32), 48, 40, 0.1, 8, name="edge")
    return sc


def dense_c16():
    sc = S.ellipsoid_surfaces(1077, 20000, 80, 80, n_channels=16, gamma=1e-2, n_track=16,
                              centre_xy=(-0.6, 0.6), centre_z=(5.0, 8.0), axes=(0.3, 1.0))
    sc.name = "dense_c16"
    return sc


SCENES = {
    "cfg0": lambda: S.config_scene(0),
    "ragged_rotated": ragged_rotated,
    "edge": edge_scene,
    "dense_c16": dense_c16,
    "gmm_gamma1e-3": lambda: S.gaussian_mixture(1031, 4000, 64, 48, gamma=1e-3, n_track=10,
                                                 mean_xy=(-0.8, 0.8)),
    "gmm_gamma1": lambda: S.gaussian_mixture(1032, 4000, 64, 48, gamma=1.0, n_track=10,
                                              mean_xy=(-0.8, 0.8)),
}
VARIANTS = [("cfg0", {}), ("cfg0", {"dist_literal": True}), ("cfg0", {"min_size": False}),
            ("ragged_rotated", {}), ("edge", {}), ("dense_c16", {}), ("gmm_gamma1e-3", {}),
            ("gmm_gamma1", {})]


def _id(v):
    name, kw = v
    return name + "".join(f"-{k}" for k in kw)


@pytest.fixture(scope="module")
def cache():
    return {}


def run_pair(orc, cache, name, kw):
    key = (name, tuple(sorted(kw.items())))
    if key not in cache:
        sc = SCENES[name]()
        okw = dict(min_size=kw.get("min_size", True), dist_literal=kw.get("dist_literal", False))
        ref = orc.render(sc, **okw)
        gpu = gpu_forward(sc, **kw)
        cache[key] = (sc, ref, gpu, okw)
    return cache[key]


@pytest.mark.parametrize("variant", VARIANTS, ids=_id)
def test_tile_lists_bit_exact(orc, cache, variant):
    sc, ref, gpu, okw = run_pair(orc, cache, *variant)
    off, oids = orc.tile_lists(sc, tile=16, min_size=okw["min_size"])
    ranges, ids = gpu_tile_lists(gpu["frame"])
    assert_tile_lists_equal(ranges, ids, off, oids)


@pytest.mark.parametrize("config", [1, 2], ids=["100k_spheres_512", "1M_spheres_1024"])
def test_tile_lists_bit_exact_full_size(orc, config):
    """Every tile's list of the full-size workloads (1,024 and 4,096 tiles, so
    the tile-key sort takes more than one digit pass) equals the oracle's
    by-definition lists (App. B, Step 1)."""
    sc = S.config_scene(config)
    gpu = gpu_forward(sc, capacity=16 << 20)
    ranges, ids = gpu_tile_lists(gpu["frame"])
    off, oids = orc.tile_lists(sc, tile=16)
    assert len(oids) > 100_000
    assert_tile_lists_equal(ranges, ids, off, oids)


@pytest.mark.parametrize("variant", VARIANTS, ids=_id)
def test_forward_matches_oracle(orc, cache, variant):
    sc, ref, gpu, okw = run_pair(orc, cache, *variant)
    img = gpu["image"].cpu().numpy().astype(np.float64)
    err = np.abs(img - ref.image).max()
    assert err <= 1e-4, err
    np.testing.assert_array_equal(gpu["tracked"].cpu().numpy(), ref.tracked)
    ld = gpu["log_norm"].cpu().numpy().astype(np.float64)
    assert np.abs(ld - ref.log_d).max() <= 1e-4 * max(1.0, np.abs(ref.log_d).max())
    # hits blended before the exact stop can only be fewer than all hits
    assert np.all(gpu["n_hits"].cpu().numpy() <= ref.n_hits)


@pytest.mark.parametrize("store", [True, False], ids=["store", "recompute"])
@pytest.mark.parametrize("variant", VARIANTS, ids=_id)
def test_backward_matches_oracle(orc, cache, variant, store):
    sc, ref, gpu, okw = run_pair(orc, cache, *variant)
    if not store:
        gpu = gpu_forward(sc, store=False, **variant[1])
    G = S.grad_image(99, sc.height, sc.width, sc.n_channels)
    want = orc.render_backward(sc, G, **okw)
    got = gpu_backward(gpu, G)
    assert_grads_close(got, want, scene=sc)


def test_store_and_recompute_agree(orc):
    sc = dense_c16()
    G = S.grad_image(5, sc.height, sc.width, sc.n_channels)
    a = gpu_backward(gpu_forward(sc, store=True), G)
    b = gpu_backward(gpu_forward(sc, store=False), G)
    for k in a:
        rel, _ = grad_error(a[k], b[k])
        assert rel <= 1e-5, (k, rel)


def test_gradients_match_central_differences(orc):
    """GPU gradients of fully tracked spheres against FP64 central differences
    of the oracle's forward pass (decisions frozen, all hits inside n_track)."""
    sc = S.config_scene(0, n=400)
    sc.n_track = 32
    G = np.zeros((sc.height, sc.width, 3))
    G[24:40, 24:40] = S.grad_image(77, 16, 16, 3)
    full = orc.render(sc, n_track=64)
    assert full.n_hits.max() <= 32          # every hit is tracked
    got = gpu_backward(gpu_forward(sc, n_track=32), G)
    seen = np.unique(full.tracked[24:40, 24:40][full.tracked[24:40, 24:40] >= 0])
    sph = np.random.default_rng(2).choice(seen, 8, replace=False)
    base = {k: getattr(sc, k).astype(np.float64) for k in ("pos", "rad", "opa", "feat", "cam", "bg")}

    def fd(name, idx, h):
        vals = []
        for s in (1, -1, 2, -2):
            arr = {k: v.copy() for k, v in base.items()}
            arr[name].reshape(-1)[idx] += s * h
            vals.append(float(np.sum(orc.render(sc, freeze_decisions=True, n_track=1, **arr).image * G)))
        return (8 * (vals[0] - vals[1]) - (vals[2] - vals[3])) / (12 * h)

    checks = [("pos", 3 * i + k) for i in sph for k in range(3)] + [("opa", i) for i in sph] + \
             [("rad", i) for i in sph] + [("feat", 3 * i) for i in sph[:3]] + [("cam", k) for k in range(11)]
    scale = {n: max(np.abs(got[n]).max(), 1e-12) for n in got}
    checked = 0
    for name, idx in checks:
        h = 2e-6 * max(1.0, abs(float(base[name].reshape(-1)[idx])))
        want, want2 = fd(name, idx, h), fd(name, idx, h / 2)
        tol = 1e-3 * (abs(want) + 1e-3 * scale[name]) + 1e-7
        if abs(want - want2) > 1e-2 * tol:
            continue   # the stencil crosses a kink of d (a sphere's rim or centre): not differentiable
        g = got[name].reshape(-1)[idx]
        assert abs(g - want) <= tol, (name, idx, g, want)
        checked += 1
    assert checked >= int(0.8 * len(checks)), (checked, len(checks))


@pytest.mark.parametrize("gamma", [1e-3, 1e-2, 0.1, 1.0])
def test_100k_spheres_512_sampled(orc, gamma):
    """The 100k-sphere, 512x512 workload at sampled pixels and a gradient crop."""
    sc = S.config_scene(1, gamma=gamma)
    gpu = gpu_forward(sc)
    g = np.random.default_rng(int(gamma * 1e5))
    n_hits = gpu["n_hits"].cpu().numpy()
    busy = np.argwhere(n_hits > 0)
    pix = np.concatenate([busy[g.choice(len(busy), 300, replace=False)][:, ::-1],
                          np.stack([g.integers(0, 512, 100), g.integers(0, 512, 100)], 1)])
    ref = orc.render_pixels(sc, pix)
    img = gpu["image"].cpu().numpy()[pix[:, 1], pix[:, 0]]
    assert np.abs(img - ref.image).max() <= 1e-4
    np.testing.assert_array_equal(gpu["tracked"].cpu().numpy()[pix[:, 1], pix[:, 0]], ref.tracked)
    # gradients through a 24 x 24 crop around a busy pixel
    v, u = busy[g.integers(len(busy))]
    v0, u0 = min(max(v - 12, 0), 512 - 24), min(max(u - 12, 0), 512 - 24)
    G = np.zeros((512, 512, 3))
    G[v0:v0 + 24, u0:u0 + 24] = S.grad_image(3, 24, 24, 3)
    want = orc.render_backward(sc, G)
    got = gpu_backward(gpu, G)
    assert_grads_close(got, want, scene=sc)


def test_1m_spheres_1024_sampled(orc):
    """The 1M-sphere, 1024x1024, 16-channel workload at sampled pixels."""
    sc = S.config_scene(2)
    gpu = gpu_forward(sc, capacity=16 << 20)
    g = np.random.default_rng(7)
    n_hits = gpu["n_hits"].cpu().numpy()
    busy = np.argwhere(n_hits > 0)
    pix = np.concatenate([busy[g.choice(len(busy), 120, replace=False)][:, ::-1],
                          np.stack([g.integers(0, 1024, 24), g.integers(0, 1024, 24)], 1)])
    ref = orc.render_pixels(sc, pix)
    img = gpu["image"].cpu().numpy()[pix[:, 1], pix[:, 0]]
    assert np.abs(img - ref.image).max() <= 1e-4
    np.testing.assert_array_equal(gpu["tracked"].cpu().numpy()[pix[:, 1], pix[:, 0]], ref.tracked)
    v, u = busy[g.integers(len(busy))]
    v0, u0 = min(max(v - 8, 0), 1024 - 16), min(max(u - 8, 0), 1024 - 16)
    G = np.zeros((1024, 1024, 16))
    G[v0:v0 + 16, u0:u0 + 16] = S.grad_image(4, 16, 16, 16)
    want = orc.render_backward(sc, G)
    for store in (True, False):
        out = gpu if store else gpu_forward(sc, store=False, capacity=16 << 20)
        assert_grads_close(gpu_backward(out, G), want, scene=sc)


_bench_ref = {}


@pytest.mark.parametrize("segment,persistent", [(2048, False), (2048, True), (3072, False), (4096, True)],
                         ids=["seg2048", "seg2048-persistent", "seg3072", "seg4096-persistent"])
def test_1m_spheres_1024_bench_schedules(orc, segment, persistent):
    """The 1M-sphere workload in the launch configurations the benchmark's
    autotuner picks between: sampled pixels bit-exact in their tracked hits and
    within the image bar, and a gradient crop within the gradient bar."""
    sc = S.config_scene(2)
    gpu = gpu_forward(sc, capacity=2 << 20, segment=segment, persistent=persistent)
    if not _bench_ref:
        g = np.random.default_rng(17)
        busy = np.argwhere(gpu["n_hits"].cpu().numpy() > 0)
        pix = busy[g.choice(len(busy), 96, replace=False)][:, ::-1]
        v, u = busy[g.integers(len(busy))]
        v0, u0 = min(max(v - 8, 0), 1024 - 16), min(max(u - 8, 0), 1024 - 16)
        G = np.zeros((1024, 1024, 16))
        G[v0:v0 + 16, u0:u0 + 16] = S.grad_image(8, 16, 16, 16)
        _bench_ref.update(pix=pix, ref=orc.render_pixels(sc, pix), G=G, want=orc.render_backward(sc, G))
    pix, ref = _bench_ref["pix"], _bench_ref["ref"]
    img = gpu["image"].cpu().numpy()[pix[:, 1], pix[:, 0]]
    assert np.abs(img - ref.image).max() <= 1e-4
    np.testing.assert_array_equal(gpu["tracked"].cpu().numpy()[pix[:, 1], pix[:, 0]], ref.tracked)
    assert_grads_close(gpu_backward(gpu, _bench_ref["G"]), _bench_ref["want"], scene=sc)


def test_5m_spheres_1920x1080_sampled(orc):
    """The largest single-scene workload (5M spheres on ellipsoid surfaces,
    1920x1080, C=3, n_track 8) at sampled pixels, with a gradient crop."""
    sc = S.config_scene(4)
    gpu = gpu_forward(sc, capacity=48 << 20)
    g = np.random.default_rng(11)
    n_hits = gpu["n_hits"].cpu().numpy()
    busy = np.argwhere(n_hits > 0)
    pix = np.concatenate([busy[g.choice(len(busy), 60, replace=False)][:, ::-1],
                          np.stack([g.integers(0, 1920, 12), g.integers(0, 1080, 12)], 1)])
    ref = orc.render_pixels(sc, pix)
    img = gpu["image"].cpu().numpy()[pix[:, 1], pix[:, 0]]
    assert np.abs(img - ref.image).max() <= 1e-4
    np.testing.assert_array_equal(gpu["tracked"].cpu().numpy()[pix[:, 1], pix[:, 0]], ref.tracked)
    v, u = busy[g.integers(len(busy))]
    v0, u0 = min(max(v - 6, 0), 1080 - 12), min(max(u - 6, 0), 1920 - 12)
    G = np.zeros((1080, 1920, 3))
    G[v0:v0 + 12, u0:u0 + 12] = S.grad_image(6, 12, 12, 3)
    want = orc.render_backward(sc, G)
    assert_grads_close(gpu_backward(gpu, G), want, scene=sc)
