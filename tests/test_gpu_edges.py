"""Edge cases and the PyTorch front end of the CUDA path."""
import math

import numpy as np
import pytest

from paper_2004_07484_gb300 import scenes as S
from helpers import assert_grads_close, gpu_backward, gpu_forward, gpu_tile_lists, assert_tile_lists_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_07484_gb300 import build
    build.build()


def _scene(pos, rad, opa, feat, W, H, gamma=0.1, K=5, bg=None, cam=None):
    feat = np.atleast_2d(np.asarray(feat, np.float32)).reshape(len(rad), -1) if len(rad) else \
        np.zeros((0, len(bg) if bg is not None else 3), np.float32)
    C = feat.shape[1]
    return S.Scene(np.asarray(pos, np.float32).reshape(-1, 3), np.asarray(rad, np.float32).ravel(),
                   np.asarray(opa, np.float32).ravel(), np.ascontiguousarray(feat),
                   S.make_cam() if cam is None else cam,
                   np.zeros(C, np.float32) if bg is None else np.asarray(bg, np.float32), W, H, gamma, K)


def _full_check(orc, sc, **kw):
    ref = orc.render(sc, **{k: v for k, v in kw.items() if k in ("min_size", "dist_literal")})
    gpu = gpu_forward(sc, **kw)
    assert np.abs(gpu["image"].cpu().numpy() - ref.image).max() <= 1e-4
    np.testing.assert_array_equal(gpu["tracked"].cpu().numpy(), ref.tracked)
    off, oids = orc.tile_lists(sc)
    assert_tile_lists_equal(*gpu_tile_lists(gpu["frame"]), off, oids)
    G = S.grad_image(11, sc.height, sc.width, sc.n_channels)
    want = orc.render_backward(sc, G)
    assert_grads_close(gpu_backward(gpu, G), want, scene=sc)
    return gpu, ref


def test_empty_scene_is_background(orc):
    sc = _scene(np.zeros((0, 3)), [], [], np.zeros((0, 4)), 40, 24, bg=[0.1, 0.2, 0.3, 0.4])
    gpu = gpu_forward(sc)
    img = gpu["image"].cpu().numpy()
    assert np.allclose(img, np.array([0.1, 0.2, 0.3, 0.4], np.float32)[None, None, :])
    G = S.grad_image(1, 24, 40, 4)
    got = gpu_backward(gpu, G)
    np.testing.assert_allclose(got["bg"], G.astype(np.float64).sum(axis=(0, 1)), rtol=1e-4)
    assert np.all(got["cam"] == 0)


def test_all_spheres_culled(orc):
    g = np.random.default_rng(0)
    pos = np.stack([g.uniform(-1, 1, 50), g.uniform(-1, 1, 50), g.uniform(-5, 0.5, 50)], 1)
    sc = _scene(pos, g.uniform(0.1, 0.3, 50), np.ones(50), g.uniform(0, 1, (50, 3)), 32, 32)
    gpu, ref = _full_check(orc, sc)
    assert gpu["n_hits"].cpu().numpy().sum() == 0


def test_single_sphere_on_axis_closed_form(orc):
    W = H = 33
    Z, r, o = 6.0, 2.0, 0.8
    f = np.array([0.3, 0.7, 0.2], np.float32)
    sc = _scene([0, 0, Z], [r], [o], f, W, H, gamma=0.1, bg=[0.1, 0.2, 0.9])
    gpu, _ = _full_check(orc, sc)
    z = (20.0 - (Z - r)) / 19.0
    a = float(np.float32(o)) * math.exp(float(np.float32(o)) * z / float(np.float32(0.1)))
    B = math.exp(float(np.float32(1e-5)) / float(np.float32(0.1)))
    want = (a * f.astype(np.float64) + B * np.array([0.1, 0.2, 0.9], np.float32)) / (B + a)
    np.testing.assert_allclose(gpu["image"].cpu().numpy()[16, 16], want, atol=1e-5)


@pytest.mark.parametrize("C,K", [(1, 1), (2, 3), (5, 9), (32, 32), (12, 17), (8, 8)])
def test_channel_and_track_counts(orc, C, K):
    sc = S.gaussian_mixture(2000 + C * 33 + K, 2500, 48, 40, n_channels=C, gamma=0.05, n_track=K,
                            mean_xy=(-0.7, 0.7), feat="normal")
    _full_check(orc, sc)


@pytest.mark.parametrize("W,H", [(1, 1), (17, 1), (1, 31), (33, 47), (16, 16)])
def test_ragged_and_tiny_images(orc, W, H):
    sc = S.uniform_cloud(3000 + W * 7 + H, 400, W, H, n_channels=3, gamma=0.1, n_track=5,
                         xy=(-0.6, 0.6), rad=(0.05, 0.5))
    _full_check(orc, sc)


def test_capacity_overflow_is_reported_and_recovered(orc):
    import torch
    from paper_2004_07484_gb300 import _lib, forward_frame
    from helpers import settings_of, to_dev
    sc = S.config_scene(0)
    dev = to_dev(sc)
    s = settings_of(sc)
    fr, _, _ = forward_frame(s, dev["pos"], dev["feat"], dev["rad"], dev["opa"], dev["cam"], dev["bg"],
                             16, check_overflow=False)
    st, need = _lib.read_status(fr.ws.data_ptr(), fr.ws_bytes, torch.cuda.current_stream().cuda_stream)
    assert st == _lib.ERR_CAPACITY and need > 16
    st2, need_bytes = _lib.last_overflow(fr.params, fr.ws.data_ptr(), fr.ws_bytes,
                                         torch.cuda.current_stream().cuda_stream)
    assert st2 == _lib.ERR_CAPACITY
    assert need_bytes == _lib.workspace_size(s.params(sc.n_spheres, need)) > fr.ws_bytes
    fr2, img, _ = forward_frame(s, dev["pos"], dev["feat"], dev["rad"], dev["opa"], dev["cam"], dev["bg"],
                                16, check_overflow=True)
    assert fr2.params.list_capacity >= need
    ref = orc.render(sc)
    assert np.abs(img.cpu().numpy() - ref.image).max() <= 1e-4


def test_decisions_are_deterministic(orc):
    sc = S.config_scene(1, n=20000, res=128)
    a = gpu_forward(sc)
    b = gpu_forward(sc)
    assert np.array_equal(a["tracked"].cpu().numpy(), b["tracked"].cpu().numpy())
    ra, ia = gpu_tile_lists(a["frame"])
    rb, ib = gpu_tile_lists(b["frame"])
    assert np.array_equal(ra, rb)
    n = int(ra[:, 1].max())
    assert np.array_equal(ia[:n], ib[:n])


@pytest.mark.parametrize("store,persistent", [(True, False), (True, True), (False, True)])
def test_repeated_calls_on_one_workspace(orc, store, persistent):
    """Binning twice after one projection, a second forward pass, and two
    backward passes of one forward pass give the single calls' results: the
    counters the kernels' last CTAs use to finish a scan or a reduction, and
    the work counter a persistent launch resets itself (shared, in recompute
    mode, by the track pass and the backward render of one call), are ready
    again after each call.  (The single calls' parity with the oracle is
    tested elsewhere.)"""
    import torch
    from paper_2004_07484_gb300 import _lib
    from paper_2004_07484_gb300.renderer import scene_args
    sc = S.config_scene(1, n=20000, res=128)
    gpu = gpu_forward(sc, store=store, persistent=persistent, segment=256)
    fr, d = gpu["frame"], gpu["dev"]
    ranges0, ids0 = gpu_tile_lists(fr)
    stream = torch.cuda.current_stream().cuda_stream
    _lib.bin(fr.params, fr.ws.data_ptr(), fr.ws_bytes, stream)   # again, on the same projection
    ranges1, ids1 = gpu_tile_lists(fr)
    assert np.array_equal(ranges0, ranges1)
    n = int(ranges0[:, 1].max())
    assert np.array_equal(ids0[:n], ids1[:n])
    image = torch.empty_like(gpu["image"])
    log_norm = torch.empty_like(gpu["log_norm"])
    sa = scene_args(d["pos"], d["feat"], d["rad"], d["opa"], d["cam"], d["bg"])
    _lib.render_fwd(fr.params, sa, fr.ws.data_ptr(), fr.ws_bytes, image.data_ptr(), log_norm.data_ptr(),
                    None, None, None, stream)
    torch.cuda.synchronize()
    assert torch.equal(image, gpu["image"]) or (image - gpu["image"]).abs().max().item() <= 1e-6
    G = S.grad_image(12, sc.height, sc.width, sc.n_channels)
    g1 = gpu_backward(gpu, G)
    g2 = gpu_backward(gpu, G)
    # every tracked hit adds to its sphere's feature gradient: a backward launch that found its
    # work counter spent would leave them zero (radius gradients can be zero throughout here:
    # spheres enlarged to the minimum projected size have none)
    assert np.abs(g1["feat"]).max() > 0 and np.abs(g2["feat"]).max() > 0
    for k in g1:
        if g1[k] is None:
            continue
        scale = max(np.abs(g1[k]).max(), 1e-30)
        assert np.abs(g1[k] - g2[k]).max() <= 1e-5 * scale, k   # float atomics may add in another order


def test_module_autograd_matches_oracle(orc):
    import torch
    from paper_2004_07484_gb300 import Renderer
    sc = S.config_scene(0)
    r = Renderer(sc.width, sc.height, sc.n_spheres, n_channels=3, n_track=sc.n_track, gamma=sc.gamma)
    t = {k: torch.from_numpy(getattr(sc, k)).cuda().requires_grad_(True)
         for k in ("pos", "feat", "rad", "opa", "cam", "bg")}
    img = r(t["pos"], t["feat"], t["rad"], t["cam"], opa=t["opa"], bg=t["bg"])
    G = S.grad_image(12, sc.height, sc.width, 3)
    (img * torch.from_numpy(G).cuda()).sum().backward()
    want = orc.render_backward(sc, G)
    got = {k: t[k].grad.cpu().numpy().astype(np.float64) for k in t}
    assert_grads_close(got, want, scene=sc)
    # only what autograd asks for is computed
    t2 = {k: torch.from_numpy(getattr(sc, k)).cuda() for k in ("pos", "feat", "rad", "opa", "cam", "bg")}
    t2["feat"].requires_grad_(True)
    img2 = r(t2["pos"], t2["feat"], t2["rad"], t2["cam"], opa=t2["opa"], bg=t2["bg"])
    (img2 * torch.from_numpy(G).cuda()).sum().backward()
    np.testing.assert_allclose(t2["feat"].grad.cpu().numpy(), want.feat, atol=1e-5)


def test_listing1_example_runs():
    """The ten-sphere, 1024 x 1024 example of Listing 1 (identity rotation)."""
    import torch
    from paper_2004_07484_gb300 import Renderer
    g = np.random.default_rng(1)
    pos = g.uniform(0, 1, (10, 3)) * 10.0
    pos[:, 2] += 25.0
    pos[:, :2] -= 5.0
    r = Renderer(1024, 1024, 10, n_channels=3)
    cam = torch.tensor([0, 0, 0, 1, 0, 0, 0, 1, 0, 5.0, 2.0], dtype=torch.float32, device="cuda")
    pos_t = torch.tensor(pos, dtype=torch.float32, device="cuda", requires_grad=True)
    col = torch.tensor(g.uniform(0, 1, (10, 3)), dtype=torch.float32, device="cuda")
    rad = torch.tensor(g.uniform(0, 1, 10), dtype=torch.float32, device="cuda")
    img = r(pos_t, col, rad, cam, gamma=0.1, max_depth=45.0)
    img.abs().sum().backward()
    assert torch.isfinite(img).all() and (img.sum(-1) > 0).any()
    assert torch.isfinite(pos_t.grad).all()


@pytest.mark.parametrize("segment,persistent", [(32, False), (64, True), (0, True), (4096, False)],
                         ids=["seg32", "seg64-persistent", "default-persistent", "seg4096"])
def test_scheduling_options_leave_results_unchanged(orc, segment, persistent):
    """Splitting tile lists into short segments (many merged partial states)
    and persistent kernels change only the scheduling: tracked hits stay
    bit-exact, images and gradients stay at oracle parity."""
    sc = S.ellipsoid_surfaces(1077, 20000, 80, 80, n_channels=16, gamma=1e-2, n_track=16,
                              centre_xy=(-0.6, 0.6), centre_z=(5.0, 8.0), axes=(0.3, 1.0))
    ref = orc.render(sc)
    for store in (True, False):
        gpu = gpu_forward(sc, store=store, segment=segment, persistent=persistent)
        assert np.abs(gpu["image"].cpu().numpy() - ref.image).max() <= 1e-4
        np.testing.assert_array_equal(gpu["tracked"].cpu().numpy(), ref.tracked)
        assert np.abs(gpu["log_norm"].cpu().numpy() - ref.log_d).max() <= 1e-4 * max(1.0, np.abs(ref.log_d).max())
        G = S.grad_image(12, sc.height, sc.width, sc.n_channels)
        assert_grads_close(gpu_backward(gpu, G), orc.render_backward(sc, G), scene=sc)


def test_fma_probe_measures_a_plausible_fp32_rate():
    import torch
    from paper_2004_07484_gb300 import _lib
    sink = torch.zeros(1, device="cuda")
    flops, ms = _lib.probe_fma_throughput(sink.data_ptr(), 2048, torch.cuda.current_stream().cuda_stream)
    assert ms > 0.0
    # 152 SMs x 128 FP32 lanes x 2 flops at 0.5..2.1 GHz
    assert 10e12 < flops < 90e12, flops
    assert float(sink.item()) == 0.0


def test_adam_steps_reduce_the_image_loss():
    """The renderer as a training component: Adam on positions, radii,
    opacities and colours lowers the L2 distance to a target rendered from
    perturbed spheres (the shape of the paper's optimisation experiments)."""
    import torch
    from paper_2004_07484_gb300 import Renderer
    sc = S.config_scene(0)
    r = Renderer(sc.width, sc.height, sc.n_spheres, n_channels=3, n_track=sc.n_track, gamma=sc.gamma)
    t = {k: torch.from_numpy(getattr(sc, k)).cuda() for k in ("pos", "feat", "rad", "opa", "cam", "bg")}
    with torch.no_grad():
        target = r(t["pos"], t["feat"], t["rad"], t["cam"], opa=t["opa"], bg=t["bg"]).clone()
    g = torch.Generator(device="cuda").manual_seed(3)
    p = {"pos": (t["pos"] + 0.02 * torch.randn(t["pos"].shape, generator=g, device="cuda")).requires_grad_(True),
         "feat": (t["feat"] * 0.7).requires_grad_(True),
         "rad": (t["rad"] * 1.2).requires_grad_(True),
         "opa": (t["opa"] * 0.9).requires_grad_(True)}
    opt = torch.optim.Adam(p.values(), lr=1e-2)
    losses = []
    for _ in range(30):
        opt.zero_grad()
        img = r(p["pos"], p["feat"], p["rad"], t["cam"], opa=p["opa"], bg=t["bg"])
        loss = ((img - target) ** 2).sum()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])


@pytest.mark.parametrize("store", [True, False], ids=["store", "recompute"])
def test_paper_gradients_match_oracle(orc, store):
    """The paper's gradient normalisations (App. B, end of "The Backward
    Pass"; Sec. 6) against the oracle's: spheres of 0.3 to 7 pixels projected
    radius under a rotated camera, upstream gradient zero on some pixels (they
    still count), one sphere set seen by two views of a batch adding into one
    set of buffers."""
    from paper_2004_07484_gb300.scenes import uniform_cloud
    sc = uniform_cloud(71, 300, 96, 72, n_channels=4, gamma=0.05, n_track=6, rad=(0.02, 1.0))
    rows = S.random_rotation(np.random.default_rng(5)).T
    centre = sc.pos.astype(np.float64).mean(axis=0)
    sc.cam = S.make_cam(t=centre - 8.0 * rows[2], rot6=S.rot6_from_matrix(rows))
    G = S.grad_image(13, sc.height, sc.width, sc.n_channels)
    G[::4, ::3] = 0.0
    gpu = gpu_forward(sc, store=store, paper=True)
    want = orc.render_backward(sc, G, paper_grad=True)
    got = gpu_backward(gpu, G)
    assert_grads_close(got, want, scene=sc)
    hit = np.abs(want.opa) > 0
    gated = np.abs(want.pos).sum(axis=1) == 0
    assert (hit & gated).any() and (hit & ~gated).any()   # both sides of the 3-pixel gate


def test_paper_gradients_accumulate_over_views(orc):
    import torch
    from dataclasses import replace
    from paper_2004_07484_gb300 import _lib, backward_batch, forward_batch
    from helpers import settings_of
    from paper_2004_07484_gb300.scenes import uniform_cloud
    sc = uniform_cloud(72, 200, 64, 64, n_channels=4, gamma=0.05, n_track=6, rad=(0.02, 1.0))
    centre = sc.pos.astype(np.float64).mean(axis=0)
    cams = S.orbit_cameras(9, centre, n_views=2, distance=6.0)
    d = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).cuda() for k in ("pos", "feat", "rad", "opa", "bg")}
    inputs = [(d["pos"], d["feat"], d["rad"], d["opa"], torch.from_numpy(c).cuda(), d["bg"]) for c in cams]
    s = replace(settings_of(sc, paper=True), accumulate=True)
    fr, images, log_norms = forward_batch([s, s], inputs, [1 << 16] * 2)
    Gs = [S.grad_image(20 + k, sc.height, sc.width, sc.n_channels) for k in range(2)]
    M, C = sc.n_spheres, sc.n_channels
    shared = (torch.zeros((M, 3), device="cuda"), torch.zeros(M, device="cuda"), torch.zeros(M, device="cuda"),
              torch.zeros((M, C), device="cuda"))
    out = [shared + (None, None)] * 2
    mask = _lib.GRAD_POS | _lib.GRAD_RAD | _lib.GRAD_OPA | _lib.GRAD_FEAT
    backward_batch(fr, inputs, images, log_norms, [torch.from_numpy(G).cuda() for G in Gs], mask, out=out)
    torch.cuda.synchronize()
    from types import SimpleNamespace
    refs = [orc.render_backward(SimpleNamespace(**{**sc.__dict__, "cam": c}), G, paper_grad=True)
            for c, G in zip(cams, Gs)]
    tot = SimpleNamespace(**{n: getattr(refs[0], n) + getattr(refs[1], n) for n in ("pos", "rad", "opa", "feat")})
    got = {n: t.cpu().numpy().astype(np.float64) for n, t in zip(("pos", "rad", "opa", "feat"), shared)}
    assert_grads_close(got, tot, names=("pos", "rad", "opa", "feat"))


@pytest.mark.parametrize("sensor,rotated", [(6.0, False), (2.4, True)], ids=["subpixel", "rotated-large"])
def test_orthographic_camera_matches_oracle(orc, sensor, rotated):
    """The orthographic camera (Sec. 1): tile lists and tracked hits
    bit-exact, image and gradients (store and recompute) at oracle parity,
    for sub-pixel spheres under the minimum size and for spheres up to 3
    pixels under a rotated camera."""
    sc = S.config_scene(0)
    sc.ortho = True
    rows, t = np.eye(3), np.zeros(3)
    if rotated:
        rows = S.random_rotation(np.random.default_rng(8)).T
        t = np.array([0.0, 0.0, 7.5]) - 7.5 * rows[2]
    sc.cam = S.make_cam(t=t, rot6=S.rot6_from_matrix(rows), focal=1.4, sensor_width=sensor)
    gpu, ref = _full_check(orc, sc)
    assert ref.n_hits.sum() > 500
    gpu2 = gpu_forward(sc, store=False)
    G = S.grad_image(11, sc.height, sc.width, sc.n_channels)
    assert_grads_close(gpu_backward(gpu2, G), orc.render_backward(sc, G), scene=sc)


def test_orthographic_batch_with_paper_gradients(orc):
    """A batch of orthographic scenes in paper-gradient mode against the oracle, scene by scene."""
    import torch
    from paper_2004_07484_gb300 import backward_batch, forward_batch
    from helpers import settings_of
    scs = []
    for k, (n, res) in enumerate([(400, 48), (900, 64), (150, 40)]):
        sc = S.uniform_cloud(300 + k, n, res, res, n_channels=4, gamma=0.05, n_track=6, rad=(0.02, 0.4))
        sc.ortho = True
        sc.cam = S.make_cam(sensor_width=3.0 + k)
        scs.append(sc)
    inputs = [tuple(torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).cuda()
                    for k in ("pos", "feat", "rad", "opa", "cam", "bg")) for sc in scs]
    sets = [settings_of(sc, paper=True) for sc in scs]
    fr, images, log_norms = forward_batch(sets, inputs, [1 << 15] * len(scs))
    Gs = [S.grad_image(40 + k, sc.height, sc.width, sc.n_channels) for k, sc in enumerate(scs)]
    grads = backward_batch(fr, inputs, images, log_norms, [torch.from_numpy(G).cuda() for G in Gs])
    torch.cuda.synchronize()
    for sc, img, G, g in zip(scs, images, Gs, grads):
        ref = orc.render(sc)
        assert np.abs(img.cpu().numpy() - ref.image).max() <= 1e-4
        want = orc.render_backward(sc, G, paper_grad=True)
        got = {n: t.cpu().numpy().astype(np.float64) for n, t in zip(("pos", "rad", "opa", "feat", "cam", "bg"), g)}
        assert_grads_close(got, want, scene=sc)


@pytest.mark.parametrize("ortho", [False, True])
def test_test_rectangles_miss_no_hit(orc, ortho):
    """The block lists test only the tangent bounds of each sphere's
    projection widened by 1/8 pixel: every pixel's hit count must still equal
    the oracle's brute-force count over all spheres, for spheres from 0.2 to
    20 pixels in radius, centred anywhere including beyond the image borders,
    under a rotated wide-angle camera."""
    g = np.random.default_rng(31 + ortho)
    W, H, n = 96, 80, 3000
    rows = S.random_rotation(g).T
    t = np.array([0.1, -0.2, 0.3])
    cam = S.make_cam(t=t, rot6=S.rot6_from_matrix(rows), focal=0.8, sensor_width=(6.0 if ortho else 2.4))
    zc = g.uniform(1.5, 15.0, n)
    k = (6.0 / W) if ortho else (2.4 / (W * 0.8))
    span = np.stack([W, H]) * 0.6 * k
    xy = g.uniform(-1, 1, (n, 2)) * (span if ortho else span[None] * zc[:, None])
    pc = np.concatenate([xy, zc[:, None]], axis=1)
    pos = (rows.T @ pc.T).T + t
    pix = k if ortho else k * zc
    rad = pix * np.exp(g.uniform(np.log(0.2), np.log(20.0), n))
    sc = S.Scene(pos.astype(np.float32), rad.astype(np.float32), g.uniform(0.3, 1, n).astype(np.float32),
                 g.uniform(0, 1, (n, 3)).astype(np.float32), cam, np.zeros(3, np.float32), W, H, 0.05, 8,
                 zfar=20.0, ortho=ortho)
    ref = orc.render(sc)
    gpu = gpu_forward(sc, capacity=1 << 20)
    assert ref.n_hits.sum() > 10000
    np.testing.assert_array_equal(gpu["n_hits"].cpu().numpy(), ref.n_hits)
    np.testing.assert_array_equal(gpu["tracked"].cpu().numpy(), ref.tracked)
    assert np.abs(gpu["image"].cpu().numpy() - ref.image).max() <= 1e-4


def _deep_cloud(seed, n, W, H, rad):
    """Spheres from depth 2 to 18 at gamma 0.05: far hits behind near ones
    fall below the 1 % of the paper's early termination at a few per cent of
    the pixels."""
    sc = S.uniform_cloud(seed, n, W, H, gamma=0.05, n_track=5, rad=rad, z=(2.0, 18.0))
    sc.paper_stop = True
    return sc


def _truncation_bound(exact, stop, sc):
    """Largest colour change from leaving out n hits (each with a weight
    numerator at most A, A / (D + A) < tau): 2 f_max n t / (1 + n t)."""
    left = exact.n_hits - stop.n_hits
    tau = float(np.float32(sc.min_contrib))
    t = tau / (1.0 - tau)
    fmax = max(float(np.abs(sc.feat).max()), float(np.abs(sc.bg).max()))
    return 2.0 * fmax * left * t / (1.0 + left * t)


@pytest.mark.parametrize("persistent,tau,segment", [(False, 0.01, 0), (True, 0.01, 0), (False, 0.05, 0),
                                                    (False, 0.01, 32), (True, 0.01, 64)],
                         ids=["items", "persistent", "5-percent", "chain-32", "chain-64-persistent"])
def test_paper_stop_forward_matches_oracle(orc, persistent, tau, segment):
    """The paper's early termination (App. B, Step 2): on every pixel whose
    decisions lie clear of the threshold (|ln(a / tau)| >= 1e-3 for every
    test the oracle takes; a float32 denominator can only decide otherwise
    nearer) the image is at oracle parity and the tracked hits are equal; every
    pixel stays within the truncation bound of the exact image."""
    sc = _deep_cloud(85, 2000, 64, 48, (0.05, 0.4))
    sc.min_contrib = tau
    ref = orc.render(sc)
    margin = orc.paper_stop_margin(sc)
    sc_exact = S.Scene(**{**sc.__dict__, "paper_stop": False})
    exact = orc.render(sc_exact)
    assert (exact.n_hits > ref.n_hits).mean() > 0.01          # the option does cut lists here
    gpu = gpu_forward(sc, persistent=persistent, segment=segment)
    img = gpu["image"].cpu().numpy()
    clear = margin >= 1e-3
    assert clear.mean() >= 0.99
    err = np.abs(img - ref.image).max(axis=2)
    assert err[clear].max() <= 1e-4
    np.testing.assert_array_equal(gpu["tracked"].cpu().numpy()[clear], ref.tracked[clear])
    bound = _truncation_bound(exact, ref, sc)
    assert np.all(np.abs(img - exact.image).max(axis=2) <= bound + 1e-4)
    # the exact renderer differs from it by the truncation
    plain = gpu_forward(sc_exact)
    assert np.abs(plain["image"].cpu().numpy() - exact.image).max() <= 1e-4


def test_paper_stop_gradients_match_oracle(orc):
    """Gradients through the hits the early termination kept (the forward
    pass records where each pixel stopped); every decision of this scene lies
    at least 2e-3 from the threshold.  Tile lists split into 32-entry segments
    walked in order give the same.  Without stored hits the backward pass
    reports an unsupported setting."""
    sc = _deep_cloud(86, 600, 48, 40, (0.1, 0.5))
    assert orc.paper_stop_margin(sc).min() >= 2e-3
    ref = orc.render(sc)
    G = S.grad_image(12, sc.height, sc.width, sc.n_channels)
    want = orc.render_backward(sc, G)
    for segment in (32, 64):
        gpu = gpu_forward(sc, segment=segment, persistent=segment == 64)
        np.testing.assert_array_equal(gpu["tracked"].cpu().numpy(), ref.tracked)
        assert np.abs(gpu["image"].cpu().numpy() - ref.image).max() <= 1e-4
        assert_grads_close(gpu_backward(gpu, G), want, scene=sc)
    gpu = gpu_forward(sc)
    assert np.abs(gpu["image"].cpu().numpy() - ref.image).max() <= 1e-4
    np.testing.assert_array_equal(gpu["tracked"].cpu().numpy(), ref.tracked)
    assert_grads_close(gpu_backward(gpu, G), want, scene=sc)
    # the gradients differ from the exact renderer's (hits were left out)
    sc_exact = S.Scene(**{**sc.__dict__, "paper_stop": False})
    full = orc.render_backward(sc_exact, G)
    assert np.abs(full.opa - want.opa).max() > 1e-5 * np.abs(full.opa).max()
    rec = gpu_forward(sc, store=False)
    with pytest.raises(Exception, match="unsupported"):
        gpu_backward(rec, G)
