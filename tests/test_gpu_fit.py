"""The scene fit (Sec. 3.4) on the GPU against its oracle (oracle/fit.py):

  - pulsar_image_loss: loss and dL/dF of both kinds, ragged and misaligned sizes;
  - pulsar_adam_step: several steps over tensors of uneven sizes with boxes,
    the device step counter and the gradient reset;
  - PULSAR_FLAG_ACCUMULATE: views sharing gradient buffers add up to the sum
    of their separate gradients, and to the oracle's summed gradients;
  - ViewFit: a few steps of the whole loop against the oracle's loop, and the
    CUDA-graph replay against eager steps.
"""
import math

import numpy as np
import pytest

from paper_2004_07484_gb300 import scenes as S
from helpers import assert_grads_close, settings_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_07484_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def fit_orc(orc):
    from oracle import fit
    return fit


def _assert_within(got, want, bound, what):
    """|got - want| <= bound elementwise (bound may be an array)."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    diff = np.abs(got - want)
    bound = np.broadcast_to(np.asarray(bound, np.float64), diff.shape)
    bad = np.flatnonzero(~(diff <= bound))
    assert bad.size == 0, (what, bad.size, [(int(i), float(got.flat[i]), float(want.flat[i]), float(bound.flat[i]))
                                            for i in bad[:5]])


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("kind", ["l2", "l1"])
@pytest.mark.parametrize("n,offset", [(0, 0), (1, 0), (3, 1), (1029, 0), (1029, 1), (1_000_003, 0),
                                      (1_000_003, 3)])
def test_image_loss_matches_oracle(fit_orc, kind, n, offset):
    import torch
    from paper_2004_07484_gb300 import _lib
    rng = np.random.default_rng(n + offset)
    F = rng.standard_normal(n + offset).astype(np.float32)
    T = rng.standard_normal(n + offset).astype(np.float32)
    if n > 2:
        T[offset + 1] = F[offset + 1]          # one exact match: sign(0) = 0
    dF, dT = torch.from_numpy(F).cuda(), torch.from_numpy(T).cuda()
    grad = torch.full((n + offset,), 7.0, device="cuda")
    loss = torch.full((1,), 7.0, device="cuda")
    scratch = torch.empty(_lib.LOSS_SCRATCH_FLOATS, device="cuda")
    scale = 0.37
    kcode = _lib.LOSS_L2 if kind == "l2" else _lib.LOSS_L1
    _lib.image_loss(kcode, dF.data_ptr() + 4 * offset, dT.data_ptr() + 4 * offset, n, scale,
                    grad.data_ptr() + 4 * offset, loss.data_ptr(), scratch.data_ptr(), _stream())
    torch.cuda.synchronize()
    ref_loss, ref_grad = fit_orc.image_loss(kind, F[offset:], T[offset:], scale)
    g = grad.cpu().numpy()
    assert np.all(g[:offset] == 7.0)           # nothing written before the range
    if kind == "l1":
        np.testing.assert_array_equal(g[offset:], ref_grad.astype(np.float32))
    else:
        # F - T, then times 2 scale (scale rounded to float32): three roundings of 2^-24
        np.testing.assert_allclose(g[offset:], ref_grad, rtol=3e-7, atol=0)
    # every term is >= 0, so the float32 sums (a few terms per thread, a warp tree, eight
    # warps, then float64 over the CTAs) stay within about 20 roundings of the total
    assert abs(float(loss.item()) - ref_loss) <= 3e-6 * abs(ref_loss)
    # without a gradient buffer only the loss is written
    loss2 = torch.zeros((1,), device="cuda")
    _lib.image_loss(kcode, dF.data_ptr() + 4 * offset, dT.data_ptr() + 4 * offset, n, scale, None,
                    loss2.data_ptr(), scratch.data_ptr(), _stream())
    torch.cuda.synchronize()
    assert float(loss2.item()) == float(loss.item())


def test_adam_steps_match_oracle(fit_orc):
    import torch
    from paper_2004_07484_gb300 import _lib
    rng = np.random.default_rng(21)
    sizes = [0, 1, 2047, 2049, 100_003]
    bounds = [(-math.inf, math.inf), (0.0, 1.0), (-0.5, math.inf), (-math.inf, math.inf), (1e-4, 2.0)]
    theta = [rng.uniform(-1, 1.5, n).astype(np.float32) for n in sizes]
    dev = {k: [torch.from_numpy(x.copy()).cuda() for x in theta] for k in ("theta",)}
    m = [torch.zeros(n, device="cuda") for n in sizes]
    v = [torch.zeros(n, device="cuda") for n in sizes]
    g = [torch.zeros(n, device="cuda") for n in sizes]
    state = torch.zeros(4, dtype=torch.int32, device="cuda")
    ts = (_lib.AdamTensor * len(sizes))(*[
        _lib.AdamTensor(dev["theta"][k].data_ptr(), g[k].data_ptr(), m[k].data_ptr(), v[k].data_ptr(),
                        sizes[k], bounds[k][0], bounds[k][1]) for k in range(len(sizes))])
    # the hyper-parameters as the library receives them (float32), for both sides
    lr, b1, b2, eps = (float(np.float32(x)) for x in (1e-2, 0.9, 0.99, 1e-8))
    hp = _lib.AdamHyper(lr, b1, b2, eps, 1)
    ref = [(x.astype(np.float64), np.zeros(x.size), np.zeros(x.size)) for x in theta]
    gmax = [np.zeros(n) for n in sizes]
    for t in range(1, 5):
        grads = [(rng.standard_normal(n) * 10.0 ** rng.uniform(-4, 1, n)).astype(np.float32) for n in sizes]
        for k in range(len(sizes)):
            g[k].copy_(torch.from_numpy(grads[k]))
            gmax[k] = np.maximum(gmax[k], np.abs(grads[k]))
        _lib.adam_step(ts, hp, state.data_ptr(), _stream())
        torch.cuda.synchronize()
        ref = [fit_orc.adam_step(ref[k][0], grads[k], ref[k][1], ref[k][2], t, lr, b1, b2, eps, *bounds[k])
               for k in range(len(sizes))]
        for k in range(len(sizes)):
            th, mm, vv = ref[k]
            # m is a weighted sum of the gradients (weights summing to < 1) that may cancel: its
            # float32 error is a few roundings of the largest gradient seen; the step divides it
            # by sqrt(v_hat), about the size of the gradients, so it carries that relative error
            # times lr; theta itself is rounded to float32 once per step
            _assert_within(dev["theta"][k].cpu().numpy(), th, 5e-6 * lr + 4e-7 * np.abs(th), ("theta", t, k))
            _assert_within(m[k].cpu().numpy(), mm, 4e-7 * t * gmax[k], ("m", t, k))
            _assert_within(v[k].cpu().numpy(), vv, 3e-6 * np.abs(vv), ("v", t, k))
            assert not g[k].any()              # gradients reset for the next accumulation
            lo, hi = bounds[k]
            th_dev = dev["theta"][k].cpu().numpy()
            assert th_dev.size == 0 or (th_dev.min() >= lo and th_dev.max() <= hi)
    st = state.cpu().numpy()
    assert st[0] == 4
    sv = st.view(np.float32)
    assert sv[1] == pytest.approx(lr / (1 - b1 ** 4), rel=1e-6)
    assert sv[2] == pytest.approx(1 / math.sqrt(1 - b2 ** 4), rel=1e-6)


def _two_views(n=3000, res=64):
    sc = S.config_scene(4, n=n, res=res)
    centre = sc.pos.astype(np.float64).mean(axis=0)
    cams = S.orbit_cameras(5, centre, n_views=2, distance=7.0)
    return sc, cams


def test_accumulate_adds_views_into_shared_buffers(orc, fit_orc):
    import torch
    from dataclasses import replace
    from paper_2004_07484_gb300 import _lib, backward_batch, forward_batch
    sc, cams = _two_views()
    M, C = sc.n_spheres, sc.n_channels
    base = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).cuda() for k in ("pos", "feat", "rad", "opa", "bg")}
    dcams = [torch.from_numpy(c).cuda() for c in cams]
    inputs = [(base["pos"], base["feat"], base["rad"], base["opa"], c, base["bg"]) for c in dcams]
    Gs = [S.grad_image(40 + k, sc.height, sc.width, C) for k in range(2)]
    dG = [torch.from_numpy(G).cuda() for G in Gs]
    s = settings_of(sc)
    caps = [max(8 * M, 1 << 14)] * 2
    fr, images, log_norms = forward_batch([s, s], inputs, caps)
    plain = backward_batch(fr, inputs, images, log_norms, dG)
    torch.cuda.synchronize()
    # the same views with the accumulate flag into one set of buffers that already holds ones
    sa = replace(s, accumulate=True)
    fra, images_a, log_norms_a = forward_batch([sa, sa], inputs, caps)
    shared = (torch.ones((M, 3), device="cuda"), torch.ones(M, device="cuda"), torch.ones(M, device="cuda"),
              torch.ones((M, C), device="cuda"))
    cam_out = [torch.ones(11, device="cuda") for _ in range(2)]
    bg_out = torch.ones(C, device="cuda")
    out = [shared + (cam_out[k], bg_out) for k in range(2)]
    backward_batch(fra, inputs, images_a, log_norms_a, dG, _lib.GRAD_ALL, out=out)
    torch.cuda.synchronize()
    for i, name in enumerate(("pos", "rad", "opa", "feat")):
        want = 1.0 + plain[0][i].cpu().numpy().astype(np.float64) + plain[1][i].cpu().numpy()
        got = shared[i].cpu().numpy()
        scale = float(np.abs(want - 1.0).max())
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-5 * scale + 1e-6, err_msg=name)
    for k in range(2):
        # the camera gradient sums per-sphere terms |dL/dp_i| max(1, |p_i - t|) whose float32
        # atomics run in a different order in the two calls
        gp = plain[k][0].cpu().numpy().astype(np.float64)
        dist = np.linalg.norm(sc.pos.astype(np.float64) - cams[k][:3].astype(np.float64), axis=1)
        terms = float((np.linalg.norm(gp, axis=1) * np.maximum(1.0, dist)).sum())
        np.testing.assert_allclose(cam_out[k].cpu().numpy(), 1.0 + plain[k][4].cpu().numpy(), rtol=0,
                                   atol=1e-6 * terms + 1e-6)
    want_bg = 1.0 + plain[0][5].cpu().numpy() + plain[1][5].cpu().numpy()
    np.testing.assert_allclose(bg_out.cpu().numpy(), want_bg, rtol=1e-5, atol=1e-6)
    # and against the oracle: the summed gradients of the two views
    tot = None
    for k in range(2):
        g = orc.render_backward(fit_orc.view_scene(sc, {n: getattr(sc, n) for n in fit_orc.PARAM_NAMES}, cams[k]),
                                Gs[k])
        tot = g if tot is None else type(g)(*[getattr(tot, n) + getattr(g, n) for n in
                                              ("pos", "rad", "opa", "feat", "cam", "bg")])
    # (the accumulated buffers equal the plain sum above; the oracle is compared with that sum,
    # which carries no rounding of the ones the buffers started from)
    got = {n: plain[0][i].cpu().numpy().astype(np.float64) + plain[1][i].cpu().numpy()
           for i, n in enumerate(("pos", "rad", "opa", "feat"))}
    assert_grads_close(got, tot, names=("pos", "rad", "opa", "feat"))


def _fit_problem(orc, fit_orc, n=1000, res=64, views=2):
    hidden = S.config_scene(4, n=n, res=res)
    centre = hidden.pos.astype(np.float64).mean(axis=0)
    cams = S.orbit_cameras(31, centre, n_views=views, distance=6.0)
    start = S.perturbed(hidden, 32)
    names = fit_orc.PARAM_NAMES
    targets = [orc.render(fit_orc.view_scene(hidden, {k: getattr(hidden, k) for k in names}, c)).image
               for c in cams]
    return hidden, start, cams, [t.astype(np.float32) for t in targets]


def _view_fit(start, cams, targets, lr):
    import torch
    from paper_2004_07484_gb300.fit import AdamSettings, ViewFit
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(start, k))).cuda()
           for k in ("pos", "rad", "opa", "feat", "bg")}
    return ViewFit(settings_of(start), [torch.from_numpy(c).cuda() for c in cams],
                   torch.from_numpy(np.stack(targets)).cuda(), dev["pos"], dev["rad"], dev["opa"], dev["feat"],
                   dev["bg"], max(16 * start.n_spheres, 1 << 14), AdamSettings(lr=lr))


def _loss_bound(F, T):
    """|L_gpu - L_oracle| for L = sum (F - T)^2 when every F is within 1e-4 of the oracle's."""
    d = np.abs(np.asarray(F, np.float64) - np.asarray(T, np.float64))
    return 2e-4 * float(d.sum()) + 1e-8 * d.size


def _adam_step_bound(history, name, lr, steps):
    """Per-element bound on |theta_gpu - theta_oracle| after the steps in history.

    Each step moves a parameter by lr m_hat / (sqrt(v_hat) + eps), a ratio of
    the gradient history that changes by about 3 (the gradient's relative
    error) times lr, and by at most 2 lr when the error flips the gradient's
    sign.  The gradient's error is held to 1e-3 |g| + 1e-5 max|g| per element
    (the gradient tolerance of the parity tests)."""
    b = 0.0
    for g in history:
        a = np.abs(np.asarray(g[name], np.float64))
        rel = 1e-3 + 1e-5 * a.max() / np.maximum(a, 1e-30)
        b = b + lr * np.minimum(2.0, 3.0 * rel)
    return b


@pytest.mark.parametrize("paper_stop", [False, True], ids=["exact", "paper-stop"])
def test_fit_steps_match_oracle_loop(orc, fit_orc, paper_stop):
    """Three Adam steps of the fit against the oracle's loop; also with the
    paper's 1 % early termination, whose decisions in these views all lie at
    least 1.5e-2 from the threshold (it cuts the lists of 1 to 2 % of the
    pixels)."""
    hidden, start, cams, targets = _fit_problem(orc, fit_orc)
    start.paper_stop = paper_stop
    steps, lr = 3, 1e-3
    vf = _view_fit(start, cams, targets, lr)
    losses = []
    for _ in range(steps):
        losses.append(float(vf.step().item()))
    final = float(vf.evaluate().item())
    assert vf.overflowed() == 0 and vf.steps_taken() == steps
    names = fit_orc.PARAM_NAMES
    hist = []
    ref_losses, ref_p, ref_final = fit_orc.fit(start, {k: getattr(start, k) for k in names}, cams, targets,
                                               steps, lr=lr, bounds={"rad": (1e-4, np.inf), "opa": (0.0, 1.0)},
                                               history=hist)
    F0 = [orc.render(fit_orc.view_scene(start, {k: getattr(start, k) for k in names}, c)).image for c in cams]
    bound0 = sum(_loss_bound(f, t) for f, t in zip(F0, targets))
    assert abs(losses[0] - ref_losses[0]) <= bound0, (losses[0], ref_losses[0], bound0)
    assert final < losses[0] and ref_final < ref_losses[0]
    for k in names:
        got = vf.params[k].cpu().numpy().astype(np.float64)
        want = ref_p[k].astype(np.float64)
        _assert_within(got, want, _adam_step_bound(hist, k, lr, steps) + 4e-7 * steps * np.abs(want), k)
    # the losses of later steps: the parameters differ by at most the bound above; a change
    # of the parameters moves the loss by at most sum |dL/dtheta| |change|
    for t in range(1, steps + 1):
        dev_bound = sum(float(np.sum(np.abs(hist[min(t, steps - 1)][k]) * _adam_step_bound(hist[:t], k, lr, t)))
                        for k in names)
        got = losses[t] if t < steps else final
        want = ref_losses[t] if t < steps else ref_final
        assert abs(got - want) <= 2 * bound0 + 2 * dev_bound, (t, got, want, bound0, dev_bound)


def test_fit_graph_replay_matches_eager_steps(orc, fit_orc):
    hidden, start, cams, targets = _fit_problem(orc, fit_orc, n=600, res=64, views=3)
    a = _view_fit(start, cams, targets, 2e-3)
    b = _view_fit(start, cams, targets, 2e-3)
    for _ in range(4):
        a.step()
    b.capture()
    for _ in range(4):
        b.replay()
    la, lb = float(a.evaluate().item()), float(b.evaluate().item())
    assert a.steps_taken() == b.steps_taken() == 4
    assert lb == pytest.approx(la, rel=1e-4)
    for k in a.params:
        # the two runs differ only in the order of the float32 atomics of the backward pass;
        # an update moves a parameter by at most about lr per step
        diff = (a.params[k] - b.params[k]).abs().flatten().cpu().numpy()
        assert diff.max() <= 2 * 4 * 2e-3 + 1e-6, k
        assert np.median(diff) <= 1e-3 * 2e-3, k


def test_fit_overflow_is_reported_and_grown(orc, fit_orc):
    import torch
    from paper_2004_07484_gb300.fit import AdamSettings, ViewFit
    hidden, start, cams, targets = _fit_problem(orc, fit_orc, n=500, res=48)
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(start, k))).cuda()
           for k in ("pos", "rad", "opa", "feat", "bg")}
    vf = ViewFit(settings_of(start), [torch.from_numpy(c).cuda() for c in cams],
                 torch.from_numpy(np.stack(targets)).cuda(), dev["pos"], dev["rad"], dev["opa"], dev["feat"],
                 dev["bg"], 64, AdamSettings())
    vf.evaluate()
    need = vf.overflowed()
    assert need > 2 * 64
    vf.grow(need)
    assert sum(vf.capacities()) >= need
    loss = float(vf.evaluate().item())
    assert vf.overflowed() == 0
    names = fit_orc.PARAM_NAMES
    ref, _ = fit_orc.loss_and_grads(start, {k: getattr(start, k) for k in names}, cams, targets)
    F0 = [orc.render(fit_orc.view_scene(start, {k: getattr(start, k) for k in names}, c)).image for c in cams]
    assert abs(loss - ref) <= sum(_loss_bound(f, t) for f, t in zip(F0, targets))


def test_listing1_camera_conversion_and_gradient(orc):
    """The 8-vector camera of Listing 1 (axis-angle rotation): the library's
    conversion against the oracle's Rodrigues formula, its gradient against
    the oracle's Jacobian (central differences in float64) applied to the
    renderer's camera gradient, and a Renderer call with either camera form."""
    import torch
    from oracle import scene_utils
    from paper_2004_07484_gb300 import _lib, Renderer
    rng = np.random.default_rng(17)
    cams8 = np.concatenate([rng.normal(size=(5, 3)), rng.normal(size=(5, 3)) * 1.2,
                            rng.uniform(0.5, 2.0, (5, 1)), rng.uniform(1.0, 3.0, (5, 1))], axis=1)
    cams8[0, 3:6] = 0.0
    cams8[1, 3:6] = [1e-5, -2e-5, 0.0]
    cams8 = cams8.astype(np.float32)
    d8 = torch.from_numpy(cams8).cuda()
    d11 = torch.empty((5, 11), device="cuda")
    _lib.camera_from_axis_angle(d8.data_ptr(), d11.data_ptr(), 5, _stream())
    g11 = rng.normal(size=(5, 11)).astype(np.float32)
    dg8 = torch.empty((5, 8), device="cuda")
    _lib.camera_axis_angle_backward(d8.data_ptr(), torch.from_numpy(g11).cuda().data_ptr(), dg8.data_ptr(), 5,
                                    _stream())
    torch.cuda.synchronize()
    for k in range(5):
        c8 = cams8[k].astype(np.float64)
        np.testing.assert_allclose(d11[k].cpu().numpy(), scene_utils.cam11_from_cam8(c8), rtol=0, atol=2e-7)
        J = np.zeros((11, 8))
        for j in range(8):
            h = 1e-6
            cp, cm = c8.copy(), c8.copy()
            cp[j] += h
            cm[j] -= h
            J[:, j] = (scene_utils.cam11_from_cam8(cp) - scene_utils.cam11_from_cam8(cm)) / (2 * h)
        want = J.T @ g11[k].astype(np.float64)
        np.testing.assert_allclose(dg8[k].cpu().numpy(), want, rtol=0, atol=2e-6 * max(1.0, np.abs(want).max()))
    # a Renderer call with the 8-vector equals one with the converted 11-vector
    sc = S.config_scene(0)
    r = Renderer(sc.width, sc.height, sc.n_spheres, n_channels=3, n_track=5, gamma=0.1)
    pos = torch.from_numpy(sc.pos).cuda()
    feat = torch.from_numpy(sc.feat).cuda()
    rad = torch.from_numpy(sc.rad).cuda()
    c8 = torch.tensor([0.02, -0.01, 0.05, 0.03, -0.02, 0.01, 1.0, 2.0], device="cuda", requires_grad=True)
    img8 = r(pos, feat, rad, c8)
    (img8 * 1.0).sum().backward()
    c11 = torch.from_numpy(scene_utils.cam11_from_cam8(c8.detach().cpu().numpy().astype(np.float64))
                           .astype(np.float32)).cuda().requires_grad_(True)
    img11 = r(pos, feat, rad, c11)
    img11.sum().backward()
    assert (img8 - img11).abs().max().item() <= 1e-5
    J = np.zeros((11, 8))
    base = c8.detach().cpu().numpy().astype(np.float64)
    for j in range(8):
        cp, cm = base.copy(), base.copy()
        cp[j] += 1e-6
        cm[j] -= 1e-6
        J[:, j] = (scene_utils.cam11_from_cam8(cp) - scene_utils.cam11_from_cam8(cm)) / 2e-6
    want = J.T @ c11.grad.cpu().numpy().astype(np.float64)
    got = c8.grad.cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-3 * np.abs(want).max())


@pytest.mark.parametrize("n", [0, 1, 2047, 2049, 100_003])
def test_prune_and_subdivide_match_oracle(n):
    """Pruning (kept set bit-exact: the same float32 decision on both sides,
    order preserved) and subdivision (children within float rounding) against
    the oracle, for sizes around the 2048-sphere tiles of the compaction."""
    import torch
    from oracle import scene_utils
    from paper_2004_07484_gb300.fit import prune_spheres, subdivide_spheres
    rng = np.random.default_rng(n + 1)
    pos = rng.normal(size=(n, 3)).astype(np.float32)
    rad = rng.uniform(0.01, 0.2, n).astype(np.float32)
    opa = rng.uniform(0, 1, n).astype(np.float32)
    feat = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    bg = np.float32([0.5, 0.4, 0.6])
    act = np.where(rng.uniform(0, 1, n) < 0.2, 0.0, rng.uniform(0, 1, n)).astype(np.float32)
    d = [torch.from_numpy(x).cuda() for x in (pos, rad, opa, feat, bg, act)]
    for activity, tol in ((None, -1.0), (d[5], -1.0), (d[5], 0.35), (None, 0.5)):
        got = prune_spheres(*d[:5], activity=activity, color_tol=tol)
        keep = scene_utils.prune_keep(feat, bg, None if activity is None else act, tol)
        for g, want in zip(got, (pos, rad, opa, feat)):
            np.testing.assert_array_equal(g.cpu().numpy(), want[keep])
    cp, cr, co, cf = subdivide_spheres(*d[:4], offset_scale=0.7, radius_scale=0.3)
    wp, wr, wo, wf = scene_utils.subdivide(pos, rad, opa, feat, 0.7, 0.3)
    np.testing.assert_allclose(cp.cpu().numpy(), wp, rtol=0, atol=4e-7 * max(1.0, np.abs(wp).max() if n else 1.0))
    np.testing.assert_allclose(cr.cpu().numpy(), wr, rtol=1e-7)
    np.testing.assert_array_equal(co.cpu().numpy(), wo.astype(np.float32))
    np.testing.assert_array_equal(cf.cpu().numpy(), wf.astype(np.float32))


def test_fit_with_l1_loss_matches_oracle(orc, fit_orc):
    """The l1 loss of Sec. 3.4 through the whole loop: two steps against the
    oracle's loop (loss within the 1e-4-per-value image tolerance summed over
    the values, parameters within the bound the gradient tolerance gives)."""
    from paper_2004_07484_gb300.fit import AdamSettings, ViewFit
    import torch
    hidden, start, cams, targets = _fit_problem(orc, fit_orc, n=800, res=56)
    steps, lr = 2, 1e-3
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(start, k))).cuda()
           for k in ("pos", "rad", "opa", "feat", "bg")}
    vf = ViewFit(settings_of(start), [torch.from_numpy(c).cuda() for c in cams],
                 torch.from_numpy(np.stack(targets)).cuda(), dev["pos"], dev["rad"], dev["opa"], dev["feat"],
                 dev["bg"], max(16 * start.n_spheres, 1 << 14), AdamSettings(lr=lr, loss="l1"))
    losses = [float(vf.step().item()) for _ in range(steps)]
    names = fit_orc.PARAM_NAMES
    hist = []
    ref_losses, ref_p, _ = fit_orc.fit(start, {k: getattr(start, k) for k in names}, cams, targets, steps, lr=lr,
                                       kind="l1", bounds={"rad": (1e-4, np.inf), "opa": (0.0, 1.0)}, history=hist)
    n_values = sum(t.size for t in targets)
    assert abs(losses[0] - ref_losses[0]) <= 1e-4 * n_values
    final = float(vf.evaluate().item())
    assert final < losses[0]
    # dL/dF = sign(F - T) is decided by float rounding wherever one sphere dominates a pixel in
    # both the start and the target (F - T of order 1e-6): whole pixel contributions flip sign
    # between float32 and float64, so the parameters are held only to Adam's step size (each
    # step moves a parameter by at most about lr)
    for k in names:
        got = vf.params[k].cpu().numpy().astype(np.float64)
        diff = np.abs(got - ref_p[k].astype(np.float64)).ravel()
        assert diff.max() <= 2 * steps * lr + 1e-6, k
