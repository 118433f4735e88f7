"""Batched rendering (several independent scenes in one launch sequence)
against the FP64 oracle, scene by scene, and against single-scene calls.

Bars as for single scenes: per-tile lists and tracked hits bit-exact, images
within 1e-4 max-abs, gradients within the 1e-3 relative rule.
"""
import numpy as np
import pytest

from paper_2004_07484_gb300 import scenes as S
from helpers import GRAD_NAMES, assert_grads_close, grad_error, settings_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_07484_gb300 import build
    build.build()


def empty_scene(width=48, height=32, n_channels=8, n_track=10):
    return S.Scene(np.zeros((0, 3), np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                   np.zeros((0, n_channels), np.float32), S.make_cam(),
                   np.linspace(0.1, 0.8, n_channels).astype(np.float32), width, height, 0.05, n_track,
                   name="empty")


def small_batch():
    """Uneven scenes (rotated cameras, mixed resolutions and gammas), one of
    them empty and one with every sphere behind the camera."""
    scs = S.batch_scenes(2024, n_scenes=6, m_range=(200, 4000), resolutions=(40, 64, 100))
    scs.insert(2, empty_scene())
    behind = S.batch_scenes(77, n_scenes=1, m_range=(300, 300), resolutions=(64,))[0]
    behind.cam = S.make_cam(t=behind.pos.astype(np.float64).mean(0) + np.array([0.0, 0.0, 30.0]))
    behind.name = "behind"
    scs.append(behind)
    return scs


def _inputs(scs):
    import torch
    return [tuple(torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).cuda()
                  for k in ("pos", "feat", "rad", "opa", "cam", "bg")) for sc in scs]


def run_batch(scs, store=True, capacities=None, segment=0, persistent=False):
    import torch
    from paper_2004_07484_gb300 import forward_batch
    inputs = _inputs(scs)
    sets = [settings_of(sc, store, segment=segment, persistent=persistent) for sc in scs]
    tracked = [torch.empty((sc.height, sc.width, sc.n_track), dtype=torch.int32, device="cuda") for sc in scs]
    n_hits = [torch.empty((sc.height, sc.width), dtype=torch.int32, device="cuda") for sc in scs]
    caps = capacities or [max(8 * sc.n_spheres, 1 << 14) for sc in scs]
    fr, images, log_norms = forward_batch(sets, inputs, caps, check_overflow=True, n_hits=n_hits,
                                          tracked=tracked)
    torch.cuda.synchronize()
    return dict(frame=fr, inputs=inputs, images=images, log_norms=log_norms, tracked=tracked, n_hits=n_hits)


def batch_backward(out, Gs, mask=None):
    import torch
    from paper_2004_07484_gb300 import _lib, backward_batch
    gs = [torch.from_numpy(np.ascontiguousarray(G.astype(np.float32))).cuda() for G in Gs]
    res = backward_batch(out["frame"], out["inputs"], out["images"], out["log_norms"], gs,
                         _lib.GRAD_ALL if mask is None else mask)
    torch.cuda.synchronize()
    return [{k: (None if v is None else v.cpu().numpy().astype(np.float64)) for k, v in zip(GRAD_NAMES, r)}
            for r in res]


def batch_tile_lists(fr):
    import torch
    from paper_2004_07484_gb300 import _lib
    nt = sum(((s.width + 15) // 16) * ((s.height + 15) // 16) for s in fr.settings)
    ranges = torch.empty((nt, 2), dtype=torch.int32, device="cuda")
    ids = torch.empty((max(sum(fr.capacities()), 1),), dtype=torch.int32, device="cuda")
    _lib.read_tile_lists_batched(fr.params, fr.ws.data_ptr(), fr.ws_bytes, ranges.data_ptr(),
                                 ids.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return ranges.cpu().numpy(), ids.cpu().numpy()


@pytest.fixture(scope="module")
def batch(orc):
    scs = small_batch()
    return scs, run_batch(scs), [orc.render(sc) for sc in scs]


def test_batched_tile_lists_bit_exact(orc, batch):
    scs, out, _ = batch
    ranges, ids = batch_tile_lists(out["frame"])
    t0 = m0 = 0
    for sc in scs:
        off, oids = orc.tile_lists(sc, tile=16)
        nt = len(off) - 1
        for t in range(nt):
            b, e = ranges[t0 + t]
            got = ids[b:e] - m0 if e > b else ids[:0]
            want = oids[off[t]:off[t + 1]]
            assert np.array_equal(got, want), (sc.name, t, got[:8], want[:8])
        t0 += nt
        m0 += sc.n_spheres
    assert t0 == len(ranges)


def test_batched_forward_matches_oracle(batch):
    scs, out, refs = batch
    for sc, ref, img, ln, tr, nh in zip(scs, refs, out["images"], out["log_norms"], out["tracked"],
                                         out["n_hits"]):
        img = img.cpu().numpy().astype(np.float64)
        assert np.abs(img - ref.image).max() <= 1e-4, sc.name
        np.testing.assert_array_equal(tr.cpu().numpy(), ref.tracked, err_msg=sc.name)
        ld = ln.cpu().numpy().astype(np.float64)
        assert np.abs(ld - ref.log_d).max() <= 1e-4 * max(1.0, np.abs(ref.log_d).max()), sc.name
        assert np.all(nh.cpu().numpy() <= ref.n_hits), sc.name


@pytest.mark.parametrize("store", [True, False], ids=["store", "recompute"])
def test_batched_backward_matches_oracle(orc, batch, store):
    scs, out, _ = batch
    if not store:
        out = run_batch(scs, store=False)
    Gs = [S.grad_image(300 + k, sc.height, sc.width, sc.n_channels) for k, sc in enumerate(scs)]
    got = batch_backward(out, Gs)
    for sc, G, g in zip(scs, Gs, got):
        want = orc.render_backward(sc, G)
        if sc.n_spheres == 0:
            for n in ("cam", "bg"):
                assert grad_error(g[n], getattr(want, n))[0] <= 1e-3, (sc.name, n)
            continue
        assert_grads_close(g, want, scene=sc)


def test_batched_equals_single_scene_calls(batch):
    """Each scene of a batch renders as it does alone: identical tracked hits,
    images equal up to float rounding, gradients up to atomics order."""
    from helpers import gpu_backward, gpu_forward
    scs, out, _ = batch
    Gs = [S.grad_image(500 + k, sc.height, sc.width, sc.n_channels) for k, sc in enumerate(scs)]
    got = batch_backward(out, Gs)
    for k, sc in enumerate(scs):
        single = gpu_forward(sc)
        a = out["images"][k].cpu().numpy()
        b = single["image"].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-6, sc.name
        np.testing.assert_array_equal(out["tracked"][k].cpu().numpy(), single["tracked"].cpu().numpy())
        g1 = gpu_backward(single, Gs[k])
        for n in GRAD_NAMES:
            if g1[n].size:
                assert grad_error(got[k][n], g1[n])[0] <= 1e-5, (sc.name, n)


def test_batched_persistent_short_segments(orc, batch):
    """Persistent kernels and 32-entry segments over the whole batch: same
    tracked hits, oracle-parity images and gradients."""
    scs, _, refs = batch
    out = run_batch(scs, store=False, segment=32, persistent=True)
    for sc, ref, img, tr in zip(scs, refs, out["images"], out["tracked"]):
        assert np.abs(img.cpu().numpy() - ref.image).max() <= 1e-4, sc.name
        np.testing.assert_array_equal(tr.cpu().numpy(), ref.tracked, err_msg=sc.name)
    Gs = [S.grad_image(700 + k, sc.height, sc.width, sc.n_channels) for k, sc in enumerate(scs)]
    for sc, G, g in zip(scs, Gs, batch_backward(out, Gs)):
        if sc.n_spheres:
            assert_grads_close(g, orc.render_backward(sc, G), scene=sc)


def test_batched_overflow_is_detected_and_recovered(orc):
    scs = S.batch_scenes(91, n_scenes=3, m_range=(1000, 3000), resolutions=(64, 100))
    out = run_batch(scs, capacities=[16, 16, 16])
    assert sum(out["frame"].capacities()) > 48
    for sc, img in zip(scs, out["images"]):
        ref = orc.render(sc)
        assert np.abs(img.cpu().numpy() - ref.image).max() <= 1e-4, sc.name


def test_32_scene_batch_sampled(orc):
    """The 32-scene batch (1e3..5e5 spheres, 128..1024 pixels square, rotated
    cameras, gamma 1e-3..0.1, C = 8, n_track = 10) at sampled pixels of a few
    scenes, and gradient sums over every scene."""
    scs = S.batch_scenes(1003)
    out = run_batch(scs, capacities=[max(6 * sc.n_spheres, 1 << 14) for sc in scs])
    # every scene's tile lists bit-exact: the batch has tens of thousands of
    # tiles, so the tile-key sort takes two digit passes
    ranges, ids = batch_tile_lists(out["frame"])
    assert len(ranges) > 256
    t0 = m0 = 0
    for sc in scs:
        off, oids = orc.tile_lists(sc, tile=16)
        nt = len(off) - 1
        b, e = ranges[t0:t0 + nt, 0], ranges[t0:t0 + nt, 1]
        assert np.array_equal(e - b, np.diff(off)), sc.name
        nz = e > b
        got = np.concatenate([ids[x:y] for x, y in zip(b[nz], e[nz])]) - m0 if nz.any() else ids[:0]
        np.testing.assert_array_equal(got, oids, err_msg=sc.name)
        t0 += nt
        m0 += sc.n_spheres
    assert t0 == len(ranges)
    g = np.random.default_rng(3)
    picks = sorted(g.choice(len(scs), 4, replace=False))
    for k in picks:
        sc = scs[k]
        nh = out["n_hits"][k].cpu().numpy()
        busy = np.argwhere(nh > 0)
        pix = busy[g.choice(len(busy), min(60, len(busy)), replace=False)][:, ::-1] if len(busy) else \
            np.zeros((0, 2), np.int64)
        pix = np.concatenate([pix, np.stack([g.integers(0, sc.width, 20), g.integers(0, sc.height, 20)], 1)])
        ref = orc.render_pixels(sc, pix)
        img = out["images"][k].cpu().numpy()[pix[:, 1], pix[:, 0]]
        assert np.abs(img - ref.image).max() <= 1e-4, sc.name
        tr = out["tracked"][k].cpu().numpy()[pix[:, 1], pix[:, 0]]
        np.testing.assert_array_equal(tr, ref.tracked, err_msg=sc.name)
    Gs = [np.ones((sc.height, sc.width, sc.n_channels)) for sc in scs]
    got = batch_backward(out, Gs)
    for sc, gr in zip(scs, got):
        # with G = 1 everywhere the loss is sum(F) = sum over pixels of
        # (sum_i w_i sum_c f_ic + w_B sum_c bg_c), so dL/dbg_c = sum_pixels w_B
        # equals the same for every channel, and dL/df_ic is the same for all c
        assert np.allclose(gr["bg"], gr["bg"][0], rtol=1e-5, atol=1e-6), sc.name
        f = gr["feat"]
        assert np.allclose(f, f[:, :1], rtol=1e-5, atol=1e-6 * max(1.0, np.abs(f).max())), sc.name
        assert np.all(np.isfinite(gr["pos"])) and np.all(np.isfinite(gr["cam"])), sc.name


def test_autotune_and_graph_replay(orc):
    """The autotuner's choice is one of its candidates with capacities that hold
    every scene's pairs, and a CUDA-graph capture of the tuned batched step
    replays to the oracle's images and to the uncaptured gradients."""
    import torch
    from paper_2004_07484_gb300 import autotune, backward_batch, forward_batch
    scs = S.batch_scenes(4242, n_scenes=5, m_range=(500, 5000), resolutions=(64, 100))
    inputs = _inputs(scs)
    sets = [settings_of(sc) for sc in scs]
    Gs = [torch.from_numpy(S.grad_image(900 + k, sc.height, sc.width, sc.n_channels).astype(np.float32)).cuda()
          for k, sc in enumerate(scs)]
    choice = autotune.tune(sets, inputs, Gs, reps=1, use_cache=False)
    assert choice.segment in autotune.SEGMENTS and choice.persistent in autotune.FORMS
    assert len(choice.ms) == len(autotune.SEGMENTS) * len(autotune.FORMS)
    pairs = autotune.pairs_per_scene(sets, inputs)
    assert all(c >= p for c, p in zip(choice.capacities, pairs))
    tuned = autotune.apply(sets, choice)

    def step():
        fr, images, log_norms = forward_batch(tuned, inputs, choice.capacities, check_overflow=False)
        return images, backward_batch(fr, inputs, images, log_norms, Gs)

    eager_images, eager_grads = step()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        g_images, g_grads = step()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for k, sc in enumerate(scs):
        ref = orc.render(sc)
        assert np.abs(g_images[k].cpu().numpy() - ref.image).max() <= 1e-4, sc.name
        for a, b in zip(g_grads[k], eager_grads[k]):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            assert np.abs(a - b).max() <= 1e-5 * max(1.0, np.abs(b).max()), sc.name


def test_one_call_batched_forward_matches_the_three_calls(batch):
    import torch
    from paper_2004_07484_gb300 import _lib
    from paper_2004_07484_gb300.renderer import BatchFrame, _scene_array
    scs, out, _ = batch
    fr = BatchFrame(out["frame"].settings, [sc.n_spheres for sc in scs], out["frame"].capacities(), "cuda")
    outs = (_lib.FwdOut * len(scs))()
    imgs, lns = [], []
    for k, sc in enumerate(scs):
        imgs.append(torch.empty((sc.height, sc.width, sc.n_channels), device="cuda"))
        lns.append(torch.empty((sc.height, sc.width), device="cuda"))
        outs[k] = _lib.FwdOut(imgs[k].data_ptr(), lns[k].data_ptr(), None, None, None)
    _lib.render_batched(fr.params, _scene_array(out["inputs"]), fr.ws.data_ptr(), fr.ws_bytes, outs,
                        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for k, sc in enumerate(scs):
        assert np.abs(imgs[k].cpu().numpy() - out["images"][k].cpu().numpy()).max() <= 1e-6, sc.name


def test_batched_paper_stop_per_scene_thresholds(orc):
    """The paper's early termination in a batch: two scenes with their own
    thresholds (1 % and 2 %) and an empty one, 32-entry segments walked in
    order by persistent kernels; tracked hits bit-exact, images and gradients
    at parity with the oracle's truncated renders (every decision of the two
    scenes lies at least 2e-3 from its threshold)."""
    scs = []
    for seed, n, W, H, rad, tau in [(86, 600, 48, 40, (0.1, 0.5), 0.01), (88, 300, 32, 32, (0.2, 0.8), 0.02)]:
        sc = S.uniform_cloud(seed, n, W, H, gamma=0.05, n_track=5, rad=rad, z=(2.0, 18.0))
        sc.paper_stop, sc.min_contrib = True, tau
        assert orc.paper_stop_margin(sc).min() >= 2e-3
        scs.append(sc)
    empty = empty_scene(n_channels=3, n_track=5)
    empty.gamma, empty.paper_stop = 0.05, True
    scs.append(empty)
    out = run_batch(scs, segment=32, persistent=True)
    Gs = [S.grad_image(310 + k, sc.height, sc.width, sc.n_channels) for k, sc in enumerate(scs)]
    got = batch_backward(out, Gs)
    for k, sc in enumerate(scs):
        ref = orc.render(sc)
        np.testing.assert_array_equal(out["tracked"][k].cpu().numpy(), ref.tracked)
        assert np.abs(out["images"][k].cpu().numpy() - ref.image).max() <= 1e-4
        want = orc.render_backward(sc, Gs[k])
        if sc.n_spheres == 0:
            assert grad_error(got[k]["bg"], want.bg)[0] <= 1e-3
            continue
        assert_grads_close(got[k], want, scene=sc)
