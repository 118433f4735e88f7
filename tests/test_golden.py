"""The stored oracle record of the 1,000-sphere 64x64 scene (tests/golden/).

CPU: the oracle still reproduces it.  GPU: the CUDA path matches it (tile
lists and tracked hits exactly, images within 1e-4, gradient sums within
1e-3 of the sums of their magnitudes)."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "config0_oracle.json")
NAMES = ("pos", "rad", "opa", "feat", "cam", "bg")


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as f:
        return json.load(f)


def test_oracle_reproduces_the_record(orc, gold):
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_golden
    now = make_golden.golden()
    for key in ("pixels", "tracked", "n_hits", "tile_lengths", "tiles", "tile_lists"):
        assert now[key] == gold[key], key
    np.testing.assert_allclose(now["image"], gold["image"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(now["log_d"], gold["log_d"], rtol=1e-12)
    for n in NAMES:
        assert now["grad_sums"][n] == pytest.approx(gold["grad_sums"][n], rel=1e-10, abs=1e-12)
    np.testing.assert_allclose(now["grad_cam"], gold["grad_cam"], rtol=1e-10, atol=1e-12)


@pytest.mark.gpu
def test_cuda_path_matches_the_record(gold):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_07484_gb300 import build
    build.build()
    from paper_2004_07484_gb300 import scenes
    from helpers import gpu_backward, gpu_forward, gpu_tile_lists
    sc = scenes.config_scene(0)
    out = gpu_forward(sc)
    ranges, ids = gpu_tile_lists(out["frame"])
    assert [int(e - b) for b, e in ranges] == gold["tile_lengths"]
    for t, want in zip(gold["tiles"], gold["tile_lists"]):
        b, e = ranges[t]
        assert [int(x) for x in ids[b:e]] == want, t
    img = out["image"].cpu().numpy()
    ld = out["log_norm"].cpu().numpy()
    tr = out["tracked"].cpu().numpy()
    for (u, v), im, l, t in zip(gold["pixels"], gold["image"], gold["log_d"], gold["tracked"]):
        assert np.abs(img[v, u] - np.asarray(im)).max() <= 1e-4, (u, v)
        assert abs(ld[v, u] - l) <= 1e-4 * max(1.0, abs(l)), (u, v)
        assert [int(x) for x in tr[v, u]] == t, (u, v)
    G = scenes.grad_image(99, sc.height, sc.width, sc.n_channels)
    got = gpu_backward(out, G)
    for n in NAMES:
        assert abs(float(got[n].sum()) - gold["grad_sums"][n]) <= 1e-3 * max(gold["grad_abs_sums"][n], 1e-12), n
