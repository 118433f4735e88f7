"""The renderer inside a training graph: its 16-channel image feeds the conv
shading net of the 1M-sphere workload (16 -> 32 -> 32 -> 3, 3x3, ReLU, FP32),
the loss is the mean squared output, and loss.backward() runs through the
renderer's torch.autograd.Function.  The renderer's gradients must equal the
oracle's analytic gradients under the net's dL/dF (taken by autograd through
the net alone), in store mode and in recompute mode (memory budget below the
workspace: the backward pass rebuilds the lists and hit lists)."""
import numpy as np
import pytest

from paper_2004_07484_gb300 import scenes as S
from helpers import assert_grads_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_07484_gb300 import build
    build.build()


def _net(torch, C):
    torch.manual_seed(2)
    return torch.nn.Sequential(torch.nn.Conv2d(C, 32, 3, padding=1), torch.nn.ReLU(),
                               torch.nn.Conv2d(32, 32, 3, padding=1), torch.nn.ReLU(),
                               torch.nn.Conv2d(32, 3, 3, padding=1)).cuda().double()


@pytest.mark.parametrize("budget", [None, 0], ids=["store", "recompute"])
def test_shading_net_gradients_match_the_oracle(orc, budget):
    import torch
    from paper_2004_07484_gb300 import Renderer
    sc = S.ellipsoid_surfaces(1078, 12000, 72, 64, n_channels=16, gamma=1e-2, n_track=16,
                              centre_xy=(-0.6, 0.6), centre_z=(5.0, 8.0), axes=(0.3, 1.0))
    net = _net(torch, 16)
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).cuda().requires_grad_(True)
         for k in ("pos", "feat", "rad", "opa", "cam", "bg")}
    r = Renderer(sc.width, sc.height, sc.n_spheres, n_channels=16, n_track=16, gamma=sc.gamma, eps=sc.eps,
                 znear=sc.znear, zfar=sc.zfar, memory_budget=budget)
    img = r(t["pos"], t["feat"], t["rad"], t["cam"], opa=t["opa"], bg=t["bg"])
    assert r.last_mode == ("store" if budget is None else "recompute")
    y = net(img.double().permute(2, 0, 1).unsqueeze(0))
    (y * y).mean().backward()
    torch.cuda.synchronize()
    ref = orc.render(sc)
    assert np.abs(img.detach().cpu().numpy() - ref.image).max() <= 1e-4
    # dL/dF of the net at the oracle's image (FP64), the upstream gradient of the render
    x = torch.from_numpy(ref.image).cuda().requires_grad_(True)
    yy = net(x.permute(2, 0, 1).unsqueeze(0))
    (yy * yy).mean().backward()
    G = x.grad.cpu().numpy()
    want = orc.render_backward(sc, G)
    got = {k: t[k].grad.cpu().numpy().astype(np.float64) for k in ("pos", "rad", "opa", "feat", "cam", "bg")}
    assert_grads_close(got, want, scene=sc)


def test_store_and_recompute_agree_through_the_net():
    """Both modes give the same gradients (up to the order of float atomics)."""
    import torch
    from paper_2004_07484_gb300 import Renderer
    sc = S.ellipsoid_surfaces(1079, 20000, 96, 80, n_channels=16, gamma=1e-2, n_track=16,
                              centre_xy=(-0.6, 0.6), centre_z=(5.0, 8.0), axes=(0.3, 1.0))
    net = _net(torch, 16).float()
    grads = []
    for budget in (None, 0):
        t = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).cuda().requires_grad_(True)
             for k in ("pos", "feat", "rad", "opa", "cam", "bg")}
        r = Renderer(sc.width, sc.height, sc.n_spheres, n_channels=16, n_track=16, gamma=sc.gamma,
                     eps=sc.eps, znear=sc.znear, zfar=sc.zfar, memory_budget=budget)
        img = r(t["pos"], t["feat"], t["rad"], t["cam"], opa=t["opa"], bg=t["bg"])
        y = net(img.permute(2, 0, 1).unsqueeze(0))
        (y * y).mean().backward()
        grads.append({k: v.grad.cpu().numpy().astype(np.float64) for k, v in t.items()})
    for k in grads[0]:
        a, b = grads[0][k], grads[1][k]
        assert np.abs(a - b).max() <= 1e-5 * max(np.abs(a).max(), 1e-12), k
