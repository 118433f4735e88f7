"""The allocation-free forward render (pulsar_render_fwd_static).

Some callers cannot allocate device memory when they render (another
component owns the device memory, or the caller must avoid the synchronising
cudaFree).  For them the library renders into a fixed device array of its own
instead of a caller-provided workspace.  This checks, through the C ABI, that
it produces the same image and log-normaliser as pulsar_render_fwd with a
caller workspace, on two calls in a row (the second call runs on whatever the
first one left in the array), and that oversized requests are refused.

The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_2004_07484_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_07484_gb300 import build
    build.build()


def _render_both(sc):
    import torch
    from paper_2004_07484_gb300 import _lib
    from paper_2004_07484_gb300.renderer import RenderSettings, scene_args
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).cuda()
           for k in ("pos", "rad", "opa", "feat", "cam", "bg")}
    n_tiles = ((sc.width + 15) // 16) * ((sc.height + 15) // 16)
    s = RenderSettings(sc.width, sc.height, sc.n_channels, sc.n_track, sc.gamma, sc.eps, sc.znear,
                       sc.zfar)
    p = s.params(sc.n_spheres, sc.n_spheres * n_tiles)   # cannot overflow
    assert _lib.workspace_size(p) <= _lib.STATIC_WORKSPACE_BYTES
    sa = scene_args(dev["pos"], dev["feat"], dev["rad"], dev["opa"], dev["cam"], dev["bg"])
    stream = torch.cuda.current_stream().cuda_stream
    H, W, C = sc.height, sc.width, sc.n_channels
    ws = torch.empty(_lib.workspace_size(p), dtype=torch.uint8, device="cuda")
    img_ref = torch.empty((H, W, C), dtype=torch.float32, device="cuda")
    ld_ref = torch.empty((H, W), dtype=torch.float32, device="cuda")
    _lib.project(p, sa, ws.data_ptr(), ws.numel(), stream)
    _lib.bin(p, ws.data_ptr(), ws.numel(), stream)
    _lib.render_fwd(p, sa, ws.data_ptr(), ws.numel(), img_ref.data_ptr(), ld_ref.data_ptr(), None,
                    None, None, stream)
    outs = []
    for _ in range(2):
        img = torch.full((H, W, C), float("nan"), dtype=torch.float32, device="cuda")
        ld = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
        _lib.render_fwd_static(p, sa, img.data_ptr(), ld.data_ptr(), stream)
        outs.append((img, ld))
    torch.cuda.synchronize()
    return img_ref.cpu().numpy(), ld_ref.cpu().numpy(), [(a.cpu().numpy(), b.cpu().numpy()) for a, b in outs]


@pytest.mark.parametrize("make", [lambda: S.config_scene(0),
                                  lambda: S.gaussian_mixture(77, 6000, 96, 80, n_channels=4, gamma=0.05,
                                                             n_track=8, mean_xy=(-0.7, 0.7))],
                         ids=["1000_spheres_64x64", "6000_spheres_96x80"])
def test_static_workspace_matches_caller_workspace(make):
    img_ref, ld_ref, outs = _render_both(make())
    for img, ld in outs:
        assert np.isfinite(img).all() and np.isfinite(ld).all()
        assert np.abs(img - img_ref).max() <= 1e-4
        assert np.abs(ld - ld_ref).max() <= 1e-4 * max(1.0, np.abs(ld_ref).max())


def test_static_workspace_refuses_oversized_requests():
    import torch
    from paper_2004_07484_gb300 import _lib
    from paper_2004_07484_gb300.renderer import RenderSettings, scene_args
    s = RenderSettings(1024, 1024, 16, 16)
    p = s.params(1_000_000, 4_000_000)
    assert _lib.workspace_size(p) > _lib.STATIC_WORKSPACE_BYTES
    x = torch.zeros(16, device="cuda")
    sa = scene_args(x, x, x, x, x, x)
    with pytest.raises(_lib.PulsarError) as err:
        _lib.render_fwd_static(p, sa, x.data_ptr(), x.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert err.value.status == _lib.ERR_CAPACITY
