"""The allocation-free forward render (pulsar_render_fwd_static).

Some callers cannot allocate device memory when they render (another
component owns the device memory, or the caller must avoid the synchronising
cudaFree).  For them the library renders into a fixed device array of its own
instead of a caller-provided workspace.  This checks, through the C ABI, that
it produces the same image and log-normaliser as pulsar_render_fwd with a
caller workspace, on two calls in a row (the second call runs on whatever the
first one left in the array), also when a larger scene is followed by a
smaller one with other settings; that a pair-list overflow is reported by
pulsar_static_read_status; and that it refuses what pulsar_render_fwd refuses,
with the same status codes, plus requests larger than its array.

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


def _inputs(sc):
    import torch
    from paper_2004_07484_gb300.renderer import scene_args
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).cuda()
           for k in ("pos", "rad", "opa", "feat", "cam", "bg")}
    return dev, scene_args(dev["pos"], dev["feat"], dev["rad"], dev["opa"], dev["cam"], dev["bg"])


def _params(sc, capacity=None, **flags):
    from paper_2004_07484_gb300 import _lib
    from paper_2004_07484_gb300.renderer import RenderSettings
    n_tiles = ((sc.width + 15) // 16) * ((sc.height + 15) // 16)
    s = RenderSettings(sc.width, sc.height, sc.n_channels, sc.n_track, sc.gamma, sc.eps, sc.znear,
                       sc.zfar, **flags)
    p = s.params(sc.n_spheres, sc.n_spheres * n_tiles if capacity is None else capacity)  # None: cannot overflow
    assert _lib.workspace_size(p) <= _lib.STATIC_WORKSPACE_BYTES
    return p


def _caller_workspace(sc, p):
    """The image and log-normaliser of pulsar_render_fwd with a caller workspace."""
    import torch
    from paper_2004_07484_gb300 import _lib
    dev, sa = _inputs(sc)
    stream = torch.cuda.current_stream().cuda_stream
    H, W, C = sc.height, sc.width, sc.n_channels
    ws = torch.empty(_lib.workspace_size(p), dtype=torch.uint8, device="cuda")
    img = torch.empty((H, W, C), dtype=torch.float32, device="cuda")
    ld = torch.empty((H, W), dtype=torch.float32, device="cuda")
    _lib.project(p, sa, ws.data_ptr(), ws.numel(), stream)
    _lib.bin(p, ws.data_ptr(), ws.numel(), stream)
    _lib.render_fwd(p, sa, ws.data_ptr(), ws.numel(), img.data_ptr(), ld.data_ptr(), None, None, None,
                    stream)
    torch.cuda.synchronize()
    return img.cpu().numpy(), ld.cpu().numpy()


def _static(sc, p):
    """The same through pulsar_render_fwd_static, into NaN-filled outputs."""
    import torch
    from paper_2004_07484_gb300 import _lib
    dev, sa = _inputs(sc)
    H, W, C = sc.height, sc.width, sc.n_channels
    img = torch.full((H, W, C), float("nan"), dtype=torch.float32, device="cuda")
    ld = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
    _lib.render_fwd_static(p, sa, img.data_ptr(), ld.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return img.cpu().numpy(), ld.cpu().numpy()


def _assert_same(got, want):
    img, ld = got
    img_ref, ld_ref = want
    assert np.isfinite(img).all() and np.isfinite(ld).all()
    assert np.abs(img - img_ref).max() <= 1e-4
    assert np.abs(ld - ld_ref).max() <= 1e-4 * max(1.0, np.abs(ld_ref).max())


def _large():
    return S.gaussian_mixture(77, 6000, 96, 80, n_channels=4, gamma=0.05, n_track=8, mean_xy=(-0.7, 0.7))


@pytest.mark.parametrize("make", [lambda: S.config_scene(0), _large],
                         ids=["1000_spheres_64x64", "6000_spheres_96x80"])
def test_static_workspace_matches_caller_workspace(make):
    sc = make()
    p = _params(sc)
    want = _caller_workspace(sc, p)
    for _ in range(2):
        _assert_same(_static(sc, p), want)


@pytest.mark.parametrize("flags", [{}, {"store_hits": True}, {"paper_stop": True, "store_hits": True}],
                         ids=["plain", "store_hits", "paper_stop"])
def test_static_workspace_larger_then_smaller_scene(flags):
    """A larger scene (more spheres, tiles and pairs, more channels) fills the
    array first; the smaller scene rendered next must not read any of it."""
    from paper_2004_07484_gb300 import _lib
    import torch
    big, small = _large(), S.config_scene(0)
    p_big, p_small = _params(big, **flags), _params(small, **flags)
    _assert_same(_static(big, p_big), _caller_workspace(big, p_big))
    _assert_same(_static(small, p_small), _caller_workspace(small, p_small))
    st, _ = _lib.static_read_status(torch.cuda.current_stream().cuda_stream)
    assert st == _lib.OK


def test_static_workspace_reports_overflow():
    """With a pair capacity below the scene's pair count the image is
    background only, and pulsar_static_read_status says so, with the count
    needed; a call with that capacity then renders the scene."""
    import torch
    from paper_2004_07484_gb300 import _lib
    sc = _large()
    stream = torch.cuda.current_stream().cuda_stream
    p = _params(sc, capacity=64)
    _static(sc, p)
    st, need = _lib.static_read_status(stream)
    assert st == _lib.ERR_CAPACITY and need > 64
    p2 = _params(sc, capacity=need)
    got = _static(sc, p2)
    st, need2 = _lib.static_read_status(stream)
    assert st == _lib.OK and need2 == need
    _assert_same(got, _caller_workspace(sc, p2))


def test_static_workspace_refuses_what_the_caller_workspace_refuses():
    import torch
    from paper_2004_07484_gb300 import _lib
    from paper_2004_07484_gb300.renderer import RenderSettings, scene_args
    x = torch.zeros(16, device="cuda")
    sa = scene_args(x, x, x, x, x, x)
    stream = torch.cuda.current_stream().cuda_stream
    # larger than the array
    p = RenderSettings(1024, 1024, 16, 16).params(1_000_000, 4_000_000)
    assert _lib.workspace_size(p) > _lib.STATIC_WORKSPACE_BYTES
    with pytest.raises(_lib.PulsarError) as err:
        _lib.render_fwd_static(p, sa, x.data_ptr(), x.data_ptr(), stream)
    assert err.value.status == _lib.ERR_CAPACITY
    # unsupported and invalid settings: the codes of pulsar_render_fwd
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    for bad, code in ((RenderSettings(64, 64, 40, 5).params(10, 100), _lib.ERR_UNSUPPORTED),
                      (RenderSettings(64, 64, 3, 5, gamma=2.0).params(10, 100), _lib.ERR_INVALID_ARG)):
        with pytest.raises(_lib.PulsarError) as e1:
            _lib.render_fwd(bad, sa, ws.data_ptr(), ws.numel(), x.data_ptr(), x.data_ptr(), None, None, None,
                            stream)
        with pytest.raises(_lib.PulsarError) as e2:
            _lib.render_fwd_static(bad, sa, x.data_ptr(), x.data_ptr(), stream)
        assert e1.value.status == e2.value.status == code
