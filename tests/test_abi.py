"""The C-ABI library loads and exports every entry point its header declares.

CPU only: no CUDA work is enqueued.  Host-side argument validation is
exercised because it returns before anything touches the device.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2004_07484_gb300 import build
    build.build()
    from paper_2004_07484_gb300 import _lib
    return _lib


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(pulsar_[a-z_0-9]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert {"pulsar_project", "pulsar_bin", "pulsar_render_fwd", "pulsar_render_bwd"} <= names
    L = ctypes.CDLL(lib.LIB_PATH)
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(lib.EXPORTED) <= names


def test_status_strings(lib):
    for s in range(6):
        assert lib.status_string(s)


def _params(lib, **kw):
    p = dict(width=64, height=48, n_spheres=10, n_channels=3, n_track=5, tile=16, list_capacity=1000,
             gamma=0.1, eps=1e-5, znear=1.0, zfar=20.0, flags=lib.FLAG_STORE_HITS)
    p.update(kw)
    return lib.Params(**p)


def test_workspace_size_validates_settings(lib):
    assert lib.lib().pulsar_workspace_size(ctypes.byref(_params(lib))) > 0
    bad = [dict(width=0), dict(height=70000), dict(n_channels=0), dict(n_track=0), dict(gamma=2.0),
           dict(gamma=1e-7), dict(znear=0.0), dict(zfar=0.5), dict(list_capacity=-1),
           dict(flags=1 << 8), dict(n_spheres=-1), dict(min_contrib=-0.01), dict(min_contrib=1.0),
           dict(min_contrib=float("nan"))]
    for b in bad:
        assert lib.lib().pulsar_workspace_size(ctypes.byref(_params(lib, **b))) == 0, b
    unsupported = [dict(n_channels=33), dict(n_track=33), dict(tile=8)]
    for b in unsupported:
        assert lib.lib().pulsar_workspace_size(ctypes.byref(_params(lib, **b))) == 0, b


def test_workspace_grows_with_capacity_channels_and_track(lib):
    a = lib.lib().pulsar_workspace_size(ctypes.byref(_params(lib)))
    b = lib.lib().pulsar_workspace_size(ctypes.byref(_params(lib, list_capacity=100000)))
    c = lib.lib().pulsar_workspace_size(ctypes.byref(_params(lib, flags=0)))
    d = lib.lib().pulsar_workspace_size(ctypes.byref(_params(lib, n_channels=16, n_track=16)))
    assert b > a and d > a
    assert c == a   # the per-pixel backward data is kept in both modes


def test_entry_points_reject_bad_arguments_before_any_launch(lib):
    L = lib.lib()
    p = _params(lib)
    scene = lib.SceneArgs(None, None, None, None, None, None)
    # null / misaligned workspace, missing scene pointers, short workspace
    assert L.pulsar_project(ctypes.byref(p), ctypes.byref(scene), None, 0, None) == lib.ERR_INVALID_ARG
    assert L.pulsar_project(ctypes.byref(p), ctypes.byref(scene), 256, 1 << 30, None) == lib.ERR_INVALID_ARG
    assert L.pulsar_project(ctypes.byref(p), ctypes.byref(scene), 257, 1 << 30, None) == lib.ERR_INVALID_ARG
    assert L.pulsar_bin(ctypes.byref(p), 256, 16, None) == lib.ERR_CAPACITY
    bad = _params(lib, gamma=5.0)
    assert L.pulsar_bin(ctypes.byref(bad), 256, 1 << 30, None) == lib.ERR_INVALID_ARG
    assert L.pulsar_read_status(None, 0, None, None) == lib.ERR_INVALID_ARG


def _batch(lib, plist):
    return (lib.Params * len(plist))(*plist)


def test_batched_workspace_size_validates_the_batch(lib):
    L = lib.lib()
    one = _params(lib)
    assert L.pulsar_workspace_size_batched(1, _batch(lib, [one])) == L.pulsar_workspace_size(ctypes.byref(one))
    two = _batch(lib, [_params(lib), _params(lib, width=300, height=20, n_spheres=500, gamma=0.01)])
    n2 = L.pulsar_workspace_size_batched(2, two)
    assert n2 > L.pulsar_workspace_size(ctypes.byref(two[1]))
    # scenes must share channels, n_track and flags; the count is 1..MAX_SCENES
    for kw in (dict(n_channels=4), dict(n_track=6), dict(flags=0)):
        assert L.pulsar_workspace_size_batched(2, _batch(lib, [_params(lib), _params(lib, **kw)])) == 0, kw
    assert L.pulsar_workspace_size_batched(0, _batch(lib, [one])) == 0
    many = [_params(lib) for _ in range(lib.MAX_SCENES + 1)]
    assert L.pulsar_workspace_size_batched(lib.MAX_SCENES, _batch(lib, many[:-1])) > 0
    assert L.pulsar_workspace_size_batched(lib.MAX_SCENES + 1, _batch(lib, many)) == 0
    # an invalid scene anywhere in the batch invalidates it
    assert L.pulsar_workspace_size_batched(2, _batch(lib, [_params(lib), _params(lib, gamma=3.0)])) == 0


def test_batched_entry_points_reject_bad_arguments_on_the_host(lib):
    L = lib.lib()
    ps = _batch(lib, [_params(lib), _params(lib, n_spheres=0)])
    ss = (lib.SceneArgs * 2)()
    # no workspace
    assert L.pulsar_project_batched(2, ps, ss, None, 0, None) == lib.ERR_INVALID_ARG
    assert L.pulsar_bin_batched(2, ps, None, 0, None) == lib.ERR_INVALID_ARG
    # a misaligned or short workspace
    assert L.pulsar_bin_batched(2, ps, 16, 1 << 30, None) == lib.ERR_INVALID_ARG
    assert L.pulsar_bin_batched(2, ps, 256, 16, None) == lib.ERR_CAPACITY
    # mixed channel counts
    bad = _batch(lib, [_params(lib), _params(lib, n_channels=5)])
    assert L.pulsar_bin_batched(2, bad, 256, 1 << 40, None) == lib.ERR_INVALID_ARG
    # missing scene pointers (checked before any launch)
    n = L.pulsar_workspace_size_batched(2, ps)
    assert L.pulsar_project_batched(2, ps, ss, 256, n, None) == lib.ERR_INVALID_ARG
    outs = (lib.FwdOut * 2)()
    assert L.pulsar_render_fwd_batched(2, ps, ss, 256, n, outs, None) == lib.ERR_INVALID_ARG
    ios = (lib.BwdIO * 2)()
    assert L.pulsar_render_bwd_batched(2, ps, ss, 256, n, ios, lib.GRAD_ALL, None) == lib.ERR_INVALID_ARG


def test_fit_entry_points_reject_bad_arguments_on_the_host(lib):
    L = lib.lib()
    # image loss: unknown kind, negative size, missing buffers
    assert L.pulsar_image_loss(7, 256, 256, 4, 1.0, None, None, 256, None) == lib.ERR_INVALID_ARG
    assert L.pulsar_image_loss(lib.LOSS_L2, 256, 256, -1, 1.0, None, None, 256, None) == lib.ERR_INVALID_ARG
    assert L.pulsar_image_loss(lib.LOSS_L1, None, 256, 4, 1.0, None, None, 256, None) == lib.ERR_INVALID_ARG
    assert L.pulsar_image_loss(lib.LOSS_L1, 256, 256, 4, 1.0, None, None, None, None) == lib.ERR_INVALID_ARG
    # Adam: tensor count, hyper-parameters, tensor descriptors
    inf = float("inf")
    good = lib.AdamTensor(256, 512, 768, 1024, 10, -inf, inf)
    ts = (lib.AdamTensor * 1)(good)
    hp = lib.AdamHyper(1e-3, 0.9, 0.999, 1e-8, 1)
    assert L.pulsar_adam_step(0, ts, ctypes.byref(hp), 256, None) == lib.ERR_INVALID_ARG
    assert L.pulsar_adam_step(lib.ADAM_MAX_TENSORS + 1, ts, ctypes.byref(hp), 256, None) == lib.ERR_INVALID_ARG
    assert L.pulsar_adam_step(1, ts, ctypes.byref(hp), None, None) == lib.ERR_INVALID_ARG
    for bad in (lib.AdamHyper(-1.0, 0.9, 0.999, 1e-8, 1), lib.AdamHyper(1e-3, 1.0, 0.999, 1e-8, 1),
                lib.AdamHyper(1e-3, 0.9, -0.1, 1e-8, 1), lib.AdamHyper(1e-3, 0.9, 0.999, -1.0, 1),
                lib.AdamHyper(float("nan"), 0.9, 0.999, 1e-8, 1)):
        assert L.pulsar_adam_step(1, ts, ctypes.byref(bad), 256, None) == lib.ERR_INVALID_ARG
    for bad in (lib.AdamTensor(256, 512, 768, 1024, -1, -inf, inf),
                lib.AdamTensor(256, 512, 768, 1024, 10, 1.0, 0.0),
                lib.AdamTensor(256, None, 768, 1024, 10, -inf, inf),
                lib.AdamTensor(256, 512, 768, 1024, 10, float("nan"), inf)):
        assert L.pulsar_adam_step(1, (lib.AdamTensor * 1)(bad), ctypes.byref(hp), 256, None) == lib.ERR_INVALID_ARG
    # the accumulate flag is a valid setting
    assert L.pulsar_workspace_size(ctypes.byref(_params(lib, flags=lib.FLAG_ACCUMULATE))) > 0
    assert L.pulsar_workspace_size(ctypes.byref(_params(lib, flags=lib.FLAG_PAPER_GRADIENTS))) > \
        L.pulsar_workspace_size(ctypes.byref(_params(lib)))   # per-sphere sums of the paper mode
    assert L.pulsar_workspace_size(ctypes.byref(_params(lib, flags=lib.FLAG_ORTHOGRAPHIC))) > 0
    # the paper's early termination keeps the workspace layout
    assert L.pulsar_workspace_size(ctypes.byref(_params(lib, flags=lib.FLAG_PAPER_STOP))) == \
        L.pulsar_workspace_size(ctypes.byref(_params(lib)))
    assert L.pulsar_workspace_size(ctypes.byref(_params(lib, flags=1 << 8))) == 0
