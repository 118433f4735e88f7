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
           dict(flags=1 << 7), dict(n_spheres=-1)]
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
