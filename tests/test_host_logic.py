"""Host-side logic that needs no GPU."""
import pytest


def test_memory_budget_selects_store_or_recompute():
    """A render keeps its workspace for the backward pass (store) when it fits
    the renderer's memory budget, and recomputes otherwise."""
    pytest.importorskip("torch")
    from paper_2004_07484_gb300 import Renderer
    assert Renderer(64, 64, 1000).keeps_workspace(1 << 40)
    r = Renderer(64, 64, 1000, memory_budget=1 << 20)
    assert r.keeps_workspace(1 << 20) and not r.keeps_workspace((1 << 20) + 1)
    assert not Renderer(64, 64, 1000, memory_budget=0).keeps_workspace(1)
