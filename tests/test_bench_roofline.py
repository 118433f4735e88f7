"""The benchmark's roofline arithmetic, on the headline workload's counts
(1M spheres, 1024x1024, C = 16, K = 16: 1,268,938 pairs, 11,127,553 pixel
tests, 7,614,537 blended hits, 1,608,415 tracked hits), against the
per-stage byte and operation counts written out by hand."""
import pytest

bench = pytest.importorskip("bench")

L, TESTS, HITS, TRACKED, M, P, C, K = 1268938, 11127553, 7614537, 1608415, 1_000_000, 1024 * 1024, 16, 16


def test_stage_work_counts():
    w = bench.stage_work(L, TESTS, HITS, TRACKED, M, P, C)
    assert w["project"] == (68.0 * M, 0.0)
    assert w["depth sort"] == (16.0 * M, 0.0)
    assert w["binning"] == (16.0 * L, 30.0 * TESTS)
    # list entry + draw records 36 B and 64 B of features per pair; image 64 B, log D + hits 8 B per pixel
    assert w["forward render"][0] == 36 * L + 64 * L + 64 * P + 8 * P == 202_391_272
    assert w["forward render"][1] == 48.0 * HITS
    # dL/dF and F 128 B + threshold 16 B per pixel; records, features, gradients, camera chain per sphere
    assert w["backward"][0] == 144 * P + (32 + 64 + 20 + 64 + 28) * M
    assert w["backward"][1] == 124.0 * TRACKED


def test_step_roofline_is_the_sum_of_stage_bounds():
    pk = {"hbm_gbs": 6786.6}
    stage_mean = {"project": 0.040, "bin": 0.320, "render_fwd": 0.380, "render_bwd": 0.270}
    r = bench.step_roofline(L, TESTS, HITS, TRACKED, M, P, C, K, stage_mean, 1.0, pk, "measured", 77.7)
    bw, fp = 6786.6e9, 77.7e12
    w = bench.stage_work(L, TESTS, HITS, TRACKED, M, P, C)
    t_roof = sum(max(b / bw, f / fp) for b, f in w.values())
    assert r["step"]["t_roof_us"] == pytest.approx(t_roof * 1e6)
    assert r["step"]["frac"] == pytest.approx(t_roof / 1.0e-3)
    # the forward render against HBM: algorithmic bytes over the forward call's time
    assert r["achieved"] == pytest.approx(202_391_272 / 0.380e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6786.6)
    # binning is the depth sort and the pair stages together
    b = w["depth sort"][0] + w["binning"][0]
    assert r["per_call"]["pulsar_bin"]["hbm_frac"] == pytest.approx(b / 0.320e-3 / bw)


def test_kernels_per_step_matches_the_launch_list():
    # depths in [1, 20]: 26-bit offset keys, three 9-bit passes; 4,096 tiles:
    # 12-bit tile keys, two 6-bit passes (the launch list of one step shows 32 kernels)
    assert bench.kernels_per_step(1.0, 20.0, 4096, False) == 2 + (9 + 2 + 6 + 4) + 3 + 6 == 32
    assert bench.kernels_per_step(1.0, 20.0, 4096, True) == 33
    # 256 tiles: one 8-bit tile pass
    assert bench.kernels_per_step(1.0, 20.0, 256, False) == 32 - 3


def test_fit_kernels_per_step():
    # 4 views of 1920x1080: 32,640 tiles, 15-bit tile keys in two 8-bit passes; depths in [1, 20]
    assert bench.binning_kernels(1.0, 20.0, 4 * 120 * 68) == 9 + 2 + 6 + 4
    assert bench.fit_kernels_per_step(1.0, 20.0, 4 * 120 * 68) == 2 + 21 + 3 + 2 + 4 + 2 == 34
