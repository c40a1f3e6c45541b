"""Host-side checks of bench.py's contract: the metric is the configured one,
every workload builds its synthetic input and names itself, and each DRAM
traffic figure the bench reports comes from a committed profile that gives it."""
import json
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_metric_is_the_configured_one():
    cfg = json.load(open(os.path.join(ROOT, "BASELINE.json")))
    assert bench.METRIC == cfg["metric"]


@pytest.mark.parametrize("name,n", [("tgv2d", 20), ("cavity", 20), ("tgv3d", 12), ("batch", 3), ("dambreak", 12)])
def test_workloads_build_and_name_themselves(name, n):
    d, wcfg = bench.make_workload(name, n, 0.0)
    insts = d if isinstance(d, list) else [d]
    assert wcfg["workload"] and wcfg["dims"] in (2, 3)
    for x in insts:
        nf = x["nf"]
        assert x["x"].shape[0] >= nf and x["v"].shape == (nf, wcfg["dims"]) and x["p"].shape == (nf,)


def test_default_run_is_one_gpu_and_short(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps <= 200 and a.impl == "ours"


def test_default_workload_is_the_batched_ensemble(monkeypatch):
    """The metric is quoted on the batched ensemble (64 Taylor-Green instances,
    FP32-compensated, one persistent launch per step): that is the default."""
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    d, wcfg = bench.make_workload(a.workload, a.n_side, a.re)
    assert a.workload == "batch" and wcfg["workload"] == "batch-64x-tgv2d" and len(d) == 64
    assert wcfg["particles"] == 1499340


def test_algorithmic_bytes_and_flops_follow_the_pair_cache_form():
    """Per particle-iteration: own state (52 / 72 B on the compensated path, 88 /
    120 B in FP64) plus one cache entry per pair (16 / 20 B, 28 / 36 B); FP64
    flops 8 dim + 3 per particle and 8 dim + 9 per pair."""
    assert bench.STATE_BYTES[(2, True)] + 27.3 * bench.PAIR_BYTES[(2, True)] == pytest.approx(488.8)
    assert bench.STATE_BYTES[(3, True)] + 112 * bench.PAIR_BYTES[(3, True)] == pytest.approx(2312)
    assert bench.fp64_flops(2) == (19.0, 25.0) and bench.fp64_flops(3) == (27.0, 33.0)


def test_algorithmic_bytes_without_the_cache():
    """The uncached form reads the particle's position at r^0 (16 B cell offset
    on the compensated path, dim doubles in FP64) and one 4-byte list entry per
    pair instead of a cache entry; the cached form's figure is unchanged."""
    f = bench.loop_bytes_per_particle_iteration
    assert f(2, True, 2, 27.3) == pytest.approx(52 + 16 + 4 * 27.3)
    assert f(3, True, 2, 112) == pytest.approx(72 + 16 + 4 * 112)
    assert f(3, False, 2, 112) == pytest.approx(120 + 24 + 4 * 112)
    assert f(2, True, 1, 27.3) == pytest.approx(488.8)


def test_loop_bytes_of_a_switched_step():
    """A step that started without the cache and switched to it after
    floor(kstar) iterations counts those iterations in the uncached form and
    the rest in the cached one, instance by instance."""
    f = bench.loop_launch_bytes
    a = bench.loop_bytes_per_particle_iteration(2, True, 2, 27.0)
    b = bench.loop_bytes_per_particle_iteration(2, True, 1, 27.0)
    assert f(2, True, 1, 27.0, [100, 50], [4, 9], 3.4) == pytest.approx(100 * 4 * b + 50 * 9 * b)
    assert f(2, True, 2, 27.0, [100, 50], [2, 3], 3.4) == pytest.approx(100 * 2 * a + 50 * 3 * a)
    assert f(2, True, 3, 27.0, [100, 50], [2, 9], 3.4) == pytest.approx(100 * 2 * a + 50 * (3 * a + 6 * b))


def test_traffic_figures_come_from_committed_profiles():
    """Every DRAM traffic figure bench.py uses comes from a committed profile
    summary that states the captured launch's DRAM bytes and its algorithmic
    bytes, the two numbers the line's traffic is scaled by."""
    for (workload, dim, lanes, stages, form), (byts, alg, src) in bench.NCU_TRAFFIC.items():
        assert form in (1, 2)
        path = os.path.join(ROOT, src)
        assert os.path.exists(path), path
        txt = open(path).read()
        assert "dram__bytes_read" in txt and "dram__bytes_write" in txt, path
        assert f"{byts / 1e9:.3f} GB" in txt, (path, byts)
        assert f"{alg / 1e9:.3f} GB" in txt, (path, alg)
        # (the form without the cache re-reads its lists and gathers from L2
        # across iterations, so its DRAM bytes may fall below the algorithmic ones)
        assert 0.1 < byts / alg < 3.0
