"""Per-stage fractions of roofline reported by bench.py (host arithmetic only).

The bench divides each stage's algorithmic work per step (bytes per moonlet
for the memory-bound stages, FLOPs per counted unit for the arithmetic ones)
by the stage's measured time and by the peak; these tests feed it stage
times and counters like those of the 1e5-moonlet bench disk and check the
arithmetic and the shape of the result.
"""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

STAGES = {"sort": 0.0948, "build": 0.0893, "climb": 0.1651, "walk": 0.1361, "m2l": 0.0519, "descend": 0.1412,
          "eval": 0.0315, "collide": 0.3833, "kdk": 0.0262, "near": 0.1912}


def test_stage_rooflines_arithmetic():
    n, m2l, inter, tests = 100_000, 137_116, 57_122_097, 22_217_601
    out = bench.stage_rooflines(STAGES, n, 6, m2l, inter, tests, 6777.6, 72.6)
    assert set(out) == set(STAGES)
    kdk = out["kdk"]
    assert kdk["bound"] == "hbm" and kdk["unit"] == "GB/s"
    gbs = 220.0 * n / (0.0262e-3) / 1e9
    assert kdk["achieved"] == pytest.approx(gbs, abs=0.05)
    assert kdk["frac"] == pytest.approx(gbs / 6777.6, abs=1e-4)
    near = out["near"]
    # the method's own counts (30 FLOPs per unordered direct pair, 3.2e3 per unordered M2L pair at p = 6,
    # 30 per collision candidate), whatever the kernels evaluate
    assert near["bound"] == "alu" and near["flops_per_step"] == 30.0 * inter
    assert near["achieved"] == pytest.approx(30.0 * inter / 0.1912e-3 / 1e12, abs=1e-3)
    assert out["m2l"]["flops_per_step"] == 3200.0 * m2l
    assert out["collide"]["flops_per_step"] == 30.0 * tests
    assert out["walk"] == {"bound": "latency", "ms": 0.1361}
    assert out["descend"]["bound"] == "latency"
    for v in out.values():
        if "frac" in v:
            assert 0.0 < v["frac"] < 1.0
    json.dumps(out)   # the bench prints it as JSON


def test_stage_rooflines_missing_stages_and_orders():
    out = bench.stage_rooflines({"near": 0.1, "m2l": 0.05, "walk": 0.0}, 1000, 5, 100, 1e6, 0, 6777.6, 80.5)
    assert set(out) == {"near"}          # no M2L FLOP count for p = 5, zero-time and absent stages skipped
    out = bench.stage_rooflines({}, 1000, 6, 0, 0, 0, 6777.6, 80.5)
    assert out == {}


def test_measured_hbm_bandwidth_or_fallback(tmp_path, monkeypatch):
    assert bench.measured_hbm_gbs() > 1000.0
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm_gbs() == 6800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.5}))
    assert bench.measured_hbm_gbs() == 7000.5


def test_near_roofline_counts_unordered_pairs():
    t = {"stage": {"near": 0.2}, "prof": {"p2p_interactions": 5e7, "m2l": 0, "col_tests": 0}}
    r = bench.near_roofline(t, 70.0, "mixed", None)
    assert r["flops_per_launch"] == 30.0 * 5e7
    assert r["achieved"] == pytest.approx(30.0 * 5e7 / 0.2e-3 / 1e12, abs=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / 70.0, abs=1e-4) and r["traffic"] is None


def test_host_cores_reports_nproc():
    h = bench.host_cores()
    assert h["nproc"] == os.cpu_count()


def test_collision_prefilter_against_the_fp32_peak(monkeypatch):
    # the pair test's prefilters run in FP32 in both precisions: its stage takes the FP32 peak even when the
    # near field and M2L (FP64 form) take the FP64 one
    monkeypatch.setattr(bench, "FP32_PEAK_TFLOPS", 78.0)
    out = bench.stage_rooflines(STAGES, 100_000, 6, 137_116, 57_122_097, 22_217_601, 6777.6, 1.25)
    assert out["collide"]["peak"] == 78.0 and out["near"]["peak"] == 1.25 and out["m2l"]["peak"] == 1.25
    assert out["collide"]["frac"] == pytest.approx(out["collide"]["achieved"] / 78.0, abs=1e-4)
