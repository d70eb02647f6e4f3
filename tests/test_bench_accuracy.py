"""The bench's accuracy report: its direct summation (numpy, FP64) is the
oracle's direct summation, and its error statistic is the per-moonlet
relative vector error of the mutual acceleration (reading c10)."""
import numpy as np

import oracle
from paper_2310_20374_gb300 import diskgen


def test_direct_sample_errors_uses_the_direct_sum():
    import bench
    d = diskgen.make_disk(3000, 5)
    ref = oracle.direct_accel(d["pos"], d["mass"])
    e = bench.direct_sample_errors(d["pos"], d["mass"], ref, k=500)
    assert e["sample"] == 500 and e["p99"] < 1e-13
    # a known perturbation of every acceleration by 1e-6 of its length is reported as 1e-6
    bumped = ref + 1e-6 * np.linalg.norm(ref, axis=1)[:, None] * np.array([1.0, 0.0, 0.0])
    e = bench.direct_sample_errors(d["pos"], d["mass"], bumped, k=500)
    assert abs(e["median"] - 1e-6) < 1e-9 and abs(e["p99"] - 1e-6) < 1e-9


def test_eval_traffic_only_for_captured_workloads(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "EVAL_DRAM_BYTES_PER_LAUNCH", {(100_000, 6, 0.5): 5.5e6, (1_000_000, 4, 0.6): 5e7})
    assert bench.eval_traffic(100_000, 6, 0.5, "mixed", 64) == 5.5e6
    assert bench.eval_traffic(1_000_000, 4, 0.6, "mixed", 64) == 5e7
    # another precision, leaf size or workload has no capture behind it
    assert bench.eval_traffic(100_000, 6, 0.5, "fp64", 64) is None
    assert bench.eval_traffic(100_000, 6, 0.5, "mixed", 32) is None
    assert bench.eval_traffic(200_000, 6, 0.5, "mixed", 64) is None
