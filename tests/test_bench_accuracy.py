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
