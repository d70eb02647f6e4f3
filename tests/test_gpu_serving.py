"""Serving on a GB300: requests arriving over time through the real batch.

Disks of two expansion orders arrive while others are being integrated; the
loop admits each at the next tick, so the work of several disks overlaps in
one ncorp_batch_run.  Every disk's final state must equal that of the same
disk integrated alone with ncorp_step (FP64: to the rounding of sums taken
in another order), whatever it shared the GPU with.
"""
import numpy as np
import pytest
import torch

from paper_2310_20374_gb300 import diskgen, ncorp, serving

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def config():
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_FP64
    cfg.leaf_size = 24
    return cfg


def alone(d, p, theta, dt, steps):
    n = len(d["pos"])
    ctx = ncorp.ncorp_init(config(), n, 0, torch.cuda.current_stream().cuda_stream)
    pos, vel = d["pos"].copy(), d["vel"].copy()
    try:
        for _ in range(steps):
            ncorp.ncorp_step(ctx, pos, vel, d["mass"], d["radius"], n, p, theta, dt)
    finally:
        ncorp.ncorp_free(ctx)
    return pos, vel


def test_each_result_is_the_same_alone_and_in_the_mix():
    theta, dt, steps = 0.5, 2e-2, 12
    plan = [(0.0, 2500, 3), (0.0, 1500, 4), (0.03, 4000, 3), (0.06, 2000, 4), (0.1, 3000, 3), (0.2, 1800, 4)]
    reqs = []
    for k, (t, n, p) in enumerate(plan):
        dense = k % 2 == 0
        d = (diskgen.make_disk(n, 900 + k, a_lo=2.0, a_hi=2.5, r_lo=2e-2, r_hi=5e-2, sigma_e=0.1, sigma_i=0.05)
             if dense else diskgen.make_disk(n, 900 + k))
        reqs.append(serving.Request(arrival=t, n=n, p=p, steps=steps, disk=d))
    results = {}

    def on_done(r):
        results[id(r)] = (np.zeros((r.n, 3)), np.zeros((r.n, 3)))
        return results[id(r)]

    b = ncorp.ncorp_batch_create(config(), 0, torch.cuda.current_stream().cuda_stream)
    try:
        st = serving.serve(serving.BatchBackend(ncorp, b, theta, dt), reqs, tick_steps=5, on_done=on_done)
    finally:
        ncorp.ncorp_batch_free(b)
    assert st["served"] == len(reqs) and st["concurrent_disks_max"] >= 2
    for r in reqs:
        xs, vs = alone(r.disk, r.p, theta, dt, steps)
        x, v = results[id(r)]
        np.testing.assert_allclose(x, xs, rtol=0, atol=1e-12 * np.abs(xs).max())
        np.testing.assert_allclose(v, vs, rtol=0, atol=1e-11 * np.abs(vs).max())
