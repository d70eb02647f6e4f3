"""The fused gravity + collision walk (ncorp_config.fused_walk), needs a GB300.

With the fused walk one traversal of each new tree takes the gravity
decisions and lists the leaf pairs of the next step's collision search,
walked with a bound on every moonlet's R + dt |v| at that step; the next step
checks the bounds and searches on its own when one is exceeded (always on the
first step, whose tree had no fused walk).  Gravity is the same walk as
without fusion, and the colliding pairs are the brute-force set either way:
steps with and without fusion give the same pairs (the search without fusion
is checked against brute force elsewhere) and the same states to the rounding
of order-dependent sums.
"""
import numpy as np
import pytest
import torch

from paper_2310_20374_gb300 import diskgen, ncorp

pytestmark = pytest.mark.gpu

STEPS = 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def run(d, fused, p, precision, graphs=True, dt=1e-3):
    n = len(d["pos"])
    cfg = ncorp.ncorp_config_default()
    cfg.precision = precision
    cfg.leaf_size = 32
    cfg.fused_walk = fused
    ctx = ncorp.ncorp_init(cfg, n, 0, torch.cuda.current_stream().cuda_stream)
    arrs = [torch.tensor(d[k], device="cuda") for k in ("pos", "vel", "mass", "radius")]
    out = []
    try:
        ncorp.ncorp_set_graphs(ctx, graphs)
        for _ in range(STEPS):
            x0, v0 = arrs[0].cpu().numpy(), arrs[1].cpu().numpy()
            ncorp.ncorp_step(ctx, *arrs, n, p, 0.5, dt)
            st = ncorp.ncorp_stats(ctx)
            buf = np.zeros((1 << 15, 2), dtype=np.int64)
            k = ncorp.ncorp_collisions(ctx, buf, len(buf))
            out.append({"x0": x0, "v0": v0, "x": arrs[0].cpu().numpy(), "v": arrs[1].cpu().numpy(),
                        "pairs": buf[:k].copy(), "fused": st["fused"], "tests": st["col_tests"]})
    finally:
        ncorp.ncorp_free(ctx)
    return out


def dense_disk(n, seed):
    return diskgen.make_disk(n, seed, a_lo=2.0, a_hi=2.5, r_lo=2e-2, r_hi=5e-2, sigma_e=0.1, sigma_i=0.05)


@pytest.mark.parametrize("precision,p", [(ncorp.NCORP_FP64, 3), (ncorp.NCORP_MIXED, 6)])
def test_fused_walk_gives_the_same_pairs_and_states(precision, p):
    d = dense_disk(20000, 311)
    a = run(d, 0, p, precision)
    b = run(d, 1, p, precision)
    assert [s["fused"] for s in a] == [0] * STEPS
    assert b[0]["fused"] == 0 and sum(s["fused"] for s in b[1:]) >= STEPS - 2   # the bounds held
    assert sum(len(s["pairs"]) for s in a) > 20                                  # the disk does collide
    tol = 1e-12 if precision == ncorp.NCORP_FP64 else 1e-9
    for sa, sb in zip(a, b):
        assert np.array_equal(sa["pairs"], sb["pairs"])
        np.testing.assert_allclose(sb["x"], sa["x"], rtol=0, atol=tol * np.abs(sa["x"]).max())
        np.testing.assert_allclose(sb["v"], sa["v"], rtol=0, atol=tol * 1e3 * np.abs(sa["v"]).max())
