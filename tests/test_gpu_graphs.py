"""CUDA graphs of resident steps (ncorp_set_graphs), needs a GB300.

From the second call on, ncorp_step runs its step as a replayed CUDA graph
(two graphs, one per buffer rotation).  The replayed step launches the same
kernels with the same arguments as the direct one, so the states agree to the
rounding of the order-dependent sums (the walk appends its interaction lists
with atomics, so their order, hence the order of the M2L and near-field sums,
varies from run to run), and the colliding pairs are the same.
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


def run(d, graphs, host, precision=ncorp.NCORP_FP64, stream=None):
    n = len(d["pos"])
    cfg = ncorp.ncorp_config_default()
    cfg.precision = precision
    cfg.leaf_size = 64
    cfg.n_cs, cfg.n_cc_pre, cfg.n_cc_post = 256, 256, 512
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    ctx = ncorp.ncorp_init(cfg, n, 0, s)
    if host:
        arrs = [d[k].copy() for k in ("pos", "vel", "mass", "radius")]
    else:
        arrs = [torch.tensor(d[k], device="cuda") for k in ("pos", "vel", "mass", "radius")]
    used, states, pairs = [], [], []
    try:
        ncorp.ncorp_set_graphs(ctx, graphs)
        for _ in range(STEPS):
            ncorp.ncorp_step(ctx, *arrs, n, 6, 0.5, 1e-3)
            used.append(ncorp.ncorp_stats(ctx)["graph"])
            x, v = arrs[0], arrs[1]
            if not host:
                x, v = x.cpu().numpy(), v.cpu().numpy()
            states.append((x.copy(), v.copy()))
            buf = np.zeros((1 << 14, 2), dtype=np.int64)
            k = ncorp.ncorp_collisions(ctx, buf, len(buf))
            pairs.append(buf[:k].copy())
    finally:
        ncorp.ncorp_free(ctx)
    return used, states, pairs


@pytest.mark.parametrize("host", [False, True])
def test_graph_steps_match_direct_steps(host):
    d = diskgen.make_disk(30000, 71, a_lo=2.0, a_hi=2.6, r_lo=1e-2, r_hi=3e-2)
    used_g, st_g, pairs_g = run(d, True, host)
    used_d, st_d, pairs_d = run(d, False, host)
    assert used_g == [0] + [1] * (STEPS - 1)
    assert used_d == [0] * STEPS
    for (xg, vg), (xd, vd) in zip(st_g, st_d):
        np.testing.assert_allclose(xg, xd, rtol=0, atol=1e-12 * np.abs(xd).max())
        np.testing.assert_allclose(vg, vd, rtol=0, atol=1e-11 * np.abs(vd).max())
    assert sum(len(p) for p in pairs_d) > 0
    for pg, pd in zip(pairs_g, pairs_d):
        assert np.array_equal(pg, pd)


def test_graph_steps_on_a_side_stream_and_after_toggling():
    """Graphs launch on the caller's stream (here a non-default one); turning
    graphs off and on again between steps keeps the state resident."""
    d = diskgen.make_disk(20000, 72)
    n = len(d["pos"])
    stream = torch.cuda.Stream()
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_MIXED
    ctx = ncorp.ncorp_init(cfg, n, 0, stream.cuda_stream)
    ref = ncorp.ncorp_init(cfg, n, 0, stream.cuda_stream)
    with torch.cuda.stream(stream):
        a = [torch.tensor(d[k], device="cuda") for k in ("pos", "vel", "mass", "radius")]
        b = [t.clone() for t in a]
    used = []
    try:
        ncorp.ncorp_set_graphs(ref, False)
        for i in range(5):
            if i == 3:
                ncorp.ncorp_set_graphs(ctx, False)
            if i == 4:
                ncorp.ncorp_set_graphs(ctx, True)
            ncorp.ncorp_step(ctx, *a, n, 4, 0.6, 2e-3)
            used.append(ncorp.ncorp_stats(ctx)["graph"])
            ncorp.ncorp_step(ref, *b, n, 4, 0.6, 2e-3)
        stream.synchronize()
        x, v = a[0].cpu().numpy(), a[1].cpu().numpy()
        xr, vr = b[0].cpu().numpy(), b[1].cpu().numpy()
    finally:
        ncorp.ncorp_free(ctx)
        ncorp.ncorp_free(ref)
    assert used == [0, 1, 1, 0, 1]
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-12 * np.abs(xr).max())
    # FP32 sums in another order: the velocities agree to about the mixed-precision error
    assert np.abs(v - vr).max() <= 1e-6 * np.abs(vr).max()


def test_radix_status_clearing_keeps_results(monkeypatch):
    """The radix sorts tag their look-back status words with a device epoch;
    at a limit the sort clears the status words and restarts the epoch.  With
    the limit lowered to 3, the clearing runs every few sorts (in directly
    launched and replayed steps, and in the colliding-pair sorts) and the
    results stay those of a context that never reaches it."""
    d = diskgen.make_disk(30000, 73, a_lo=2.0, a_hi=2.6, r_lo=1e-2, r_hi=3e-2)
    monkeypatch.setenv("NCORP_RADIX_EPOCH_LIMIT", "3")
    used_w, st_w, pairs_w = run(d, True, False)
    monkeypatch.delenv("NCORP_RADIX_EPOCH_LIMIT")
    used_r, st_r, pairs_r = run(d, True, False)
    assert used_w == used_r == [0] + [1] * (STEPS - 1)
    for (xw, vw), (xr, vr) in zip(st_w, st_r):
        np.testing.assert_allclose(xw, xr, rtol=0, atol=1e-12 * np.abs(xr).max())
        np.testing.assert_allclose(vw, vr, rtol=0, atol=1e-11 * np.abs(vr).max())
    assert sum(len(p) for p in pairs_r) > 0
    for pw, pr in zip(pairs_w, pairs_r):
        assert np.array_equal(pw, pr)
