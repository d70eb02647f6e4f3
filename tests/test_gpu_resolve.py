"""Collision resolution in ncorp_step (Sect. 5.1, 5.2) against the oracle (needs a GB300).

With gravity made negligible (central mass 0, moonlet masses ~1e-30) a step
is a drift with resolved impacts, computed on both sides with exactly rounded
FP64 operations in the same order: the GPU states must equal the oracle's bit
for bit, through clumps dense enough that many moonlets are in several pairs
per step (the one-impact-per-moonlet matching runs several rounds).  With
real gravity (a disk with inflated radii) the states agree to the FP64 falcON
tolerance of the plain KDK test and the resolved counts are equal.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_20374_gb300 import diskgen, ncorp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def clump(seed, n, spread=1.0):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-spread, spread, (n, 3)) + np.array([20.0, 0.0, 0.0])
    vel = rng.normal(size=(n, 3)) * 0.5
    return pos, vel, rng.uniform(0.5, 2.0, n) * 1e-30, rng.uniform(0.05, 0.12, n)


def make_ctx(n, f, precision=ncorp.NCORP_FP64, central_mass=0.0, s=16, graphs=True):
    cfg = ncorp.ncorp_config_default()
    cfg.precision = precision
    cfg.central_mass = central_mass
    cfg.leaf_size = s
    cfg.resolve_f = f
    ctx = ncorp.ncorp_init(cfg, n, 0, torch.cuda.current_stream().cuda_stream)
    ncorp.ncorp_set_graphs(ctx, graphs)
    return ctx


def gpu_steps(ctx, pos, vel, m, R, p, theta, dt, steps, device):
    n = len(pos)
    arrs = [pos.copy(), vel.copy(), m, R]
    if device:
        arrs = [torch.tensor(a, device="cuda") for a in arrs]
    out = []
    for _ in range(steps):
        ncorp.ncorp_step(ctx, *arrs, n, p, theta, dt)
        st = ncorp.ncorp_stats(ctx)
        buf = np.zeros((1 << 15, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, buf, len(buf))
        x, v = arrs[0], arrs[1]
        if device:
            x, v = x.cpu().numpy(), v.cpu().numpy()
        out.append((x.copy(), v.copy(), buf[:k].copy(), st["resolved"], st["graph"]))
    return out


def oracle_steps(P, pos, vel, m, R, dt, steps):
    out, acc = [], None
    x, v = pos, vel
    for _ in range(steps):
        info = {}
        x, v, acc, pairs = oracle.kdk(P, x, v, m, R, dt, 1, acc0=acc, info=info)
        out.append((x, v, pairs[:, 1:], info["resolved"]))
    return out


@pytest.mark.parametrize("f,device", [(2.0, True), (1.3, False), (1.0, True)])
def test_resolved_drift_equals_oracle_bit_for_bit(f, device):
    n, steps, dt = 3000, 4, 0.05
    pos, vel, m, R = clump(31, n, spread=1.6)
    P = oracle.params(p=3, theta=0.5, leaf_size=16, central_mass=0.0, resolve_f=f)
    ref = oracle_steps(P, pos, vel, m, R, dt, steps)
    ctx = make_ctx(n, f)
    try:
        got = gpu_steps(ctx, pos, vel, m, R, 3, 0.5, dt, steps, device)
    finally:
        ncorp.ncorp_free(ctx)
    assert [g[4] for g in got] == [0] + [1] * (steps - 1)     # replayed graphs from the second step
    for k, ((xg, vg, pg, rg, _), (xo, vo, po, ro)) in enumerate(zip(got, ref)):
        assert np.array_equal(pg, po), k
        assert rg == ro, (k, rg, ro)
        assert np.array_equal(xg, xo), (k, np.abs(xg - xo).max())
        assert np.array_equal(vg, vo), (k, np.abs(vg - vo).max())
    total_pairs = sum(len(r[2]) for r in ref)
    total_res = sum(r[3] for r in ref)
    # dense enough that moonlets meet several others in a step
    assert total_res > 100 and total_pairs > total_res + 20


def test_resolution_matching_with_many_conflicts():
    """A tight clump: hundreds of pairs per step, most sharing moonlets, so the
    matching takes several rounds; still equal to the sequential oracle."""
    n, dt = 1500, 0.1
    pos, vel, m, R = clump(32, n, spread=0.9)
    P = oracle.params(p=3, theta=0.5, leaf_size=16, central_mass=0.0, resolve_f=2.0)
    ref = oracle_steps(P, pos, vel, m, R, dt, 2)
    ctx = make_ctx(n, 2.0)
    try:
        got = gpu_steps(ctx, pos, vel, m, R, 3, 0.5, dt, 2, True)
    finally:
        ncorp.ncorp_free(ctx)
    assert len(ref[0][2]) > 2 * ref[0][3] > 200
    for (xg, vg, pg, rg, _), (xo, vo, po, ro) in zip(got, ref):
        assert np.array_equal(pg, po) and rg == ro
        assert np.array_equal(xg, xo) and np.array_equal(vg, vo)


@pytest.mark.parametrize("precision", [ncorp.NCORP_FP64, ncorp.NCORP_MIXED])
def test_resolution_in_a_disk_with_gravity(precision):
    n, p, theta, s, dt, steps = 20000, 3, 0.5, 16, 0.02, 3
    d = diskgen.make_disk(n, 52, a_lo=2.0, a_hi=2.6, r_lo=1e-2, r_hi=4e-2, sigma_e=0.1, sigma_i=0.05)
    P = oracle.params(p=p, theta=theta, leaf_size=s, resolve_f=1.5)
    ref = oracle_steps(P, d["pos"], d["vel"], d["mass"], d["radius"], dt, steps)
    ctx = make_ctx(n, 1.5, precision=precision, central_mass=1.0, s=s)
    try:
        got = gpu_steps(ctx, d["pos"], d["vel"], d["mass"], d["radius"], p, theta, dt, steps, True)
    finally:
        ncorp.ncorp_free(ctx)
    assert sum(r[3] for r in ref) > 20
    # mixed precision: mutual accelerations to ~2e-5 of their size, and close pairs (no softening) have
    # large ones; the step's kicks carry that into v and the drift into x
    tol_x, tol_v = (1e-12, 1e-11) if precision == ncorp.NCORP_FP64 else (1e-9, 1e-6)
    for (xg, vg, pg, rg, _), (xo, vo, po, ro) in zip(got, ref):
        assert np.array_equal(pg, po) and rg == ro
        np.testing.assert_allclose(xg, xo, rtol=0, atol=tol_x * np.abs(xo).max())
        np.testing.assert_allclose(vg, vo, rtol=0, atol=tol_v * np.abs(vo).max())


def test_resolution_off_reports_the_same_pairs_without_changing_the_drift():
    """resolve_f = 0 (the default) leaves the step as before: the pairs are
    reported and the moonlets pass through each other."""
    n, dt = 2000, 0.05
    pos, vel, m, R = clump(33, n, spread=1.6)
    P = oracle.params(p=3, theta=0.5, leaf_size=16, central_mass=0.0)
    ref = oracle_steps(P, pos, vel, m, R, dt, 2)
    ctx = make_ctx(n, 0.0)
    try:
        got = gpu_steps(ctx, pos, vel, m, R, 3, 0.5, dt, 2, True)
    finally:
        ncorp.ncorp_free(ctx)
    for (xg, vg, pg, rg, _), (xo, vo, po, ro) in zip(got, ref):
        assert rg == 0 and ro == 0 and len(po) > 0
        assert np.array_equal(pg, po)
        assert np.array_equal(xg, xo) and np.array_equal(vg, vo)
