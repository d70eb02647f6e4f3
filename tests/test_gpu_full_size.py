"""Parity at the full sizes of the three single-disk workloads (needs a GB300).

  1. N = 1e4 disk (seed 1), p = 3, theta_min = 0.5, FP64: one force evaluation
     and one collision search over dt = 1e-3.
  2. N = 1e5 disk (seed 2), p = 6, theta_min = 0.5, FP64 and mixed: the
     benchmark's workload, in the launch configuration the benchmark times
     (leaf size 64, thresholds (256, 256, 512), collisions (12, 0, 16)); one
     force evaluation each and one full step in FP64, against the oracle.
  3. N = 1e6 disk (seed 3), p = 4, theta_min = 0.6, mixed: keys, order,
     cells, climb geometry and the colliding pairs against the oracle
     exactly; the mutual accelerations against the oracle's falcON per
     moonlet (2e-5) with equal walk decision counts (one oracle evaluation
     at this size takes about 15 s); momentum and the error against direct
     summation on a seeded sample.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_20374_gb300 import diskgen, ncorp

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
MIXED_TOL = 2e-5
LAUNCH = {3: (32, (64, 8, 64)), 4: (48, (64, 8, 64)), 6: (64, (256, 256, 512))}   # p -> (leaf size, thresholds)
COLL = (12, 0, 16)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def ctx_for(n, p, precision):
    s, grav = LAUNCH[p]
    cfg = ncorp.ncorp_config_default()
    cfg.precision = precision
    cfg.leaf_size = s
    cfg.n_cs, cfg.n_cc_pre, cfg.n_cc_post = grav
    cfg.c_cs, cfg.c_cc_pre, cfg.c_cc_post = COLL
    return ncorp.ncorp_init(cfg, n, 0, torch.cuda.current_stream().cuda_stream)


def params_for(p, theta):
    s, grav = LAUNCH[p]
    return oracle.params(p=p, theta=theta, leaf_size=s, gravity_thresholds=grav, collision_thresholds=COLL)


def gpu_mutual(ctx, d, p, theta):
    n = len(d["pos"])
    pos = torch.tensor(d["pos"], device="cuda")
    m = torch.tensor(d["mass"], device="cuda")
    acc = torch.empty_like(pos)
    mut = torch.empty_like(pos)
    ncorp.ncorp_accel(ctx, pos, m, n, p, theta, acc, mut)
    return mut.cpu().numpy(), ncorp.ncorp_stats(ctx)


def rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


DECISIONS = ("cells", "leaves", "depth", "m2l", "p2p_pairs", "p2p_self", "p2p_interactions")


# ------------------------------------------------------------------ workload 1
def test_disk_1e4_p3_fp64_forces_and_collisions():
    n, p, theta, dt = 10_000, 3, 0.5, 1e-3
    d = diskgen.make_disk(n, 1)
    ctx = ctx_for(n, p, ncorp.NCORP_FP64)
    try:
        mut, st = gpu_mutual(ctx, d, p, theta)
        ncorp.ncorp_collide(ctx, torch.tensor(d["pos"], device="cuda"), torch.tensor(d["vel"], device="cuda"),
                            torch.tensor(d["radius"], device="cuda"), n, dt)
        pairs = np.zeros((1 << 12, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, pairs, len(pairs))
    finally:
        ncorp.ncorp_free(ctx)
    P = params_for(p, theta)
    ref, ost = oracle.falcon_accel(P, d["pos"], d["mass"])
    assert all(st[key] == ost[key] for key in DECISIONS), {key: (st[key], ost[key]) for key in DECISIONS}
    assert rel_err(mut, ref).max() <= FP64_TOL
    brute = oracle.collide_brute(d["pos"], d["vel"], d["radius"], dt)
    assert np.array_equal(pairs[:k], brute)


# ------------------------------------------------------------------ workload 2
@pytest.fixture(scope="module")
def disk_1e5():
    d = diskgen.make_disk(100_000, 2)
    P = params_for(6, 0.5)
    ref, ost = oracle.falcon_accel(P, d["pos"], d["mass"])
    return d, ref, ost


@pytest.mark.parametrize("precision,tol", [(ncorp.NCORP_FP64, FP64_TOL), (ncorp.NCORP_MIXED, MIXED_TOL)])
def test_disk_1e5_p6_forces_match_oracle(disk_1e5, precision, tol):
    d, ref, ost = disk_1e5
    n = len(d["pos"])
    ctx = ctx_for(n, 6, precision)
    try:
        mut, st = gpu_mutual(ctx, d, 6, 0.5)
    finally:
        ncorp.ncorp_free(ctx)
    assert all(st[key] == ost[key] for key in DECISIONS), {key: (st[key], ost[key]) for key in DECISIONS}
    e = rel_err(mut, ref)
    assert e.max() <= tol, (e.max(), np.percentile(e, 99))
    # accuracy of the method against direct summation on a seeded 10^3 sample, central body
    # included as in Sect. 4.2 (the oracle itself gives median 1.7e-6, p99 1.6e-5 on this
    # 0.02-mass disk; the paper quotes ~1e-7 at p = 6 for its runs)
    idx = np.random.default_rng(2).choice(n, 1000, replace=False)
    direct = oracle.direct_accel(d["pos"], d["mass"], targets=idx)
    ext = oracle.external_accel(params_for(6, 0.5), d["pos"][idx])
    ed = rel_err(mut[idx] + ext, direct + ext)
    assert np.median(ed) < 1e-5 and np.percentile(ed, 99) < 1e-4, (np.median(ed), np.percentile(ed, 99))


def test_disk_1e5_p6_fp64_step_matches_oracle_kdk(disk_1e5):
    d, _, _ = disk_1e5
    n, dt = len(d["pos"]), 1e-3
    ctx = ctx_for(n, 6, ncorp.NCORP_FP64)
    pos = torch.tensor(d["pos"], device="cuda")
    vel = torch.tensor(d["vel"], device="cuda")
    try:
        ncorp.ncorp_step(ctx, pos, vel, torch.tensor(d["mass"], device="cuda"),
                         torch.tensor(d["radius"], device="cuda"), n, 6, 0.5, dt)
        pairs = np.zeros((1 << 12, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, pairs, len(pairs))
    finally:
        ncorp.ncorp_free(ctx)
    xo, vo, _, po = oracle.kdk(params_for(6, 0.5), d["pos"], d["vel"], d["mass"], d["radius"], dt, 1)
    np.testing.assert_allclose(pos.cpu().numpy(), xo, rtol=0, atol=1e-13 * np.abs(xo).max())
    np.testing.assert_allclose(vel.cpu().numpy(), vo, rtol=0, atol=1e-12 * np.abs(vo).max())
    assert [tuple(r) for r in po[:, 1:].tolist()] == [tuple(r) for r in pairs[:k].tolist()]


# ------------------------------------------------------------------ workload 3
def test_disk_1e6_p4_mixed_tree_collisions_and_accuracy():
    n, p, theta, dt = 1_000_000, 4, 0.6, 1e-3
    d = diskgen.make_disk(n, 3)
    ctx = ctx_for(n, p, ncorp.NCORP_MIXED)
    try:
        mut, st = gpu_mutual(ctx, d, p, theta)
        cap = n // 2
        order = np.zeros(n, dtype=np.int64)
        keys = np.zeros(n, dtype=np.uint64)
        root = np.zeros(4)
        cells = np.zeros((cap, 7), dtype=np.int64)
        gg = np.zeros((cap, 6))
        nc = ncorp.ncorp_tree_export(ctx, order, keys, root, cells, gg, None, cap)
        assert nc <= cap
        ncorp.ncorp_collide(ctx, torch.tensor(d["pos"], device="cuda"), torch.tensor(d["vel"], device="cuda"),
                            torch.tensor(d["radius"], device="cuda"), n, dt)
        pairs = np.zeros((1 << 14, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, pairs, len(pairs))
    finally:
        ncorp.ncorp_free(ctx)
    P = params_for(p, theta)
    o = oracle.tree_export(P, d["pos"], d["mass"])
    assert np.array_equal(root, o["root"])
    assert np.array_equal(order, o["order"])
    assert np.array_equal(keys, o["keys"][o["order"]])
    assert np.array_equal(cells[:nc], o["cells"])
    assert np.array_equal(gg[:nc], o["ggeo"])
    assert st["cells"] == nc
    ref_pairs, _ = oracle.collide_tree(P, d["pos"], d["vel"], d["radius"], dt)
    assert np.array_equal(pairs[:k], ref_pairs)
    # element-wise parity with the oracle's falcON at the full size, same walk decisions
    ref, ost = oracle.falcon_accel(P, d["pos"], d["mass"])
    assert all(st[key] == ost[key] for key in DECISIONS), {key: (st[key], ost[key]) for key in DECISIONS}
    e = rel_err(mut, ref)
    assert e.max() <= MIXED_TOL, (e.max(), np.median(e))
    # momentum: the symmetric M2L and the pairwise near field conserve it up to FP32 rounding
    f = d["mass"][:, None] * mut
    assert np.linalg.norm(f.sum(axis=0)) <= 1e-6 * np.linalg.norm(f, axis=1).sum()
    # accuracy against direct summation on a seeded sample, central body included (the oracle
    # gives median 3e-5, p99 1.9e-4 at p = 4, theta_min = 0.6 on a 2e5 disk of this kind)
    idx = np.random.default_rng(3).choice(n, 500, replace=False)
    direct = oracle.direct_accel(d["pos"], d["mass"], targets=idx)
    ext = oracle.external_accel(P, d["pos"][idx])
    ed = rel_err(mut[idx] + ext, direct + ext)
    assert np.median(ed) < 3e-4 and np.percentile(ed, 99) < 3e-3, (np.median(ed), np.percentile(ed, 99))
