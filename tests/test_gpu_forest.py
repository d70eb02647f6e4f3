"""Forests: many independent disks in one context (ncorp_set_disks), needs a GB300.

A forest runs every stage once over all its disks.  Each disk must come out
as the same disk alone: per disk, the Hilbert keys, moonlet order, cells and
climb geometry equal the oracle's bit for bit, the walk takes the oracle's
decisions (the forest's counts are the sums over its disks), the colliding
pairs equal brute force, and the accelerations match the oracle's falcON to
1e-11 (FP64) / 2e-5 (mixed) per moonlet.  Disks of one and two moonlets are
in the mix (a root that is a leaf).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_20374_gb300 import diskgen, ncorp

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
MIXED_TOL = 2e-5
DECISIONS = ("m2l", "p2p_pairs", "p2p_self", "p2p_interactions")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def make_ctx(n_max, precision=ncorp.NCORP_FP64, s=16, grav=(64, 8, 64)):
    cfg = ncorp.ncorp_config_default()
    cfg.precision = precision
    cfg.leaf_size = s
    cfg.n_cs, cfg.n_cc_pre, cfg.n_cc_post = grav
    return ncorp.ncorp_init(cfg, n_max, 0, torch.cuda.current_stream().cuda_stream)


def tiny(n, seed):
    """A disk of n < 3 moonlets (the generator's smallest disks are larger)."""
    rng = np.random.default_rng(seed)
    pos = np.array([[3.0, 0.5, 0.1], [3.05, 0.45, 0.1]])[:n] + rng.normal(size=(n, 3)) * 1e-3
    vel = np.array([[-0.2, 0.55, 0.0], [-0.19, 0.56, 0.0]])[:n]
    return {"pos": pos, "vel": vel, "mass": np.full(n, 1e-4), "radius": np.full(n, 1e-3)}


def disks_for(sizes, seed, dense=()):
    out = []
    for k, n in enumerate(sizes):
        if n < 3:
            out.append(tiny(n, seed + k))
        elif k in dense:
            out.append(diskgen.make_disk(n, seed + k, a_lo=2.0, a_hi=2.5, r_lo=2e-2, r_hi=5e-2, sigma_e=0.1,
                                         sigma_i=0.05))
        else:
            out.append(diskgen.make_disk(n, seed + k))
    return out


def concat(disks):
    return {f: np.concatenate([d[f] for d in disks]) for f in ("pos", "vel", "mass", "radius")}


def offsets(sizes):
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


def export_tree(ctx, n, nd):
    cap = 8 * n + 64 * nd
    order = np.zeros(n, dtype=np.int64)
    keys = np.zeros(n, dtype=np.uint64)
    root = np.zeros((nd, 4))
    cells = np.zeros((cap, 7), dtype=np.int64)
    gg = np.zeros((cap, 6))
    cg = np.zeros((cap, 5))
    nc = ncorp.ncorp_tree_export(ctx, order, keys, root, cells, gg, cg, cap)
    return {"order": order, "keys": keys, "root": root, "cells": cells[:nc], "ggeo": gg[:nc], "cgeo": cg[:nc]}


def disk_part(g, lo, hi):
    """The cells of the forest's disk holding moonlets [lo, hi), in the forest's order, with moonlet
    indices made disk-local."""
    sel = (g["cells"][:, 4] >= lo) & (g["cells"][:, 4] < hi)
    cells = g["cells"][sel].copy()
    cells[:, 4] -= lo
    return cells, g["ggeo"][sel], g["cgeo"][sel]


def test_forest_tree_geometry_decisions_and_fp64_accel_per_disk():
    sizes = [5000, 1, 2, 700, 9000, 33]
    p, theta, s = 3, 0.5, 16
    disks = disks_for(sizes, 300)
    a = concat(disks)
    n, off = sum(sizes), offsets(sizes)
    ctx = make_ctx(n, s=s)
    try:
        ncorp.ncorp_set_disks(ctx, sizes)
        acc = np.zeros((n, 3))
        mut = np.zeros((n, 3))
        ncorp.ncorp_accel(ctx, a["pos"], a["mass"], n, p, theta, acc, mut)
        st = ncorp.ncorp_stats(ctx)
        g = export_tree(ctx, n, len(sizes))
    finally:
        ncorp.ncorp_free(ctx)
    P = oracle.params(p=p, theta=theta, leaf_size=s)
    sums = {k: 0 for k in DECISIONS + ("cells", "leaves")}
    for k, d in enumerate(disks):
        lo, hi = off[k], off[k + 1]
        o = oracle.tree_export(P, d["pos"], d["mass"])
        assert np.array_equal(g["root"][k], o["root"])
        assert np.array_equal(g["order"][lo:hi] - lo, o["order"])
        assert np.array_equal(g["keys"][lo:hi], o["keys"][o["order"]])
        cells, gg, _ = disk_part(g, lo, hi)
        assert np.array_equal(cells, o["cells"])
        assert np.array_equal(gg, o["ggeo"])          # M, s, r_max, r_crit bit for bit
        ref, ost = oracle.falcon_accel(P, d["pos"], d["mass"])
        for key in sums:
            sums[key] += ost[key]
        if sizes[k] == 1:
            assert np.all(mut[lo:hi] == 0.0)
        else:
            assert rel_err(mut[lo:hi], ref).max() <= FP64_TOL
        ext = oracle.external_accel(P, d["pos"])
        np.testing.assert_allclose(acc[lo:hi], ref + ext, rtol=1e-12, atol=1e-15)
    for key, v in sums.items():
        assert st[key] == v, (key, st[key], v)


@pytest.mark.parametrize("p,theta,s", [(6, 0.5, 64), (4, 0.6, 48)])
def test_forest_mixed_accel_matches_oracle_per_disk(p, theta, s):
    sizes = [20000, 3000, 12000, 2]
    grav = (256, 256, 512) if p == 6 else (64, 8, 64)
    disks = disks_for(sizes, 310 + p)
    a = concat(disks)
    n, off = sum(sizes), offsets(sizes)
    ctx = make_ctx(n, precision=ncorp.NCORP_MIXED, s=s, grav=grav)
    try:
        ncorp.ncorp_set_disks(ctx, sizes)
        pos = torch.tensor(a["pos"], device="cuda")
        m = torch.tensor(a["mass"], device="cuda")
        acc = torch.empty_like(pos)
        mut = torch.empty_like(pos)
        ncorp.ncorp_accel(ctx, pos, m, n, p, theta, acc, mut)
        mut = mut.cpu().numpy()
    finally:
        ncorp.ncorp_free(ctx)
    P = oracle.params(p=p, theta=theta, leaf_size=s, gravity_thresholds=grav)
    for k, d in enumerate(disks):
        ref, _ = oracle.falcon_accel(P, d["pos"], d["mass"])
        e = rel_err(mut[off[k]:off[k + 1]], ref)
        assert e.max() <= MIXED_TOL, (k, e.max(), np.median(e))


def test_forest_collision_pairs_and_geometry_bit_exact():
    sizes = [3000, 2500, 1, 4000, 2]
    dt = 0.05
    disks = disks_for(sizes, 320, dense=(0, 1, 3))
    a = concat(disks)
    n, off = sum(sizes), offsets(sizes)
    ctx = make_ctx(n, s=16)
    try:
        ncorp.ncorp_set_disks(ctx, sizes)
        ncorp.ncorp_collide(ctx, torch.tensor(a["pos"], device="cuda"), torch.tensor(a["vel"], device="cuda"),
                            torch.tensor(a["radius"], device="cuda"), n, dt)
        out = np.zeros((1 << 15, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, out, len(out))
        st = ncorp.ncorp_stats(ctx)
        g = export_tree(ctx, n, len(sizes))
    finally:
        ncorp.ncorp_free(ctx)
    P = oracle.params(p=3, leaf_size=16)
    want, tests = [], 0
    for j, d in enumerate(disks):
        lo, hi = off[j], off[j + 1]
        brute = oracle.collide_brute(d["pos"], d["vel"], d["radius"], dt)
        want.append(brute + lo)
        o = oracle.tree_export(P, d["pos"], None, d["vel"], d["radius"], dt)
        cells, _, cg = disk_part(g, lo, hi)
        assert np.array_equal(cells, o["cells"])
        assert np.array_equal(cg, o["cgeo"])
        _, ost = oracle.collide_tree(P, d["pos"], d["vel"], d["radius"], dt)
        tests += ost["col_tests"]
    want = np.concatenate(want)
    assert len(want) > 20
    assert np.array_equal(out[:k], want)
    assert st["col_tests"] == tests


def single_steps(d, p, theta, dt, steps, s):
    n = len(d["pos"])
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_FP64
    cfg.leaf_size = s
    ctx = ncorp.ncorp_init(cfg, n, 0, torch.cuda.current_stream().cuda_stream)
    pos, vel = d["pos"].copy(), d["vel"].copy()
    try:
        for _ in range(steps):
            ncorp.ncorp_step(ctx, pos, vel, d["mass"], d["radius"], n, p, theta, dt)
        pairs = np.zeros((1 << 14, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, pairs, len(pairs))
    finally:
        ncorp.ncorp_free(ctx)
    return pos, vel, pairs[:k]


def forest_steps(disks, p, theta, dt, steps, s):
    sizes = [len(d["pos"]) for d in disks]
    a = concat(disks)
    n = sum(sizes)
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_FP64
    cfg.leaf_size = s
    ctx = ncorp.ncorp_init(cfg, n, 0, torch.cuda.current_stream().cuda_stream)
    pos, vel = torch.tensor(a["pos"], device="cuda"), torch.tensor(a["vel"], device="cuda")
    m, R = torch.tensor(a["mass"], device="cuda"), torch.tensor(a["radius"], device="cuda")
    launches = []
    try:
        ncorp.ncorp_set_disks(ctx, sizes)
        for _ in range(steps):
            ncorp.ncorp_step(ctx, pos, vel, m, R, n, p, theta, dt)
            launches.append(ncorp.ncorp_stats(ctx)["launches"])
        pairs = np.zeros((1 << 15, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, pairs, len(pairs))
    finally:
        ncorp.ncorp_free(ctx)
    return pos.cpu().numpy(), vel.cpu().numpy(), pairs[:k], launches


def test_forest_steps_equal_each_disk_alone_with_launches_independent_of_disks():
    p, theta, dt, s, steps = 4, 0.5, 2e-2, 24, 3
    sizes = [3000, 2000, 5000, 1500, 2500, 4000]
    disks = disks_for(sizes, 330, dense=(0, 3))
    pos, vel, pairs, launches6 = forest_steps(disks, p, theta, dt, steps, s)
    off = offsets(sizes)
    for k, d in enumerate(disks):
        xs, vs, ps = single_steps(d, p, theta, dt, steps, s)
        lo, hi = off[k], off[k + 1]
        np.testing.assert_allclose(pos[lo:hi], xs, rtol=0, atol=1e-12 * np.abs(xs).max())
        np.testing.assert_allclose(vel[lo:hi], vs, rtol=0, atol=1e-11 * np.abs(vs).max())
        mine = pairs[(pairs[:, 0] >= lo) & (pairs[:, 0] < hi)] - lo
        assert np.array_equal(mine, ps)
        if k in (0, 3):
            assert len(ps) > 0
    # one launch per stage: half the disks, the same launches per step
    _, _, _, launches3 = forest_steps(disks[:3], p, theta, dt, steps, s)
    assert launches3 == launches6


def test_set_disks_rejections_and_return_to_one_disk():
    d = diskgen.make_disk(3000, 340)
    ctx = make_ctx(3000)
    try:
        for bad in ([], [0, 10], [-1], list(range(1, ncorp.NCORP_MAX_DISKS + 2))):
            with pytest.raises(ncorp.NcorpError) as e:
                ncorp.ncorp_set_disks(ctx, bad)
            assert e.value.code == ncorp.NCORP_EINVAL
        ncorp.ncorp_set_disks(ctx, [1000, 2000])
        acc = np.zeros((3000, 3))
        with pytest.raises(ncorp.NcorpError) as e:   # n is not the disks' total
            ncorp.ncorp_accel(ctx, d["pos"], d["mass"], 2999, 3, 0.5, acc, None)
        assert e.value.code == ncorp.NCORP_EINVAL and "total" in str(e.value)
        with pytest.raises(ncorp.NcorpError) as e:   # the standard tree code walks one disk
            ncorp.ncorp_accel_standard(ctx, d["pos"], d["mass"], 3000, 3, 0.5, acc, None)
        assert e.value.code == ncorp.NCORP_EINVAL
        ncorp.ncorp_accel(ctx, d["pos"], d["mass"], 3000, 3, 0.5, acc, None)
        two = acc.copy()
        ncorp.ncorp_set_disks(ctx, [3000])
        ncorp.ncorp_accel(ctx, d["pos"], d["mass"], 3000, 3, 0.5, acc, None)
        one = acc.copy()
    finally:
        ncorp.ncorp_free(ctx)
    # one disk again: the whole disk's field, which differs from that of its two halves
    P = oracle.params(p=3, theta=0.5, leaf_size=16)
    ref, _ = oracle.falcon_accel(P, d["pos"], d["mass"])
    ext = oracle.external_accel(P, d["pos"])
    np.testing.assert_allclose(one, ref + ext, rtol=1e-12, atol=1e-15)
    assert not np.allclose(two, one, rtol=1e-9, atol=0)
