"""CUDA path vs the CPU oracle, through the C ABI (needs a GB300).

Bit-exact: Hilbert keys, moonlet order, cells, the tree-climb geometry that
decides the walk, the walk's decision counts and the colliding-pair sets.
Tolerances (relative, per moonlet, on the mutual acceleration): 1e-11 for
the FP64 path and 2e-5 for the mixed FP32/FP64 path, against the oracle's
falcON at the same p, theta_min, leaf size and thresholds.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2310_20374_gb300 import diskgen, ncorp

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
MIXED_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def make_ctx(n_max, precision=ncorp.NCORP_FP64, s=16, grav=(64, 8, 64), col=(12, 0, 16), collisions=1, star=None,
             bulge=None):
    cfg = ncorp.ncorp_config_default()
    if bulge:
        cfg.central_radius, cfg.central_J2 = bulge
    cfg.precision = precision
    cfg.leaf_size = s
    cfg.n_cs, cfg.n_cc_pre, cfg.n_cc_post = grav
    cfg.c_cs, cfg.c_cc_pre, cfg.c_cc_post = col
    cfg.collisions = collisions
    if star:
        cfg.star_mass, cfg.star_a, cfg.star_obliquity = star
    return ncorp.ncorp_init(cfg, n_max, 0, torch.cuda.current_stream().cuda_stream)


def gpu_accel(ctx, d, p, theta):
    n = len(d["pos"])
    pos = torch.tensor(d["pos"], device="cuda")
    m = torch.tensor(d["mass"], device="cuda")
    acc = torch.empty_like(pos)
    mut = torch.empty_like(pos)
    ncorp.ncorp_accel(ctx, pos, m, n, p, theta, acc, mut)
    return acc.cpu().numpy(), mut.cpu().numpy(), ncorp.ncorp_stats(ctx)


def rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


def export_tree(ctx, n):
    cap = 8 * n + 64
    order = np.zeros(n, dtype=np.int64)
    keys = np.zeros(n, dtype=np.uint64)
    root = np.zeros(4)
    cells = np.zeros((cap, 7), dtype=np.int64)
    gg = np.zeros((cap, 6))
    cg = np.zeros((cap, 5))
    nc = ncorp.ncorp_tree_export(ctx, order, keys, root, cells, gg, cg, cap)
    return {"order": order, "keys": keys, "root": root, "cells": cells[:nc], "ggeo": gg[:nc], "cgeo": cg[:nc]}


# ----------------------------------------------------------------- tree parity
@pytest.mark.parametrize("n,s,seed", [(5000, 16, 1), (20000, 40, 2), (777, 3, 3)])
def test_keys_order_cells_and_geometry_bit_exact(n, s, seed):
    d = diskgen.make_disk(n, seed)
    ctx = make_ctx(n, s=s)
    try:
        gpu_accel(ctx, d, 3, 0.5)
        g = export_tree(ctx, n)
    finally:
        ncorp.ncorp_free(ctx)
    P = oracle.params(p=3, theta=0.5, leaf_size=s)
    o = oracle.tree_export(P, d["pos"], d["mass"])
    assert np.array_equal(g["root"], o["root"])
    assert np.array_equal(g["keys"], o["keys"][o["order"]])
    assert np.array_equal(g["order"], o["order"])
    assert np.array_equal(g["cells"], o["cells"])
    assert np.array_equal(g["ggeo"], o["ggeo"])        # M, s, r_max, r_crit bit for bit


def test_collision_geometry_bit_exact():
    n = 4000
    d = diskgen.make_disk(n, 5)
    ctx = make_ctx(n, s=16)
    try:
        ncorp.ncorp_collide(ctx, torch.tensor(d["pos"], device="cuda"), torch.tensor(d["vel"], device="cuda"),
                            torch.tensor(d["radius"], device="cuda"), n, 1e-3)
        g = export_tree(ctx, n)
        st = ncorp.ncorp_stats(ctx)
    finally:
        ncorp.ncorp_free(ctx)
    P = oracle.params(p=3, leaf_size=16)
    o = oracle.tree_export(P, d["pos"], None, d["vel"], d["radius"], 1e-3)
    assert np.array_equal(g["cells"], o["cells"])
    assert np.array_equal(g["cgeo"], o["cgeo"])
    _, ost = oracle.collide_tree(P, d["pos"], d["vel"], d["radius"], 1e-3)
    assert (st["col_pairs"], st["col_self"], st["col_tests"]) == (ost["col_pairs"], ost["col_self"], ost["col_tests"])


# ------------------------------------------------------------- gravity parity
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_fp64_accel_matches_oracle_falcon(p):
    n, s, theta = 6000, 24, 0.5
    grav = (256, 256, 512) if p == 6 else (64, 8, 64)
    d = diskgen.make_disk(n, 10 + p)
    ctx = make_ctx(n, s=s, grav=grav)
    try:
        acc, mut, st = gpu_accel(ctx, d, p, theta)
    finally:
        ncorp.ncorp_free(ctx)
    P = oracle.params(p=p, theta=theta, leaf_size=s, gravity_thresholds=grav)
    ref, ost = oracle.falcon_accel(P, d["pos"], d["mass"])
    # identical walk decisions
    for k in ("cells", "leaves", "depth", "m2l", "p2p_pairs", "p2p_self", "p2p_interactions"):
        assert st[k] == ost[k], (k, st[k], ost[k])
    assert rel_err(mut, ref).max() <= FP64_TOL
    ext = oracle.external_accel(P, d["pos"])
    np.testing.assert_allclose(acc, ref + ext, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("p,theta,s", [(3, 0.5, 32), (4, 0.6, 48), (6, 0.5, 64)])
def test_mixed_accel_matches_oracle_falcon(p, theta, s):
    n = 8000
    grav = (256, 256, 512) if p == 6 else (64, 8, 64)
    d = diskgen.make_disk(n, 20 + p)
    ctx = make_ctx(n, precision=ncorp.NCORP_MIXED, s=s, grav=grav)
    try:
        acc, mut, st = gpu_accel(ctx, d, p, theta)
    finally:
        ncorp.ncorp_free(ctx)
    P = oracle.params(p=p, theta=theta, leaf_size=s, gravity_thresholds=grav)
    ref, ost = oracle.falcon_accel(P, d["pos"], d["mass"])
    assert st["m2l"] == ost["m2l"] and st["p2p_interactions"] == ost["p2p_interactions"]
    e = rel_err(mut, ref)
    assert e.max() <= MIXED_TOL, (e.max(), np.percentile(e, 99))


def test_momentum_conserved_fp64():
    n = 20000
    d = diskgen.make_disk(n, 31)
    ctx = make_ctx(n, s=32, grav=(256, 256, 512))
    try:
        _, mut, _ = gpu_accel(ctx, d, 6, 0.5)
    finally:
        ncorp.ncorp_free(ctx)
    ma = d["mass"][:, None] * mut
    assert np.linalg.norm(ma.sum(0)) <= 1e-13 * np.abs(ma).sum()


def test_star_tide_and_central_force():
    n = 2000
    d = diskgen.make_disk(n, 41)
    star = (3.3e5, 2.3e4, 0.41)
    ctx = make_ctx(n, s=16, star=star)
    try:
        acc, mut, _ = gpu_accel(ctx, d, 3, 0.5)
    finally:
        ncorp.ncorp_free(ctx)
    P = oracle.params(p=3, star=star)
    ext = oracle.external_accel(P, d["pos"], 0.0)
    np.testing.assert_allclose(acc - mut, ext, rtol=1e-13, atol=1e-18)


def test_equatorial_bulge_and_star():
    """External forces with the central body's bulge (App. B.2) and the star
    (App. B.3) together, FP64: the acceleration minus the mutual part is the
    oracle's external acceleration; three KDK steps (the later ones replayed
    from a graph) follow the oracle's."""
    n, dt = 2000, 2e-3
    d = diskgen.make_disk(n, 42)
    star, bulge = (3.3e5, 2.3e4, 0.41), (1.0, 1.08e-3)
    ctx = make_ctx(n, s=16, star=star, bulge=bulge)
    try:
        acc, mut, _ = gpu_accel(ctx, d, 3, 0.5)
    finally:
        ncorp.ncorp_free(ctx)
    P = oracle.params(p=3, star=star, bulge=bulge, leaf_size=16, gravity_thresholds=(64, 8, 64))
    ext = oracle.external_accel(P, d["pos"], 0.0)
    np.testing.assert_allclose(acc - mut, ext, rtol=1e-13, atol=1e-18)
    no_bulge = oracle.external_accel(oracle.params(p=3, star=star), d["pos"], 0.0)
    assert np.abs(ext - no_bulge).max() > 1e-7 * np.abs(ext).max()   # the term is there
    ctx = make_ctx(n, s=16, bulge=bulge)
    x, v = d["pos"].copy(), d["vel"].copy()
    try:
        for _ in range(3):
            ncorp.ncorp_step(ctx, x, v, d["mass"], d["radius"], n, 3, 0.5, dt)
    finally:
        ncorp.ncorp_free(ctx)
    Pk = oracle.params(p=3, bulge=bulge, leaf_size=16, gravity_thresholds=(64, 8, 64))
    xo, vo, _, _ = oracle.kdk(Pk, d["pos"], d["vel"], d["mass"], d["radius"], dt, 3)
    np.testing.assert_allclose(x, xo, rtol=0, atol=1e-13 * np.abs(xo).max())
    np.testing.assert_allclose(v, vo, rtol=0, atol=1e-12 * np.abs(vo).max())


# ------------------------------------------------------------- collisions
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_collision_pairs_bit_exact_vs_brute_force(seed):
    n = 3000 + 500 * seed
    d = diskgen.make_disk(n, 9 + seed, a_lo=2.0, a_hi=2.5, r_lo=2e-2, r_hi=5e-2, sigma_e=0.1, sigma_i=0.05)
    ctx = make_ctx(n, s=16 + 8 * seed)
    try:
        ncorp.ncorp_collide(ctx, torch.tensor(d["pos"], device="cuda"), torch.tensor(d["vel"], device="cuda"),
                            torch.tensor(d["radius"], device="cuda"), n, 0.05)
        out = np.zeros((1 << 14, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, out, len(out))
    finally:
        ncorp.ncorp_free(ctx)
    brute = oracle.collide_brute(d["pos"], d["vel"], d["radius"], 0.05)
    assert len(brute) > 10
    assert np.array_equal(out[:k], brute)


def test_collision_pairs_host_buffers_and_overflow_report():
    n = 3000
    d = diskgen.make_disk(n, 9, a_lo=2.0, a_hi=2.5, r_lo=2e-2, r_hi=5e-2, sigma_e=0.1, sigma_i=0.05)
    ctx = make_ctx(n)
    try:
        ncorp.ncorp_collide(ctx, d["pos"], d["vel"], d["radius"], n, 0.05)
        small = np.zeros((3, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, small, 3)
    finally:
        ncorp.ncorp_free(ctx)
    brute = oracle.collide_brute(d["pos"], d["vel"], d["radius"], 0.05)
    assert k == len(brute) and np.array_equal(small, brute[:3])


# ------------------------------------------------------------------ KDK
def test_kdk_steps_match_oracle_fp64():
    n, p, theta, s, dt, steps = 2500, 3, 0.5, 16, 0.02, 3
    d = diskgen.make_disk(n, 51, a_lo=2.0, a_hi=2.6, r_lo=1e-2, r_hi=4e-2, sigma_e=0.1, sigma_i=0.05)
    P = oracle.params(p=p, theta=theta, leaf_size=s)
    xo, vo, _, pairs_o = oracle.kdk(P, d["pos"], d["vel"], d["mass"], d["radius"], dt, steps)
    ctx = make_ctx(n, s=s)
    pos = torch.tensor(d["pos"], device="cuda")
    vel = torch.tensor(d["vel"], device="cuda")
    m = torch.tensor(d["mass"], device="cuda")
    R = torch.tensor(d["radius"], device="cuda")
    got_pairs = []
    try:
        for k in range(steps):
            ncorp.ncorp_step(ctx, pos, vel, m, R, n, p, theta, dt)
            out = np.zeros((4096, 2), dtype=np.int64)
            c = ncorp.ncorp_collisions(ctx, out, 4096)
            got_pairs += [(k, i, j) for i, j in out[:c]]
    finally:
        ncorp.ncorp_free(ctx)
    np.testing.assert_allclose(pos.cpu().numpy(), xo, rtol=0, atol=1e-12 * np.abs(xo).max())
    np.testing.assert_allclose(vel.cpu().numpy(), vo, rtol=0, atol=1e-11 * np.abs(vo).max())
    assert len(pairs_o) > 0
    assert [tuple(r) for r in pairs_o.tolist()] == got_pairs


def test_step_resident_state_and_host_arrays():
    n, p, theta, dt = 3000, 4, 0.6, 1e-3
    d = diskgen.make_disk(n, 61)
    ctx = make_ctx(n, precision=ncorp.NCORP_MIXED, s=32)
    pos, vel = d["pos"].copy(), d["vel"].copy()
    try:
        for _ in range(3):
            ncorp.ncorp_step(ctx, pos, vel, d["mass"], d["radius"], n, p, theta, dt)
        x2, v2 = np.zeros_like(pos), np.zeros_like(vel)
        ncorp.ncorp_get_state(ctx, x2, v2)
    finally:
        ncorp.ncorp_free(ctx)
    assert np.array_equal(x2, pos) and np.array_equal(v2, vel)
    P = oracle.params(p=p, theta=theta, leaf_size=32)
    xo, vo, _, _ = oracle.kdk(P, d["pos"], d["vel"], d["mass"], d["radius"], dt, 3)
    assert np.abs(pos - xo).max() < 1e-9
    assert np.abs(vel - vo).max() < 1e-8


# ------------------------------------------------------------- edge cases
def test_single_and_two_moonlets():
    ctx = make_ctx(8)
    try:
        d = {"pos": np.array([[3.0, 0.5, 0.1]]), "mass": np.array([1e-3])}
        acc, mut, _ = gpu_accel(ctx, d, 3, 0.5)
        assert np.all(mut == 0.0)
        d = {"pos": np.array([[3.0, 0.5, 0.1], [3.1, 0.4, 0.1]]), "mass": np.array([1e-3, 2e-3])}
        acc, mut, _ = gpu_accel(ctx, d, 6, 0.5)
        ref = oracle.direct_accel(d["pos"], d["mass"])
        assert rel_err(mut, ref).max() <= 1e-14
    finally:
        ncorp.ncorp_free(ctx)


def test_coincident_and_clustered_moonlets():
    rng = np.random.default_rng(4)
    pos = np.vstack([np.repeat([[4.0, 1.0, 0.0]], 40, axis=0), rng.normal(size=(500, 3)) * 1e-9 + [5.0, 0, 0],
                     rng.normal(size=(1000, 3)) + [6.0, 0, 0]])
    m = rng.random(len(pos)) * 1e-6 + 1e-7
    d = {"pos": pos, "mass": m}
    ctx = make_ctx(len(pos), s=8)
    try:
        _, mut, st = gpu_accel(ctx, d, 4, 0.5)
        g = export_tree(ctx, len(pos))
    finally:
        ncorp.ncorp_free(ctx)
    P = oracle.params(p=4, theta=0.5, leaf_size=8)
    ref, ost = oracle.falcon_accel(P, pos, m)
    o = oracle.tree_export(P, pos, m)
    assert np.array_equal(g["cells"], o["cells"]) and st["depth"] == 21
    assert np.allclose(mut, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_equal_keys_ordered_by_caller_index_after_a_step():
    """Ties in the key order are broken by caller index (reading c4), also in
    a step, where the sort's input is the previous tree order: moonlet 0 drifts
    exactly onto moonlet 1, which preceded it in the tree order of x_0."""
    rng = np.random.default_rng(9)
    bg = rng.uniform(-3.9, 3.9, size=(200, 3))
    bg[0], bg[1] = [-4, -4, -4], [4, 4, 4]          # root cube [-8, 8)^3, cells of side 2^-17
    h, dt = 2.0 ** -17, 2.0 ** -10
    target = np.array([0.5, 0.25, 0.125]) + h / 2    # centre of a quantisation cell
    P = oracle.params(p=3, theta=0.5, leaf_size=8)
    mass = np.full(202, 1e-30)                       # gravity negligible: the drift is exact
    for axis in range(3):
        for sgn in (1.0, -1.0):
            off = np.zeros(3)
            off[axis] = sgn * 4 * h
            pos = np.vstack([target + off, target, bg])
            keys = oracle.tree_export(P, pos, mass)["keys"]
            if keys[1] < keys[0]:
                break
        if keys[1] < keys[0]:
            break
    assert keys[1] < keys[0]
    vel = np.zeros_like(pos)
    vel[0] = -off / dt
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_FP64
    cfg.leaf_size = 8
    cfg.central_mass = 0.0
    ctx = ncorp.ncorp_init(cfg, len(pos), 0, torch.cuda.current_stream().cuda_stream)
    x, v = pos.copy(), vel.copy()
    try:
        ncorp.ncorp_step(ctx, x, v, mass, np.full(202, 1e-12), len(pos), 3, 0.5, dt)
        g = export_tree(ctx, len(pos))
    finally:
        ncorp.ncorp_free(ctx)
    assert np.array_equal(x[0], target) and np.array_equal(x[1], target)
    o = oracle.tree_export(P, x, mass)
    assert o["keys"][0] == o["keys"][1]
    assert np.array_equal(g["order"], o["order"])
    assert np.array_equal(g["keys"], o["keys"][o["order"]])
    assert np.array_equal(g["cells"], o["cells"])


def test_bad_arguments():
    ctx = make_ctx(16)
    try:
        x = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
        m = torch.ones(4, dtype=torch.float64, device="cuda")
        a = torch.empty_like(x)
        for p, th in ((0, 0.5), (7, 0.5), (3, 0.0), (3, 1.0)):
            with pytest.raises(ncorp.NcorpError) as e:
                ncorp.ncorp_accel(ctx, x, m, 4, p, th, a)
            assert e.value.code == ncorp.NCORP_EINVAL
        with pytest.raises(ncorp.NcorpError):
            ncorp.ncorp_step(ctx, x, x.clone(), m, m, 4, 3, 0.5, 0.0)
        x[1, 0] = float("nan")
        with pytest.raises(ncorp.NcorpError) as e:
            ncorp.ncorp_accel(ctx, x, m, 4, 3, 0.5, a)
        assert e.value.code == ncorp.NCORP_EINVAL
    finally:
        ncorp.ncorp_free(ctx)


def test_context_grows_beyond_initial_capacity():
    n = 30000
    d = diskgen.make_disk(n, 71)
    ctx = make_ctx(100, s=16)
    try:
        _, mut, _ = gpu_accel(ctx, d, 3, 0.5)
    finally:
        ncorp.ncorp_free(ctx)
    ref, _ = oracle.falcon_accel(oracle.params(p=3, theta=0.5, leaf_size=16), d["pos"], d["mass"])
    assert rel_err(mut, ref).max() <= FP64_TOL


# ------------------------------------------------- per-stage expansion parity
def _oracle_multi(P, pos, mass):
    M, Cc = oracle.expansions(P, pos, mass)
    p = P.p
    Mm = [np.concatenate([oracle.full_to_multi(row[oracle.off(n):oracle.off(n + 1)], n) for n in range(p) if n != 1])
          for row in M]
    Cm = [np.concatenate([oracle.full_to_multi(row[oracle.off(n):oracle.off(n + 1)], n) for n in range(1, p + 1)])
          for row in Cc]
    return np.array(Mm), np.array(Cm)


@pytest.mark.parametrize("p,prec,tol", [(4, ncorp.NCORP_FP64, 1e-12), (6, ncorp.NCORP_FP64, 1e-12),
                                        (6, ncorp.NCORP_MIXED, 3e-5)])
def test_multipoles_and_local_expansions_match_oracle(p, prec, tol):
    """P2M + M2M (Eq. multipole_moment, App. C) and the complete local expansion
    of each cell (M2L of Eq. phi_expanded + descent of Eq. shifting) against the
    oracle's full-tensor versions."""
    n, s = 4000, 24
    grav = (64, 8, 64)
    d = diskgen.make_disk(n, 81 + p)
    ctx = make_ctx(n, precision=prec, s=s, grav=grav)
    try:
        gpu_accel(ctx, d, p, 0.5)
        cap = 4 * n
        mult = np.zeros((cap, ncorp.num_m(p)))
        loc = np.zeros((cap, ncorp.num_c(p)))
        rho = np.zeros(cap)
        nc, pp = ncorp.ncorp_expansions(ctx, mult, loc, rho, cap)
    finally:
        ncorp.ncorp_free(ctx)
    P = oracle.params(p=p, theta=0.5, leaf_size=s, gravity_thresholds=grav)
    Mo, Co = _oracle_multi(P, d["pos"], d["mass"])
    assert nc == len(Mo) and pp == p
    mult, loc, rho = mult[:nc], loc[:nc], rho[:nc]
    assert np.isfinite(mult).all() and np.isfinite(loc).all()
    # compare in the scaled representation M_beta/(beta! rho^|beta|) and C_alpha rho^|alpha|, in which every
    # component of a cell is bounded by its mass (multipoles) or by its largest component (locals)
    em, ec = [], []
    for n_, (lo, hi) in [(0, (0, 1))] + [(k, (ncorp.num_m(k), ncorp.num_m(k + 1))) for k in range(2, p)]:
        f = np.array([1.0 / np.prod([math.factorial(e) for e in ab]) for ab in _exps(n_)])
        w = f[None, :] / rho[:, None] ** n_
        em.append(np.abs(mult[:, lo:hi] - Mo[:, lo:hi]) * w / Mo[:, :1])
    Cs_g, Cs_o = [], []
    for m in range(1, p + 1):
        lo, hi = ncorp.num_c(m - 1), ncorp.num_c(m)
        Cs_g.append(loc[:, lo:hi] * rho[:, None] ** m)
        Cs_o.append(Co[:, lo:hi] * rho[:, None] ** m)
    Cg, Cr = np.hstack(Cs_g), np.hstack(Cs_o)
    has = np.abs(Cr).max(axis=1) > 0
    ec = np.abs(Cg[has] - Cr[has]) / np.abs(Cr[has]).max(axis=1, keepdims=True)
    assert max(e.max() for e in em) <= tol
    assert ec.max() <= tol * 10


def _exps(n):
    return [(n - k, k - c, c) for k in range(n + 1) for c in range(k + 1)]
