"""Pins of the oracle's standard tree code (Algorithm StandardTree, Sect. 3.4.4).

M2P (a cell's expansion evaluated at a moonlet) is pinned against the
symmetric M2L of the oracle (itself pinned) with the target reduced to a
point, and against the direct sum it converges to as p grows.  The whole
algorithm reduces to direct summation when nothing can be well separated (a
vanishing opening angle, or N_cb,pre above N), its error against direct
summation falls with p, and it is of the order of falcON's at the same p and
theta_min (Fig. 4 caption: the errors are similar).
"""
import numpy as np
import pytest

import oracle
from paper_2310_20374_gb300 import diskgen


def cluster(seed, n, radius=0.3):
    rng = np.random.default_rng(seed)
    pos = rng.normal(size=(n, 3)) * radius
    mu = rng.uniform(0.5, 1.5, n)
    s = (mu[:, None] * pos).sum(0) / mu.sum()
    return pos, mu, s


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_m2p_is_the_point_target_m2l(p):
    pos, mu, s = cluster(1, 40)
    M = oracle.p2m(p, pos, mu, s)
    x = np.array([3.0, -2.0, 1.5])
    got = oracle.m2p(p, x, s, M)
    # a target cell reduced to a point: monopole only, expansion about x itself
    MA = np.zeros(oracle.off(p))
    MA[0] = 1.0
    CA, _ = oracle.m2l(p, x, MA, s, M)
    np.testing.assert_allclose(got, CA[oracle.off(1):oracle.off(2)], rtol=1e-13, atol=0)


def test_m2p_converges_to_the_direct_pull():
    pos, mu, s = cluster(2, 60)
    x = np.array([2.0, 1.0, -0.5])
    direct = -(mu[:, None] * (x - pos) / np.linalg.norm(x - pos, axis=1)[:, None] ** 3).sum(0)
    errs = []
    for p in range(1, 7):
        M = oracle.p2m(p, pos, mu, s)
        errs.append(np.linalg.norm(oracle.m2p(p, x, s, M) - direct) / np.linalg.norm(direct))
    # the multipole series converges like (r_max / R)^p with r_max / R ~ 0.4
    assert all(b < 0.8 * a for a, b in zip(errs[1:], errs[2:])), errs
    assert errs[-1] < 1e-3


def disk(n, seed=3):
    d = diskgen.make_disk(n, seed)
    return d["pos"], d["mass"]


def test_nothing_separated_is_direct_summation():
    pos, m = disk(1200)
    ref = oracle.direct_accel(pos, m)
    # a vanishing opening angle: r_crit = r_max / theta(M) covers the disk
    a1, st1 = oracle.standard_accel(oracle.params(p=3, theta=1e-6, leaf_size=16), pos, m)
    # N_cb,pre above N: brute force from the root
    a2, st2 = oracle.standard_accel(oracle.params(p=3, leaf_size=16, standard_thresholds=(10**9, 16)), pos, m)
    scale = np.linalg.norm(ref, axis=1)
    for a, st in ((a1, st1), (a2, st2)):
        assert st["m2l"] == 0
        assert st["p2p_interactions"] == len(pos) ** 2
        assert (np.linalg.norm(a - ref, axis=1) / scale).max() < 1e-12


def rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


def test_error_falls_with_p_to_the_papers_orders():
    pos, m = disk(2000, 4)
    ref = oracle.direct_accel(pos, m)
    med = []
    for p in range(1, 7):
        a, st = oracle.standard_accel(oracle.params(p=p, theta=0.5, leaf_size=16), pos, m)
        assert st["m2l"] > 0 and st["p2p_pairs"] > 0
        med.append(np.median(rel_err(a, ref)))
    # p = 2 adds nothing at a point (the dipole about the barycentre vanishes); beyond, every order helps
    assert med[1] == med[0] and all(b < 0.8 * a for a, b in zip(med[1:], med[2:])), med
    # (the paper's ~1e-5 at p = 3 is for 4e5 moonlets; mutual accelerations of a 2000-moonlet disk
    # cancel more, and falcON's own median error here is ~2e-3 at p = 3)
    assert med[2] < 1e-2 and med[5] < 1e-3, med


def test_thresholds_only_move_work_between_branches():
    pos, m = disk(1500, 5)
    ref = oracle.direct_accel(pos, m)
    out = []
    for th in ((0, 0), (6, 16), (32, 128)):
        a, st = oracle.standard_accel(oracle.params(p=4, theta=0.5, leaf_size=16, standard_thresholds=th), pos, m)
        out.append((np.median(rel_err(a, ref)), st["m2l"], st["p2p_interactions"]))
    # more brute force with larger thresholds: fewer expansions, more direct pairs, no larger error
    assert out[0][1] > out[1][1] > out[2][1]
    assert out[0][2] < out[1][2] < out[2][2]
    assert out[2][0] <= out[0][0] * 1.01


def test_errors_similar_to_falcon():
    pos, m = disk(2000, 6)
    ref = oracle.direct_accel(pos, m)
    P = oracle.params(p=3, theta=0.5, leaf_size=16)
    e_std = np.median(rel_err(oracle.standard_accel(P, pos, m)[0], ref))
    e_fal = np.median(rel_err(oracle.falcon_accel(P, pos, m)[0], ref))
    assert 0.1 < e_std / e_fal < 10.0, (e_std, e_fal)


@pytest.mark.parametrize("thresholds", [(0, 16), (0, 0), (8, 64)])
def test_standard_collision_search_equals_brute_force(thresholds):
    """The collision variant of StandardTree prunes only cells no moonlet of
    which can reach a within the step, and tests each pair from its lower
    index: the pair set is the brute-force one, on random sets and a dense
    ring, at any thresholds."""
    P = oracle.params(p=3, leaf_size=6, standard_collision_thresholds=thresholds)
    for seed in range(6):
        rng = np.random.default_rng(100 + seed)
        n = 300
        pos = rng.uniform(-1.0, 1.0, (n, 3))
        vel = rng.normal(size=(n, 3))
        rad = rng.uniform(0.01, 0.05, n)
        got, st = oracle.collide_standard(P, pos, vel, rad, 0.05)
        ref = oracle.collide_brute(pos, vel, rad, 0.05)
        assert np.array_equal(got, ref)
        assert st["col_tests"] < n * (n - 1) // 2 or thresholds[0] > n
    d = diskgen.make_disk(4000, 9, a_lo=2.0, a_hi=2.5, r_lo=2e-2, r_hi=5e-2, sigma_e=0.1, sigma_i=0.05)
    got, st = oracle.collide_standard(P, d["pos"], d["vel"], d["radius"], 0.05)
    ref = oracle.collide_brute(d["pos"], d["vel"], d["radius"], 0.05)
    tree, _ = oracle.collide_tree(P, d["pos"], d["vel"], d["radius"], 0.05)
    assert len(ref) > 10 and np.array_equal(got, ref) and np.array_equal(tree, ref)
    assert st["col_tests"] < 4000 * 3999 // 20
