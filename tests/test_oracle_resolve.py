"""Pins of the oracle's collision resolution (Sect. 5.1 elastic, 5.2 inelastic).

The impulse J = alpha (dr.dv) dr with alpha = f m1 m2 / ((m1 + m2)(R1 + R2)^2)
is checked against what mechanics fixes independently of its formula: the
textbook 1-D restitution law (coefficient of restitution e = f - 1), momentum
conservation, the unchanged tangential relative velocity, the reversal of the
normal relative velocity by the factor (1 - f), the kinetic energy change
(f (f - 2) / 2) mu (dv.n)^2 of a hard-sphere impact with that restitution,
contact at the impact time (|dr| = R1 + R2), and a trajectory that passes
through the impact point.  The multi-pair policy (one impact per moonlet per
step, earliest first, ties by index) is pinned on crafted lines of moonlets,
and the KDK step with resolution on the tree search against the same step on
the brute-force search.

Gravity is made negligible in the KDK cases (central mass 0, moonlet masses
of order 1e-30 in G = 1 units), so a step is a pure drift plus resolution.
"""
import numpy as np
import pytest

import oracle


def drift_params(f, brute=True, leaf_size=4):
    return oracle.params(p=3, theta=0.5, leaf_size=leaf_size, G=1.0, central_mass=0.0,
                         brute_collisions=brute, resolve_f=f)


def one_step(f, pos, vel, m, R, dt, brute=True):
    info = {}
    x, v, _, pairs = oracle.kdk(drift_params(f, brute), pos, vel, m, R, dt, 1, info=info)
    return x, v, pairs[:, 1:], info["resolved"]


def test_head_on_equal_masses_exchange_velocities_exactly():
    # dyadic inputs: every operation of the step is exact
    pos = np.array([[5.0, 0, 0], [6.0, 0, 0]])
    vel = np.array([[1.0, 0, 0], [-1.0, 0, 0]])
    m, R = np.array([1e-30, 1e-30]), np.array([0.25, 0.25])
    x, v, pairs, nres = one_step(2.0, pos, vel, m, R, 0.5)
    # contact at t = 0.25 (gap 0.5 closed at relative speed 2), then back out for 0.25
    assert nres == 1 and pairs.tolist() == [[0, 1]]
    assert np.array_equal(v, [[-1.0, 0, 0], [1.0, 0, 0]])
    assert np.array_equal(x, pos)


@pytest.mark.parametrize("f", [1.0, 1.3, 1.75, 2.0])
def test_head_on_follows_the_restitution_law(f):
    m1, m2, u1, u2 = 3e-30, 1e-30, 0.7, -0.4
    pos = np.array([[4.0, 1.0, 0.5], [4.6, 1.0, 0.5]])
    vel = np.array([[u1, 0, 0], [u2, 0, 0]])
    x, v, pairs, nres = one_step(f, pos, vel, np.array([m1, m2]), np.array([0.1, 0.2]), 1.0)
    e = f - 1.0
    w1 = (m1 * u1 + m2 * u2 - m2 * e * (u1 - u2)) / (m1 + m2)
    w2 = (m1 * u1 + m2 * u2 + m1 * e * (u1 - u2)) / (m1 + m2)
    assert nres == 1
    np.testing.assert_allclose(v[:, 0], [w1, w2], rtol=1e-14, atol=1e-15)
    assert np.all(v[:, 1:] == 0.0)
    # contact after the gap 0.3 closes at speed 1.1; then the new velocities for the rest of the step
    tc = 0.3 / 1.1
    np.testing.assert_allclose(x[:, 0], [4.0 + tc * u1 + (1.0 - tc) * w1, 4.6 + tc * u2 + (1.0 - tc) * w2],
                               rtol=1e-14)


def random_impacts(seed, count):
    """Pairs of moonlets on straight-line courses that touch within dt = 1."""
    rng = np.random.default_rng(seed)
    cases = []
    while len(cases) < count:
        R1, R2 = rng.uniform(0.05, 0.3, 2)
        m1, m2 = rng.uniform(0.1, 5.0, 2)
        v1, v2 = rng.normal(size=3), rng.normal(size=3)
        x1 = rng.normal(size=3) * 3.0
        dv = v1 - v2
        # place moonlet 2 so the relative motion reaches contact at t0 in (0, 1) with impact parameter b
        t0 = rng.uniform(0.1, 0.9)
        n = rng.normal(size=3)
        n -= n.dot(dv) / dv.dot(dv) * dv
        n /= np.linalg.norm(n)
        b = rng.uniform(0.0, 0.95) * (R1 + R2)
        along = np.sqrt((R1 + R2) ** 2 - b * b)
        dr_contact = b * n - along * dv / np.linalg.norm(dv)      # r1 - r2 at contact, approaching
        x2 = x1 + t0 * v1 - t0 * v2 - dr_contact
        cases.append((np.array([x1, x2]), np.array([v1, v2]), np.array([m1, m2]), np.array([R1, R2])))
    return cases


@pytest.mark.parametrize("f", [1.0, 1.5, 2.0])
def test_oblique_impacts_conserve_momentum_and_follow_the_hard_sphere_laws(f):
    for pos, vel, m, R in random_impacts(11 + int(10 * f), 50):
        assert oracle.collide_pair(pos[0], vel[0], R[0], pos[1], vel[1], R[1], 1.0)
        xs, w, done = oracle.resolve(pos, vel, m, R, f, np.array([[0, 1]]))
        assert done.tolist() == [True]
        # the impact: the trajectory x_start + t w passes through the impact point x + t_c v
        dv = vel[0] - vel[1]
        dr0 = pos[0] - pos[1]
        tc = (-(dr0 @ dv) - np.sqrt((dr0 @ dv) ** 2 - dv @ dv * (dr0 @ dr0 - (R[0] + R[1]) ** 2))) / (dv @ dv)
        hit = pos + tc * vel
        np.testing.assert_allclose(xs + tc * w, hit, rtol=0, atol=1e-13 * np.abs(hit).max())
        dr = hit[0] - hit[1]
        assert abs(np.linalg.norm(dr) - (R[0] + R[1])) <= 1e-12
        nh = dr / np.linalg.norm(dr)
        dw = w[0] - w[1]
        P0, P1 = m @ vel, m @ w
        np.testing.assert_allclose(P1, P0, rtol=0, atol=1e-14 * np.abs(m[:, None] * vel).max())
        # tangential relative velocity unchanged, normal one reversed by (1 - f)
        np.testing.assert_allclose(dw - (dw @ nh) * nh, dv - (dv @ nh) * nh, rtol=0, atol=1e-13)
        # (|dr| at the computed impact equals R1 + R2 only to a few 1e-14 after the cancellations)
        np.testing.assert_allclose(dw @ nh, (1.0 - f) * (dv @ nh), rtol=0, atol=2e-13 * np.linalg.norm(dv))
        # kinetic energy change of a hard-sphere impact with restitution e = f - 1
        mu = m[0] * m[1] / (m[0] + m[1])
        dE = 0.5 * (m @ (w * w).sum(1) - m @ (vel * vel).sum(1))
        np.testing.assert_allclose(dE, 0.5 * f * (f - 2.0) * mu * (dv @ nh) ** 2, rtol=0,
                                   atol=1e-13 * (m @ (vel * vel).sum(1)))


def test_one_impact_per_moonlet_the_earliest():
    # a line of three moonlets: (1, 2) touch at t = 0.2, (0, 1) at t = 0.3, (0, 2) at t = 0.35
    pos = np.array([[10.0, 0, 0], [10.5, 0, 0], [10.9, 0, 0]])
    vel = np.array([[1.0, 0, 0], [0.0, 0, 0], [-1.0, 0, 0]])
    m, R = np.full(3, 1e-30), np.full(3, 0.1)
    x, v, pairs, nres = one_step(2.0, pos, vel, m, R, 0.5)
    assert pairs.tolist() == [[0, 1], [0, 2], [1, 2]]     # all three are reported
    assert nres == 1                                      # only the earliest is resolved
    np.testing.assert_allclose(v[:, 0], [1.0, -1.0, 0.0], rtol=0, atol=1e-13)   # 10.9 is not dyadic
    np.testing.assert_allclose(x[:, 0], [10.5, 10.5 - 0.3, 10.9 - 0.2], rtol=1e-14)
    _, _, done = oracle.resolve(pos, vel, m, R, 2.0, pairs)
    assert done.tolist() == [False, False, True]


def test_equal_impact_times_go_to_the_lower_indices():
    # moonlet 1 at rest between 0 and 2, which approach it symmetrically: t_c(0,1) = t_c(1,2) = 0.25,
    # t_c(0,2) = 0.375
    pos = np.array([[7.0, 0, 0], [8.0, 0, 0], [9.0, 0, 0]])
    vel = np.array([[2.0, 0, 0], [0.0, 0, 0], [-2.0, 0, 0]])
    m, R = np.full(3, 1e-30), np.full(3, 0.25)
    x, v, pairs, nres = one_step(2.0, pos, vel, m, R, 0.5)
    assert pairs.tolist() == [[0, 1], [0, 2], [1, 2]] and nres == 1
    # (moonlet 0 is left at rest but for the ~1e-30 gravity of its neighbours)
    np.testing.assert_allclose(v[:, 0], [0.0, 2.0, -2.0], rtol=0, atol=1e-25)
    assert np.array_equal(x[:, 0], [7.5, 8.5, 8.0])


def test_non_colliding_or_invalid_rows_are_skipped():
    pos = np.array([[1.0, 0, 0], [3.0, 0, 0]])
    vel = np.array([[0.0, 0, 0], [0.0, 0, 0]])     # dv = 0: no impact time
    xs, w, done = oracle.resolve(pos, vel, np.ones(2), np.full(2, 0.1), 2.0, np.array([[0, 1], [1, 0], [0, 5]]))
    assert done.tolist() == [False, False, False]
    assert np.array_equal(xs, pos) and np.array_equal(w, vel)


def clump(seed, n):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-1.0, 1.0, (n, 3)) + np.array([20.0, 0.0, 0.0])
    vel = rng.normal(size=(n, 3)) * 0.5
    return pos, vel, rng.uniform(0.5, 2.0, n) * 1e-30, rng.uniform(0.05, 0.12, n)


@pytest.mark.parametrize("f", [1.2, 2.0])
def test_kdk_resolution_on_the_tree_search_equals_the_brute_force_one(f):
    pos, vel, m, R = clump(5, 300)
    out = []
    for brute in (True, False):
        info = {}
        x, v, _, pairs = oracle.kdk(drift_params(f, brute), pos, vel, m, R, 0.1, 3, info=info)
        out.append((x, v, pairs, info["resolved"]))
    (xb, vb, pb, nb), (xt, vt, pt, nt) = out
    assert nb == nt and nb > 20
    assert np.array_equal(pb, pt)
    assert np.array_equal(xb, xt) and np.array_equal(vb, vt)
    # more pairs than impacts: the one-per-moonlet rule was exercised
    assert len(pb) > nb


def test_kdk_with_resolution_conserves_momentum_and_elastic_energy():
    pos, vel, m, R = clump(6, 200)
    info = {}
    x, v, _, pairs = oracle.kdk(drift_params(2.0), pos, vel, m, R, 0.1, 4, info=info)
    assert info["resolved"] > 10
    np.testing.assert_allclose(m @ v, m @ vel, rtol=0, atol=1e-14 * np.abs(m @ np.abs(vel)).max())
    E0, E1 = m @ (vel * vel).sum(1), m @ (v * v).sum(1)
    assert abs(E1 - E0) <= 1e-13 * E0


def test_kdk_without_resolution_is_unchanged():
    pos, vel, m, R = clump(7, 150)
    x0, v0, _, p0 = oracle.kdk(drift_params(0.0), pos, vel, m, R, 0.1, 2)
    # with f = 0 the pairs are found but the moonlets pass through each other: a pure drift
    xd = pos.copy()
    for _ in range(2):
        xd = xd + 0.1 * vel
    assert len(p0) > 0
    np.testing.assert_allclose(x0, xd, rtol=0, atol=1e-14)
    np.testing.assert_allclose(v0, vel, rtol=0, atol=1e-14)


def test_self_gravitating_clump_with_resolution_conserves_momentum():
    """falcON's mutual forces come in equal and opposite pairs (symmetric M2L
    and P2P) and every impulse is +-J: with no central body the total momentum
    of a self-gravitating clump with impacts stays at its initial value."""
    rng = np.random.default_rng(8)
    n = 400
    pos = rng.uniform(-1.0, 1.0, (n, 3))
    vel = rng.normal(size=(n, 3)) * 0.3
    m = rng.uniform(0.5, 2.0, n) * 1e-4
    R = rng.uniform(0.03, 0.08, n)
    P = oracle.params(p=4, theta=0.5, leaf_size=8, G=1.0, central_mass=0.0, resolve_f=1.5)
    info = {}
    x, v, _, pairs = oracle.kdk(P, pos, vel, m, R, 0.02, 5, info=info)
    assert info["resolved"] > 20 and len(pairs) >= info["resolved"]
    p0, p1 = m @ vel, m @ v
    assert np.abs(p1 - p0).max() <= 1e-12 * (m @ np.linalg.norm(vel, axis=1))
    assert np.all(np.isfinite(x)) and not np.array_equal(v, vel)
