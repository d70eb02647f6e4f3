"""Exact pins of the oracle's tree climbing (Sect. 3.4.2).

The oracle climbs the tree recursively in C.  These tests recompute every
cell's geometry from the moonlets and the exported cell list alone, in numpy,
without calling the oracle's climb:

  gravity   (Eqs. expansion_center, rmax_2, rcrit_2):
    s_A = sum_a M_a s_a / M_A over the children (the moonlets' barycentre),
    r_max,A = max_a (r_max,a + |s_a - s_A|) over the children (a moonlet has
    r_max = 0), then replaced by the distance from s_A to the farthest corner
    of A's cube when that is smaller (the corner cap), and
    r_crit,A = r_max,A / theta(M_A) with Dehnen's law
    theta^5 / (1 - theta)^2 = theta_min^5 / (1 - theta_min)^2 (M_A / M_tot)^(-1/3);
  collisions (Eqs. center, rmax, rcrit): the same with the moonlets' mean
    position and r_crit = r_max + max over the members of (R + dt |v|).

The farthest corner is found by enumerating the cube's eight corners (the
oracle uses a per-axis form); the cube is the cell's integer cube widened by
L 2^-48 on each side (reading c8).  theta is found by scipy's root finder,
not the oracle's bisection and Newton steps.  Every cell is compared to a
few ulps, and a crafted cell checks that the cap binds where it must.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

from paper_2310_20374_gb300 import diskgen

pytestmark = pytest.mark.filterwarnings("ignore")


def children(cells):
    where = {(int(c[0]), int(c[1]), int(c[2]), int(c[3])): k for k, c in enumerate(cells)}
    kids = [[] for _ in cells]
    for k, (lv, cx, cy, cz, first, cnt, nch) in enumerate(cells):
        if lv > 0:
            kids[where[(int(lv) - 1, int(cx) >> 1, int(cy) >> 1, int(cz) >> 1)]].append(k)
    return kids


def farthest_corner(root, cell, s):
    lv, cx, cy, cz = (int(v) for v in cell[:4])
    L = root[3]
    h = L / 2.0 ** lv
    eps = L * 2.0 ** -48
    lo = root[:3] + np.array([cx, cy, cz], dtype=np.float64) * h - eps
    hi = root[:3] + np.array([cx, cy, cz], dtype=np.float64) * h + h + eps
    corners = np.array([[(lo, hi)[i][0], (lo, hi)[j][1], (lo, hi)[k][2]]
                        for i in (0, 1) for j in (0, 1) for k in (0, 1)])
    return np.linalg.norm(corners - s, axis=1).max()


def dehnen_theta(M, Mtot, theta_min):
    K = theta_min ** 5 / (1.0 - theta_min) ** 2 * (M / Mtot) ** (-1.0 / 3.0)
    if M >= Mtot:
        return theta_min
    return brentq(lambda t: t ** 5 / (1.0 - t) ** 2 - K, theta_min, 1.0 - 1e-15, xtol=1e-17, rtol=8.9e-16)


def recompute(t, pos, m, vel, R, dt, theta_min):
    """numpy geometry of every cell, bottom-up over the exported cells, and
    whether the corner cap decided r_max (gravity, collisions)."""
    cells, order, root = t["cells"], t["order"], t["root"]
    kids = children(cells)
    nc = len(cells)
    M = np.zeros(nc)
    s = np.zeros((nc, 3))
    rmax = np.zeros(nc)
    sb = np.zeros((nc, 3))
    rmax_c = np.zeros(nc)
    reach = np.zeros(nc)
    capped = np.zeros(nc, bool)
    capped_c = np.zeros(nc, bool)
    for k in np.argsort(-cells[:, 0], kind="stable"):   # deepest level first
        first, cnt = int(cells[k, 4]), int(cells[k, 5])
        idx = order[first:first + cnt]
        if not kids[k]:   # a leaf: its moonlets are the children (r_max = 0)
            M[k] = m[idx].sum()
            s[k] = (m[idx, None] * pos[idx]).sum(0) / M[k]
            rec = np.linalg.norm(pos[idx] - s[k], axis=1).max()
            sb[k] = pos[idx].sum(0) / cnt
            rec_c = np.linalg.norm(pos[idx] - sb[k], axis=1).max()
            reach[k] = (R[idx] + dt * np.linalg.norm(vel[idx], axis=1)).max()
        else:
            ch = np.array(kids[k])
            M[k] = M[ch].sum()
            s[k] = (M[ch, None] * s[ch]).sum(0) / M[k]
            rec = (rmax[ch] + np.linalg.norm(s[ch] - s[k], axis=1)).max()
            w = cells[ch, 5].astype(np.float64)
            sb[k] = (w[:, None] * sb[ch]).sum(0) / cnt
            rec_c = (rmax_c[ch] + np.linalg.norm(sb[ch] - sb[k], axis=1)).max()
            reach[k] = reach[ch].max()
        cap = farthest_corner(root, cells[k], s[k])
        rmax[k] = min(rec, cap)
        capped[k] = cap < rec
        cap_c = farthest_corner(root, cells[k], sb[k])
        rmax_c[k] = min(rec_c, cap_c)
        capped_c[k] = cap_c < rec_c
    Mtot = M[0]
    rcrit = np.array([rmax[k] / dehnen_theta(M[k], Mtot, theta_min) for k in range(nc)])
    return dict(M=M, s=s, rmax=rmax, rcrit=rcrit, sb=sb, rmax_c=rmax_c, rcrit_c=rmax_c + reach,
                capped=capped, capped_c=capped_c)


def assert_close(got, want, ulps, what):
    scale = np.maximum(np.abs(want), np.finfo(np.float64).tiny)
    err = np.abs(got - want) / scale
    assert err.max() <= ulps * 2.0 ** -52, f"{what}: max relative difference {err.max():.3e}"


def check_geometry(oracle_lib, d, leaf_size, theta_min, dt):
    pos, vel, m, R = d["pos"], d["vel"], d["mass"], d["radius"]
    P = oracle_lib.params(p=3, theta=theta_min, leaf_size=leaf_size)
    t = oracle_lib.tree_export(P, pos, m, vel, R, dt)
    g, c = t["ggeo"], t["cgeo"]
    ref = recompute(t, pos, m, vel, R, dt, theta_min)
    assert_close(g[:, 0], ref["M"], 64, "M")
    span = np.abs(pos).max()
    assert np.abs(g[:, 1:4] - ref["s"]).max() <= 64 * 2.0 ** -52 * span, "s"
    assert_close(g[:, 4], ref["rmax"], 64, "r_max (gravity)")
    assert_close(g[:, 5], ref["rcrit"], 256, "r_crit (gravity)")
    assert np.abs(c[:, 0:3] - ref["sb"]).max() <= 64 * 2.0 ** -52 * span, "sbar"
    assert_close(c[:, 3], ref["rmax_c"], 64, "r_max (collisions)")
    assert_close(c[:, 4], ref["rcrit_c"], 64, "r_crit (collisions)")
    return ref


@pytest.mark.parametrize("n,seed,leaf,theta", [(3000, 21, 16, 0.5), (2500, 22, 4, 0.6), (1200, 23, 1, 0.5)])
def test_climb_equals_independent_recomputation(oracle_lib, n, seed, leaf, theta):
    d = diskgen.make_disk(n, seed)
    check_geometry(oracle_lib, d, leaf, theta, 1e-3)


def crafted_cell():
    """Eight octants of the unit cube, each a leaf of two moonlets: a heavy
    one near the cube's centre in x and y but at the octant's outer face in
    z, and a light one at the octant's outer corner, with uneven masses.
    An octant's span then points away from the root's barycentre, so Eq.
    rmax_2's recursion (the octant's r_max plus its offset from the
    barycentre) overshoots the distance to the root cube's farthest corner,
    for the barycentre (gravity) and the mean position (collisions) alike:
    the cap must decide r_max at the root."""
    pos, m = [], []
    rng = np.random.default_rng(5)
    for ox in (0, 1):
        for oy in (0, 1):
            for oz in (0, 1):
                o = np.array([ox, oy, oz], dtype=np.float64)
                heavy = 0.5 + (o - 0.5) * np.array([0.02, 0.02, 0.98])
                outer = o * 0.999 + (1 - o) * 0.001
                pos += [heavy, outer]
                m += [1.0 + 0.5 * ox + 0.25 * oy * (1 - oz) + 0.1 * rng.random(), 1e-3]
    pos = np.array(pos)
    n = len(pos)
    return {"pos": pos, "vel": np.zeros((n, 3)), "mass": np.array(m), "radius": np.full(n, 1e-3)}


def test_corner_cap_binds_in_crafted_cell(oracle_lib):
    d = crafted_cell()
    ref = check_geometry(oracle_lib, d, 2, 0.5, 1e-3)
    P = oracle_lib.params(p=3, theta=0.5, leaf_size=2)
    t = oracle_lib.tree_export(P, d["pos"], d["mass"], d["vel"], d["radius"], 1e-3)
    assert t["cells"][0, 6] == 8 and ref["capped"][0] and ref["capped_c"][0]
    # at the root, r_max is the farthest-corner distance, strictly below the recursion
    assert t["ggeo"][0, 4] == pytest.approx(farthest_corner(t["root"], t["cells"][0], ref["s"][0]), rel=1e-15)
    assert t["cgeo"][0, 3] == pytest.approx(farthest_corner(t["root"], t["cells"][0], ref["sb"][0]), rel=1e-15)
