"""Standard tree code (ncorp_accel_standard, Algorithm StandardTree) against the oracle (needs a GB300).

The walk decisions are taken in FP64 on both sides, so the counters (moonlet-
cell expansions, direct sums, direct pairs) must be equal, and the FP64
accelerations agree to the rounding of the sums (1e-11 relative, per moonlet,
mutual part).  Mixed precision (FP32 expansions and direct sums) is held to
2e-5.  With nothing separable the result is direct summation.
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


def run(pos, m, p, theta, precision, s=16, thresholds=(6, 16), G=1.0, central_mass=1.0):
    n = len(pos)
    cfg = ncorp.ncorp_config_default()
    cfg.precision = precision
    cfg.leaf_size = s
    cfg.n_cb_pre, cfg.n_cb_post = thresholds
    cfg.G, cfg.central_mass = G, central_mass
    ctx = ncorp.ncorp_init(cfg, n, 0, torch.cuda.current_stream().cuda_stream)
    acc, mut = np.zeros((n, 3)), np.zeros((n, 3))
    try:
        ncorp.ncorp_accel_standard(ctx, pos, m, n, p, theta, acc, mut)
        st = ncorp.ncorp_stats(ctx)
    finally:
        ncorp.ncorp_free(ctx)
    return acc, mut, st


def rel(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("p,n,seed", [(3, 20011, 21), (6, 5003, 22), (1, 3001, 23)])
def test_fp64_equals_oracle(p, n, seed):
    d = diskgen.make_disk(n, seed)
    P = oracle.params(p=p, theta=0.5, leaf_size=16)
    ref, ost = oracle.standard_accel(P, d["pos"], d["mass"])
    acc, mut, st = run(d["pos"], d["mass"], p, 0.5, ncorp.NCORP_FP64)
    assert (st["m2l"], st["p2p_pairs"], st["p2p_interactions"]) == (ost["m2l"], ost["p2p_pairs"],
                                                                     ost["p2p_interactions"])
    assert st["m2l"] > 0 and st["p2p_pairs"] > 0
    assert rel(mut, ref).max() <= 1e-11
    ext = oracle.external_accel(oracle.params(), d["pos"])
    np.testing.assert_allclose(acc, mut + ext, rtol=0, atol=1e-13 * np.abs(ext).max())


@pytest.mark.parametrize("p,n", [(3, 30011), (6, 8009)])
def test_mixed_within_2e5(p, n):
    d = diskgen.make_disk(n, 24)
    P = oracle.params(p=p, theta=0.5, leaf_size=32)
    ref, ost = oracle.standard_accel(P, d["pos"], d["mass"])
    _, mut, st = run(d["pos"], d["mass"], p, 0.5, ncorp.NCORP_MIXED, s=32)
    assert st["m2l"] == ost["m2l"] and st["p2p_interactions"] == ost["p2p_interactions"]
    e = rel(mut, ref)
    assert e.max() <= 2e-5, (e.max(), np.median(e))


@pytest.mark.parametrize("thresholds", [(0, 0), (40, 200)])
def test_thresholds_match_oracle(thresholds):
    d = diskgen.make_disk(8009, 25)
    P = oracle.params(p=4, theta=0.6, leaf_size=8, standard_thresholds=thresholds)
    ref, ost = oracle.standard_accel(P, d["pos"], d["mass"])
    _, mut, st = run(d["pos"], d["mass"], 4, 0.6, ncorp.NCORP_FP64, s=8, thresholds=thresholds)
    assert (st["m2l"], st["p2p_pairs"], st["p2p_interactions"]) == (ost["m2l"], ost["p2p_pairs"],
                                                                     ost["p2p_interactions"])
    assert rel(mut, ref).max() <= 1e-11


def test_nothing_separable_is_direct_summation_and_tiny_inputs():
    d = diskgen.make_disk(3001, 26)
    ref = oracle.direct_accel(d["pos"], d["mass"])
    _, mut, st = run(d["pos"], d["mass"], 3, 0.5, ncorp.NCORP_FP64, thresholds=(10 ** 9, 16))
    assert st["m2l"] == 0 and st["p2p_interactions"] == 3001 ** 2
    assert rel(mut, ref).max() <= 1e-12
    # one moonlet: no mutual force; two: the closed form
    one = run(np.array([[3.0, 0.5, 0.1]]), np.array([1e-3]), 3, 0.5, ncorp.NCORP_FP64)[1]
    assert np.all(one == 0.0)
    x = np.array([[3.0, 0.0, 0.0], [3.5, 0.0, 0.0]])
    two = run(x, np.array([2e-3, 1e-3]), 3, 0.5, ncorp.NCORP_FP64)[1]
    np.testing.assert_allclose(two, [[1e-3 / 0.25, 0, 0], [-2e-3 / 0.25, 0, 0]], rtol=1e-14, atol=1e-20)


def test_standard_and_falcon_agree_to_their_errors():
    """Both approximate the same direct sum: on a 20k disk at p = 6 (mixed
    precision) the median error of each against direct summation stays small."""
    d = diskgen.make_disk(20011, 27)
    n = len(d["pos"])
    idx = np.random.default_rng(1).choice(n, 500, replace=False)
    ref = oracle.direct_accel(d["pos"], d["mass"], targets=idx)
    _, mut_s, _ = run(d["pos"], d["mass"], 6, 0.5, ncorp.NCORP_MIXED)
    cfg = ncorp.ncorp_config_default()
    ctx = ncorp.ncorp_init(cfg, n, 0, torch.cuda.current_stream().cuda_stream)
    acc, mut_f = np.zeros((n, 3)), np.zeros((n, 3))
    try:
        ncorp.ncorp_accel(ctx, d["pos"], d["mass"], n, 6, 0.5, acc, mut_f)
    finally:
        ncorp.ncorp_free(ctx)
    e_s, e_f = np.median(rel(mut_s[idx], ref)), np.median(rel(mut_f[idx], ref))
    assert e_s < 1e-2 and e_f < 1e-2, (e_s, e_f)


# ---------------------------------------------------------------- collision search (StandardTree)
def collide_standard(d, dt, s=16, thresholds=(0, 16)):
    n = len(d["pos"])
    cfg = ncorp.ncorp_config_default()
    cfg.leaf_size = s
    cfg.c_cb_pre, cfg.c_cb_post = thresholds
    ctx = ncorp.ncorp_init(cfg, n, 0, torch.cuda.current_stream().cuda_stream)
    try:
        ncorp.ncorp_collide_standard(ctx, d["pos"], d["vel"], d["radius"], n, dt)
        pairs = np.zeros((1 << 15, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, pairs, len(pairs))
        st = ncorp.ncorp_stats(ctx)
    finally:
        ncorp.ncorp_free(ctx)
    return pairs[:k], st


@pytest.mark.parametrize("n,seed,dense,thresholds", [(4000, 31, True, (0, 16)), (3000, 32, True, (6, 40)),
                                                     (20000, 33, False, (0, 16))])
def test_collision_search_equals_oracle_and_brute_force(n, seed, dense, thresholds):
    """Algorithm StandardTree's collision search on the GPU: the same pair set as the oracle's tree search
    and as brute force (bit-exact), the same direct-search decisions and tested pairs as the oracle.  The
    wide disk has moonlets ten times larger than the workloads' so that it has pairs to find."""
    if dense:
        d = diskgen.make_disk(n, seed, a_lo=2.0, a_hi=2.5, r_lo=2e-2, r_hi=5e-2, sigma_e=0.1, sigma_i=0.05)
    else:
        d = diskgen.make_disk(n, seed, r_lo=1e-2, r_hi=1e-1)
    dt = 0.05
    got, st = collide_standard(d, dt, thresholds=thresholds)
    P = oracle.params(p=3, theta=0.5, leaf_size=16, standard_collision_thresholds=thresholds)
    ref, ost = oracle.collide_standard(P, d["pos"], d["vel"], d["radius"], dt)
    assert len(ref) > 0 and np.array_equal(got, ref)
    assert np.array_equal(got, oracle.collide_brute(d["pos"], d["vel"], d["radius"], dt))
    assert (st["col_pairs"], st["col_tests"]) == (ost["col_pairs"], ost["col_tests"])


def test_collision_search_matches_dual_walk():
    d = diskgen.make_disk(6000, 34, a_lo=2.0, a_hi=2.5, r_lo=2e-2, r_hi=5e-2, sigma_e=0.1, sigma_i=0.05)
    got, _ = collide_standard(d, 0.05)
    cfg = ncorp.ncorp_config_default()
    cfg.leaf_size = 16
    ctx = ncorp.ncorp_init(cfg, len(d["pos"]), 0, torch.cuda.current_stream().cuda_stream)
    try:
        ncorp.ncorp_collide(ctx, d["pos"], d["vel"], d["radius"], len(d["pos"]), 0.05)
        pairs = np.zeros((1 << 15, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, pairs, len(pairs))
    finally:
        ncorp.ncorp_free(ctx)
    assert np.array_equal(got, pairs[:k])
