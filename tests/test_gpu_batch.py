"""Batches of independent disks (ncorp_batch_*), needs a GB300.

Every disk of a batch must evolve as the same disk stepped alone with
ncorp_step: the batch only changes how the work is scheduled (disks of the
same (p, theta, dt) side by side in one forest, one launch per stage over
them, runs replayed from CUDA graphs, forests on separate streams), so FP64
states agree to the rounding of sums taken in another order and the
colliding pairs are the same.
"""
import numpy as np
import pytest
import torch

from paper_2310_20374_gb300 import diskgen, ncorp

pytestmark = pytest.mark.gpu

MIXED_TOL = 2e-5   # relative error of the mixed-precision mutual acceleration, per moonlet

DISKS = [  # n, p, theta, dt, seed, dense ring
    (3000, 3, 0.5, 2e-2, 61, True),
    (7000, 4, 0.6, 2e-3, 62, False),
    (1500, 6, 0.5, 2e-2, 63, True),
    (12000, 3, 0.5, 5e-4, 64, False),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def make_disk(n, seed, dense):
    if dense:
        return diskgen.make_disk(n, seed, a_lo=2.0, a_hi=2.5, r_lo=2e-2, r_hi=5e-2, sigma_e=0.1, sigma_i=0.05)
    return diskgen.make_disk(n, seed)


def config(precision=ncorp.NCORP_FP64):
    cfg = ncorp.ncorp_config_default()
    cfg.precision = precision
    cfg.leaf_size = 24
    return cfg


def single_disk_run(d, p, theta, dt, steps, leaf_size=24):
    n = len(d["pos"])
    cfg = config()
    cfg.leaf_size = leaf_size
    ctx = ncorp.ncorp_init(cfg, n, 0, torch.cuda.current_stream().cuda_stream)
    pos = torch.tensor(d["pos"], device="cuda")
    vel = torch.tensor(d["vel"], device="cuda")
    m = torch.tensor(d["mass"], device="cuda")
    R = torch.tensor(d["radius"], device="cuda")
    try:
        for _ in range(steps):
            ncorp.ncorp_step(ctx, pos, vel, m, R, n, p, theta, dt)
        pairs = np.zeros((1 << 14, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, pairs, len(pairs))
    finally:
        ncorp.ncorp_free(ctx)
    return pos.cpu().numpy(), vel.cpu().numpy(), pairs[:k]


def test_batch_disks_evolve_as_single_disks():
    disks = [make_disk(n, seed, dense) for n, _, _, _, seed, dense in DISKS]
    b = ncorp.ncorp_batch_create(config(), 0, torch.cuda.current_stream().cuda_stream)
    try:
        ids = []
        for i, ((n, p, theta, dt, _, _), d) in enumerate(zip(DISKS, disks)):
            # host arrays for some disks, device arrays for others
            if i % 2:
                args = (d["pos"], d["vel"], d["mass"], d["radius"])
            else:
                args = tuple(torch.tensor(d[k], device="cuda") for k in ("pos", "vel", "mass", "radius"))
            ids.append(ncorp.ncorp_batch_add_disk(b, *args, n, p, theta, dt))
        assert len(set(ids)) == len(ids)
        ncorp.ncorp_batch_run(b, 3)
        ncorp.ncorp_batch_run(b, 2)
        info = ncorp.ncorp_batch_info(b)
        assert info["disks"] == len(DISKS) and info["moonlets"] == sum(x[0] for x in DISKS)
        assert info["launches"] > 0 and info["forests"] == len(DISKS)
        for (n, p, theta, dt, _, dense), d, did in zip(DISKS, disks, ids):
            pos = np.zeros((n, 3))
            vel = np.zeros((n, 3))
            ncorp.ncorp_batch_get_state(b, did, pos, vel)
            pairs = np.zeros((1 << 14, 2), dtype=np.int64)
            k = ncorp.ncorp_batch_collisions(b, did, pairs, len(pairs))
            xs, vs, ps = single_disk_run(d, p, theta, dt, 5)
            np.testing.assert_allclose(pos, xs, rtol=0, atol=1e-12 * np.abs(xs).max())
            np.testing.assert_allclose(vel, vs, rtol=0, atol=1e-11 * np.abs(vs).max())
            assert np.array_equal(pairs[:k], ps)
            if dense:
                assert k > 0
        # removing a disk returns its state and leaves the others running
        out_p = torch.zeros((DISKS[0][0], 3), dtype=torch.float64, device="cuda")
        out_v = torch.zeros_like(out_p)
        ncorp.ncorp_batch_remove_disk(b, ids[0], out_p, out_v)
        xs, vs, _ = single_disk_run(disks[0], *DISKS[0][1:4], 5)
        np.testing.assert_allclose(out_p.cpu().numpy(), xs, rtol=0, atol=1e-12 * np.abs(xs).max())
        ncorp.ncorp_batch_run(b, 1)
        assert ncorp.ncorp_batch_info(b)["disks"] == len(DISKS) - 1
    finally:
        ncorp.ncorp_batch_free(b)


def batch_of(disks, p, theta, dt):
    b = ncorp.ncorp_batch_create(config(), 0, torch.cuda.current_stream().cuda_stream)
    ids = [ncorp.ncorp_batch_add_disk(b, d["pos"], d["vel"], d["mass"], d["radius"], len(d["pos"]), p, theta, dt)
           for d in disks]
    return b, ids


def check_disk(b, did, d, p, theta, dt, steps):
    n = len(d["pos"])
    pos, vel = np.zeros((n, 3)), np.zeros((n, 3))
    ncorp.ncorp_batch_get_state(b, did, pos, vel)
    pairs = np.zeros((1 << 14, 2), dtype=np.int64)
    k = ncorp.ncorp_batch_collisions(b, did, pairs, len(pairs))
    xs, vs, ps = single_disk_run(d, p, theta, dt, steps)
    np.testing.assert_allclose(pos, xs, rtol=0, atol=1e-12 * np.abs(xs).max())
    np.testing.assert_allclose(vel, vs, rtol=0, atol=1e-11 * np.abs(vs).max())
    assert np.array_equal(pairs[:k], ps)
    return k


def test_forest_of_many_disks_evolves_as_single_disks():
    """Twelve disks of mixed size with one (p, theta, dt): one forest, launches per run independent of the
    number of disks; a disk removed or added in the middle leaves the others' evolution unchanged."""
    p, theta, dt = 4, 0.5, 2e-2
    sizes = np.exp(np.random.default_rng(5).uniform(np.log(500), np.log(8000), 12)).astype(int)
    disks = [make_disk(int(n), 400 + k, k % 4 == 0) for k, n in enumerate(sizes)]
    b, ids = batch_of(disks, p, theta, dt)
    try:
        ncorp.ncorp_batch_run(b, 3)
        ncorp.ncorp_batch_run(b, 2)   # a second graph (another length), then the first one replayed
        ncorp.ncorp_batch_run(b, 3)
        info = ncorp.ncorp_batch_info(b)
        assert info["forests"] == 1 and info["disks"] == 12 and info["fallbacks"] == 0
        launches12 = info["launches"]
        found = sum(check_disk(b, did, d, p, theta, dt, 8) for did, d in zip(ids, disks))
        assert found > 0
        # remove one in the middle, add a new one: both take effect at the next run
        ncorp.ncorp_batch_remove_disk(b, ids[5])
        extra = make_disk(3000, 450, True)
        new_id = ncorp.ncorp_batch_add_disk(b, extra["pos"], extra["vel"], extra["mass"], extra["radius"], 3000, p,
                                            theta, dt)
        ncorp.ncorp_batch_run(b, 2)
        assert ncorp.ncorp_batch_info(b)["disks"] == 12
        for k in (0, 4, 6, 11):
            check_disk(b, ids[k], disks[k], p, theta, dt, 10)
        check_disk(b, new_id, extra, p, theta, dt, 2)
    finally:
        ncorp.ncorp_batch_free(b)
    # the same runs with a quarter of the disks: the same launches (one per stage, not per disk)
    b, _ = batch_of(disks[:3], p, theta, dt)
    try:
        for k in (3, 2, 3):
            ncorp.ncorp_batch_run(b, k)
        assert ncorp.ncorp_batch_info(b)["launches"] == launches12
    finally:
        ncorp.ncorp_batch_free(b)


def test_autotuned_forest_equals_single_disks_at_the_chosen_leaf_size():
    """leaf_size = 0: the tuner times candidate leaf sizes on the forest's own state and keeps one; the
    disks then evolve as single disks with that leaf size (the trials leave the state as it was)."""
    p, theta, dt, steps = 3, 0.5, 2e-2, 3
    sizes = [20000, 15000, 8000]
    disks = [make_disk(n, 470 + k, k == 0) for k, n in enumerate(sizes)]
    cfg = config()
    cfg.leaf_size = 0
    b = ncorp.ncorp_batch_create(cfg, 0, torch.cuda.current_stream().cuda_stream)
    try:
        ids = [ncorp.ncorp_batch_add_disk(b, d["pos"], d["vel"], d["mass"], d["radius"], len(d["pos"]), p, theta, dt)
               for d in disks]
        ncorp.ncorp_batch_run(b, steps)
        info = ncorp.ncorp_batch_info(b)
        assert info["tuned"] == 1 and info["leaf_size"] in (16, 24, 32, 48)
        s = info["leaf_size"]
        for did, d in zip(ids, disks):
            n = len(d["pos"])
            pos, vel = np.zeros((n, 3)), np.zeros((n, 3))
            ncorp.ncorp_batch_get_state(b, did, pos, vel)
            xs, vs, _ = single_disk_run(d, p, theta, dt, steps, leaf_size=s)
            np.testing.assert_allclose(pos, xs, rtol=0, atol=1e-12 * np.abs(xs).max())
            np.testing.assert_allclose(vel, vs, rtol=0, atol=1e-11 * np.abs(vs).max())
    finally:
        ncorp.ncorp_batch_free(b)


def test_a_full_forest_starts_another():
    """More than NCORP_MAX_DISKS disks of one (p, theta, dt): the batch starts a second forest, and a disk
    in it evolves as the same disk alone."""
    p, theta, dt = 3, 0.5, 2e-2
    disks = [diskgen.make_disk(300, 1000 + k) for k in range(ncorp.NCORP_MAX_DISKS + 3)]
    b, ids = batch_of(disks, p, theta, dt)
    try:
        ncorp.ncorp_batch_run(b, 2)
        info = ncorp.ncorp_batch_info(b)
        assert info["forests"] == 2 and info["disks"] == len(disks)
        for k in (0, ncorp.NCORP_MAX_DISKS, len(disks) - 1):
            check_disk(b, ids[k], disks[k], p, theta, dt, 2)
    finally:
        ncorp.ncorp_batch_free(b)


def test_batch_mixed_precision_runs_and_matches_single_disk():
    n, p, theta, dt = 20000, 6, 0.5, 1e-3
    d = diskgen.make_disk(n, 65)
    b = ncorp.ncorp_batch_create(config(ncorp.NCORP_MIXED), 0, torch.cuda.current_stream().cuda_stream)
    try:
        did = ncorp.ncorp_batch_add_disk(b, d["pos"], d["vel"], d["mass"], d["radius"], n, p, theta, dt)
        did2 = ncorp.ncorp_batch_add_disk(b, d["pos"], d["vel"], d["mass"], d["radius"], n, p, theta, dt)
        ncorp.ncorp_batch_run(b, 4)
        pos, vel = np.zeros((n, 3)), np.zeros((n, 3))
        pos2, vel2 = np.zeros((n, 3)), np.zeros((n, 3))
        ncorp.ncorp_batch_get_state(b, did, pos, vel)
        ncorp.ncorp_batch_get_state(b, did2, pos2, vel2)
    finally:
        ncorp.ncorp_batch_free(b)
    ctx = ncorp.ncorp_init(config(ncorp.NCORP_MIXED), n, 0, torch.cuda.current_stream().cuda_stream)
    xs, vs = d["pos"].copy(), d["vel"].copy()
    try:
        for _ in range(4):
            ncorp.ncorp_step(ctx, xs, vs, d["mass"], d["radius"], n, p, theta, dt)
    finally:
        ncorp.ncorp_free(ctx)
    # Two mixed runs may each differ from the FP64 forces by up to MIXED_TOL of a moonlet's mutual
    # acceleration (FP32 sums in a different order), so over k steps their velocities may differ by
    # about k dt 2 MIXED_TOL |a_mut| per moonlet (taken twice for safety); positions by dt times less.
    ctx = ncorp.ncorp_init(config(ncorp.NCORP_FP64), n, 0, torch.cuda.current_stream().cuda_stream)
    acc, mut = np.zeros((n, 3)), np.zeros((n, 3))
    try:
        ncorp.ncorp_accel(ctx, d["pos"], d["mass"], n, p, theta, acc, mut)
    finally:
        ncorp.ncorp_free(ctx)
    bound = 2 * 4 * dt * 2 * MIXED_TOL * np.linalg.norm(mut, axis=1) + 1e-15
    for x, v in ((pos, vel), (pos2, vel2)):
        np.testing.assert_allclose(x, xs, rtol=0, atol=1e-12 * np.abs(xs).max())
        assert np.all(np.linalg.norm(v - vs, axis=1) <= bound)


def test_batch_rejections():
    d = diskgen.make_disk(2000, 66)
    b = ncorp.ncorp_batch_create(config(), 1 << 20, torch.cuda.current_stream().cuda_stream)   # 1 MiB budget
    try:
        with pytest.raises(ncorp.NcorpError) as e:
            ncorp.ncorp_batch_add_disk(b, d["pos"], d["vel"], d["mass"], d["radius"], 2000, 3, 0.5, 1e-3)
        assert e.value.code == ncorp.NCORP_ENOMEM and "budget" in str(e.value)
        assert ncorp.ncorp_batch_info(b)["disks"] == 0
        for bad in ((0, 3, 0.5, 1e-3), (2000, 7, 0.5, 1e-3), (2000, 3, 1.0, 1e-3), (2000, 3, 0.5, 0.0)):
            with pytest.raises(ncorp.NcorpError) as e:
                ncorp.ncorp_batch_add_disk(b, d["pos"], d["vel"], d["mass"], d["radius"], *bad)
            assert e.value.code == ncorp.NCORP_EINVAL
        with pytest.raises(ncorp.NcorpError) as e:
            ncorp.ncorp_batch_remove_disk(b, 12345)
        assert e.value.code == ncorp.NCORP_EINVAL
        with pytest.raises(ncorp.NcorpError):
            ncorp.ncorp_batch_run(b, -1)
        ncorp.ncorp_batch_run(b, 3)   # empty batch: nothing to do
    finally:
        ncorp.ncorp_batch_free(b)


def test_a_layout_that_runs_out_of_memory_leaves_nothing_behind():
    """A run whose forest cannot be laid out (device memory taken by another allocation) fails with
    NCORP_ENOMEM, steps nothing, and releases every buffer it had taken: the device's free memory is
    the same after the batch is freed, and the run succeeds once memory is available again."""
    d = diskgen.make_disk(200000, 67)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    b = ncorp.ncorp_batch_create(config(), 0, torch.cuda.current_stream().cuda_stream)
    try:
        i = ncorp.ncorp_batch_add_disk(b, d["pos"], d["vel"], d["mass"], d["radius"], len(d["pos"]), 3, 0.5, 1e-3)
        # leave about 60 MB free: not enough for the forest's context
        hog = torch.empty(max(0, torch.cuda.mem_get_info()[0] - (60 << 20)), dtype=torch.uint8, device="cuda")
        with pytest.raises(ncorp.NcorpError) as e:
            ncorp.ncorp_batch_run(b, 2)
        assert e.value.code == ncorp.NCORP_ENOMEM
        pos, vel = np.zeros((len(d["pos"]), 3)), np.zeros((len(d["pos"]), 3))
        ncorp.ncorp_batch_get_state(b, i, pos, vel)
        assert np.array_equal(pos, d["pos"]) and np.array_equal(vel, d["vel"])   # nothing was stepped
        del hog
        torch.cuda.empty_cache()
        ncorp.ncorp_batch_run(b, 2)
    finally:
        ncorp.ncorp_batch_free(b)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    assert torch.cuda.mem_get_info()[0] >= free0 - (16 << 20)
