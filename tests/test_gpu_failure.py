"""Failure paths of the step library on a GB300, made without a GPU fault.

  * A bounded device-side wait that runs out: NCORP_TEST_STALL_STEP=k makes
    the grid barriers of a context's k-th ncorp_step wait for one arrival
    that no block makes; with NCORP_WAIT_LIMIT_MS=20 every block gives up
    after 20 ms and returns, the call fails with NCORP_ETIMEOUT, the caller's
    arrays are left as they were, and the next call succeeds with the result
    a fresh context gives from the same state.  Nothing traps, faults or
    waits without a limit.
  * Buffers that overflow: NCORP_TEST_LIST_CAP / NCORP_TEST_PAIR_CAP start
    the walk lists / the colliding-pair buffer far too small, so the step
    overflows, grows them and reruns from the resident state (ncorp_step), or
    the batch reruns the disk from its snapshot (counted in
    NCORP_BATCH_FALLBACKS); results equal those of an unforced run.

The knobs are read by ncorp_init, so each context is created with the
environment set and the variables are removed again afterwards.
"""
import numpy as np
import pytest
import torch

from paper_2310_20374_gb300 import diskgen, ncorp

pytestmark = pytest.mark.gpu

P, THETA, DT = 3, 0.5, 2e-2


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def ring(n, seed):
    """A dense ring with many colliding pairs per step."""
    return diskgen.make_disk(n, seed, a_lo=2.0, a_hi=2.5, r_lo=2e-2, r_hi=5e-2, sigma_e=0.1, sigma_i=0.05)


def config():
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_FP64
    cfg.leaf_size = 16
    return cfg


def device_state(d):
    return [torch.tensor(d[k], device="cuda") for k in ("pos", "vel", "mass", "radius")]


def run_steps(d, steps, env=None, monkeypatch=None):
    """(pos, vel, pairs of the last step) after `steps` ncorp_step calls of a new context."""
    if env:
        for k, v in env.items():
            monkeypatch.setenv(k, str(v))
    n = len(d["pos"])
    ctx = ncorp.ncorp_init(config(), n, 0, torch.cuda.current_stream().cuda_stream)
    if env:
        for k in env:
            monkeypatch.delenv(k)
    pos, vel, m, R = device_state(d)
    try:
        for _ in range(steps):
            ncorp.ncorp_step(ctx, pos, vel, m, R, n, P, THETA, DT)
        pairs = np.zeros((1 << 15, 2), dtype=np.int64)
        k = ncorp.ncorp_collisions(ctx, pairs, len(pairs))
    finally:
        ncorp.ncorp_free(ctx)
    return pos.cpu().numpy(), vel.cpu().numpy(), pairs[:k]


def close(a, b, rtol):
    return np.abs(a - b).max() <= rtol * np.abs(b).max()


def test_barrier_wait_runs_out_and_the_next_step_recovers(monkeypatch):
    n = 6000
    d = ring(n, 81)
    monkeypatch.setenv("NCORP_WAIT_LIMIT_MS", "20")
    monkeypatch.setenv("NCORP_TEST_STALL_STEP", "3")
    ctx = ncorp.ncorp_init(config(), n, 0, torch.cuda.current_stream().cuda_stream)
    monkeypatch.delenv("NCORP_WAIT_LIMIT_MS")
    monkeypatch.delenv("NCORP_TEST_STALL_STEP")
    pos, vel, m, R = device_state(d)
    try:
        for _ in range(2):
            ncorp.ncorp_step(ctx, pos, vel, m, R, n, P, THETA, DT)
        before_p, before_v = pos.clone(), vel.clone()
        with pytest.raises(ncorp.NcorpError) as e:
            ncorp.ncorp_step(ctx, pos, vel, m, R, n, P, THETA, DT)   # the stalled step
        assert e.value.code == ncorp.NCORP_ETIMEOUT
        assert "timed out" in ncorp.ncorp_last_error(ctx)
        torch.cuda.synchronize()
        assert torch.equal(pos, before_p) and torch.equal(vel, before_v)   # nothing written
        ncorp.ncorp_step(ctx, pos, vel, m, R, n, P, THETA, DT)         # re-reads the arrays
        got_p, got_v = pos.cpu().numpy(), vel.cpu().numpy()
        pairs = np.zeros((1 << 15, 2), dtype=np.int64)
        got_pairs = pairs[:ncorp.ncorp_collisions(ctx, pairs, len(pairs))]
        for _ in range(2):   # and stays usable (resident, graph-replayed steps)
            ncorp.ncorp_step(ctx, pos, vel, m, R, n, P, THETA, DT)
    finally:
        ncorp.ncorp_free(ctx)
    start = dict(d, pos=before_p.cpu().numpy(), vel=before_v.cpu().numpy())
    ref_p, ref_v, ref_pairs = run_steps(start, 1)
    assert close(got_p, ref_p, 1e-13) and close(got_v, ref_v, 1e-12)
    assert len(ref_pairs) > 0 and np.array_equal(got_pairs, ref_pairs)


@pytest.mark.parametrize("knob,cap", [("NCORP_TEST_LIST_CAP", 64), ("NCORP_TEST_PAIR_CAP", 4)])
def test_forced_overflow_grows_and_reruns_the_step(monkeypatch, knob, cap):
    d = ring(5000, 82)
    ref = run_steps(d, 3)
    got = run_steps(d, 3, {knob: cap}, monkeypatch)
    if knob == "NCORP_TEST_PAIR_CAP":
        assert len(ref[2]) > cap   # the pair buffer must overflow (the lists overflow at any size here)
    assert close(got[0], ref[0], 1e-13) and close(got[1], ref[1], 1e-12)
    assert np.array_equal(got[2], ref[2])


def test_batch_overflow_reruns_the_disk_from_its_snapshot(monkeypatch):
    disks = [ring(4000, 83), diskgen.make_disk(6000, 84)]
    steps = 3
    refs = [run_steps(d, steps) for d in disks]
    monkeypatch.setenv("NCORP_TEST_PAIR_CAP", "4")   # the dense ring finds more pairs than that
    b = ncorp.ncorp_batch_create(config(), 0, torch.cuda.current_stream().cuda_stream)
    try:
        ids = [ncorp.ncorp_batch_add_disk(b, *device_state(d), len(d["pos"]), P, THETA, DT) for d in disks]
        monkeypatch.delenv("NCORP_TEST_PAIR_CAP")
        assert ncorp.ncorp_batch_info(b)["fallbacks"] == 0
        ncorp.ncorp_batch_run(b, steps)
        assert ncorp.ncorp_batch_info(b)["fallbacks"] >= 1
        for did, d, (rp, rv, rpairs) in zip(ids, disks, refs):
            n = len(d["pos"])
            gp, gv = np.zeros((n, 3)), np.zeros((n, 3))
            ncorp.ncorp_batch_get_state(b, did, gp, gv)
            pairs = np.zeros((1 << 15, 2), dtype=np.int64)
            k = ncorp.ncorp_batch_collisions(b, did, pairs, len(pairs))
            assert close(gp, rp, 1e-13) and close(gv, rv, 1e-12)
            assert np.array_equal(pairs[:k], rpairs)
    finally:
        ncorp.ncorp_batch_free(b)
