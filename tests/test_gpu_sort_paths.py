"""Key sort of a step's new tree, on each of its paths (needs a GB300).

In a step the keys of the drifted positions are computed in the previous
tree order, so they are nearly sorted: the keys next to a descent, and the
keys out of order with the nearest such-free keys on either side, are taken
out ("movers"), sorted apart (ranked when at most 4096: path 1; radix-sorted
when more: path 2) and merged back into the rest.  When there are more than
65536 movers the launch sorts all keys with the radix sort instead (path 0),
and when the keys left in place are not in order it does the same after the
check (path -1).  Whichever path runs, the new tree must be the oracle's
tree of the new positions, bit for bit; the path is read from the step's
statistics and predicted here from the oracle's keys.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_20374_gb300 import diskgen, ncorp

pytestmark = pytest.mark.gpu

MOVERS_RANKED = 4096
MOVERS_MAX = 65536
REACH = 16   # a key with this many keys next to descents beside it is a mover


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def predicted_path(P, x_prev, x_new):
    """The path the sort takes for keys of x_new listed in the tree order of x_prev."""
    order_prev = oracle.tree_export(P, x_prev)["order"]
    seq = oracle.tree_export(P, x_new)["keys"][order_prev]
    n = len(seq)
    desc = seq[:-1] > seq[1:]
    near = np.zeros(n, dtype=bool)       # next to a descent
    near[:-1] |= desc
    near[1:] |= desc
    mover = near.copy()
    for i in np.flatnonzero(~near):      # out of order with the nearest keys not next to a descent
        j = i - 1
        while j >= 0 and near[j] and i - j < REACH:
            j -= 1
        if j >= 0 and (near[j] or seq[j] > seq[i]):
            mover[i] = True
            continue
        j = i + 1
        while j < n and near[j] and j - i < REACH:
            j += 1
        if j < n and (near[j] or seq[i] > seq[j]):
            mover[i] = True
    if mover.sum() > MOVERS_MAX:
        return 0
    kept = seq[~mover]
    if not np.all(kept[:-1] <= kept[1:]):
        return -1
    return 1 if mover.sum() <= MOVERS_RANKED else 2


@pytest.mark.parametrize("n,dt,jump,first_path", [(20011, 1e-3, 0, 1), (20011, 0.05, 0, 2), (20011, 0.2, 0, -1),
                                                  (140000, 0.2, 0, 0), (20011, 1e-3, 300, 1)])
def test_step_tree_matches_oracle_on_every_sort_path(n, dt, jump, first_path):
    s = 16
    d = diskgen.make_disk(n, 81)
    x, v = d["pos"].copy(), d["vel"].copy()
    if jump:   # these moonlets cross to the other side of the disk in one step
        v[:jump] = -2.0 * x[:jump] / dt
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_FP64
    cfg.leaf_size = s
    cfg.collisions = 0
    ctx = ncorp.ncorp_init(cfg, n, 0, torch.cuda.current_stream().cuda_stream)
    P = oracle.params(p=3, theta=0.5, leaf_size=s)
    paths = []
    try:
        for step in range(2):
            x_prev = x.copy()
            ncorp.ncorp_step(ctx, x, v, d["mass"], d["radius"], n, 3, 0.5, dt)
            path = ncorp.ncorp_stats(ctx)["sort_path"]
            paths.append(path)
            assert path == predicted_path(P, x_prev, x), (step, path)
            cap = 8 * n + 64
            order = np.zeros(n, dtype=np.int64)
            keys = np.zeros(n, dtype=np.uint64)
            cells = np.zeros((cap, 7), dtype=np.int64)
            nc = ncorp.ncorp_tree_export(ctx, order, keys, np.zeros(4), cells, None, None, cap)
            o = oracle.tree_export(P, x)
            assert np.array_equal(order, o["order"])
            assert np.array_equal(keys, o["keys"][o["order"]])
            assert np.array_equal(cells[:nc], o["cells"])
    finally:
        ncorp.ncorp_free(ctx)
    assert paths[0] == first_path
