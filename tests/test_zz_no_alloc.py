"""GPU test of ncorp_hilbert_sort_static, the allocation-free keys + sort call.

Compares it, on two calls in a row, with the Hilbert keys and tree order that
ncorp_tree_export reports after ncorp_accel on the same positions (bit-exact:
integer results), at a ragged size, at one moonlet and at the largest size
the static scratch array holds, and checks the rejections made before any
device work.  This file is collected last so that it also runs after every
other test has used the device.
"""
import numpy as np
import pytest
import torch

from paper_2310_20374_gb300 import diskgen, ncorp

pytestmark = pytest.mark.gpu


def reference_keys_order(pos_np, mass_np):
    n = len(pos_np)
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_FP64
    cfg.leaf_size = 32
    ctx = ncorp.ncorp_init(cfg, n, 0, torch.cuda.current_stream().cuda_stream)
    try:
        pos = torch.tensor(pos_np, device="cuda")
        m = torch.tensor(mass_np, device="cuda")
        acc = torch.empty_like(pos)
        ncorp.ncorp_accel(ctx, pos, m, n, 3, 0.5, acc)
        cap = 8 * n + 64
        order = np.zeros(n, dtype=np.int64)
        keys = np.zeros(n, dtype=np.uint64)
        ncorp.ncorp_tree_export(ctx, order, keys, np.zeros(4), np.zeros((cap, 7), dtype=np.int64),
                                np.zeros((cap, 6)), np.zeros((cap, 5)), cap)
    finally:
        ncorp.ncorp_free(ctx)
    return keys, order


@pytest.mark.parametrize("n,seed", [(20000, 41), (1, 42), (ncorp.NCORP_STATIC_MAX_N, 43)])
def test_static_sort_matches_tree_export_twice(n, seed):
    d = diskgen.make_disk(n, seed)
    ref_keys, ref_order = reference_keys_order(d["pos"], d["mass"])
    pos = torch.tensor(d["pos"], device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        keys = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        order = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        ncorp.ncorp_hilbert_sort_static(pos, n, keys, order, stream)
        torch.cuda.synchronize()
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref_keys)
        assert np.array_equal(order.cpu().numpy(), ref_order)


def test_static_sort_rejects_before_device_work():
    n = ncorp.NCORP_STATIC_MAX_N + 1
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    order = torch.empty(n, dtype=torch.int64, device="cuda")
    with pytest.raises(ncorp.NcorpError) as e:
        ncorp.ncorp_hilbert_sort_static(pos, n, keys, order)
    assert e.value.code == ncorp.NCORP_EINVAL
    with pytest.raises(ncorp.NcorpError) as e:   # host array
        ncorp.ncorp_hilbert_sort_static(np.zeros((8, 3)), 8, keys, order)
    assert e.value.code == ncorp.NCORP_EINVAL
    bad = torch.zeros((8, 3), dtype=torch.float64, device="cuda")
    bad[3, 1] = float("nan")
    with pytest.raises(ncorp.NcorpError) as e:   # non-finite position, found on the device
        ncorp.ncorp_hilbert_sort_static(bad, 8, keys, order)
    assert e.value.code == ncorp.NCORP_EINVAL


def test_static_sort_takes_no_device_memory():
    """After one warm-up call (which may load the module and look up the
    scratch array), further calls leave the device's free memory unchanged."""
    n = 30000
    d = diskgen.make_disk(n, 44)
    pos = torch.tensor(d["pos"], device="cuda")
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    order = torch.empty(n, dtype=torch.int64, device="cuda")
    ncorp.ncorp_hilbert_sort_static(pos, n, keys, order)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        ncorp.ncorp_hilbert_sort_static(pos, n, keys, order)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
