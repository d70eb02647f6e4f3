"""C ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every function include/ncorp.h declares, and rejects bad arguments before any
device work."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2310_20374_gb300 import build as B
from paper_2310_20374_gb300 import ncorp


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ncorp.load()


def test_exports_every_declared_symbol(lib):
    names = ncorp.declared_functions()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(names) <= exported


def test_build_flags_target_sm103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_config_default(lib):
    cfg = ncorp.ncorp_config_default()
    assert cfg.G == 1.0 and cfg.central_mass == 1.0 and cfg.central_radius == 1.0
    assert cfg.precision == ncorp.NCORP_MIXED and cfg.collisions == 1
    assert cfg.leaf_size == 0 and cfg.star_mass == 0.0 and cfg.central_J2 == 0.0
    assert cfg.resolve_f == 0.0
    assert (cfg.n_cb_pre, cfg.n_cb_post) == (6, 16)


def test_bad_arguments_rejected_without_device_work(lib):
    cfg = ncorp.ncorp_config_default()
    h = C.c_void_p()
    assert lib.ncorp_init(C.byref(h), C.byref(cfg), 0, 0, None) == ncorp.NCORP_EINVAL
    assert lib.ncorp_init(None, C.byref(cfg), 10, 0, None) == ncorp.NCORP_EINVAL
    bad = ncorp.ncorp_config_default()
    bad.precision = 7
    assert lib.ncorp_init(C.byref(h), C.byref(bad), 10, 0, None) == ncorp.NCORP_EINVAL
    for f in (0.5, 2.5, -1.0, float("nan"), float("inf")):   # resolution needs 1 <= f <= 2 (or 0 = off)
        bad = ncorp.ncorp_config_default()
        bad.resolve_f = f
        assert lib.ncorp_init(C.byref(h), C.byref(bad), 10, 0, None) == ncorp.NCORP_EINVAL
        assert lib.ncorp_batch_create(C.byref(h), C.byref(bad), 0, None) == ncorp.NCORP_EINVAL
    bad = ncorp.ncorp_config_default()
    bad.n_cb_pre = -1
    assert lib.ncorp_init(C.byref(h), C.byref(bad), 10, 0, None) == ncorp.NCORP_EINVAL
    assert lib.ncorp_accel_standard(None, None, None, 10, 3, 0.5, None, None) == ncorp.NCORP_EINVAL
    assert lib.ncorp_step(None, None, None, None, None, 10, 3, 0.5, 1e-3) == ncorp.NCORP_EINVAL
    assert lib.ncorp_accel(None, None, None, 10, 3, 0.5, None, None) == ncorp.NCORP_EINVAL
    assert lib.ncorp_collisions(None, None, 0, None) == ncorp.NCORP_EINVAL
    assert lib.ncorp_last_error(None) == b"null context"
    lib.ncorp_free(None)


def test_header_documents_every_entry_point():
    with open(ncorp.HEADER) as f:
        text = f.read()
    for name in ncorp.declared_functions():
        m = re.search(r"^(?:const )?[a-z_0-9]+ \**" + name + r"\(", text, re.M)   # the declaration line
        assert m, f"{name} has no declaration line"
        assert text[:m.start()].rstrip().endswith("*/"), f"{name} has no comment right above it"
