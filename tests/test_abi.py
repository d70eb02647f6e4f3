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


# ---- the ctypes binding and the oracle wrapper against the C declarations they mirror
_CTYPES = {"double": C.c_double, "int": C.c_int, "int64_t": C.c_int64}


def _struct_fields(text, name):
    """[(field, ctypes type)] of `typedef struct { ... } name;` in C source text."""
    m = re.search(r"typedef struct \{(.*?)\}\s*" + name + ";", text, re.S)
    assert m, name
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = decl.split(None, 1)
        out += [(n.strip(), _CTYPES[ctype]) for n in names.split(",")]
    return out


def test_config_struct_matches_the_header():
    text = open(ncorp.HEADER).read()
    assert [(n, t) for n, t in ncorp.ncorp_config._fields_] == _struct_fields(text, "ncorp_config")


def test_stat_and_stage_slots_match_the_header():
    text = open(ncorp.HEADER).read()
    stats = {n: int(i) for n, i in re.findall(r"#define NCORP_STAT_(\w+)\s+(\d+)", text)}
    assert int(re.search(r"#define NCORP_NSTATS\s+(\d+)", text).group(1)) == len(ncorp.STAT_NAMES) == len(stats)
    for name, i in stats.items():
        assert ncorp.STAT_NAMES[i] == name.lower().replace("p2p_inter", "p2p_interactions"), (name, i)
    stages = {n: int(i) for n, i in re.findall(r"#define NCORP_STAGE_(\w+)\s+(\d+)", text)}
    assert int(re.search(r"#define NCORP_NSTAGES\s+(\d+)", text).group(1)) == len(ncorp.STAGE_NAMES) == len(stages)
    for name, i in stages.items():
        assert ncorp.STAGE_NAMES[i] == name.lower(), (name, i)


def test_oracle_params_match_its_c_struct():
    import oracle
    text = open(os.path.join(os.path.dirname(oracle.__file__), "ncorp_oracle.c")).read()
    assert [(n, t) for n, t in oracle.Params._fields_] == _struct_fields(text, "or_params")
