"""Thin Python binding of libncorp.so (the C ABI declared in include/ncorp.h).

Functions carry the C names and only marshal arguments: array arguments may
be torch tensors (CPU or CUDA), numpy arrays or raw integer addresses; all
computation happens in the CUDA library.  A non-zero status raises NcorpError
with the library's message.  There is no fallback: if the library has not been
built (``paper_2310_20374_gb300.build``) or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import build as _build

NCORP_OK, NCORP_EINVAL, NCORP_ENOMEM, NCORP_ECUDA, NCORP_EOVERFLOW, NCORP_ETIMEOUT, NCORP_ESTATE = 0, -1, -2, -3, -4, -5, -6
NCORP_FP64, NCORP_MIXED = 0, 1
NCORP_MAX_DISKS = 256
STAT_NAMES = ["cells", "leaves", "depth", "m2l", "p2p_pairs", "p2p_self", "p2p_interactions", "col_pairs",
              "col_self", "col_tests", "col_found", "walk_iters", "m2l_directed", "p2p_directed", "launches", "col_iters",
              "graph", "sort_path", "resolved", "fused"]
STAGE_NAMES = ["sort", "build", "climb", "walk", "m2l", "descend", "eval", "collide", "kdk", "near"]
HEADER = os.path.join(os.path.dirname(_build.HERE), "include", "ncorp.h")


class NcorpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ncorp error {code}: {msg}")
        self.code = code


class ncorp_config(C.Structure):
    _fields_ = [("G", C.c_double), ("central_mass", C.c_double), ("central_radius", C.c_double),
                ("leaf_size", C.c_int), ("n_cs", C.c_int), ("n_cc_pre", C.c_int), ("n_cc_post", C.c_int),
                ("c_cs", C.c_int), ("c_cc_pre", C.c_int), ("c_cc_post", C.c_int),
                ("precision", C.c_int), ("collisions", C.c_int),
                ("star_mass", C.c_double), ("star_a", C.c_double), ("star_obliquity", C.c_double),
                ("t0", C.c_double), ("central_J2", C.c_double), ("resolve_f", C.c_double),
                ("n_cb_pre", C.c_int), ("n_cb_post", C.c_int), ("c_cb_pre", C.c_int), ("c_cb_post", C.c_int),
                ("fused_walk", C.c_int)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Loads libncorp.so (raises if it is missing: no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build the CUDA library first (paper_2310_20374_gb300.build.build())")
    L = C.CDLL(path)
    vp, i64, dbl, ip = C.c_void_p, C.c_int64, C.c_double, C.c_int
    L.ncorp_config_default.argtypes = [C.POINTER(ncorp_config)]
    L.ncorp_config_default.restype = None
    L.ncorp_init.argtypes = [C.POINTER(vp), C.POINTER(ncorp_config), i64, ip, vp]
    L.ncorp_set_stream.argtypes = [vp, vp]
    L.ncorp_step.argtypes = [vp, vp, vp, vp, vp, i64, ip, dbl, dbl]
    L.ncorp_reset.argtypes = [vp]
    L.ncorp_set_disks.argtypes = [vp, ip, vp]
    L.ncorp_set_graphs.argtypes = [vp, ip]
    L.ncorp_collisions.argtypes = [vp, vp, i64, C.POINTER(i64)]
    L.ncorp_accel.argtypes = [vp, vp, vp, i64, ip, dbl, vp, vp]
    L.ncorp_accel_standard.argtypes = [vp, vp, vp, i64, ip, dbl, vp, vp]
    L.ncorp_collide.argtypes = [vp, vp, vp, vp, i64, dbl]
    L.ncorp_collide_standard.argtypes = [vp, vp, vp, vp, i64, dbl]
    L.ncorp_get_state.argtypes = [vp, vp, vp]
    L.ncorp_stats.argtypes = [vp, C.POINTER(i64), ip]
    L.ncorp_tree_export.argtypes = [vp, vp, vp, vp, vp, vp, vp, i64, C.POINTER(i64)]
    L.ncorp_expansions.argtypes = [vp, vp, vp, vp, i64, C.POINTER(i64), C.POINTER(ip)]
    L.ncorp_profile.argtypes = [vp, ip]
    L.ncorp_stage_times.argtypes = [vp, C.POINTER(dbl), ip]
    L.ncorp_hilbert_sort_static.argtypes = [vp, i64, vp, vp, vp]
    L.ncorp_fma_peak.argtypes = [ip, ip, vp, C.POINTER(dbl)]
    L.ncorp_batch_create.argtypes = [C.POINTER(vp), C.POINTER(ncorp_config), C.c_size_t, vp]
    L.ncorp_batch_add_disk.argtypes = [vp, vp, vp, vp, vp, i64, ip, dbl, dbl, C.POINTER(C.c_int32)]
    L.ncorp_batch_run.argtypes = [vp, ip]
    L.ncorp_batch_get_state.argtypes = [vp, C.c_int32, vp, vp]
    L.ncorp_batch_collisions.argtypes = [vp, C.c_int32, vp, i64, C.POINTER(i64)]
    L.ncorp_batch_remove_disk.argtypes = [vp, C.c_int32, vp, vp]
    L.ncorp_batch_info.argtypes = [vp, C.POINTER(i64), ip]
    L.ncorp_batch_free.argtypes = [vp]
    L.ncorp_batch_free.restype = None
    L.ncorp_batch_last_error.argtypes = [vp]
    L.ncorp_batch_last_error.restype = C.c_char_p
    L.ncorp_free.argtypes = [vp]
    L.ncorp_free.restype = None
    L.ncorp_last_error.argtypes = [vp]
    L.ncorp_last_error.restype = C.c_char_p
    for name in ("ncorp_init", "ncorp_set_stream", "ncorp_step", "ncorp_reset", "ncorp_set_disks", "ncorp_set_graphs", "ncorp_collisions", "ncorp_accel",
                 "ncorp_accel_standard", "ncorp_collide", "ncorp_collide_standard", "ncorp_get_state", "ncorp_stats", "ncorp_tree_export", "ncorp_expansions", "ncorp_profile", "ncorp_stage_times",
                 "ncorp_hilbert_sort_static", "ncorp_fma_peak", "ncorp_batch_create", "ncorp_batch_add_disk", "ncorp_batch_run",
                 "ncorp_batch_get_state", "ncorp_batch_collisions", "ncorp_batch_remove_disk", "ncorp_batch_info"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def declared_functions() -> list[str]:
    """Names of the functions declared in include/ncorp.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ncorp_[a-z_0-9]+)\s*\(", text)))


def _ptr(a):
    """Address of a tensor / ndarray / int (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a)}")


_KINDS = {"f8": ("float64",), "i8": ("int64", "uint64"), "i4": ("int32",)}


def _arr(a, kind, count, name):
    """Address of an array argument after checking what can be checked here:
    a torch tensor or numpy array must have the element type `kind` ("f8":
    float64, "i8": 8-byte integer), be contiguous and hold at least `count`
    elements, else NcorpError(NCORP_EINVAL) is raised before the library is
    called (the library cannot see how large an allocation is).  None and raw
    integer addresses pass through unchecked."""
    if a is None or isinstance(a, int):
        return _ptr(a)
    if hasattr(a, "data_ptr"):   # torch tensor
        dt = str(a.dtype).replace("torch.", "")
        contiguous, size = a.is_contiguous(), a.numel()
    elif hasattr(a, "ctypes"):   # numpy array
        dt = str(a.dtype)
        contiguous, size = bool(a.flags["C_CONTIGUOUS"]), a.size
    else:
        return _ptr(a)
    if dt not in _KINDS[kind]:
        raise NcorpError(NCORP_EINVAL, f"{name}: element type {dt}, expected {' or '.join(_KINDS[kind])}")
    if not contiguous:
        raise NcorpError(NCORP_EINVAL, f"{name}: array is not contiguous")
    if size < count:
        raise NcorpError(NCORP_EINVAL, f"{name}: {size} elements, at least {count} needed")
    return _ptr(a)


def _check(ctx, st):
    if st != NCORP_OK:
        msg = load().ncorp_last_error(ctx)
        raise NcorpError(st, msg.decode() if msg else "")
    return st


def ncorp_config_default() -> ncorp_config:
    cfg = ncorp_config()
    load().ncorp_config_default(C.byref(cfg))
    return cfg


def ncorp_init(cfg: ncorp_config, n_max: int, device: int = 0, stream=None):
    h = C.c_void_p()
    st = load().ncorp_init(C.byref(h), C.byref(cfg), int(n_max), int(device), _ptr(stream))
    if st != NCORP_OK:
        raise NcorpError(st, "ncorp_init failed")
    return h


def ncorp_set_stream(ctx, stream):
    return _check(ctx, load().ncorp_set_stream(ctx, _ptr(stream)))


def ncorp_step(ctx, positions, velocities, masses, radii, n, p, theta, dt):
    n = int(n)
    return _check(ctx, load().ncorp_step(ctx, _arr(positions, "f8", 3 * n, "positions"),
                                         _arr(velocities, "f8", 3 * n, "velocities"), _arr(masses, "f8", n, "masses"),
                                         _arr(radii, "f8", n, "radii"), n, int(p), float(theta), float(dt)))


def ncorp_reset(ctx):
    return _check(ctx, load().ncorp_reset(ctx))


def ncorp_set_disks(ctx, sizes):
    """Lays the context's moonlets out as len(sizes) independent disks (sizes: moonlets per disk, in the
    order the disks follow one another in the arrays of later calls); [n] returns to one disk."""
    sz = np.ascontiguousarray(np.asarray(sizes, dtype=np.int64).reshape(-1))
    return _check(ctx, load().ncorp_set_disks(ctx, int(sz.size), sz.ctypes.data if sz.size else None))


def ncorp_set_graphs(ctx, enable):
    return _check(ctx, load().ncorp_set_graphs(ctx, 1 if enable else 0))


def ncorp_collisions(ctx, pairs, cap):
    """Fills pairs [cap][2] int64; returns the total number found."""
    found = C.c_int64(0)
    st = load().ncorp_collisions(ctx, _arr(pairs, "i8", 2 * int(cap), "pairs"), int(cap), C.byref(found))
    if st not in (NCORP_OK, NCORP_EOVERFLOW):
        _check(ctx, st)
    return int(found.value)


def ncorp_accel(ctx, positions, masses, n, p, theta, acc, acc_mutual=None):
    n = int(n)
    return _check(ctx, load().ncorp_accel(ctx, _arr(positions, "f8", 3 * n, "positions"),
                                          _arr(masses, "f8", n, "masses"), n, int(p), float(theta),
                                          _arr(acc, "f8", 3 * n, "acc"), _arr(acc_mutual, "f8", 3 * n, "acc_mutual")))


def ncorp_accel_standard(ctx, positions, masses, n, p, theta, acc, acc_mutual=None):
    n = int(n)
    return _check(ctx, load().ncorp_accel_standard(ctx, _arr(positions, "f8", 3 * n, "positions"),
                                                   _arr(masses, "f8", n, "masses"), n, int(p), float(theta),
                                                   _arr(acc, "f8", 3 * n, "acc"),
                                                   _arr(acc_mutual, "f8", 3 * n, "acc_mutual")))


def ncorp_collide(ctx, positions, velocities, radii, n, dt):
    n = int(n)
    return _check(ctx, load().ncorp_collide(ctx, _arr(positions, "f8", 3 * n, "positions"),
                                            _arr(velocities, "f8", 3 * n, "velocities"),
                                            _arr(radii, "f8", n, "radii"), n, float(dt)))


def ncorp_collide_standard(ctx, positions, velocities, radii, n, dt):
    n = int(n)
    return _check(ctx, load().ncorp_collide_standard(ctx, _arr(positions, "f8", 3 * n, "positions"),
                                                     _arr(velocities, "f8", 3 * n, "velocities"),
                                                     _arr(radii, "f8", n, "radii"), n, float(dt)))


def ncorp_get_state(ctx, positions, velocities):
    return _check(ctx, load().ncorp_get_state(ctx, _ptr(positions), _ptr(velocities)))


def ncorp_stats(ctx) -> dict:
    arr = (C.c_int64 * len(STAT_NAMES))()
    _check(ctx, load().ncorp_stats(ctx, arr, len(STAT_NAMES)))
    return {k: int(v) for k, v in zip(STAT_NAMES, arr) if not k.startswith("_")}


def ncorp_tree_export(ctx, order=None, keys=None, root=None, cells=None, ggeo=None, cgeo=None, cap=0):
    nc = C.c_int64(0)
    st = load().ncorp_tree_export(ctx, _ptr(order), _ptr(keys), _ptr(root), _ptr(cells), _ptr(ggeo), _ptr(cgeo),
                                  int(cap), C.byref(nc))
    if st not in (NCORP_OK, NCORP_EOVERFLOW):
        _check(ctx, st)
    return int(nc.value)


def ncorp_expansions(ctx, mult=None, local=None, rho=None, cap=0):
    """Returns (n_cells, p); fills the given [cap][...] float64 arrays."""
    nc = C.c_int64(0)
    pp = C.c_int(0)
    st = load().ncorp_expansions(ctx, _ptr(mult), _ptr(local), _ptr(rho), int(cap), C.byref(nc), C.byref(pp))
    if st not in (NCORP_OK, NCORP_EOVERFLOW):
        _check(ctx, st)
    return int(nc.value), int(pp.value)


def num_m(p):
    return 1 if p < 2 else p * (p + 1) * (p + 2) // 6 - 3


def num_c(p):
    return (p + 1) * (p + 2) * (p + 3) // 6 - 1


def ncorp_profile(ctx, enable=True):
    return _check(ctx, load().ncorp_profile(ctx, int(bool(enable))))


def ncorp_stage_times(ctx) -> dict:
    arr = (C.c_double * len(STAGE_NAMES))()
    _check(ctx, load().ncorp_stage_times(ctx, arr, len(STAGE_NAMES)))
    return dict(zip(STAGE_NAMES, (float(v) for v in arr)))


NCORP_STATIC_MAX_N = 65536
BATCH_INFO_NAMES = ["disks", "moonlets", "bytes", "forests", "fallbacks", "launches", "tuned", "leaf_size"]


def _bcheck(b, st, ok=(NCORP_OK,)):
    if st not in ok:
        msg = load().ncorp_batch_last_error(b)
        raise NcorpError(st, msg.decode() if msg else "")
    return st


def ncorp_batch_create(cfg: ncorp_config, hbm_budget_bytes: int = 0, stream=None):
    h = C.c_void_p()
    st = load().ncorp_batch_create(C.byref(h), C.byref(cfg), int(hbm_budget_bytes), _ptr(stream))
    if st != NCORP_OK:
        raise NcorpError(st, "ncorp_batch_create failed")
    return h


def ncorp_batch_add_disk(b, positions, velocities, masses, radii, n, p, theta, dt) -> int:
    did = C.c_int32(-1)
    n = int(n)
    _bcheck(b, load().ncorp_batch_add_disk(b, _arr(positions, "f8", 3 * n, "positions"),
                                           _arr(velocities, "f8", 3 * n, "velocities"),
                                           _arr(masses, "f8", n, "masses"), _arr(radii, "f8", n, "radii"), n,
                                           int(p), float(theta), float(dt), C.byref(did)))
    return int(did.value)


def ncorp_batch_run(b, n_steps):
    return _bcheck(b, load().ncorp_batch_run(b, int(n_steps)))


def ncorp_batch_get_state(b, disk_id, positions, velocities):
    return _bcheck(b, load().ncorp_batch_get_state(b, int(disk_id), _ptr(positions), _ptr(velocities)))


def ncorp_batch_collisions(b, disk_id, pairs, cap):
    found = C.c_int64(0)
    _bcheck(b, load().ncorp_batch_collisions(b, int(disk_id), _arr(pairs, "i8", 2 * int(cap), "pairs"), int(cap),
                                             C.byref(found)),
            ok=(NCORP_OK, NCORP_EOVERFLOW))
    return int(found.value)


def ncorp_batch_remove_disk(b, disk_id, positions=None, velocities=None):
    return _bcheck(b, load().ncorp_batch_remove_disk(b, int(disk_id), _ptr(positions), _ptr(velocities)))


def ncorp_batch_info(b) -> dict:
    arr = (C.c_int64 * len(BATCH_INFO_NAMES))()
    _bcheck(b, load().ncorp_batch_info(b, arr, len(BATCH_INFO_NAMES)))
    return dict(zip(BATCH_INFO_NAMES, (int(v) for v in arr)))


def ncorp_batch_free(b):
    if b:
        load().ncorp_batch_free(b)


def ncorp_batch_last_error(b) -> str:
    m = load().ncorp_batch_last_error(b)
    return m.decode() if m else ""


def ncorp_hilbert_sort_static(positions, n, keys, order, stream=None):
    """Allocation-free keys + stable sort (device arrays only); raises NcorpError on failure."""
    n = int(n)
    st = load().ncorp_hilbert_sort_static(_arr(positions, "f8", 3 * n, "positions"), n, _arr(keys, "i8", n, "keys"),
                                          _arr(order, "i8", n, "order"), _ptr(stream))
    if st != NCORP_OK:
        why = {NCORP_EINVAL: f"invalid argument (n must be 1..{NCORP_STATIC_MAX_N}, arrays device memory of the "
                             f"current device, positions finite)",
               NCORP_ETIMEOUT: "grid barrier timed out", NCORP_ECUDA: "CUDA call failed"}.get(st, "")
        raise NcorpError(st, why)
    return st


def ncorp_fma_peak(device=0, precision=NCORP_MIXED, stream=None) -> float:
    """Measured FMA throughput in FLOP/s: FP32 (NCORP_MIXED) or FP64 (NCORP_FP64)."""
    out = C.c_double(0.0)
    st = load().ncorp_fma_peak(int(device), int(precision), _ptr(stream), C.byref(out))
    if st != NCORP_OK:
        raise NcorpError(st, "ncorp_fma_peak failed")
    return float(out.value)


def ncorp_free(ctx):
    if ctx:
        load().ncorp_free(ctx)


def ncorp_last_error(ctx) -> str:
    m = load().ncorp_last_error(ctx)
    return m.decode() if m else ""
