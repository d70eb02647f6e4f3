"""CPU oracle for the falcON step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``ncorp_oracle.c`` (plain C,
FP64, compiled with ``-O2 -ffp-contract=off``) through ctypes and shares no
code with the CUDA library.  See the C file's header for what each function
follows in the paper.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ncorp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libncorp_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build (only when the source is newer)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [("G", C.c_double), ("central_mass", C.c_double), ("p", C.c_int),
                ("theta_min", C.c_double), ("leaf_size", C.c_int),
                ("n_cs", C.c_int64), ("n_cc_pre", C.c_int64), ("n_cc_post", C.c_int64),
                ("c_cs", C.c_int64), ("c_cc_pre", C.c_int64), ("c_cc_post", C.c_int64),
                ("star_mass", C.c_double), ("star_a", C.c_double), ("star_obliquity", C.c_double),
                ("time", C.c_double), ("m2m_direct", C.c_int), ("brute_collisions", C.c_int),
                ("central_radius", C.c_double), ("central_J2", C.c_double), ("resolve_f", C.c_double),
                ("n_cb_pre", C.c_int64), ("n_cb_post", C.c_int64),
                ("c_cb_pre", C.c_int64), ("c_cb_post", C.c_int64)]


STAT_NAMES = ["cells", "leaves", "depth", "m2l", "p2p_pairs", "p2p_self", "p2p_interactions",
              "col_pairs", "col_self", "col_tests", "col_found"]

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def _opt(ptr_type):
    """ndpointer that also accepts None."""
    class _Opt(ptr_type):
        @classmethod
        def from_param(cls, obj):
            if obj is None:
                return None
            return ptr_type.from_param(obj)
    return _Opt


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def build_variant(source_text: str, out_dir: str) -> str:
    """Compiles an edited copy of the oracle's source (tests that plant a
    mistake in the oracle use this) with the oracle's flags; returns the
    library path."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "ncorp_oracle_variant.c")
    with open(src, "w") as f:
        f.write(source_text)
    out = os.path.join(out_dir, "libncorp_oracle_variant.so")
    subprocess.check_call(["gcc", *CFLAGS, src, "-o", out, "-lm"])
    return out


def source() -> str:
    with open(_SRC) as f:
        return f.read()


class use_library:
    """Context manager: every function of this module calls the library at
    `path` (an oracle variant) instead of the oracle itself."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        build()
        with _lock:
            self.saved = _lib
            _lib = _bind(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def _bind(path):
    L = C.CDLL(path)
    PP = C.POINTER(Params)
    i64, dbl = C.c_int64, C.c_double
    L.or_root.argtypes = [i64, _dp, _dp]
    L.or_hilbert_key.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_int]
    L.or_hilbert_key.restype = C.c_uint64
    L.or_keys.argtypes = [i64, _dp, _dp, _u32p, _up]
    L.or_theta.argtypes = [dbl, dbl, dbl]
    L.or_theta.restype = dbl
    L.or_dtensor.argtypes = [C.c_int, _dp, _dp]
    L.or_p2m.argtypes = [C.c_int, i64, _dp, _dp, _dp, _dp]
    L.or_m2m.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
    L.or_m2l.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    L.or_l2l.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
    L.or_l2p.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
    L.or_direct_accel.argtypes = [i64, _dp, _dp, dbl, i64, _opt(_ip), _dp]
    L.or_external_accel.argtypes = [PP, i64, _dp, dbl, _dp]
    L.or_collide_pair.argtypes = [_dp, _dp, dbl, _dp, _dp, dbl, dbl]
    L.or_collide_pair.restype = C.c_int
    L.or_collide_brute.argtypes = [i64, _dp, _dp, _dp, dbl, _ip, i64]
    L.or_collide_brute.restype = i64
    L.or_resolve.argtypes = [i64, _dp, _dp, _dp, _dp, dbl, _ip, i64, _opt(_ip)]
    L.or_resolve.restype = i64
    L.or_falcon_accel.argtypes = [PP, i64, _dp, _dp, _dp, _ip]
    L.or_falcon_accel.restype = C.c_int
    L.or_standard_accel.argtypes = [PP, i64, _dp, _dp, _dp, _ip]
    L.or_standard_accel.restype = C.c_int
    L.or_m2p.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
    L.or_collide_tree.argtypes = [PP, i64, _dp, _dp, _dp, dbl, _ip, i64, _ip]
    L.or_collide_tree.restype = i64
    L.or_collide_standard.argtypes = [PP, i64, _dp, _dp, _dp, dbl, _ip, i64, _ip]
    L.or_collide_standard.restype = i64
    L.or_tree_export.argtypes = [PP, i64, _dp, _opt(_dp), _opt(_dp), _opt(_dp), dbl,
                                 _opt(_ip), _opt(_up), _opt(_dp), _opt(_ip), _opt(_dp), _opt(_dp), i64]
    L.or_tree_export.restype = i64
    L.or_expansions.argtypes = [PP, i64, _dp, _dp, _opt(_dp), _opt(_dp), i64]
    L.or_expansions.restype = i64
    L.or_kdk.argtypes = [PP, i64, _dp, _dp, _dp, _dp, dbl, C.c_int, _opt(_dp), _opt(_dp), _ip, i64,
                         _opt(_ip)]
    L.or_kdk.restype = i64
    return L


# Thresholds used in the paper's performance runs (Sect. 4.2): collisions
# N_cs = 12, N_cc,pre = 0, N_cc,post = 16; gravity p = 3: 64 / 8 / 64;
# gravity p = 6: 256 / 256 / 512.
def default_gravity_thresholds(p: int):
    return (256, 256, 512) if p >= 6 else (64, 8, 64)


def params(p=3, theta=0.5, leaf_size=17, G=1.0, central_mass=1.0, gravity_thresholds=None,
           collision_thresholds=(12, 0, 16), star=None, time=0.0, m2m_direct=False,
           brute_collisions=False, bulge=None, resolve_f=0.0, standard_thresholds=(6, 16),
           standard_collision_thresholds=(0, 16)) -> Params:
    """bulge: (R_c, J2) of the central body's equatorial bulge (App. B.2), None = no bulge.
    resolve_f: 0 = colliding pairs are only reported; 1 <= f <= 2 = kdk() resolves them (Sect. 5).
    standard_thresholds: (N_cb,pre, N_cb,post) of Algorithm StandardTree (Sect. 3.4.4; 6 and 16 in Sect. 4.2),
    and standard_collision_thresholds the same for its collision search (0 and 16 in Sect. 4.2)."""
    g = gravity_thresholds if gravity_thresholds is not None else default_gravity_thresholds(p)
    P = Params()
    P.G, P.central_mass, P.p, P.theta_min, P.leaf_size = G, central_mass, int(p), theta, int(leaf_size)
    P.n_cs, P.n_cc_pre, P.n_cc_post = (int(v) for v in g)
    P.c_cs, P.c_cc_pre, P.c_cc_post = (int(v) for v in collision_thresholds)
    if star:
        P.star_mass, P.star_a, P.star_obliquity = star
    P.time = time
    P.m2m_direct = int(bool(m2m_direct))
    P.brute_collisions = int(bool(brute_collisions))
    if bulge:
        P.central_radius, P.central_J2 = bulge
    P.resolve_f = float(resolve_f)
    P.n_cb_pre, P.n_cb_post = (int(v) for v in standard_thresholds)
    P.c_cb_pre, P.c_cb_post = (int(v) for v in standard_collision_thresholds)
    return P


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


# ---- keys -------------------------------------------------------------------
def root(pos):
    pos = _f64(pos)
    out = np.zeros(4)
    lib().or_root(len(pos), pos.reshape(-1), out)
    return out


def keys(pos):
    """(root[4], q[n,3] uint32, keys[n] uint64)"""
    pos = _f64(pos)
    n = len(pos)
    r = np.zeros(4)
    q = np.zeros((max(n, 1), 3), dtype=np.uint32)
    k = np.zeros(max(n, 1), dtype=np.uint64)
    lib().or_keys(n, pos.reshape(-1), r, q.reshape(-1), k)
    return r, q[:n], k[:n]


def hilbert_key(x, y, z, bits=21) -> int:
    return int(lib().or_hilbert_key(int(x), int(y), int(z), int(bits)))


def theta(M, Mtot, theta_min) -> float:
    return float(lib().or_theta(float(M), float(Mtot), float(theta_min)))


# ---- tensors ------------------------------------------------------------------
def off(n):
    return (3 ** n - 1) // 2


def dtensor(n, R):
    out = np.zeros(3 ** n)
    lib().or_dtensor(int(n), _f64(R), out)
    return out.reshape((3,) * n) if n > 0 else out


def p2m(p, pos, mu, s):
    pos = _f64(pos)
    out = np.zeros(off(p))
    lib().or_p2m(int(p), len(pos), pos.reshape(-1), _f64(mu), _f64(s), out)
    return out


def m2m(p, M_child, s_child, s_parent):
    out = np.zeros(off(p))
    lib().or_m2m(int(p), _f64(M_child), _f64(s_child), _f64(s_parent), out)
    return out


def m2l(p, sA, MA, sB, MB):
    CA, CB = np.zeros(off(p + 1)), np.zeros(off(p + 1))
    lib().or_m2l(int(p), _f64(sA), _f64(MA), _f64(sB), _f64(MB), CA, CB)
    return CA, CB


def l2l(p, Cin, s0, s1):
    out = np.zeros(off(p + 1))
    lib().or_l2l(int(p), _f64(Cin), _f64(s0), _f64(s1), out)
    return out


def l2p(p, Cin, s, x):
    out = np.zeros(3)
    lib().or_l2p(int(p), _f64(Cin), _f64(s), _f64(x), out)
    return out


# ---- forces ---------------------------------------------------------------------
def direct_accel(pos, mass, G=1.0, targets=None):
    pos = _f64(pos)
    n = len(pos)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if t is None else len(t)
    out = np.zeros((max(nt, 1), 3))
    lib().or_direct_accel(n, pos.reshape(-1), _f64(mass), float(G), nt, t, out.reshape(-1))
    return out[:nt]


def external_accel(P: Params, pos, t=0.0):
    pos = _f64(pos)
    out = np.zeros((max(len(pos), 1), 3))
    lib().or_external_accel(C.byref(P), len(pos), pos.reshape(-1), float(t), out.reshape(-1))
    return out[:len(pos)]


def falcon_accel(P: Params, pos, mass):
    """(mutual acceleration [n,3], stats dict)"""
    pos = _f64(pos)
    n = len(pos)
    out = np.zeros((max(n, 1), 3))
    st = np.zeros(16, dtype=np.int64)
    lib().or_falcon_accel(C.byref(P), n, pos.reshape(-1), _f64(mass), out.reshape(-1), st)
    return out[:n], dict(zip(STAT_NAMES, (int(v) for v in st)))


def standard_accel(P: Params, pos, mass):
    """Mutual acceleration by the standard tree code (Algorithm StandardTree), and its counters
    (m2l = moonlet-cell expansions, p2p_pairs = brute-force moonlet-cell interactions)."""
    pos = _f64(pos)
    n = len(pos)
    out = np.zeros((max(n, 1), 3))
    st = np.zeros(16, dtype=np.int64)
    lib().or_standard_accel(C.byref(P), n, pos.reshape(-1), _f64(mass), out.reshape(-1), st)
    return out[:n], dict(zip(STAT_NAMES, (int(v) for v in st)))


def m2p(p, x, sB, MB):
    """C^(1) at x of the expansion MB (packed full tensors, orders 0..p-1) about sB."""
    out = np.zeros(3)
    lib().or_m2p(int(p), _f64(x), _f64(sB), _f64(MB), out)
    return out


# ---- collisions -------------------------------------------------------------------
def collide_pair(x1, v1, R1, x2, v2, R2, dt) -> bool:
    return bool(lib().or_collide_pair(_f64(x1), _f64(v1), float(R1), _f64(x2), _f64(v2), float(R2), float(dt)))


def collide_brute(pos, vel, rad, dt, cap=1 << 16):
    pos, vel = _f64(pos), _f64(vel)
    out = np.zeros((cap, 2), dtype=np.int64)
    n = lib().or_collide_brute(len(pos), pos.reshape(-1), vel.reshape(-1), _f64(rad), float(dt), out.reshape(-1), cap)
    if n > cap:
        return collide_brute(pos, vel, rad, dt, cap=int(n))
    return out[:n]


def collide_tree(P: Params, pos, vel, rad, dt, cap=1 << 16):
    pos, vel = _f64(pos), _f64(vel)
    out = np.zeros((cap, 2), dtype=np.int64)
    st = np.zeros(16, dtype=np.int64)
    n = lib().or_collide_tree(C.byref(P), len(pos), pos.reshape(-1), vel.reshape(-1), _f64(rad), float(dt),
                              out.reshape(-1), cap, st)
    if n > cap:
        return collide_tree(P, pos, vel, rad, dt, cap=int(n))
    return out[:n], dict(zip(STAT_NAMES, (int(v) for v in st)))


def resolve(pos, vel, mass, rad, f, pairs):
    """Resolves colliding pairs (rows i < j) of one step (Sect. 5.1-5.2); returns (positions the drift
    starts from, new velocities, per-pair resolved flags)."""
    pos, vel = _f64(pos).copy(), _f64(vel).copy()
    pr = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    done = np.zeros(max(len(pr), 1), dtype=np.int64)
    lib().or_resolve(len(pos), pos.reshape(-1), vel.reshape(-1), _f64(mass), _f64(rad), float(f),
                     pr.reshape(-1) if len(pr) else np.zeros(2, dtype=np.int64), len(pr), done)
    return pos, vel, done[:len(pr)].astype(bool)


def collide_standard(P: Params, pos, vel, rad, dt, cap=1 << 16):
    """Colliding pairs found by the standard tree code's collision search, and its counters."""
    pos, vel = _f64(pos), _f64(vel)
    out = np.zeros((cap, 2), dtype=np.int64)
    st = np.zeros(16, dtype=np.int64)
    n = lib().or_collide_standard(C.byref(P), len(pos), pos.reshape(-1), vel.reshape(-1), _f64(rad), float(dt),
                                  out.reshape(-1), cap, st)
    if n > cap:
        return collide_standard(P, pos, vel, rad, dt, cap=int(n))
    return out[:n], dict(zip(STAT_NAMES, (int(v) for v in st)))


def tree_export(P: Params, pos, mass=None, vel=None, rad=None, dt=0.0):
    """Canonical order, keys, root, cells[k,7], gravity geometry[k,6], collision geometry[k,5]."""
    pos = _f64(pos)
    n = len(pos)
    cap = 4 * n + 64
    ord_ = np.zeros(n, dtype=np.int64)
    k = np.zeros(n, dtype=np.uint64)
    r = np.zeros(4)
    cells = np.zeros((cap, 7), dtype=np.int64)
    gg = np.zeros((cap, 6)) if mass is not None else None
    cg = np.zeros((cap, 5)) if vel is not None else None
    m = None if mass is None else _f64(mass)
    v = None if vel is None else _f64(vel).reshape(-1)
    rd = None if rad is None else _f64(rad)
    nc = lib().or_tree_export(C.byref(P), n, pos.reshape(-1), m, v, rd, float(dt), ord_, k, r,
                              cells.reshape(-1), None if gg is None else gg.reshape(-1),
                              None if cg is None else cg.reshape(-1), cap)
    return {"order": ord_, "keys": k, "root": r, "cells": cells[:nc],
            "ggeo": None if gg is None else gg[:nc], "cgeo": None if cg is None else cg[:nc]}


def expansions(P: Params, pos, mass):
    """Per-cell multipoles M[k][(3^p-1)/2] and M2L sums C[k][(3^(p+1)-1)/2] (full tensors, packed by order),
    level-major cell order, before the descent."""
    pos = _f64(pos)
    n = len(pos)
    cap = 4 * n + 64
    M = np.zeros((cap, off(P.p)))
    Cc = np.zeros((cap, off(P.p + 1)))
    nc = lib().or_expansions(C.byref(P), n, pos.reshape(-1), _f64(mass), M.reshape(-1), Cc.reshape(-1), cap)
    return M[:nc], Cc[:nc]


def full_to_multi(T, order):
    """Symmetric multi-index components (a, b, c) of a full order-n tensor given flat, in the library's
    packed order (k = b + c = 0..n, c = 0..k)."""
    out = []
    for k in range(order + 1):
        for c in range(k + 1):
            a, b = order - k, k - c
            idx = 0
            for d in [0] * a + [1] * b + [2] * c:
                idx = idx * 3 + d
            out.append(T[idx])
    return np.array(out)


def kdk(P: Params, pos, vel, mass, rad, dt, nsteps, acc0=None, cap=1 << 16, info=None):
    """Runs nsteps KDK steps; returns (pos, vel, acc, pairs[k,3] as (step, i, j)).  With a dict as
    info, info["resolved"] receives the number of resolved impacts (-1: the pair buffer overflowed)."""
    pos, vel = _f64(pos).copy(), _f64(vel).copy()
    n = len(pos)
    acc = np.zeros((max(n, 1), 3))
    out = np.zeros((cap, 3), dtype=np.int64)
    a0 = None if acc0 is None else _f64(acc0).reshape(-1)
    res = np.zeros(1, dtype=np.int64)
    tot = lib().or_kdk(C.byref(P), n, pos.reshape(-1), vel.reshape(-1), _f64(mass), _f64(rad), float(dt),
                       int(nsteps), a0, acc.reshape(-1), out.reshape(-1), cap, res)
    if info is not None:
        info["resolved"] = int(res[0])
    return pos, vel, acc[:n], out[:min(tot, cap)]
