"""ctypes binding of the serial CPU oracle (oracle.cpp).

Test infrastructure only: the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this module; the GPU package never does. The oracle is built from source
with g++ on first use (or by `build()`), into `oracle/_build/`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_HDR = os.path.join(_HERE, "oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EDEGENERATE, ETOOSMALL, EINTERNAL = 0, -1, -2, -3, -4
BAD_ORIENT, BAD_ADJACENCY, BAD_DELAUNAY, BAD_GHOST, BAD_HULLCOUNT = 1, 2, 4, 8, 16


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "n_points", "n_unique", "n_dups", "n_tets", "n_ghosts", "n_hull_vertices",
        "sum_cavity", "sum_ball", "sum_walk", "n_insphere", "n_exact", "n_sos",
        "validate_flags")]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain g++, no contraction of multiply-adds)."""
    with _lock:
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                   "-o", tmp, _SRC]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        p = ctypes.c_void_p
        i64 = ctypes.c_int64
        u64 = ctypes.c_uint64
        L.oracle_moore_keys.argtypes = [p, i64, p]
        L.oracle_moore_index.argtypes = [p, i64, ctypes.c_int, p]
        L.oracle_brio_rounds.argtypes = [i64, u64, p]
        L.oracle_insertion_order.argtypes = [p, i64, u64, p]
        L.oracle_dedup.argtypes = [p, i64, p]
        L.oracle_orient3d.argtypes = [p]
        L.oracle_insphere.argtypes = [p]
        L.oracle_insphere_sos.argtypes = [p, p]
        L.oracle_insphere_value.argtypes = [p]
        L.oracle_insphere_value.restype = ctypes.c_double
        L.oracle_orient3d_value.argtypes = [p]
        L.oracle_orient3d_value.restype = ctypes.c_double
        L.oracle_delaunay.argtypes = [p, i64, u64, p, p, i64, ctypes.c_int, ctypes.POINTER(Stats)]
        L.oracle_delaunay.restype = i64
        L.oracle_brute_force.argtypes = [p, i64, p, i64]
        L.oracle_brute_force.restype = i64
        L.oracle_adjacency.argtypes = [p, i64, p]
        L.oracle_set_mutation.argtypes = [ctypes.c_int]
        L.oracle_set_mutation.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _xyz(xyz):
    a = np.ascontiguousarray(xyz, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("xyz must be [n, 3]")
    return a


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}")
        self.code = code


def moore_keys(xyz) -> np.ndarray:
    a = _xyz(xyz)
    keys = np.empty(len(a), dtype=np.uint64)
    rc = lib().oracle_moore_keys(_ptr(a), len(a), _ptr(keys))
    if rc:
        raise OracleError(rc)
    return keys


def moore_index(q, m: int) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.uint32).reshape(-1, 3)
    keys = np.empty(len(q), dtype=np.uint64)
    rc = lib().oracle_moore_index(_ptr(q), len(q), m, _ptr(keys))
    if rc:
        raise OracleError(rc)
    return keys


def brio_rounds(n: int, seed: int) -> np.ndarray:
    r = np.empty(n, dtype=np.uint8)
    rc = lib().oracle_brio_rounds(n, seed, _ptr(r))
    if rc:
        raise OracleError(rc)
    return r


def insertion_order(xyz, seed: int) -> np.ndarray:
    a = _xyz(xyz)
    perm = np.empty(len(a), dtype=np.uint32)
    rc = lib().oracle_insertion_order(_ptr(a), len(a), seed, _ptr(perm))
    if rc:
        raise OracleError(rc)
    return perm


def dedup(xyz) -> np.ndarray:
    a = _xyz(xyz)
    rep = np.empty(len(a), dtype=np.uint32)
    rc = lib().oracle_dedup(_ptr(a), len(a), _ptr(rep))
    if rc:
        raise OracleError(rc)
    return rep


def orient3d(a, b, c, d) -> int:
    p = np.ascontiguousarray(np.array([a, b, c, d], dtype=np.float64).reshape(12))
    return lib().oracle_orient3d(_ptr(p))


def insphere(a, b, c, d, e) -> int:
    p = np.ascontiguousarray(np.array([a, b, c, d, e], dtype=np.float64).reshape(15))
    return lib().oracle_insphere(_ptr(p))


def insphere_sos(pts, ids) -> int:
    p = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(15))
    i = np.ascontiguousarray(np.asarray(ids, dtype=np.int64).reshape(5))
    return lib().oracle_insphere_sos(_ptr(p), _ptr(i))


def insphere_value(a, b, c, d, e) -> float:
    p = np.ascontiguousarray(np.array([a, b, c, d, e], dtype=np.float64).reshape(15))
    return lib().oracle_insphere_value(_ptr(p))


def orient3d_value(a, b, c, d) -> float:
    p = np.ascontiguousarray(np.array([a, b, c, d], dtype=np.float64).reshape(12))
    return lib().oracle_orient3d_value(_ptr(p))


def delaunay(xyz, seed: int = 0, order=None, validate: bool = False, cap: int | None = None):
    """Canonical sorted finite tetrahedra [T, 4] (uint32 input indices) and the stats dict."""
    a = _xyz(xyz)
    n = len(a)
    if cap is None:
        cap = max(64, 8 * n + 64)
    out = np.empty((cap, 4), dtype=np.uint32)
    st = Stats()
    order_arr = None
    if order is not None:
        order_arr = np.ascontiguousarray(order, dtype=np.int64)
    rc = lib().oracle_delaunay(_ptr(a), n, seed,
                               _ptr(order_arr) if order_arr is not None else None,
                               _ptr(out), cap, 1 if validate else 0, ctypes.byref(st))
    if rc == ETOOSMALL:
        return delaunay(xyz, seed, order, validate, cap=st.n_tets)
    if rc < 0:
        raise OracleError(rc)
    return out[:rc].copy(), st.as_dict()


def brute_force(xyz) -> np.ndarray:
    a = _xyz(xyz)
    cap = 200000
    out = np.empty((cap, 4), dtype=np.uint32)
    rc = lib().oracle_brute_force(_ptr(a), len(a), _ptr(out), cap)
    if rc < 0:
        raise OracleError(rc)
    return out[:rc].copy()


def adjacency(tets) -> np.ndarray:
    t = np.ascontiguousarray(tets, dtype=np.uint32).reshape(-1, 4)
    nbr = np.empty_like(t)
    rc = lib().oracle_adjacency(_ptr(t), len(t), _ptr(nbr))
    if rc:
        raise OracleError(rc)
    return nbr


def set_mutation(k: int) -> None:
    lib().oracle_set_mutation(k)


__all__ = [name for name in dir() if not name.startswith("_")]
