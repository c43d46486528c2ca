"""ctypes binding of the paper's CPU parallel insertion (paper_cpu.cpp, Sections 3.2 to 3.4), a
second host baseline beside the serial oracle.

Test and baseline infrastructure only: the tests and the CPU legs of `bench.py` use it; the GPU
package never does. Built from source with g++ on first use (or by `build()`), into
`oracle/_build/`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "paper_cpu.cpp")
_DEPS = [_SRC, os.path.join(_HERE, "oracle.cpp"), os.path.join(_HERE, "oracle.h")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libpaper_cpu.so")
_lock = threading.Lock()
_lib = None

STATS = ("n_unique", "n_tets", "passes", "aborted", "one_thread_passes", "max_threads", "sum_cavity", "sum_ball",
         "sum_walk")


def build(force: bool = False) -> str:
    """Compile libpaper_cpu.so (g++, threads, no contraction of multiply-adds)."""
    with _lock:
        stale = not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(d) for d in _DEPS)
        if force or stale:
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                            "-o", tmp, _SRC], check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        p, i64 = ctypes.c_void_p, ctypes.c_int64
        L.paper_cpu_delaunay.argtypes = [p, i64, ctypes.c_uint64, ctypes.c_int, i64, p, i64, p]
        L.paper_cpu_delaunay.restype = i64
        _lib = L
    return _lib


def delaunay(xyz, threads: int, seed: int = 0, min_per_thread: int = 3000):
    """Canonical sorted finite tetrahedra [T, 4] (uint32 input indices, as oracle.delaunay) and a
    stats dict, from the paper's thread scheme with up to `threads` threads."""
    a = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64))
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("xyz must be [n, 3]")
    n = len(a)
    cap = max(64, 8 * n + 64)
    st = np.zeros(len(STATS), dtype=np.int64)
    while True:
        out = np.empty((cap, 4), dtype=np.uint32)
        rc = lib().paper_cpu_delaunay(a.ctypes.data, n, seed, int(threads), int(min_per_thread), out.ctypes.data,
                                      cap, st.ctypes.data)
        if rc == -3 and st[1] > cap:  # too small: the count is in the stats
            cap = int(st[1])
            continue
        break
    if rc < 0:
        raise RuntimeError(f"paper_cpu_delaunay failed ({rc})")
    return out[:rc].copy(), dict(zip(STATS, (int(v) for v in st)))
