"""Python binding of the GB300 concurrent 3D Delaunay library (C ABI in include/dt.h).

Argument marshalling only: every step of the triangulation runs in the CUDA kernels of
libdt_gb300.so. PyTorch supplies device memory and streams. There is no CPU fallback: if the
library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dt.h")

DT_OK, DT_EINVAL, DT_ENOMEM, DT_ETOOSMALL, DT_EDEGENERATE, DT_ELIMIT, DT_ECUDA, DT_ESTATE = (
    0, -1, -2, -3, -4, -5, -6, -7)
DT_SCHED_PLAIN, DT_SCHED_LEARNED = 0, 1
DT_FLAG_NO_CANONICAL_SORT = 1
DT_FLAG_PROFILE = 2
DT_FLAG_LOG = 4
DT_MLP_PARAMS = 1410
DT_FEATURES = 8


class Config(ctypes.Structure):
    _fields_ = [
        ("tet_capacity_factor", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("stream", ctypes.c_void_p),
        ("schedule", ctypes.c_uint32),
        ("max_walk_steps", ctypes.c_uint32),
        ("max_rounds", ctypes.c_uint32),
        ("segments", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32 * 5),
    ]


_STAT_FIELDS = ["n_points", "n_unique", "n_dups", "n_tets", "n_slots", "n_rounds", "n_passes",
                "n_attempts", "n_conflicts", "n_big", "sum_cavity", "sum_ball", "sum_walk",
                "n_exact", "n_sos"]


class Stats(ctypes.Structure):
    _fields_ = ([(f, ctypes.c_uint64) for f in _STAT_FIELDS]
                + [("ms_sort", ctypes.c_double), ("ms_insert", ctypes.c_double),
                   ("n_launches", ctypes.c_uint64), ("ms_walk", ctypes.c_double),
                   ("ms_cavity", ctypes.c_double), ("ms_insert_k", ctypes.c_double),
                   ("n_profiled", ctypes.c_uint64), ("device_error", ctypes.c_uint64),
                   ("device_error_info", ctypes.c_uint64), ("n_rounds_wave", ctypes.c_uint64),
                   ("n_rounds_retry", ctypes.c_uint64), ("n_rounds_big", ctypes.c_uint64),
                   ("ms_first_round", ctypes.c_double), ("n_walk_limit", ctypes.c_uint64),
                   ("free_slots", ctypes.c_uint64), ("max_walk", ctypes.c_uint64),
                   ("n_clouds_degenerate", ctypes.c_uint64), ("batch_warps", ctypes.c_uint64),
                   ("batch_alpha", ctypes.c_double), ("ms_batch_tune", ctypes.c_double),
                   ("batch_graph", ctypes.c_uint64), ("batch_min_blocks", ctypes.c_uint64),
                   ("ms_async", ctypes.c_double), ("n_async", ctypes.c_uint64),
                   ("n_restarts", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                   ("n_exact_handoff", ctypes.c_uint64), ("n_inserted_async", ctypes.c_uint64),
                   ("reserved", ctypes.c_uint64 * 2)])

    def as_dict(self):
        d = {f: getattr(self, f) for f in _STAT_FIELDS}
        for f in ("ms_sort", "ms_insert", "n_launches", "ms_walk", "ms_cavity", "ms_insert_k",
                  "n_profiled", "device_error", "device_error_info", "n_rounds_wave",
                  "n_rounds_retry", "n_rounds_big", "ms_first_round", "n_walk_limit", "free_slots",
                  "max_walk", "n_clouds_degenerate", "batch_warps", "batch_alpha", "ms_batch_tune",
                  "batch_graph", "batch_min_blocks", "ms_async", "n_async", "n_restarts", "device_bytes", "n_exact_handoff", "n_inserted_async"):
            d[f] = getattr(self, f)
        return d


class DTError(RuntimeError):
    def __init__(self, code, what=""):
        lib_ = _lib
        msg = lib_.dt_strerror(code).decode() if lib_ is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")
        self.code = code


_lib = None


def exported_names():
    """Names of the functions declared in include/dt.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:int|void|const char\*)\s+(dt_\w+)\s*\(", text, re.M)))


def lib():
    """Loads libdt_gb300.so, building it first when it is missing or stale."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        p, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
        L.dt_create.argtypes = [ctypes.POINTER(p), ctypes.POINTER(Config)]
        L.dt_insert.argtypes = [p, p, u64]
        L.dt_insert_host.argtypes = [p, p, u64]
        L.dt_batch.argtypes = [p, p, p, u32]
        L.dt_get_tets.argtypes = [p, p, u64, ctypes.POINTER(u64), p, ctypes.c_int]
        L.dt_get_tets_host.argtypes = [p, p, u64, ctypes.POINTER(u64), ctypes.c_int]
        L.dt_get_order.argtypes = [p, p, p, p]
        L.dt_get_stats.argtypes = [p, ctypes.POINTER(Stats)]
        L.dt_load_model.argtypes = [p, p, u32]
        L.dt_clear.argtypes = [p]
        L.dt_destroy.argtypes = [p]
        L.dt_destroy.restype = None
        L.dt_strerror.argtypes = [ctypes.c_int]
        L.dt_strerror.restype = ctypes.c_char_p
        L.dt_eval_predicates.argtypes = [ctypes.c_int, p, p, p, u64, p]
        L.dt_order_noalloc.argtypes = [p, u64, u64, p, p, p, p]
        L.dt_get_features.argtypes = [p, p, p, p, u64]
        L.dt_mlp_forward.argtypes = [p, p, u64, p, p]
        L.dt_mlp_grad.argtypes = [p, p, p, u64, p, p, p]
        L.dt_mlp_train.argtypes = [p, p, p, u64, u32, u32, ctypes.c_float, u64, p, p]
        L.dt_refine.argtypes = [p, ctypes.c_double, ctypes.c_double, ctypes.c_double, p, u32,
                                ctypes.POINTER(u64), ctypes.POINTER(u32)]
        L.dt_get_points.argtypes = [p, p, u64, ctypes.POINTER(u64)]
        L.dt_check.argtypes = [p, p]
        for name in exported_names():
            getattr(L, name)
        _lib = L
    return _lib


def _check(rc, what):
    if rc != DT_OK:
        raise DTError(rc, what)


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream)


class Triangulation:
    """One triangulation on the current CUDA device (a dt_handle)."""

    def __init__(self, seed: int = 0, stream=None, schedule: int = DT_SCHED_PLAIN,
                 tet_capacity_factor: float = 0.0, segments: int = 0, max_walk_steps: int = 0,
                 max_rounds: int = 0, flags: int = 0):
        L = lib()
        cfg = Config()
        cfg.tet_capacity_factor = tet_capacity_factor
        cfg.seed = seed
        cfg.stream = _stream_ptr(stream)
        cfg.schedule = schedule
        cfg.max_walk_steps = max_walk_steps
        cfg.max_rounds = max_rounds
        cfg.segments = segments
        cfg.flags = flags
        self._stream = stream
        self._h = ctypes.c_void_p()
        _check(L.dt_create(ctypes.byref(self._h), ctypes.byref(cfg)), "dt_create")

    def close(self):
        if self._h:
            lib().dt_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def clear(self):
        """Starts over with an empty triangulation, keeping the device memory."""
        _check(lib().dt_clear(self._h), "dt_clear")

    def _check_dev(self, rc, what):
        if rc != DT_OK:
            st = Stats()
            lib().dt_get_stats(self._h, ctypes.byref(st))
            raise DTError(rc, f"{what} (device error {st.device_error}, info {st.device_error_info:#x})")

    def insert(self, xyz):
        """Inserts a CUDA float64 tensor [n, 3] (device pointer path)."""
        torch = _torch()
        if not (isinstance(xyz, torch.Tensor) and xyz.is_cuda and xyz.dtype == torch.float64):
            raise TypeError("xyz must be a CUDA float64 tensor [n, 3]")
        xyz = xyz.contiguous()
        if xyz.dim() != 2 or xyz.shape[1] != 3:
            raise ValueError("xyz must be [n, 3]")
        self._check_dev(lib().dt_insert(self._h, ctypes.c_void_p(xyz.data_ptr()), xyz.shape[0]), "dt_insert")

    def insert_host(self, xyz):
        """Inserts host float64 points [n, 3] (copied to the device inside the call)."""
        a = np.ascontiguousarray(xyz, dtype=np.float64)
        if a.ndim != 2 or a.shape[1] != 3:
            raise ValueError("xyz must be [n, 3]")
        self._check_dev(lib().dt_insert_host(self._h, a.ctypes.data_as(ctypes.c_void_p), a.shape[0]),
                        "dt_insert_host")

    def refine(self, size: float, box=(0.0, 0.0, 0.0, 1.0, 1.0, 1.0), ratio: float = 1.4,
               spacing: float = 0.7, max_iters: int = 100):
        """Delaunay refinement inside the box (dt_refine): circumcentres of tetrahedra with
        r > ratio * size, spaced at least spacing * size from every point, inserted until none
        is left. Returns (points added, iterations)."""
        b = (ctypes.c_double * 6)(*[float(v) for v in box])
        added, iters = ctypes.c_uint64(), ctypes.c_uint32()
        self._check_dev(lib().dt_refine(self._h, float(size), float(ratio), float(spacing), b, int(max_iters),
                                        ctypes.byref(added), ctypes.byref(iters)), "dt_refine")
        return added.value, iters.value

    def points(self):
        """Every point given to the handle, by input index, as a CUDA float64 tensor [n, 3]."""
        torch = _torch()
        n = ctypes.c_uint64()
        _check(lib().dt_get_points(self._h, None, 0, ctypes.byref(n)), "dt_get_points")
        out = torch.empty((n.value, 3), dtype=torch.float64, device="cuda")
        if n.value:
            _check(lib().dt_get_points(self._h, ctypes.c_void_p(out.data_ptr()), n.value, ctypes.byref(n)),
                   "dt_get_points")
        return out

    def check(self):
        """Device certificate of the mesh (dt_check): dict of live finite tetrahedra, bad
        adjacencies, non-positive orientations, non-locally-Delaunay facets and vertices used."""
        out = (ctypes.c_uint64 * 5)()
        self._check_dev(lib().dt_check(self._h, out), "dt_check")
        return {"tets": out[0], "bad_adjacency": out[1], "bad_orientation": out[2],
                "not_delaunay": out[3], "vertices": out[4]}

    def batch(self, xyz, offsets):
        """Triangulates independent clouds in one call: xyz is a CUDA float64 tensor [N, 3] with
        the clouds back to back, offsets the n_clouds + 1 row offsets (host, offsets[0] = 0)."""
        torch = _torch()
        if not (isinstance(xyz, torch.Tensor) and xyz.is_cuda and xyz.dtype == torch.float64):
            raise TypeError("xyz must be a CUDA float64 tensor [N, 3]")
        xyz = xyz.contiguous()
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        if off.ndim != 1 or off.size < 2:
            raise ValueError("offsets must hold n_clouds + 1 entries")
        self._check_dev(lib().dt_batch(self._h, ctypes.c_void_p(xyz.data_ptr()),
                                       off.ctypes.data_as(ctypes.c_void_p), off.size - 1), "dt_batch")
        self._n_clouds = off.size - 1

    def tets_batch(self, canonical: bool = True, out=None):
        """After batch(): (tets numpy uint32 [T, 4] with cloud-local ids, cloud_offsets numpy
        uint64 [n_clouds + 1]); each cloud's rows are canonical on their own. out: a page-locked
        host uint32 array [rows, 4] (e.g. from torch's pin_memory) that receives the rows
        directly when it is large enough."""
        torch = _torch()
        nc = self._n_clouds
        coff = np.zeros(nc + 1, dtype=np.uint64)
        n = ctypes.c_uint64()
        if out is not None:
            if not (isinstance(out, np.ndarray) and out.dtype == np.uint32 and out.ndim == 2
                    and out.shape[1] == 4 and out.flags.c_contiguous):
                raise TypeError("out must be a C-contiguous uint32 array [rows, 4]")
            rc = lib().dt_get_tets(self._h, out.ctypes.data_as(ctypes.c_void_p), out.shape[0], ctypes.byref(n),
                                   coff.ctypes.data_as(ctypes.c_void_p), 1 if canonical else 0)
            if rc == DT_OK:
                return out[: n.value], coff
            if rc not in (DT_ETOOSMALL, DT_EINVAL):  # DT_EINVAL: pageable memory, not written
                _check(rc, "dt_get_tets")
        rc = lib().dt_get_tets(self._h, None, 0, ctypes.byref(n), coff.ctypes.data_as(ctypes.c_void_p), 0)
        if rc not in (DT_OK, DT_ETOOSMALL):
            _check(rc, "dt_get_tets")
        T = n.value
        out = torch.empty((max(T, 1), 4), dtype=torch.int32, device="cuda")
        _check(lib().dt_get_tets(self._h, ctypes.c_void_p(out.data_ptr()), T, ctypes.byref(n),
                                 coff.ctypes.data_as(ctypes.c_void_p), 1 if canonical else 0), "dt_get_tets")
        return out[: n.value].cpu().numpy().view(np.uint32), coff

    def num_tets(self) -> int:
        n = ctypes.c_uint64()
        rc = lib().dt_get_tets(self._h, None, 0, ctypes.byref(n), None, 0)
        if rc not in (DT_OK, DT_ETOOSMALL):
            _check(rc, "dt_get_tets")
        return n.value

    def tets(self, canonical: bool = True):
        """Finite tetrahedra as a CUDA int32 tensor [T, 4] (uint32 bit patterns)."""
        torch = _torch()
        T = self.num_tets()
        out = torch.empty((max(T, 1), 4), dtype=torch.int32, device="cuda")
        n = ctypes.c_uint64()
        _check(lib().dt_get_tets(self._h, ctypes.c_void_p(out.data_ptr()), T, ctypes.byref(n), None,
                                 1 if canonical else 0), "dt_get_tets")
        return out[: n.value]

    def tets_numpy(self, canonical: bool = True) -> np.ndarray:
        return self.tets(canonical).cpu().numpy().view(np.uint32)

    def tets_host(self, canonical: bool = True, out=None) -> np.ndarray:
        """Finite tetrahedra as a host uint32 array [T, 4] (dt_get_tets_host). out: a C-contiguous
        uint32 [rows, 4] host array to fill (page-locked memory copies fastest); a new array
        is allocated when it is None or too small."""
        n = ctypes.c_uint64()
        if out is not None:
            if not (isinstance(out, np.ndarray) and out.dtype == np.uint32 and out.ndim == 2
                    and out.shape[1] == 4 and out.flags.c_contiguous):
                raise TypeError("out must be a C-contiguous uint32 array [rows, 4]")
            rc = lib().dt_get_tets_host(self._h, out.ctypes.data_as(ctypes.c_void_p), out.shape[0],
                                        ctypes.byref(n), 1 if canonical else 0)
            if rc == DT_OK:
                return out[: n.value]
            if rc != DT_ETOOSMALL:
                _check(rc, "dt_get_tets_host")
        T = self.num_tets()
        out = np.empty((max(T, 1), 4), dtype=np.uint32)
        _check(lib().dt_get_tets_host(self._h, out.ctypes.data_as(ctypes.c_void_p), T, ctypes.byref(n),
                                      1 if canonical else 0), "dt_get_tets_host")
        return out[: n.value]

    def order(self, n: int):
        """(keys uint64, perm uint32, rounds uint8) numpy arrays of the last insert of n points."""
        torch = _torch()
        keys = torch.empty(n, dtype=torch.int64, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        rounds = torch.empty(n, dtype=torch.uint8, device="cuda")
        _check(lib().dt_get_order(self._h, ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(perm.data_ptr()),
                                  ctypes.c_void_p(rounds.data_ptr())), "dt_get_order")
        return (keys.cpu().numpy().view(np.uint64), perm.cpu().numpy().view(np.uint32),
                rounds.cpu().numpy())

    def load_model(self, params):
        """Loads the learned scheduler's 1410 float32 parameters (host array)."""
        a = np.ascontiguousarray(params, dtype=np.float32).ravel()
        _check(lib().dt_load_model(self._h, a.ctypes.data_as(ctypes.c_void_p), a.size), "dt_load_model")

    def features(self, n: int, labels: bool = True):
        """Features [n, 8] of the last insert's points in insertion order (CUDA float32), and
        with labels=True (needs DT_FLAG_LOG) the labels [n, 2] and their validity [n] (uint8)."""
        torch = _torch()
        x = torch.empty((n, DT_FEATURES), dtype=torch.float32, device="cuda")
        y = torch.empty((n, 2), dtype=torch.float32, device="cuda") if labels else None
        v = torch.empty(n, dtype=torch.uint8, device="cuda") if labels else None
        _check(lib().dt_get_features(self._h, ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(y.data_ptr()) if labels else None,
                                     ctypes.c_void_p(v.data_ptr()) if labels else None, n), "dt_get_features")
        return (x, y, v) if labels else x

    def stats(self) -> dict:
        st = Stats()
        _check(lib().dt_get_stats(self._h, ctypes.byref(st)), "dt_get_stats")
        return st.as_dict()


def delaunay(xyz, seed: int = 0, **kw) -> np.ndarray:
    """Canonical sorted tetrahedra of a CUDA float64 tensor [n, 3] (numpy uint32 [T, 4])."""
    with Triangulation(seed=seed, **kw) as t:
        t.insert(xyz)
        return t.tets_numpy(canonical=True)


def eval_predicates(kind: int, pts, ids=None, stream=None):
    """Device predicate signs: kind 0 orient3d, 1 insphere, 2 perturbed insphere.
    pts: CUDA float64 [n, 5, 3]; ids: CUDA int64 [n, 5] (kind 2). Returns int8 CUDA tensor."""
    torch = _torch()
    pts = pts.contiguous()
    n = pts.shape[0]
    out = torch.empty(n, dtype=torch.int8, device=pts.device)
    idp = None
    if ids is not None:
        ids = ids.contiguous()
        idp = ctypes.c_void_p(ids.data_ptr())
    _check(lib().dt_eval_predicates(kind, ctypes.c_void_p(pts.data_ptr()), idp, ctypes.c_void_p(out.data_ptr()),
                                    n, _stream_ptr(stream)), "dt_eval_predicates")
    return out


def mlp_forward(params, x):
    """The learned scheduler's network on CUDA float32 rows x [n, 8]: [n, 2]."""
    torch = _torch()
    out = torch.empty((x.shape[0], 2), dtype=torch.float32, device=x.device)
    _check(lib().dt_mlp_forward(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(x.contiguous().data_ptr()),
                                x.shape[0], ctypes.c_void_p(out.data_ptr()), None), "dt_mlp_forward")
    return out


def mlp_grad(params, x, y):
    """(mean loss, gradient [1410]) of the network on CUDA float32 samples (x [n, 8], y [n, 2])."""
    torch = _torch()
    g = torch.empty(DT_MLP_PARAMS, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(lib().dt_mlp_grad(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(x.contiguous().data_ptr()),
                             ctypes.c_void_p(y.contiguous().data_ptr()), x.shape[0], ctypes.c_void_p(g.data_ptr()),
                             ctypes.c_void_p(loss.data_ptr()), None), "dt_mlp_grad")
    return float(loss.item()), g


def mlp_train(params, x, y, steps: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0):
    """Trains CUDA float32 params [1410] in place with the library's Adam kernels; returns the
    per-step minibatch losses (numpy)."""
    losses = np.zeros(max(steps, 1), dtype=np.float32)
    _check(lib().dt_mlp_train(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(x.contiguous().data_ptr()),
                              ctypes.c_void_p(y.contiguous().data_ptr()), x.shape[0], steps, batch, lr, seed,
                              losses.ctypes.data_as(ctypes.c_void_p), None), "dt_mlp_train")
    return losses[:steps]


def init_params(seed: int = 0) -> np.ndarray:
    """He-scaled random initial parameters (float32 [1410]) in the dt_load_model layout."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2 / 8), (8, 32)), np.zeros(32), rng.normal(0, np.sqrt(2 / 32), (32, 32)),
             np.zeros(32), rng.normal(0, np.sqrt(1 / 32), (32, 2)), np.zeros(2)]
    return np.concatenate([q.ravel() for q in parts]).astype(np.float32)

