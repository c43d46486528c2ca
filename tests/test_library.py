"""CPU-side checks of the native library: it builds for sm_103a, loads, and exports the C ABI."""
import ctypes

import paper_1805_08831_gb300 as dt


def test_library_exports_every_declared_symbol():
    L = dt.lib()
    names = dt.exported_names()
    assert "dt_create" in names and "dt_insert" in names and "dt_get_tets" in names
    for name in names:
        assert hasattr(L, name), name


def test_strerror_and_argument_checks_need_no_gpu():
    L = dt.lib()
    assert L.dt_strerror(dt.DT_EDEGENERATE).decode().startswith("fewer than four")
    assert L.dt_create(None, None) == dt.DT_EINVAL
    cfg = dt.Config()
    cfg.reserved[0] = 1
    h = ctypes.c_void_p()
    assert L.dt_create(ctypes.byref(h), ctypes.byref(cfg)) == dt.DT_EINVAL
    assert L.dt_insert(None, None, 0) == dt.DT_EINVAL
    assert L.dt_get_stats(None, None) == dt.DT_EINVAL
    assert L.dt_eval_predicates(7, None, None, None, 0, None) == dt.DT_EINVAL
    L.dt_destroy(None)
