"""The C ABI: the library loads on a CPU-only host and exports every symbol that
include/tschrod.h declares (no compute calls: there may be no GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*[A-Za-z_][A-Za-z_0-9 \t]*[\s*]+(ts_[a-z_0-9]+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_2605_20491_b300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("ts_plan_create", "ts_plan_destroy", "ts_apply_inverse", "ts_apply_exp", "ts_pcg",
                     "ts_split_step", "ts_inverse_iteration", "ts_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    import ctypes
    lib = ctypes.CDLL(built_lib)
    for name in sorted(declared_symbols()):
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2605_20491_b300 import tschrod
    assert set(tschrod.EXPORTS) == declared_symbols()


def test_version_and_error_string_without_gpu(built_lib):
    from paper_2605_20491_b300 import tschrod
    assert "sm_103a" in tschrod.ts_version()
    assert tschrod.lib().ts_plan_destroy(None) == tschrod.TS_OK  # a successful call clears the message
    assert tschrod.ts_last_error() == ""


def test_invalid_arguments_rejected_on_host(built_lib):
    """Validation happens before any device work, so it runs without a GPU."""
    import ctypes as C
    from paper_2605_20491_b300 import tschrod as T
    L = T.lib()
    out = C.c_void_p()
    assert L.ts_plan_create(None, 0, None, C.byref(out)) == T.TS_ERR_INVALID_ARG
    assert "NULL" in T.ts_last_error()
    d = 13
    desc = T._Desc(d, (C.c_int * d)(*([4] * d)), (C.c_double * d)(*([1.0] * d)), None, 0, 1)
    assert L.ts_plan_create(C.byref(desc), 0, None, C.byref(out)) == T.TS_ERR_INVALID_ARG
    assert out.value is None
    assert L.ts_apply_inverse(None, 1.0, None, None, 0, None) == T.TS_ERR_INVALID_ARG
    assert L.ts_plan_destroy(None) == T.TS_OK


def test_grid_nodes_on_host_match_the_oracle(built_lib):
    """ts_grid_nodes needs no GPU: its GLL nodes and lumped masses (Newton on the Legendre
    recurrence, barycentric derivative matrix) against the numpy oracle (Legendre roots,
    Legendre Vandermonde); invalid Q^k grids are rejected."""
    import ctypes as C
    import numpy as np
    from oracle import sem
    from paper_2605_20491_b300 import tschrod as T
    for n, L, k in ((99, 8.0, 20), (1099, 1.0, 2), (599, 8.0, 10), (31, 2.0, 32), (37, 3.5, 1), (37, 3.5, 0)):
        x, m = T.ts_grid_nodes(n, L, k)
        ax = sem.axis_1d(n, L, max(k, 1))
        assert np.max(np.abs(x - ax.x)) < 1e-14 * L
        assert np.max(np.abs(m / ax.m - 1)) < 1e-13
    with pytest.raises(T.TsError):
        T.ts_grid_nodes(100, 1.0, 3)
    f = (C.POINTER(C.c_double) * 1)((C.c_double * 100)())
    desc = T._Desc(1, (C.c_int * 1)(100), (C.c_double * 1)(1.0), f, 0, 3)
    out = C.c_void_p()
    assert T.lib().ts_plan_create(C.byref(desc), 0, None, C.byref(out)) == T.TS_ERR_INVALID_ARG
    assert "multiple of 3" in T.ts_last_error()


def test_plan_handle_is_freed_once(monkeypatch):
    """ts_plan_destroy clears the Python handle, so a later close() or garbage collection of
    the same Plan does not free the native plan a second time (a double free of the host
    object)."""
    import gc
    from paper_2605_20491_b300 import tschrod as T
    freed = []

    class FakeLib:
        def ts_plan_destroy(self, h):
            freed.append(h.value)
            return T.TS_OK

    monkeypatch.setattr(T, "lib", lambda: FakeLib())
    P = T.Plan(0x1234, (4, 4), (1.0, 1.0))
    T.ts_plan_destroy(P)
    P.close()
    T.ts_plan_destroy(P)
    del P
    gc.collect()
    Q = T.Plan(0x5678, (4,), (1.0,))
    del Q
    gc.collect()
    assert freed == [0x1234, 0x5678]


def test_tile_config_refuses_clusters_other_than_single_and_pairs(built_lib):
    """ts_tc_config_set accepts cluster 1 (single CTAs) and TS_TC_PAIR only: no tile of the
    contraction is shared through a multicast load.  The check is host-side (no GPU)."""
    from paper_2605_20491_b300 import tschrod as T
    L = T.lib()
    for cluster in (2, 4, 8, 0, -1, 3):
        assert L.ts_tc_config_set(0, 64, 64, 128, cluster) == T.TS_ERR_INVALID_ARG, cluster
        assert "cluster" in T.ts_last_error()
    for cluster in (1, T.TS_TC_PAIR):
        assert L.ts_tc_config_set(0, 64, 64, 128, cluster) == T.TS_OK
        assert L.ts_tc_config_set(0, 64, 0, 0, 0) == T.TS_OK  # forget it again


def test_unassigned_precisions_are_refused_on_host(built_lib):
    """Precision values 3 and 4 are not assigned: a plan mask with those bits is refused
    before any device work."""
    import ctypes as C
    from paper_2605_20491_b300 import tschrod as T
    L = T.lib()
    n = (C.c_int * 1)(8)
    Lx = (C.c_double * 1)(1.0)
    f0 = (C.c_double * 8)(*([0.0] * 8))
    f = (C.POINTER(C.c_double) * 1)(C.cast(f0, C.POINTER(C.c_double)))
    out = C.c_void_p()
    for bit in (3, 4):
        desc = T._Desc(1, n, Lx, f, 0, 1)
        assert L.ts_plan_create(C.byref(desc), 1 << bit, None, C.byref(out)) == T.TS_ERR_INVALID_ARG
        assert "not assigned" in T.ts_last_error() and out.value is None


def test_server_config_checked_before_device_work(built_lib):
    """max_inflight above TS_SERVER_MAX_INFLIGHT is refused before any CUDA call; on a
    host without a device a valid config fails in its first CUDA call instead, and both
    return no handle (the half-built server is released)."""
    import ctypes as C
    from paper_2605_20491_b300 import tschrod as T
    L = T.lib()
    out = C.c_void_p()
    cfg = T._ServerConfig(0, T.TS_SERVER_MAX_INFLIGHT + 1, 0, 0, 0)
    assert L.ts_server_create(C.byref(cfg), C.byref(out)) == T.TS_ERR_INVALID_ARG
    assert "max_inflight" in T.ts_last_error() and out.value is None
    import torch
    if not torch.cuda.is_available():
        cfg = T._ServerConfig(0, 4, 0, 0, 0)
        assert L.ts_server_create(C.byref(cfg), C.byref(out)) != T.TS_OK
        assert out.value is None
