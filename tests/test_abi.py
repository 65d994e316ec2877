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
    desc = T._Desc(d, (C.c_int * d)(*([4] * d)), (C.c_double * d)(*([1.0] * d)), None, 0)
    assert L.ts_plan_create(C.byref(desc), 0, None, C.byref(out)) == T.TS_ERR_INVALID_ARG
    assert out.value is None
    assert L.ts_apply_inverse(None, 1.0, None, None, 0, None) == T.TS_ERR_INVALID_ARG
    assert L.ts_plan_destroy(None) == T.TS_OK
