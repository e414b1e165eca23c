"""Host-side checks of the C ABI: the library builds and loads, exports every
function include/mw.h declares, and the binding refuses to run without it."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mw_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libmw():
    from paper_1110_6298_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("mw_plan_create", "mw_forward", "mw_inverse", "mw_forward_adjoint", "mw_inverse_adjoint",
              "mw_plan_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libmw):
    missing = [n for n in declared_functions() if not hasattr(libmw, n)]
    assert not missing, missing


def test_host_only_calls(libmw):
    libmw.mw_map_size.restype = ctypes.c_size_t
    libmw.mw_flm_size.restype = ctypes.c_size_t
    libmw.mw_status_string.restype = ctypes.c_char_p
    assert libmw.mw_map_size(2048) == 8382466 and libmw.mw_map_size(1) == 1 and libmw.mw_map_size(0) == 0
    assert libmw.mw_flm_size(256) == 65536
    assert b"MW_EINVAL" in libmw.mw_status_string(1)
    assert libmw.mw_plan_destroy(None) == 0
    # invalid arguments are rejected before any device work
    h = ctypes.c_void_p()
    assert libmw.mw_plan_create(None, 8, 0, 1, 0) == 1
    assert libmw.mw_plan_create(ctypes.byref(h), 0, 0, 1, 0) == 1
    assert libmw.mw_plan_create(ctypes.byref(h), 8, 8, 1, 0) == 1
    assert libmw.mw_plan_create(ctypes.byref(h), 8, 0, 0, 0) == 1
    assert libmw.mw_plan_create(ctypes.byref(h), 8, 0, 1, 7) == 1
    assert libmw.mw_forward(None, None, None, None) == 1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_1110_6298_gb300.mw as mw
    monkeypatch.setattr(mw, "_lib", None)
    monkeypatch.setattr(mw, "LIB_PATH", str(tmp_path / "libmw.so"))
    with pytest.raises(RuntimeError):
        mw.lib()
