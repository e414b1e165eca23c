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


def header_constants():
    """name -> value of the enum constants of include/mw.h (integers and 1 << k)."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "mw.h")).read(), flags=re.S)
    out = {}
    for body in re.findall(r"enum\s*\{([^}]*)\}", src):
        for item in body.split(","):
            m = re.match(r"\s*(MW_[A-Z0-9_]+)\s*=\s*(.+?)\s*$", item)
            if m:
                expr = m.group(2)
                if re.fullmatch(r"[0-9<\s]+", expr):
                    out[m.group(1)] = eval(expr)  # integer literals and shifts only
    return out


def test_binding_constants_match_header():
    import paper_1110_6298_gb300.mw as mw
    c = header_constants()
    assert c["MW_FLAG_GRAPH"] == mw.FLAG_GRAPH
    assert c["MW_FLAG_REAL"] == mw.FLAG_REAL
    assert c["MW_FLAG_DELTA_TN"] == mw.FLAG_DELTA_TN == mw.DELTA["tn"]
    assert c["MW_FLAG_DELTA_RISBO"] == mw.FLAG_DELTA_RISBO == mw.DELTA["risbo"]
    assert c["MW_FLAG_AUTOTUNE"] == mw.FLAG_AUTOTUNE
    assert c["MW_PREC_FP64"] == mw.PRECISIONS["fp64"]
    assert c["MW_PREC_MIXED_BF16X3"] == mw.PRECISIONS["mixed"] == mw.PRECISIONS["mixed_bf16"]
    assert c["MW_PREC_MIXED_TF32X3"] == mw.PRECISIONS["mixed_tf32"]
    assert (c["MW_OK"], c["MW_EINVAL"], c["MW_EUNSUPPORTED"]) == (mw.MW_OK, mw.MW_EINVAL, mw.MW_EUNSUPPORTED)


def test_flag_rules_checked_before_device_work(libmw):
    c = header_constants()
    h = ctypes.c_void_p()
    tn, rb, real = c["MW_FLAG_DELTA_TN"], c["MW_FLAG_DELTA_RISBO"], c["MW_FLAG_REAL"]
    mixed, fp64 = c["MW_PREC_MIXED"], c["MW_PREC_FP64"]
    # both recursions at once
    assert libmw.mw_plan_create(ctypes.byref(h), 8, 0, 1, mixed | tn | rb) == c["MW_EINVAL"]
    # Trapani-Navaza is for the mixed precisions only
    assert libmw.mw_plan_create(ctypes.byref(h), 8, 0, 1, fp64 | tn) == c["MW_EUNSUPPORTED"]
    # real-signal plans are spin 0 and not ragged
    assert libmw.mw_plan_create(ctypes.byref(h), 8, 1, 2, mixed | real) == c["MW_EINVAL"]
    Ls = (ctypes.c_int * 2)(8, 4)
    ss = (ctypes.c_int * 2)(0, 0)
    assert libmw.mw_plan_create_ragged(ctypes.byref(h), 2, Ls, ss, mixed | real) == c["MW_EINVAL"]
    # an unknown flag bit
    assert libmw.mw_plan_create(ctypes.byref(h), 8, 0, 1, mixed | (1 << 13)) == c["MW_EINVAL"]
    assert not h.value


def test_ragged_layout_prefix_sums(libmw):
    """mw_layout_ragged: prefix sums of (L-1)(2L-1)+1 and L^2 in the caller's
    order (Sec. IV-C sample count, Sec. III-B coefficient count), the total in
    the last entry; bad band limits rejected; the per-plan queries answer -1 /
    0 for a NULL plan."""
    ll = ctypes.c_longlong
    libmw.mw_layout_ragged.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ll),
                                       ctypes.POINTER(ll)]
    Ls = [64, 512, 1, 2, 384, 2048, 128]
    n = len(Ls)
    la = (ctypes.c_int * n)(*Ls)
    mo, fo = (ll * (n + 1))(), (ll * (n + 1))()
    assert libmw.mw_layout_ragged(n, la, mo, fo) == 0
    em = ef = 0
    for b, L in enumerate(Ls):
        assert mo[b] == em and fo[b] == ef
        em += (L - 1) * (2 * L - 1) + 1
        ef += L * L
    assert mo[n] == em and fo[n] == ef
    assert libmw.mw_layout_ragged(n, la, None, fo) == 0
    bad = (ctypes.c_int * 2)(8, 2049)
    assert libmw.mw_layout_ragged(2, bad, mo, fo) == 1
    assert libmw.mw_layout_ragged(0, la, mo, fo) == 1
    for name in ("mw_plan_map_offset", "mw_plan_flm_offset"):
        getattr(libmw, name).restype = ll
        getattr(libmw, name).argtypes = [ctypes.c_void_p, ctypes.c_int]
        assert getattr(libmw, name)(None, 0) == -1
    libmw.mw_plan_band_limit.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert libmw.mw_plan_band_limit(None, 0) == -1
    assert libmw.mw_plan_batch(None) == 0
