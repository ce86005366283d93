"""CPU checks of the native boundary: the library builds for sm_103a, loads, and
exports every entry point that include/phs.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "phs.h")) as fh:
        txt = fh.read()
    return sorted(set(re.findall(r"^\s*(?:phs_status|void|int64_t|const char \*)\s*(phs_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def native():
    from paper_2608_11462_b300 import build
    build.build()
    from paper_2608_11462_b300 import _native
    return _native


def test_header_declares_entry_points():
    names = _declared()
    for must in ["phs_plan_create", "phs_matvec", "phs_fit", "phs_eval", "phs_plan_destroy", "phs_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(native):
    L = ctypes.CDLL(native.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(native.EXPORTS) == _declared()


def test_options_default_host_only(native):
    o = native.PhsOptions()
    native.lib().phs_options_default(ctypes.byref(o), 2)
    assert o.tol == 1e-8 and o.domain_halfwidth == 0.25 and abs(o.alpha - 0.35) < 1e-15 and o.nu == 1.0
    assert o.m2l_tensor == 1 and o.precond_lowrank == 0 and o.ordering == 3
    # the ctypes mirror is as large as the C struct: phs_options_default clears
    # sizeof(phs_options) bytes, so nothing past the mirror's size may change
    size = ctypes.sizeof(native.PhsOptions)
    buf = (ctypes.c_ubyte * (size + 64))(*([0xA5] * (size + 64)))
    native.lib().phs_options_default(ctypes.cast(buf, ctypes.POINTER(native.PhsOptions)), 2)
    assert bytes(buf[size:]) == bytes([0xA5] * 64)
    assert ctypes.cast(buf, ctypes.POINTER(native.PhsOptions)).contents.ordering == 3
    native.lib().phs_options_default(ctypes.byref(o), 4)
    assert o.domain_halfwidth == 1.0 and o.alpha == 0.5 and o.nu == 2.0
    native.lib().phs_options_default(ctypes.byref(o), 3)
    assert o.nu == 1.5
    assert native.lib().phs_last_error() is not None


def test_build_targets_sm103a_only():
    from paper_2608_11462_b300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _header_struct(name):
    """(type, field) pairs of a `typedef struct { ... } name;` in include/phs.h, comments
    stripped."""
    with open(os.path.join(ROOT, "include", "phs.h")) as fh:
        txt = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", txt).group(1)
    return re.findall(r"^\s*(int|double|float|uint64_t|int64_t)\s+(\w+)\s*;", body, re.M)


def test_ctypes_mirrors_follow_the_header(native):
    """PhsOptions, PhsFitInfo and PhsServerConfig list the header's fields in its order
    with matching C types, so a field added on one side only is caught on CPU."""
    ctype = {"int": ctypes.c_int, "double": ctypes.c_double, "float": ctypes.c_float,
             "uint64_t": ctypes.c_uint64, "int64_t": ctypes.c_int64}
    for cname, mirror in (("phs_options", native.PhsOptions), ("phs_fit_info", native.PhsFitInfo),
                          ("phs_server_config", native.PhsServerConfig)):
        want = [(f, ctype[t]) for t, f in _header_struct(cname)]
        assert want, cname
        assert [(f, t) for f, t in mirror._fields_] == want, cname
