"""The C-ABI library builds, loads and exports every symbol that
include/lms.h declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1510_01041_gb300 import build, lms
    build.build()
    return lms


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(r"LMS_API\s+[\w\s\*]+?\b(lms_\w+)\s*\(", src)))


def test_header_declares_entry_points():
    names = _declared("lms.h")
    for must in ("lms_fit", "lms_fit_host", "lms_workspace_size", "lms_set_workspace",
                 "lms_reserve", "lms_status_str", "lms_version"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    lib = ctypes.CDLL(L.library_path())
    for header in sorted(os.listdir(os.path.join(ROOT, "include"))):
        for name in _declared(header):
            assert hasattr(lib, name), f"{name} declared in {header} but not exported"


def test_status_strings(L):
    assert L.status_str(0) == "ok"
    assert "slope" in L.status_str(3)
    assert L.version().startswith("lms-gb300")


def test_argument_errors_before_any_device_work(L):
    lib = L.lib()
    x = np.zeros(8, np.int16)
    res = np.zeros(1, dtype=L.RESULT_DTYPE)
    vp = ctypes.c_void_p
    cases = [
        (None, x.ctypes.data, 8, 0, 0),          # null pointer
        (x.ctypes.data, x.ctypes.data, 1, 0, 0),  # n < 2
        (x.ctypes.data, x.ctypes.data, 70000, 0, 0),  # n > 65536
        (x.ctypes.data, x.ctypes.data, 8, 9, 0),  # h > n
        (x.ctypes.data, x.ctypes.data, 8, -1, 0),  # h < 0
        (x.ctypes.data, x.ctypes.data, 8, 0, 5),  # bad dtype
    ]
    for xp, yp, n, h, dt in cases:
        rc = lib.lms_fit(vp(xp), vp(yp), n, h, dt, None, vp(res.ctypes.data), None)
        assert rc == L.LMS_ERR_ARG
    bad = L.options("plain")
    bad.algorithm = 5                             # beyond the last algorithm
    rc = lib.lms_fit(vp(x.ctypes.data), vp(x.ctypes.data), 8, 0, 0, ctypes.byref(bad),
                     vp(res.ctypes.data), None)
    assert rc == L.LMS_ERR_ARG
    bad = L.options("plain")
    bad.reserved[1] = 1
    rc = lib.lms_fit(vp(x.ctypes.data), vp(x.ctypes.data), 8, 0, 0, ctypes.byref(bad),
                     vp(res.ctypes.data), None)
    assert rc == L.LMS_ERR_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1510_01041_gb300 import build, lms
    monkeypatch.setattr(build, "LIB", str(tmp_path / "nope.so"))
    monkeypatch.setattr(lms, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        lms.lib()
