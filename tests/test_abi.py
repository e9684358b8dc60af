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


def test_argument_errors_of_every_entry_point(L):
    """Each entry point refuses what include/lms.h documents as LMS_ERR_ARG
    (LMS_ERR_TOO_LARGE for the allocation-free fit) before it touches a
    device, so these run without a GPU.  A private handle of the library
    carries the prototypes set here, leaving the binding's untouched."""
    lib = ctypes.CDLL(L.library_path())
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.lms_fit_host.argtypes = [vp, vp, i64, i64, i32, vp, vp, vp]
    lib.lms_fit_host.restype = ctypes.c_int
    x = np.zeros(8, np.int16)
    res = np.zeros(1, dtype=L.RESULT_DTYPE)
    px, pr = x.ctypes.data, res.ctypes.data
    ARG = L.LMS_ERR_ARG
    for fn in (lib.lms_fit_host,):
        for args in ((None, px, 8, 0), (px, px, 1, 0), (px, px, 70000, 0), (px, px, 8, 9), (px, px, 8, -1)):
            assert fn(*args, 0, None, pr, None) == ARG
        assert fn(px, px, 8, 0, 0, None, None, None) == ARG
        assert fn(px, px, 8, 0, 5, None, pr, None) == ARG
    bnb = lib.lms_fit_bnb
    bnb.argtypes = [vp, vp, i64, i64, vp, vp, vp, vp, vp]
    bnb.restype = ctypes.c_int
    for args in ((None, px, 8, 0), (px, px, 1, 0), (px, px, 70000, 0), (px, px, 8, 9)):
        assert bnb(*args, None, None, pr, None, None) == ARG
    bad = L.options("bnb")
    bad.seed_mode = 2
    assert bnb(px, px, 8, 0, None, ctypes.addressof(bad), pr, None, None) == ARG
    na = lib.lms_fit_noalloc
    na.argtypes = [vp, vp, i64, i64, vp, vp]
    na.restype = ctypes.c_int
    assert na(None, px, 8, 0, pr, None) == ARG
    assert na(px, px, 1, 0, pr, None) == ARG
    assert na(px, px, 8, 9, pr, None) == ARG
    big = np.zeros(1025, np.int16)
    assert na(big.ctypes.data, big.ctypes.data, 1025, 0, pr, None) == L.LMS_ERR_TOO_LARGE
    # the learned fits check every argument before queueing the network's
    # forward pass; a stand-in handle is never dereferenced on these paths
    handle = ctypes.create_string_buffer(64)
    for name in ("lms_fit_learned", "lms_fit_learned_host"):
        f = getattr(lib, name)
        f.argtypes = [vp, vp, vp, i64, i64, vp, vp, vp, vp]
        f.restype = ctypes.c_int
        assert f(None, px, px, 8, 0, None, pr, None, None) == ARG
        h = ctypes.addressof(handle)
        for args in ((None, px, 8, 0), (px, px, 1, 0), (px, px, 70000, 0), (px, px, 8, 9), (px, px, 8, -2)):
            assert f(h, *args, None, pr, None, None) == ARG, (name, args[2:])
    plan = vp()
    cre = lib.lms_batch_plan_create_ex
    cre.argtypes = [vp, i64, vp, i32, i32, i32, ctypes.POINTER(vp)]
    cre.restype = ctypes.c_int
    off = np.array([0, 10, 11, 30], np.int64)        # a set of one point
    assert cre(None, 3, None, 0, 4, 0, ctypes.byref(plan)) == ARG
    assert cre(off.ctypes.data, 0, None, 0, 4, 0, ctypes.byref(plan)) == ARG
    assert cre(off.ctypes.data, 3, None, 0, 4, 0, ctypes.byref(plan)) == ARG
    off = np.array([0, 10, 40010], np.int64)         # a set above 32768 points
    assert cre(off.ctypes.data, 2, None, 0, 4, 0, ctypes.byref(plan)) == ARG
    assert not plan.value
    hr = lib.lms_hough_refine
    hr.argtypes = [vp, i64, i32, i32, i32, i32, i32, ctypes.c_float, i32, i32, i32, ctypes.c_uint64, vp, vp, vp, vp]
    hr.restype = ctypes.c_int
    img = np.zeros((16, 16), np.uint8)
    lines = np.zeros(64 * 64, np.uint8)
    pi, pl = img.ctypes.data, lines.ctypes.data
    good = dict(edges=pi, B=1, H=16, W=16, n_theta=90, n_rho=64, top_k=2, band=1.0, nt=2, nr=2, mp=0)
    for k, v in (("edges", None), ("B", 0), ("H", 1), ("W", 40000), ("n_theta", 0), ("n_rho", 1),
                 ("top_k", 65), ("band", float("nan")), ("band", -1.0), ("nt", -1), ("mp", -1)):
        a = dict(good, **{k: v})
        assert hr(a["edges"], a["B"], a["H"], a["W"], a["n_theta"], a["n_rho"], a["top_k"], a["band"], a["nt"],
                  a["nr"], a["mp"], 0, None, None, pl, None) == ARG, k
    assert hr(pi, 1, 16, 16, 90, 64, 2, 1.0, 2, 2, 0, 0, None, None, None, None) == ARG
    pk = lib.lms_measure_int_peak
    pk.argtypes = [i32, i64, vp, vp]
    pk.restype = ctypes.c_int
    v = ctypes.c_double()
    assert pk(2, 10, ctypes.addressof(v), None) == ARG
    assert pk(0, 0, ctypes.addressof(v), None) == ARG
    assert pk(0, 10, None, None) == ARG
    ws = lib.lms_workspace_size
    ws.argtypes = [i64, i32, vp]
    ws.restype = ctypes.c_size_t
    assert ws(1, 0, None) == 0 and ws(70000, 0, None) == 0 and ws(8, 5, None) == 0
