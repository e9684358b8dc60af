"""CPU oracle for the exact 2D LMS line estimator (Shapira & Hassner).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; the product package never imports
it.  It shares no code with the CUDA path (see ``lms_oracle.c`` for the
definition it implements).

* ``lms_i16`` / ``lms_f32``  -- O1 brute force or O2 exact sweep (C, OpenMP).
* ``eval_slope_i16``         -- narrowest h-window at one given slope.
* ``tiny``                   -- O3 exhaustive subset search (pure Python).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lms_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblms_oracle.so")

OK, ERR_ARG, ERR_VERTICAL, ERR_UNSUPPORTED, ERR_NOMEM = 0, 1, 3, 7, 8


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (strict IEEE: no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Result(ctypes.Structure):
    _fields_ = [("w_num", ctypes.c_int64), ("w_den", ctypes.c_int64),
                ("s_num", ctypes.c_int64), ("s_den", ctypes.c_int64),
                ("t_num", ctypes.c_int64), ("t_den", ctypes.c_int64),
                ("theta1", ctypes.c_double), ("theta2", ctypes.c_double),
                ("med_sq", ctypes.c_double),
                ("i", ctypes.c_int32), ("j", ctypes.c_int32),
                ("status", ctypes.c_int32), ("scale_exp", ctypes.c_int32),
                ("ints_valid", ctypes.c_int32), ("pad", ctypes.c_int32)]


@dataclass(frozen=True)
class OracleResult:
    w_num: int
    w_den: int
    s_num: int
    s_den: int
    t_num: int
    t_den: int
    theta1: float
    theta2: float
    med_sq: float
    i: int
    j: int
    status: int
    scale_exp: int = 0

    def exact(self):
        """The bit-exact fields compared against the CUDA path."""
        return (self.status, self.w_num, self.w_den, self.s_num, self.s_den,
                self.t_num, self.t_den, self.i, self.j)


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        p16 = ctypes.POINTER(ctypes.c_int16)
        pf = ctypes.POINTER(ctypes.c_float)
        pres = ctypes.POINTER(_Result)
        for name, pt in (("oracle_lms_i16_brute", p16), ("oracle_lms_i16_sweep", p16),
                         ("oracle_lms_f32_brute", pf), ("oracle_lms_f32_sweep", pf)):
            f = getattr(L, name)
            f.argtypes = [pt, pt, ctypes.c_int64, ctypes.c_int64, pres]
            f.restype = ctypes.c_int
        L.oracle_eval_slope_i16.argtypes = [p16, p16, ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_int64, ctypes.c_int64, pres]
        L.oracle_eval_slope_i16.restype = ctypes.c_int
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _conv(r: _Result) -> OracleResult:
    return OracleResult(r.w_num, r.w_den, r.s_num, r.s_den, r.t_num, r.t_den,
                        r.theta1, r.theta2, r.med_sq, r.i, r.j, r.status, r.scale_exp)


def set_threads(t: int) -> None:
    lib().oracle_set_threads(int(t))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def lms_i16(x, y, h: int = 0, method: str = "brute") -> OracleResult:
    """Exact LMS of int16 points; method 'brute' (O1) or 'sweep' (O2)."""
    x = np.ascontiguousarray(x, dtype=np.int16)
    y = np.ascontiguousarray(y, dtype=np.int16)
    assert x.shape == y.shape and x.ndim == 1
    r = _Result()
    fn = {"brute": lib().oracle_lms_i16_brute, "sweep": lib().oracle_lms_i16_sweep}[method]
    p16 = ctypes.POINTER(ctypes.c_int16)
    fn(x.ctypes.data_as(p16), y.ctypes.data_as(p16), x.size, int(h), ctypes.byref(r))
    return _conv(r)


def lms_f32(x, y, h: int = 0, method: str = "brute") -> OracleResult:
    """Exact LMS of float32 points taken as real numbers (reported as doubles)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    assert x.shape == y.shape and x.ndim == 1
    r = _Result()
    fn = {"brute": lib().oracle_lms_f32_brute, "sweep": lib().oracle_lms_f32_sweep}[method]
    pf = ctypes.POINTER(ctypes.c_float)
    fn(x.ctypes.data_as(pf), y.ctypes.data_as(pf), x.size, int(h), ctypes.byref(r))
    return _conv(r)


def eval_slope_i16(x, y, s_num: int, s_den: int, h: int = 0) -> OracleResult:
    """Narrowest window of h projections at the slope s_num/s_den (s_den > 0)."""
    x = np.ascontiguousarray(x, dtype=np.int16)
    y = np.ascontiguousarray(y, dtype=np.int16)
    r = _Result()
    p16 = ctypes.POINTER(ctypes.c_int16)
    lib().oracle_eval_slope_i16(x.ctypes.data_as(p16), y.ctypes.data_as(p16), x.size,
                                int(h), int(s_num), int(s_den), ctypes.byref(r))
    return _conv(r)


def default_h(n: int) -> int:
    """The order statistic used throughout: floor(n/2) + 1 (upper median)."""
    return n // 2 + 1
