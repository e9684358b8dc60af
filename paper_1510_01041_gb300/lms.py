"""Thin Python binding of the C ABI in ``include/lms.h`` (ctypes).

Argument marshalling only: every step of a fit runs in the CUDA kernels of
``_build/liblms.so``.  PyTorch supplies device memory and streams.  There is
no CPU fallback: if the library is missing or a GPU is absent, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LMS_OK, LMS_ERR_ARG, LMS_ERR_RANGE, LMS_ERR_VERTICAL = 0, 1, 2, 3
LMS_ERR_TIMEOUT, LMS_ERR_CUDA, LMS_ERR_WORKSPACE, LMS_ERR_UNSUPPORTED, LMS_ERR_INTERNAL = 4, 5, 6, 7, 8
LMS_I16, LMS_F32 = 0, 1
ALGOS = {"auto": 0, "plain": 1, "sweep": 2, "bnb": 3}

# lms_result: 6 x int64, 3 x double, 4 x int32 = 88 bytes
RESULT_DTYPE = np.dtype([("w_num", "<i8"), ("w_den", "<i8"), ("s_num", "<i8"), ("s_den", "<i8"),
                         ("t_num", "<i8"), ("t_den", "<i8"), ("theta1", "<f8"), ("theta2", "<f8"),
                         ("med_sq", "<f8"), ("i", "<i4"), ("j", "<i4"), ("status", "<i4"),
                         ("algorithm", "<i4")])
assert RESULT_DTYPE.itemsize == 88


class Options(ctypes.Structure):
    _fields_ = [("algorithm", ctypes.c_int32), ("sweepers", ctypes.c_int32),
                ("buckets", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class LmsError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        super().__init__(f"{what}: {status_str(code)} ({code})" if what else f"{status_str(code)} ({code})")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load liblms.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(path)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        popt = ctypes.POINTER(Options)
        for name in ("lms_fit", "lms_fit_host"):
            f = getattr(L, name)
            f.argtypes = [vp, vp, i64, i64, i32, popt, vp, vp]
            f.restype = ctypes.c_int
        L.lms_workspace_size.argtypes = [i64, i32, popt]
        L.lms_workspace_size.restype = ctypes.c_size_t
        L.lms_set_workspace.argtypes = [vp, ctypes.c_size_t]
        L.lms_set_workspace.restype = ctypes.c_int
        L.lms_reserve.argtypes = [i64, i32, popt]
        L.lms_reserve.restype = ctypes.c_int
        L.lms_status_str.argtypes = [ctypes.c_int]
        L.lms_status_str.restype = ctypes.c_char_p
        L.lms_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def status_str(code: int) -> str:
    return lib().lms_status_str(int(code)).decode()


def version() -> str:
    return lib().lms_version().decode()


def options(algorithm: str = "auto", sweepers: int = 0, buckets: int = 0) -> Options:
    o = Options()
    o.algorithm = ALGOS[algorithm]
    o.sweepers = int(sweepers)
    o.buckets = int(buckets)
    return o


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.int16:
        return LMS_I16
    if t.dtype == torch.float32:
        return LMS_F32
    raise TypeError(f"coordinates must be int16 or float32, got {t.dtype}")


def fit(x, y, h: int = 0, algorithm: str = "auto", sweepers: int = 0, buckets: int = 0,
        out=None, stream=None):
    """Enqueue lms_fit on CUDA tensors x, y (int16 or float32, 1-D, same length).

    Returns ``out`` (a uint8 CUDA tensor of 88 bytes holding one lms_result);
    decode it with :func:`decode` after synchronising.
    """
    import torch
    if not (x.is_cuda and y.is_cuda):
        raise ValueError("fit() takes CUDA tensors; use fit_host() for host arrays")
    if x.shape != y.shape or x.dim() != 1 or x.dtype != y.dtype:
        raise ValueError("x and y must be 1-D tensors of one dtype and length")
    x = x.contiguous()
    y = y.contiguous()
    if out is None:
        out = torch.empty(RESULT_DTYPE.itemsize, dtype=torch.uint8, device=x.device)
    opt = options(algorithm, sweepers, buckets)
    rc = lib().lms_fit(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.numel(), int(h),
                       _dtype_code(x), ctypes.byref(opt), ctypes.c_void_p(out.data_ptr()),
                       _stream_handle(stream))
    if rc != LMS_OK:
        raise LmsError(rc, "lms_fit")
    return out


def fit_host(x, y, h: int = 0, algorithm: str = "auto", sweepers: int = 0, buckets: int = 0,
             stream=None) -> dict:
    """lms_fit_host on numpy arrays: host copies in, fit, result copied back."""
    x = np.ascontiguousarray(x)
    y = np.ascontiguousarray(y)
    if x.dtype == np.int16:
        code = LMS_I16
    elif x.dtype == np.float32:
        code = LMS_F32
    else:
        raise TypeError("coordinates must be int16 or float32")
    if x.shape != y.shape or x.ndim != 1 or y.dtype != x.dtype:
        raise ValueError("x and y must be 1-D arrays of one dtype and length")
    res = np.zeros(1, dtype=RESULT_DTYPE)
    opt = options(algorithm, sweepers, buckets)
    rc = lib().lms_fit_host(ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(y.ctypes.data), x.size, int(h),
                            code, ctypes.byref(opt), ctypes.c_void_p(res.ctypes.data),
                            _stream_handle(stream))
    if rc != LMS_OK:
        raise LmsError(rc, "lms_fit_host")
    return _row(res[0])


def _row(r) -> dict:
    return {k: (float(r[k]) if RESULT_DTYPE[k].kind == "f" else int(r[k])) for k in RESULT_DTYPE.names}


def decode(buf) -> list:
    """Decode lms_result records from a uint8 tensor/array (host or device)."""
    try:
        import torch
        if isinstance(buf, torch.Tensor):
            buf = buf.detach().cpu().numpy()
    except ImportError:
        pass
    arr = np.frombuffer(np.ascontiguousarray(buf).tobytes(), dtype=RESULT_DTYPE)
    return [_row(r) for r in arr]


def workspace_size(n: int, dtype: int = LMS_I16, algorithm: str = "auto") -> int:
    opt = options(algorithm)
    return int(lib().lms_workspace_size(int(n), int(dtype), ctypes.byref(opt)))


def reserve(n: int, dtype: int = LMS_I16, algorithm: str = "auto") -> None:
    opt = options(algorithm)
    rc = lib().lms_reserve(int(n), int(dtype), ctypes.byref(opt))
    if rc != LMS_OK:
        raise LmsError(rc, "lms_reserve")


def exact_fields(r: dict):
    """The fields compared bit for bit against the oracle."""
    return (r["status"], r["w_num"], r["w_den"], r["s_num"], r["s_den"], r["t_num"], r["t_den"],
            r["i"], r["j"])


# ------------------------------------------------------------------ profiling
def _prof_sigs():
    L = lib()
    if not getattr(L, "_prof_ready", False):
        L.lms_profile_enable.argtypes = [ctypes.c_int]
        L.lms_profile_enable.restype = None
        L.lms_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.lms_profile_read.restype = ctypes.c_int
        L.lms_stage_name.argtypes = [ctypes.c_int]
        L.lms_stage_name.restype = ctypes.c_char_p
        L.lms_launch_count.restype = ctypes.c_int64
        L._prof_ready = True
    return L


def profile_enable(on: bool = True) -> None:
    _prof_sigs().lms_profile_enable(1 if on else 0)


def profile_read() -> dict:
    """{stage name: (milliseconds, launches)} accumulated since the last read."""
    L = _prof_sigs()
    ms = np.zeros(64, dtype=np.float64)
    cnt = np.zeros(64, dtype=np.int64)
    ns = L.lms_profile_read(ctypes.c_void_p(ms.ctypes.data), ctypes.c_void_p(cnt.ctypes.data), 64)
    return {L.lms_stage_name(s).decode(): (float(ms[s]), int(cnt[s])) for s in range(ns) if cnt[s]}


def launch_count() -> int:
    return int(_prof_sigs().lms_launch_count())
