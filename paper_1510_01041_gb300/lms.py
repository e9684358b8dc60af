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
LMS_ERR_TOO_LARGE = 9
LMS_I16, LMS_F32 = 0, 1
ALGOS = {"auto": 0, "plain": 1, "sweep": 2, "bnb": 3, "paper": 4}

# lms_result: 6 x int64, 3 x double, 4 x int32 = 88 bytes
RESULT_DTYPE = np.dtype([("w_num", "<i8"), ("w_den", "<i8"), ("s_num", "<i8"), ("s_den", "<i8"),
                         ("t_num", "<i8"), ("t_den", "<i8"), ("theta1", "<f8"), ("theta2", "<f8"),
                         ("med_sq", "<f8"), ("i", "<i4"), ("j", "<i4"), ("status", "<i4"),
                         ("algorithm", "<i4")])
assert RESULT_DTYPE.itemsize == 88


class Options(ctypes.Structure):
    _fields_ = [("algorithm", ctypes.c_int32), ("sweepers", ctypes.c_int32),
                ("buckets", ctypes.c_int32), ("seed_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


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


SEED_MODES = {"quantiles": 0, "angles": 1}


def options(algorithm: str = "auto", sweepers: int = 0, buckets: int = 0, seed_mode: str = "quantiles") -> Options:
    o = Options()
    o.algorithm = ALGOS[algorithm]
    o.sweepers = int(sweepers)
    o.buckets = int(buckets)
    o.seed_mode = SEED_MODES[seed_mode]
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


def measure_int_peak(kind: int = 0, iters: int = 20000, stream=None) -> float:
    """lms_measure_int_peak: int32 instructions per second of this GPU
    (kind 0: add/xor, kind 1: multiply-add)."""
    L = lib()
    L.lms_measure_int_peak.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    L.lms_measure_int_peak.restype = ctypes.c_int
    v = ctypes.c_double(0.0)
    rc = L.lms_measure_int_peak(int(kind), int(iters), ctypes.byref(v), _stream_handle(stream))
    if rc != LMS_OK:
        raise LmsError(rc, "lms_measure_int_peak")
    return float(v.value)


# ------------------------------------------------------------------ branch and bound
class BnbStats(ctypes.Structure):
    _fields_ = [("events_total", ctypes.c_int64), ("events_swept", ctypes.c_int64),
                ("nodes_evaluated", ctypes.c_int64), ("nodes_pruned", ctypes.c_int64),
                ("buckets_total", ctypes.c_int32), ("buckets_swept", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("seeded", ctypes.c_int32),
                ("upper_bound", ctypes.c_double)]


def fit_bnb(x, y, h: int = 0, seed=None, out=None, stream=None, sweepers: int = 0, buckets: int = 0,
            seed_mode: str = "quantiles", stats: bool = True):
    """Exact LMS by branch-and-bound (lms_fit_bnb).  ``seed``: a CUDA float32
    tensor holding a predicted slope, or None.  Returns (out, stats dict); with
    stats=False the call does not wait for the fit and the dict is None."""
    import torch
    L = lib()
    if not getattr(L, "_bnb_ready", False):
        L.lms_fit_bnb.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_void_p, ctypes.POINTER(Options), ctypes.c_void_p,
                                  ctypes.POINTER(BnbStats), ctypes.c_void_p]
        L.lms_fit_bnb.restype = ctypes.c_int
        L._bnb_ready = True
    if x.dtype != torch.int16 or not x.is_cuda:
        raise TypeError("fit_bnb takes int16 CUDA tensors")
    x = x.contiguous()
    y = y.contiguous()
    if out is None:
        out = torch.empty(RESULT_DTYPE.itemsize, dtype=torch.uint8, device=x.device)
    st = BnbStats()
    sp = ctypes.c_void_p(seed.data_ptr()) if seed is not None else ctypes.c_void_p(0)
    opt = options("bnb", sweepers, buckets, seed_mode)
    rc = L.lms_fit_bnb(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.numel(), int(h), sp,
                       ctypes.byref(opt), ctypes.c_void_p(out.data_ptr()), ctypes.byref(st) if stats else None,
                       _stream_handle(stream))
    if rc != LMS_OK:
        raise LmsError(rc, "lms_fit_bnb")
    return out, ({f: getattr(st, f) for f, _ in BnbStats._fields_} if stats else None)


# ------------------------------------------------------------------ learned slope proposal
def _setnet_sigs():
    L = lib()
    if not getattr(L, "_setnet_ready", False):
        vp, i64, f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_float
        L.lms_setnet_create.argtypes = [ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p)]
        L.lms_setnet_create.restype = ctypes.c_int
        L.lms_setnet_destroy.argtypes = [vp]
        L.lms_setnet_destroy.restype = None
        L.lms_setnet_param_count.restype = ctypes.c_int64
        L.lms_setnet_params.argtypes = [vp, vp, i64, ctypes.c_int32]
        L.lms_setnet_params.restype = ctypes.c_int
        L.lms_setnet_forward.argtypes = [vp, vp, vp, vp, i64, vp, vp]
        L.lms_setnet_forward.restype = ctypes.c_int
        L.lms_setnet_backward.argtypes = [vp, vp, vp, vp, i64, vp, f32, vp, vp, vp]
        L.lms_setnet_backward.restype = ctypes.c_int
        L.lms_setnet_train_step.argtypes = [vp, vp, vp, vp, i64, vp, f32, f32, vp, vp]
        L.lms_setnet_train_step.restype = ctypes.c_int
        L.lms_setnet_save.argtypes = [vp, ctypes.c_char_p]
        L.lms_setnet_save.restype = ctypes.c_int
        L.lms_setnet_load.argtypes = [vp, ctypes.c_char_p]
        L.lms_setnet_load.restype = ctypes.c_int
        L.lms_fit_learned.argtypes = [vp, vp, vp, i64, i64, ctypes.POINTER(Options), vp,
                                      ctypes.POINTER(BnbStats), vp]
        L.lms_fit_learned.restype = ctypes.c_int
        L.lms_fit_learned_host.argtypes = [vp, vp, vp, i64, i64, ctypes.POINTER(Options), vp,
                                           ctypes.POINTER(BnbStats), vp]
        L.lms_fit_learned_host.restype = ctypes.c_int
        L._setnet_ready = True
    return L


class SetNet:
    """Handle of the device set network (lms_setnet_*)."""

    def __init__(self, seed: int = 1):
        self.L = _setnet_sigs()
        h = ctypes.c_void_p()
        rc = self.L.lms_setnet_create(ctypes.c_uint64(seed), ctypes.byref(h))
        if rc != LMS_OK:
            raise LmsError(rc, "lms_setnet_create")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            self.L.lms_setnet_destroy(self.h)
            self.h = None

    @property
    def nparam(self) -> int:
        return int(self.L.lms_setnet_param_count())

    def get_params(self):
        a = np.zeros(self.nparam, dtype=np.float32)
        rc = self.L.lms_setnet_params(self.h, ctypes.c_void_p(a.ctypes.data), a.size, 0)
        if rc != LMS_OK:
            raise LmsError(rc, "lms_setnet_params")
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        rc = self.L.lms_setnet_params(self.h, ctypes.c_void_p(a.ctypes.data), a.size, 1)
        if rc != LMS_OK:
            raise LmsError(rc, "lms_setnet_params")

    def forward(self, x, y, offsets, stream=None):
        """CUDA int16 x, y and int64 offsets[B+1] -> CUDA float32 [B, 4]
        (angle, normalised intercept, slope, intercept)."""
        import torch
        B = offsets.numel() - 1
        pred = torch.empty((B, 4), dtype=torch.float32, device=x.device)
        rc = self.L.lms_setnet_forward(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       ctypes.c_void_p(offsets.data_ptr()), B, ctypes.c_void_p(pred.data_ptr()),
                                       _stream_handle(stream))
        if rc != LMS_OK:
            raise LmsError(rc, "lms_setnet_forward")
        return pred

    def backward(self, x, y, offsets, targets, lam: float, stream=None):
        import torch
        B = offsets.numel() - 1
        g = torch.empty(self.nparam, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        rc = self.L.lms_setnet_backward(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                        ctypes.c_void_p(offsets.data_ptr()), B,
                                        ctypes.c_void_p(targets.data_ptr()), float(lam),
                                        ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                        _stream_handle(stream))
        if rc != LMS_OK:
            raise LmsError(rc, "lms_setnet_backward")
        return loss, g

    def train_step(self, x, y, offsets, targets, lam: float, lr: float, loss=None, stream=None):
        import torch
        B = offsets.numel() - 1
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=x.device)
        rc = self.L.lms_setnet_train_step(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                          ctypes.c_void_p(offsets.data_ptr()), B,
                                          ctypes.c_void_p(targets.data_ptr()), float(lam), float(lr),
                                          ctypes.c_void_p(loss.data_ptr()), _stream_handle(stream))
        if rc != LMS_OK:
            raise LmsError(rc, "lms_setnet_train_step")
        return loss

    def save(self, path: str):
        rc = self.L.lms_setnet_save(self.h, path.encode())
        if rc != LMS_OK:
            raise LmsError(rc, "lms_setnet_save")

    def load(self, path: str):
        rc = self.L.lms_setnet_load(self.h, path.encode())
        if rc != LMS_OK:
            raise LmsError(rc, "lms_setnet_load")
        return self

    def fit(self, x, y, h: int = 0, out=None, stream=None, stats: bool = True):
        """lms_fit_learned: predict the slope, then exact branch-and-bound.
        Returns (out, stats dict); with stats=False the call does not wait for
        the fit and the dict is None."""
        import torch
        if out is None:
            out = torch.empty(RESULT_DTYPE.itemsize, dtype=torch.uint8, device=x.device)
        st = BnbStats()
        opt = options("bnb")
        rc = self.L.lms_fit_learned(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                    x.numel(), int(h), ctypes.byref(opt), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.byref(st) if stats else None, _stream_handle(stream))
        if rc != LMS_OK:
            raise LmsError(rc, "lms_fit_learned")
        return out, ({f: getattr(st, f) for f, _ in BnbStats._fields_} if stats else None)

    def fit_host(self, x, y, h: int = 0, out=None, stream=None, stats: bool = True):
        """lms_fit_learned_host on host int16 arrays (numpy or CPU tensors;
        pinned tensors copy asynchronously).  ``out``: optional host uint8
        buffer of 88 bytes that receives the lms_result.  Returns (out, stats)
        (stats None with stats=False)."""
        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        n = x.numel() if hasattr(x, "numel") else x.size
        if out is None:
            out = np.zeros(RESULT_DTYPE.itemsize, dtype=np.uint8)
        st = BnbStats()
        opt = options("bnb")
        rc = self.L.lms_fit_learned_host(self.h, ctypes.c_void_p(ptr(x)), ctypes.c_void_p(ptr(y)), int(n), int(h),
                                         ctypes.byref(opt), ctypes.c_void_p(ptr(out)),
                                         ctypes.byref(st) if stats else None, _stream_handle(stream))
        if rc != LMS_OK:
            raise LmsError(rc, "lms_fit_learned_host")
        return out, ({f: getattr(st, f) for f, _ in BnbStats._fields_} if stats else None)


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "setnet.bin")


def pretrained(path: str = WEIGHTS, seed: int = 1) -> SetNet:
    """The set network with the weights trained by train_setnet.py."""
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path}: run python -m paper_1510_01041_gb300.train_setnet")
    return SetNet(seed).load(path)


# ------------------------------------------------------------------ batched fits
class BatchPlan:
    """lms_batch_plan for a fixed list of set sizes (CSR offsets)."""

    def __init__(self, offsets, h=None, plain_max_n: int = 0, streams: int = 0, bnb_min_n: int = 0):
        L = lib()
        if not getattr(L, "_batch_ready", False):
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            L.lms_batch_plan_create.argtypes = [vp, i64, vp, i32, i32, ctypes.POINTER(ctypes.c_void_p)]
            L.lms_batch_plan_create.restype = ctypes.c_int
            L.lms_batch_plan_create_ex.argtypes = [vp, i64, vp, i32, i32, i32, ctypes.POINTER(ctypes.c_void_p)]
            L.lms_batch_plan_create_ex.restype = ctypes.c_int
            L.lms_batch_plan_destroy.argtypes = [vp]
            L.lms_batch_plan_destroy.restype = ctypes.c_int
            L.lms_batch_plan_bytes.argtypes = [vp]
            L.lms_batch_plan_bytes.restype = ctypes.c_size_t
            L.lms_fit_batched.argtypes = [vp, vp, vp, vp, vp, vp]
            L.lms_fit_batched.restype = ctypes.c_int
            L._batch_ready = True
        self.L = L
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.B = self.offsets.size - 1
        hh = None if h is None else np.ascontiguousarray(h, dtype=np.int32)
        handle = ctypes.c_void_p()
        rc = L.lms_batch_plan_create_ex(ctypes.c_void_p(self.offsets.ctypes.data), self.B,
                                        ctypes.c_void_p(hh.ctypes.data) if hh is not None else None,
                                        int(plain_max_n), int(streams), int(bnb_min_n), ctypes.byref(handle))
        if rc != LMS_OK:
            raise LmsError(rc, "lms_batch_plan_create")
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None):
            self.L.lms_batch_plan_destroy(self.h)
            self.h = None

    @property
    def nbytes(self) -> int:
        return int(self.L.lms_batch_plan_bytes(self.h))

    def fit(self, x, y, offsets_dev, out=None, stream=None):
        """Enqueue the batch; returns a uint8 CUDA tensor of B lms_result records."""
        import torch
        if out is None:
            out = torch.empty((self.B, RESULT_DTYPE.itemsize), dtype=torch.uint8, device=x.device)
        rc = self.L.lms_fit_batched(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                    ctypes.c_void_p(offsets_dev.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    _stream_handle(stream))
        if rc != LMS_OK:
            raise LmsError(rc, "lms_fit_batched")
        return out


# ------------------------------------------------------------------ Hough + LMS
class _LmsResultC(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in ("w_num", "w_den", "s_num", "s_den", "t_num", "t_den")] + \
               [(name, ctypes.c_double) for name in ("theta1", "theta2", "med_sq")] + \
               [(name, ctypes.c_int32) for name in ("i", "j", "status", "algorithm")]


class LmsLine(ctypes.Structure):
    _fields_ = [("theta_index", ctypes.c_int32), ("rho_index", ctypes.c_int32), ("votes", ctypes.c_int32),
                ("transposed", ctypes.c_int32), ("npoints", ctypes.c_int32), ("nfit", ctypes.c_int32),
                ("pad", ctypes.c_int32 * 2), ("fit", _LmsResultC), ("ols_theta1", ctypes.c_double),
                ("ols_theta2", ctypes.c_double)]


def hough_refine(edges, n_theta=1024, n_rho=2896, top_k=32, band_px=4.0, nms_theta=5, nms_rho=5,
                 cos_sin=None, acc_out=None, stream=None, max_points=0, sample_seed=0):
    """lms_hough_refine on a CUDA uint8 tensor [B, H, W]; returns a list of
    B * top_k dicts (peak, band size, points fitted, transposed flag, exact
    LMS fit, least-squares line of the same points)."""
    L = lib()
    if not getattr(L, "_hough_ready", False):
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.lms_hough_refine.argtypes = [vp, i64, i32, i32, i32, i32, i32, ctypes.c_float, i32, i32, i32,
                                       ctypes.c_uint64, vp, vp, vp, vp]
        L.lms_hough_refine.restype = ctypes.c_int
        L._hough_ready = True
    B, H, W = edges.shape
    edges = edges.contiguous()
    out = (LmsLine * (B * top_k))()
    rc = L.lms_hough_refine(ctypes.c_void_p(edges.data_ptr()), B, H, W, n_theta, n_rho, top_k, float(band_px),
                            nms_theta, nms_rho, int(max_points), int(sample_seed) & 0xFFFFFFFFFFFFFFFF,
                            ctypes.c_void_p(cos_sin.data_ptr()) if cos_sin is not None else None,
                            ctypes.c_void_p(acc_out.data_ptr()) if acc_out is not None else None,
                            ctypes.byref(out), _stream_handle(stream))
    if rc != LMS_OK:
        raise LmsError(rc, "lms_hough_refine")
    res = []
    for ln in out:
        d = {f: getattr(ln, f) for f in ("theta_index", "rho_index", "votes", "transposed", "npoints", "nfit",
                                         "ols_theta1", "ols_theta2")}
        d["fit"] = {f: getattr(ln.fit, f) for f, _ in _LmsResultC._fields_}
        res.append(d)
    return res
