"""ctypes binding of libnomad (include/nomad.h): argument marshalling only.

Every function of the C ABI is exposed under the same name; ``Nomad`` is a
small convenience wrapper that owns a handle and accepts torch tensors (on
the handle's GPU or on the host) or numpy arrays.  All computation happens
in the CUDA kernels of the library; if the library cannot be loaded, every
call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libnomad.so")

NOMAD_OK = 0
NOMAD_ERR_INVALID_ARG = -1
NOMAD_ERR_OOM = -2
NOMAD_ERR_DUP_ENTRY = -3
NOMAD_ERR_TIMEOUT = -4
NOMAD_ERR_OWNERSHIP = -5
NOMAD_ERR_CUDA = -6
NOMAD_ERR_RANGE = -7
NOMAD_ERR_UNSUPPORTED = -8
NOMAD_ERR_STATE = -9

NOMAD_MODE_EPOCH = 0
NOMAD_MODE_UNIFORM = 1
NOMAD_FP32 = 0
NOMAD_BF16 = 1
NOMAD_FP8 = 2
NOMAD_PARTITION_RATINGS = 0
NOMAD_PARTITION_USERS = 1
NOMAD_VARIANT_BATCHED = 0
NOMAD_VARIANT_SIMPLE = 1
NOMAD_CIRCULATION_FLAT = 0
NOMAD_CIRCULATION_BLOCK = 1
NOMAD_ROUTING_UNIFORM = 0
NOMAD_ROUTING_SHORTER = 1
NOMAD_COO = 0
NOMAD_CSC = 1


class nomad_schedule(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("mode", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("partition", ctypes.c_int32), ("n_workers", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("debug", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("spin_timeout_ns", ctypes.c_int64),
                ("device", ctypes.c_int32), ("debug_drop_item", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("routing", ctypes.c_int32),
                ("circulation", ctypes.c_int32), ("batch_tokens", ctypes.c_int32),
                ("epochs_per_launch", ctypes.c_int32), ("reserved32", ctypes.c_int32),
                ("reserved", ctypes.c_int64 * 3)]


class nomad_info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int32),
                ("p", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("n_segments", ctypes.c_int64), ("epochs_done", ctypes.c_int64),
                ("pitch", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("blocks", ctypes.c_int32), ("sm_count", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("predrawn_ratings", ctypes.c_int64), ("reserved", ctypes.c_int64 * 2)]


# name -> (restype, argtypes); mirrors include/nomad.h
_P = ctypes.c_void_p
_I32, _I64 = ctypes.c_int32, ctypes.c_int64
SIGNATURES = {
    "nomad_schedule_default": (None, [ctypes.POINTER(nomad_schedule)]),
    "nomad_create": (_I32, [_I64, _I64, _I32, ctypes.c_float,
                            ctypes.POINTER(nomad_schedule), ctypes.POINTER(_P)]),
    "nomad_load_ratings": (_I32, [_P, _I32, _I64, _P, _P, _P, _I32, _P]),
    "nomad_epoch": (_I32, [_P, _I32, _P]),
    "nomad_epoch_many": (_I32, [ctypes.POINTER(_P), _I32, _I32, _P]),
    "nomad_last_epoch_span_ns": (_I32, [_P, ctypes.POINTER(ctypes.c_int64), _P]),
    "nomad_check": (_I32, [_P, _P]),
    "nomad_rmse": (_I32, [_P, _I64, _P, _P, _P, _I32,
                          ctypes.POINTER(ctypes.c_double), _P]),
    "nomad_objective": (_I32, [_P, ctypes.POINTER(ctypes.c_double), _P]),
    "nomad_get_factors": (_I32, [_P, _P, _P, _I32, _P]),
    "nomad_set_factors": (_I32, [_P, _P, _P, _I32, _I64, _P]),
    "nomad_get_info": (_I32, [_P, ctypes.POINTER(nomad_info)]),
    "nomad_last_epoch_kernel_ms": (_I32, [_P, ctypes.POINTER(ctypes.c_float)]),
    "nomad_get_layout": (_I32, [_P, _P, _P, _P, _P, _P, _P]),
    "nomad_get_replay_log": (_I32, [_P, _I64, _P, _P, ctypes.POINTER(_I64)]),
    "nomad_get_debug_counts": (_I32, [_P, _P, ctypes.POINTER(_I64)]),
    "nomad_rmse_noalloc": (_I32, [_P, _P, _I64, _I64, _I32, _I64, _I64, _P, _P, _P, _P,
                                  _P]),
    "nomad_destroy": (None, [_P]),
    "nomad_error_string": (ctypes.c_char_p, [_I32]),
    "nomad_last_error_message": (ctypes.c_char_p, [_P]),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libnomad.so (build it with ``paper_1312_0193_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(
                "libnomad.so is not built (%s); run __graft_entry__.build() or "
                "python paper_1312_0193_gb300/build.py" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class NomadError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        lib = load_library()
        text = lib.nomad_error_string(code).decode()
        super().__init__("%s (%d)%s" % (text, code, (": " + msg) if msg else ""))


def _check(code, handle=None):
    if code != NOMAD_OK:
        msg = ""
        if handle is not None:
            msg = load_library().nomad_last_error_message(handle).decode()
        raise NomadError(code, msg)


# ---------------------------------------------------------------- C-named API
def nomad_schedule_default() -> nomad_schedule:
    s = nomad_schedule()
    load_library().nomad_schedule_default(ctypes.byref(s))
    return s


def nomad_create(m, n, k, lam, sched: nomad_schedule):
    h = _P()
    _check(load_library().nomad_create(m, n, k, lam, ctypes.byref(sched),
                                       ctypes.byref(h)))
    return h


def nomad_load_ratings(h, fmt, nnz, major, minor, vals, device_ptrs, stream):
    _check(load_library().nomad_load_ratings(h, fmt, nnz, major, minor, vals,
                                             device_ptrs, stream), h)


def nomad_epoch(h, n_epochs, stream):
    _check(load_library().nomad_epoch(h, n_epochs, stream), h)


def nomad_epoch_many(handles, n_epochs, stream):
    arr = (_P * len(handles))(*handles)
    _check(load_library().nomad_epoch_many(arr, len(handles), n_epochs, stream),
           handles[0] if handles else None)


def nomad_check(h, stream):
    _check(load_library().nomad_check(h, stream), h)


def nomad_rmse(h, nnz, rows, cols, vals, device_ptrs, stream) -> float:
    out = ctypes.c_double()
    _check(load_library().nomad_rmse(h, nnz, rows, cols, vals, device_ptrs,
                                     ctypes.byref(out), stream), h)
    return out.value


def nomad_objective(h, stream) -> float:
    out = ctypes.c_double()
    _check(load_library().nomad_objective(h, ctypes.byref(out), stream), h)
    return out.value


def nomad_get_factors(h, W, H, device_ptrs, stream):
    _check(load_library().nomad_get_factors(h, W, H, device_ptrs, stream), h)


def nomad_set_factors(h, W, H, device_ptrs, epochs_done, stream):
    _check(load_library().nomad_set_factors(h, W, H, device_ptrs, epochs_done,
                                            stream), h)


def nomad_get_info(h) -> nomad_info:
    info = nomad_info()
    _check(load_library().nomad_get_info(h, ctypes.byref(info)), h)
    return info


def nomad_destroy(h):
    load_library().nomad_destroy(h)


# ---------------------------------------------------------------- marshalling
def _stream_ptr(stream):
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return _P(torch.cuda.current_stream().cuda_stream)
        return _P(0)
    if isinstance(stream, int):
        return _P(stream)
    return _P(stream.cuda_stream)


def _arg(x, dtype):
    """(pointer, on_device, keepalive) for a torch tensor or numpy array."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            want = {np.int32: torch.int32, np.int64: torch.int64,
                    np.float32: torch.float32}[dtype]
            if x.dtype != want:
                raise TypeError("expected %s, got %s" % (want, x.dtype))
            x = x.contiguous()
            return _P(x.data_ptr()), 1 if x.is_cuda else 0, x
    except ImportError:
        pass
    a = np.ascontiguousarray(x, dtype=dtype)
    return _P(a.ctypes.data), 0, a


class Nomad:
    """One NOMAD problem on one GPU (wraps a nomad_t handle)."""

    def __init__(self, m, n, k, lam, alpha=0.012, beta=0.05, mode="epoch",
                 precision="fp32", partition="ratings", n_workers=0,
                 warps_per_block=0, debug=False, seed=1, spin_timeout_ns=0,
                 device=0, debug_drop_item=-1, variant="batched", routing="uniform",
                 circulation="flat", batch_tokens=0, epochs_per_launch=0):
        s = nomad_schedule_default()
        s.alpha, s.beta = alpha, beta
        s.mode = {"epoch": NOMAD_MODE_EPOCH, "uniform": NOMAD_MODE_UNIFORM}[mode]
        s.precision = {"fp32": NOMAD_FP32, "bf16": NOMAD_BF16, "fp8": NOMAD_FP8}[precision]
        s.partition = {"ratings": NOMAD_PARTITION_RATINGS,
                       "users": NOMAD_PARTITION_USERS}[partition]
        s.n_workers = n_workers
        s.warps_per_block = warps_per_block
        s.debug = 1 if debug else 0
        s.seed = seed
        s.spin_timeout_ns = spin_timeout_ns
        s.device = device
        s.debug_drop_item = debug_drop_item
        s.variant = {"batched": NOMAD_VARIANT_BATCHED, "simple": NOMAD_VARIANT_SIMPLE}[variant]
        s.routing = {"uniform": NOMAD_ROUTING_UNIFORM, "shorter": NOMAD_ROUTING_SHORTER}[routing]
        s.circulation = {"flat": NOMAD_CIRCULATION_FLAT,
                         "block": NOMAD_CIRCULATION_BLOCK}[circulation]
        s.batch_tokens = batch_tokens
        s.epochs_per_launch = epochs_per_launch
        self.schedule = s
        self.m, self.n, self.k, self.lam = m, n, k, lam
        self.h = nomad_create(m, n, k, lam, s)

    # lifetime
    def close(self):
        if self.h is not None:
            nomad_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # the path
    def load_coo(self, rows, cols, vals, stream=None):
        r, dr, kr = _arg(rows, np.int32)
        c, dc, kc = _arg(cols, np.int32)
        v, dv, kv = _arg(vals, np.float32)
        if not (dr == dc == dv):
            raise ValueError("rows, cols and vals must all be on the GPU or all on the host")
        nnz = len(kr)
        nomad_load_ratings(self.h, NOMAD_COO, nnz, r, c, v, dr, _stream_ptr(stream))

    def load_csc(self, colptr, rows, vals, stream=None):
        cp, dp, kp = _arg(colptr, np.int64)
        r, dr, kr = _arg(rows, np.int32)
        v, dv, kv = _arg(vals, np.float32)
        if not (dp == dr == dv):
            raise ValueError("colptr, rows and vals must all be on the GPU or all on the host")
        nomad_load_ratings(self.h, NOMAD_CSC, len(kr), cp, r, v, dr, _stream_ptr(stream))

    def epoch(self, n_epochs=1, stream=None):
        nomad_epoch(self.h, n_epochs, _stream_ptr(stream))

    @staticmethod
    def epoch_many(nomads, n_epochs=1, stream=None):
        """n_epochs epochs of several independent problems, one launch per
        epoch (nomad_epoch_many): each handle runs on its own blocks."""
        nomad_epoch_many([nm.h for nm in nomads], n_epochs, _stream_ptr(stream))

    def check(self, stream=None):
        nomad_check(self.h, _stream_ptr(stream))

    def rmse(self, rows, cols, vals, stream=None) -> float:
        r, dr, kr = _arg(rows, np.int32)
        c, dc, kc = _arg(cols, np.int32)
        v, dv, kv = _arg(vals, np.float32)
        if not (dr == dc == dv):
            raise ValueError("rows, cols and vals must all be on the GPU or all on the host")
        return nomad_rmse(self.h, len(kr), r, c, v, dr, _stream_ptr(stream))

    def objective(self, stream=None) -> float:
        return nomad_objective(self.h, _stream_ptr(stream))

    def factors(self, stream=None):
        """(W, H) as float32 numpy arrays of shape (m, k) and (n, k)."""
        W = np.zeros((self.m, self.k), dtype=np.float32)
        H = np.zeros((self.n, self.k), dtype=np.float32)
        nomad_get_factors(self.h, _P(W.ctypes.data), _P(H.ctypes.data), 0,
                          _stream_ptr(stream))
        return W, H

    def factors_into(self, W, H, stream=None):
        """Copy the factors into device tensors W (m, k) and H (n, k)."""
        w, dw, kw = _arg(W, np.float32)
        h, dh, kh = _arg(H, np.float32)
        nomad_get_factors(self.h, w, h, dw, _stream_ptr(stream))

    def set_factors(self, W, H, epochs_done=0, stream=None):
        w, dw, kw = _arg(W, np.float32)
        h, dh, kh = _arg(H, np.float32)
        if dw != dh:
            raise ValueError("W and H must both be on the GPU or both on the host")
        nomad_set_factors(self.h, w, h, dw, epochs_done, _stream_ptr(stream))

    def last_epoch_span_ns(self, stream=None) -> int:
        """Device time of this handle's workers in the last batched epoch
        call (first start to last end), in nanoseconds."""
        ns = ctypes.c_int64(0)
        _check(load_library().nomad_last_epoch_span_ns(self.h, ctypes.byref(ns),
                                                       _stream_ptr(stream)), self.h)
        return int(ns.value)

    def last_epoch_kernel_ms(self) -> float:
        """Device time of the last persistent kernel (CUDA events)."""
        ms = ctypes.c_float()
        _check(load_library().nomad_last_epoch_kernel_ms(self.h, ctypes.byref(ms)), self.h)
        return ms.value

    def info(self) -> dict:
        i = nomad_get_info(self.h)
        return {name: getattr(i, name) for name, _ in nomad_info._fields_
                if name != "reserved"}

    def layout(self) -> dict:
        info = nomad_get_info(self.h)
        S, nnz, m = info.n_segments, info.nnz, info.m
        out = dict(row_worker=np.zeros(m, np.int32), seg_worker=np.zeros(S, np.int32),
                   seg_col=np.zeros(S, np.int32), seg_ptr=np.zeros(S + 1, np.int64),
                   rec_row=np.zeros(nnz, np.int32), rec_val=np.zeros(nnz, np.float32))
        p = {k: _P(v.ctypes.data) for k, v in out.items()}
        _check(load_library().nomad_get_layout(
            self.h, p["row_worker"], p["seg_worker"], p["seg_col"], p["seg_ptr"],
            p["rec_row"], p["rec_val"]), self.h)
        return out

    def replay_log(self):
        """(seg, epoch) arrays of the last nomad_epoch call, in ticket order."""
        lib = load_library()
        count = ctypes.c_int64()
        _check(lib.nomad_get_replay_log(self.h, 0, None, None, ctypes.byref(count)), self.h)
        seg = np.zeros(count.value, np.int32)
        ep = np.zeros(count.value, np.int32)
        _check(lib.nomad_get_replay_log(self.h, count.value, _P(seg.ctypes.data),
                                        _P(ep.ctypes.data), ctypes.byref(count)), self.h)
        return seg, ep

    def debug_counts(self):
        """(per-record update counts in layout order, ownership violations)."""
        info = nomad_get_info(self.h)
        cnt = np.zeros(info.nnz, np.int32)
        viol = ctypes.c_int64()
        _check(load_library().nomad_get_debug_counts(self.h, _P(cnt.ctypes.data),
                                                     ctypes.byref(viol)), self.h)
        return cnt, viol.value
